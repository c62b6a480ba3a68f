/* cddt_example.c -- the C ABI used from plain C (no Python, no PyTorch): build
 * a CDDT of a 64 x 48 box (walls on the border, one pillar), cast rays along
 * the axes, and check them against the closed forms of Section IV's
 * axis-aligned case (the distance from the query cell's centre to the wall or
 * pillar cell's centre along the ray).  Device memory comes from the CUDA
 * runtime; everything else goes through include/cddt.h.
 *
 * Exit status: 0 on success, 1 on a wrong range or failed call, 2 when there
 * is no CUDA device (after checking that the library reports that as
 * CDDT_ERR_CUDA and still answers argument errors with CDDT_ERR_ARG). */
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cddt.h"

#define MAP_W 64
#define MAP_H 48

static int fail(const char *what, cddt_status s)
{
    fprintf(stderr, "%s: %s (%d)\n", what, cddt_status_string(s), (int)s);
    return 1;
}

int main(void)
{
    cddt_t h = NULL;
    printf("libcddt version %d, checked build %d\n", (int)cddt_version(), (int)cddt_checked_build());
    /* argument errors come back before any device work */
    if (cddt_build(NULL, MAP_W, MAP_H, 108, 100.0f, 0, NULL, &h) != CDDT_ERR_ARG || h) return fail("null grid", CDDT_OK);

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        uint8_t fake[1];
        const cddt_status s = cddt_build(fake, MAP_W, MAP_H, 108, 100.0f, 0, NULL, &h);
        if (s != CDDT_ERR_CUDA) return fail("build without a device", s);
        printf("no CUDA device: %s\n", cddt_status_string(s));
        return 2;
    }

    static uint8_t grid[MAP_H][MAP_W];
    memset(grid, 0, sizeof(grid));
    for (int i = 0; i < MAP_W; ++i) grid[0][i] = grid[MAP_H - 1][i] = 1;
    for (int j = 0; j < MAP_H; ++j) grid[j][0] = grid[j][MAP_W - 1] = 1;
    grid[20][40] = 1; /* a pillar at (x = 40, y = 20) */

    /* queries (x, y, theta) and their closed-form ranges */
    const float PI = 3.14159265358979f;
    const float q[][3] = {{10, 20, 0}, {50, 20, PI}, {10, 20, PI}, {10, 10, PI / 2}, {10, 10, -PI / 2},
                          {30, 20, 0}, {0, 5, 0}, {-3, 5, 0}};
    const float want[] = {30, 10, 10, 37, 10, 10, 0, 0};
    enum { NQ = sizeof(want) / sizeof(want[0]) };

    uint8_t *grid_dev = NULL;
    float *pose_dev = NULL, *range_dev = NULL;
    if (cudaMalloc((void **)&grid_dev, sizeof(grid)) != cudaSuccess ||
        cudaMalloc((void **)&pose_dev, sizeof(q)) != cudaSuccess ||
        cudaMalloc((void **)&range_dev, sizeof(float) * NQ) != cudaSuccess)
        return fail("cudaMalloc", CDDT_ERR_OOM);
    cudaMemcpy(grid_dev, grid, sizeof(grid), cudaMemcpyHostToDevice);
    cudaMemcpy(pose_dev, q, sizeof(q), cudaMemcpyHostToDevice);

    cddt_status s = cddt_build(grid_dev, MAP_W, MAP_H, 108, 100.0f, 0, NULL, &h);
    if (s != CDDT_OK) return fail("cddt_build", s);
    cddt_stats st;
    if ((s = cddt_get_stats(h, &st)) != CDDT_OK) return fail("cddt_get_stats", s);
    printf("%d x %d, %d slices, %lld zero points in %lld bytes\n", st.W, st.H, st.n_slices,
           (long long)st.n_zero_points, (long long)st.store_bytes);

    float got[NQ];
    int bad = 0;
    for (int sorted = 0; sorted < 2; ++sorted) {
        if ((s = cddt_calc_range_many(h, pose_dev, range_dev, NQ, sorted, NULL)) != CDDT_OK)
            return fail("cddt_calc_range_many", s);
        cudaMemcpy(got, range_dev, sizeof(got), cudaMemcpyDeviceToHost);
        for (int i = 0; i < NQ; ++i)
            if (got[i] != want[i]) {
                fprintf(stderr, "query %d (sorted %d): got %g, want %g\n", i, sorted, got[i], want[i]);
                bad = 1;
            }
    }
    if ((s = cddt_get_status(h)) != CDDT_OK) return fail("device status", s);
    cddt_destroy(h);
    cudaFree(grid_dev);
    cudaFree(pose_dev);
    cudaFree(range_dev);
    if (!bad) printf("%d ray casts match their closed forms\n", 2 * (int)NQ);
    return bad;
}
