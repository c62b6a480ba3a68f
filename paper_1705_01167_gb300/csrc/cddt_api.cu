// cddt_api.cu -- the C ABI of libcddt.so: handle lifecycle, argument checks,
// export and statistics.  Compute happens in the kernels of cddt_build.cu,
// cddt_query.cu and cddt_maintain.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"
#include "cddt_trace.cuh"

namespace {

bool device_ok()
{
    int n = 0;
    return cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
}

cddt_status check_handle(cddt_t h)
{
    if (!h) return CDDT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CDDT_ERR_CUDA;
    if (dev != h->device) return CDDT_ERR_ARG;
    return CDDT_OK;
}

void free_handle(cddt_s *h)
{
    if (!h) return;
    cudaFree(h->slices);
    cudaFree(h->hdr);
    cudaFree(h->store);
    cudaFree(h->grid);
    cudaFree(h->edge);
    cudaFree(h->status);
    cudaFree(h->last_writer);
    cudaFree(h->stamp);
    cudaFree(h->qscratch);
    cudaFree(h->spare);
    cudaFree(h->ws);
    cudaFree(h->ws_keys);
    delete h;
}

cddt_status sensor_common(cddt_t h, const float *part, int64_t P, const float *beam_off, const float *obs,
                          int32_t B, int32_t D, const cddt_beam_model *m)
{
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    if (P < 0 || B < 1 || B > 8192 || !m) return CDDT_ERR_ARG;
    if (P > 0 && (!part || !beam_off || !obs)) return CDDT_ERR_ARG;
    if (D != 0 && (D >= B || 2 * D < B)) return CDDT_ERR_ARG;
    if (!(m->sigma_hit > 0) || !(m->max_range > 0) || !(m->lambda_short > 0)) return CDDT_ERR_ARG;
    return CDDT_OK;
}

}  // namespace

extern "C" {

int32_t cddt_version(void) { return 1; }

int32_t cddt_checked_build(void) { return CDDT_CHECKED; }

const char *cddt_status_string(cddt_status s)
{
    switch (s) {
    case CDDT_OK: return "ok";
    case CDDT_ERR_ARG: return "invalid argument";
    case CDDT_ERR_CUDA: return "CUDA runtime error or no CUDA device";
    case CDDT_ERR_OOM: return "device out of memory";
    case CDDT_ERR_PRUNED: return "incremental update of a pruned CDDT";
    case CDDT_ERR_TIMEOUT: return "a bounded device wait gave up";
    case CDDT_ERR_DEVICE: return "a kernel flagged bad input";
    case CDDT_ERR_BOUNDS: return "a gather failed its bounds check (checked build)";
    }
    return "unknown status";
}

cddt_status cddt_build(const uint8_t *grid_dev, int32_t W, int32_t H, int32_t theta_disc, float max_range,
                       uint32_t flags, void *stream, cddt_t *out)
{
    CDDT_RANGE("cddt_build", stream);
    if (!out) return CDDT_ERR_ARG;
    *out = nullptr;
    if (!grid_dev || W < 1 || H < 1 || W > 32767 || H > 32767) return CDDT_ERR_ARG;
    if (theta_disc < 2 || (theta_disc & 1) || theta_disc > 65536) return CDDT_ERR_ARG;
    if (!(max_range > 0) || !std::isfinite(max_range)) return CDDT_ERR_ARG;
    if (flags & ~CDDT_ZP_U16) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_build");
    if (!device_ok()) return CDDT_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cddt_s *h = new cddt_s();
    cudaGetDevice(&h->device);
    h->W = W;
    h->H = H;
    h->N = theta_disc;
    h->S = theta_disc / 2;
    h->max_range = max_range;
    h->flags = flags;
    h->u16 = (flags & CDDT_ZP_U16) ? 1 : 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    cddt_status rc = cddt::init_handle(h, grid_dev, st);
    if (rc == CDDT_OK) {
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = CDDT_ERR_CUDA;
        else cudaEventElapsedTime(&h->build_ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CDDT_OK) {
        cudaStreamSynchronize(st);
        free_handle(h);
        return rc;
    }
    *out = h;
    return CDDT_OK;
}

cddt_status cddt_import(const uint8_t *grid_dev, int32_t W, int32_t H, int32_t theta_disc, float max_range,
                        uint32_t flags, int32_t pruned, int64_t total_bins, const int64_t *bin_start_host,
                        const float *zp_host, void *stream, cddt_t *out)
{
    CDDT_RANGE("cddt_import", stream);
    if (!out) return CDDT_ERR_ARG;
    *out = nullptr;
    if (!grid_dev || W < 1 || H < 1 || W > 32767 || H > 32767) return CDDT_ERR_ARG;
    if (theta_disc < 2 || (theta_disc & 1) || theta_disc > 65536) return CDDT_ERR_ARG;
    if (!(max_range > 0) || !std::isfinite(max_range)) return CDDT_ERR_ARG;
    if (flags & ~CDDT_ZP_U16) return CDDT_ERR_ARG;
    if (total_bins < 0 || !bin_start_host) return CDDT_ERR_ARG;
    if (bin_start_host[total_bins] > 0 && !zp_host) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_import");
    if (!device_ok()) return CDDT_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cddt_s *h = new cddt_s();
    cudaGetDevice(&h->device);
    h->W = W;
    h->H = H;
    h->N = theta_disc;
    h->S = theta_disc / 2;
    h->max_range = max_range;
    h->flags = flags;
    h->u16 = (flags & CDDT_ZP_U16) ? 1 : 0;
    h->pruned = pruned ? 1 : 0;
    cddt_status rc = cddt::init_handle(h, grid_dev, st, false);
    if (rc == CDDT_OK && h->total_bins != total_bins) rc = CDDT_ERR_ARG;  // exported with other parameters
    if (rc == CDDT_OK) rc = cddt::import_store(h, bin_start_host, zp_host, st);
    if (rc == CDDT_OK) {
        int flag = 0;
        if (cudaMemcpy(&flag, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = CDDT_ERR_CUDA;
        else if (flag) rc = CDDT_ERR_ARG;  // a bin of the CSR was not sorted
    }
    if (rc != CDDT_OK) {
        cudaStreamSynchronize(st);
        free_handle(h);
        return rc;
    }
    *out = h;
    return CDDT_OK;
}

cddt_status cddt_destroy(cddt_t h)
{
    if (!h) return CDDT_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_handle(h);
    if (cur != h->device) cudaSetDevice(cur);
    return CDDT_OK;
}

cddt_status cddt_prune(cddt_t h, void *stream)
{
    CDDT_RANGE("cddt_prune", stream);
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    if (h->pruned) return CDDT_ERR_PRUNED;
    CDDT_FAULT_POINT("cddt_prune");
    return cddt::prune(h, (cudaStream_t)stream);
}

cddt_status cddt_update_cells(cddt_t h, const int32_t *xy_dev, const uint8_t *occ_dev, int32_t n, void *stream)
{
    CDDT_RANGE("cddt_update_cells", stream);
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    if (n < 0 || (n > 0 && (!xy_dev || !occ_dev))) return CDDT_ERR_ARG;
    if (h->pruned) return CDDT_ERR_PRUNED;
    CDDT_FAULT_POINT("cddt_update_cells");
    if (n == 0) return CDDT_OK;
    return cddt::update_cells(h, xy_dev, occ_dev, n, (cudaStream_t)stream);
}

cddt_status cddt_calc_range_many(cddt_t h, const float *pose_dev, float *range_dev, int64_t n, int32_t sort_by_slice,
                                 void *stream)
{
    CDDT_RANGE("cddt_calc_range_many", stream);
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    if (n < 0 || (n > 0 && (!pose_dev || !range_dev))) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_calc_range_many");
    return cddt::calc_range(h, pose_dev, range_dev, n, sort_by_slice, (cudaStream_t)stream);
}

cddt_status cddt_calc_range_timed(cddt_t h, const float *pose_dev, float *range_dev, int64_t n,
                                  int64_t *warp_cycles_dev, void *stream)
{
    CDDT_RANGE("cddt_calc_range_timed", stream);
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    if (n < 0 || (n > 0 && (!pose_dev || !range_dev || !warp_cycles_dev))) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_calc_range_timed");
    return cddt::calc_range_timed(h, pose_dev, range_dev, n, reinterpret_cast<long long *>(warp_cycles_dev),
                                  (cudaStream_t)stream);
}

cddt_status cddt_sensor_weights(cddt_t h, const float *particles_dev, int64_t P, const float *beam_off_dev,
                                const float *obs_dev, int32_t B, int32_t pair_offset, const cddt_beam_model *m,
                                float *logw_dev, float *ranges_dev, void *stream)
{
    CDDT_RANGE("cddt_sensor_weights", stream);
    cddt_status rc = sensor_common(h, particles_dev, P, beam_off_dev, obs_dev, B, pair_offset, m);
    if (rc != CDDT_OK) return rc;
    if (P > 0 && !logw_dev) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_sensor_weights");
    if (P == 0) return CDDT_OK;
    cddt::SensorArgs a{};
    a.part = particles_dev;
    a.P = P;
    a.beam_off = beam_off_dev;
    a.obs = obs_dev;
    a.B = B;
    a.D = pair_offset;
    a.bc = cddt::make_beam_consts(*m);
    a.logw = logw_dev;
    a.ranges = ranges_dev;
    return cddt::launch_sensor(h, a, 0, (cudaStream_t)stream);
}

cddt_status cddt_sensor_weights_backward(cddt_t h, const float *particles_dev, int64_t P, const float *beam_off_dev,
                                         const float *obs_dev, int32_t B, int32_t pair_offset,
                                         const cddt_beam_model *m, const float *grad_logw_dev, float *grad_xy_dev,
                                         void *stream)
{
    CDDT_RANGE("cddt_sensor_weights_backward", stream);
    cddt_status rc = sensor_common(h, particles_dev, P, beam_off_dev, obs_dev, B, pair_offset, m);
    if (rc != CDDT_OK) return rc;
    if (P > 0 && (!grad_logw_dev || !grad_xy_dev)) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_sensor_weights_backward");
    if (P == 0) return CDDT_OK;
    cddt::SensorArgs a{};
    a.part = particles_dev;
    a.P = P;
    a.beam_off = beam_off_dev;
    a.obs = obs_dev;
    a.B = B;
    a.D = pair_offset;
    a.bc = cddt::make_beam_consts(*m);
    a.grad_logw = grad_logw_dev;
    a.grad_xy = grad_xy_dev;
    return cddt::launch_sensor(h, a, 1, (cudaStream_t)stream);
}

cddt_status cddt_sensor_weights_fwd_bwd(cddt_t h, const float *particles_dev, int64_t P, const float *beam_off_dev,
                                        const float *obs_dev, int32_t B, int32_t pair_offset,
                                        const cddt_beam_model *m, float *logw_dev, float *grad_xy_dev, void *stream)
{
    CDDT_RANGE("cddt_sensor_weights_fwd_bwd", stream);
    cddt_status rc = sensor_common(h, particles_dev, P, beam_off_dev, obs_dev, B, pair_offset, m);
    if (rc != CDDT_OK) return rc;
    if (P > 0 && (!logw_dev || !grad_xy_dev)) return CDDT_ERR_ARG;
    CDDT_FAULT_POINT("cddt_sensor_weights_fwd_bwd");
    if (P == 0) return CDDT_OK;
    cddt::SensorArgs a{};
    a.part = particles_dev;
    a.P = P;
    a.beam_off = beam_off_dev;
    a.obs = obs_dev;
    a.B = B;
    a.D = pair_offset;
    a.bc = cddt::make_beam_consts(*m);
    a.logw = logw_dev;
    a.grad_xy = grad_xy_dev;
    return cddt::launch_sensor(h, a, 2, (cudaStream_t)stream);
}

cddt_status cddt_sensor_work(cddt_t h, const float *particles_dev, int64_t P, const float *beam_off_dev, int32_t B,
                             int32_t pair_offset, int64_t *out_host, void *stream)
{
    cddt_beam_model dummy{1, 0, 0, 0, 1, 1, 1, 0};
    // obs are not read for work figures; beam_off stands in as a valid pointer
    cddt_status rc = sensor_common(h, particles_dev, P, beam_off_dev, beam_off_dev, B, pair_offset, &dummy);
    if (rc != CDDT_OK) return rc;
    if (!out_host) return CDDT_ERR_ARG;
    std::memset(out_host, 0, sizeof(int64_t) * 7);
    if (P == 0) return CDDT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *w = nullptr;
    CDDT_CUDA(cudaMalloc(&w, sizeof(unsigned long long) * 7));
    cudaMemsetAsync(w, 0, sizeof(unsigned long long) * 7, st);
    cddt::SensorArgs a{};
    a.part = particles_dev;
    a.P = P;
    a.beam_off = beam_off_dev;
    a.obs = beam_off_dev;
    a.B = B;
    a.D = pair_offset;
    a.bc = cddt::make_beam_consts(dummy);
    a.work = w;
    rc = cddt::launch_sensor(h, a, 3, st);
    unsigned long long host[7] = {0, 0, 0, 0, 0, 0, 0};
    if (rc == CDDT_OK) {
        cudaError_t e = cudaMemcpyAsync(host, w, sizeof(host), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cddt::cuda_status(e);
    }
    cudaFree(w);
    for (int q = 0; q < 7; ++q) out_host[q] = (int64_t)host[q];
    return rc;
}

cddt_status cddt_set_search(cddt_t h, int32_t search)
{
    if (!h) return CDDT_ERR_ARG;
    if (search != CDDT_SEARCH_TREE && search != CDDT_SEARCH_BINARY) return CDDT_ERR_ARG;
    if (h->search != search) h->generation++;
    h->search = search;
    return CDDT_OK;
}

cddt_status cddt_get_stats(cddt_t h, cddt_stats *out)
{
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    if (!out) return CDDT_ERR_ARG;
    CDDT_CUDA(cudaDeviceSynchronize());
    out->W = h->W;
    out->H = h->H;
    out->theta_disc = h->N;
    out->n_slices = h->S;
    out->max_range = h->max_range;
    out->flags = h->flags;
    out->pruned = h->pruned;
    out->total_bins = h->total_bins;
    out->n_zero_points = h->n_zp;
    out->n_edge_cells = h->n_edge;
    out->store_bytes = h->store_nodes * 32 + h->total_bins * (int64_t)sizeof(cddt::BinHdr);
    out->max_bin = h->max_bin;
    out->build_ms = h->build_ms;
    out->prune_ms = h->prune_ms;
    out->update_ms = h->update_ms;
    return CDDT_OK;
}

cddt_status cddt_get_status(cddt_t h)
{
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    int s = 0;
    CDDT_CUDA(cudaDeviceSynchronize());
    CDDT_CUDA(cudaMemcpy(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    CDDT_CUDA(cudaMemset(h->status, 0, sizeof(int)));
    return (cddt_status)s;
}

cddt_status cddt_export(cddt_t h, int64_t *slice_base_host, int64_t *bin_start_host, float *zp_host)
{
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    CDDT_CUDA(cudaDeviceSynchronize());
    std::vector<cddt::SliceInfo> sl(h->S);
    CDDT_CUDA(cudaMemcpy(sl.data(), h->slices, sizeof(cddt::SliceInfo) * h->S, cudaMemcpyDeviceToHost));
    if (slice_base_host) {
        for (int s = 0; s < h->S; ++s) slice_base_host[s] = sl[s].sbase;
        slice_base_host[h->S] = h->total_bins;
    }
    if (!bin_start_host && !zp_host) return CDDT_OK;
    std::vector<cddt::BinHdr> hdr((size_t)h->total_bins);
    CDDT_CUDA(cudaMemcpy(hdr.data(), h->hdr, sizeof(cddt::BinHdr) * hdr.size(), cudaMemcpyDeviceToHost));
    if (bin_start_host) {
        int64_t o = 0;
        for (int64_t g = 0; g < h->total_bins; ++g) {
            bin_start_host[g] = o;
            o += cddt::bin_count(hdr[g].nm);
        }
        bin_start_host[h->total_bins] = o;
    }
    if (!zp_host) return CDDT_OK;
    const int LK = h->u16 ? 4 : 3, R = h->u16 ? 12 : 6;
    std::vector<unsigned char> store((size_t)h->store_nodes * 32);
    if (!store.empty())
        CDDT_CUDA(cudaMemcpy(store.data(), h->store, store.size(), cudaMemcpyDeviceToHost));
    int64_t o = 0;
    int s = 0;
    for (int64_t g = 0; g < h->total_bins; ++g) {
        while (s + 1 < h->S && (int64_t)sl[s + 1].sbase <= g) ++s;
        uint32_t n = cddt::bin_count(hdr[g].nm);
        if (!n) continue;
        size_t leaf = (size_t)(hdr[g].off + cddt::internal_nodes(n, LK, R)) * 32;
        if (h->u16) {
            const uint16_t *k = reinterpret_cast<const uint16_t *>(store.data() + leaf);
            volatile float invQ = h->invQ;
            for (uint32_t i = 0; i < n; ++i) {
                volatile float t = (float)k[i] * invQ;  // exact: invQ is a power of two
                zp_host[o + i] = t - sl[s].X;
            }
        } else {
            std::memcpy(zp_host + o, store.data() + leaf, sizeof(float) * n);
        }
        o += n;
    }
    return CDDT_OK;
}

cddt_status cddt_export_grid(cddt_t h, uint8_t *grid_host, uint8_t *edge_host)
{
    cddt_status rc = check_handle(h);
    if (rc != CDDT_OK) return rc;
    CDDT_CUDA(cudaDeviceSynchronize());
    size_t n = (size_t)h->W * h->H;
    if (grid_host) CDDT_CUDA(cudaMemcpy(grid_host, h->grid, n, cudaMemcpyDeviceToHost));
    if (edge_host) CDDT_CUDA(cudaMemcpy(edge_host, h->edge, n, cudaMemcpyDeviceToHost));
    return CDDT_OK;
}

}  // extern "C"
