// cddt_probe.cu -- random 32-byte sector gather probe (cddt_gather_probe):
// the bandwidth that bounds a gather of tree nodes, measured on this GPU.
#include <cuda_runtime.h>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"

namespace cddt {

// SplitMix64 finaliser of (seed, i): the sector each read takes.
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) gather_probe_kernel(const char *buf, uint64_t nsec, int64_t reads,
                                                            uint64_t seed, unsigned long long *sink)
{
    uint32_t acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < reads;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t sec = mix64(seed ^ (uint64_t)i) % nsec;
        uint32_t w[8];
        ld_node(buf + (sec << 5), w);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc ^= w[q];
    }
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicXor(sink, (unsigned long long)acc);
}

}  // namespace cddt

extern "C" cddt_status cddt_gather_probe(const void *buf_dev, int64_t bytes, int64_t sectors, uint64_t seed,
                                         uint64_t *sink_dev, void *stream)
{
    if (!buf_dev || !sink_dev || bytes < 32 || (bytes & 31) || sectors < 0) return CDDT_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(buf_dev) & 31) return CDDT_ERR_ARG;  // 256-bit loads
    if (sectors == 0) return CDDT_OK;
    const unsigned blocks = cddt::grid_cap(sectors, 256, 16);
    cddt::gather_probe_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const char *>(buf_dev), (uint64_t)bytes >> 5, sectors, seed,
        reinterpret_cast<unsigned long long *>(sink_dev));
    CDDT_CUDA(cudaGetLastError());
    return CDDT_OK;
}
