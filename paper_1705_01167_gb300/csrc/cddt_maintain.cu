// cddt_maintain.cu -- pruning (Section IV-C) and incremental update
// (Section IV-D) of a built CDDT.
#include <cuda_runtime.h>

#include "cddt_internal.cuh"
#include "cddt_kernels.cuh"

namespace cddt {

cddt_status prune(cddt_s *, cudaStream_t) { return CDDT_ERR_ARG; }

cddt_status update_cells(cddt_s *, const int32_t *, const uint8_t *, int32_t, cudaStream_t)
{
    return CDDT_ERR_ARG;
}

}  // namespace cddt
