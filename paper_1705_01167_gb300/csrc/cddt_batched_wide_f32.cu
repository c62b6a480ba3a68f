// cddt_batched_wide_f32.cu -- persistent batched sensor-model kernels with 16
// and 32 lanes per particle, float32 zero points.
#include "cddt_sensor.cuh"

namespace cddt {

BatchedFn batched_fn_wide_f32(int search, int tpp, int block, int regcap)
{
    if (search == CDDT_SEARCH_BINARY)
        return regcap ? batched_fn_kt_wide<float, CDDT_SEARCH_BINARY, 48>(tpp, block)
                      : batched_fn_kt_wide<float, CDDT_SEARCH_BINARY, 32>(tpp, block);
    return regcap ? batched_fn_kt_wide<float, CDDT_SEARCH_TREE, 48>(tpp, block)
                  : batched_fn_kt_wide<float, CDDT_SEARCH_TREE, 32>(tpp, block);
}

}  // namespace cddt
