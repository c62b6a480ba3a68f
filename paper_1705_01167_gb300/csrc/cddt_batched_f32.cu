// cddt_batched_f32.cu -- persistent batched sensor-model kernels, float32 zero points.
#include "cddt_sensor.cuh"

namespace cddt {

BatchedFn batched_fn_f32(int search, int tpp, int block, int regcap)
{
    if (tpp >= 16) return batched_fn_wide_f32(search, tpp, block, regcap);
    if (search == CDDT_SEARCH_BINARY)
        return regcap ? batched_fn_kt<float, CDDT_SEARCH_BINARY, 48>(tpp, block)
                      : batched_fn_kt<float, CDDT_SEARCH_BINARY, 32>(tpp, block);
    return regcap ? batched_fn_kt<float, CDDT_SEARCH_TREE, 48>(tpp, block)
                  : batched_fn_kt<float, CDDT_SEARCH_TREE, 32>(tpp, block);
}

}  // namespace cddt
