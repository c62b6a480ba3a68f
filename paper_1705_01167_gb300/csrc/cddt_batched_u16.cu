// cddt_batched_u16.cu -- persistent batched sensor-model kernels, 16-bit zero points.
#include "cddt_sensor.cuh"

namespace cddt {

BatchedFn batched_fn_u16(int search, int tpp, int block, int regcap)
{
    if (tpp >= 16) return batched_fn_wide_u16(search, tpp, block, regcap);
    if (search == CDDT_SEARCH_BINARY)
        return regcap ? batched_fn_kt<uint16_t, CDDT_SEARCH_BINARY, 48>(tpp, block)
                      : batched_fn_kt<uint16_t, CDDT_SEARCH_BINARY, 32>(tpp, block);
    return regcap ? batched_fn_kt<uint16_t, CDDT_SEARCH_TREE, 48>(tpp, block)
                  : batched_fn_kt<uint16_t, CDDT_SEARCH_TREE, 32>(tpp, block);
}

}  // namespace cddt
