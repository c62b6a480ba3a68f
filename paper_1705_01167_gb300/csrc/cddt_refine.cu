// cddt_refine.cu -- the plan's gradient pose refinement kernels (both key
// types, every lanes-per-particle count); the kernel is in cddt_sensor.cuh.
#include "cddt_sensor.cuh"

namespace cddt {

RefineFn refine_fn(bool u16, int tpp) { return u16 ? refine_fn_kt<uint16_t>(tpp) : refine_fn_kt<float>(tpp); }

}  // namespace cddt
