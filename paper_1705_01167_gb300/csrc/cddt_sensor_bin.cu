// cddt_sensor_bin.cu -- single-filter sensor-model kernels with the
// binary-search layout (forward mode), for comparison with the tree.
#include "cddt_sensor.cuh"

namespace cddt {

cddt_status launch_sensor_binary(const cddt_s *h, const SensorArgs &a, int tpp, int threads, cudaStream_t st)
{
    if (h->u16) return launch_sensor_tpp<uint16_t, MODE_FWD, CDDT_SEARCH_BINARY>(h, a, tpp, threads, st);
    return launch_sensor_tpp<float, MODE_FWD, CDDT_SEARCH_BINARY>(h, a, tpp, threads, st);
}

}  // namespace cddt
