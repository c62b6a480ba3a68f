// cddt_sensor_u16.cu -- single-filter sensor-model kernels, 16-bit zero points.
#include "cddt_sensor.cuh"

namespace cddt {

cddt_status launch_sensor_u16(const cddt_s *h, const SensorArgs &a, int mode, int tpp, int threads, cudaStream_t st)
{
    return launch_sensor_mode<uint16_t>(h, a, mode, tpp, threads, st);
}

}  // namespace cddt
