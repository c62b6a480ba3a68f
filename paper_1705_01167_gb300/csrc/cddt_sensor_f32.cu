// cddt_sensor_f32.cu -- single-filter sensor-model kernels, float32 zero points.
#include "cddt_sensor.cuh"

namespace cddt {

cddt_status launch_sensor_f32(const cddt_s *h, const SensorArgs &a, int mode, int tpp, int threads, cudaStream_t st)
{
    return launch_sensor_mode<float>(h, a, mode, tpp, threads, st);
}

}  // namespace cddt
