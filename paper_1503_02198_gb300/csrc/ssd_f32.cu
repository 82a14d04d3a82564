// FP32 path: interpolation, flux and divergence arithmetic in float; state,
// Runge-Kutta accumulation, rotation angle and mortar geometry stay FP64.
#include "ssd_engine.cuh"

namespace ssd {
Engine *make_engine_f32(int N) { return make_engine_t<float>(N); }
}  // namespace ssd
