// FP32 path: interpolation, flux and divergence arithmetic in float; the
// state and its Runge-Kutta accumulation in double-float; rotation angles and
// mortar offsets in extended FP64.
#include "ssd_engine.cuh"

namespace ssd {
Engine *make_engine_f32(int N) { return make_engine_t<float>(N); }
}  // namespace ssd
