// FP32 state storage: as the FP32 path, with the state kept as one float per
// value (the Runge-Kutta stage result rounded to float once per stage).
#include "ssd_engine.cuh"

namespace ssd {
Engine *make_engine_f32s(int N) { return make_engine_t<float, false>(N); }
}  // namespace ssd
