// FP64 path: every kernel of ssd_engine.cuh instantiated with T = double.
#include "ssd_engine.cuh"

namespace ssd {
Engine *make_engine_f64(int N) { return make_engine_t<double>(N); }
}  // namespace ssd
