// Per-event kernels for at most 10 K* resonances and 0 Z resonance(s).
#include "amp4d_eval.cuh"

namespace amp4d {
template cudaError_t launch_eval_t<10, 0>(const LaunchArgs &, int);
template cudaError_t launch_grad_t<10, 0>(const LaunchArgs &, bool);
template cudaError_t launch_lcache_t<10, 0>(const LaunchArgs &, float2 *);
}  // namespace amp4d
