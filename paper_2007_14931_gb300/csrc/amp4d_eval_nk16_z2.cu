// Per-event kernels for at most 16 K* resonances and 2 Z resonance(s).
#include "amp4d_eval.cuh"

namespace amp4d {
template cudaError_t launch_eval_t<16, 2>(const LaunchArgs &, int);
template cudaError_t launch_grad_t<16, 2>(const LaunchArgs &, bool);
template cudaError_t launch_lcache_t<16, 2>(const LaunchArgs &, float2 *);
}  // namespace amp4d
