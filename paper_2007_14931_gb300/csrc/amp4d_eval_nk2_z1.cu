// Per-event kernels for at most 2 K* resonances and 1 Z resonance(s).
#include "amp4d_eval.cuh"

namespace amp4d {
template cudaError_t launch_eval_t<2, 1>(const LaunchArgs &, int);
template cudaError_t launch_grad_t<2, 1>(const LaunchArgs &, bool);
template cudaError_t launch_lcache_t<2, 1>(const LaunchArgs &, float2 *);
}  // namespace amp4d
