// Instantiation of the per-event kernels for at most 2 K* resonances.
#include "amp4d_eval.cuh"

namespace amp4d {
template cudaError_t launch_eval_nk<2>(const LaunchArgs &, int);
template cudaError_t launch_grad_nk<2>(const LaunchArgs &, bool);
template cudaError_t launch_lcache_nk<2>(const LaunchArgs &, float2 *);
}  // namespace amp4d
