// Dispatch of the per-event kernels for at most 2 K* resonances; the kernels
// for each number of Z resonances are instantiated in amp4d_eval_nk2_z*.cu,
// which compile in parallel.
#include "amp4d_eval.cuh"

namespace amp4d {
extern template cudaError_t launch_eval_t<2, 0>(const LaunchArgs &, int);
extern template cudaError_t launch_eval_t<2, 1>(const LaunchArgs &, int);
extern template cudaError_t launch_eval_t<2, 2>(const LaunchArgs &, int);
extern template cudaError_t launch_grad_t<2, 0>(const LaunchArgs &, bool);
extern template cudaError_t launch_grad_t<2, 1>(const LaunchArgs &, bool);
extern template cudaError_t launch_grad_t<2, 2>(const LaunchArgs &, bool);
extern template cudaError_t launch_lcache_t<2, 0>(const LaunchArgs &, float2 *);
extern template cudaError_t launch_lcache_t<2, 1>(const LaunchArgs &, float2 *);
extern template cudaError_t launch_lcache_t<2, 2>(const LaunchArgs &, float2 *);
template cudaError_t launch_eval_nk<2>(const LaunchArgs &, int);
template cudaError_t launch_grad_nk<2>(const LaunchArgs &, bool);
template cudaError_t launch_lcache_nk<2>(const LaunchArgs &, float2 *);
}  // namespace amp4d
