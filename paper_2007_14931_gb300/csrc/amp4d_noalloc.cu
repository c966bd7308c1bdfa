// Allocation-free variant of the proposal-training gradient.
//
// amp4d_mlp_loss_grad allocates its scratch (per-block partial sums and a BF16
// copy of the weights) with cudaMalloc on every call.  Some callers cannot do
// that: code that runs while another component owns the whole device memory
// budget through its own pool, or code that must not trigger the implicit
// device synchronisation that cudaMalloc/cudaFree can cause.  For them this
// file keeps that scratch in one file-scope device array of fixed size, which
// every GPU that loads the library holds until the process exits, and the
// entry point below takes only caller-owned inputs and outputs.
#include <cstdint>

#include <cuda_bf16.h>

#include "../../include/amp4d.h"
#include "amp4d_launch.h"
#include "amp4d_mlp.cuh"

namespace amp4d {

namespace {

// At most one CTA per MLP_GRAD_TILE rows of each set, one partial row each.
constexpr int NA_MAX_BLOCKS = 2 * ((AMP4D_NOALLOC_MAX_ROWS + MLP_GRAD_TILE - 1) / MLP_GRAD_TILE);
constexpr size_t NA_PART_FLOATS = (size_t)NA_MAX_BLOCKS * (MLP_P + 1);   // multiple of 64
static_assert(NA_PART_FLOATS % 64 == 0, "the BF16 weights start 256-byte aligned");
constexpr size_t NA_SCRATCH_FLOATS = NA_PART_FLOATS + (MLP_P + 1) / 2 + 64;

// Partial sums (NA_MAX_BLOCKS x 4546 floats), then the BF16 weights.
static __device__ __align__(256) float g_noalloc_scratch[NA_SCRATCH_FLOATS];

thread_local const char *g_na_error = "";

// Device address of the scratch array in the current context.  Host code cannot
// use the symbol itself as a device pointer.  The address is looked up on every
// call rather than cached: a context that was reset and re-created reloads the
// module, and a cached address would then point into freed memory.  The lookup
// is a host-side query that neither allocates nor synchronises once the module
// is loaded (the first call on a device may load it).
cudaError_t scratch_address(float **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<float *>(p);
    return cudaSuccess;
}

}  // namespace

}  // namespace amp4d

using namespace amp4d;

extern "C" amp4d_status amp4d_mlp_loss_grad_noalloc(const float *theta, const float *xd, int64_t nd,
                                                    const float *xu, int64_t nu, double *out,
                                                    void *stream)
{
    if (!theta || !xd || !xu || !out) {
        g_na_error = "mlp_loss_grad_noalloc: null pointer";
        return AMP4D_ERR_ARG;
    }
    if (nd < 1 || nu < 1 || nd > AMP4D_NOALLOC_MAX_ROWS || nu > AMP4D_NOALLOC_MAX_ROWS) {
        g_na_error = "mlp_loss_grad_noalloc: nd and nu must lie in [1, AMP4D_NOALLOC_MAX_ROWS = 4096]"
                     " (the size of the static scratch)";
        return AMP4D_ERR_ARG;
    }
    if (mlp_grad_blocks(nd, nu) > NA_MAX_BLOCKS) {
        g_na_error = "mlp_loss_grad_noalloc: the gradient kernel needs more partial rows than the static scratch holds";
        return AMP4D_ERR_ARG;
    }
    float *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        g_na_error = cudaGetErrorString(e);
        return AMP4D_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    float *part = scratch;
    __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(scratch + NA_PART_FLOATS);
    // Every block of the gradient kernel writes its whole partial row and the
    // finishing kernel reads only those rows: nothing has to start at zero.
    e = launch_to_bf16(theta, wb, st);
    if (e == cudaSuccess) e = launch_mlp_grad(wb, xd, nd, xu, nu, part, out, st);
    if (e != cudaSuccess) {
        g_na_error = cudaGetErrorString(e);
        return AMP4D_ERR_CUDA;
    }
    return AMP4D_OK;
}

extern "C" const char *amp4d_noalloc_last_error(void) { return g_na_error; }
