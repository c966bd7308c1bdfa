// Host-side launch interface between the C ABI (amp4d_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace amp4d {

struct ModelDev;
struct ModelStatic;

struct LaunchArgs {
    const float *rec;        // event records, REC_* x npad
    int64_t npad, n;         // padded and true event counts
    int wrec;                // record index of the weights (normalisation points)
    const ModelDev *md;      // device model table
    double *part;            // per-block partials
    float *out;              // per-event output (MODE_WRITE)
    unsigned *status;        // error flags
    int grid;
    int nk_max, nz;          // template bucket
    cudaStream_t stream;
};

int nk_bucket(int nk);
int grad_num_slots(int nk_max, int nz);
int eval_block();
int grad_block();

cudaError_t launch_eval(const LaunchArgs &a, int mode);  // 0 ln S, 1 w S, 2 write S
cudaError_t launch_grad(const LaunchArgs &a, bool norm);
cudaError_t launch_reduce_cols(const double *part, int nblk, int ncol, double *out,
                               cudaStream_t s);
cudaError_t launch_finish(const double *rd, const double *rn, const int *slot_param,
                          const double *pscale, int nslot, int nparam, double n_events,
                          double lnpq, double vol_over_n, const unsigned *status, double *out,
                          cudaStream_t s);

cudaError_t launch_build_table(const ModelStatic *st, const double *params, ModelDev *md,
                               double *pscale, unsigned *status, cudaStream_t s);
cudaError_t launch_finish_gram(const double *rd, const int *slot_param, const double *pscale,
                               int nslot, int ncol, int nparam, double n_events, double lnpq,
                               double vol_over_n, const double *params, const double *G,
                               const unsigned *status, double *out, int with_grad, cudaStream_t s);

// Normalisation Gram matrix (amp4d_gram.cu).
struct GramArgs {
    const float *rec;        // normalisation-point records (weights in record wrec)
    int64_t npad, n;
    int wrec;
    const ModelDev *md;
    unsigned *colmax;        // 64 (scratch)
    float *gscale;           // 64 (scratch): fixed-point scale per real column
    long long *part;         // grid_tc x 4096 INT64 partials (scratch)
    int *err;                // set to 1 if a bounded wait expired
    double *G;               // dim x dim output
    int dim;                 // 2 K
    int grid_colmax, grid_tc;
    int nk_max, nz;
    cudaStream_t stream;
};
cudaError_t launch_gram(const GramArgs &a);
cudaError_t launch_gram_selftest(const int *synth, int64_t n, const ModelDev *md, long long *part,
                                 int grid, int *err, long long *out, cudaStream_t st);
int gram_chunk_points();

// One-time FP64 preparation of an event set (amp4d_prepare.cu).
struct PrepArgs {
    float *rec;
    int64_t npad, n;
    int has_z;
    int wrec;                 // >= 0: weights record; with have_w = 0 it is filled with p q
    int have_w;
    double mB, mpsi, mK, mpi, m_lo, m_hi;
    double *part_lnpq;        // per-block partials of sum ln(p q) (nullable)
    unsigned long long *bad;  // first bad index (init to ~0ull)
    int grid;
    cudaStream_t stream;
};
cudaError_t launch_prepare(const PrepArgs &a);
int prepare_block();

}  // namespace amp4d
