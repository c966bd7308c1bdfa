// Host-side launch interface between the C ABI (amp4d_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace amp4d {

struct ModelDev;
struct ModelStatic;

// Inputs of the Gram-path finishing step (finish_gram_body in amp4d_finish.cuh).
struct FinishArgs {
    const unsigned long long *ad = nullptr;  // the data pass's 128-bit sums
    const int *slot_param = nullptr;
    const double *pscale = nullptr;
    int nslot = 0, ncol = 0, nparam = 0;
    double n_events = 0.0, lnpq = 0.0, vol_over_n = 0.0;
    const double *params = nullptr, *G = nullptr;
    const unsigned *status = nullptr;
    double *out = nullptr;
    int with_grad = 0;
    double n_points = 0.0;
    int partials = 0;
    const unsigned long long *ar = nullptr;
    ModelDev *alpha_md = nullptr;
    double purity = 1.0;
    // fused into the data kernel: the CTA that draws the last ticket finishes, and
    // CTAs 0 .. dim/2 - 1 write the rows of G u and G v (2 dim doubles) to guv
    unsigned *ticket = nullptr;
    double *guv = nullptr;
};

struct LaunchArgs {
    const float *rec;        // event records, REC_* x npad
    int64_t npad, n;         // padded and true event counts
    int wrec;                // record index of the weights (normalisation points)
    const ModelDev *md;      // device model table
    double *part;            // per-block partials (ingest)
    unsigned long long *acc = nullptr;  // 128-bit accumulators of the sums (evaluation kernels)
    float *out;              // per-event output (MODE_WRITE)
    unsigned *status;        // error flags
    int grid;
    int nk_max, nz;          // template bucket
    cudaStream_t stream;
    const float2 *lcache = nullptr;  // basis cache of the set, or null (recompute)
    int nrow = 0;                    // rows of the basis cache: lineshapes, then 4 per Z
    int nk = -1;                     // K* resonances of the model (at most the bucket nk_max)
    int nj0 = 0;                     // of which scalar (J = 0): the last nj0 in internal order
    bool zboth = false;              // every Z has both columns (l' = 0 and l' = +-1)
    int nslot = 0;                   // gradient slots (grad_num_slots)
    bool all_fixed = false;          // no mass or width floats (with lcache: all lineshapes cached)
    bool kstar_fixed = false;        // no K* mass or width floats
    // Eq. 14 with a background (data sets): eps and hb per event, and the
    // accumulator of the signal probabilities r = alpha eps S / g.
    const float *mix_eps = nullptr, *mix_hb = nullptr;
    unsigned long long *acc_r = nullptr;
    bool mt = false;                 // data sets with a flavour mistag: S and S(-phi) per event
    // Gram path: the data kernel's last CTA finishes the evaluation (fin.ticket set)
    FinishArgs fin;
};

// Resident CTAs per SM of the adjoint kernels (their __launch_bounds__).  The
// all-cached variant (k_grad_fx) evaluates two events per thread in lock-step,
// reading each resonance's constants and each gradient slot once for both, and
// holds the state of both in about 150 registers: 3 CTAs per SM.
constexpr int GRAD_CTAS_PER_SM = 4;
constexpr int GRAD_CTAS_PER_SM_CACHED = 3;
constexpr int GRAD_EVENTS_PER_THREAD_CACHED = 2;
// With floated K* lineshapes computed per event the all-cached kernel takes one
// event per thread (the two-event form spills).
constexpr int GRAD_CTAS_PER_SM_KFLOAT = 4;

int nk_bucket(int nk);
// Gradient slots: ln S (or w S), 6 per K* of the bucket, 4 per Z, and 2 (mass,
// width) per floated resonance, in the order of their parameters.
int grad_num_slots(int nk_max, int nz, int n_float);
int eval_block();
int grad_block();

cudaError_t launch_eval(const LaunchArgs &a, int mode);  // 0 ln S, 1 w S, 2 write S
cudaError_t launch_grad(const LaunchArgs &a, bool norm);
cudaError_t launch_lcache(const LaunchArgs &a, float2 *lc);
cudaError_t launch_reduce_cols(const double *part, int nblk, int ncol, double *out,
                               cudaStream_t s);
// Generator with Eq. 14 templates: S <- alpha eps S + beta hb per candidate.
cudaError_t launch_eq14_density(float *S, const float *eps, const float *hb, int64_t n, double alpha,
                                double beta, cudaStream_t s);
cudaError_t launch_pdf_scale(const float *rec, int64_t npad, int64_t n, double alpha, double beta,
                             const float *eps, const float *hb, float *S, cudaStream_t s);
cudaError_t launch_finish(const unsigned long long *ad, const unsigned long long *an, const int *slot_param,
                          const double *pscale, int nslot, int nparam, double n_events,
                          double lnpq, double vol_over_n, const unsigned *status, double *out,
                          cudaStream_t s, const unsigned long long *ar = nullptr);
// Eq. 14 with a background: alpha = P / I_eps into the device table, I_eps =
// vol_over_n times the point sum in an.
cudaError_t launch_mix_alpha(const unsigned long long *an, double vol_over_n, double purity,
                             ModelDev *md, unsigned *status, cudaStream_t s);

// couplings_only: refresh the folded couplings of a table whose masses and
// widths are all fixed and which has had one full build.
// acc (nacc words, may be null): the evaluation's 128-bit accumulators, zeroed.
cudaError_t launch_build_table(const ModelStatic *st, const double *params, ModelDev *md,
                               double *pscale, unsigned *status, cudaStream_t s,
                               bool couplings_only = false, unsigned long long *acc = nullptr,
                               int nacc = 0);
cudaError_t launch_finish_gram(const unsigned long long *ad, const int *slot_param, const double *pscale,
                               int nslot, int ncol, int nparam, double n_events, double lnpq,
                               double vol_over_n, const double *params, const double *G,
                               const unsigned *status, double *out, int with_grad, cudaStream_t s,
                               double n_points = 0.0, int partials = 0,
                               const unsigned long long *ar = nullptr, ModelDev *alpha_md = nullptr,
                               double purity = 1.0);
cudaError_t launch_partials(const unsigned long long *ad, const unsigned long long *an, const int *slot_param,
                            const double *pscale, int nslot, int nparam, double n_events,
                            double lnpq, double n_points, double volume, const unsigned *status,
                            double *out, cudaStream_t s);

// Normalisation Gram matrix (amp4d_gram.cu).
struct GramArgs {
    const float *rec;        // normalisation-point records (weights in record wrec)
    int64_t npad, n;
    int wrec;
    const ModelDev *md;
    float *xb;               // basis matrix (scratch): 2 dim x gram_basis_points(n) floats
    unsigned *colmax;        // 64 (scratch)
    float *gscale;           // 64 (scratch): fixed-point scale per real column
    long long *part;         // grid_tc x 4096 INT64 partials (scratch)
    int *err;                // set to 1 if a bounded wait expired
    double *G;               // dim x dim output
    int dim;                 // 2 K
    int nsm, grid_tc;
    int nk_max, nz;
    cudaStream_t stream;
};
cudaError_t launch_gram(const GramArgs &a);
cudaError_t launch_gram_selftest(const int *synth, int64_t n, long long *part, int grid, int *err,
                                 long long *out, cudaStream_t st);
int gram_chunk_points();
// Points the basis matrix holds for n points: n rounded up to whole chunks.
int64_t gram_basis_points(int64_t n);

// Generator and learned proposal (amp4d_proposal.cu).
cudaError_t launch_gen_candidates(float *rec, int64_t npad, int64_t n, uint64_t first,
                                  uint32_t stream_id, uint64_t seed, double m_lo, double m_hi,
                                  float *uacc, cudaStream_t st);
int gen_tile();
cudaError_t launch_gen_accept(const float *rec, int64_t npad, int64_t n, const float *S,
                              const float *uacc, double fmax, unsigned *blk_count, unsigned *over,
                              unsigned *fmax_bits, cudaStream_t st);
cudaError_t launch_gen_scatter(const float *rec, int64_t npad, int64_t n, const float *S,
                               const float *uacc, double fmax, const unsigned *blk_count,
                               unsigned long long *off, int64_t base, int64_t n_want, float *om,
                               float *ocK, float *ocpsi, float *ophi, cudaStream_t st);
int mlp_num_params();
void mlp_init_params(float *th, uint64_t seed);
cudaError_t launch_mlp_forward(const __nv_bfloat16 *wb, const float *x, int64_t n, float *g,
                               cudaStream_t st);
cudaError_t launch_mlp_grid(const __nv_bfloat16 *wb, const int nb[4], float *g, cudaStream_t st);
size_t mlp_grad_smem();
int mlp_grad_blocks(int64_t nd, int64_t nu);
cudaError_t launch_mlp_grad(const __nv_bfloat16 *wb, const float *xd, int64_t nd, const float *xu,
                            int64_t nu, float *part, double *out, cudaStream_t st);
cudaError_t launch_adam(float *th, float *m, float *v, const double *grad, float lr, float b1,
                        float b2, float eps, int64_t t, __nv_bfloat16 *wb, cudaStream_t st);
cudaError_t launch_to_bf16(const float *th, __nv_bfloat16 *wb, cudaStream_t st);
cudaError_t launch_mlp_batch(const float *em, const float *ecK, const float *ecpsi, const float *ephi,
                             int64_t n, int64_t nd, int64_t nu, uint64_t seed, uint64_t step,
                             double m_lo, double m_hi, float *xd, float *xu, cudaStream_t st);
int64_t cdf_scratch(int64_t ncell);
cudaError_t launch_grid_cdf(const float *g, int64_t ncell, double alpha, double *scratch,
                            double *cdf, cudaStream_t st);
cudaError_t launch_grid_sample(const double *cdf, const int nb[4], uint64_t seed, int64_t n,
                               double m_lo, double m_hi, double mB, double mpsi, double mK,
                               double mpi, float *om, float *ocK, float *ocpsi, float *ophi, float *w,
                               int64_t *cell, cudaStream_t st);

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

// Eq. 14 templates of one set (k_templates): per point eps and hb, or for a
// normalisation set the weight record rewritten as w0 eps; per-block FP64
// partials of sum ln eps (data) or sum w0 hb (points).
struct TplDev {
    const float *h;   // nullptr: unset
    int nx, ny;
    double xlo, xhi, ylo, yhi;
};
struct TplArgs {
    const float *rec;
    int64_t npad, n;
    float *eps, *hb;          // data sets: per-event outputs (npad values each)
    const float *w0;          // normalisation sets: weights as loaded
    const float *tag;         // data sets: flavour tags (the stored phi is tag x observed phi), or null
    float *wout;              // normalisation sets: the weight record to rewrite
    TplDev t[4];              // efficiency x masses, x angles; background x masses, x angles
    double mB, mpsi, mK, mpi;
    double *part;             // per-block partials (grid values)
    int grid;
    cudaStream_t stream;
};
cudaError_t launch_templates(const TplArgs &a);
// Flavour-align the stored events: the phi-odd records of event e are multiplied
// by old_tag[e] x new_tag[e] (null = all +1).
cudaError_t launch_flavour(float *rec, int64_t npad, int64_t n, const float *old_tag,
                           const float *new_tag, int has_z, int grid, cudaStream_t st);

}  // namespace amp4d
