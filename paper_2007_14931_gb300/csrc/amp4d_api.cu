// C ABI of the amplitude-fit library: model set-up, event ingest, evaluation.
//
// An evaluation is a fixed sequence on one stream: k_build_table turns the
// parameter vector (device memory) into the FP32 table of Eq. 2-3 constants,
// the per-event kernels run over the data events and the normalisation points,
// the block partials are reduced in a fixed order and k_finish assembles the
// NLL (and gradient) into a device output block.  The synchronous calls stage
// the host parameters into a device buffer, enqueue that sequence and copy the
// output block back in one transfer.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/amp4d.h"
#include "amp4d_device.cuh"
#include "amp4d_launch.h"

using namespace amp4d;

namespace {

struct EventSet {
    float *rec = nullptr;
    int64_t n = 0, npad = 0;
    int nrec = 0, wrec = -1;
    double lnpq = 0.0;
    double volume = 0.0;
    int grid_eval = 0, grid_grad = 0, grid_grad_cached = 0;
    double *part = nullptr;     // per-block partials (grid_grad x nslot)
    size_t part_cap = 0;
    float2 *lcache = nullptr;   // basis cache [resonance][npad] (cached path)
    bool lcache_valid = false;
    // Eq. 14 templates: data sets hold eps and hb per event (npad each); a
    // normalisation set keeps its weights as loaded in w0 and its weight record
    // holds w0 eps.
    float *eps = nullptr, *hb = nullptr, *w0 = nullptr;
    float *tag = nullptr;       // data: flavour tags (+1 B0, -1 B0bar); the stored phi is tag x phi
    double lneps = 0.0;         // data: sum ln eps over the events
    double whb = 0.0;           // points: sum w0 hb
};

thread_local std::string g_create_error;

}  // namespace

struct amp4d_model {
    int device = 0;
    int nsm = 0;
    amp4d_particle_masses mass{};
    std::vector<amp4d_resonance> res;
    std::vector<int> internal;   // internal order (K* first, then Z) -> user index
    std::vector<int> res_col;    // user resonance -> first column
    std::vector<int> res_fpos;   // user resonance -> float position or -1
    std::vector<int> col_res, col_lam;
    int nK = 0, nZ = 0, n_col = 0, n_float = 0, n_param = 0, nk_max = 2;
    int nslot = 0;
    double m_lo = 0, m_hi = 0;
    int path = AMP4D_PATH_PLAIN;
    EventSet ev, mc;
    ModelDev *d_md = nullptr;
    ModelStatic *d_static = nullptr;
    double *d_params = nullptr, *h_params = nullptr;
    double *d_pscale = nullptr;   // per-parameter gradient scale (folded column constants)
    // per-phase device timing: table, data kernel, normalisation kernel, reductions
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::vector<cudaEvent_t>> prof_pending;
    double prof_ms[4] = {0, 0, 0, 0};
    int64_t prof_n[4] = {0, 0, 0, 0};
    int *d_slot_param = nullptr;
    unsigned long long *d_acc = nullptr;   // 128-bit sums: [data, points][nslot][hi, lo], R
    double *d_guv = nullptr;               // G u and G v of the fused Gram finish (2 x 64)
    double *d_out = nullptr, *h_out = nullptr;
    // Replay of the synchronous evaluations (run_eval) as CUDA graphs of the
    // parameter copy, the evaluation's launches and the result copy, captured on a
    // private stream.  state_gen counts the calls that may change what an
    // evaluation enqueues; a graph is captured on the second call at one
    // generation (the first may build the table, the caches or the Gram) and
    // replayed while the generation holds.
    uint64_t state_gen = 0;
    cudaStream_t cap_stream = nullptr;
    struct EvalGraph {
        cudaGraphExec_t exec = nullptr;
        uint64_t gen = ~0ull;
        int calls = 0;
        bool failed = false;
    } graphs[2][2];   // [with_grad][partials]
    unsigned *d_status = nullptr;
    unsigned long long *d_bad = nullptr;
    double *d_tmp = nullptr;     // scratch for set-up reductions
    size_t tmp_cap = 0;
    // normalisation Gram matrix (cached path)
    double *d_G = nullptr;           // 2K x 2K, folded basis
    long long *d_gram_part = nullptr;
    float *d_gram_x = nullptr;       // basis matrix of the points (Gram build scratch)
    size_t gram_x_cap = 0;           // its size in floats
    unsigned *d_colmax = nullptr;
    float *d_gscale = nullptr;
    int *d_gram_err = nullptr;
    int gram_grid = 0;
    bool gram_valid = false;
    bool table_built = false;    // one full table build enqueued (all masses fixed)
    // Eq. 14: templates [efficiency x masses, x angles, background x masses, x angles]
    float *d_tpl[4] = {nullptr, nullptr, nullptr, nullptr};
    TplDev tpl[4] = {};
    bool has_eff = false, has_bkg = false;
    double purity = 1.0;
    bool eff_phi_even = true;    // the angular efficiency template is even in phi
    bool kstar_fixed = true;     // no K* has a floating mass or width
    double mistag = 0.0;         // flavour mistag fraction
    // learned proposal
    float *d_th = nullptr, *d_am = nullptr, *d_av = nullptr;   // FP32 master weights, Adam moments
    __nv_bfloat16 *d_wb = nullptr;                              // BF16 weights
    float *d_gcell = nullptr;
    double *d_cdf = nullptr;
    int nb[4] = {0, 0, 0, 0};
    bool proposal_ready = false;
    std::string err;
};

namespace {

amp4d_status fail(amp4d_model *m, amp4d_status code, const std::string &msg)
{
    if (m) m->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(model, e_ == cudaErrorMemoryAllocation ? AMP4D_ERR_OOM       \
                                                               : AMP4D_ERR_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

void build_slot_map(const amp4d_model *mo, std::vector<int> &map)
{
    const int NK = mo->nk_max, NZ = mo->nZ;
    map.assign(mo->nslot, -1);
    const int Z0 = 1 + 6 * NK, MG0 = 1 + 6 * NK + 4 * NZ;
    for (int i = 0; i < mo->nK; ++i) {
        const int u = mo->internal[i];
        const amp4d_resonance &r = mo->res[u];
        const int c = mo->res_col[u];
        if (r.J == 0) {
            map[1 + 6 * i + 2] = 2 * c;
            map[1 + 6 * i + 3] = 2 * c + 1;
        } else {
            for (int l = 0; l < 3; ++l) {
                map[1 + 6 * i + 2 * l] = 2 * (c + l);
                map[1 + 6 * i + 2 * l + 1] = 2 * (c + l) + 1;
            }
        }
        if (r.float_mg) {
            map[MG0 + 2 * mo->res_fpos[u]] = 2 * mo->n_col + 2 * mo->res_fpos[u];
            map[MG0 + 2 * mo->res_fpos[u] + 1] = 2 * mo->n_col + 2 * mo->res_fpos[u] + 1;
        }
    }
    for (int z = 0; z < mo->nZ; ++z) {
        const int u = mo->internal[mo->nK + z];
        const amp4d_resonance &r = mo->res[u];
        int c = mo->res_col[u];
        const int eta = -r.P * ((r.J % 2) ? -1 : 1);
        if (eta == 1) { map[Z0 + 4 * z] = 2 * c; map[Z0 + 4 * z + 1] = 2 * c + 1; ++c; }
        if (r.J >= 1) { map[Z0 + 4 * z + 2] = 2 * c; map[Z0 + 4 * z + 3] = 2 * c + 1; }
        if (r.float_mg) {
            map[MG0 + 2 * mo->res_fpos[u]] = 2 * mo->n_col + 2 * mo->res_fpos[u];
            map[MG0 + 2 * mo->res_fpos[u] + 1] = 2 * mo->n_col + 2 * mo->res_fpos[u] + 1;
        }
    }
}

amp4d_status ensure_tmp(amp4d_model *model, size_t n)
{
    if (model->tmp_cap >= n) return AMP4D_OK;
    if (model->d_tmp) cudaFree(model->d_tmp);
    model->d_tmp = nullptr;
    model->tmp_cap = 0;
    CK(cudaMalloc(&model->d_tmp, n * sizeof(double)));
    model->tmp_cap = n;
    return AMP4D_OK;
}

amp4d_status load_set(amp4d_model *model, EventSet &s, const float *m, const float *cK,
                      const float *cpsi, const float *phi, const float *w, int64_t n,
                      bool is_norm, cudaStream_t st)
{
    if (!m || !cK || !cpsi || !phi || n < 1) return fail(model, AMP4D_ERR_ARG, "null array or n < 1");
    CK(cudaSetDevice(model->device));
    if (s.rec) { cudaFree(s.rec); s.rec = nullptr; }
    if (s.part) { cudaFree(s.part); s.part = nullptr; }
    if (s.lcache) { cudaFree(s.lcache); s.lcache = nullptr; }
    for (float **b : {&s.eps, &s.hb, &s.w0, &s.tag})
        if (*b) { cudaFree(*b); *b = nullptr; }
    s.lneps = s.whb = 0.0;
    s.lcache_valid = false;
    s.n = 0;
    const int64_t npad = (n + 3) & ~int64_t(3);
    const int nrec = model->nZ > 0 ? REC_NZ : REC_NK;
    const int tot = nrec + (is_norm ? 1 : 0);
    CK(cudaMalloc(&s.rec, (size_t)tot * npad * sizeof(float)));
    const float *src[4] = {m, cK, cpsi, phi};
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(s.rec + k * npad, src[k], n * sizeof(float), cudaMemcpyDefault, st));
    if (is_norm && w)
        CK(cudaMemcpyAsync(s.rec + nrec * npad, w, n * sizeof(float), cudaMemcpyDefault, st));
    s.nrec = nrec;
    s.wrec = is_norm ? nrec : -1;
    s.npad = npad;
    PrepArgs a{};
    a.rec = s.rec;
    a.npad = npad;
    a.n = n;
    a.has_z = model->nZ > 0;
    a.wrec = s.wrec;
    a.have_w = (w != nullptr);
    a.mB = model->mass.mB; a.mpsi = model->mass.mpsi; a.mK = model->mass.mK; a.mpi = model->mass.mpi;
    a.m_lo = model->m_lo; a.m_hi = model->m_hi;
    a.grid = (int)std::min<int64_t>((npad + prepare_block() - 1) / prepare_block(), model->nsm * 8);
    amp4d_status rc = ensure_tmp(model, a.grid + 2);
    if (rc) return rc;
    a.part_lnpq = model->d_tmp;
    a.bad = model->d_bad;
    a.stream = st;
    CK(cudaMemsetAsync(model->d_bad, 0xff, sizeof(unsigned long long), st));
    CK(launch_prepare(a));
    CK(launch_reduce_cols(model->d_tmp, a.grid, 1, model->d_tmp + a.grid, st));
    double lnpq = 0;
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&lnpq, model->d_tmp + a.grid, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&bad, model->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad != ~0ull) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "%s %llu outside the box or not finite",
                      is_norm ? "normalisation point" : "event", bad);
        return fail(model, AMP4D_ERR_INPUT, buf);
    }
    s.lnpq = lnpq;
    s.grid_eval = (int)std::max<int64_t>(1, std::min<int64_t>((n + eval_block() - 1) / eval_block(),
                                                              (int64_t)model->nsm * 4));
    s.grid_grad = (int)std::max<int64_t>(1, std::min<int64_t>((n + grad_block() - 1) / grad_block(),
                                                              (int64_t)model->nsm * GRAD_CTAS_PER_SM));
    s.grid_grad_cached = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + grad_block() - 1) / grad_block(), (int64_t)model->nsm * GRAD_CTAS_PER_SM_CACHED));
    s.part_cap = (size_t)std::max(s.grid_eval, std::max(s.grid_grad, s.grid_grad_cached)) * model->nslot;
    CK(cudaMalloc(&s.part, s.part_cap * sizeof(double)));
    s.n = n;
    return AMP4D_OK;
}

// The per-evaluation table: a full FP64 build the first time, and always when a
// mass or width floats; afterwards only the folded couplings are rewritten.
cudaError_t enqueue_table(amp4d_model *mo, const double *d_params, cudaStream_t st)
{
    const bool fast = mo->n_float == 0 && mo->table_built;
    cudaError_t e = launch_build_table(mo->d_static, d_params, mo->d_md, mo->d_pscale, mo->d_status,
                                       st, fast, mo->d_acc, 4 * mo->nslot + 3);
    if (e == cudaSuccess && mo->n_float == 0) mo->table_built = true;
    return e;
}

// Grid of the adjoint kernel over a set: one full wave of the variant that runs.
int grad_grid(const amp4d_model *mo, const EventSet &s)
{
    // the all-cached kernel: two events per thread at GRAD_CTAS_PER_SM_CACHED, or one
    // per thread at GRAD_CTAS_PER_SM_KFLOAT (= GRAD_CTAS_PER_SM) with floated K*
    static_assert(GRAD_CTAS_PER_SM_KFLOAT == GRAD_CTAS_PER_SM, "one-event grid");
    const bool cached = mo->path == AMP4D_PATH_CACHED && s.lcache_valid && mo->kstar_fixed;
    return cached ? s.grid_grad_cached : s.grid_grad;
}

LaunchArgs args_for(amp4d_model *mo, EventSet &s, double *part, float *out, cudaStream_t st,
                    int grid)
{
    LaunchArgs a{};
    a.rec = s.rec;
    a.npad = s.npad;
    a.n = s.n;
    a.wrec = s.wrec;
    a.md = mo->d_md;
    a.part = part;
    a.out = out;
    a.status = mo->d_status;
    a.grid = grid;
    a.nk_max = mo->nk_max;
    a.nz = mo->nZ;
    a.stream = st;
    a.lcache = (mo->path == AMP4D_PATH_CACHED && s.lcache_valid) ? s.lcache : nullptr;
    a.nrow = (int)mo->res.size() + 4 * mo->nZ;
    a.nk = (int)mo->res.size() - mo->nZ;
    a.nj0 = 0;
    a.zboth = true;
    for (int u : mo->internal) {
        const amp4d_resonance &r = mo->res[u];
        if (r.chain == AMP4D_CHAIN_KSTAR && r.J == 0) ++a.nj0;
        // a Z has the l' = 0 column when its parity factor is +1, l' = +-1 when J >= 1
        if (r.chain == AMP4D_CHAIN_Z && (-r.P * ((r.J % 2) ? -1 : 1) != 1 || r.J < 1)) a.zboth = false;
    }
    a.nslot = mo->nslot;
    a.all_fixed = mo->n_float == 0;
    a.kstar_fixed = mo->kstar_fixed;
    a.acc = (&s == &mo->ev) ? mo->d_acc : mo->d_acc + 2 * mo->nslot;
    a.mt = (&s == &mo->ev) && mo->mistag > 0.0;
    if (&s == &mo->ev && mo->has_bkg && mo->purity < 1.0 && s.eps && s.hb) {
        a.mix_eps = s.eps;
        a.mix_hb = s.hb;
        a.acc_r = mo->d_acc + 4 * mo->nslot;
    }
    return a;
}

// Basis cache of a set for the current (fixed) masses and widths; the table
// must already be on the stream.  Allocates on first use.
amp4d_status ensure_lcache(amp4d_model *model, EventSet &s, cudaStream_t st)
{
    if (s.lcache_valid || s.n == 0) return AMP4D_OK;
    // lineshape rows, then the four angular-factor rows of each Z
    const size_t rows = model->res.size() + 4 * (size_t)model->nZ;
    if (!s.lcache) CK(cudaMalloc(&s.lcache, rows * s.npad * sizeof(float2)));
    LaunchArgs a = args_for(model, s, nullptr, nullptr, st, model->nsm * 8);
    CK(launch_lcache(a, s.lcache));
    s.lcache_valid = true;
    return AMP4D_OK;
}

amp4d_status check_params(amp4d_model *model, const double *params)
{
    if (!params) return fail(model, AMP4D_ERR_ARG, "params is null");
    for (int i = 0; i < model->n_param; ++i)
        if (!std::isfinite(params[i])) return fail(model, AMP4D_ERR_ARG, "non-finite parameter");
    for (size_t u = 0; u < model->res.size(); ++u) {
        if (!model->res[u].float_mg) continue;
        const double M = params[2 * model->n_col + 2 * model->res_fpos[u]];
        const double G = params[2 * model->n_col + 2 * model->res_fpos[u] + 1];
        if (!(M > 0.0) || !(G > 0.0)) return fail(model, AMP4D_ERR_ARG, "mass and width must be > 0");
    }
    return AMP4D_OK;
}

cudaEvent_t prof_event(amp4d_model *m)
{
    if (!m->ev_pool.empty()) {
        cudaEvent_t e = m->ev_pool.back();
        m->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Eq. 14 with a background: the data term mixes signal and background.
bool mixing(const amp4d_model *m) { return m->has_bkg && m->purity < 1.0; }

bool use_gram(const amp4d_model *m)
{
    return m->path == AMP4D_PATH_CACHED && m->n_float == 0 && 2 * m->n_col <= 64;
}

// Build the normalisation Gram matrix for the masses and widths in d_params
// (synchronous; checks the kernel's bounded-wait flag).
amp4d_status build_gram(amp4d_model *model, cudaStream_t st)
{
    if (model->mc.n == 0) return fail(model, AMP4D_ERR_STATE, "no normalisation points");
    if (2 * model->n_col > 64) return fail(model, AMP4D_ERR_ARG, "Gram matrix supports at most 32 columns");
    if (!model->d_G) {
        model->gram_grid = model->nsm;
        CK(cudaMalloc(&model->d_G, 64 * 64 * sizeof(double)));
        CK(cudaMalloc(&model->d_gram_part, (size_t)model->gram_grid * 4096 * sizeof(long long)));
        CK(cudaMalloc(&model->d_colmax, 64 * sizeof(unsigned)));
        CK(cudaMalloc(&model->d_gscale, 64 * sizeof(float)));
        CK(cudaMalloc(&model->d_gram_err, sizeof(int)));
    }
    // the basis matrix: 2 dim floats per point (kept for later builds at new masses)
    const size_t nx = (size_t)gram_basis_points(model->mc.n) * 2 * (2 * model->n_col);
    if (nx > model->gram_x_cap) {
        if (model->d_gram_x) CK(cudaFree(model->d_gram_x));
        model->d_gram_x = nullptr;
        model->gram_x_cap = 0;
        CK(cudaMalloc(&model->d_gram_x, nx * sizeof(float)));
        model->gram_x_cap = nx;
    }
    CK(cudaMemsetAsync(model->d_gram_err, 0, sizeof(int), st));
    CK(enqueue_table(model, model->d_params, st));
    GramArgs g{};
    g.rec = model->mc.rec;
    g.npad = model->mc.npad;
    g.n = model->mc.n;
    g.wrec = model->mc.wrec;
    g.md = model->d_md;
    g.xb = model->d_gram_x;
    g.colmax = model->d_colmax;
    g.gscale = model->d_gscale;
    g.part = model->d_gram_part;
    g.err = model->d_gram_err;
    g.G = model->d_G;
    g.dim = 2 * model->n_col;
    g.nsm = model->nsm;
    const int64_t nchunks = (model->mc.n + gram_chunk_points() - 1) / gram_chunk_points();
    g.grid_tc = (int)std::max<int64_t>(1, std::min<int64_t>(model->gram_grid, nchunks));
    g.nk_max = model->nk_max;
    g.nz = model->nZ;
    g.stream = st;
    CK(launch_gram(g));
    int err = 0;
    CK(cudaMemcpyAsync(&err, model->d_gram_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) return fail(model, AMP4D_ERR_TIMEOUT, "Gram kernel: a bounded wait expired");
    model->gram_valid = true;
    return AMP4D_OK;
}

// Enqueue one evaluation on stream st (no synchronisation).
// partials: write the shard partials (k_partials layout) instead of the NLL.
amp4d_status enqueue(amp4d_model *model, bool with_grad, const double *d_params, double *d_out,
                     cudaStream_t st, bool partials = false)
{
    if (model->ev.n == 0 || model->mc.n == 0)
        return fail(model, AMP4D_ERR_STATE, "set_events and set_norm_points must come first");
    const bool mix = mixing(model);
    if (mix && partials)
        return fail(model, AMP4D_ERR_STATE, "shard partials are not available with a background");
    if (mix && !(model->mc.whb > 0.0))
        return fail(model, AMP4D_ERR_DOMAIN, "the background template is 0 over the normalisation points");
    // Parameter-independent part of ln f per event: ln(p q), and ln eps with an
    // efficiency but no background (with a background eps sits inside g).
    const double lnconst = model->ev.lnpq + (mix ? 0.0 : model->ev.lneps);
    const unsigned long long *ar = mix ? model->d_acc + 4 * model->nslot : nullptr;
    std::vector<cudaEvent_t> marks;
    auto mark = [&]() {
        if (!model->prof_on) return cudaSuccess;
        cudaEvent_t e = prof_event(model);
        marks.push_back(e);
        return cudaEventRecord(e, st);
    };
    CK(mark());
    CK(enqueue_table(model, d_params, st));
    if (model->path == AMP4D_PATH_CACHED) {
        amp4d_status rc = ensure_lcache(model, model->ev, st);
        if (rc == AMP4D_OK && !use_gram(model)) rc = ensure_lcache(model, model->mc, st);
        if (rc) return rc;
    }
    CK(mark());
    // The kernels add their sums to the 128-bit accumulators the table kernel
    // zeroed; the finishing kernel reads them (no separate reduction launch).
    const unsigned long long *ad = model->d_acc, *an = model->d_acc + 2 * model->nslot;
    if (use_gram(model)) {
        if (!model->gram_valid) {
            amp4d_status rc = build_gram(model, st);
            if (rc) return rc;
        }
        const double von = model->mc.volume / (double)model->mc.n;
        if (mix)   // alpha = P / I_eps from the Gram quadratic form, before the data pass
            CK(launch_finish_gram(ad, model->d_slot_param, model->d_pscale, model->nslot, model->n_col,
                                  model->n_param, (double)model->ev.n, lnconst, von, d_params,
                                  model->d_G, model->d_status, d_out, 0, st, (double)model->mc.n, 0,
                                  nullptr, model->d_md, model->purity));
        // With the gradient the data kernel's last CTA finishes
        // the evaluation (no separate launch).
        bool fused = false;
        if (with_grad) {
            LaunchArgs la = args_for(model, model->ev, model->ev.part, nullptr, st, grad_grid(model, model->ev));
            // the all-cached kernel carries the finish (with a background too: alpha was
            // set before the data pass, and the signal-probability sum is added before
            // the CTA takes its ticket); its first n_col CTAs form G u, G v
            fused = la.lcache != nullptr && la.grid >= model->n_col;
            if (fused) {
                FinishArgs &f = la.fin;
                f.ad = ad; f.slot_param = model->d_slot_param; f.pscale = model->d_pscale;
                f.nslot = model->nslot; f.ncol = model->n_col; f.nparam = model->n_param;
                f.n_events = (double)model->ev.n; f.lnpq = lnconst; f.vol_over_n = von;
                f.params = d_params; f.G = model->d_G; f.status = model->d_status; f.out = d_out;
                f.with_grad = 1; f.n_points = (double)model->mc.n; f.partials = partials ? 1 : 0;
                f.ar = ar;
                f.ticket = reinterpret_cast<unsigned *>(model->d_acc + 4 * model->nslot + 2);
                f.guv = model->d_guv;
            }
            CK(launch_grad(la, false));
        } else {
            LaunchArgs la = args_for(model, model->ev, model->ev.part, nullptr, st, model->ev.grid_eval);
            CK(launch_eval(la, 0));
        }
        CK(mark());
        CK(mark());
        if (!fused)
            CK(launch_finish_gram(ad, model->d_slot_param, model->d_pscale, model->nslot, model->n_col,
                                  model->n_param, (double)model->ev.n, lnconst, von, d_params,
                                  model->d_G, model->d_status, d_out, with_grad ? 1 : 0, st,
                                  (double)model->mc.n, partials ? 1 : 0, ar));
        CK(mark());
        if (model->prof_on) model->prof_pending.push_back(marks);
        return AMP4D_OK;
    }
    // Data pass and point pass.  With a background the point pass runs first:
    // the data pass needs alpha = P / I_eps (the profile's second interval is
    // then the point pass, the third the data pass).
    const double von = model->mc.volume / (double)model->mc.n;
    auto data_pass = [&]() -> cudaError_t {
        LaunchArgs ld = args_for(model, model->ev, model->ev.part, nullptr, st,
                                 with_grad ? grad_grid(model, model->ev) : model->ev.grid_eval);
        return with_grad ? launch_grad(ld, false) : launch_eval(ld, 0);
    };
    auto point_pass = [&]() -> cudaError_t {
        LaunchArgs ln = args_for(model, model->mc, model->mc.part, nullptr, st,
                                 with_grad ? grad_grid(model, model->mc) : model->mc.grid_eval);
        return with_grad ? launch_grad(ln, true) : launch_eval(ln, 1);
    };
    if (mix) {
        CK(point_pass());
        CK(mark());
        CK(launch_mix_alpha(an, von, model->purity, model->d_md, model->d_status, st));
        CK(data_pass());
        CK(mark());
    } else {
        CK(data_pass());
        CK(mark());
        CK(point_pass());
        CK(mark());
    }
    const int *slots = with_grad ? model->d_slot_param : nullptr;
    const int nsl = with_grad ? model->nslot : 1, npar = with_grad ? model->n_param : 0;
    if (partials)
        CK(launch_partials(ad, an, slots, model->d_pscale, nsl, npar, (double)model->ev.n, lnconst,
                           (double)model->mc.n, model->mc.volume, model->d_status, d_out, st));
    else
        CK(launch_finish(ad, an, slots, model->d_pscale, nsl, npar, (double)model->ev.n, lnconst,
                         von, model->d_status, d_out, st, ar));
    CK(mark());
    if (model->prof_on) model->prof_pending.push_back(marks);
    return AMP4D_OK;
}

// Synchronous evaluation from host parameters; leaves the output block in h_out.
// The copy-in, the evaluation and the copy-out of run_eval on stream st.
amp4d_status enqueue_sync_eval(amp4d_model *model, bool with_grad, bool partials, cudaStream_t st)
{
    CK(cudaMemcpyAsync(model->d_params, model->h_params, model->n_param * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    amp4d_status rc = enqueue(model, with_grad, model->d_params, model->d_out, st, partials);
    if (rc) return rc;
    const size_t nout = 6 + (with_grad ? (partials ? 2 : 1) * model->n_param : 0);
    CK(cudaMemcpyAsync(model->h_out, model->d_out, nout * sizeof(double), cudaMemcpyDeviceToHost, st));
    return AMP4D_OK;
}

void drop_graph(amp4d_model::EvalGraph &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = amp4d_model::EvalGraph{};
}

// Capture the evaluation into g.exec, on the pinned parameter and result
// buffers; false if it cannot be captured (the call then runs
// enqueue_sync_eval directly).
bool capture_eval_graph(amp4d_model *model, bool with_grad, bool partials, amp4d_model::EvalGraph &g)
{
    if (!model->cap_stream &&
        cudaStreamCreateWithFlags(&model->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        model->cap_stream = nullptr;
        return false;
    }
    cudaStream_t cs = model->cap_stream;
    const std::string saved_err = model->err;
    // The graph's kernels read the parameters from, and write the result block to,
    // the model's pinned host buffers directly (their device-side addresses), so it
    // holds no copy nodes.  Every call writes h_params before the launch and reads
    // h_out after the synchronisation.
    double *dp = nullptr, *dout = nullptr;
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&dp), model->h_params, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&dout), model->h_out, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const amp4d_status rc = enqueue(model, with_grad, dp, dout, cs, partials);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    bool ok = rc == AMP4D_OK && e == cudaSuccess && graph != nullptr;
    if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        g.exec = nullptr;
        cudaGetLastError();   // a failed capture leaves no sticky error; clear the last one
        model->err = saved_err;
    }
    return ok;
}

// Synchronous evaluation from host parameters; leaves the output block in h_out.
// Repeated calls at one state generation replay a CUDA graph of the sequence.
amp4d_status run_eval(amp4d_model *model, const double *params, bool with_grad, cudaStream_t st,
                      bool partials = false)
{
    amp4d_status rc = check_params(model, params);
    if (rc) return rc;
    CK(cudaSetDevice(model->device));
    std::memcpy(model->h_params, params, model->n_param * sizeof(double));
    amp4d_model::EvalGraph &g = model->graphs[with_grad ? 1 : 0][partials ? 1 : 0];
    if (g.gen != model->state_gen) {
        drop_graph(g);
        g.gen = model->state_gen;
    }
    ++g.calls;
    if (!g.exec && !g.failed && !model->prof_on && g.calls >= 2)
        g.failed = !capture_eval_graph(model, with_grad, partials, g);
    if (g.exec && !model->prof_on) {
        CK(cudaGraphLaunch(g.exec, st));
    } else {
        rc = enqueue_sync_eval(model, with_grad, partials, st);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(st));
    if (((unsigned)model->h_out[5]) & 2u) return fail(model, AMP4D_ERR_ARG, "invalid parameters");
    return AMP4D_OK;
}

ModelStatic make_static(const amp4d_model *mo)
{
    ModelStatic s;
    std::memset(&s, 0, sizeof s);
    s.mB = mo->mass.mB; s.mpsi = mo->mass.mpsi; s.mK = mo->mass.mK; s.mpi = mo->mass.mpi;
    s.n_res = (int)mo->res.size();
    s.n_col = mo->n_col;
    s.n_float = mo->n_float;
    s.n_param = mo->n_param;
    // Eq. 14: beta = (1 - P) / B, B = (V / n) sum w0 hb over the normalisation points
    const double B = mo->mc.n > 0 ? mo->mc.volume / (double)mo->mc.n * mo->mc.whb : 0.0;
    s.mix_beta = (mixing(mo) && B > 0.0) ? (1.0 - mo->purity) / B : 0.0;
    s.mistag = mo->mistag;
    for (size_t i = 0; i < mo->internal.size(); ++i) {
        const int u = mo->internal[i];
        const amp4d_resonance &r = mo->res[u];
        ResStatic &d = s.res[i];
        d.M = r.M; d.G0 = r.G0; d.r = r.r;
        d.chain = r.chain; d.J = r.J; d.LB = r.LB; d.LR = r.LR;
        d.shape = r.shape;
        if (r.shape == AMP4D_SHAPE_LASS) {
            // Eq. 7 is the whole mass dependence: no barrier factors.
            d.LB = d.LR = 0;
            d.lass_a = r.lass_a; d.lass_b = r.lass_b; d.lass_R = r.lass_R;
        }
        d.col = mo->res_col[u];
        d.fpos = mo->res_fpos[u];
        d.eta = -r.P * ((r.J % 2) ? -1 : 1);
        d.zcol0 = d.zcol1 = -1;
        if (r.chain == AMP4D_CHAIN_Z) {
            int c = mo->res_col[u];
            if (d.eta == 1) d.zcol0 = c++;
            if (r.J >= 1) d.zcol1 = c;
        }
    }
    return s;
}

// Eq. 14 templates over one loaded set: a data set gets eps and hb per event and
// sum ln eps; a normalisation set gets the weight record w0 eps (w0 = the weights
// as loaded, kept) and sum w0 hb.  Without templates the set is restored.
amp4d_status apply_templates(amp4d_model *model, EventSet &s, bool is_norm, cudaStream_t st)
{
    if (s.n == 0) return AMP4D_OK;
    const bool any = model->has_eff || model->has_bkg;
    float *wrec = is_norm ? s.rec + (size_t)s.wrec * s.npad : nullptr;
    const size_t bytes = (size_t)s.npad * sizeof(float);
    if (!any) {
        if (is_norm && s.w0) {
            CK(cudaMemcpyAsync(wrec, s.w0, bytes, cudaMemcpyDeviceToDevice, st));
            CK(cudaStreamSynchronize(st));
            cudaFree(s.w0);
            s.w0 = nullptr;
            model->gram_valid = false;
        }
        for (float **b : {&s.eps, &s.hb})
            if (*b) { cudaFree(*b); *b = nullptr; }
        s.lneps = s.whb = 0.0;
        return AMP4D_OK;
    }
    if (is_norm) {
        if (!s.w0) {
            CK(cudaMalloc(&s.w0, bytes));
            CK(cudaMemcpyAsync(s.w0, wrec, bytes, cudaMemcpyDeviceToDevice, st));
        }
    } else {
        if (!s.eps) CK(cudaMalloc(&s.eps, bytes));
        if (!s.hb) CK(cudaMalloc(&s.hb, bytes));
    }
    TplArgs a{};
    a.rec = s.rec;
    a.npad = s.npad;
    a.n = s.n;
    a.eps = is_norm ? nullptr : s.eps;
    a.hb = is_norm ? nullptr : s.hb;
    a.w0 = is_norm ? s.w0 : nullptr;
    a.tag = is_norm ? nullptr : s.tag;
    a.wout = wrec;
    for (int i = 0; i < 4; ++i) a.t[i] = model->tpl[i];
    if (!model->has_eff) a.t[0].h = a.t[1].h = nullptr;
    if (!model->has_bkg) a.t[2].h = a.t[3].h = nullptr;
    a.mB = model->mass.mB; a.mpsi = model->mass.mpsi; a.mK = model->mass.mK; a.mpi = model->mass.mpi;
    a.grid = (int)std::min<int64_t>((s.npad + prepare_block() - 1) / prepare_block(), model->nsm * 8);
    amp4d_status rc = ensure_tmp(model, a.grid + 2);
    if (rc) return rc;
    a.part = model->d_tmp;
    a.stream = st;
    CK(launch_templates(a));
    CK(launch_reduce_cols(model->d_tmp, a.grid, 1, model->d_tmp + a.grid, st));
    double sum = 0.0;
    CK(cudaMemcpyAsync(&sum, model->d_tmp + a.grid, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (is_norm) {
        s.whb = sum;
        model->gram_valid = false;
    } else {
        s.lneps = sum;
    }
    return AMP4D_OK;
}

// After a change of templates or sets: the static table (beta of Eq. 14) and a
// full table build on the next evaluation.
amp4d_status refresh_static(amp4d_model *model)
{
    ModelStatic ms = make_static(model);
    CK(cudaMemcpy(model->d_static, &ms, sizeof ms, cudaMemcpyHostToDevice));
    model->table_built = false;
    return AMP4D_OK;
}

// Copy one template pair (mass, angle) into model slots t0, t0 + 1.
amp4d_status set_template_pair(amp4d_model *model, int t0, const amp4d_hist2d *mass,
                               const amp4d_hist2d *angle, cudaStream_t st)
{
    const amp4d_hist2d *src[2] = {mass, angle};
    for (int j = 0; j < 2; ++j) {
        const amp4d_hist2d *h = src[j];
        if (!h->h || h->nx < 1 || h->ny < 1 || (int64_t)h->nx * h->ny > (1 << 26) ||
            !(h->x_hi > h->x_lo) || !(h->y_hi > h->y_lo) || !std::isfinite(h->x_lo) ||
            !std::isfinite(h->x_hi) || !std::isfinite(h->y_lo) || !std::isfinite(h->y_hi))
            return fail(model, AMP4D_ERR_ARG, "bad template (null contents, bins or ranges)");
    }
    // contents must be finite and >= 0 (an efficiency or a density)
    for (int j = 0; j < 2; ++j) {
        const amp4d_hist2d *h = src[j];
        std::vector<float> c((size_t)h->nx * h->ny);
        CK(cudaMemcpy(c.data(), h->h, c.size() * sizeof(float), cudaMemcpyDefault));
        for (size_t i = 0; i < c.size(); ++i)
            if (!(c[i] >= 0.0f) || !std::isfinite(c[i])) {
                char buf[96];
                std::snprintf(buf, sizeof buf, "template bin %zu is negative or not finite", i);
                return fail(model, AMP4D_ERR_ARG, buf);
            }
    }
    for (int j = 0; j < 2; ++j) {
        const amp4d_hist2d *h = src[j];
        const int t = t0 + j;
        if (model->d_tpl[t]) { cudaFree(model->d_tpl[t]); model->d_tpl[t] = nullptr; }
        const size_t bytes = (size_t)h->nx * h->ny * sizeof(float);
        if (cudaMalloc(&model->d_tpl[t], bytes) != cudaSuccess)
            return fail(model, AMP4D_ERR_OOM, "template allocation failed");
        CK(cudaMemcpyAsync(model->d_tpl[t], h->h, bytes, cudaMemcpyDefault, st));
        model->tpl[t] = TplDev{model->d_tpl[t], h->nx, h->ny, h->x_lo, h->x_hi, h->y_lo, h->y_hi};
    }
    CK(cudaStreamSynchronize(st));
    return AMP4D_OK;
}

// Whether the angular efficiency template (slot 1: x = cos theta_psi, y = phi) is
// even in phi: a range symmetric about 0 and mirror-symmetric contents.
amp4d_status angular_template_phi_even(amp4d_model *model, int t, bool *even)
{
    const TplDev &d = model->tpl[t];
    *even = false;
    if (!(d.ylo == -d.yhi)) return AMP4D_OK;
    std::vector<float> h((size_t)d.nx * d.ny);
    CK(cudaMemcpy(h.data(), d.h, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (int iy = 0; iy < d.ny; ++iy)
        for (int ix = 0; ix < d.nx; ++ix)
            if (h[(size_t)iy * d.nx + ix] != h[(size_t)(d.ny - 1 - iy) * d.nx + ix]) return AMP4D_OK;
    *even = true;
    return AMP4D_OK;
}

bool flavour_active(const amp4d_model *m) { return m->mistag > 0.0 || m->ev.tag != nullptr; }

amp4d_status reapply_templates(amp4d_model *model, cudaStream_t st)
{
    amp4d_status rc = apply_templates(model, model->ev, false, st);
    if (rc == AMP4D_OK) rc = apply_templates(model, model->mc, true, st);
    if (rc == AMP4D_OK) rc = refresh_static(model);
    return rc;
}

}  // namespace

extern "C" {

amp4d_status amp4d_model_create(const amp4d_particle_masses *masses, const amp4d_resonance *res,
                                int n_res, double m_lo, double m_hi, int path, amp4d_model **out)
{
    amp4d_model *model = nullptr;
    if (!masses || !res || !out) return fail(nullptr, AMP4D_ERR_ARG, "null argument");
    *out = nullptr;
    if (n_res < 1 || n_res > AMP4D_MAX_RES) return fail(nullptr, AMP4D_ERR_ARG, "n_res out of range");
    if (!(m_lo > masses->mK + masses->mpi) || !(m_hi > m_lo))
        return fail(nullptr, AMP4D_ERR_ARG, "bad m_Kpi box");
    if (path != AMP4D_PATH_PLAIN && path != AMP4D_PATH_CACHED)
        return fail(nullptr, AMP4D_ERR_ARG, "unknown path");
    int nz = 0;
    for (int i = 0; i < n_res; ++i) {
        const amp4d_resonance &r = res[i];
        if (r.chain != AMP4D_CHAIN_KSTAR && r.chain != AMP4D_CHAIN_Z)
            return fail(nullptr, AMP4D_ERR_ARG, "bad chain");
        if (r.J < 0 || r.J > 4 || r.LB < 0 || r.LB > 4 || r.LR < 0 || r.LR > 4 ||
            (r.P != 1 && r.P != -1) || !(r.M > 0) || !(r.G0 > 0) || !(r.r >= 0))
            return fail(nullptr, AMP4D_ERR_ARG, "bad resonance record");
        if (r.shape != AMP4D_SHAPE_BW && r.shape != AMP4D_SHAPE_LASS)
            return fail(nullptr, AMP4D_ERR_ARG, "bad lineshape kind");
        if (r.shape == AMP4D_SHAPE_LASS &&
            (r.chain != AMP4D_CHAIN_KSTAR || r.J != 0 || r.float_mg || !(r.lass_a > 0) ||
             !(r.lass_b >= 0) || !(r.lass_R >= 0) || !std::isfinite(r.lass_a) ||
             !std::isfinite(r.lass_b) || !std::isfinite(r.lass_R)))
            return fail(nullptr, AMP4D_ERR_ARG,
                        "LASS: a fixed J = 0 K* with a > 0, b >= 0, R >= 0 (finite)");
        if (r.chain == AMP4D_CHAIN_Z) {
            ++nz;
            const int eta = -r.P * ((r.J % 2) ? -1 : 1);
            if (r.J == 0 && eta != 1) return fail(nullptr, AMP4D_ERR_ARG, "Z with no allowed helicity");
        }
    }
    if (nz > 2) return fail(nullptr, AMP4D_ERR_ARG, "at most 2 Z resonances");
    model = new amp4d_model();
    model->mass = *masses;
    model->res.assign(res, res + n_res);
    model->m_lo = m_lo;
    model->m_hi = m_hi;
    model->path = path;
    model->res_col.assign(n_res, 0);
    model->res_fpos.assign(n_res, -1);
    for (int i = 0; i < n_res; ++i) {
        const amp4d_resonance &r = res[i];
        model->res_col[i] = model->n_col;
        if (r.float_mg) {
            model->res_fpos[i] = model->n_float++;
            if (r.chain == AMP4D_CHAIN_KSTAR) model->kstar_fixed = false;
        }
        if (r.chain == AMP4D_CHAIN_KSTAR) {
            if (r.J == 0) { model->col_res.push_back(i); model->col_lam.push_back(0); }
            else for (int l = -1; l <= 1; ++l) { model->col_res.push_back(i); model->col_lam.push_back(l); }
        } else {
            const int eta = -r.P * ((r.J % 2) ? -1 : 1);
            if (eta == 1) { model->col_res.push_back(i); model->col_lam.push_back(0); }
            if (r.J >= 1) { model->col_res.push_back(i); model->col_lam.push_back(1); }
        }
        model->n_col = (int)model->col_res.size();
    }
    // Internal order: the K* of spin > 0, then the scalar K* (J = 0), then the Z,
    // each in the caller's order.  With the scalars last, a kernel specialised
    // for the number of scalars knows each K*'s class at compile time.
    for (int i = 0; i < n_res; ++i)
        if (res[i].chain == AMP4D_CHAIN_KSTAR && res[i].J != 0) model->internal.push_back(i);
    for (int i = 0; i < n_res; ++i)
        if (res[i].chain == AMP4D_CHAIN_KSTAR && res[i].J == 0) model->internal.push_back(i);
    for (int i = 0; i < n_res; ++i)
        if (res[i].chain == AMP4D_CHAIN_Z) model->internal.push_back(i);
    model->nZ = nz;
    model->nK = n_res - nz;
    model->n_param = 2 * model->n_col + 2 * model->n_float;
    model->nk_max = nk_bucket(model->nK);
    model->nslot = grad_num_slots(model->nk_max, nz, model->n_float);
    cudaError_t e = cudaGetDevice(&model->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&model->nsm, cudaDevAttrMultiProcessorCount, model->device);
    if (e == cudaSuccess) e = cudaMalloc(&model->d_md, sizeof(ModelDev));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_static, sizeof(ModelStatic));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_params, std::max(1, model->n_param) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_pscale, std::max(1, model->n_param) * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&model->h_params, std::max(1, model->n_param) * sizeof(double));
    if (e == cudaSuccess) {
        ModelStatic ms = make_static(model);
        e = cudaMemcpy(model->d_static, &ms, sizeof ms, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc(&model->d_slot_param, model->nslot * sizeof(int));
    // [data, points][nslot][hi, lo], then the Eq. 14 signal-probability sum
    // and the finishing ticket of the data kernel (zeroed with the sums)
    if (e == cudaSuccess) e = cudaMalloc(&model->d_acc, (4 * model->nslot + 3) * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_guv, 128 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_out, (6 + 2 * model->n_param) * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&model->h_out, (6 + 2 * model->n_param) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&model->d_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        std::vector<int> map;
        build_slot_map(model, map);
        e = cudaMemcpy(model->d_slot_param, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        std::string msg = std::string("model_create: ") + cudaGetErrorString(e);
        amp4d_status code = e == cudaErrorMemoryAllocation ? AMP4D_ERR_OOM : AMP4D_ERR_CUDA;
        amp4d_model_destroy(model);
        return fail(nullptr, code, msg);
    }
    *out = model;
    return AMP4D_OK;
}

amp4d_status amp4d_model_destroy(amp4d_model *model)
{
    if (!model) return AMP4D_OK;
    cudaSetDevice(model->device);
    for (EventSet *s : {&model->ev, &model->mc}) {
        if (s->rec) cudaFree(s->rec);
        if (s->part) cudaFree(s->part);
        if (s->lcache) cudaFree(s->lcache);
        for (float *b : {s->eps, s->hb, s->w0, s->tag})
            if (b) cudaFree(b);
    }
    for (float *t : model->d_tpl)
        if (t) cudaFree(t);
    if (model->d_md) cudaFree(model->d_md);
    if (model->d_static) cudaFree(model->d_static);
    if (model->d_params) cudaFree(model->d_params);
    if (model->d_pscale) cudaFree(model->d_pscale);
    if (model->h_params) cudaFreeHost(model->h_params);
    for (auto &v : model->prof_pending)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    for (cudaEvent_t e : model->ev_pool) cudaEventDestroy(e);
    if (model->d_slot_param) cudaFree(model->d_slot_param);
    if (model->d_acc) cudaFree(model->d_acc);
    if (model->d_guv) cudaFree(model->d_guv);
    if (model->d_out) cudaFree(model->d_out);
    if (model->h_out) cudaFreeHost(model->h_out);
    if (model->d_status) cudaFree(model->d_status);
    if (model->d_bad) cudaFree(model->d_bad);
    if (model->d_tmp) cudaFree(model->d_tmp);
    if (model->d_G) cudaFree(model->d_G);
    for (auto &row : model->graphs)
        for (auto &g : row) drop_graph(g);
    if (model->cap_stream) cudaStreamDestroy(model->cap_stream);
    if (model->d_gram_part) cudaFree(model->d_gram_part);
    if (model->d_gram_x) cudaFree(model->d_gram_x);
    if (model->d_colmax) cudaFree(model->d_colmax);
    if (model->d_gscale) cudaFree(model->d_gscale);
    if (model->d_gram_err) cudaFree(model->d_gram_err);
    for (void *ptr : {(void *)model->d_th, (void *)model->d_am, (void *)model->d_av, (void *)model->d_wb,
                      (void *)model->d_gcell, (void *)model->d_cdf})
        if (ptr) cudaFree(ptr);
    delete model;
    return AMP4D_OK;
}

const char *amp4d_last_error(const amp4d_model *model)
{
    return model ? model->err.c_str() : g_create_error.c_str();
}

int amp4d_num_columns(const amp4d_model *model) { return model ? model->n_col : -1; }
int amp4d_num_params(const amp4d_model *model) { return model ? model->n_param : -1; }

amp4d_status amp4d_set_events(amp4d_model *model, const float *m, const float *cK,
                              const float *cpsi, const float *phi, int64_t n, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model) return AMP4D_ERR_ARG;
    amp4d_status rc = load_set(model, model->ev, m, cK, cpsi, phi, nullptr, n, false, (cudaStream_t)stream);
    if (rc == AMP4D_OK) rc = apply_templates(model, model->ev, false, (cudaStream_t)stream);
    return rc;
}

amp4d_status amp4d_set_efficiency(amp4d_model *model, const amp4d_hist2d *mass,
                                  const amp4d_hist2d *angle, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || (!mass) != (!angle)) return model ? fail(model, AMP4D_ERR_ARG, "give both templates or neither") : AMP4D_ERR_ARG;
    CK(cudaSetDevice(model->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (mass) {
        amp4d_status rc = set_template_pair(model, 0, mass, angle, st);
        if (rc) return rc;
    }
    bool even = true;
    if (mass) {
        amp4d_status rc = angular_template_phi_even(model, 1, &even);
        if (rc) return rc;
    }
    if (mass && !even && flavour_active(model))
        return fail(model, AMP4D_ERR_STATE, "with flavour tags or a mistag the efficiency must be even in phi");
    model->has_eff = mass != nullptr;
    model->eff_phi_even = even;
    return reapply_templates(model, st);
}

amp4d_status amp4d_set_flavour(amp4d_model *model, const float *tag, double mistag, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model) return AMP4D_ERR_ARG;
    if (!(mistag >= 0.0 && mistag <= 0.5)) return fail(model, AMP4D_ERR_ARG, "mistag must lie in [0, 0.5]");
    EventSet &s = model->ev;
    if (tag && s.n == 0) return fail(model, AMP4D_ERR_STATE, "set_events must come first");
    if ((tag || mistag > 0.0) && model->has_eff && !model->eff_phi_even)
        return fail(model, AMP4D_ERR_STATE, "with flavour tags or a mistag the efficiency must be even in phi");
    CK(cudaSetDevice(model->device));
    cudaStream_t st = (cudaStream_t)stream;
    float *nt = nullptr;
    if (tag) {
        std::vector<float> h((size_t)s.n);
        CK(cudaMemcpy(h.data(), tag, h.size() * sizeof(float), cudaMemcpyDefault));
        for (int64_t e = 0; e < s.n; ++e)
            if (h[e] != 1.0f && h[e] != -1.0f) {
                char buf[96];
                std::snprintf(buf, sizeof buf, "tag %lld is not +1 or -1", (long long)e);
                return fail(model, AMP4D_ERR_ARG, buf);
            }
        if (cudaMalloc(&nt, (size_t)s.n * sizeof(float)) != cudaSuccess)
            return fail(model, AMP4D_ERR_OOM, "tag allocation failed");
        const cudaError_t e = cudaMemcpy(nt, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(nt);
            return fail(model, AMP4D_ERR_CUDA, std::string("set_flavour: ") + cudaGetErrorString(e));
        }
    }
    if (s.n > 0 && (s.tag || nt)) {
        const int grid = (int)std::min<int64_t>((s.npad + prepare_block() - 1) / prepare_block(), model->nsm * 8);
        cudaError_t e = launch_flavour(s.rec, s.npad, s.n, s.tag, nt, model->nZ > 0, grid, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            if (nt) cudaFree(nt);
            return fail(model, AMP4D_ERR_CUDA, std::string("set_flavour: ") + cudaGetErrorString(e));
        }
        // the cached Z-chain angular factors follow the rewritten phi-odd records
        if (model->nZ > 0) s.lcache_valid = false;
    }
    if (s.tag) cudaFree(s.tag);
    s.tag = nt;
    model->mistag = mistag;
    amp4d_status rc = apply_templates(model, s, false, st);
    if (rc == AMP4D_OK) rc = refresh_static(model);
    return rc;
}

amp4d_status amp4d_set_background(amp4d_model *model, const amp4d_hist2d *mass,
                                  const amp4d_hist2d *angle, double purity, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || (!mass) != (!angle)) return model ? fail(model, AMP4D_ERR_ARG, "give both templates or neither") : AMP4D_ERR_ARG;
    if (mass && !(purity >= 0.0 && purity <= 1.0)) return fail(model, AMP4D_ERR_ARG, "purity must lie in [0, 1]");
    CK(cudaSetDevice(model->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (mass) {
        amp4d_status rc = set_template_pair(model, 2, mass, angle, st);
        if (rc) return rc;
    }
    model->has_bkg = mass != nullptr;
    model->purity = mass ? purity : 1.0;
    return reapply_templates(model, st);
}

amp4d_status amp4d_set_norm_points(amp4d_model *model, const float *m, const float *cK,
                                   const float *cpsi, const float *phi, const float *w,
                                   int64_t n, double volume, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model) return AMP4D_ERR_ARG;
    if (!(volume > 0.0)) return fail(model, AMP4D_ERR_ARG, "volume must be > 0");
    model->gram_valid = false;
    amp4d_status rc = load_set(model, model->mc, m, cK, cpsi, phi, w, n, true, (cudaStream_t)stream);
    if (rc == AMP4D_OK) model->mc.volume = volume;
    if (rc == AMP4D_OK) rc = apply_templates(model, model->mc, true, (cudaStream_t)stream);
    if (rc == AMP4D_OK && model->has_bkg) rc = refresh_static(model);
    return rc;
}

amp4d_status amp4d_eval_nll(amp4d_model *model, const double *params, double *nll, void *stream)
{
    if (!model || !nll) return AMP4D_ERR_ARG;
    amp4d_status rc = run_eval(model, params, false, (cudaStream_t)stream);
    if (rc) return rc;
    *nll = model->h_out[0];
    if (model->h_out[5] != 0.0 || !std::isfinite(model->h_out[0])) {
        *nll = INFINITY;
        return fail(model, AMP4D_ERR_DOMAIN, "S <= 0 at a data event, p q = 0, or I <= 0");
    }
    return AMP4D_OK;
}

amp4d_status amp4d_eval_nll_grad(amp4d_model *model, const double *params, double *nll,
                                 double *grad, void *stream)
{
    if (!model || !nll || !grad) return AMP4D_ERR_ARG;
    amp4d_status rc = run_eval(model, params, true, (cudaStream_t)stream);
    if (rc) return rc;
    *nll = model->h_out[0];
    std::memcpy(grad, model->h_out + 6, model->n_param * sizeof(double));
    if (model->h_out[5] != 0.0 || !std::isfinite(model->h_out[0])) {
        *nll = INFINITY;
        return fail(model, AMP4D_ERR_DOMAIN, "S <= 0 at a data event, p q = 0, or I <= 0");
    }
    return AMP4D_OK;
}

amp4d_status amp4d_eval_terms(amp4d_model *model, const double *params, double *out, void *stream)
{
    if (!model || !out) return AMP4D_ERR_ARG;
    amp4d_status rc = run_eval(model, params, false, (cudaStream_t)stream);
    if (rc) return rc;
    out[0] = model->h_out[1];
    out[1] = model->h_out[2];
    out[2] = model->h_out[3];
    out[3] = model->h_out[4];
    return AMP4D_OK;
}

amp4d_status amp4d_eval_density(amp4d_model *model, const double *params, int which,
                                float *S_out, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !params || !S_out || (which != 0 && which != 1)) return AMP4D_ERR_ARG;
    EventSet &s = which == 0 ? model->ev : model->mc;
    if (s.n == 0) return fail(model, AMP4D_ERR_STATE, "no events loaded");
    cudaStream_t st = (cudaStream_t)stream;
    amp4d_status rc = check_params(model, params);
    if (rc) return rc;
    CK(cudaSetDevice(model->device));
    std::memcpy(model->h_params, params, model->n_param * sizeof(double));
    CK(cudaMemcpyAsync(model->d_params, model->h_params, model->n_param * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CK(enqueue_table(model, model->d_params, st));
    LaunchArgs a = args_for(model, s, s.part, S_out, st, s.grid_eval);
    CK(launch_eval(a, 2));
    CK(cudaStreamSynchronize(st));
    return AMP4D_OK;
}

amp4d_status amp4d_eval_pdf(amp4d_model *model, const double *params, float *pdf_out, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !params || !pdf_out) return AMP4D_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    amp4d_status rc = run_eval(model, params, false, st);   // I over the current points
    if (rc) return rc;
    const double I = model->h_out[3];   // I_eps with an efficiency
    if (!(I > 0.0) || !std::isfinite(I)) return fail(model, AMP4D_ERR_DOMAIN, "I <= 0");
    rc = amp4d_eval_density(model, params, 0, pdf_out, stream);
    if (rc) return rc;
    const bool mix = mixing(model);
    const double P = mix ? model->purity : 1.0;
    const double B = model->mc.volume / (double)model->mc.n * model->mc.whb;
    CK(launch_pdf_scale(model->ev.rec, model->ev.npad, model->ev.n, P / I,
                        mix ? (1.0 - P) / B : 0.0, model->has_eff ? model->ev.eps : nullptr,
                        mix ? model->ev.hb : nullptr, pdf_out, st));
    CK(cudaStreamSynchronize(st));
    return AMP4D_OK;
}

amp4d_status amp4d_enqueue_eval(amp4d_model *model, int what, const double *params, double *out,
                                void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !params || !out || (what != AMP4D_EVAL_NLL && what != AMP4D_EVAL_NLL_GRAD))
        return model ? fail(model, AMP4D_ERR_ARG, "bad enqueue arguments") : AMP4D_ERR_ARG;
    CK(cudaSetDevice(model->device));
    return enqueue(model, what == AMP4D_EVAL_NLL_GRAD, params, out, (cudaStream_t)stream);
}

amp4d_status amp4d_enqueue_partials(amp4d_model *model, int what, const double *params,
                                    double *out, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !params || !out || (what != AMP4D_EVAL_NLL && what != AMP4D_EVAL_NLL_GRAD))
        return model ? fail(model, AMP4D_ERR_ARG, "bad enqueue arguments") : AMP4D_ERR_ARG;
    CK(cudaSetDevice(model->device));
    return enqueue(model, what == AMP4D_EVAL_NLL_GRAD, params, out, (cudaStream_t)stream, true);
}

amp4d_status amp4d_eval_partials(amp4d_model *model, int what, const double *params, double *out,
                                 void *stream)
{
    if (!model || !params || !out || (what != AMP4D_EVAL_NLL && what != AMP4D_EVAL_NLL_GRAD))
        return model ? fail(model, AMP4D_ERR_ARG, "bad partials arguments") : AMP4D_ERR_ARG;
    const bool g = what == AMP4D_EVAL_NLL_GRAD;
    amp4d_status rc = run_eval(model, params, g, (cudaStream_t)stream, true);
    if (rc) return rc;
    std::memcpy(out, model->h_out, (6 + (g ? 2 * model->n_param : 0)) * sizeof(double));
    return AMP4D_OK;
}

amp4d_status amp4d_build_gram(amp4d_model *model, const double *params, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model) return AMP4D_ERR_ARG;
    amp4d_status rc = check_params(model, params);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(model->device));
    std::memcpy(model->h_params, params, model->n_param * sizeof(double));
    CK(cudaMemcpyAsync(model->d_params, model->h_params, model->n_param * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    return build_gram(model, st);
}

amp4d_status amp4d_fit_fractions(amp4d_model *model, const double *params, double *ff, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !params || !ff) return AMP4D_ERR_ARG;
    if (model->mc.n == 0) return fail(model, AMP4D_ERR_STATE, "set_norm_points must come first");
    cudaStream_t st = (cudaStream_t)stream;
    // Fit fractions are defined on S over phase space.  With an efficiency the
    // weight record holds w0 eps: the Gram for them is built over the weights as
    // loaded (w0), and the efficiency-weighted record is restored afterwards (the
    // evaluation Gram is then rebuilt on the next evaluation).
    const bool unweight = model->has_eff && model->mc.w0;
    float *wrec = model->mc.rec + (size_t)model->mc.wrec * model->mc.npad;
    const size_t wbytes = (size_t)model->mc.npad * sizeof(float);
    if (unweight) {
        CK(cudaMemcpyAsync(wrec, model->mc.w0, wbytes, cudaMemcpyDeviceToDevice, st));
        model->gram_valid = false;
    }
    // The Gram matrix at these masses and widths (fixed-mass models reuse it).
    amp4d_status rc0 = AMP4D_OK;
    if (model->n_float > 0 || !model->gram_valid) rc0 = amp4d_build_gram(model, params, stream);
    else rc0 = check_params(model, params);
    if (unweight) {
        const amp4d_status rc1 = apply_templates(model, model->mc, true, st);   // w0 eps again
        model->gram_valid = false;
        if (rc0 == AMP4D_OK) rc0 = rc1;
    }
    if (rc0) return rc0;
    const int K = model->n_col, dim = 2 * K;
    std::vector<double> G((size_t)dim * dim), kap(model->n_param);
    CK(cudaMemcpyAsync(G.data(), model->d_G, G.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(kap.data(), model->d_pscale, kap.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // q(c) = u^T G u + v^T G v with u = (Re c', -Im c'), v = (Im c', Re c') per column,
    // c'_k = kappa_k c_k the folded couplings (the Gram rows are the folded basis).
    auto q_of = [&](int only_res) {
        std::vector<double> u(dim, 0.0), v(dim, 0.0);
        for (int k = 0; k < K; ++k) {
            if (only_res >= 0 && model->col_res[k] != only_res) continue;
            const double re = kap[2 * k] * params[2 * k], im = kap[2 * k] * params[2 * k + 1];
            u[2 * k] = re; u[2 * k + 1] = -im;
            v[2 * k] = im; v[2 * k + 1] = re;
        }
        double q = 0.0;
        for (int i = 0; i < dim; ++i) {
            double gu = 0.0, gv = 0.0;
            for (int j = 0; j < dim; ++j) {
                gu += G[(size_t)i * dim + j] * u[j];
                gv += G[(size_t)i * dim + j] * v[j];
            }
            q += u[i] * gu + v[i] * gv;
        }
        return q;
    };
    const double qt = q_of(-1);
    if (!(qt > 0.0)) return fail(model, AMP4D_ERR_DOMAIN, "I <= 0");
    for (int r = 0; r < (int)model->res.size(); ++r) ff[r] = q_of(r) / qt;
    return AMP4D_OK;
}

amp4d_status amp4d_get_gram(amp4d_model *model, double *G, void *stream)
{
    if (!model || !G) return AMP4D_ERR_ARG;
    if (!model->gram_valid) return fail(model, AMP4D_ERR_STATE, "no Gram matrix built");
    cudaStream_t st = (cudaStream_t)stream;
    const int dim = 2 * model->n_col;
    std::vector<double> gp(dim * dim), ps(model->n_param);
    CK(cudaMemcpyAsync(gp.data(), model->d_G, dim * dim * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ps.data(), model->d_pscale, model->n_param * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) G[i * dim + j] = gp[i * dim + j] * ps[i] * ps[j];
    return AMP4D_OK;
}

amp4d_status amp4d_gram_selftest(const int32_t *X, int64_t n, long long *G_int, void *stream)
{
    amp4d_model *model = nullptr;
    if (!X || !G_int || n < 1) return fail(nullptr, AMP4D_ERR_ARG, "bad self-test arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t nchunks = (n + gram_chunk_points() - 1) / gram_chunk_points();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nsm, nchunks));
    int *d_X = nullptr, *d_err = nullptr;
    long long *d_part = nullptr, *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_X, (size_t)n * 128 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_part, (size_t)grid * 4096 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_out, 4096 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_X, X, (size_t)n * 128 * sizeof(int), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = launch_gram_selftest(d_X, n, d_part, grid, d_err, d_out, st);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(G_int, d_out, 4096 * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_X); cudaFree(d_part); cudaFree(d_out); cudaFree(d_err);
    if (e != cudaSuccess) return fail(nullptr, AMP4D_ERR_CUDA, std::string("gram self-test: ") + cudaGetErrorString(e));
    if (err) return fail(nullptr, AMP4D_ERR_TIMEOUT, "gram self-test: a bounded wait expired");
    return AMP4D_OK;
}

amp4d_status amp4d_generate(amp4d_model *model, const double *params, uint64_t seed, int64_t n,
                            float *m, float *cK, float *cpsi, float *phi, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !m || !cK || !cpsi || !phi || n < 1) return AMP4D_ERR_ARG;
    amp4d_status rc = check_params(model, params);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(model->device));
    std::memcpy(model->h_params, params, model->n_param * sizeof(double));
    CK(cudaMemcpyAsync(model->d_params, model->h_params, model->n_param * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CK(enqueue_table(model, model->d_params, st));
    // With Eq. 14 templates the events follow f = p q [P eps S / I_eps + (1 - P) hb / B]
    // (without a background, p q eps S): the accept-reject weight becomes
    // alpha eps S + beta hb, alpha = P / I_eps and beta = (1 - P) / B from the
    // normalisation points.
    const bool tpl = model->has_eff || model->has_bkg;
    const bool mix = mixing(model);
    double g_alpha = 1.0, g_beta = 0.0;
    if (mix) {
        if (model->mc.n == 0) return fail(model, AMP4D_ERR_STATE, "generate with a background needs normalisation points");
        if (!(model->mc.whb > 0.0)) return fail(model, AMP4D_ERR_DOMAIN, "the background template is 0 over the normalisation points");
        LaunchArgs ln = args_for(model, model->mc, model->mc.part, nullptr, st, model->mc.grid_eval);
        CK(launch_eval(ln, 1));
        unsigned long long a2[2];
        CK(cudaMemcpyAsync(a2, model->d_acc + 2 * model->nslot, sizeof a2, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const double T = (double)(long long)a2[0] + (double)a2[1] * 0x1p-64;
        const double von = model->mc.volume / (double)model->mc.n;
        const double Ie = von * T, Bn = von * model->mc.whb;
        if (!(Ie > 0.0)) return fail(model, AMP4D_ERR_DOMAIN, "generate: I_eps <= 0");
        g_alpha = model->purity / Ie;
        g_beta = (1.0 - model->purity) / Bn;
    }
    const int64_t B = 1 << 22, nscan = 1 << 20;
    const int nrec = model->nZ > 0 ? REC_NZ : REC_NK;
    const int nblk = (int)((B + gen_tile() - 1) / gen_tile());
    EventSet g;
    g.npad = B;
    g.nrec = nrec;
    float *S = nullptr, *ua = nullptr;
    unsigned *cnt = nullptr, *flag = nullptr;
    unsigned long long *off = nullptr;
    double *part = nullptr;
    auto cleanup = [&]() {
        for (void *ptr : {(void *)g.rec, (void *)S, (void *)ua, (void *)cnt, (void *)flag, (void *)off,
                          (void *)part, (void *)g.eps, (void *)g.hb})
            if (ptr) cudaFree(ptr);
        g.eps = g.hb = nullptr;
    };
#define CKG(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cleanup();                                                                     \
            return fail(model, e_ == cudaErrorMemoryAllocation ? AMP4D_ERR_OOM : AMP4D_ERR_CUDA, \
                        std::string("generate: ") + cudaGetErrorString(e_));              \
        }                                                                                  \
    } while (0)
    CKG(cudaMalloc(&g.rec, (size_t)nrec * B * sizeof(float)));
    CKG(cudaMalloc(&S, B * sizeof(float)));
    CKG(cudaMalloc(&ua, B * sizeof(float)));
    CKG(cudaMalloc(&cnt, nblk * sizeof(unsigned)));
    CKG(cudaMalloc(&flag, 2 * sizeof(unsigned)));
    CKG(cudaMalloc(&off, (nblk + 1) * sizeof(unsigned long long)));
    CKG(cudaMalloc(&part, (size_t)model->nsm * 8 * sizeof(double)));
    if (tpl) {
        CKG(cudaMalloc(&g.eps, B * sizeof(float)));
        CKG(cudaMalloc(&g.hb, B * sizeof(float)));
    }
    // Evaluate S p q at count candidates of the given Philox stream starting at first.
    auto eval_batch = [&](uint64_t first, int64_t count, uint32_t sid, float *uacc) -> cudaError_t {
        cudaError_t e = launch_gen_candidates(g.rec, B, count, first, sid, seed, model->m_lo,
                                              model->m_hi, uacc, st);
        if (e != cudaSuccess) return e;
        PrepArgs a{};
        a.rec = g.rec; a.npad = B; a.n = count; a.has_z = model->nZ > 0; a.wrec = -1; a.have_w = 0;
        a.mB = model->mass.mB; a.mpsi = model->mass.mpsi; a.mK = model->mass.mK; a.mpi = model->mass.mpi;
        a.m_lo = model->m_lo; a.m_hi = model->m_hi;
        a.grid = model->nsm * 8; a.part_lnpq = nullptr; a.bad = model->d_bad; a.stream = st;
        e = launch_prepare(a);
        if (e != cudaSuccess) return e;
        g.n = count;
        LaunchArgs la = args_for(model, g, part, S, st, model->nsm * 8);
        e = launch_eval(la, 2);
        if (e != cudaSuccess || !tpl) return e;
        TplArgs t{};
        t.rec = g.rec; t.npad = B; t.n = count; t.eps = g.eps; t.hb = g.hb;
        for (int i = 0; i < 4; ++i) t.t[i] = model->tpl[i];
        if (!model->has_eff) t.t[0].h = t.t[1].h = nullptr;
        if (!model->has_bkg) t.t[2].h = t.t[3].h = nullptr;
        t.mB = model->mass.mB; t.mpsi = model->mass.mpsi; t.mK = model->mass.mK; t.mpi = model->mass.mpi;
        t.part = part;
        t.grid = (int)std::min<int64_t>((count + prepare_block() - 1) / prepare_block(), model->nsm * 8);
        t.stream = st;
        e = launch_templates(t);
        if (e != cudaSuccess) return e;
        return launch_eq14_density(S, g.eps, mix ? g.hb : nullptr, count, g_alpha, g_beta, st);
    };
    // f_max: 1.5 x the largest S p q over the scan candidates (stream 2)
    CKG(cudaMemsetAsync(flag, 0, 2 * sizeof(unsigned), st));
    CKG(eval_batch(0, nscan, 2u, nullptr));
    CKG(launch_gen_accept(g.rec, B, nscan, S, nullptr, 0.0, cnt, flag, flag + 1, st));
    unsigned fbits = 0;
    CKG(cudaMemcpyAsync(&fbits, flag + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CKG(cudaStreamSynchronize(st));
    float fm32;
    std::memcpy(&fm32, &fbits, sizeof fm32);
    double fmax = 1.5 * (double)fm32;
    if (!(fmax > 0.0)) { cleanup(); return fail(model, AMP4D_ERR_DOMAIN, "generate: S p q vanishes"); }
    int64_t got = 0;
    uint64_t first = 0;
    int restarts = 0;
    while (got < n) {
        if (first > (uint64_t)(4000 * n + (1 << 24))) { cleanup(); return fail(model, AMP4D_ERR_DOMAIN, "generate: candidate budget exhausted"); }
        CKG(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
        CKG(eval_batch(first, B, 0u, ua));
        CKG(launch_gen_accept(g.rec, B, B, S, ua, fmax, cnt, flag, nullptr, st));
        unsigned over = 0;
        CKG(cudaMemcpyAsync(&over, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CKG(cudaStreamSynchronize(st));
        if (over) {
            fmax *= 2.0;
            got = 0;
            first = 0;
            if (++restarts > 20) { cleanup(); return fail(model, AMP4D_ERR_DOMAIN, "generate: f_max did not settle"); }
            continue;
        }
        CKG(launch_gen_scatter(g.rec, B, B, S, ua, fmax, cnt, off, got, n, m, cK, cpsi, phi, st));
        unsigned long long tot = 0;
        CKG(cudaMemcpyAsync(&tot, off + nblk, sizeof(tot), cudaMemcpyDeviceToHost, st));
        CKG(cudaStreamSynchronize(st));
        got += (int64_t)tot;
        first += B;
    }
#undef CKG
    cleanup();
    return AMP4D_OK;
}

amp4d_status amp4d_proposal_train(amp4d_model *model, const float *m, const float *cK,
                                  const float *cpsi, const float *phi, int64_t n,
                                  const amp4d_mlp_cfg *cfg, uint64_t seed, double *loss, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !m || !cK || !cpsi || !phi || !cfg || n < 1 || cfg->batch < 1 || cfg->steps < 1)
        return AMP4D_ERR_ARG;
    for (int d = 0; d < 4; ++d)
        if (cfg->nb[d] < 1) return fail(model, AMP4D_ERR_ARG, "grid cells must be >= 1");
    if (!(cfg->alpha > 0.0 && cfg->alpha <= 1.0)) return fail(model, AMP4D_ERR_ARG, "alpha in (0, 1]");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(model->device));
    const int P = mlp_num_params();
    if (!model->d_th) {
        CK(cudaMalloc(&model->d_th, P * sizeof(float)));
        CK(cudaMalloc(&model->d_am, P * sizeof(float)));
        CK(cudaMalloc(&model->d_av, P * sizeof(float)));
        CK(cudaMalloc(&model->d_wb, P * sizeof(__nv_bfloat16)));
    }
    std::vector<float> th(P);
    mlp_init_params(th.data(), seed);
    CK(cudaMemcpyAsync(model->d_th, th.data(), P * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(model->d_am, 0, P * sizeof(float), st));
    CK(cudaMemsetAsync(model->d_av, 0, P * sizeof(float), st));
    CK(launch_to_bf16(model->d_th, model->d_wb, st));
    const int64_t nd = cfg->batch, nu = cfg->batch;
    float *xd = nullptr, *xu = nullptr, *part = nullptr;
    double *gout = nullptr;
    auto cleanup = [&]() {
        for (void *ptr : {(void *)xd, (void *)xu, (void *)part, (void *)gout})
            if (ptr) cudaFree(ptr);
    };
    cudaError_t e = cudaMalloc(&xd, nd * 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&xu, nu * 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)mlp_grad_blocks(nd, nu) * (P + 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&gout, (P + 1) * sizeof(double));
    for (int64_t t = 1; e == cudaSuccess && t <= cfg->steps; ++t) {
        e = launch_mlp_batch(m, cK, cpsi, phi, n, nd, nu, seed, (uint64_t)t, model->m_lo, model->m_hi,
                             xd, xu, st);
        if (e == cudaSuccess) e = launch_mlp_grad(model->d_wb, xd, nd, xu, nu, part, gout, st);
        if (e == cudaSuccess)
            e = launch_adam(model->d_th, model->d_am, model->d_av, gout, (float)cfg->lr, 0.9f, 0.999f,
                            1e-8f, t, model->d_wb, st);
    }
    double L = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&L, gout + P, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return fail(model, AMP4D_ERR_CUDA, std::string("proposal_train: ") + cudaGetErrorString(e));
    if (loss) *loss = L;
    // Grid of cell-centre values and the FP64 CDF of the defensive mixture.
    const int64_t nc = (int64_t)cfg->nb[0] * cfg->nb[1] * cfg->nb[2] * cfg->nb[3];
    if (model->d_gcell) { cudaFree(model->d_gcell); model->d_gcell = nullptr; }
    if (model->d_cdf) { cudaFree(model->d_cdf); model->d_cdf = nullptr; }
    CK(cudaMalloc(&model->d_gcell, nc * sizeof(float)));
    CK(cudaMalloc(&model->d_cdf, nc * sizeof(double)));
    {
        amp4d_status rc = ensure_tmp(model, 2 * cdf_scratch(nc) + 2);
        if (rc) return rc;
    }
    for (int d = 0; d < 4; ++d) model->nb[d] = cfg->nb[d];
    CK(launch_mlp_grid(model->d_wb, model->nb, model->d_gcell, st));
    CK(launch_grid_cdf(model->d_gcell, nc, cfg->alpha, model->d_tmp, model->d_cdf, st));
    CK(cudaStreamSynchronize(st));
    model->proposal_ready = true;
    return AMP4D_OK;
}

amp4d_status amp4d_proposal_train_gram(amp4d_model *model, const double *params, int64_t n,
                                       const amp4d_mlp_cfg *cfg, uint64_t seed, uint64_t gen_seed,
                                       double *loss, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !params || !cfg || n < 1) return AMP4D_ERR_ARG;
    if (model->mc.n == 0) return fail(model, AMP4D_ERR_STATE, "set_norm_points must come first");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(model->device));
    // The Gram diagonal over the current points at these masses and widths:
    // G_kk = int |B_k|^2 p q (times the points' weights), the normalisation of
    // column k with a unit coupling.
    amp4d_status rc = amp4d_build_gram(model, params, stream);
    if (rc) return rc;
    const int K = model->n_col, dim = 2 * K, P = model->n_param;
    std::vector<double> G((size_t)dim * dim);
    rc = amp4d_get_gram(model, G.data(), stream);
    if (rc) return rc;
    std::vector<double> gd(K);
    double gsum = 0.0;
    for (int k = 0; k < K; ++k) {
        gd[k] = G[(size_t)(2 * k) * dim + 2 * k] + G[(size_t)(2 * k + 1) * dim + 2 * k + 1];
        if (!(gd[k] >= 0.0)) return fail(model, AMP4D_ERR_DOMAIN, "proposal_train_gram: a Gram diagonal element is not >= 0");
        gsum += gd[k];
    }
    if (!(gsum > 0.0)) return fail(model, AMP4D_ERR_DOMAIN, "proposal_train_gram: the Gram diagonal is 0");
    // Column k contributes max(1, round(n G_kk / sum G)) events of the model with
    // the single unit coupling c_k = 1 (density |B_k|^2 p q), drawn by the
    // generator with seed gen_seed + k: together a draw from sum_k |B_k|^2 p q.
    std::vector<int64_t> nk(K), off(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        nk[k] = std::max<int64_t>(1, (int64_t)std::llround((double)n * gd[k] / gsum));
        off[k + 1] = off[k] + nk[k];
    }
    const int64_t tot = off[K];
    float *ev = nullptr;
    CK(cudaMalloc(&ev, (size_t)4 * tot * sizeof(float)));
    std::vector<double> pk(params, params + P);
    for (int k = 0; k < K && rc == AMP4D_OK; ++k) {
        std::fill(pk.begin(), pk.begin() + 2 * K, 0.0);
        pk[2 * k] = 1.0;
        rc = amp4d_generate(model, pk.data(), gen_seed + (uint64_t)k, nk[k], ev + off[k],
                            ev + tot + off[k], ev + 2 * tot + off[k], ev + 3 * tot + off[k], stream);
    }
    if (rc == AMP4D_OK)
        rc = amp4d_proposal_train(model, ev, ev + tot, ev + 2 * tot, ev + 3 * tot, tot, cfg, seed, loss,
                                  stream);
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(ev);
    if (rc == AMP4D_OK && e != cudaSuccess) return fail(model, AMP4D_ERR_CUDA, cudaGetErrorString(e));
    return rc;
}

amp4d_status amp4d_proposal_sample(amp4d_model *model, int64_t n, uint64_t seed, float *m, float *cK,
                                   float *cpsi, float *phi, float *w, void *stream)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model || !m || !cK || !cpsi || !phi || !w || n < 1) return AMP4D_ERR_ARG;
    if (!model->proposal_ready) return fail(model, AMP4D_ERR_STATE, "proposal not trained");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(model->device));
    CK(launch_grid_sample(model->d_cdf, model->nb, seed, n, model->m_lo, model->m_hi, model->mass.mB,
                          model->mass.mpsi, model->mass.mK, model->mass.mpi, m, cK, cpsi, phi, w,
                          nullptr, st));
    CK(cudaStreamSynchronize(st));
    return AMP4D_OK;
}

amp4d_status amp4d_mlp_forward(const float *theta, const float *x, int64_t n, float *g, void *stream)
{
    amp4d_model *model = nullptr;
    if (!theta || !x || !g || n < 1) return fail(nullptr, AMP4D_ERR_ARG, "bad mlp_forward arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int P = mlp_num_params();
    float *th = nullptr;
    __nv_bfloat16 *wb = nullptr;
    CK(cudaMalloc(&th, P * sizeof(float)));
    cudaError_t e = cudaMalloc(&wb, P * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemcpyAsync(th, theta, P * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = launch_to_bf16(th, wb, st);
    if (e == cudaSuccess) e = launch_mlp_forward(wb, x, n, g, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(th);
    if (wb) cudaFree(wb);
    if (e != cudaSuccess) return fail(nullptr, AMP4D_ERR_CUDA, std::string("mlp_forward: ") + cudaGetErrorString(e));
    return AMP4D_OK;
}

amp4d_status amp4d_mlp_loss_grad(const float *theta, const float *xd, int64_t nd, const float *xu,
                                 int64_t nu, double *out, void *stream)
{
    amp4d_model *model = nullptr;
    if (!theta || !xd || !xu || !out || nd < 1 || nu < 1) return fail(nullptr, AMP4D_ERR_ARG, "bad mlp_loss_grad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int P = mlp_num_params();
    float *th = nullptr, *part = nullptr;
    __nv_bfloat16 *wb = nullptr;
    double *go = nullptr;
    CK(cudaMalloc(&th, P * sizeof(float)));
    cudaError_t e = cudaMalloc(&wb, P * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)mlp_grad_blocks(nd, nu) * (P + 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&go, (P + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(th, theta, P * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = launch_to_bf16(th, wb, st);
    if (e == cudaSuccess) e = launch_mlp_grad(wb, xd, nd, xu, nu, part, go, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, go, (P + 1) * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void *ptr : {(void *)th, (void *)wb, (void *)part, (void *)go})
        if (ptr) cudaFree(ptr);
    if (e != cudaSuccess) return fail(nullptr, AMP4D_ERR_CUDA, std::string("mlp_loss_grad: ") + cudaGetErrorString(e));
    return AMP4D_OK;
}

amp4d_status amp4d_grid_sample(const float *gcell, const int *nb, double alpha, uint64_t seed,
                               int64_t n, double m_lo, double m_hi, const amp4d_particle_masses *masses,
                               float *m, float *cK, float *cpsi, float *phi, float *w, int64_t *cell,
                               void *stream)
{
    amp4d_model *model = nullptr;
    if (!gcell || !nb || !masses || !m || !cK || !cpsi || !phi || !w || n < 1 || !(alpha > 0.0 && alpha <= 1.0))
        return fail(nullptr, AMP4D_ERR_ARG, "bad grid_sample arguments");
    for (int d = 0; d < 4; ++d)
        if (nb[d] < 1) return fail(nullptr, AMP4D_ERR_ARG, "grid cells must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nc = (int64_t)nb[0] * nb[1] * nb[2] * nb[3];
    float *gc = nullptr;
    double *cdf = nullptr, *scr = nullptr;
    CK(cudaMalloc(&gc, nc * sizeof(float)));
    cudaError_t e = cudaMalloc(&cdf, nc * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&scr, (2 * cdf_scratch(nc) + 2) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(gc, gcell, nc * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = launch_grid_cdf(gc, nc, alpha, scr, cdf, st);
    if (e == cudaSuccess)
        e = launch_grid_sample(cdf, nb, seed, n, m_lo, m_hi, masses->mB, masses->mpsi, masses->mK,
                               masses->mpi, m, cK, cpsi, phi, w, cell, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void *ptr : {(void *)gc, (void *)cdf, (void *)scr})
        if (ptr) cudaFree(ptr);
    if (e != cudaSuccess) return fail(nullptr, AMP4D_ERR_CUDA, std::string("grid_sample: ") + cudaGetErrorString(e));
    return AMP4D_OK;
}

amp4d_status amp4d_profile_enable(amp4d_model *model, int on)
{
    if (model) ++model->state_gen;   // may change what an evaluation enqueues
    if (!model) return AMP4D_ERR_ARG;
    model->prof_on = on != 0;
    return AMP4D_OK;
}

amp4d_status amp4d_profile_read(amp4d_model *model, double *ms, int64_t *count)
{
    if (!model || !ms || !count) return AMP4D_ERR_ARG;
    for (auto &v : model->prof_pending) {
        CK(cudaEventSynchronize(v.back()));
        for (size_t i = 0; i + 1 < v.size() && i < 4; ++i) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, v[i], v[i + 1]));
            model->prof_ms[i] += t;
            model->prof_n[i] += 1;
        }
        for (cudaEvent_t e : v) model->ev_pool.push_back(e);
    }
    model->prof_pending.clear();
    for (int i = 0; i < 4; ++i) {
        ms[i] = model->prof_ms[i];
        count[i] = model->prof_n[i];
        model->prof_ms[i] = 0.0;
        model->prof_n[i] = 0;
    }
    return AMP4D_OK;
}

}  // extern "C"
