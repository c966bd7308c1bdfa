// Recombination of shard partials (host code only).
//
// The unbinned likelihood (Introduction) is a product over data events of the
// PDF S p q / I (Eq. 5), and I is an integral estimated as a sum over
// points, so a fit whose events and points are split into shards needs, per
// evaluation, only the sums each shard produces (amp4d_eval_partials):
//   ln L terms  l_r = sum ln S,  sum ln(p q),  N_r,
//   T_r = V sum_n w_n S_n,  M_r points,
// and their parameter derivatives.  Over the union of the shards
//   I = (sum_r T_r) / (sum_r M_r),
//   NLL = -2 [ sum_r l_r + sum_r ln(pq)_r - N ln I ],
//   dNLL/dtheta = -2 [ sum_r dl_r - N (sum_r dT_r) / (sum_r T_r) ].
// Shards are summed in the order given, with Neumaier compensation, so every
// rank that combines the same gathered partials gets the same bits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/amp4d.h"

namespace {

struct Neumaier {
    double s = 0.0, c = 0.0;
    void add(double x)
    {
        const double t = s + x;
        c += (std::fabs(s) >= std::fabs(x)) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

thread_local const char *g_shard_error = "";

}  // namespace

extern "C" amp4d_status amp4d_combine_partials(const double *parts, int n_shards, int n_param,
                                               int what, double *out)
{
    if (!parts || !out || n_shards < 1 || n_param < 0 ||
        (what != AMP4D_EVAL_NLL && what != AMP4D_EVAL_NLL_GRAD)) {
        g_shard_error = "combine_partials: null pointer, n_shards < 1, n_param < 0 or bad what";
        return AMP4D_ERR_ARG;
    }
    const bool g = what == AMP4D_EVAL_NLL_GRAD;
    const int64_t stride = 6 + (g ? 2 * (int64_t)n_param : 0);
    Neumaier l, lnpq, N, T, M;
    std::vector<Neumaier> dl(g ? n_param : 0), dT(g ? n_param : 0);
    unsigned st = 0;
    for (int r = 0; r < n_shards; ++r) {
        const double *p = parts + r * stride;
        if (!(p[2] >= 0.0) || !(p[4] >= 0.0) || !(p[5] >= 0.0)) {
            g_shard_error = "combine_partials: a shard has a negative or NaN count or status";
            return AMP4D_ERR_ARG;
        }
        l.add(p[0]);
        lnpq.add(p[1]);
        N.add(p[2]);
        T.add(p[3]);
        M.add(p[4]);
        st |= (unsigned)p[5];
        for (int k = 0; k < (g ? n_param : 0); ++k) {
            dl[k].add(p[6 + k]);
            dT[k].add(p[6 + n_param + k]);
        }
    }
    const double Mv = M.value(), Tv = T.value(), Nv = N.value();
    if (!(Mv > 0.0)) {
        g_shard_error = "combine_partials: no normalisation points in any shard";
        return AMP4D_ERR_STATE;
    }
    const double I = Tv / Mv;
    const double nll = -2.0 * (l.value() + lnpq.value() - Nv * std::log(I));
    if (!(I > 0.0) || !std::isfinite(nll)) st |= 1u;
    out[0] = st ? INFINITY : nll;
    out[1] = l.value();
    out[2] = lnpq.value();
    out[3] = I;
    out[4] = Nv;
    out[5] = (double)st;
    for (int k = 0; k < (g ? n_param : 0); ++k)
        out[6 + k] = st ? 0.0 : -2.0 * (dl[k].value() - Nv * dT[k].value() / Tv);
    if (st & 2u) {
        g_shard_error = "combine_partials: a shard reported invalid parameters";
        return AMP4D_ERR_ARG;
    }
    if (st & 1u) {
        g_shard_error = "combine_partials: S <= 0 at a data event, p q = 0, or I <= 0";
        return AMP4D_ERR_DOMAIN;
    }
    return AMP4D_OK;
}

extern "C" const char *amp4d_shard_last_error(void) { return g_shard_error; }
