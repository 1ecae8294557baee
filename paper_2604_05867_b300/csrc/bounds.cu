// Bound post-processing on the host (Sec. 6): turning certified upper bounds
// on exact-channel capacities C_{n,k} (or on C_n(d)) into upper bounds on the
// capacity C(d) of the binary deletion channel.  No kernels: these are a few
// hundred floating-point operations per bound.
//
// Every sum is formed in long double from non-negative terms and the result
// is rounded up to the next double, so that exact inputs give a valid upper
// bound (the weights C(n,k) d^(n-k) (1-d)^k are products of non-negative
// factors; the rounding of each product and addition in long double is far
// below the double ulp that is added at the end).
#include "bdc_internal.cuh"

#include <cmath>

namespace {

long double binom_ld(int n, int k) {
    if (k < 0 || k > n || n < 0) return 0.0L;
    long double r = 1.0L;
    for (int i = 1; i <= k; i++) r = r * (long double)(n - k + i) / (long double)i;
    return floorl(r + 0.5L);
}

double round_up(long double v) {
    double r = (double)v;
    if ((long double)r < v) r = std::nextafter(r, INFINITY);
    return r;
}

}  // namespace

// Lemma prob-vs-exact (Sec. 2.2): C_n(d) <= sum_{k=1}^n C(n,k) d^(n-k) (1-d)^k C_{n,k}.
extern "C" bdc_status bdc_bound_prob_vs_exact(int n, double d, const double *Cnk, double *Cn_d) {
    if (n < 1 || n > 64 || !Cnk || !Cn_d || !(d >= 0.0 && d <= 1.0)) {
        bdc_set_error("bdc_bound_prob_vs_exact: need 1 <= n <= 64, 0 <= d <= 1, non-NULL arrays");
        return BDC_EINVAL;
    }
    long double s = 0.0L, dl = d, dm = 1.0L - (long double)d;
    for (int k = 1; k <= n; k++) {
        if (!(Cnk[k] >= 0.0) || !std::isfinite(Cnk[k])) {
            bdc_set_error("bdc_bound_prob_vs_exact: every C_{n,k} bound must be finite and non-negative");
            return BDC_EINVAL;
        }
        long double w = binom_ld(n, k) * powl(dl, (long double)(n - k)) * powl(dm, (long double)k);
        s += w * (long double)Cnk[k];
    }
    *Cn_d = round_up(s);
    return BDC_OK;
}

// Lemma worse-UB (Sec. 6): splitting the n input symbols into the first s
// and the other n - s,
//   C_{n,k} <= sum_{i=0}^{s} [C(s,i) C(n-s,k-i) / C(n,k)] (C_{s,i} + C_{n-s,k-i}).
extern "C" bdc_status bdc_bound_split(int n, int k, int s, const double *Cs, const double *Cns, double *Cnk) {
    if (n < 2 || n > 64 || k < 0 || k > n || s < 1 || s >= n || !Cs || !Cns || !Cnk) {
        bdc_set_error("bdc_bound_split: need 2 <= n <= 64, 0 <= k <= n, 1 <= s < n, non-NULL arrays");
        return BDC_EINVAL;
    }
    const long double ck = binom_ld(n, k);
    long double acc = 0.0L;
    for (int i = 0; i <= s; i++) {
        const int j = k - i;
        if (j < 0 || j > n - s) continue;  // no way to keep i of the first s and j of the rest
        const long double w = binom_ld(s, i) * binom_ld(n - s, j) / ck;
        if (!(Cs[i] >= 0.0) || !(Cns[j] >= 0.0) || !std::isfinite(Cs[i]) || !std::isfinite(Cns[j])) {
            bdc_set_error("bdc_bound_split: the bounds used must be finite and non-negative");
            return BDC_EINVAL;
        }
        acc += w * ((long double)Cs[i] + (long double)Cns[j]);
    }
    *Cnk = round_up(acc);
    return BDC_OK;
}

// Lemma convex (Sec. 6, Rahmati and Duman): for d = lambda d' + 1 - lambda
// with lambda in [0, 1], i.e. every d in [d', 1],
//   C(d) / (1 - d) <= C(d') / (1 - d').
// Given an upper bound C_dp on C(d'), writes the bound on C(d) and on the
// ratio C(d') / (1 - d') itself.
extern "C" bdc_status bdc_bound_high_noise(double d_prime, double C_dp, double d, double *Cd, double *ratio) {
    if (!(d_prime >= 0.0 && d_prime < 1.0) || !(d >= d_prime && d <= 1.0) || !(C_dp >= 0.0) || !std::isfinite(C_dp)) {
        bdc_set_error("bdc_bound_high_noise: need 0 <= d' < 1, d' <= d <= 1 and a finite C(d') >= 0");
        return BDC_EINVAL;
    }
    const long double r = (long double)C_dp / (1.0L - (long double)d_prime);
    if (ratio) *ratio = round_up(r);
    if (Cd) *Cd = round_up(r * (1.0L - (long double)d));
    return BDC_OK;
}
