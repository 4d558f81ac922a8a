// plan.h -- host-side planning of the split form's plain-FP32 integrals.
// Pure C++ (no CUDA), shared by the library and its CPU tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace qdt {

// Per class: which kept quartets may have their integrals in plain FP32.
//   w[i]      = Q_i Dmax_i of shell pair i (Schwarz factor times density maximum)
//   nfp[i]    = function pairs of shell pair i
//   order[q]  = shell pair at sorted ket position q (w descending)
//   prefix[i] = kept ket positions of bra row i (a prefix of the sorted order)
// The FP32 set is {(i, order[q]) : q < prefix[i], w_i w_order[q] <= t}: a suffix
// split[i] .. prefix[i] of every row, and the same decision for (j, i) as for
// (i, j).  t is the largest threshold (to 1 %) whose bound
//     scale * sum (w_i nfp_i) (w_j nfp_j)
// over the FP32 set stays within budget; budget <= 0 gives no FP32 quartets.
// Returns t (or -1 when none); *bound receives the bound of the chosen set.
inline double f32_tail_split(const std::vector<double> &w, const std::vector<int> &nfp, const std::vector<int> &order,
                             const std::vector<int> &prefix, double scale, double budget, std::vector<int> &split,
                             double *bound) {
    const int n = (int)w.size();
    split = prefix;
    *bound = 0.0;
    if (budget <= 0.0 || n == 0) return -1.0;
    // sorted w and suffix sums of w nfp, accumulated from the smallest products up so
    // that the FP32 tails (the small products) are summed without cancellation
    std::vector<double> ws(n), S(n + 1, 0.0);
    for (int q = 0; q < n; ++q) ws[q] = w[order[q]];
    for (int q = n - 1; q >= 0; --q) S[q] = S[q + 1] + ws[q] * (double)nfp[order[q]];
    // first kept position of row a whose product with w_a is <= t
    auto start = [&](int a, double t) {
        int lo = 0, hi = prefix[a];
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (w[a] * ws[mid] <= t) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    auto total = [&](double t) {
        double b = 0.0;
        for (int a = 0; a < n; ++a) {
            const int s0 = start(a, t), e = prefix[a];
            if (s0 < e) b += w[a] * (double)nfp[a] * (S[s0] - S[e]);
        }
        return scale * b;
    };
    double lo = 0.0, hi = 0.0;                             // total(lo) within budget, search up to w_max^2
    for (int i = 0; i < n; ++i) hi = std::max(hi, w[i]);
    hi = hi * hi;
    if (total(hi) <= budget) {
        lo = hi;
    } else {
        // bisection on the exponent scale, to 1 % in t (each step is one pass over the
        // rows, host time inside the transform)
        for (int it = 0; it < 60; ++it) {
            const double mid = lo > 0.0 ? std::sqrt(lo) * std::sqrt(hi) : hi * 1e-30;
            if (mid <= lo || mid >= hi) break;
            if (total(mid) <= budget) lo = mid; else hi = mid;
            if (lo > 0.0 && hi <= lo * 1.01) break;
        }
    }
    for (int a = 0; a < n; ++a) split[a] = start(a, lo);
    *bound = total(lo);
    return lo;
}

}  // namespace qdt
