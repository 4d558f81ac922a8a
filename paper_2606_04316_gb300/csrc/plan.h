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

// Ket list of one row batch when a class runs in row batches with bra-ket
// symmetry (bra positions [b0, b1) in this batch; shell pairs 0..n-1):
//   order[q]   shell pair at global ket position q (w descending)
//   kpos[i]    global ket position of pair i (the inverse of order)
//   prefix[i]  kept ket prefix of pair i: row i keeps the positions q < prefix[i]
//   bpos[i]    bra position of pair i
//   batch      the batch's pairs
// A kept block (AB|CD) whose mirror (CD|AB) is kept too (kpos(AB) < prefix(CD))
// and whose ket pair CD lies in an earlier batch came, transposed, from CD's
// batch, so such a CD needs no column here -- unless some row of this batch
// keeps CD one way only (kpos(AB) >= prefix(CD)), whose block must be computed
// here.  The list holds the pairs of this and later batches and those earlier
// pairs, in global ket order; the kernel skips the rows of an earlier pair kept
// both ways.  Outputs: list (shell pairs), pos[i] (index in list or -1), and
// cnt[q] (list entries among the global positions < q, q = 0..n): row AB's
// kept entries are the first cnt[prefix[AB]] of the list.
struct BatchKets {
    std::vector<int> list, pos, cnt;
};

inline BatchKets batch_kets(const std::vector<int> &order, const std::vector<int> &kpos,
                            const std::vector<int> &prefix, const std::vector<int> &bpos, int b0,
                            const std::vector<int> &batch) {
    const int n = (int)order.size();
    // the batch's rows by ket position, and the largest prefix among the rows at
    // or after each one
    std::vector<int> rows(batch);
    std::sort(rows.begin(), rows.end(), [&](int x, int y) { return kpos[x] < kpos[y]; });
    std::vector<int> kk(rows.size()), smax(rows.size() + 1, -1);
    for (size_t i = 0; i < rows.size(); ++i) kk[i] = kpos[rows[i]];
    for (int i = (int)rows.size() - 1; i >= 0; --i) smax[i] = std::max(smax[i + 1], prefix[rows[i]]);
    BatchKets b;
    b.pos.assign(n, -1);
    b.cnt.assign(n + 1, 0);
    for (int q = 0; q < n; ++q) {
        const int sp = order[q];
        bool keep = bpos[sp] >= b0;
        if (!keep) {
            // rows AB with kpos(AB) >= prefix(CD) are not kept by CD; does one of them keep CD?
            const size_t i = (size_t)(std::lower_bound(kk.begin(), kk.end(), prefix[sp]) - kk.begin());
            keep = smax[i] > q;
        }
        if (keep) {
            b.pos[sp] = (int)b.list.size();
            b.list.push_back(sp);
        }
        b.cnt[q + 1] = (int)b.list.size();
    }
    return b;
}

}  // namespace qdt
