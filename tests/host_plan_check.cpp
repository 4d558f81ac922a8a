// CPU check of the host planning (plan.h) on seeded random classes.  The split
// form's FP32 set: a per-row suffix of the kept kets, the same decision for
// (i, j) and (j, i), the reported bound is the brute-force sum and stays within
// the budget, and a 2 % larger threshold would exceed it.  The ket lists of row
// batches with bra-ket symmetry: every kept block reaches its row exactly once.
#include <cstdio>
#include <random>

#include "plan.h"

int main() {
    int fails = 0;
    for (int seed = 1; seed <= 40; ++seed) {
        std::mt19937_64 rng(seed);
        const int n = 50 + (int)(rng() % 400);
        std::uniform_real_distribution<double> lg(-14.0, 0.0);
        std::vector<double> w(n);
        std::vector<int> nfp(n), order(n), prefix(n), pos(n);
        for (int i = 0; i < n; ++i) {
            w[i] = (rng() % 17 == 0) ? 0.0 : std::pow(10.0, lg(rng));
            nfp[i] = 1 + (int)(rng() % 36);
            order[i] = i;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
        for (int q = 0; q < n; ++q) pos[order[q]] = q;
        for (int i = 0; i < n; ++i) prefix[i] = (int)(rng() % (n + 1));
        const double scale = 18.0 * 1024.0 / 16777216.0;
        const double budget = std::pow(10.0, -10.0 - (double)(rng() % 8));
        std::vector<int> split;
        double bound = 0.0;
        const double t = qdt::f32_tail_split(w, nfp, order, prefix, scale, budget, split, &bound);
        double brute = 0.0, brute_up = 0.0, wmax = 0.0;
        for (int i = 0; i < n; ++i) wmax = std::max(wmax, w[i]);
        for (int i = 0; i < n; ++i) {
            if (split[i] < 0 || split[i] > prefix[i]) { std::printf("seed %d: split out of range\n", seed); ++fails; }
            for (int q = 0; q < prefix[i]; ++q) {
                const int j = order[q];
                const bool f32 = q >= split[i];
                if (f32 != (w[i] * w[j] <= t)) { std::printf("seed %d: not a suffix\n", seed); ++fails; break; }
                if (q < prefix[i] && pos[i] < prefix[j] && f32 != (pos[i] >= split[j])) {
                    std::printf("seed %d: (i, j) and (j, i) differ\n", seed);
                    ++fails;
                    break;
                }
                const double c = scale * w[i] * nfp[i] * w[j] * nfp[j];
                if (f32) brute += c;
                if (w[i] * w[j] <= t * 1.02) brute_up += c;
            }
        }
        if (std::fabs(brute - bound) > 1e-9 * std::max(bound, 1e-300)) {
            std::printf("seed %d: bound %.6e, brute force %.6e\n", seed, bound, brute);
            ++fails;
        }
        if (bound > budget) { std::printf("seed %d: bound %.3e over budget %.3e\n", seed, bound, budget); ++fails; }
        if (t < wmax * wmax && brute_up <= budget) {
            std::printf("seed %d: a 2 %% larger threshold still fits (%.3e <= %.3e)\n", seed, brute_up, budget);
            ++fails;
        }
        // no budget, no FP32 quartets
        std::vector<int> s0;
        double b0 = 1.0;
        qdt::f32_tail_split(w, nfp, order, prefix, scale, 0.0, s0, &b0);
        if (s0 != prefix || b0 != 0.0) { std::printf("seed %d: zero budget\n", seed); ++fails; }
    }
    // row batches with bra-ket symmetry (batch_kets): on seeded random classes
    // split into batches, every kept ordered pair (AB, CD) reaches row AB exactly
    // once -- computed by AB's task, written transposed by CD's task in the same
    // batch (the lower pair id computes a block kept both ways), or written into
    // W2 by CD's task in CD's (earlier) batch -- under the integral kernel's rules.
    long long one_way_earlier = 0, dropped_earlier = 0;      // the cases the list must handle
    for (int seed = 101; seed <= 160; ++seed) {
        std::mt19937_64 rng(seed);
        const int n = 20 + (int)(rng() % 200);
        std::uniform_real_distribution<double> lg(-8.0, 0.0);
        std::vector<double> Q(n), Dm(n), w(n);
        for (int i = 0; i < n; ++i) {
            Q[i] = std::pow(10.0, lg(rng));
            Dm[i] = (rng() % 13 == 0) ? 0.0 : std::pow(10.0, lg(rng));
            w[i] = Q[i] * Dm[i];
        }
        const double tau = std::pow(10.0, -6.0 - (double)(rng() % 8));
        std::vector<int> order(n), kpos(n), prefix(n), bord(n), bpos(n);
        for (int i = 0; i < n; ++i) order[i] = bord[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
        std::stable_sort(bord.begin(), bord.end(), [&](int a, int b) { return Q[a] > Q[b]; });
        for (int q = 0; q < n; ++q) { kpos[order[q]] = q; bpos[bord[q]] = q; }
        for (int i = 0; i < n; ++i) {
            int p = 0;
            while (p < n && Q[i] * w[order[p]] >= tau) ++p;
            prefix[i] = p;
        }
        // contiguous batches of the bra order
        std::vector<int> cuts{0};
        while (cuts.back() < n) cuts.push_back(std::min(n, cuts.back() + 1 + (int)(rng() % 40)));
        std::vector<int> batch_of(n);
        for (size_t bi = 0; bi + 1 < cuts.size(); ++bi)
            for (int k = cuts[bi]; k < cuts[bi + 1]; ++k) batch_of[bord[k]] = (int)bi;
        std::vector<std::vector<int>> got(n, std::vector<int>(n, 0));
        auto kept = [&](int a, int c) { return kpos[c] < prefix[a]; };      // row a keeps ket c
        for (size_t bi = 0; bi + 1 < cuts.size(); ++bi) {
            const int b0 = cuts[bi], b1 = cuts[bi + 1];
            std::vector<int> batch(bord.begin() + b0, bord.begin() + b1);
            const qdt::BatchKets bk = qdt::batch_kets(order, kpos, prefix, bpos, b0, batch);
            for (int ab : batch)
                for (int c = 0; c < n; ++c)
                    if (bpos[c] < b0 && kept(ab, c)) {
                        if (!kept(c, ab)) ++one_way_earlier;
                        else if (bk.pos[c] < 0) ++dropped_earlier;
                    }
            for (int ab : batch) {
                // the task of row ab walks the first cnt[prefix[ab]] list entries
                for (int p = 0; p < bk.cnt[prefix[ab]]; ++p) {
                    const int cd = bk.list[p];
                    if (!kept(ab, cd)) { std::printf("seed %d: list entry not kept by its row\n", seed); ++fails; }
                    const bool both = cd != ab && kept(cd, ab);
                    bool rev = both, mir = false;
                    if (both) {
                        if (bpos[cd] < b0) continue;
                        rev = bpos[cd] < b1;
                        mir = !rev;
                    }
                    if (rev && cd < ab) continue;
                    ++got[ab][cd];                    // (ab|cd) into row ab
                    if (rev || mir) ++got[cd][ab];    // its transpose into row cd (W, or W2 of a later batch)
                    if (rev && bk.pos[ab] < 0) { std::printf("seed %d: rev column missing\n", seed); ++fails; }
                }
            }
        }
        for (int a = 0; a < n && fails < 20; ++a)
            for (int c = 0; c < n; ++c) {
                const int want = kept(a, c) ? 1 : 0;
                if (got[a][c] != want) {
                    std::printf("seed %d: pair (%d, %d) reaches its row %d times, want %d\n", seed, a, c, got[a][c], want);
                    ++fails;
                    break;
                }
            }
    }
    if (one_way_earlier == 0 || dropped_earlier == 0) {
        std::printf("batch lists: no one-way (%lld) or dropped (%lld) earlier kets in the sample\n", one_way_earlier,
                    dropped_earlier);
        ++fails;
    }
    std::printf(fails ? "FAILED %d\n" : "ok\n", fails);
    return fails ? 1 : 0;
}
