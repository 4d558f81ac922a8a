// CPU check of the split form's FP32 planning (plan.h) on seeded random
// classes: the FP32 set is a per-row suffix of the kept kets, the decision is
// the same for (i, j) and (j, i), the reported bound is the brute-force sum and
// stays within the budget, and a 2 % larger threshold would exceed it.
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
    std::printf(fails ? "FAILED %d\n" : "ok\n", fails);
    return fails ? 1 : 0;
}
