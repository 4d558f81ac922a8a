// basis_kernels.cu -- shell-pair setup on the GPU: Boys-function table,
// per-component normalisation and the McMurchie-Davidson Hermite expansion
// coefficients of every primitive pair, derivative (small-component)
// functions included.  Stage (i) set-up of the AO integrals (paper Sec. 2.4,
// "quaternion scalar integrals"; restricted kinetic balance, Eq. RKB).
#include <math.h>

#include "qdt_internal.cuh"

namespace qdt {

// ------------------------------------------------------------- Boys table
// tab[i][n] = F_n(i * delta) for n < kBoysCols, by the power series of the
// top order followed by downward recursion F_n = (2T F_{n+1} + e^{-T}) / (2n+1).
__global__ void boys_table_kernel(double *tab) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kBoysGrid) return;
    double T = i * kBoysDelta;
    int M = kBoysCols - 1;
    double term = 1.0 / (2.0 * M + 1.0), sum = term;
    for (int k = 1; k < 2000; ++k) {
        term *= 2.0 * T / (2.0 * M + 2.0 * k + 1.0);
        sum += term;
        if (term < 1e-19 * sum) break;
    }
    double e = exp(-T);
    double *row = tab + (size_t)i * kBoysCols;
    row[M] = e * sum;
    for (int n = M - 1; n >= 0; --n) row[n] = (2.0 * T * row[n + 1] + e) / (2.0 * n + 1.0);
    // after the FP64 table: its FP32 copy (header of the plain-FP32 integrals), its
    // split into FP32 pairs hi + lo, and per grid point exp(-T_i) and T_i as pairs
    // (header of the compensated-FP32 integrals); layout in boys_tables()
    BoysTables t = boys_tables(tab);
    for (int n = 0; n <= M; ++n) {
        t.f32[(size_t)i * kBoysCols + n] = (float)row[n];
        t.pair[(size_t)i * kBoysCols + n] = split_pair(row[n]);
    }
    t.exp_pair[i] = split_pair(e);
    t.t_pair[i] = split_pair(T);
}

void launch_boys_table(double *d_tab, cudaStream_t s) {
    boys_table_kernel<<<(kBoysGrid + 127) / 128, 128, 0, s>>>(d_tab);
    QDT_CHECK_LAUNCH();
}

// Cartesian triple of component c of order l (x-major order).
__device__ inline void cart_triple(int l, int c, int &i, int &j, int &k) {
    int n = 0;
    for (int a = l; a >= 0; --a)
        for (int b = l - a; b >= 0; --b) {
            if (n == c) { i = a; j = b; k = l - a - b; return; }
            ++n;
        }
    i = j = k = 0;
}

__device__ inline double dfact_odd(int n) {  // (2n-1)!!
    double r = 1.0;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

// ----------------------------------------------------------- normalisation
// norms[noff + c] = 1 / sqrt(<g_c|g_c>) of the contracted component c.
__global__ void shell_norm_kernel(const ShellDev *shells, int nsh, const double *exps,
                                  const double *coefs, double *norms) {
    int s = blockIdx.x;
    if (s >= nsh) return;
    ShellDev sh = shells[s];
    int nc = ncart(sh.l);
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int ix, iy, iz;
        cart_triple(sh.l, c, ix, iy, iz);
        double S = 0.0;
        for (int p = 0; p < sh.nprim; ++p)
            for (int q = 0; q < sh.nprim; ++q) {
                double g = exps[sh.poff + p] + exps[sh.poff + q];
                double v = coefs[sh.poff + p] * coefs[sh.poff + q] * pow(M_PI / g, 1.5);
                v *= dfact_odd(ix) / pow(2.0 * g, ix);
                v *= dfact_odd(iy) / pow(2.0 * g, iy);
                v *= dfact_odd(iz) / pow(2.0 * g, iz);
                S += v;
            }
        norms[sh.noff + c] = 1.0 / sqrt(S);
    }
}

void launch_shell_norms(const ShellDev *shells, int nL_shells, const double *exps,
                        const double *coefs, double *norms, cudaStream_t s) {
    if (nL_shells <= 0) return;
    shell_norm_kernel<<<nL_shells, 32, 0, s>>>(shells, nL_shells, exps, coefs, norms);
    QDT_CHECK_LAUNCH();
}

// ------------------------------------------------- Hermite coefficients
// For primitive pair (alpha at A, beta at B) the 1D McMurchie-Davidson
// coefficients E^{ij}_t of (x-A)^i (x-B)^j exp(-alpha (x-A)^2 - beta (x-B)^2)
// = sum_t E^{ij}_t Lambda_t(x; p, P):
//   E^{00}_0 = exp(-alpha beta / p X_AB^2),
//   E^{i+1,j}_t = E^{ij}_{t-1} / (2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1},
//   E^{i,j+1}_t = E^{ij}_{t-1} / (2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}.
constexpr int kE1 = kMaxLFunc + 1;          // i, j <= kMaxLFunc
constexpr int kEt = 2 * kMaxLFunc + 1;      // t <= i + j

struct FuncTerms {              // a basis function as <= 2 primitive Cartesian terms
    int n;
    int pw[2][3];
    double w[2];
};

// Terms of local function f of shell `sh` for primitive prim (coefficient
// d, exponent a, normalisation of its parent component).
__device__ inline void func_terms(const ShellDev &sh, int f, double a, double d, const double *norms,
                                  FuncTerms &t) {
    if (!sh.isS) {
        int i, j, k;
        cart_triple(sh.l, f, i, j, k);
        t.n = 1;
        t.pw[0][0] = i; t.pw[0][1] = j; t.pw[0][2] = k;
        t.w[0] = norms[sh.noff + f] * d;
        return;
    }
    if (sh.red) {
        // p shell: d/dr_K (x_i g) = delta_iK g - 2a x_i x_K g is symmetric in (i, K);
        // function f is the pair i <= K in the order of the Cartesian d components
        int pw2[3];
        cart_triple(2, f, pw2[0], pw2[1], pw2[2]);
        int i = pw2[0] ? 0 : (pw2[1] ? 1 : 2);           // first axis of the pair
        double N = norms[sh.noff + i] * d;               // the three p components share N
        t.pw[0][0] = pw2[0]; t.pw[0][1] = pw2[1]; t.pw[0][2] = pw2[2];
        t.w[0] = -2.0 * a * N;
        t.n = 1;
        if (pw2[i] == 2) {                               // i == K: the delta_iK g term
            t.pw[1][0] = t.pw[1][1] = t.pw[1][2] = 0;
            t.w[1] = N;
            t.n = 2;
        }
        return;
    }
    // d/dr_K of N (x-A)^i.. e^{-a r^2} = N (i (x-A)^{i-1} - 2 a (x-A)^{i+1}) ..
    int c = f / 3, K = f % 3, pw[3];
    cart_triple(sh.l, c, pw[0], pw[1], pw[2]);
    double N = norms[sh.noff + c] * d;
    t.n = 0;
    t.pw[0][0] = pw[0]; t.pw[0][1] = pw[1]; t.pw[0][2] = pw[2];
    t.pw[0][K] += 1;
    t.w[0] = -2.0 * a * N;
    t.n = 1;
    if (pw[K] > 0) {
        t.pw[1][0] = pw[0]; t.pw[1][1] = pw[1]; t.pw[1][2] = pw[2];
        t.pw[1][K] -= 1;
        t.w[1] = pw[K] * N;
        t.n = 2;
    }
}

__device__ inline void pair_fp_decode(const PairDev &pr, int nfb, int fp, int &fa, int &fb) {
    if (pr.sa == pr.sb) {
        // upper triangle, row-major: fp = fa*n - fa(fa-1)/2 + (fb - fa)
        int n = nfb, a = 0, base = 0;
        while (base + (n - a) <= fp) { base += n - a; ++a; }
        fa = a; fb = a + (fp - base);
    } else {
        fa = fp / nfb; fb = fp % nfb;
    }
}

__device__ inline void htrip(int h, int &t, int &u, int &v) {
    int s = 0;
    while (nherm(s) <= h) ++s;
    int rem = h - (s ? nherm(s - 1) : 0);
    int uv = 0;
    while ((uv + 1) * (uv + 2) / 2 <= rem) ++uv;
    v = rem - uv * (uv + 1) / 2;
    u = uv - v;
    t = s - uv;
}

// One CTA per primitive pair: 1D tables in shared memory, then the E matrix
// E[h][fp] over the pair's Hermite functions h of order <= Lab and its
// function pairs fp (function pairs contiguous, for coalesced reads).
__global__ void prim_pair_kernel(const ShellDev *shells, const PairDev *pairs, const int *pp_pair,
                                 const double *exps, const double *coefs, const double *norms,
                                 PrimPairDev *pp, double *E) {
    __shared__ double Ex[3][kE1][kE1][kEt];
    int ipp = blockIdx.x;
    int ip = pp_pair[ipp];
    PairDev pr = pairs[ip];
    ShellDev A = shells[pr.sa], B = shells[pr.sb];
    int ia = pp[ipp].ia, ib = pp[ipp].ib;
    double a = exps[A.poff + ia], b = exps[B.poff + ib];
    double da = coefs[A.poff + ia], db = coefs[B.poff + ib];
    double p = a + b;
    if (threadIdx.x < 3) {
        int x = threadIdx.x;
        double Px = (a * A.A[x] + b * B.A[x]) / p;
        double XAB = A.A[x] - B.A[x], XPA = Px - A.A[x], XPB = Px - B.A[x];
        for (int i = 0; i < kE1; ++i)
            for (int j = 0; j < kE1; ++j)
                for (int t = 0; t < kEt; ++t) Ex[x][i][j][t] = 0.0;
        Ex[x][0][0][0] = exp(-a * b / p * XAB * XAB);
        for (int i = 0; i < kE1; ++i) {
            if (i > 0)
                for (int t = 0; t <= i; ++t) {
                    double v = XPA * Ex[x][i - 1][0][t];
                    if (t > 0) v += Ex[x][i - 1][0][t - 1] / (2.0 * p);
                    if (t + 1 < kEt) v += (t + 1) * Ex[x][i - 1][0][t + 1];
                    Ex[x][i][0][t] = v;
                }
            for (int j = 1; j < kE1; ++j)
                for (int t = 0; t <= i + j && t < kEt; ++t) {
                    double v = XPB * Ex[x][i][j - 1][t];
                    if (t > 0) v += Ex[x][i][j - 1][t - 1] / (2.0 * p);
                    if (t + 1 < kEt) v += (t + 1) * Ex[x][i][j - 1][t + 1];
                    Ex[x][i][j][t] = v;
                }
        }
        if (x == 0) {
            PrimPairDev o;
            o.p = p;
            o.inv_p = 1.0 / p;
            for (int d = 0; d < 3; ++d) o.P[d] = (a * A.A[d] + b * B.A[d]) / p;
            o.eoff = pp[ipp].eoff;
            o.ia = ia;
            o.ib = ib;
            pp[ipp] = o;
        }
    }
    __syncthreads();
    int nh = nherm(pr.Lab);
    double *Eo = E + pp[ipp].eoff;
    for (int fp = threadIdx.x; fp < pr.nfp; fp += blockDim.x) {
        int fa, fb;
        pair_fp_decode(pr, B.nfunc, fp, fa, fb);
        FuncTerms ta, tb;
        func_terms(A, fa, a, da, norms, ta);
        func_terms(B, fb, b, db, norms, tb);
        for (int h = 0; h < nh; ++h) {
            int t, u, v;
            htrip(h, t, u, v);
            double s = 0.0;
            for (int x = 0; x < ta.n; ++x)
                for (int y = 0; y < tb.n; ++y) {
                    const int *pa = ta.pw[x], *pb = tb.pw[y];
                    if (t > pa[0] + pb[0] || u > pa[1] + pb[1] || v > pa[2] + pb[2]) continue;
                    s += ta.w[x] * tb.w[y] * Ex[0][pa[0]][pb[0]][t] * Ex[1][pa[1]][pb[1]][u] *
                         Ex[2][pa[2]][pb[2]][v];
                }
            Eo[(size_t)h * pr.nfp + fp] = s;          // [h][fp]: function pairs contiguous
        }
    }
}

// Launcher (pp_pair maps every primitive pair to its shell pair).
void launch_prim_pairs_map(const ShellDev *shells, const PairDev *pairs, const int *pp_pair,
                           long long npp, const double *exps, const double *coefs,
                           const double *norms, PrimPairDev *pp, double *E, cudaStream_t s) {
    if (npp <= 0) return;
    prim_pair_kernel<<<(unsigned)npp, 64, 0, s>>>(shells, pairs, pp_pair, exps, coefs, norms, pp, E);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
