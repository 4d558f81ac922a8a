// density_kernels.cu -- quaternion pair densities (paper Eqs. Den and
// QuaternionScatter), density-weighted Schwarz screening order (Eq. SchwarzDen)
// and the row gathers / packing that feed and drain the contractions.
#include <math.h>

#include "qdt_internal.cuh"

namespace qdt {

struct cplx { double re, im; };
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ inline cplx cconj(cplx a) { return {a.re, -a.im}; }
__device__ inline cplx cneg(cplx a) { return {-a.re, -a.im}; }
__device__ inline cplx ctimes_i(cplx a) { return {-a.im, a.re}; }

// Compensated FP32 pair x = h + l (~48-bit significand): products by the
// exact-product FMA plus the cross terms, sums by the error-free two-sum,
// both renormalised.  The intrinsics keep the compiler from contracting the
// rounded operations into FMAs.  FP32 issues 64 times faster than FP64 on this
// part, so the split form's density (whose digits keep 42 bits) runs in these.
struct dfl { float h, l; };
__device__ inline dfl dfl_of(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ inline double dfl_val(dfl a) { return (double)a.h + (double)a.l; }
__device__ inline dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ inline dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bv = __fsub_rn(s, a.h);
    float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
    err = __fadd_rn(err, __fadd_rn(a.l, b.l));
    const float t = __fadd_rn(s, err);
    return {t, __fsub_rn(err, __fsub_rn(t, s))};
}
__device__ inline dfl operator-(dfl a) { return {-a.h, -a.l}; }
__device__ inline dfl operator-(dfl a, dfl b) { return a + (-b); }

// Complex numbers over the real type R (double, or dfl in the split form).
template <class R> struct Cx { R re, im; };
template <class R> __device__ inline Cx<R> operator*(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __device__ inline Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __device__ inline Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __device__ inline Cx<R> conj_(Cx<R> a) { return {a.re, -a.im}; }
template <class R> __device__ inline Cx<R> neg_(Cx<R> a) { return {-a.re, -a.im}; }
template <class R> __device__ inline Cx<R> times_i(Cx<R> a) { return {-a.im, a.re}; }
__device__ inline double val_(double x) { return x; }
__device__ inline double val_(dfl x) { return dfl_val(x); }
__device__ inline double real_of(double x, double) { return x; }
__device__ inline dfl real_of(double x, dfl) { return dfl_of(x); }

// Two-spinor coefficients of row f, Kramers pair k: alpha = q0 + i q1, beta = q2 + i q3.
__device__ inline void spinor(const double *Cq, int nK, int f, int k, cplx &al, cplx &be) {
    const double *q = Cq + ((size_t)f * nK + k) * 4;
    al = {q[0], q[1]};
    be = {q[2], q[3]};
}

__device__ inline void decode_fp(const PairDev &pr, int nfb, int fp, int &fa, int &fb) {
    if (pr.sa == pr.sb) {
        int a = 0, base = 0;
        while (base + (nfb - a) <= fp) { base += nfb - a; ++a; }
        fa = a; fb = a + (fp - base);
    } else {
        fa = fp / nfb; fb = fp % nfb;
    }
}

__device__ inline void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// Maximum over a warp by shuffles, then over the block's warps (result in thread 0).
__device__ inline double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ inline double block_max(double v) {
    __shared__ double wm[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    v = warp_max(v);
    if (l == 0) wm[w] = v;
    __syncthreads();
    if (w == 0) v = warp_max(l < (int)(blockDim.x >> 5) ? wm[l] : 0.0);
    return v;
}

// Coulomb: row (a,b) of a class-0 pair, columns (RS, part):
//   A = D^{RS}_{ab} + D^{RS}_{ba},  B = D^{R'S}_{ab} + D^{R'S}_{ba}  (a != b; a == b: single term)
//   D^{xy}_{ab} = sum_tau conj(C[a,tau,x]) C[b,tau,y];  for the partner R':
//   conj(C[a,alpha,R']) = -C[a,beta,R],  conj(C[a,beta,R']) = C[a,alpha,R].
// KU (Kramers-unrestricted input): R, S are spinors with their own
// coefficients; only A is formed, 2 parts (Re A, Im A) per spinor pair.
//
// One CTA per shell pair: the coefficient rows of its shells (active range)
// are staged in shared memory once, then the threads run over the flattened
// (function pair, column pair RS) range, each element's parts written as
// 16-byte stores next to its neighbours' (a warp writes contiguous runs of a
// row).  One barrier per CTA.
constexpr int kDensityThreads = 256;

// Shared-memory layout of a density CTA: rows of shell A, rows of shell B
// (none for a diagonal pair), then the packed (a, b) of every function pair.
template <class R>
struct DensityStage {
    const R *ca, *cb;
    const int *ftab;
};

template <class R>
__device__ inline DensityStage<R> stage_pair(const PairDev &pr, const ShellDev &A, const ShellDev &B,
                                             const double *Cq, int nK, int k0, int nKa, double *raw) {
    const int row = 4 * nKa;
    const bool diag = pr.sa == pr.sb;
    R *ca = reinterpret_cast<R *>(raw);
    R *cb = diag ? ca : ca + (size_t)A.nfunc * row;
    int *ftab = reinterpret_cast<int *>(ca + (size_t)(A.nfunc + (diag ? 0 : B.nfunc)) * row);
    for (int i = threadIdx.x; i < A.nfunc * row; i += blockDim.x) {
        const int f = i / row, j = i - f * row;
        ca[i] = real_of(Cq[((size_t)(A.foff + f) * nK + k0) * 4 + j], R{});
    }
    if (!diag)
        for (int i = threadIdx.x; i < B.nfunc * row; i += blockDim.x) {
            const int f = i / row, j = i - f * row;
            cb[i] = real_of(Cq[((size_t)(B.foff + f) * nK + k0) * 4 + j], R{});
        }
    for (int fp = threadIdx.x; fp < pr.nfp; fp += blockDim.x) {
        int fa, fb;
        decode_fp(pr, B.nfunc, fp, fa, fb);
        ftab[fp] = fa | (fb << 16);
    }
    __syncthreads();
    return {ca, cb, ftab};
}

template <class R>
__device__ inline void spinor_s(const R *c, int k, Cx<R> &al, Cx<R> &be) {
    al = {c[4 * k], c[4 * k + 1]};
    be = {c[4 * k + 2], c[4 * k + 3]};
}

template <bool KU, class R>
__global__ void __launch_bounds__(kDensityThreads) density_coulomb_kernel(
    const PairDev *pairs, const int *bra_order, const ShellDev *shells, const double *Cq, int nK, int k0, int nKa,
    const int *rsR, const int *rsS, int nRS, double *D, double *Dmax) {
    extern __shared__ double crow_raw[];
    const int sp = bra_order[blockIdx.x];
    const PairDev pr = pairs[sp];
    const ShellDev A = shells[pr.sa], B = shells[pr.sb];
    constexpr int parts = KU ? 2 : 4;
    const long long ld = (long long)parts * nRS;
    const DensityStage<R> st = stage_pair<R>(pr, A, B, Cq, nK, k0, nKa, crow_raw);
    const int row = 4 * nKa;
    double vmax = 0.0;
    int fp = threadIdx.x / nRS, rs = threadIdx.x - fp * nRS;
    while (fp < pr.nfp) {
        const int f = st.ftab[fp], fa = f & 0xffff, fb = f >> 16;
        const R *ca = st.ca + (size_t)fa * row, *cb = st.cb + (size_t)fb * row;
        const bool two = A.foff + fa != B.foff + fb;        // a != b: both orders
        const int Rr = rsR[rs], Ss = rsS[rs];
        Cx<R> aaR, abR, aaS, abS, baR, bbR, baS, bbS;
        spinor_s(ca, Rr, aaR, abR);
        spinor_s(ca, Ss, aaS, abS);
        spinor_s(cb, Rr, baR, bbR);
        spinor_s(cb, Ss, baS, bbS);
        Cx<R> Av = conj_(aaR) * baS + conj_(abR) * bbS;
        if (two) Av = Av + (conj_(baR) * aaS + conj_(bbR) * abS);
        const double are = val_(Av.re), aim = val_(Av.im);
        double2 *o = reinterpret_cast<double2 *>(D + (pr.rowoff + fp) * ld + (long long)parts * rs);
        o[0] = make_double2(are, aim);
        vmax = fmax(vmax, fmax(fabs(are), fabs(aim)));
        if (!KU) {
            Cx<R> Bv = aaR * bbS - abR * baS;
            if (two) Bv = Bv + (baR * abS - bbR * aaS);
            const double bre = val_(Bv.re), bim = val_(Bv.im);
            o[1] = make_double2(bre, bim);
            vmax = fmax(vmax, fmax(fabs(bre), fabs(bim)));
        }
        rs += blockDim.x;
        while (rs >= nRS) { rs -= nRS; ++fp; }
    }
    // block max -> Dmax[sp]
    vmax = block_max(vmax);
    if (threadIdx.x == 0) atomic_max_nonneg(Dmax + sp, vmax);
}

// sigma_J between the spin components: c = (conj(C[u,alpha,x]), conj(C[u,beta,x])),
// d = (C[v,alpha,y], C[v,beta,y]).
template <class R>
__device__ inline Cx<R> sigma_form(int J, Cx<R> c1, Cx<R> c2, Cx<R> d1, Cx<R> d2) {
    if (J == 0) return c1 * d2 + c2 * d1;                          // sigma_x
    if (J == 1) return times_i(c2 * d1 - c1 * d2);                 // sigma_y
    return c1 * d1 - c2 * d2;                                      // sigma_z
}

// Gaunt / gauge: rows (a in L, b in S), columns (J, RS, part) of the folded
// L-S alpha densities D^J_{ab} + D^J_{ba} (Eqs. GauntInt, gaugeInt).  Same
// work layout as the Coulomb kernel.
template <bool KU, class R>
__global__ void __launch_bounds__(kDensityThreads) density_gaunt_kernel(
    const PairDev *pairs, const int *bra_order, const ShellDev *shells, const double *Cq, int nK, int k0, int nKa,
    const int *rsR, const int *rsS, int nRS, double *D, double *Dmax) {
    extern __shared__ double crow_raw[];
    const int sp = bra_order[blockIdx.x];
    const PairDev pr = pairs[sp];
    const ShellDev A = shells[pr.sa], B = shells[pr.sb];
    constexpr int parts = KU ? 2 : 4;
    const long long ld = 3LL * parts * nRS;
    const DensityStage<R> st = stage_pair<R>(pr, A, B, Cq, nK, k0, nKa, crow_raw);
    const int row = 4 * nKa;
    double vmax = 0.0;
    int fp = threadIdx.x / nRS, rs = threadIdx.x - fp * nRS;
    while (fp < pr.nfp) {
        const int f = st.ftab[fp], fa = f & 0xffff, fb = f >> 16;
        const R *ca = st.ca + (size_t)fa * row, *cb = st.cb + (size_t)fb * row;
        double *drow = D + (pr.rowoff + fp) * ld;
        const int Rr = rsR[rs], Ss = rsS[rs];
        Cx<R> aaR, abR, aaS, abS, baR, bbR, baS, bbS;
        spinor_s(ca, Rr, aaR, abR);
        spinor_s(ca, Ss, aaS, abS);
        spinor_s(cb, Rr, baR, bbR);
        spinor_s(cb, Ss, baS, bbS);
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            // x = R: (conj alpha, conj beta); x = R': (-beta, alpha)
            const Cx<R> Av = sigma_form(J, conj_(aaR), conj_(abR), baS, bbS) +
                             sigma_form(J, conj_(baR), conj_(bbR), aaS, abS);
            const double are = val_(Av.re), aim = val_(Av.im);
            double2 *o = reinterpret_cast<double2 *>(drow + (long long)J * parts * nRS + (long long)parts * rs);
            o[0] = make_double2(are, aim);
            vmax = fmax(vmax, fmax(fabs(are), fabs(aim)));
            if (!KU) {
                const Cx<R> Bv = sigma_form(J, neg_(abR), aaR, baS, bbS) + sigma_form(J, neg_(bbR), baR, aaS, abS);
                const double bre = val_(Bv.re), bim = val_(Bv.im);
                o[1] = make_double2(bre, bim);
                vmax = fmax(vmax, fmax(fabs(bre), fabs(bim)));
            }
        }
        rs += blockDim.x;
        while (rs >= nRS) { rs -= nRS; ++fp; }
    }
    vmax = block_max(vmax);
    if (threadIdx.x == 0) atomic_max_nonneg(Dmax + sp, vmax);
}

template <bool KU, class R>
void launch_density_t(bool gaunt, const PairDev *pairs, const int *bra_order, int nsp, const ShellDev *shells,
                      const double *Cq, int nK, int k0, int nKa, int maxnf, int maxnfp, const int *rsR,
                      const int *rsS, int nRS, double *D, double *Dmax, cudaStream_t s) {
    // two shells' coefficient rows (active range) and the function-pair table
    const size_t smem = 2 * (size_t)maxnf * 4 * (size_t)(nKa > 0 ? nKa : 1) * sizeof(R) +
                        (size_t)maxnfp * sizeof(int) + 16;
    if (smem > (size_t)200 * 1024) throw Error{QDT_ERR_ARG, "density: too many active columns"};
    if (gaunt) {
        if (smem > (size_t)48 * 1024)
            QDT_CUDA_TRY(cudaFuncSetAttribute(density_gaunt_kernel<KU, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        density_gaunt_kernel<KU, R><<<nsp, kDensityThreads, smem, s>>>(pairs, bra_order, shells, Cq, nK, k0, nKa, rsR,
                                                                       rsS, nRS, D, Dmax);
    } else {
        if (smem > (size_t)48 * 1024)
            QDT_CUDA_TRY(cudaFuncSetAttribute(density_coulomb_kernel<KU, R>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        density_coulomb_kernel<KU, R><<<nsp, kDensityThreads, smem, s>>>(pairs, bra_order, shells, Cq, nK, k0, nKa,
                                                                         rsR, rsS, nRS, D, Dmax);
    }
    QDT_CHECK_LAUNCH();
}

// The split form (pairs = true) computes the density in compensated FP32
// pairs, the FP64 form in FP64.  maxnf: functions of the largest shell;
// maxnfp: function pairs of the largest shell pair.
void launch_density(bool gaunt, bool ku, bool pairs_arith, const PairDev *pairs, const int *bra_order, int nsp,
                    const ShellDev *shells, int maxnf, int maxnfp, const double *Cq, int nK, int k0, const int *rsR,
                    const int *rsS, int nRS, double *D, double *Dmax, cudaStream_t s) {
    if (nsp <= 0) return;
    // active units: every R and S index of the column list lies in [0, nKa)
    // (Kramers pairs, or spinors of unrestricted input: the same triangular list)
    int nKa = 0;
    while ((long long)nKa * (nKa + 1) / 2 < nRS) ++nKa;
    if (ku) {
        if (pairs_arith) launch_density_t<true, dfl>(gaunt, pairs, bra_order, nsp, shells, Cq, nK, k0, nKa, maxnf, maxnfp, rsR, rsS, nRS, D, Dmax, s);
        else launch_density_t<true, double>(gaunt, pairs, bra_order, nsp, shells, Cq, nK, k0, nKa, maxnf, maxnfp, rsR, rsS, nRS, D, Dmax, s);
    } else {
        if (pairs_arith) launch_density_t<false, dfl>(gaunt, pairs, bra_order, nsp, shells, Cq, nK, k0, nKa, maxnf, maxnfp, rsR, rsS, nRS, D, Dmax, s);
        else launch_density_t<false, double>(gaunt, pairs, bra_order, nsp, shells, Cq, nK, k0, nKa, maxnf, maxnfp, rsR, rsS, nRS, D, Dmax, s);
    }
}

// Dmax of one MO block (MO-driven route): the largest |entry| of the density
// rows of each shell pair over the block's columns [c0, c1) of each of the nJ
// column groups (row length ld, group stride N4).
__global__ void block_dmax_kernel(const PairDev *pairs, const double *D, long long ld, int nJ, long long N4,
                                  long long c0, long long c1, double *Dmax) {
    const PairDev pr = pairs[blockIdx.x];
    const long long w = c1 - c0, per_row = (long long)nJ * w;
    double vmax = 0.0;
    for (long long i = threadIdx.x; i < (long long)pr.nfp * per_row; i += blockDim.x) {
        const long long r = i / per_row, rem = i - r * per_row, J = rem / w, c = rem - J * w;
        vmax = fmax(vmax, fabs(D[(pr.rowoff + r) * ld + J * N4 + c0 + c]));
    }
    vmax = block_max(vmax);
    if (threadIdx.x == 0) Dmax[blockIdx.x] = vmax;
}

void launch_block_dmax(const PairDev *pairs, int nsp, const double *D, long long ld, int nJ, long long N4,
                       long long c0, long long c1, double *Dmax, cudaStream_t s) {
    if (nsp <= 0) return;
    block_dmax_kernel<<<nsp, 256, 0, s>>>(pairs, D, ld, nJ, N4, c0, c1, Dmax);
    QDT_CHECK_LAUNCH();
}

// ----------------------------------------------------------- ket ordering
// w_CD = Q_CD * Dmax_CD; ket positions sorted by w descending (ties: pair id
// ascending) by rank counting.  A bra pair AB keeps exactly the ket prefix
// with Q_AB * w >= tau (the product is monotone in w).
__global__ void ket_rank_kernel(const double *Q, const double *Dmax, int n, double *w_sorted,
                                int *ket_sp) {
    __shared__ double tile[1024];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double wi = (i < n) ? Q[i] * Dmax[i] : 0.0;
    int rank = 0;
    for (int j0 = 0; j0 < n; j0 += 1024) {
        __syncthreads();
        for (int j = threadIdx.x; j < 1024; j += blockDim.x)
            tile[j] = (j0 + j < n) ? Q[j0 + j] * Dmax[j0 + j] : -1.0;
        __syncthreads();
        if (i < n) {
            int jn = min(1024, n - j0);
            for (int j = 0; j < jn; ++j) {
                double wj = tile[j];
                rank += (wj > wi) || (wj == wi && j0 + j < i);
            }
        }
    }
    if (i < n) {
        ket_sp[rank] = i;
        w_sorted[rank] = wi;
    }
}

// exclusive prefix sums of nfp over the sorted ket order (single CTA): warp
// scans by shuffles, then a scan of the warp totals by the first warp
__global__ void ket_col_kernel(const PairDev *pairs, const int *ket_sp, int n, long long *col) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = (i < n) ? pairs[ket_sp[i]].nfp : 0;
        long long x = v;                                   // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {                                      // inclusive scan of the warp totals
            long long t = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) wsum[lane] = t;
        }
        __syncthreads();
        if (i < n) col[i] = carry + (w > 0 ? wsum[w - 1] : 0) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) col[n] = carry;
}

// prefix[sp] = number of sorted ket positions kept by bra pair sp
__global__ void prefix_kernel(const double *Q, const double *w_sorted, int n, double tau, int *prefix) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double q = Q[i];
    int lo = 0, hi = n;                       // first position with q * w < tau
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (q * w_sorted[mid] >= tau) lo = mid + 1; else hi = mid;
    }
    prefix[i] = lo;
}

void launch_ket_order(const double *Q, const double *Dmax, int nsp, double *w, int *ket_sp,
                      cudaStream_t s) {
    if (nsp <= 0) return;
    ket_rank_kernel<<<(nsp + 255) / 256, 256, 0, s>>>(Q, Dmax, nsp, w, ket_sp);
    QDT_CHECK_LAUNCH();
}

void launch_ket_columns(const PairDev *pairs, const int *ket_sp, int nsp, long long *ket_col,
                        cudaStream_t s) {
    ket_col_kernel<<<1, 1024, 0, s>>>(pairs, ket_sp, nsp, ket_col);
    QDT_CHECK_LAUNCH();
}

void launch_prefix_lengths(const double *Q, const double *w_sorted, int nsp, double tau, int *prefix,
                           cudaStream_t s) {
    if (nsp <= 0) return;
    prefix_kernel<<<(nsp + 255) / 256, 256, 0, s>>>(Q, w_sorted, nsp, tau, prefix);
    QDT_CHECK_LAUNCH();
}

// dst rows of sorted ket position k  <-  src rows of its pair (bra order)
__global__ void gather_rows_kernel(const double *src, const PairDev *pairs, const int *ket_sp,
                                   const long long *ket_col, long long rowlen, double *dst) {
    int k = blockIdx.x;
    PairDev pr = pairs[ket_sp[k]];
    const double *s = src + pr.rowoff * rowlen;
    double *d = dst + ket_col[k] * rowlen;
    long long n = (long long)pr.nfp * rowlen;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

void launch_gather_rows(const double *src, const PairDev *pairs, const int *ket_sp,
                        const long long *ket_col, int nsp, long long rowlen, double *dst,
                        cudaStream_t s) {
    if (nsp <= 0) return;
    gather_rows_kernel<<<nsp, 256, 0, s>>>(src, pairs, ket_sp, ket_col, rowlen, dst);
    QDT_CHECK_LAUNCH();
}

__global__ void merge_rows_kernel(const double *in, const int *m0, const int *m1, int nrows, int rowlen,
                                  double *out) {
    int r = blockIdx.x;
    if (r >= nrows) return;
    const double *a = in + (size_t)m0[r] * rowlen;
    const double *b = m1[r] >= 0 ? in + (size_t)m1[r] * rowlen : nullptr;
    double *o = out + (size_t)r * rowlen;
    for (int i = threadIdx.x; i < rowlen; i += blockDim.x) o[i] = b ? a[i] + b[i] : a[i];
}

void launch_merge_rows(const double *in, const int *m0, const int *m1, int nrows, int rowlen, double *out,
                       cudaStream_t s) {
    if (nrows <= 0) return;
    merge_rows_kernel<<<nrows, 128, 0, s>>>(in, m0, m1, nrows, rowlen, out);
    QDT_CHECK_LAUNCH();
}

// Restricted kinetic balance (Eq. RKB): the small-component spinor
// (1/2c) sigma.p chi_mu c_mu, p = -i grad, expands over the derivative
// functions d_K chi_mu with coefficients (-i/2c) sigma_K c_mu.  in[nL][n][4]
// holds (Re a, Im a, Re b, Im b) of each two-spinor c_mu; out[3 nL][n][4]
// rows 3 mu + K.  sigma.p commutes with time reversal, so quaternion columns
// (one spinor of a Kramers pair) map the same way as unrestricted spinors.
__global__ void rkb_map_kernel(const double *in, long long nL, long long n, double h, double *out) {
    const long long total = nL * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long mu = e / n, p = e - mu * n;
        const double ar = in[4 * e], ai = in[4 * e + 1], br = in[4 * e + 2], bi = in[4 * e + 3];
        double *o = out + 4 * (3 * mu * n + p);
        // x: sigma_x (a, b) = (b, a);  y: (-i b, i a);  z: (a, -b); then times -i h
        const double v[3][4] = {{bi * h, -br * h, ai * h, -ar * h},
                                {-br * h, -bi * h, ar * h, ai * h},
                                {ai * h, -ar * h, -bi * h, br * h}};
#pragma unroll
        for (int K = 0; K < 3; ++K)
#pragma unroll
            for (int j = 0; j < 4; ++j) o[4 * K * n + j] = v[K][j];
    }
}

void launch_rkb_map(const double *in, long long nL, long long n, double c_light, double *out,
                    cudaStream_t s) {
    if (nL <= 0 || n <= 0) return;
    long long blocks = (nL * n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    rkb_map_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, nL, n, 0.5 / c_light, out);
    QDT_CHECK_LAUNCH();
}

__global__ void zero_kernel(double *p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

void launch_zero(double *p, long long n, cudaStream_t s) {
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    zero_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, n);
    QDT_CHECK_LAUNCH();
}

// Integral rows zeroed only as far as a contraction reads them: row r up to
// the larger K extent of the two 64-row tiles of its 128-row tile, rounded up
// to 64 (the split form's row tiles are 128 rows and its K subtiles 64 wide),
// at most ld.  One CTA per row.
__global__ void zero_rows_kernel(double *W, long long ld, long long rows, const long long *kt64, long long nt64) {
    const long long r = blockIdx.x;
    if (r >= rows) return;
    const long long t = (r / 128) * 2;
    long long e = kt64[t];
    if (t + 1 < nt64) e = max(e, kt64[t + 1]);
    e = min(ld, (e + 63) / 64 * 64);
    double *row = W + r * ld;
    for (long long k = threadIdx.x; k < e; k += blockDim.x) row[k] = 0.0;
}

void launch_zero_rows(double *W, long long ld, long long rows, const long long *kt64, long long nt64,
                      cudaStream_t s) {
    if (rows <= 0 || ld <= 0) return;
    zero_rows_kernel<<<(unsigned)rows, 256, 0, s>>>(W, ld, rows, kt64, nt64);
    QDT_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- packing
// out[t][parts^2], t = pq nP - pq(pq-1)/2 + (rs - pq) for pq <= rs:
// out[t][parts i + j] = O[parts pq + i][parts rs + j]  (parts 4: Kramers pairs,
// parts 2: spinor pairs of Kramers-unrestricted input)
template <int PARTS>
__global__ void pack_kernel(const double *O, long long ldo, int nP, double *out) {
    int pq = blockIdx.y;
    for (int rs = pq + blockIdx.x * blockDim.x + threadIdx.x; rs < nP; rs += gridDim.x * blockDim.x) {
        long long t = (long long)pq * nP - (long long)pq * (pq - 1) / 2 + (rs - pq);
        double *o = out + t * PARTS * PARTS;
#pragma unroll
        for (int i = 0; i < PARTS; ++i) {
            const double *src = O + ((long long)PARTS * pq + i) * ldo + (long long)PARTS * rs;
#pragma unroll
            for (int j = 0; j < PARTS; ++j) o[PARTS * i + j] = src[j];
        }
    }
}

void launch_pack(const double *O, long long ldo, int nP, int parts, double *out, cudaStream_t s) {
    if (nP <= 0) return;
    dim3 grid((nP + 255) / 256, nP);
    if (parts == 2) pack_kernel<2><<<grid, 256, 0, s>>>(O, ldo, nP, out);
    else pack_kernel<4><<<grid, 256, 0, s>>>(O, ldo, nP, out);
    QDT_CHECK_LAUNCH();
}

// -------------------------------------------------------------- unpacking
// Symmetrised spinor density of spinor pair (x, y) as sign * [conj] Z with
// Z = A (which 0) or B (which 1) of Kramers pairs X <= Y:
//   (x, y) = (X, Y): A;  (X', Y): B;  (X, Y'): -conj B (Coulomb), +conj B (alpha);
//   (X', Y'): conj A (Coulomb), -conj A (alpha);  X > Y: conj of the swapped pair.
struct DMap { int X, Y, which; double sign; bool cj; };

__device__ inline DMap dmap(int x, int y, bool alpha) {
    int X = x >> 1, bx = x & 1, Y = y >> 1, by = y & 1;
    bool swap = X > Y;
    if (swap) { int t = X; X = Y; Y = t; t = bx; bx = by; by = t; }
    DMap m;
    m.X = X; m.Y = Y;
    if (!bx && !by) { m.which = 0; m.sign = 1.0; m.cj = false; }
    else if (bx && !by) { m.which = 1; m.sign = 1.0; m.cj = false; }
    else if (!bx && by) { m.which = 1; m.sign = alpha ? 1.0 : -1.0; m.cj = true; }
    else { m.which = 0; m.sign = alpha ? -1.0 : 1.0; m.cj = true; }
    if (swap) m.cj = !m.cj;
    return m;
}

__global__ void unpack_kernel(const double *packed, int nKa, int alpha, double *full) {
    const int n = 2 * nKa;
    const long long total = (long long)n * n * n * n;
    const int nP = nKa * (nKa + 1) / 2;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        int s = (int)(id % n), r = (int)((id / n) % n), q = (int)((id / n / n) % n), p = (int)(id / n / n / n);
        DMap m1 = dmap(p, q, alpha != 0), m2 = dmap(r, s, alpha != 0);
        int i1 = m1.X * nKa - m1.X * (m1.X - 1) / 2 + (m1.Y - m1.X);
        int i2 = m2.X * nKa - m2.X * (m2.X - 1) / 2 + (m2.Y - m2.X);
        int re1 = 2 * m1.which, im1 = re1 + 1, re2 = 2 * m2.which, im2 = re2 + 1;
        const double *blk;
        bool tr = i1 > i2;
        if (!tr) blk = packed + ((long long)i1 * nP - (long long)i1 * (i1 - 1) / 2 + (i2 - i1)) * 16;
        else blk = packed + ((long long)i2 * nP - (long long)i2 * (i2 - 1) / 2 + (i1 - i2)) * 16;
        auto O = [&](int a, int b) { return tr ? blk[4 * b + a] : blk[4 * a + b]; };
        double t1 = m1.cj ? -1.0 : 1.0, t2 = m2.cj ? -1.0 : 1.0;
        double vr = O(re1, re2) - t1 * t2 * O(im1, im2);
        double vi = t2 * O(re1, im2) + t1 * O(im1, re2);
        double sg = m1.sign * m2.sign;
        full[2 * id] = sg * vr;
        full[2 * id + 1] = sg * vi;
    }
}

// Kramers-unrestricted input: D^{pq} = Dr + i c Di of the spinor pair
// (min, max), c = -1 when p > q; (pq|rs) = (RR - c1 c2 II) + i (c2 RI + c1 IR).
__global__ void unpack_ku_kernel(const double *packed, int n, double *full) {
    const long long total = (long long)n * n * n * n;
    const int nP = n * (n + 1) / 2;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        int s = (int)(id % n), r = (int)((id / n) % n), q = (int)((id / n / n) % n), p = (int)(id / n / n / n);
        const int a1 = min(p, q), b1 = max(p, q), a2 = min(r, s), b2 = max(r, s);
        const int i1 = a1 * n - a1 * (a1 - 1) / 2 + (b1 - a1), i2 = a2 * n - a2 * (a2 - 1) / 2 + (b2 - a2);
        const bool tr = i1 > i2;
        const double *blk = tr ? packed + ((long long)i2 * nP - (long long)i2 * (i2 - 1) / 2 + (i1 - i2)) * 4
                               : packed + ((long long)i1 * nP - (long long)i1 * (i1 - 1) / 2 + (i2 - i1)) * 4;
        auto O = [&](int u, int v) { return tr ? blk[2 * v + u] : blk[2 * u + v]; };
        const double c1 = p > q ? -1.0 : 1.0, c2 = r > s ? -1.0 : 1.0;
        full[2 * id] = O(0, 0) - c1 * c2 * O(1, 1);
        full[2 * id + 1] = c2 * O(0, 1) + c1 * O(1, 0);
    }
}

void launch_unpack(const double *packed, int n_units, int gaunt_like, bool ku, double *full, cudaStream_t s) {
    long long n = ku ? (long long)n_units : 2LL * n_units, total = n * n * n * n;
    if (total <= 0) return;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (ku) unpack_ku_kernel<<<(unsigned)blocks, 256, 0, s>>>(packed, n_units, full);
    else unpack_kernel<<<(unsigned)blocks, 256, 0, s>>>(packed, n_units, gaunt_like, full);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
