// eri_kernels.cu -- AO two-electron integral tiles on the GPU (stage (i) of
// the paper's Sec. 3.3.1 decomposition), McMurchie-Davidson in FP64:
//
//   (xy|K|zw) = sum_{ij in X, kl in Y} sum_{h, h'} E^{ij}_{xy,h} (-1)^{|h'|}
//               E^{kl}_{zw,h'} R^K_{h+h'}(rho, P - Q)
//
//   1/r12 (Eq. Coulomb):    R^n_000 = (-2 rho)^n F_n(T) * 2 pi^{5/2} / (p q sqrt(p+q))
//   r12 (for Eq. gaugeInt): R^n_000 = (-2 rho)^n (F_n - F_{n-1})(T) * pi^{5/2} sqrt(p+q) / (p q)^2,
//                           F_{-1}(T) = -(2 T F_0 + e^{-T})  (Gaussian-smeared distance)
//   gauge kernel:  (xy|r_I r_J/r^3|zw) = delta_IJ (xy|1/r|zw) - (xy|d_I d_J r|zw),
//                  the last term shifting the Hermite index of the r12 tensor by e_I + e_J,
//   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}  (same in u, v).
//
// Work layout: a CTA owns one bra shell pair and a run of ket shell pairs.
// For every shell quartet the cheaper orientation is contracted (the pair with
// more function pairs takes the outer role X).  The primitive quartets of a
// quartet are processed in groups -- several outer primitive pairs times all
// inner ones when they fit in shared memory -- so that every phase (Boys
// values, one recursion level, the ket contraction T = sum R E', the bra
// contraction G += E T) keeps the CTA's lanes busy between two barriers.
//
// FP64 issue rate is the limit of this kernel, so the FP64 pipe does only
// arithmetic of the method: no pow, one exp, two divisions and one sqrt per
// primitive quartet; recursion sources and coefficients come from tables; the
// sign (-1)^{|h'|} is a negated FMA operand (even and odd Hermite orders run in
// separate loops) instead of a multiplication.
//
// Split form (DF): Boys values, prefactors and the Hermite recursion stay in
// FP64; the two contraction passes run in compensated FP32 pairs (x = hi + lo,
// ~48-bit significands): products by the exact-product FMA, sums by the
// error-free two-sum, so each multiply-add costs about twelve FP32
// operations, which issue 64 times faster than FP64 on this part.
#include <math.h>

#include <algorithm>
#include <cstdlib>

#include "qdt_internal.cuh"

namespace qdt {

namespace {

constexpr double kPi52 = 17.493418327624862;        // pi^{5/2}
constexpr double kTwoPi52 = 34.986836655249725;     // 2 pi^{5/2}
constexpr double kHalfSqrtPi = 0.88622692545275801;  // sqrt(pi) / 2
constexpr double kBoysInvDelta = 1.0 / kBoysDelta;

static_assert(kBoysNMax <= 15, "constant tables below hold 16 orders");
static_assert(kBoysTaylor == 7, "constant table below holds 1/k for k < 8");

__constant__ double c_inv_int[8] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7};
__constant__ double c_odd[16] = {1, 3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31};
__constant__ double c_inv_odd[16] = {1.0,      1.0 / 3,  1.0 / 5,  1.0 / 7,  1.0 / 9,  1.0 / 11,
                                     1.0 / 13, 1.0 / 15, 1.0 / 17, 1.0 / 19, 1.0 / 21, 1.0 / 23,
                                     1.0 / 25, 1.0 / 27, 1.0 / 29, 1.0 / 31};

__device__ inline void htrip_d(int h, int &t, int &u, int &v) {
    int s = 0;
    while (nherm(s) <= h) ++s;
    int rem = h - (s ? nherm(s - 1) : 0);
    int uv = 0;
    while ((uv + 1) * (uv + 2) / 2 <= rem) ++uv;
    v = rem - uv * (uv + 1) / 2;
    u = uv - v;
    t = s - uv;
}

// F_0..F_nmax at T into F[0..nmax]; returns exp(-T).  Inside the table: Taylor
// expansion of the top order about the nearest grid point (Horner form), then
// the downward recursion.  Beyond it erf(sqrt T) = 1 to double precision, so
// F_0 = sqrt(pi / T) / 2, then the upward recursion.
__device__ __forceinline__ double boys_eval(const double *tab, double T, int nmax, double *F) {
    const double e = exp(-T);
    if (T < kBoysTMax) {
        const double ti = rint(T * kBoysInvDelta);
        const int i = (int)ti;
        const double md = fma(ti, kBoysDelta, -T);      // -(T - T_i)
        const double *row = tab + (size_t)i * kBoysCols + nmax;
        double f = __ldg(row + kBoysTaylor - 1);
#pragma unroll
        for (int k = kBoysTaylor - 1; k > 0; --k) f = fma(f, md * c_inv_int[k], __ldg(row + k - 1));
        F[nmax] = f;
        const double t2 = T + T;
        for (int n = nmax - 1; n >= 0; --n) {
            f = fma(t2, f, e) * c_inv_odd[n];
            F[n] = f;
        }
    } else {
        double f = kHalfSqrtPi * rsqrt(T);
        const double inv2t = 0.5 / T;
        F[0] = f;
        for (int n = 0; n < nmax; ++n) {
            f = fma(c_odd[n], f, -e) * inv2t;
            F[n + 1] = f;
        }
    }
    return e;
}

// Compensated FP32 pair arithmetic.  The intrinsics keep the compiler from
// fusing the rounded product into the following sum.
__device__ __forceinline__ float2 df_split(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// The same split by integer operations on the bits (no FP64 instruction):
// hi = the top 24 significand bits of x, lo = the remaining 29 bits rounded to
// FP32.  Magnitudes outside [2^-70, 2^120) take the FP64 route.
__device__ __forceinline__ float2 df_split_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    const int e = (int)((hi32 >> 20) & 0x7FF);
    if (e < 1023 - 70 || e >= 1023 + 120) return df_split(x);
    const unsigned sign = hi32 & 0x80000000u;
    const float h = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((hi32 & 0xFFFFFu) << 3) |
                                    (lo32 >> 29));
    const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);   // 2^(e - 1075) >= 2^-122
    const float l = __fmul_rn(__uint2float_rn(lo32 & 0x1FFFFFFFu), scale);
    return make_float2(h, __uint_as_float(__float_as_uint(l) | sign));
}

// (ah, al) += sign * a * b: exact product error of the high parts plus the
// cross terms, then the two-sum of the high parts.
template <bool NEG>
__device__ __forceinline__ void df_madd(float2 a, float2 b, float &ah, float &al) {
    float p = __fmul_rn(a.x, b.x);
    float pe = __fmaf_rn(a.x, b.x, -p);
    pe = __fmaf_rn(a.x, b.y, pe);
    pe = __fmaf_rn(a.y, b.x, pe);
    if (NEG) { p = -p; pe = -pe; }
    const float t = __fadd_rn(ah, p);
    const float bv = __fsub_rn(t, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    ah = t;
    al = __fadd_rn(al, __fadd_rn(err, pe));
}

// x a + cf c in compensated FP32 pairs, renormalised (one Hermite recursion step).
__device__ __forceinline__ float2 df_rec(float2 x, float2 a, float cf, float2 c) {
    const float p1 = __fmul_rn(x.x, a.x);
    float e1 = __fmaf_rn(x.x, a.x, -p1);
    e1 = __fmaf_rn(x.x, a.y, e1);
    e1 = __fmaf_rn(x.y, a.x, e1);
    const float p2 = __fmul_rn(cf, c.x);
    float e2 = __fmaf_rn(cf, c.x, -p2);
    e2 = __fmaf_rn(cf, c.y, e2);
    const float t = __fadd_rn(p1, p2);
    const float bv = __fsub_rn(t, p1);
    const float err = __fadd_rn(__fsub_rn(p1, __fsub_rn(t, bv)), __fsub_rn(p2, bv));
    const float lo = __fadd_rn(err, __fadd_rn(e1, e2));
    const float hi = __fadd_rn(t, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t)));
}

__global__ void split_pairs_kernel(const double *E, long long n, float2 *E2, float *E1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 v = df_split(E[i]);
        E2[i] = v;
        E1[i] = v.x;
    }
}

// Doubles of one primitive quartet's header: X_PQ (3), R^n_000 of the Coulomb
// tensor (n = 0..L) and, for the gauge kernel, of the r12 tensor (n = 0..L+2).
__host__ __device__ inline int header_len(int L, bool gauge) { return gauge ? 2 * L + 7 : L + 4; }
// Doubles per primitive quartet: header, then the recursion's two buffers per
// tensor -- even auxiliary orders (order 0 ends there: nherm(L) entries) and
// odd orders (the largest is order 1: nherm(L - 1) entries); the r12 tensor of
// the gauge kernel has top order L + 2.
__host__ __device__ inline int odd_len(int Ltop) { return Ltop >= 1 ? nherm(Ltop - 1) : 0; }
__host__ __device__ inline int quartet_len(int L, bool gauge) {
    return header_len(L, gauge) + nherm(L) + odd_len(L) + (gauge ? nherm(L + 2) + odd_len(L + 2) : 0);
}

template <bool GAUGE, bool DF>
__device__ __forceinline__ void quartet_header(const double *boys, const PrimPairDev *pa, const PrimPairDev *pc,
                                               int L, double *hd) {
    const double p = pa->p, q = pc->p, s = p + q;
    const double X = pa->P[0] - pc->P[0], Y = pa->P[1] - pc->P[1], Z = pa->P[2] - pc->P[2];
    const double inv_s = 1.0 / s;
    const double rho = p * q * inv_s;
    const double T = rho * fma(X, X, fma(Y, Y, Z * Z));
    hd[0] = X;
    hd[1] = Y;
    hd[2] = Z;
    const double sq = sqrt(s);
    const double d = pa->inv_p * pc->inv_p * inv_s * sq;      // 1 / (p q sqrt(p + q))
    const double m2r = -2.0 * rho;
    double fC = kTwoPi52 * d;
    if (!GAUGE) {
        double *F = hd + 3;
        boys_eval(boys, T, L, F);
        for (int n = 0; n <= L; ++n) {
            F[n] *= fC;
            fC *= m2r;
        }
    } else {
        double *RC = hd + 3, *RR = hd + 4 + L;
        const double e = boys_eval(boys, T, L + 2, RR);
        double fR = kPi52 * s * sq * d * d;
        double prev = -fma(T + T, RR[0], e);            // F_{-1}
        for (int n = 0; n <= L + 2; ++n) {
            const double cur = RR[n];
            if (n <= L) {
                RC[n] = cur * fC;
                fC *= m2r;
            }
            RR[n] = (cur - prev) * fR;
            fR *= m2r;
            prev = cur;
        }
    }
    if (DF) {       // the recursion runs in compensated FP32 pairs: X_PQ and R^n_000 as (hi, lo)
        float2 *h2 = reinterpret_cast<float2 *>(hd);
        const int len = header_len(L, GAUGE);
        for (int i = 0; i < len; ++i) h2[i] = df_split_bits(hd[i]);
    }
}

// ---------------------------------------------------------------------------
// FP32-pair arithmetic (x = hi + lo, ~2^-47 relative per operation) for the
// header of the compensated-FP32 integrals: error-free product and two-sum,
// renormalised.  The intrinsics keep the compiler from contracting the
// rounded operations.
__device__ __forceinline__ float2 pr_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bv = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bv)), __fsub_rn(b.x, bv));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float t = __fadd_rn(s, e);
    return make_float2(t, __fsub_rn(e, __fsub_rn(t, s)));
}
__device__ __forceinline__ float2 pr_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 pr_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float t = __fadd_rn(p, e);
    return make_float2(t, __fsub_rn(e, __fsub_rn(t, p)));
}
// times a power of two (exact)
__device__ __forceinline__ float2 pr_pow2(float2 a, float f) { return make_float2(a.x * f, a.y * f); }
// 1/a: the FP32 reciprocal y and one Newton step y + y (1 - a y), the residual in pairs
__device__ __forceinline__ float2 pr_rcp(float2 a) {
    const float y = __frcp_rn(a.x);
    const float2 r = pr_add(make_float2(1.f, 0.f), pr_neg(pr_mul(a, make_float2(y, 0.f))));
    return pr_add(make_float2(y, 0.f), make_float2(__fmul_rn(y, r.x), 0.f));
}
// sqrt(a): the FP32 root y and one Newton step y + (a - y^2) / (2 y)
__device__ __forceinline__ float2 pr_sqrt(float2 a) {
    const float y = __fsqrt_rn(a.x);
    const float2 r = pr_add(a, pr_neg(pr_mul(make_float2(y, 0.f), make_float2(y, 0.f))));
    return pr_add(make_float2(y, 0.f), make_float2(__fdiv_rn(r.x, y + y), 0.f));
}
__host__ __device__ constexpr float2 pair_const(double x) { return float2{(float)x, (float)(x - (double)(float)x)}; }
__constant__ float2 c_inv_int_p[8] = {pair_const(0.0),       pair_const(1.0),       pair_const(1.0 / 2),
                                      pair_const(1.0 / 3),   pair_const(1.0 / 4),   pair_const(1.0 / 5),
                                      pair_const(1.0 / 6),   pair_const(1.0 / 7)};
__constant__ float2 c_inv_odd_p[16] = {
    pair_const(1.0),      pair_const(1.0 / 3),  pair_const(1.0 / 5),  pair_const(1.0 / 7),
    pair_const(1.0 / 9),  pair_const(1.0 / 11), pair_const(1.0 / 13), pair_const(1.0 / 15),
    pair_const(1.0 / 17), pair_const(1.0 / 19), pair_const(1.0 / 21), pair_const(1.0 / 23),
    pair_const(1.0 / 25), pair_const(1.0 / 27), pair_const(1.0 / 29), pair_const(1.0 / 31)};

// F_0..F_nmax at T (a pair) into F[0..nmax] as pairs; returns exp(-T).  Inside
// the table: Taylor expansion of the top order about the nearest grid point
// T_i, exp(-T) = exp(-T_i) exp(T_i - T) (|T_i - T| <= 0.025, eight terms), then
// the downward recursion; beyond it F_0 = sqrt(pi / T) / 2 and the upward
// recursion (exp(-T) < 3e-16 F_0 there, so its FP32 value suffices).
__device__ __forceinline__ float2 boys_eval_pairs(const BoysTables &bt, float2 T, int nmax, float2 *F) {
    if (T.x < (float)kBoysTMax) {
        const int i = min((int)rintf(T.x * (float)kBoysInvDelta), kBoysGrid - 1);
        const float2 md = pr_add(bt.t_pair[i], pr_neg(T));        // T_i - T
        const float2 *row = bt.pair + (size_t)i * kBoysCols + nmax;
        float2 f = row[kBoysTaylor - 1];
#pragma unroll
        for (int k = kBoysTaylor - 1; k > 0; --k) f = pr_add(pr_mul(f, pr_mul(md, c_inv_int_p[k])), row[k - 1]);
        F[nmax] = f;
        float2 em = make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 7; k > 0; --k) em = pr_add(make_float2(1.f, 0.f), pr_mul(em, pr_mul(md, c_inv_int_p[k])));
        const float2 e = pr_mul(bt.exp_pair[i], em);
        const float2 t2 = pr_pow2(T, 2.f);
        for (int n = nmax - 1; n >= 0; --n) {
            f = pr_mul(pr_add(pr_mul(t2, f), e), c_inv_odd_p[n]);
            F[n] = f;
        }
        return e;
    }
    const float2 e = make_float2(expf(-T.x), 0.f);
    float2 f = pr_mul(pair_const(kHalfSqrtPi), pr_rcp(pr_sqrt(T)));
    const float2 inv2t = pr_pow2(pr_rcp(T), 0.5f);
    F[0] = f;
    for (int n = 0; n < nmax; ++n) {
        f = pr_mul(pr_add(pr_mul(f, make_float2((float)(2 * n + 1), 0.f)), pr_neg(e)), inv2t);
        F[n + 1] = f;
    }
    return e;
}

// Header of a primitive quartet whose integrals run in compensated FP32 pairs:
// the same quantities as quartet_header<GAUGE, true> computed in FP32 pairs
// (X_PQ and p + q from FP64 sums, the rest in pairs), so the FP64 pipe does four
// additions per quartet instead of the whole header.  Layout as quartet_header.
template <bool GAUGE>
__device__ __forceinline__ void quartet_header_pairs(const double *boys, const PrimPairDev *pa, const PrimPairDev *pc,
                                                     int L, double *hd) {
    float2 *h2 = reinterpret_cast<float2 *>(hd);
    const BoysTables bt = boys_tables(boys);
    const float2 p = df_split_bits(pa->p), q = df_split_bits(pc->p);
    const float2 s = df_split_bits(pa->p + pc->p);
    const float2 X = df_split_bits(pa->P[0] - pc->P[0]), Y = df_split_bits(pa->P[1] - pc->P[1]),
                 Z = df_split_bits(pa->P[2] - pc->P[2]);
    const float2 inv_s = pr_rcp(s);
    const float2 rho = pr_mul(pr_mul(p, q), inv_s);
    const float2 T = pr_mul(rho, pr_add(pr_add(pr_mul(X, X), pr_mul(Y, Y)), pr_mul(Z, Z)));
    h2[0] = X;
    h2[1] = Y;
    h2[2] = Z;
    const float2 sq = pr_sqrt(s);
    const float2 d = pr_mul(pr_mul(pr_mul(df_split_bits(pa->inv_p), df_split_bits(pc->inv_p)), inv_s), sq);
    const float2 m2r = pr_pow2(rho, -2.f);
    float2 fC = pr_mul(pair_const(kTwoPi52), d);
    if (!GAUGE) {
        float2 *F = h2 + 3;
        boys_eval_pairs(bt, T, L, F);
        for (int n = 0; n <= L; ++n) {
            F[n] = pr_mul(F[n], fC);
            fC = pr_mul(fC, m2r);
        }
    } else {
        float2 *RC = h2 + 3, *RR = h2 + 4 + L;
        const float2 e = boys_eval_pairs(bt, T, L + 2, RR);
        float2 fR = pr_mul(pr_mul(pr_mul(pair_const(kPi52), s), sq), pr_mul(d, d));
        float2 prev = pr_neg(pr_add(pr_mul(pr_pow2(T, 2.f), RR[0]), e));     // F_{-1}
        for (int n = 0; n <= L + 2; ++n) {
            const float2 cur = RR[n];
            if (n <= L) {
                RC[n] = pr_mul(cur, fC);
                fC = pr_mul(fC, m2r);
            }
            RR[n] = pr_mul(pr_add(cur, pr_neg(prev)), fR);
            fR = pr_mul(fR, m2r);
            prev = cur;
        }
    }
}

// Header of a primitive quartet whose integrals run in plain FP32 (only the
// high parts are read): the geometry -- X_PQ, 1/(p+q), rho and T = rho |PQ|^2
// -- in FP64, so that T keeps its absolute accuracy (the Boys values are
// sensitive to it), and the Boys values, exp(-T) and the prefactors in FP32
// from the table's FP32 copy (the FP64 Boys evaluation would hold the FP64
// pipe for most of the header).  Layout as quartet_header, as (value, 0) pairs.
__constant__ float c_inv_int_f[8] = {0.f, 1.f, 1.f / 2, 1.f / 3, 1.f / 4, 1.f / 5, 1.f / 6, 1.f / 7};
__constant__ float c_odd_f[16] = {1, 3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31};
__constant__ float c_inv_odd_f[16] = {1.f,      1.f / 3,  1.f / 5,  1.f / 7,  1.f / 9,  1.f / 11,
                                      1.f / 13, 1.f / 15, 1.f / 17, 1.f / 19, 1.f / 21, 1.f / 23,
                                      1.f / 25, 1.f / 27, 1.f / 29, 1.f / 31};

// F_0..F_nmax at T into F[0..nmax].x (FP32; Taylor offset from the FP64 T);
// returns exp(-T).
__device__ __forceinline__ float boys_eval_f32(const float *tab, double T, int nmax, float2 *F) {
    const float Tf = (float)T;
    const float e = expf(-Tf);
    if (T < kBoysTMax) {
        const double ti = rint(T * kBoysInvDelta);
        const float md = (float)fma(ti, kBoysDelta, -T);       // -(T - T_i), exact to FP32 rounding
        const float *row = tab + (size_t)(int)ti * kBoysCols + nmax;
        float f = __ldg(row + kBoysTaylor - 1);
#pragma unroll
        for (int k = kBoysTaylor - 1; k > 0; --k) f = fmaf(f, md * c_inv_int_f[k], __ldg(row + k - 1));
        F[nmax] = make_float2(f, 0.f);
        const float t2 = Tf + Tf;
        for (int n = nmax - 1; n >= 0; --n) {
            f = fmaf(t2, f, e) * c_inv_odd_f[n];
            F[n] = make_float2(f, 0.f);
        }
    } else {
        float f = (float)kHalfSqrtPi * rsqrtf(Tf);
        const float inv2t = 0.5f / Tf;
        F[0] = make_float2(f, 0.f);
        for (int n = 0; n < nmax; ++n) {
            f = fmaf(c_odd_f[n], f, -e) * inv2t;
            F[n + 1] = make_float2(f, 0.f);
        }
    }
    return e;
}

template <bool GAUGE>
__device__ __forceinline__ void quartet_header_f32(const double *boys, const PrimPairDev *pa, const PrimPairDev *pc,
                                                   int L, double *hd) {
    float2 *h2 = reinterpret_cast<float2 *>(hd);
    const float *boysf = boys_tables(boys).f32;
    const double p = pa->p, q = pc->p, s = p + q;
    const double X = pa->P[0] - pc->P[0], Y = pa->P[1] - pc->P[1], Z = pa->P[2] - pc->P[2];
    const double inv_s = 1.0 / s;
    const double rho = p * q * inv_s;
    const double T = rho * fma(X, X, fma(Y, Y, Z * Z));
    h2[0] = make_float2((float)X, 0.f);
    h2[1] = make_float2((float)Y, 0.f);
    h2[2] = make_float2((float)Z, 0.f);
    const float sf = (float)s;
    const float d = (float)pa->inv_p * (float)pc->inv_p * (float)inv_s * sqrtf(sf);    // 1 / (p q sqrt(p + q))
    const float m2r = (float)(-2.0 * rho);
    float fC = (float)kTwoPi52 * d;
    if (!GAUGE) {
        float2 *F = h2 + 3;
        boys_eval_f32(boysf, T, L, F);
        for (int n = 0; n <= L; ++n) {
            F[n].x *= fC;
            fC *= m2r;
        }
    } else {
        float2 *RC = h2 + 3, *RR = h2 + 4 + L;
        const float e = boys_eval_f32(boysf, T, L + 2, RR);
        const float Tf = (float)T;
        float fR = (float)kPi52 * sf * sqrtf(sf) * d * d;
        float prev = -fmaf(Tf + Tf, RR[0].x, e);                 // F_{-1}
        for (int n = 0; n <= L + 2; ++n) {
            const float cur = RR[n].x;
            if (n <= L) {
                RC[n] = make_float2(cur * fC, 0.f);
                fC *= m2r;
            }
            RR[n] = make_float2((cur - prev) * fR, 0.f);
            fR *= m2r;
            prev = cur;
        }
    }
}

}  // namespace

// Shared-memory plan (class maxima); plan_smem() gives its size.
struct Plan {
    int NC;          // 1 Coulomb, 7 gauge
    int ach, cch;    // chunk of outer / inner function pairs
    int nhMax;       // nherm(max Lab)
    int LtC, LtR;    // top Hermite orders of the Coulomb and r12 tensors (LtR < 0: none)
    int nTab;        // Hermite triples tabulated: nherm(top order)
    int maxnpp;      // primitive pairs of a shell pair
    int threads;
    long long pool;  // doubles shared by T, quartet headers and the R tensors
};

struct BlockSmem {
    double *G, *P, *cf;
    long long *eX, *eY;
    int *trip, *src;
};

size_t plan_smem(const Plan &p) {
    return ((size_t)p.NC * p.ach * p.cch + p.pool + p.nTab + 2 * (size_t)p.maxnpp) * sizeof(double) +
           2 * (size_t)p.nTab * sizeof(int) + 16;
}

__device__ inline BlockSmem carve(double *sm, const Plan &p) {
    BlockSmem b;
    b.G = sm; sm += (size_t)p.NC * p.ach * p.cch;
    b.P = sm; sm += p.pool;
    b.cf = sm; sm += p.nTab;
    b.eX = (long long *)sm; sm += p.maxnpp;
    b.eY = (long long *)sm; sm += p.maxnpp;
    b.trip = (int *)sm;
    b.src = b.trip + p.nTab;
    return b;
}

// Hermite triple h -> packed (t, u, v); recursion sources of R_h: direction,
// h - e_dir, h - 2 e_dir and the coefficient (component - 1) of the latter
// (also packed into bits 22..25 of the source word for the FP32-pair path).
__device__ void build_tables(const Plan &p, BlockSmem &b) {
    for (int h = threadIdx.x; h < p.nTab; h += blockDim.x) {
        int t, u, v;
        htrip_d(h, t, u, v);
        b.trip[h] = t | (u << 8) | (v << 16);
        int dir, c;
        if (t > 0) { dir = 0; c = t; }
        else if (u > 0) { dir = 1; c = u; }
        else { dir = 2; c = v; }
        int i1 = 0, i2 = 0;
        if (h > 0) {
            const int dt = dir == 0, du = dir == 1, dv = dir == 2;
            i1 = hidx(t - dt, u - du, v - dv);
            if (c >= 2) i2 = hidx(t - 2 * dt, u - 2 * du, v - 2 * dv);
        }
        b.src[h] = dir | (i1 << 2) | (i2 << 12) | ((c >= 2 ? c - 1 : 0) << 22);
        b.cf[h] = c >= 2 ? (double)(c - 1) : 0.0;
    }
    __syncthreads();
}

// Rows of T per outer primitive pair: the Hermite triples h of X for the
// Coulomb tensor and, for the gauge kernel, the triples g with 2 <= |g| <= Lx+2
// of the r12 tensor (g = h + e_I + e_J covers all six second derivatives).
__host__ __device__ inline int t_rows(int Lx, bool gauge) { return nherm(Lx) + (gauge ? nherm(Lx + 2) - 4 : 0); }

// FP64 multiply-adds of the contraction of a shell quartet with X outer: the
// ket pass (T rows x inner function pairs x inner Hermite terms per primitive
// quartet) plus the bra pass (components x function pairs x outer Hermite
// terms per outer primitive pair).
__host__ __device__ inline double orient_cost(const PairDev &X, const PairDev &Y, bool gauge) {
    const double nhx = nherm(X.Lab), nhy = nherm(Y.Lab);
    return (double)X.npp * Y.npp * t_rows(X.Lab, gauge) * Y.nfp * nhy +
           (double)X.npp * X.nfp * Y.nfp * nhx * (gauge ? 7 : 1);
}

// acc += sign * sum_{h' of orders n0, n0+2, ...} sum_kl R_{kl}[h + h'] E^{kl}[h'][y],
// sign = -1 (NEG) for the odd orders.
template <bool NEG>
__device__ __forceinline__ void ket_orders(int n0, int Ly, int tx, int ux, int vx, const int *trip,
                                           const double *Rq, int nr, const double *ey, int nfpY,
                                           const long long *eoff, int nk, double &acc) {
    for (int n = n0; n <= Ly; n += 2) {
        const int hb = n ? nherm(n - 1) : 0, he = nherm(n);
        for (int hp = hb; hp < he; ++hp) {
            const int tq = trip[hp];
            const int T0 = tx + (tq & 255), U0 = ux + ((tq >> 8) & 255), V0 = vx + (tq >> 16);
            const int s = T0 + U0 + V0, w = U0 + V0;
            const int i0 = s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + V0;
            const double *e = ey + (size_t)hp * nfpY;
            double a = acc;
            for (int kl = 0; kl < nk; ++kl) {
                const double r = Rq[kl * nr + i0];
                const double ev = __ldg(e + eoff[kl]);
                a = NEG ? fma(-r, ev, a) : fma(r, ev, a);
            }
            acc = a;
        }
    }
}

// The same in compensated FP32 pairs (R, E and the accumulator as hi + lo).
template <bool NEG>
__device__ __forceinline__ void ket_orders_df(int n0, int Ly, int tx, int ux, int vx, const int *trip,
                                              const float2 *Rq, int nr, const float2 *ey, int nfpY,
                                              long long sE, int nk, float &ah, float &al) {
    for (int n = n0; n <= Ly; n += 2) {
        const int hb = n ? nherm(n - 1) : 0, he = nherm(n);
        for (int hp = hb; hp < he; ++hp) {
            const int tq = trip[hp];
            const int T0 = tx + (tq & 255), U0 = ux + ((tq >> 8) & 255), V0 = vx + (tq >> 16);
            const int s = T0 + U0 + V0, w = U0 + V0;
            const int i0 = s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + V0;
            const float2 *e = ey + (size_t)hp * nfpY;
            const float2 *rk = Rq + i0;
#pragma unroll 4
            for (int kl = 0; kl < nk; ++kl) {
                df_madd<NEG>(*rk, __ldg(e), ah, al);
                rk += nr;
                e += sE;
            }
        }
    }
}

// The same in plain FP32 (the high parts of R and E): quartets whose error
// bound the host has admitted to the FP32 budget.
template <bool NEG>
__device__ __forceinline__ void ket_orders_f32(int n0, int Ly, int tx, int ux, int vx, const int *trip,
                                               const float2 *Rq, int nr, const float *ey, int nfpY,
                                               long long sE, int nk, float &acc) {
    for (int n = n0; n <= Ly; n += 2) {
        const int hb = n ? nherm(n - 1) : 0, he = nherm(n);
        for (int hp = hb; hp < he; ++hp) {
            const int tq = trip[hp];
            const int T0 = tx + (tq & 255), U0 = ux + ((tq >> 8) & 255), V0 = vx + (tq >> 16);
            const int s = T0 + U0 + V0, w = U0 + V0;
            const int i0 = s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + V0;
            const float *e = ey + (size_t)hp * nfpY;
            const float *rk = reinterpret_cast<const float *>(Rq + i0);
            float a = acc;
#pragma unroll 4
            for (int kl = 0; kl < nk; ++kl) {
                a = NEG ? fmaf(-*rk, __ldg(e), a) : fmaf(*rk, __ldg(e), a);
                rk += 2 * nr;
                e += sE;
            }
            acc = a;
        }
    }
}

// The same for two T rows (Hermite indices a, b) of one inner function pair:
// each E value is loaded once for both rows (the FP32 tiles wait on these loads).
template <bool NEG>
__device__ __forceinline__ void ket_orders_f32x2(int n0, int Ly, int txa, int uxa, int vxa, int txb, int uxb,
                                                 int vxb, const int *trip, const float2 *Rq, int nr,
                                                 const float *ey, int nfpY, long long sE, int nk, float &acca,
                                                 float &accb) {
    for (int n = n0; n <= Ly; n += 2) {
        const int hb = n ? nherm(n - 1) : 0, he = nherm(n);
        for (int hp = hb; hp < he; ++hp) {
            const int tq = trip[hp];
            const int tp = tq & 255, up = (tq >> 8) & 255, vp = tq >> 16;
            const int Ta = txa + tp, Ua = uxa + up, Va = vxa + vp, sa = Ta + Ua + Va, wa = Ua + Va;
            const int Tb = txb + tp, Ub = uxb + up, Vb = vxb + vp, sb = Tb + Ub + Vb, wb = Ub + Vb;
            const int ia = sa * (sa + 1) * (sa + 2) / 6 + wa * (wa + 1) / 2 + Va;
            const int ib = sb * (sb + 1) * (sb + 2) / 6 + wb * (wb + 1) / 2 + Vb;
            const float *e = ey + (size_t)hp * nfpY;
            const float *ra = reinterpret_cast<const float *>(Rq + ia);
            const float *rb = reinterpret_cast<const float *>(Rq + ib);
            float a = acca, b2 = accb;
#pragma unroll 4
            for (int kl = 0; kl < nk; ++kl) {
                const float ev = __ldg(e);
                a = NEG ? fmaf(-*ra, ev, a) : fmaf(*ra, ev, a);
                b2 = NEG ? fmaf(-*rb, ev, b2) : fmaf(*rb, ev, b2);
                ra += 2 * nr;
                rb += 2 * nr;
                e += sE;
            }
            acca = a;
            accb = b2;
        }
    }
}

// The same for two adjacent inner function pairs y, y + 1 at once (the second
// when has1): R and the primitive-pair offsets are loaded once for both, and
// the two accumulator chains are independent (gauge kernel, whose larger
// plan leaves registers for the second chain).
template <bool NEG>
__device__ __forceinline__ void ket_orders_df2(int n0, int Ly, int tx, int ux, int vx, const int *trip,
                                               const float2 *Rq, int nr, const float2 *ey, int nfpY,
                                               long long sE, int nk, bool has1, float &ah0, float &al0,
                                               float &ah1, float &al1) {
    for (int n = n0; n <= Ly; n += 2) {
        const int hb = n ? nherm(n - 1) : 0, he = nherm(n);
        for (int hp = hb; hp < he; ++hp) {
            const int tq = trip[hp];
            const int T0 = tx + (tq & 255), U0 = ux + ((tq >> 8) & 255), V0 = vx + (tq >> 16);
            const int s = T0 + U0 + V0, w = U0 + V0;
            const int i0 = s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + V0;
            const float2 *e = ey + (size_t)hp * nfpY;
            const float2 *rk = Rq + i0;
            if (has1) {
#pragma unroll 2
                for (int kl = 0; kl < nk; ++kl) {
                    const float2 r = *rk;
                    const float2 e0 = __ldg(e), e1 = __ldg(e + 1);
                    df_madd<NEG>(r, e0, ah0, al0);
                    df_madd<NEG>(r, e1, ah1, al1);
                    rk += nr;
                    e += sE;
                }
            } else {
                for (int kl = 0; kl < nk; ++kl) {
                    df_madd<NEG>(*rk, __ldg(e), ah0, al0);
                    rk += nr;
                    e += sE;
                }
            }
        }
    }
}

// Register tile of the ket pass: TH rows of T (Hermite rows of the outer pair,
// each with its own R tensor base and stride: the Coulomb tensor, or for the
// gauge kernel the r12 tensor) times TY adjacent inner function pairs, for one
// outer primitive pair:
//   acc[r][c] += sum_{kl} sum_{h'} (-1)^{|h'|} R_kl[h_r + h'] E^kl[h'][y_c].
// Each E value is loaded once for the TH rows and each R value once for the TY
// columns, and the TH x TY accumulators are independent chains.  DF: compensated
// FP32 pairs (R, E and the accumulators as hi + lo); else plain FP32 (the high
// parts).  Rows and columns past the chunk are clamped by the caller (their sums
// are discarded).
template <int TH, int TY, bool DF>
struct KetTile {
    float ah[TH][TY], al[TH][TY];
};

template <int TH, int TY, bool DF, bool NEG>
__device__ __forceinline__ void ket_tile_orders(int n0, int Ly, const int (&rs)[TH], const int (&rw)[TH],
                                                const int (&rv)[TH], const float2 *const (&Rb)[TH],
                                                const int (&nr)[TH], const int *trip, const void *eyv, int nfpY,
                                                long long sE, int nk, const int (&yo)[TY], KetTile<TH, TY, DF> &t) {
    for (int n = n0; n <= Ly; n += 2) {
        const int hb = n ? nherm(n - 1) : 0, he = nherm(n);
        for (int hp = hb; hp < he; ++hp) {
            const int tq = trip[hp];
            const int up = (tq >> 8) & 255, vp = tq >> 16, wp = up + vp, sp = (tq & 255) + wp;
            const float2 *rp[TH];
#pragma unroll
            for (int r = 0; r < TH; ++r) {
                const int s = rs[r] + sp, w = rw[r] + wp;
                rp[r] = Rb[r] + (s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + rv[r] + vp);
            }
            if constexpr (DF) {
                const float2 *e = reinterpret_cast<const float2 *>(eyv) + (size_t)hp * nfpY;
#pragma unroll 2
                for (int kl = 0; kl < nk; ++kl) {
                    float2 ev[TY];
#pragma unroll
                    for (int c = 0; c < TY; ++c) ev[c] = __ldg(e + yo[c]);
#pragma unroll
                    for (int r = 0; r < TH; ++r) {
                        const float2 rvv = *rp[r];
                        rp[r] += nr[r];
#pragma unroll
                        for (int c = 0; c < TY; ++c) df_madd<NEG>(rvv, ev[c], t.ah[r][c], t.al[r][c]);
                    }
                    e += sE;
                }
            } else {
                const float *e = reinterpret_cast<const float *>(eyv) + (size_t)hp * nfpY;
#pragma unroll 3
                for (int kl = 0; kl < nk; ++kl) {
                    float ev[TY];
#pragma unroll
                    for (int c = 0; c < TY; ++c) ev[c] = __ldg(e + yo[c]);
#pragma unroll
                    for (int r = 0; r < TH; ++r) {
                        const float rvv = rp[r]->x;
                        rp[r] += nr[r];
#pragma unroll
                        for (int c = 0; c < TY; ++c)
                            t.ah[r][c] = NEG ? fmaf(-rvv, ev[c], t.ah[r][c]) : fmaf(rvv, ev[c], t.ah[r][c]);
                    }
                    e += sE;
                }
            }
        }
    }
}

// The tiled ket pass over every (outer primitive pair, row block, column
// block) of a chunk: T[ij][hh][y] (float2 slots) += the sums above.  Rows hh <
// nhx use the Coulomb tensor RC (Hermite index hh); for the gauge kernel rows
// hh >= nhx use the r12 tensor RR (Hermite index hh - nhx + 4).
template <int TH, int TY, bool DF, bool GAUGE>
__device__ __forceinline__ void ket_pass_tiled(int nij, int nT, int nhx, int ych, int Ly, const int *trip,
                                               float2 *T, int tsz, const float2 *RC, int nrC, const float2 *RR,
                                               int nrR, int nk, const void *ey0, int nfpY, long long sE) {
    const int nHB = (nT + TH - 1) / TH, nYB = (ych + TY - 1) / TY;
    for (int it = threadIdx.x; it < nij * nHB * nYB; it += blockDim.x) {
        const int ijl = it / (nHB * nYB);
        const int rem = it - ijl * nHB * nYB;
        const int hb = rem / nYB, yb = rem - hb * nYB;
        const int h0 = hb * TH, y0 = yb * TY;
        int rs[TH], rw[TH], rv[TH], nr[TH], hh[TH];
        const float2 *Rb[TH];
#pragma unroll
        for (int r = 0; r < TH; ++r) {
            hh[r] = min(h0 + r, nT - 1);
            const bool r12 = GAUGE && hh[r] >= nhx;
            const int tr = trip[r12 ? hh[r] - nhx + 4 : hh[r]];
            const int u = (tr >> 8) & 255, v = tr >> 16;
            rv[r] = v;
            rw[r] = u + v;
            rs[r] = (tr & 255) + u + v;
            nr[r] = r12 ? nrR : nrC;
            Rb[r] = r12 ? RR + (size_t)ijl * nk * nrR : RC + (size_t)ijl * nk * nrC;
        }
        int yo[TY];
#pragma unroll
        for (int c = 0; c < TY; ++c) yo[c] = min(y0 + c, ych - 1) - y0;
        KetTile<TH, TY, DF> t;
        float2 *Tq = T + (size_t)ijl * tsz + y0;
#pragma unroll
        for (int r = 0; r < TH; ++r)
#pragma unroll
            for (int c = 0; c < TY; ++c) {
                const float2 v = Tq[(size_t)hh[r] * ych + yo[c]];
                t.ah[r][c] = v.x;
                t.al[r][c] = DF ? v.y : 0.f;
            }
        const void *ey = DF ? (const void *)(reinterpret_cast<const float2 *>(ey0) + y0)
                            : (const void *)(reinterpret_cast<const float *>(ey0) + y0);
        ket_tile_orders<TH, TY, DF, false>(0, Ly, rs, rw, rv, Rb, nr, trip, ey, nfpY, sE, nk, yo, t);
        ket_tile_orders<TH, TY, DF, true>(1, Ly, rs, rw, rv, Rb, nr, trip, ey, nfpY, sE, nk, yo, t);
#pragma unroll
        for (int r = 0; r < TH; ++r)
#pragma unroll
            for (int c = 0; c < TY; ++c)
                if (h0 + r < nT && y0 + c < ych) Tq[(size_t)(h0 + r) * ych + c] = make_float2(t.ah[r][c], DF ? t.al[r][c] : 0.f);
    }
}

// One chunk (x in [x0,x1) of X, y in [y0,y1) of Y) of the block (X|Y);
// results in b.G[comp][x][y].  NC = 1 (Coulomb) or 7 (gauge: [0] Coulomb,
// [1..6] (xy|d_I d_J r|zw) for IJ = xx,xy,xz,yy,yz,zz).
template <bool GAUGE, bool DF, bool F32 = false>
__device__ void block_chunk(const PrimPairDev *pp, const double *E, const float2 *E2, const float *E1,
                            const double *boys,
                            const PairDev &X, const PairDev &Y, int x0, int x1, int y0, int y1, const Plan &pl,
                            BlockSmem &b) {
    constexpr int NC = GAUGE ? 7 : 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Lx = X.Lab, Ly = Y.Lab;
    const int nhx = nherm(Lx);
    const int L = Lx + Ly, Lr = L + 2, Ltop = GAUGE ? Lr : L;
    const int nrC = nherm(L), nrR = GAUGE ? nherm(Lr) : 0;
    const int hs = header_len(L, GAUGE), perq = quartet_len(L, GAUGE);
    const int xch = x1 - x0, ych = y1 - y0;
    const int nT = t_rows(Lx, GAUGE);                   // T rows per outer primitive pair
    // the E matrices of a pair's primitive pairs are stored back to back,
    // nherm(L) x nfp each: inner primitive kl starts kl sE past the first (the
    // compensated-FP32 ket pass walks them by this stride)
    const long long sE = (long long)Y.nfp * nherm(Ly);
    const int tsz = nT * ych;                           // T doubles per outer primitive pair

    // primitive grouping: nij outer pairs x nkl inner pairs at a time
    int nijMax, nkl;
    if ((long long)Y.npp * perq + tsz <= pl.pool) {
        nkl = Y.npp;
        nijMax = (int)min((long long)X.npp, pl.pool / ((long long)Y.npp * perq + tsz));
    } else {
        nkl = (int)((pl.pool - tsz) / perq);
        nijMax = 1;
    }
    nijMax = max(nijMax, 1);
    nkl = max(nkl, 1);
    double *T = b.P;
    double *H = T + (size_t)nijMax * tsz;
    const int nqMax = nijMax * nkl;
    // order-0 (and even-order) buffers RC, RR [nqMax][nrC | nrR]; odd-order buffers RC1, RR1
    const int nrC1 = odd_len(L), nrR1 = GAUGE ? odd_len(Lr) : 0;
    double *RC = H + (size_t)nqMax * hs;
    double *RC1 = RC + (size_t)nqMax * nrC;
    double *RR = RC1 + (size_t)nqMax * nrC1;
    double *RR1 = RR + (size_t)nqMax * nrR;

    for (int i = tid; i < X.npp; i += nt) b.eX[i] = pp[X.ppoff + i].eoff;
    for (int i = tid; i < Y.npp; i += nt) b.eY[i] = pp[Y.ppoff + i].eoff;
    for (int i = tid; i < NC * xch * ych; i += nt) b.G[i] = 0.0;
    __syncthreads();

    for (int i0 = 0; i0 < X.npp; i0 += nijMax) {
        const int nij = min(nijMax, X.npp - i0);
        for (int i = tid; i < nij * tsz; i += nt) T[i] = 0.0;
        for (int k0 = 0; k0 < Y.npp; k0 += nkl) {
            const int nk = min(nkl, Y.npp - k0);
            const int nq = nij * nk;
            // Boys values, prefactors and X_PQ of every primitive quartet of the group
            for (int q = tid; q < nq; q += nt) {
                const int ijl = q / nk, kl = q - ijl * nk;
                // plain-FP32 quartets of the Coulomb kernel: FP32 header; those of
                // the gauge kernel take the FP32-pair header (its r12 tensor takes
                // differences F_n - F_{n-1} that lose digits in FP32: measured 13x
                // the Coulomb kernel's error ratio with an FP32 header), of which
                // the FP32 recursion reads the high parts
                if constexpr (DF && F32 && !GAUGE)
                    quartet_header_f32<GAUGE>(boys, pp + X.ppoff + i0 + ijl, pp + Y.ppoff + k0 + kl, L, H + (size_t)q * hs);
                else if constexpr (DF)
                    quartet_header_pairs<GAUGE>(boys, pp + X.ppoff + i0 + ijl, pp + Y.ppoff + k0 + kl, L,
                                                H + (size_t)q * hs);
                else
                    quartet_header<GAUGE, false>(boys, pp + X.ppoff + i0 + ijl, pp + Y.ppoff + k0 + kl, L,
                                                 H + (size_t)q * hs);
            }
            __syncthreads();
            // Hermite recursion, one auxiliary order per pass; order 0 ends in buffer 0.
            // Each warp runs all orders of its own primitive quartets (q = warp,
            // warp + nwarps, ...), so consecutive orders need only a warp barrier;
            // one CTA barrier after the last order.
            const int nw = nt >> 5, wq = tid >> 5, lane = tid & 31;
            const int nqw = wq < nq ? (nq - wq + nw - 1) / nw : 0;
            for (int m = Ltop; m >= 0; --m) {
                const int cC = m <= L ? nherm(L - m) : 0;
                const int cR = GAUGE ? nherm(Lr - m) : 0;
                const int cnt = cC + cR;
                const int cur = m & 1, prv = cur ^ 1;
                // items (quartet of this warp, Hermite entry) of the order; for cnt >= 2
                // the quotient it / cnt by a multiply-high with ceil(2^32 / cnt) =
                // floor((2^32 - 1) / cnt) + 1 (exact while it * cnt < 2^32; here
                // it * cnt < 2^16 * 2^8); cnt == 1 (the top order) has quotient it
                const unsigned magic = cnt > 1 ? 0xFFFFFFFFu / (unsigned)cnt + 1u : 0u;
                for (int it = lane; it < nqw * cnt; it += 32) {
                    const int qi = cnt > 1 ? (int)__umulhi((unsigned)it, magic) : it;
                    const int q = wq + qi * nw;
                    const int hh = it - qi * cnt;
                    const double *hd = H + (size_t)q * hs;
                    const bool cpart = !GAUGE || hh < cC;
                    const int h = cpart ? hh : hh - cC;
                    double *dst = cpart ? (cur ? RC1 + (size_t)q * nrC1 : RC + (size_t)q * nrC)
                                        : (cur ? RR1 + (size_t)q * nrR1 : RR + (size_t)q * nrR);
                    const double *src = cpart ? (prv ? RC1 + (size_t)q * nrC1 : RC + (size_t)q * nrC)
                                              : (prv ? RR1 + (size_t)q * nrR1 : RR + (size_t)q * nrR);
                    const int i0h = cpart ? 3 + m : 4 + L + m;
                    if constexpr (DF && F32) {
                        const float2 *hd2 = reinterpret_cast<const float2 *>(hd);
                        const float2 *src2 = reinterpret_cast<const float2 *>(src);
                        float r = hd2[i0h].x;
                        if (h > 0) {
                            const int sw = b.src[h];
                            r = fmaf(hd2[sw & 3].x, src2[(sw >> 2) & 1023].x,
                                     (float)((sw >> 22) & 15) * src2[(sw >> 12) & 1023].x);
                        }
                        reinterpret_cast<float2 *>(dst)[h] = make_float2(r, 0.f);
                    } else if constexpr (DF) {
                        const float2 *hd2 = reinterpret_cast<const float2 *>(hd);
                        const float2 *src2 = reinterpret_cast<const float2 *>(src);
                        float2 r = hd2[i0h];
                        if (h > 0) {
                            const int sw = b.src[h];
                            r = df_rec(hd2[sw & 3], src2[(sw >> 2) & 1023], (float)((sw >> 22) & 15),
                                       src2[(sw >> 12) & 1023]);
                        }
                        reinterpret_cast<float2 *>(dst)[h] = r;
                    } else {
                        double r = hd[i0h];
                        if (h > 0) {
                            const int sw = b.src[h];
                            r = fma(b.cf[h], src[(sw >> 12) & 1023], hd[sw & 3] * src[(sw >> 2) & 1023]);
                        }
                        dst[h] = r;
                    }
                }
                __syncwarp();
            }
            __syncthreads();
            // T[ij][h][y] += sum_kl sum_h' (-1)^{|h'|} R[h+h'] E^{kl}[h'][y]: rows h < nhx
            // with the Coulomb tensor, then (gauge) rows g = 4.. with the r12 tensor
            if (DF && nT >= 4 && ych >= 2) {
                // register tiles: 4 T rows x 2 inner function pairs per thread
                if constexpr (DF) {
                    float2 *T2 = reinterpret_cast<float2 *>(T);
                    const float2 *RC2 = reinterpret_cast<const float2 *>(RC), *RR2 = reinterpret_cast<const float2 *>(RR);
                    const void *ey = F32 ? (const void *)(E1 + b.eY[k0] + y0) : (const void *)(E2 + b.eY[k0] + y0);
                    // plain FP32 waits on the loads: 3 inner function pairs per thread when the
                    // chunk comes in threes (the derivative functions do), so 7 loads serve 12 FMAs
                    if (F32 && ych % 3 == 0)
                        ket_pass_tiled<4, 3, false, GAUGE>(nij, nT, nhx, ych, Ly, b.trip, T2, tsz, RC2, nrC, RR2, nrR,
                                                           nk, ey, Y.nfp, sE);
                    else
                        ket_pass_tiled<4, 2, !F32, GAUGE>(nij, nT, nhx, ych, Ly, b.trip, T2, tsz, RC2, nrC, RR2, nrR,
                                                          nk, ey, Y.nfp, sE);
                }
            } else if constexpr (DF && F32 && !GAUGE) {
                // two T rows per thread sharing the E loads
                const int nT2 = (nT + 1) / 2;
                for (int it = tid; it < nij * nT2 * ych; it += nt) {
                    const int ijl = it / (nT2 * ych);
                    const int rem = it - ijl * nT2 * ych;
                    const int h0 = 2 * (rem / ych), yy = rem - (rem / ych) * ych;
                    const bool has1 = h0 + 1 < nT;
                    const int h1 = has1 ? h0 + 1 : h0;
                    const int tra = b.trip[h0], trb = b.trip[h1];
                    float2 *T2 = reinterpret_cast<float2 *>(T + (size_t)ijl * tsz + (size_t)h0 * ych + yy);
                    float acca = T2[0].x, accb = has1 ? T2[ych].x : 0.f;
                    const float2 *R2 = reinterpret_cast<const float2 *>(RC + (size_t)ijl * nk * nrC);
                    const float *ey = E1 + b.eY[k0] + (y0 + yy);
                    ket_orders_f32x2<false>(0, Ly, tra & 255, (tra >> 8) & 255, tra >> 16, trb & 255, (trb >> 8) & 255,
                                            trb >> 16, b.trip, R2, nrC, ey, Y.nfp, sE, nk, acca, accb);
                    ket_orders_f32x2<true>(1, Ly, tra & 255, (tra >> 8) & 255, tra >> 16, trb & 255, (trb >> 8) & 255,
                                           trb >> 16, b.trip, R2, nrC, ey, Y.nfp, sE, nk, acca, accb);
                    T2[0] = make_float2(acca, 0.f);
                    if (has1) T2[ych] = make_float2(accb, 0.f);
                }
            } else if constexpr (DF && F32) {
                for (int it = tid; it < nij * nT * ych; it += nt) {
                    const int ijl = it / (nT * ych);
                    const int rem = it - ijl * nT * ych;
                    const int hh = rem / ych, yy = rem - hh * ych;
                    const bool r12 = GAUGE && hh >= nhx;
                    const int h = r12 ? hh - nhx + 4 : hh;
                    const int tr = b.trip[h];
                    const int tx = tr & 255, ux = (tr >> 8) & 255, vx = tr >> 16;
                    float2 *T2 = reinterpret_cast<float2 *>(T + (size_t)ijl * tsz + (size_t)hh * ych + yy);
                    float acc = T2[0].x;
                    const float2 *R2 = reinterpret_cast<const float2 *>(r12 ? RR + (size_t)ijl * nk * nrR
                                                                            : RC + (size_t)ijl * nk * nrC);
                    const int nr = r12 ? nrR : nrC;
                    const float *ey = E1 + b.eY[k0] + (y0 + yy);
                    ket_orders_f32<false>(0, Ly, tx, ux, vx, b.trip, R2, nr, ey, Y.nfp, sE, nk, acc);
                    ket_orders_f32<true>(1, Ly, tx, ux, vx, b.trip, R2, nr, ey, Y.nfp, sE, nk, acc);
                    T2[0] = make_float2(acc, 0.f);
                }
            } else if constexpr (DF) {
                // gauge kernel: pairs of adjacent y per thread when the chunk has enough
                // of them to keep the lanes busy; single y otherwise (same sums either way)
                const int yb = (GAUGE && ych >= 8) ? 2 : 1;
                const int ych2 = (ych + yb - 1) / yb;
                for (int it = tid; it < nij * nT * ych2; it += nt) {
                    const int ijl = it / (nT * ych2);
                    const int rem = it - ijl * nT * ych2;
                    const int hh = rem / ych2, yy = yb * (rem - hh * ych2);
                    const bool has1 = yb == 2 && yy + 1 < ych;
                    const bool r12 = GAUGE && hh >= nhx;
                    const int h = r12 ? hh - nhx + 4 : hh;
                    const int tr = b.trip[h];
                    const int tx = tr & 255, ux = (tr >> 8) & 255, vx = tr >> 16;
                    float2 *T2 = reinterpret_cast<float2 *>(T + (size_t)ijl * tsz + (size_t)hh * ych + yy);
                    float ah0 = T2[0].x, al0 = T2[0].y, ah1 = 0.f, al1 = 0.f;
                    if (has1) { ah1 = T2[1].x; al1 = T2[1].y; }
                    const float2 *R2 = reinterpret_cast<const float2 *>(r12 ? RR + (size_t)ijl * nk * nrR
                                                                            : RC + (size_t)ijl * nk * nrC);
                    const int nr = r12 ? nrR : nrC;
                    const float2 *ey = E2 + b.eY[k0] + (y0 + yy);
                    if constexpr (GAUGE) {
                        ket_orders_df2<false>(0, Ly, tx, ux, vx, b.trip, R2, nr, ey, Y.nfp, sE, nk, has1, ah0,
                                              al0, ah1, al1);
                        ket_orders_df2<true>(1, Ly, tx, ux, vx, b.trip, R2, nr, ey, Y.nfp, sE, nk, has1, ah0,
                                             al0, ah1, al1);
                    } else {
                        ket_orders_df<false>(0, Ly, tx, ux, vx, b.trip, R2, nr, ey, Y.nfp, sE, nk, ah0, al0);
                        ket_orders_df<true>(1, Ly, tx, ux, vx, b.trip, R2, nr, ey, Y.nfp, sE, nk, ah0, al0);
                    }
                    T2[0] = make_float2(ah0, al0);
                    if (has1) T2[1] = make_float2(ah1, al1);
                }
            } else
            for (int it = tid; it < nij * nT * ych; it += nt) {
                const int ijl = it / (nT * ych);
                const int rem = it - ijl * nT * ych;
                const int hh = rem / ych, yy = rem - hh * ych;
                const bool r12 = GAUGE && hh >= nhx;
                const int h = r12 ? hh - nhx + 4 : hh;
                const int tr = b.trip[h];
                const int tx = tr & 255, ux = (tr >> 8) & 255, vx = tr >> 16;
                double *Tq = T + (size_t)ijl * tsz + (size_t)hh * ych + yy;
                const double *Rq = r12 ? RR + (size_t)ijl * nk * nrR : RC + (size_t)ijl * nk * nrC;
                const int nr = r12 ? nrR : nrC;
                double acc = *Tq;
                const double *ey = E + (y0 + yy);
                ket_orders<false>(0, Ly, tx, ux, vx, b.trip, Rq, nr, ey, Y.nfp, b.eY + k0, nk, acc);
                ket_orders<true>(1, Ly, tx, ux, vx, b.trip, Rq, nr, ey, Y.nfp, b.eY + k0, nk, acc);
                *Tq = acc;
            }
            // the next group's header pass touches neither T nor R, and its
            // barrier orders this pass before the recursion overwrites R
            if (k0 + nkl >= Y.npp) __syncthreads();
        }
        // G[0][x][y] += sum_{ij} sum_h E^{ij}[h][x] T[ij][h][y]; gauge: G[1+IJ] from
        // the r12 rows h + e_I + e_J (order |h| + 2) for IJ = xx, xy, xz, yy, yz, zz
        for (int it = tid; it < xch * ych; it += nt) {
            const int xx = it / ych, yy = it - xx * ych;
            double s[NC];
            float sh[NC], sl[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) { s[c] = 0.0; sh[c] = 0.f; sl[c] = 0.f; }
            for (int ijl = 0; ijl < nij; ++ijl) {
                const size_t off = (size_t)ijl * tsz + yy;
#pragma unroll 4
                for (int h = 0; h < nhx; ++h) {
                    int g[6] = {0, 0, 0, 0, 0, 0};               // r12 rows, offset by nhx - 4
                    if (GAUGE) {
                        const int tr = b.trip[h];
                        const int u = (tr >> 8) & 255, v = tr >> 16;
                        const int o = (tr & 255) + u + v, w = u + v;
                        const int b2 = (o + 2) * (o + 3) * (o + 4) / 6 + nhx - 4;
                        g[0] = b2 + w * (w + 1) / 2 + v;
                        g[1] = b2 + (w + 1) * (w + 2) / 2 + v;
                        g[2] = g[1] + 1;
                        g[3] = b2 + (w + 2) * (w + 3) / 2 + v;
                        g[4] = g[3] + 1;
                        g[5] = g[3] + 2;
                    }
                    if constexpr (DF && F32) {
                        const float *T1 = reinterpret_cast<const float *>(reinterpret_cast<const float2 *>(T) + off);
                        const float ev = __ldg(E1 + b.eX[i0 + ijl] + (x0 + xx) + (size_t)h * X.nfp);
                        sh[0] = fmaf(ev, T1[2 * (size_t)h * ych], sh[0]);
                        if (GAUGE)
#pragma unroll
                            for (int c = 1; c < NC; ++c) sh[c] = fmaf(ev, T1[2 * (size_t)g[c - 1] * ych], sh[c]);
                    } else if constexpr (DF) {
                        const float2 *T2 = reinterpret_cast<const float2 *>(T) + off;
                        const float2 ev = __ldg(E2 + b.eX[i0 + ijl] + (x0 + xx) + (size_t)h * X.nfp);
                        df_madd<false>(ev, T2[(size_t)h * ych], sh[0], sl[0]);
                        if (GAUGE)
#pragma unroll
                            for (int c = 1; c < NC; ++c) df_madd<false>(ev, T2[(size_t)g[c - 1] * ych], sh[c], sl[c]);
                    } else {
                        const double *Tq = T + off;
                        const double ev = __ldg(E + b.eX[i0 + ijl] + (x0 + xx) + (size_t)h * X.nfp);
                        s[0] = fma(ev, Tq[(size_t)h * ych], s[0]);
                        if (GAUGE)
#pragma unroll
                            for (int c = 1; c < NC; ++c) s[c] = fma(ev, Tq[(size_t)g[c - 1] * ych], s[c]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c)
                b.G[((size_t)c * xch + xx) * ych + yy] += DF ? (double)sh[c] + (double)sl[c] : s[c];
        }
        __syncthreads();
    }
}

// Screened rows as a persistent kernel: every CTA builds its tables once, then
// takes tiles (bra shell pair x range of sorted ket positions) from the shared
// counter until none are left.  A tile's parameter set comes from prms[req],
// so one launch can mix the tiles of several transformations.
template <bool GAUGE, bool DF>
__global__ void __launch_bounds__(256, 2) eri_rows_kernel(const EriParams *prms, const EriTask *tasks, int ntasks,
                                                          int *next, Plan pl) {
    extern __shared__ double sm[];
    BlockSmem b = carve(sm, pl);
    int *slot = b.src + pl.nTab;                     // in the plan's 16 spare bytes
    build_tables(pl, b);
    const int ij_of[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (;;) {
        if (threadIdx.x == 0) *slot = atomicAdd(next, 1);
        __syncthreads();
        const int t = *slot;
        __syncthreads();
        if (t >= ntasks) break;
        const EriTask tk = tasks[t];
        const EriParams &prm = prms[tk.req];
        const PairDev AB = prm.pairs[tk.bra_sp];
        for (int kp = tk.k0; kp < tk.k1; ++kp) {
            const int cd_id = prm.ket_sp[kp];
            const PairDev CD = prm.pairs[cd_id];
            const long long col = prm.ket_col[kp];
            // (CD|AB) also kept?  Then one block serves both (EriParams::sym):
            // rev writes it at (cd, ab) of W, mir into W2 for a later batch
            const bool both = prm.sym && cd_id != tk.bra_sp && prm.ket_pos[tk.bra_sp] < prm.prefix[cd_id];
            bool rev = both, mir = false;
            if (both && prm.sym == 2) {
                const int bp = prm.bra_pos[cd_id];
                if (bp < prm.b0) continue;           // its transpose came from W2 of CD's batch
                rev = bp < prm.b1;
                mir = !rev;
            }
            if (rev && cd_id < tk.bra_sp) continue;
            const long long col_rev = rev ? prm.ket_col[prm.ket_pos[tk.bra_sp]] : 0;
            // contract the orientation with the smaller cost; swapped -> G is (CD|AB)
            const bool swap = orient_cost(CD, AB, GAUGE) < orient_cost(AB, CD, GAUGE);
            const PairDev &X = swap ? CD : AB, &Y = swap ? AB : CD;
            double *W = prm.W, *Wc = prm.Wc;
            const long long ldw = prm.ldw, ldwc = prm.ldwc, row0 = prm.row0;
            const bool wc = prm.with_coulomb != 0;
            for (int x0 = 0; x0 < X.nfp; x0 += pl.ach) {
                const int x1 = min(X.nfp, x0 + pl.ach);
                for (int y0 = 0; y0 < Y.nfp; y0 += pl.cch) {
                    const int y1 = min(Y.nfp, y0 + pl.cch);
                    if constexpr (DF) {
                        if (tk.f32)
                            block_chunk<GAUGE, true, true>(prm.pp, prm.E, prm.E2, prm.E1, prm.boys, X, Y, x0, x1, y0, y1,
                                                           pl, b);
                        else
                            block_chunk<GAUGE, true, false>(prm.pp, prm.E, prm.E2, prm.E1, prm.boys, X, Y, x0, x1, y0,
                                                            y1, pl, b);
                    } else {
                        block_chunk<GAUGE, false>(prm.pp, prm.E, prm.E2, prm.E1, prm.boys, X, Y, x0, x1, y0, y1, pl, b);
                    }
                    const int xch = x1 - x0, ych = y1 - y0;
                    for (int idx = threadIdx.x; idx < xch * ych; idx += blockDim.x) {
                        const int xx = idx / ych, yy = idx - xx * ych;
                        const int a = swap ? y0 + yy : x0 + xx;      // bra function pair
                        const int c = swap ? x0 + xx : y0 + yy;      // ket function pair
                        // the block's entry into row `r`, column `k` of an output
                        // (gauge: rows (r, I), columns (k, J); K_IJ is symmetric, so the
                        // transposed entry needs no index change)
                        auto put = [&](double *Wo, long long ldo, double *Wco, long long ldco, long long r,
                                       long long k) {
                            if (!GAUGE) {
                                Wo[r * ldo + k] = b.G[idx];
                            } else {
                                const double C = b.G[idx];
                                const double *Hh = b.G + (size_t)xch * ych;
                                for (int I = 0; I < 3; ++I)
                                    for (int J = 0; J < 3; ++J) {
                                        const double h = Hh[(size_t)ij_of[I][J] * xch * ych + idx];
                                        Wo[(r * 3 + I) * ldo + k * 3 + J] = (I == J ? C : 0.0) - h;
                                    }
                                if (wc) Wco[r * ldco + k] = C;
                            }
                        };
                        put(W, ldw, Wc, ldwc, AB.rowoff + a - row0, col + c);
                        // the same integrals at (cd, ab): rows of CD, columns of AB
                        if (rev) put(W, ldw, Wc, ldwc, CD.rowoff + c - row0, col_rev + a);
                        if (mir) put(prm.W2, prm.ldw2, prm.Wc2, prm.ldwc2, CD.rowoff + c - prm.row2,
                                     prm.col2[tk.bra_sp] + a);
                    }
                    __syncthreads();
                }
            }
        }
    }
}

// Plan for a class: the largest function-pair chunk (halved while needed) such
// that the pool holds the T of one outer primitive pair plus at least eight
// primitive quartets of the highest order.  Small classes run as 128-thread
// CTAs in 56 KB, four per SM, so that a CTA waiting at a barrier leaves the
// FP64 pipe to the others; classes that do not fit take 112 KB or 200 KB.
Plan eri_plan(int maxnfp, int maxLab, int maxnpp, bool gauge) {
    struct Tier { int kb, threads; };
    const Tier tiers[3] = {{56, 128}, {112, 256}, {200, 256}};
    Plan p{};
    for (int ti = gauge ? 1 : 0; ti < 3; ++ti) {
        p.NC = gauge ? 7 : 1;
        p.nhMax = nherm(maxLab);
        p.LtC = 2 * maxLab;
        p.LtR = gauge ? p.LtC + 2 : -1;
        p.nTab = nherm(gauge ? p.LtR : p.LtC);
        p.maxnpp = maxnpp > 0 ? maxnpp : 1;
        p.threads = tiers[ti].threads;
        p.ach = p.cch = maxnfp > 0 ? maxnfp : 1;
        const long long perq = quartet_len(p.LtC, gauge);
        const long long budget = (long long)tiers[ti].kb * 1024;
        long long tsz = 0;
        for (;;) {
            p.pool = 0;
            const long long fixed = (long long)plan_smem(p);
            tsz = (long long)t_rows(maxLab, gauge) * p.cch;
            const long long pool = (budget - fixed) / (long long)sizeof(double);
            if (pool >= tsz + 8 * perq || p.ach <= 8) {
                p.pool = pool > tsz + perq ? pool : tsz + perq;
                break;
            }
            p.ach = p.cch = (p.ach + 1) / 2;
        }
        const int want = maxnfp < 32 ? maxnfp : 32;
        if ((p.ach >= want && p.pool >= tsz + 8 * perq) || ti == 2) break;
    }
    return p;
}

int eri_default_threads(const EriShape &shape, bool gauge) {
    return eri_plan(shape.maxnfp, shape.maxLab, shape.maxnpp, gauge).threads;
}

namespace {
template <bool GAUGE, bool DF>
int resident_ctas(int threads, size_t smem) {
    int nb = 0, dev = 0, nsm = 0;
    QDT_CUDA_TRY(cudaGetDevice(&dev));
    QDT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    QDT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, eri_rows_kernel<GAUGE, DF>, threads, smem));
    return (nb > 0 ? nb : 1) * nsm;
}

template <bool GAUGE, bool DF>
void launch_rows(const EriParams *prms, const EriTask *tasks, int ntasks, int *next, const Plan &pl, int threads,
                 size_t smem, cudaStream_t s) {
    QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_kernel<GAUGE, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    const int grid = min(ntasks, resident_ctas<GAUGE, DF>(threads, smem));
    QDT_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(int), s));
    eri_rows_kernel<GAUGE, DF><<<grid, threads, smem, s>>>(prms, tasks, ntasks, next, pl);
}
}  // namespace

void launch_eri(const EriParams *prms, const EriTask *tasks, int ntasks, int *next, const EriShape &shape,
                bool gauge, bool df, const EriLaunch &how, cudaStream_t s) {
    if (ntasks <= 0) return;
    const Plan pl = eri_plan(shape.maxnfp, shape.maxLab, shape.maxnpp, gauge);
    const size_t smem = plan_smem(pl);
    const int threads = how.threads > 0 ? how.threads : pl.threads;
    if (threads % 32 || threads > 256) throw Error{QDT_ERR_ARG, "integral kernel: threads must be 32..256, a multiple of 32"};
    if (gauge) {
        if (df) launch_rows<true, true>(prms, tasks, ntasks, next, pl, threads, smem, s);
        else launch_rows<true, false>(prms, tasks, ntasks, next, pl, threads, smem, s);
    } else {
        if (df) launch_rows<false, true>(prms, tasks, ntasks, next, pl, threads, smem, s);
        else launch_rows<false, false>(prms, tasks, ntasks, next, pl, threads, smem, s);
    }
    QDT_CHECK_KERNEL("eri_rows_kernel");
}

// max over the entries of two integral-row blocks of |A - B| / (Q_row Q_col),
// rows and columns mapped to their shell pairs (mult 3: gauge rows (ab, I)).
__global__ void ratio_kernel(const double *A, const double *B, long long rows, long long ldw, int mult,
                             const int *row_pair, const int *col_pair, long long ncols, const double *Q,
                             double *out) {
    double m = 0.0;
    const long long total = rows * ldw;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / ldw, c = e - r * ldw;
        if (c / mult >= ncols) continue;
        const double q = Q[row_pair[r / mult]] * Q[col_pair[c / mult]];
        const double d = fabs(A[e] - B[e]);
        if (d > 0.0) m = fmax(m, q > 0.0 ? d / q : INFINITY);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong(m));
}

void launch_ratio(const double *A, const double *B, long long rows, long long ldw, int mult, const int *row_pair,
                  const int *col_pair, long long ncols, const double *Q, double *out, cudaStream_t s) {
    if (rows <= 0 || ldw <= 0) return;
    long long blocks = std::min<long long>((rows * ldw + 255) / 256, 152 * 8);
    ratio_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, B, rows, ldw, mult, row_pair, col_pair, ncols, Q, out);
    QDT_CHECK_LAUNCH();
}

void launch_split_pairs(const double *E, long long n, float2 *E2, float *E1, cudaStream_t s) {
    if (n <= 0) return;
    split_pairs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E, n, E2, E1);
    QDT_CHECK_KERNEL("split_pairs_kernel");
}

// Schwarz diagonals: Q[AB] = max over ab of sqrt(|(ab|ab)|), Coulomb kernel.
__global__ void __launch_bounds__(256, 2) schwarz_kernel(const PrimPairDev *pp, const PairDev *pairs, const double *E,
                                                         const double *boys, Plan pl, double *Q) {
    extern __shared__ double sm[];
    const PairDev AB = pairs[blockIdx.x];
    BlockSmem b = carve(sm, pl);
    build_tables(pl, b);
    double qmax = 0.0;
    for (int a0 = 0; a0 < AB.nfp; a0 += pl.ach) {
        const int a1 = min(AB.nfp, a0 + pl.ach);
        block_chunk<false, false>(pp, E, nullptr, nullptr, boys, AB, AB, a0, a1, a0, a1, pl, b);
        const int ach = a1 - a0;
        if (threadIdx.x == 0)
            for (int a = 0; a < ach; ++a) qmax = fmax(qmax, sqrt(fabs(b.G[(size_t)a * ach + a])));
        __syncthreads();
    }
    if (threadIdx.x == 0) Q[blockIdx.x] = qmax;
}

void launch_schwarz(const ShellDev *shells, const PairDev *pairs, const PrimPairDev *pp, const double *E,
                    const double *boys, int npairs, int maxnfp, int maxLab, int maxnpp, double *Q,
                    cudaStream_t s) {
    (void)shells;
    if (npairs <= 0) return;
    const Plan pl = eri_plan(maxnfp, maxLab, maxnpp, false);
    const size_t smem = plan_smem(pl);
    QDT_CUDA_TRY(cudaFuncSetAttribute(schwarz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    schwarz_kernel<<<npairs, pl.threads, smem, s>>>(pp, pairs, E, boys, pl, Q);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
