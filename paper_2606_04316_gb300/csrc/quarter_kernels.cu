// quarter_kernels.cu -- the conventional two-quarter first half of the Coulomb
// block (Sec. 2.2, appendix operation counts), kept as a measured comparator to
// the density route of Eq. firsthalf.  For a bra function pair ab:
//   T1^sigma_ab[c, S] = sum_d (ab|cd) C^sigma_{dS}                 (quarter 1)
//   V^{RS}_ab  = sum_{c,sigma} conj(C^sigma_{cR}) T1^sigma_ab[c, S]    (quarter 2)
//   V^{R~S}_ab = sum_c alpha_{cR} T1^beta_ab[c, S] - beta_{cR} T1^alpha_ab[c, S]
// (R~ the Kramers partner of R), which is V_ab = sum_cd (ab|cd) D^{RS}_{cd} of
// the density route without forming the density.  Both quarters run as real
// GEMMs on the contraction engine; the kernels here re-lay the operands.
#include <math.h>

#include <algorithm>

#include "qdt_internal.cuh"

namespace qdt {

// Global function indices (c, d) of every column of the ket-ordered integral
// rows: sorted ket position q covers columns ket_col[q] .. + nfp.
__global__ void ket_functions_kernel(const PairDev *pairs, const ShellDev *shells, const int *ket_sp,
                                     const long long *ket_col, int2 *cols) {
    const int q = blockIdx.x;
    const PairDev pr = pairs[ket_sp[q]];
    const ShellDev A = shells[pr.sa], B = shells[pr.sb];
    const long long c0 = ket_col[q];
    for (int fp = threadIdx.x; fp < pr.nfp; fp += blockDim.x) {
        int fa, fb;
        if (pr.sa == pr.sb) {
            int a = 0, base = 0;
            while (base + (B.nfunc - a) <= fp) { base += B.nfunc - a; ++a; }
            fa = a; fb = a + (fp - base);
        } else {
            fa = fp / B.nfunc; fb = fp % B.nfunc;
        }
        cols[c0 + fp] = make_int2(A.foff + fa, B.foff + fb);
    }
}

void launch_ket_functions(const PairDev *pairs, const ShellDev *shells, const int *ket_sp,
                          const long long *ket_col, int nsp, int2 *cols, cudaStream_t s) {
    if (nsp <= 0) return;
    ket_functions_kernel<<<nsp, 64, 0, s>>>(pairs, shells, ket_sp, ket_col, cols);
    QDT_CHECK_LAUNCH();
}

// Screening bound of the quarter route, which never forms the density: for
// every density element of a shell pair, |D^{RS}_{cd} + D^{RS}_{dc}| <=
// 2 m_C m_D with m_F the largest two-spinor norm |C_{fR}| over the pair's
// functions f and the active columns (Cauchy-Schwarz; the Kramers partner has
// the same norm).  Replaces Dmax[sp] by this bound.
__global__ void coef_bound_kernel(const PairDev *pairs, const ShellDev *shells, const double *Cq, int nK,
                                  int k0, int nKa, double *Dmax) {
    const int sp = blockIdx.x;
    const PairDev pr = pairs[sp];
    __shared__ double red[2][32];
    for (int side = 0; side < 2; ++side) {
        const ShellDev S = shells[side ? pr.sb : pr.sa];
        double m = 0.0;
        for (int i = threadIdx.x; i < S.nfunc * nKa; i += blockDim.x) {
            const int f = S.foff + i / nKa, k = k0 + i % nKa;
            const double *q = Cq + ((size_t)f * nK + k) * 4;
            // ((q0^2 + q1^2) + q2^2) + q3^2 without contraction, so the
            // screening decision is reproducible in plain FP64
            const double n2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])),
                                                  __dmul_rn(q[2], q[2])),
                                        __dmul_rn(q[3], q[3]));
            m = fmax(m, n2);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[side][threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ma = 0.0, mb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ma = fmax(ma, red[0][w]); mb = fmax(mb, red[1][w]); }
        Dmax[sp] = 2.0 * sqrt(ma) * sqrt(mb);
    }
}

void launch_coef_bound(const PairDev *pairs, const ShellDev *shells, const double *Cq, int nK, int k0,
                       int nKa, int nsp, double *Dmax, cudaStream_t s) {
    if (nsp <= 0) return;
    coef_bound_kernel<<<nsp, 128, 0, s>>>(pairs, shells, Cq, nK, k0, nKa, Dmax);
    QDT_CHECK_LAUNCH();
}

// Quarter-1 coefficients Cr1[f][j n + S] = Cq[f][k0 + S][j] (j: Re alpha,
// Im alpha, Re beta, Im beta), and the quarter-2 map Cr2[j nX + c][R P + part]
// (P = 4: parts Re/Im V^{RS}, Re/Im V^{R~S}; P = 2: the first two).
__global__ void quarter_coefs_kernel(const double *Cq, int nK, int k0, int n, int nX, int P, double *Cr1,
                                     double *Cr2) {
    const long long total = (long long)nX * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(e / n), R = (int)(e % n);
        const double *q = Cq + ((size_t)f * nK + k0 + R) * 4;
        const double ar = q[0], ai = q[1], br = q[2], bi = q[3];
        for (int j = 0; j < 4; ++j) Cr1[(size_t)f * 4 * n + (size_t)j * n + R] = q[j];
        // rows j = 0..3 (T1 components Re/Im alpha, Re/Im beta), columns part
        const double m[4][4] = {{ar, -ai, -br, -bi},
                                {ai, ar, bi, -br},
                                {br, -bi, ar, ai},
                                {bi, br, -ai, ar}};
        for (int j = 0; j < 4; ++j)
            for (int part = 0; part < P; ++part)
                Cr2[((size_t)j * nX + f) * (size_t)(P * n) + (size_t)R * P + part] = m[j][part];
    }
}

void launch_quarter_coefs(const double *Cq, int nK, int k0, int n, int nX, int P, double *Cr1, double *Cr2,
                          cudaStream_t s) {
    const long long total = (long long)nX * n;
    if (total <= 0) return;
    long long blocks = std::min<long long>((total + 255) / 256, 152 * 8);
    quarter_coefs_kernel<<<(unsigned)blocks, 256, 0, s>>>(Cq, nK, k0, n, nX, P, Cr1, Cr2);
    QDT_CHECK_LAUNCH();
}

// Integral rows (ket-ordered columns, row length ldw, zero past each row's
// kept prefix) -> square blocks WL[r][c][d] (L functions) and WS[r][c][d]
// (S functions); every (c, d) of a block belongs to exactly one ket column,
// so both triangles are written and nothing needs clearing first.
__global__ void square_rows_kernel(const double *W, long long ldw, const int2 *cols, long long ncols, int nL,
                                   int nS, double *WL, double *WS) {
    const long long r = blockIdx.y;
    const double *w = W + r * ldw;
    double *wl = WL + r * (long long)nL * nL, *ws = WS + r * (long long)nS * nS;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < ncols;
         j += (long long)gridDim.x * blockDim.x) {
        const int2 cd = cols[j];
        const double v = j < ldw ? w[j] : 0.0;
        if (cd.x < nL) {
            wl[(long long)cd.x * nL + cd.y] = v;
            wl[(long long)cd.y * nL + cd.x] = v;
        } else {
            const int c = cd.x - nL, d = cd.y - nL;
            ws[(long long)c * nS + d] = v;
            ws[(long long)d * nS + c] = v;
        }
    }
}

void launch_square_rows(const double *W, long long ldw, const int2 *cols, long long ncols, int nL, int nS,
                        long long rows, double *WL, double *WS, cudaStream_t s) {
    if (rows <= 0 || ncols <= 0) return;
    const unsigned gx = (unsigned)std::min<long long>((ncols + 255) / 256, 64);
    for (long long r0 = 0; r0 < rows; r0 += 65535) {
        const long long rr = std::min<long long>(65535, rows - r0);
        square_rows_kernel<<<dim3(gx, (unsigned)rr), 256, 0, s>>>(W + r0 * ldw, ldw, cols, ncols, nL, nS,
                                                                  WL + r0 * (long long)nL * nL,
                                                                  WS + r0 * (long long)nS * nS);
        QDT_CHECK_LAUNCH();
    }
}

// Quarter-1 output T1[r][c][j n + S] (L rows then S rows per block of r) ->
// quarter-2 operand T[r n + S][j nX + c], through 32 x 32 shared tiles.
__global__ void t1_transpose_kernel(const double *TL, const double *TS, int nL, int nS, int n, double *T) {
    __shared__ double tile[32][33];
    const int nX = nL + nS;
    const long long rj = blockIdx.z;
    const long long r = rj / 4;
    const int j = (int)(rj % 4);
    const int c0 = blockIdx.y * 32, s0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, S = s0 + threadIdx.x;
        double v = 0.0;
        if (c < nX && S < n)
            v = c < nL ? TL[(r * nL + c) * 4 * n + (long long)j * n + S]
                       : TS[(r * nS + (c - nL)) * 4 * n + (long long)j * n + S];
        tile[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int S = s0 + i, c = c0 + threadIdx.x;
        if (S < n && c < nX) T[(r * n + S) * 4 * (long long)nX + (long long)j * nX + c] = tile[threadIdx.x][i];
    }
}

void launch_t1_transpose(const double *TL, const double *TS, int nL, int nS, int n, long long rows, double *T,
                         cudaStream_t s) {
    if (rows <= 0 || n <= 0) return;
    const int nX = nL + nS;
    for (long long r0 = 0; r0 < rows; r0 += 16383) {
        const long long rr = std::min<long long>(16383, rows - r0);
        dim3 grid((unsigned)((n + 31) / 32), (unsigned)((nX + 31) / 32), (unsigned)(rr * 4));
        t1_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(TL + r0 * nL * 4LL * n, TS + r0 * nS * 4LL * n, nL, nS,
                                                         n, T + r0 * n * 4LL * nX);
        QDT_CHECK_LAUNCH();
    }
}

// Vfull[r n + S][R P + part] -> V[r][rs P + part] for the canonical column
// pairs rs = (rsR[rs], rsS[rs]), R <= S.
__global__ void quarter_gather_kernel(const double *Vf, int n, int P, const int *rsR, const int *rsS, int nRS,
                                      long long rows, double *V) {
    const long long total = rows * nRS * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / ((long long)nRS * P);
        const int rem = (int)(e - r * nRS * P), rs = rem / P, part = rem % P;
        V[e] = Vf[(r * n + rsS[rs]) * (long long)(P * n) + (long long)rsR[rs] * P + part];
    }
}

void launch_quarter_gather(const double *Vf, int n, int P, const int *rsR, const int *rsS, int nRS,
                           long long rows, double *V, cudaStream_t s) {
    const long long total = rows * nRS * P;
    if (total <= 0) return;
    long long blocks = std::min<long long>((total + 255) / 256, 152 * 16);
    quarter_gather_kernel<<<(unsigned)blocks, 256, 0, s>>>(Vf, n, P, rsR, rsS, nRS, rows, V);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
