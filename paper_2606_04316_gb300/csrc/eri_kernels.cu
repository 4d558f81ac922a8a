// eri_kernels.cu -- AO two-electron integral tiles on the GPU (stage (i) of
// the paper's Sec. 3.3.1 decomposition), McMurchie-Davidson in FP64:
//
//   (ab|K|cd) = sum_{ij in AB, kl in CD} sum_{h, h'} E^{ij}_{ab,h} (-1)^{|h'|}
//               E^{kl}_{cd,h'} R^K_{h+h'}(rho, P - Q)
//
//   1/r12 (Eq. Coulomb):   R^n_000 = (-2 rho)^n F_n(T) * 2 pi^{5/2} / (p q sqrt(p+q))
//   r12 (for Eq. gaugeInt): R^n_000 = (-2 rho)^n (F_n - F_{n-1})(T) * pi^{5/2} sqrt(p+q) / (p q)^2,
//                          F_{-1}(T) = -(2 T F_0 + e^{-T})  (Gaussian-smeared distance)
//   gauge kernel:  (ab|r_I r_J/r^3|cd) = delta_IJ (ab|1/r|cd) - (ab|d_I d_J r|cd),
//                  the last term shifting the Hermite index of the r12 tensor by e_I + e_J,
//   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}  (same in u, v).
#include <math.h>

#include "qdt_internal.cuh"

namespace qdt {

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

// F_0..F_nmax at T: Taylor expansion of the tabulated top order, then the
// downward recursion; beyond the table F_0 = sqrt(pi/T) erf(sqrt T) / 2 and
// upward recursion.
__device__ void boys_eval(const double *tab, double T, int nmax, double *F) {
    double e = exp(-T);
    if (T < kBoysTMax) {
        int i = (int)(T * (1.0 / kBoysDelta) + 0.5);
        double d = T - i * kBoysDelta;
        const double *row = tab + (size_t)i * kBoysCols;
        double f = 0.0, term = 1.0;
        for (int k = 0; k < kBoysTaylor; ++k) {
            f += row[nmax + k] * term;
            term *= -d / (k + 1);
        }
        F[nmax] = f;
        for (int n = nmax - 1; n >= 0; --n) F[n] = (2.0 * T * F[n + 1] + e) / (2.0 * n + 1.0);
    } else {
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int n = 0; n < nmax; ++n) F[n + 1] = ((2.0 * n + 1.0) * F[n] - e) / (2.0 * T);
    }
}

struct BlockSmem {
    double *G, *T, *RC[2], *RR[2], *F, *scal;
    int *trA, *trC;
};

// Shared-memory plan of one block chunk (must match eri_smem_bytes()).
__device__ inline BlockSmem carve(double *sm, int NC, int ach, int cch, int nhaMax, int LtC, int LtR) {
    BlockSmem b;
    b.G = sm; sm += (size_t)NC * ach * cch;
    b.T = sm; sm += (size_t)NC * nhaMax * cch;
    b.RC[0] = sm; sm += nherm(LtC);
    b.RC[1] = sm; sm += nherm(LtC);
    b.RR[0] = sm; sm += (LtR >= 0 ? nherm(LtR) : 0);
    b.RR[1] = sm; sm += (LtR >= 0 ? nherm(LtR) : 0);
    b.F = sm; sm += kBoysNMax + 3;
    b.scal = sm; sm += 8;
    b.trA = (int *)sm;
    b.trC = b.trA + 3 * nherm(kMaxLPair);
    return b;
}

size_t eri_smem_bytes(int NC, int ach, int cch, int maxLab, bool gauge) {
    int LtC = 2 * maxLab, LtR = gauge ? 2 * maxLab + 2 : -1;
    size_t d = (size_t)NC * ach * cch + (size_t)NC * nherm(maxLab) * cch + 2 * nherm(LtC) +
               (LtR >= 0 ? 2 * nherm(LtR) : 0) + kBoysNMax + 3 + 8;
    return d * sizeof(double) + 6 * nherm(kMaxLPair) * sizeof(int);
}

// One chunk (ab in [a0,a1), cd in [c0,c1)) of the block (AB|CD); results in
// b.G[comp][a][c].  NC = 1 (Coulomb) or 7 (gauge: [0] Coulomb, [1..6]
// (ab|d_I d_J r|cd) for IJ = xx,xy,xz,yy,yz,zz).
template <bool GAUGE>
__device__ void block_chunk(const PrimPairDev *pp, const double *E, const double *boys,
                            const PairDev &AB, const PairDev &CD, int a0, int a1, int c0, int c1,
                            BlockSmem &b) {
    constexpr int NC = GAUGE ? 7 : 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int La = AB.Lab, Lc = CD.Lab;
    const int nha = nherm(La), nhc = nherm(Lc);
    const int L = La + Lc, Lr = L + 2;
    const int ach = a1 - a0, cch = c1 - c0;
    for (int h = tid; h < nha; h += nt) htrip_d(h, b.trA[3 * h], b.trA[3 * h + 1], b.trA[3 * h + 2]);
    for (int h = tid; h < nhc; h += nt) htrip_d(h, b.trC[3 * h], b.trC[3 * h + 1], b.trC[3 * h + 2]);
    for (int i = tid; i < NC * ach * cch; i += nt) b.G[i] = 0.0;
    __syncthreads();
    for (int ij = 0; ij < AB.npp; ++ij) {
        const PrimPairDev pa = pp[AB.ppoff + ij];
        for (int i = tid; i < NC * nha * cch; i += nt) b.T[i] = 0.0;
        for (int kl = 0; kl < CD.npp; ++kl) {
            const PrimPairDev pc = pp[CD.ppoff + kl];
            if (tid == 0) {
                double p = pa.p, q = pc.p, rho = p * q / (p + q);
                double X = pa.P[0] - pc.P[0], Y = pa.P[1] - pc.P[1], Z = pa.P[2] - pc.P[2];
                double T = rho * (X * X + Y * Y + Z * Z);
                int nmax = GAUGE ? Lr : L;
                boys_eval(boys, T, nmax, b.F + 1);
                b.F[0] = -(2.0 * T * b.F[1] + exp(-T));        // F_{-1}
                b.scal[0] = X; b.scal[1] = Y; b.scal[2] = Z;
                b.scal[3] = -2.0 * rho;
                b.scal[4] = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
                b.scal[5] = pow(M_PI, 2.5) * sqrt(p + q) / (p * p * q * q);
            }
            __syncthreads();
            const double X = b.scal[0], Y = b.scal[1], Z = b.scal[2], m2r = b.scal[3];
            const int Ltop = GAUGE ? Lr : L;
            for (int n = Ltop; n >= 0; --n) {
                double *dC = b.RC[n & 1], *sC = b.RC[(n + 1) & 1];
                double *dR = b.RR[n & 1], *sR = b.RR[(n + 1) & 1];
                int cntR = GAUGE ? nherm(Lr - n) : 0;
                int cntC = (n <= L) ? nherm(L - n) : 0;
                int cnt = cntR > cntC ? cntR : cntC;
                for (int h = tid; h < cnt; h += nt) {
                    int t, u, v;
                    htrip_d(h, t, u, v);
                    double base = 0.0;
                    if (h == 0) base = pow(m2r, n);
                    // Coulomb tensor
                    if (h < cntC) {
                        double r;
                        if (h == 0) r = base * b.F[n + 1] * b.scal[4];
                        else if (t > 0) r = (t > 1 ? (t - 1) * sC[hidx(t - 2, u, v)] : 0.0) + X * sC[hidx(t - 1, u, v)];
                        else if (u > 0) r = (u > 1 ? (u - 1) * sC[hidx(t, u - 2, v)] : 0.0) + Y * sC[hidx(t, u - 1, v)];
                        else r = (v > 1 ? (v - 1) * sC[hidx(t, u, v - 2)] : 0.0) + Z * sC[hidx(t, u, v - 1)];
                        dC[h] = r;
                    }
                    if (GAUGE && h < cntR) {
                        double r;
                        if (h == 0) r = base * (b.F[n + 1] - b.F[n]) * b.scal[5];
                        else if (t > 0) r = (t > 1 ? (t - 1) * sR[hidx(t - 2, u, v)] : 0.0) + X * sR[hidx(t - 1, u, v)];
                        else if (u > 0) r = (u > 1 ? (u - 1) * sR[hidx(t, u - 2, v)] : 0.0) + Y * sR[hidx(t, u - 1, v)];
                        else r = (v > 1 ? (v - 1) * sR[hidx(t, u, v - 2)] : 0.0) + Z * sR[hidx(t, u, v - 1)];
                        dR[h] = r;
                    }
                }
                __syncthreads();
            }
            const double *RC0 = b.RC[0], *RR0 = b.RR[0];
            const double *Ekl = E + pc.eoff;
            for (int idx = tid; idx < nha * cch; idx += nt) {
                int h = idx / cch, c = idx - h * cch;
                int t = b.trA[3 * h], u = b.trA[3 * h + 1], v = b.trA[3 * h + 2];
                const double *e = Ekl + (size_t)(c0 + c) * nhc;
                double sc = 0.0;
                double sr[6] = {0, 0, 0, 0, 0, 0};
                for (int hp = 0; hp < nhc; ++hp) {
                    int tp = b.trC[3 * hp], up = b.trC[3 * hp + 1], vp = b.trC[3 * hp + 2];
                    double ev = ((tp + up + vp) & 1) ? -e[hp] : e[hp];
                    int T0 = t + tp, U0 = u + up, V0 = v + vp;
                    sc += RC0[hidx(T0, U0, V0)] * ev;
                    if (GAUGE) {
                        sr[0] += RR0[hidx(T0 + 2, U0, V0)] * ev;
                        sr[1] += RR0[hidx(T0 + 1, U0 + 1, V0)] * ev;
                        sr[2] += RR0[hidx(T0 + 1, U0, V0 + 1)] * ev;
                        sr[3] += RR0[hidx(T0, U0 + 2, V0)] * ev;
                        sr[4] += RR0[hidx(T0, U0 + 1, V0 + 1)] * ev;
                        sr[5] += RR0[hidx(T0, U0, V0 + 2)] * ev;
                    }
                }
                b.T[(size_t)h * cch + c] += sc;
                if (GAUGE)
                    for (int k = 0; k < 6; ++k) b.T[((size_t)(k + 1) * nha + h) * cch + c] += sr[k];
            }
            __syncthreads();
        }
        const double *Eij = E + pa.eoff;
        for (int idx = tid; idx < ach * cch; idx += nt) {
            int a = idx / cch, c = idx - a * cch;
            const double *e = Eij + (size_t)(a0 + a) * nha;
            double s[NC];
            for (int k = 0; k < NC; ++k) s[k] = 0.0;
            for (int h = 0; h < nha; ++h) {
                double ev = e[h];
                for (int k = 0; k < NC; ++k) s[k] += ev * b.T[((size_t)k * nha + h) * cch + c];
            }
            for (int k = 0; k < NC; ++k) b.G[((size_t)k * ach + a) * cch + c] += s[k];
        }
        __syncthreads();
    }
}

struct ChunkCfg { int ach, cch; };

// Screened rows: one CTA per task (bra shell pair x range of sorted ket positions).
template <bool GAUGE>
__global__ void __launch_bounds__(128) eri_rows_kernel(EriParams prm, const EriTask *tasks, ChunkCfg cfg) {
    extern __shared__ double sm[];
    const EriTask tk = tasks[blockIdx.x];
    const PairDev AB = prm.pairs[tk.bra_sp];
    constexpr int NC = GAUGE ? 7 : 1;
    BlockSmem b = carve(sm, NC, cfg.ach, cfg.cch, nherm(kMaxLPair), 2 * kMaxLPair,
                        GAUGE ? 2 * kMaxLPair + 2 : -1);
    for (int kp = tk.k0; kp < tk.k1; ++kp) {
        const PairDev CD = prm.pairs[prm.ket_sp[kp]];
        const long long col = prm.ket_col[kp];
        for (int a0 = 0; a0 < AB.nfp; a0 += cfg.ach) {
            int a1 = min(AB.nfp, a0 + cfg.ach);
            for (int c0 = 0; c0 < CD.nfp; c0 += cfg.cch) {
                int c1 = min(CD.nfp, c0 + cfg.cch);
                block_chunk<GAUGE>(prm.pp, prm.E, prm.boys, AB, CD, a0, a1, c0, c1, b);
                int ach = a1 - a0, cch = c1 - c0;
                for (int idx = threadIdx.x; idx < ach * cch; idx += blockDim.x) {
                    int a = idx / cch, c = idx - a * cch;
                    long long row = AB.rowoff + a0 + a - prm.row0;
                    long long cc = col + c0 + c;
                    if (!GAUGE) {
                        prm.W[row * prm.ldw + cc] = b.G[idx];
                    } else {
                        double C = b.G[idx];
                        const double *H = b.G + (size_t)ach * cch;
                        const int ij_of[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
                        for (int I = 0; I < 3; ++I)
                            for (int J = 0; J < 3; ++J) {
                                double h = H[(size_t)ij_of[I][J] * ach * cch + idx];
                                prm.W[(row * 3 + I) * prm.ldw + cc * 3 + J] = (I == J ? C : 0.0) - h;
                            }
                        if (prm.with_coulomb) prm.Wc[row * prm.ldwc + cc] = C;
                    }
                }
                __syncthreads();
            }
        }
    }
}

ChunkCfg eri_chunks(int maxnfp, int maxLab, bool gauge, size_t *smem) {
    int NC = gauge ? 7 : 1;
    ChunkCfg c;
    c.ach = c.cch = maxnfp < 96 ? maxnfp : 96;
    const size_t budget = 200 * 1024;
    while (eri_smem_bytes(NC, c.ach, c.cch, kMaxLPair, gauge) > budget && c.ach > 8) {
        c.ach = (c.ach + 1) / 2;
        c.cch = (c.cch + 1) / 2;
    }
    *smem = eri_smem_bytes(NC, c.ach, c.cch, kMaxLPair, gauge);
    return c;
}

void launch_eri(const EriParams &prm, const EriTask *tasks, int ntasks, int maxnfp, int maxLab,
                cudaStream_t s) {
    if (ntasks <= 0) return;
    size_t smem;
    ChunkCfg cfg = eri_chunks(maxnfp, maxLab, prm.gauge != 0, &smem);
    if (prm.gauge) {
        QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        eri_rows_kernel<true><<<ntasks, 128, smem, s>>>(prm, tasks, cfg);
    } else {
        QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        eri_rows_kernel<false><<<ntasks, 128, smem, s>>>(prm, tasks, cfg);
    }
    QDT_CHECK_LAUNCH();
}

// Schwarz diagonals: Q[AB] = max over ab of sqrt(|(ab|ab)|), Coulomb kernel.
__global__ void __launch_bounds__(128) schwarz_kernel(const PrimPairDev *pp, const PairDev *pairs,
                                                      const double *E, const double *boys,
                                                      ChunkCfg cfg, double *Q) {
    extern __shared__ double sm[];
    const PairDev AB = pairs[blockIdx.x];
    BlockSmem b = carve(sm, 1, cfg.ach, cfg.cch, nherm(kMaxLPair), 2 * kMaxLPair, -1);
    double qmax = 0.0;
    for (int a0 = 0; a0 < AB.nfp; a0 += cfg.ach) {
        int a1 = min(AB.nfp, a0 + cfg.ach);
        block_chunk<false>(pp, E, boys, AB, AB, a0, a1, a0, a1, b);
        int ach = a1 - a0;
        if (threadIdx.x == 0)
            for (int a = 0; a < ach; ++a) qmax = fmax(qmax, sqrt(fabs(b.G[(size_t)a * ach + a])));
        __syncthreads();
    }
    if (threadIdx.x == 0) Q[blockIdx.x] = qmax;
}

void launch_schwarz(const ShellDev *shells, const PairDev *pairs, const PrimPairDev *pp,
                    const double *E, const double *boys, int npairs, int maxnfp, int maxLab,
                    double *Q, double *scratch, cudaStream_t s) {
    (void)shells; (void)scratch;
    if (npairs <= 0) return;
    size_t smem;
    ChunkCfg cfg = eri_chunks(maxnfp, maxLab, false, &smem);
    cfg.cch = cfg.ach;
    QDT_CUDA_TRY(cudaFuncSetAttribute(schwarz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    schwarz_kernel<<<npairs, 128, smem, s>>>(pp, pairs, E, boys, cfg, Q);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
