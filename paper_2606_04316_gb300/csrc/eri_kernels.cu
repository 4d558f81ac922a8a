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
// For every shell quartet the cheaper orientation is contracted (the pair
// with more function pairs takes the outer, per-primitive-pair role), and for
// every outer primitive pair all inner primitive pairs are processed together:
// Boys values in parallel, one barrier per recursion level, then the
// contraction T = R E' and the accumulation G += E T.
#include <math.h>
#include <stdlib.h>

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

// Shared-memory plan (sizes from the class maxima; must match eri_smem_bytes()).
struct Plan {
    int NC;         // 1 Coulomb, 7 gauge
    int ach, cch;   // chunk of outer / inner function pairs
    int nhMax;      // nherm(max Lab)
    int LtC, LtR;   // top Hermite orders of the Coulomb and r12 tensors (LtR < 0: none)
    int klg;        // inner primitive pairs per group
};

struct BlockSmem {
    double *G, *T, *RC, *RR, *F, *sc;
    int *trX, *trY;
};

__host__ __device__ inline size_t smem_doubles(const Plan &p) {
    size_t nrC = nherm(p.LtC), nrR = p.LtR >= 0 ? nherm(p.LtR) : 0;
    return (size_t)p.NC * p.ach * p.cch + (size_t)p.NC * p.nhMax * p.cch + 2 * p.klg * nrC + 2 * p.klg * nrR +
           (size_t)p.klg * (kBoysNMax + 3) + (size_t)p.klg * 8;
}

size_t eri_smem_bytes(const Plan &p) { return smem_doubles(p) * sizeof(double) + 6 * p.nhMax * sizeof(int) + 64; }

__device__ inline BlockSmem carve(double *sm, const Plan &p) {
    BlockSmem b;
    size_t nrC = nherm(p.LtC), nrR = p.LtR >= 0 ? nherm(p.LtR) : 0;
    b.G = sm; sm += (size_t)p.NC * p.ach * p.cch;
    b.T = sm; sm += (size_t)p.NC * p.nhMax * p.cch;
    b.RC = sm; sm += 2 * p.klg * nrC;
    b.RR = sm; sm += 2 * p.klg * nrR;
    b.F = sm; sm += (size_t)p.klg * (kBoysNMax + 3);
    b.sc = sm; sm += (size_t)p.klg * 8;
    b.trX = (int *)sm;
    b.trY = b.trX + 3 * p.nhMax;
    return b;
}

__host__ __device__ inline double orient_cost(const PairDev &X, const PairDev &Y) {
    double nhx = nherm(X.Lab), nhy = nherm(Y.Lab);
    return (double)X.npp * Y.npp * nhx * Y.nfp * nhy + (double)X.npp * X.nfp * Y.nfp * nhx;
}

// One chunk (x in [x0,x1) of X, y in [y0,y1) of Y) of the block (X|Y);
// results in b.G[comp][x][y].  NC = 1 (Coulomb) or 7 (gauge: [0] Coulomb,
// [1..6] (xy|d_I d_J r|zw) for IJ = xx,xy,xz,yy,yz,zz).
template <bool GAUGE>
__device__ void block_chunk(const PrimPairDev *pp, const double *E, const double *boys, const PairDev &X,
                            const PairDev &Y, int x0, int x1, int y0, int y1, const Plan &pl, BlockSmem &b) {
    constexpr int NC = GAUGE ? 7 : 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Lx = X.Lab, Ly = Y.Lab;
    const int nhx = nherm(Lx), nhy = nherm(Ly);
    const int L = Lx + Ly, Lr = L + 2, Ltop = GAUGE ? Lr : L;
    const int nrC = nherm(pl.LtC), nrR = GAUGE ? nherm(pl.LtR) : 0;
    const int xch = x1 - x0, ych = y1 - y0;
    for (int h = tid; h < nhx; h += nt) htrip_d(h, b.trX[3 * h], b.trX[3 * h + 1], b.trX[3 * h + 2]);
    for (int h = tid; h < nhy; h += nt) htrip_d(h, b.trY[3 * h], b.trY[3 * h + 1], b.trY[3 * h + 2]);
    for (int i = tid; i < NC * xch * ych; i += nt) b.G[i] = 0.0;
    __syncthreads();
    for (int ij = 0; ij < X.npp; ++ij) {
        const PrimPairDev pa = pp[X.ppoff + ij];
        for (int i = tid; i < NC * nhx * ych; i += nt) b.T[i] = 0.0;
        for (int g0 = 0; g0 < Y.npp; g0 += pl.klg) {
            const int ng = min(pl.klg, Y.npp - g0);
            // Boys values and geometry of the group's primitive quartets
            for (int g = tid; g < ng; g += nt) {
                const PrimPairDev pc = pp[Y.ppoff + g0 + g];
                double p = pa.p, q = pc.p, rho = p * q / (p + q);
                double Xq = pa.P[0] - pc.P[0], Yq = pa.P[1] - pc.P[1], Zq = pa.P[2] - pc.P[2];
                double Tv = rho * (Xq * Xq + Yq * Yq + Zq * Zq);
                double *F = b.F + g * (kBoysNMax + 3);
                boys_eval(boys, Tv, Ltop, F + 1);
                F[0] = -(2.0 * Tv * F[1] + exp(-Tv));       // F_{-1}
                double *sc = b.sc + g * 8;
                sc[0] = Xq; sc[1] = Yq; sc[2] = Zq; sc[3] = -2.0 * rho;
                sc[4] = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
                sc[5] = pow(M_PI, 2.5) * sqrt(p + q) / (p * p * q * q);
            }
            __syncthreads();
            // Hermite recursion, all primitive quartets of the group per level
            for (int n = Ltop; n >= 0; --n) {
                const int cntC = (n <= L) ? nherm(L - n) : 0;
                const int cntR = GAUGE ? nherm(Lr - n) : 0;
                const int cnt = cntR > cntC ? cntR : cntC;
                for (int it = tid; it < ng * cnt; it += nt) {
                    const int g = it / cnt, h = it - g * cnt;
                    const double *sc = b.sc + g * 8;
                    const double Xq = sc[0], Yq = sc[1], Zq = sc[2];
                    int t, u, v;
                    htrip_d(h, t, u, v);
                    if (h < cntC) {
                        double *d = b.RC + ((size_t)(n & 1) * pl.klg + g) * nrC;
                        const double *s = b.RC + ((size_t)((n + 1) & 1) * pl.klg + g) * nrC;
                        double r;
                        if (h == 0) r = pow(sc[3], n) * b.F[g * (kBoysNMax + 3) + n + 1] * sc[4];
                        else if (t > 0) r = (t > 1 ? (t - 1) * s[hidx(t - 2, u, v)] : 0.0) + Xq * s[hidx(t - 1, u, v)];
                        else if (u > 0) r = (u > 1 ? (u - 1) * s[hidx(t, u - 2, v)] : 0.0) + Yq * s[hidx(t, u - 1, v)];
                        else r = (v > 1 ? (v - 1) * s[hidx(t, u, v - 2)] : 0.0) + Zq * s[hidx(t, u, v - 1)];
                        d[h] = (n == 0 && ((t + u + v) & 1)) ? -r : r;   // level 0 keeps (-1)^|k| R_k
                    }
                    if (GAUGE && h < cntR) {
                        double *d = b.RR + ((size_t)(n & 1) * pl.klg + g) * nrR;
                        const double *s = b.RR + ((size_t)((n + 1) & 1) * pl.klg + g) * nrR;
                        const double *F = b.F + g * (kBoysNMax + 3);
                        double r;
                        if (h == 0) r = pow(sc[3], n) * (F[n + 1] - F[n]) * sc[5];
                        else if (t > 0) r = (t > 1 ? (t - 1) * s[hidx(t - 2, u, v)] : 0.0) + Xq * s[hidx(t - 1, u, v)];
                        else if (u > 0) r = (u > 1 ? (u - 1) * s[hidx(t, u - 2, v)] : 0.0) + Yq * s[hidx(t, u - 1, v)];
                        else r = (v > 1 ? (v - 1) * s[hidx(t, u, v - 2)] : 0.0) + Zq * s[hidx(t, u, v - 1)];
                        d[h] = (n == 0 && ((t + u + v) & 1)) ? -r : r;
                    }
                }
                __syncthreads();
            }
            // T[c][h][y] += sum_{kl in group} sum_h' R[h+h'] (-1)^|h'| E^{kl}[y][h']
            //            = (-1)^|h| sum_h' Rs[h+h'] E^{kl}[y][h'],  Rs_k = (-1)^|k| R_k
            // two output columns per thread: one R load feeds two FMAs
            const int ych2 = (ych + 1) >> 1;
            for (int idx = tid; idx < nhx * ych2; idx += nt) {
                const int h = idx / ych2, y1 = idx - h * ych2, y2 = y1 + ych2;
                const bool two = y2 < ych;
                const int t = b.trX[3 * h], u = b.trX[3 * h + 1], v = b.trX[3 * h + 2];
                double sc1 = 0.0, sc2 = 0.0, sr1[6] = {0, 0, 0, 0, 0, 0}, sr2[6] = {0, 0, 0, 0, 0, 0};
                for (int g = 0; g < ng; ++g) {
                    const double *e = E + pp[Y.ppoff + g0 + g].eoff + (y0 + y1);   // E[h'][y], stride nfp
                    const double *RC0 = b.RC + (size_t)g * nrC;
                    const double *RR0 = b.RR + (size_t)g * nrR;
                    for (int hp = 0; hp < nhy; ++hp) {
                        const int tp = b.trY[3 * hp], up = b.trY[3 * hp + 1], vp = b.trY[3 * hp + 2];
                        const double e1 = __ldg(e + (size_t)hp * Y.nfp);
                        const double e2 = two ? __ldg(e + (size_t)hp * Y.nfp + ych2) : 0.0;
                        const int T0 = t + tp, U0 = u + up, V0 = v + vp;
                        const double rc = RC0[hidx(T0, U0, V0)];
                        sc1 = fma(rc, e1, sc1);
                        sc2 = fma(rc, e2, sc2);
                        if (GAUGE) {
                            const double r[6] = {RR0[hidx(T0 + 2, U0, V0)], RR0[hidx(T0 + 1, U0 + 1, V0)],
                                                 RR0[hidx(T0 + 1, U0, V0 + 1)], RR0[hidx(T0, U0 + 2, V0)],
                                                 RR0[hidx(T0, U0 + 1, V0 + 1)], RR0[hidx(T0, U0, V0 + 2)]};
#pragma unroll
                            for (int k = 0; k < 6; ++k) {
                                sr1[k] = fma(r[k], e1, sr1[k]);
                                sr2[k] = fma(r[k], e2, sr2[k]);
                            }
                        }
                    }
                }
                const bool odd = (t + u + v) & 1;
                b.T[(size_t)h * ych + y1] += odd ? -sc1 : sc1;
                if (two) b.T[(size_t)h * ych + y2] += odd ? -sc2 : sc2;
                if (GAUGE)
                    for (int k = 0; k < 6; ++k) {
                        b.T[((size_t)(k + 1) * nhx + h) * ych + y1] += odd ? -sr1[k] : sr1[k];
                        if (two) b.T[((size_t)(k + 1) * nhx + h) * ych + y2] += odd ? -sr2[k] : sr2[k];
                    }
            }
            __syncthreads();
        }
        // G[c][x][y] += sum_h E^{ij}[x][h] T[c][h][y], two columns per thread
        const double *Eij = E + pa.eoff;
        const int ych2 = (ych + 1) >> 1;
        for (int idx = tid; idx < xch * ych2; idx += nt) {
            const int xx = idx / ych2, y1 = idx - xx * ych2, y2 = y1 + ych2;
            const bool two = y2 < ych;
            const double *e = Eij + (x0 + xx);                                 // E[h][x], stride nfp
            double s1[NC], s2[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) s1[k] = s2[k] = 0.0;
            for (int h = 0; h < nhx; ++h) {
                const double ev = __ldg(e + (size_t)h * X.nfp);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const double *Tk = b.T + ((size_t)k * nhx + h) * ych;
                    s1[k] = fma(ev, Tk[y1], s1[k]);
                    if (two) s2[k] = fma(ev, Tk[y2], s2[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                b.G[((size_t)k * xch + xx) * ych + y1] += s1[k];
                if (two) b.G[((size_t)k * xch + xx) * ych + y2] += s2[k];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ warp engine
// Each warp owns whole shell quartets: its phases synchronise with __syncwarp
// only, so a warp in the Hermite recursion never waits for another warp.
constexpr int kWGroup = 16;   // primitive quartets whose Boys values a warp evaluates at once

struct WPlan {
    int NC, ach, cch, nhMax, LtC, LtR;
    int nwarps;           // warps per CTA
    int warp_doubles;     // shared doubles per warp
};

__host__ __device__ inline int wplan_doubles(int NC, int ach, int cch, int nhMax, int LtC, int LtR) {
    int nrC = nherm(LtC), nrR = LtR >= 0 ? nherm(LtR) : 0;
    return NC * ach * cch + NC * nhMax * cch + 2 * nrC + 2 * nrR + kWGroup * (kBoysNMax + 3) + kWGroup * 8 +
           (3 * nhMax * 2 + 1) / 2 + 2;
}

struct WSmem {
    double *G, *T, *RC, *RR, *F, *sc;
    int *trX, *trY;
};

__device__ inline WSmem wcarve(double *sm, const WPlan &p) {
    WSmem b;
    int nrC = nherm(p.LtC), nrR = p.LtR >= 0 ? nherm(p.LtR) : 0;
    b.G = sm; sm += p.NC * p.ach * p.cch;
    b.T = sm; sm += p.NC * p.nhMax * p.cch;
    b.RC = sm; sm += 2 * nrC;
    b.RR = sm; sm += 2 * nrR;
    b.F = sm; sm += kWGroup * (kBoysNMax + 3);
    b.sc = sm; sm += kWGroup * 8;
    b.trX = (int *)sm;
    b.trY = b.trX + 3 * p.nhMax;
    return b;
}

// One chunk of the block (X|Y) by one warp; results in b.G[comp][x][y].
template <bool GAUGE>
__device__ void warp_chunk(const PrimPairDev *pp, const double *E, const double *boys, const PairDev &X,
                           const PairDev &Y, int x0, int x1, int y0, int y1, const WPlan &pl, WSmem &b) {
    constexpr int NC = GAUGE ? 7 : 1;
    const int lane = threadIdx.x & 31;
    const int Lx = X.Lab, Ly = Y.Lab;
    const int nhx = nherm(Lx), nhy = nherm(Ly);
    const int L = Lx + Ly, Lr = L + 2, Ltop = GAUGE ? Lr : L;
    const int xch = x1 - x0, ych = y1 - y0;
    for (int h = lane; h < nhx; h += 32) htrip_d(h, b.trX[3 * h], b.trX[3 * h + 1], b.trX[3 * h + 2]);
    for (int h = lane; h < nhy; h += 32) htrip_d(h, b.trY[3 * h], b.trY[3 * h + 1], b.trY[3 * h + 2]);
    for (int i = lane; i < NC * xch * ych; i += 32) b.G[i] = 0.0;
    __syncwarp();
    for (int ij = 0; ij < X.npp; ++ij) {
        const PrimPairDev pa = pp[X.ppoff + ij];
        for (int i = lane; i < NC * nhx * ych; i += 32) b.T[i] = 0.0;
        for (int g0 = 0; g0 < Y.npp; g0 += kWGroup) {
            const int ng = min(kWGroup, Y.npp - g0);
            // Boys values of up to kWGroup primitive quartets, one per lane
            if (lane < ng) {
                const PrimPairDev pc = pp[Y.ppoff + g0 + lane];
                double p = pa.p, q = pc.p, rho = p * q / (p + q);
                double Xq = pa.P[0] - pc.P[0], Yq = pa.P[1] - pc.P[1], Zq = pa.P[2] - pc.P[2];
                double Tv = rho * (Xq * Xq + Yq * Yq + Zq * Zq);
                double *F = b.F + lane * (kBoysNMax + 3);
                boys_eval(boys, Tv, Ltop, F + 1);
                F[0] = -(2.0 * Tv * F[1] + exp(-Tv));
                double *sc = b.sc + lane * 8;
                sc[0] = Xq; sc[1] = Yq; sc[2] = Zq; sc[3] = -2.0 * rho;
                double pw = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
                sc[4] = pw;
                sc[5] = pow(M_PI, 2.5) * sqrt(p + q) / (p * p * q * q);
            }
            __syncwarp();
            for (int g = 0; g < ng; ++g) {
                const double *sc = b.sc + g * 8;
                const double *F = b.F + g * (kBoysNMax + 3);
                const double Xq = sc[0], Yq = sc[1], Zq = sc[2], m2r = sc[3];
                const int nrC = nherm(pl.LtC), nrR = GAUGE ? nherm(pl.LtR) : 0;
                for (int n = Ltop; n >= 0; --n) {
                    const int cntC = (n <= L) ? nherm(L - n) : 0;
                    const int cntR = GAUGE ? nherm(Lr - n) : 0;
                    const int cnt = cntR > cntC ? cntR : cntC;
                    double *dC = b.RC + (n & 1) * nrC, *sC = b.RC + ((n + 1) & 1) * nrC;
                    double *dR = b.RR + (n & 1) * nrR, *sR = b.RR + ((n + 1) & 1) * nrR;
                    for (int h = lane; h < cnt; h += 32) {
                        int t, u, v;
                        htrip_d(h, t, u, v);
                        const bool flip = (n == 0) && ((t + u + v) & 1);   // level 0 keeps (-1)^|k| R_k
                        if (h < cntC) {
                            double r;
                            if (h == 0) {
                                double mp = 1.0;                 // (-2 rho)^n
                                for (int k = 0; k < n; ++k) mp *= m2r;
                                r = mp * F[n + 1] * sc[4];
                            }
                            else if (t > 0) r = (t > 1 ? (t - 1) * sC[hidx(t - 2, u, v)] : 0.0) + Xq * sC[hidx(t - 1, u, v)];
                            else if (u > 0) r = (u > 1 ? (u - 1) * sC[hidx(t, u - 2, v)] : 0.0) + Yq * sC[hidx(t, u - 1, v)];
                            else r = (v > 1 ? (v - 1) * sC[hidx(t, u, v - 2)] : 0.0) + Zq * sC[hidx(t, u, v - 1)];
                            dC[h] = flip ? -r : r;
                        }
                        if (GAUGE && h < cntR) {
                            double r;
                            if (h == 0) {
                                double mp = 1.0;
                                for (int k = 0; k < n; ++k) mp *= m2r;
                                r = mp * (F[n + 1] - F[n]) * sc[5];
                            }
                            else if (t > 0) r = (t > 1 ? (t - 1) * sR[hidx(t - 2, u, v)] : 0.0) + Xq * sR[hidx(t - 1, u, v)];
                            else if (u > 0) r = (u > 1 ? (u - 1) * sR[hidx(t, u - 2, v)] : 0.0) + Yq * sR[hidx(t, u - 1, v)];
                            else r = (v > 1 ? (v - 1) * sR[hidx(t, u, v - 2)] : 0.0) + Zq * sR[hidx(t, u, v - 1)];
                            dR[h] = flip ? -r : r;
                        }
                    }
                    __syncwarp();
                }
                // T[c][h][y] += (-1)^|h| sum_h' Rs[h+h'] E^{kl}[h'][y]
                const double *e = E + pp[Y.ppoff + g0 + g].eoff + y0;
                const double *RC0 = b.RC, *RR0 = b.RR;
                for (int idx = lane; idx < nhx * ych; idx += 32) {
                    const int h = idx / ych, yy = idx - h * ych;
                    const int t = b.trX[3 * h], u = b.trX[3 * h + 1], v = b.trX[3 * h + 2];
                    double s0 = 0.0, s6[6] = {0, 0, 0, 0, 0, 0};
                    for (int hp = 0; hp < nhy; ++hp) {
                        const int T0 = t + b.trY[3 * hp], U0 = u + b.trY[3 * hp + 1], V0 = v + b.trY[3 * hp + 2];
                        const double ev = __ldg(e + (size_t)hp * Y.nfp + yy);
                        s0 = fma(RC0[hidx(T0, U0, V0)], ev, s0);
                        if (GAUGE) {
                            s6[0] = fma(RR0[hidx(T0 + 2, U0, V0)], ev, s6[0]);
                            s6[1] = fma(RR0[hidx(T0 + 1, U0 + 1, V0)], ev, s6[1]);
                            s6[2] = fma(RR0[hidx(T0 + 1, U0, V0 + 1)], ev, s6[2]);
                            s6[3] = fma(RR0[hidx(T0, U0 + 2, V0)], ev, s6[3]);
                            s6[4] = fma(RR0[hidx(T0, U0 + 1, V0 + 1)], ev, s6[4]);
                            s6[5] = fma(RR0[hidx(T0, U0, V0 + 2)], ev, s6[5]);
                        }
                    }
                    const bool odd = (t + u + v) & 1;
                    b.T[(size_t)h * ych + yy] += odd ? -s0 : s0;
                    if (GAUGE)
                        for (int k = 0; k < 6; ++k) b.T[((size_t)(k + 1) * nhx + h) * ych + yy] += odd ? -s6[k] : s6[k];
                }
                __syncwarp();
            }
        }
        // G[c][x][y] += sum_h E^{ij}[h][x] T[c][h][y]
        const double *Eij = E + pa.eoff + x0;
        for (int idx = lane; idx < xch * ych; idx += 32) {
            const int xx = idx / ych, yy = idx - xx * ych;
            double s[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) s[k] = 0.0;
            for (int h = 0; h < nhx; ++h) {
                const double ev = __ldg(Eij + (size_t)h * X.nfp + xx);
#pragma unroll
                for (int k = 0; k < NC; ++k) s[k] = fma(ev, b.T[((size_t)k * nhx + h) * ych + yy], s[k]);
            }
#pragma unroll
            for (int k = 0; k < NC; ++k) b.G[((size_t)k * xch + xx) * ych + yy] += s[k];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ GEMM engine
// For Hermite orders <= 4 per pair (s and p shells and their derivatives) the
// two contractions of a block are dense register-blocked FP64 micro-GEMMs:
//   T[h][y] += Rt[h][h'] E^{kl}[h'][y],   Rt[h][h'] = Rs[h + h'] (one primitive quartet)
//   G[x][y] += E^{ij}[h][x] T[h][y]
// Each of 128 threads owns a 4 x 4 block of T and of G in registers; Rt and E
// are staged k-major in shared memory so one k step is 8 loads for 16 FMAs.
// The gauge kernel runs its seven components one after the other.
constexpr int kDM = 4;          // Hermite order limit of a pair for this engine (nherm 35)
constexpr int kGT = 36;         // function pairs per chunk side (9 blocks of 4)
constexpr int kGH = 36;         // nherm(4) = 35 padded to blocks of 4

struct GSmem {
    double *Rt;      // [kGH (h')][kGH (h)]  k-major
    double *Ek;      // [kGH (h')][kGT (y)]
    double *T;       // [kGH (h)][kGT (y)]
    double *Ei;      // [kGH (h)][kGT (x)]
    double *RB;      // recursion ping-pong
    double *F, *sc;
    int *trX, *trY;
};

__host__ __device__ inline int gsmem_doubles(int Lt) {
    return kGH * kGH + 3 * kGH * kGT + 2 * nherm(Lt) + kWGroup * (kBoysNMax + 3) + kWGroup * 8 + 105 + 2;
}

__device__ inline GSmem gcarve(double *sm, int Lt) {
    GSmem b;
    b.Rt = sm; sm += kGH * kGH;
    b.Ek = sm; sm += kGH * kGT;
    b.T = sm; sm += kGH * kGT;
    b.Ei = sm; sm += kGH * kGT;
    b.RB = sm; sm += 2 * nherm(Lt);
    b.F = sm; sm += kWGroup * (kBoysNMax + 3);
    b.sc = sm; sm += kWGroup * 8;
    b.trX = (int *)sm;
    b.trY = b.trX + 3 * 35;
    return b;
}

// One chunk of block (X|Y), component comp (0: 1/r12; 1..6: r12 shifted by
// e_I + e_J); returns this thread's 4 x 4 block of G (rows x = 4 bi + r,
// columns y = 4 bj + c with bi = tid / 9, bj = tid % 9; tid >= 81 idle).
template <bool GAUGE>
__device__ void gemm_chunk(const PrimPairDev *pp, const double *E, const double *boys, const PairDev &X,
                           const PairDev &Y, int x0, int x1, int y0, int y1, int Lt, int comp, GSmem &b,
                           double g[4][4]) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int bi = tid / 9, bj = tid - 9 * bi;
    const bool act = tid < 81;
    const int Lx = X.Lab, Ly = Y.Lab;
    const int nhx = nherm(Lx), nhy = nherm(Ly);
    const int L = Lx + Ly;
    const bool useR = GAUGE && comp > 0;
    const int Ltop = useR ? L + 2 : L;
    const int xch = x1 - x0, ych = y1 - y0;
    const int nr = nherm(Lt);
    int dx = 0, dy = 0, dz = 0;
    if (useR) {
        const int IJ[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        const int I = IJ[comp - 1][0], J = IJ[comp - 1][1];
        dx = (I == 0) + (J == 0); dy = (I == 1) + (J == 1); dz = (I == 2) + (J == 2);
    }
    for (int h = tid; h < nhx; h += nt) htrip_d(h, b.trX[3 * h], b.trX[3 * h + 1], b.trX[3 * h + 2]);
    for (int h = tid; h < nhy; h += nt) htrip_d(h, b.trY[3 * h], b.trY[3 * h + 1], b.trY[3 * h + 2]);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) g[r][c] = 0.0;
    __syncthreads();
    for (int ij = 0; ij < X.npp; ++ij) {
        const PrimPairDev pa = pp[X.ppoff + ij];
        double t[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) t[r][c] = 0.0;
        for (int g0 = 0; g0 < Y.npp; g0 += kWGroup) {
            const int ng = min(kWGroup, Y.npp - g0);
            if (tid < ng) {
                const PrimPairDev pc = pp[Y.ppoff + g0 + tid];
                double p = pa.p, q = pc.p, rho = p * q / (p + q);
                double Xq = pa.P[0] - pc.P[0], Yq = pa.P[1] - pc.P[1], Zq = pa.P[2] - pc.P[2];
                double Tv = rho * (Xq * Xq + Yq * Yq + Zq * Zq);
                double *F = b.F + tid * (kBoysNMax + 3);
                boys_eval(boys, Tv, Ltop, F + 1);
                F[0] = -(2.0 * Tv * F[1] + exp(-Tv));
                double *sc = b.sc + tid * 8;
                sc[0] = Xq; sc[1] = Yq; sc[2] = Zq; sc[3] = -2.0 * rho;
                sc[4] = useR ? pow(M_PI, 2.5) * sqrt(p + q) / (p * p * q * q) : 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
            }
            __syncthreads();
            for (int g = 0; g < ng; ++g) {
                const double *sc = b.sc + g * 8;
                const double *F = b.F + g * (kBoysNMax + 3);
                const double Xq = sc[0], Yq = sc[1], Zq = sc[2], m2r = sc[3];
                for (int n = Ltop; n >= 0; --n) {
                    const int cnt = nherm(Ltop - n);
                    double *d = b.RB + (n & 1) * nr, *s = b.RB + ((n + 1) & 1) * nr;
                    for (int h = tid; h < cnt; h += nt) {
                        int tt, u, v;
                        htrip_d(h, tt, u, v);
                        double r;
                        if (h == 0) {
                            double mp = 1.0;
                            for (int k = 0; k < n; ++k) mp *= m2r;
                            r = mp * (useR ? F[n + 1] - F[n] : F[n + 1]) * sc[4];
                        } else if (tt > 0) r = (tt > 1 ? (tt - 1) * s[hidx(tt - 2, u, v)] : 0.0) + Xq * s[hidx(tt - 1, u, v)];
                        else if (u > 0) r = (u > 1 ? (u - 1) * s[hidx(tt, u - 2, v)] : 0.0) + Yq * s[hidx(tt, u - 1, v)];
                        else r = (v > 1 ? (v - 1) * s[hidx(tt, u, v - 2)] : 0.0) + Zq * s[hidx(tt, u, v - 1)];
                        d[h] = (n == 0 && ((tt + u + v) & 1)) ? -r : r;     // level 0 keeps (-1)^|k| R_k
                    }
                    __syncthreads();
                }
                // stage Rt (k-major) and E^{kl}, zero padded
                const double *ekl = E + pp[Y.ppoff + g0 + g].eoff;
                for (int i = tid; i < kGH * kGH; i += nt) {
                    const int hp = i / kGH, h = i - hp * kGH;
                    double v = 0.0;
                    if (h < nhx && hp < nhy)
                        v = b.RB[hidx(b.trX[3 * h] + b.trY[3 * hp] + dx, b.trX[3 * h + 1] + b.trY[3 * hp + 1] + dy,
                                      b.trX[3 * h + 2] + b.trY[3 * hp + 2] + dz)];
                    b.Rt[i] = v;
                }
                for (int i = tid; i < kGH * kGT; i += nt) {
                    const int hp = i / kGT, y = i - hp * kGT;
                    b.Ek[i] = (hp < nhy && y < ych) ? __ldg(ekl + (size_t)hp * Y.nfp + y0 + y) : 0.0;
                }
                __syncthreads();
                if (act) {
                    for (int k = 0; k < nhy; ++k) {
                        const double2 a01 = *reinterpret_cast<const double2 *>(b.Rt + k * kGH + 4 * bi);
                        const double2 a23 = *reinterpret_cast<const double2 *>(b.Rt + k * kGH + 4 * bi + 2);
                        const double2 e01 = *reinterpret_cast<const double2 *>(b.Ek + k * kGT + 4 * bj);
                        const double2 e23 = *reinterpret_cast<const double2 *>(b.Ek + k * kGT + 4 * bj + 2);
                        const double a[4] = {a01.x, a01.y, a23.x, a23.y}, ev[4] = {e01.x, e01.y, e23.x, e23.y};
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) t[r][c] = fma(a[r], ev[c], t[r][c]);
                    }
                }
                __syncthreads();
            }
        }
        // T with the sign (-1)^|h| of its row, and E^{ij}, into shared memory
        if (act) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int h = 4 * bi + r;
                const bool odd = h < nhx && ((b.trX[3 * h] + b.trX[3 * h + 1] + b.trX[3 * h + 2]) & 1);
#pragma unroll
                for (int c = 0; c < 4; ++c) b.T[h * kGT + 4 * bj + c] = odd ? -t[r][c] : t[r][c];
            }
        }
        const double *eij = E + pa.eoff;
        for (int i = tid; i < kGH * kGT; i += nt) {
            const int h = i / kGT, x = i - h * kGT;
            b.Ei[i] = (h < nhx && x < xch) ? __ldg(eij + (size_t)h * X.nfp + x0 + x) : 0.0;
        }
        __syncthreads();
        if (act) {
            for (int k = 0; k < nhx; ++k) {
                const double2 a01 = *reinterpret_cast<const double2 *>(b.Ei + k * kGT + 4 * bi);
                const double2 a23 = *reinterpret_cast<const double2 *>(b.Ei + k * kGT + 4 * bi + 2);
                const double2 t01 = *reinterpret_cast<const double2 *>(b.T + k * kGT + 4 * bj);
                const double2 t23 = *reinterpret_cast<const double2 *>(b.T + k * kGT + 4 * bj + 2);
                const double a[4] = {a01.x, a01.y, a23.x, a23.y}, tv[4] = {t01.x, t01.y, t23.x, t23.y};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) g[r][c] = fma(a[r], tv[c], g[r][c]);
            }
        }
        __syncthreads();
    }
}

template <bool GAUGE>
__global__ void __launch_bounds__(128) eri_rows_gemm_kernel(EriParams prm, const EriTask *tasks, int Lt) {
    extern __shared__ double sm[];
    const EriTask tk = tasks[blockIdx.x];
    const PairDev AB = prm.pairs[tk.bra_sp];
    const int tid = threadIdx.x, bi = tid / 9, bj = tid - 9 * bi;
    GSmem b = gcarve(sm, Lt);
    const int IJ[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int kp = tk.k0; kp < tk.k1; ++kp) {
        const int cd_id = prm.ket_sp[kp];
        const PairDev CD = prm.pairs[cd_id];
        const long long col = prm.ket_col[kp];
        const bool rev = prm.sym && cd_id != tk.bra_sp && prm.ket_pos[tk.bra_sp] < prm.prefix[cd_id];
        if (rev && cd_id < tk.bra_sp) continue;
        const long long col_rev = rev ? prm.ket_col[prm.ket_pos[tk.bra_sp]] : 0;
        const bool swap = orient_cost(CD, AB) < orient_cost(AB, CD);
        const PairDev &X = swap ? CD : AB, &Y = swap ? AB : CD;
        for (int x0 = 0; x0 < X.nfp; x0 += kGT) {
            const int x1 = min(X.nfp, x0 + kGT);
            for (int y0 = 0; y0 < Y.nfp; y0 += kGT) {
                const int y1 = min(Y.nfp, y0 + kGT);
                const int ncomp = GAUGE ? 7 : 1;
                for (int comp = 0; comp < ncomp; ++comp) {
                    double g[4][4];
                    gemm_chunk<GAUGE>(prm.pp, prm.E, prm.boys, X, Y, x0, x1, y0, y1, Lt, comp, b, g);
                    if (tid >= 81) continue;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int xx = 4 * bi + r, yy = 4 * bj + c;
                            if (x0 + xx >= x1 || y0 + yy >= y1) continue;
                            const int a = swap ? y0 + yy : x0 + xx;
                            const int cq = swap ? x0 + xx : y0 + yy;
                            const long long row = AB.rowoff + a - prm.row0, cc = col + cq;
                            const long long row2 = rev ? CD.rowoff + cq - prm.row0 : 0, cc2 = col_rev + a;
                            const double v = g[r][c];
                            if (!GAUGE) {
                                prm.W[row * prm.ldw + cc] = v;
                                if (rev) prm.W[row2 * prm.ldw + cc2] = v;
                            } else if (comp == 0) {
                                // Coulomb part: Gaunt block and the delta_IJ term of the gauge kernel
                                for (int I = 0; I < 3; ++I)
                                    for (int J = 0; J < 3; ++J) {
                                        const double w = I == J ? v : 0.0;
                                        prm.W[(row * 3 + I) * prm.ldw + cc * 3 + J] = w;
                                        if (rev) prm.W[(row2 * 3 + I) * prm.ldw + cc2 * 3 + J] = w;
                                    }
                                if (prm.with_coulomb) {
                                    prm.Wc[row * prm.ldwc + cc] = v;
                                    if (rev) prm.Wc[row2 * prm.ldwc + cc2] = v;
                                }
                            } else {
                                // - (xy|d_I d_J r|zw), symmetric in I, J and in the electrons
                                const int I = IJ[comp - 1][0], J = IJ[comp - 1][1];
                                prm.W[(row * 3 + I) * prm.ldw + cc * 3 + J] -= v;
                                if (I != J) prm.W[(row * 3 + J) * prm.ldw + cc * 3 + I] -= v;
                                if (rev) {
                                    prm.W[(row2 * 3 + I) * prm.ldw + cc2 * 3 + J] -= v;
                                    if (I != J) prm.W[(row2 * 3 + J) * prm.ldw + cc2 * 3 + I] -= v;
                                }
                            }
                        }
                }
            }
        }
    }
}

bool eri_gemm_fits(int maxLab) { return maxLab <= kDM; }

// Screened rows: one CTA per task (bra shell pair x range of sorted ket
// positions); the CTA's warps take the ket positions round robin.
template <bool GAUGE>
__global__ void __launch_bounds__(128) eri_rows_kernel(EriParams prm, const EriTask *tasks, WPlan pl) {
    extern __shared__ double sm[];
    const EriTask tk = tasks[blockIdx.x];
    const PairDev AB = prm.pairs[tk.bra_sp];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WSmem b = wcarve(sm + (size_t)warp * pl.warp_doubles, pl);
    const int ij_of[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int kp = tk.k0 + warp; kp < tk.k1; kp += pl.nwarps) {
        const int cd_id = prm.ket_sp[kp];
        const PairDev CD = prm.pairs[cd_id];
        const long long col = prm.ket_col[kp];
        // (CD|AB) also kept?  Then the lower pair id computes both blocks.
        const bool rev = prm.sym && cd_id != tk.bra_sp && prm.ket_pos[tk.bra_sp] < prm.prefix[cd_id];
        if (rev && cd_id < tk.bra_sp) continue;
        const long long col_rev = rev ? prm.ket_col[prm.ket_pos[tk.bra_sp]] : 0;
        const bool swap = orient_cost(CD, AB) < orient_cost(AB, CD);
        const PairDev &X = swap ? CD : AB, &Y = swap ? AB : CD;
        for (int x0 = 0; x0 < X.nfp; x0 += pl.ach) {
            const int x1 = min(X.nfp, x0 + pl.ach);
            for (int y0 = 0; y0 < Y.nfp; y0 += pl.cch) {
                const int y1 = min(Y.nfp, y0 + pl.cch);
                warp_chunk<GAUGE>(prm.pp, prm.E, prm.boys, X, Y, x0, x1, y0, y1, pl, b);
                const int xch = x1 - x0, ych = y1 - y0;
                for (int idx = lane; idx < xch * ych; idx += 32) {
                    const int xx = idx / ych, yy = idx - xx * ych;
                    const int a = swap ? y0 + yy : x0 + xx;      // bra function pair
                    const int c = swap ? x0 + xx : y0 + yy;      // ket function pair
                    const long long row = AB.rowoff + a - prm.row0;
                    const long long cc = col + c;
                    const double C = b.G[idx];
                    if (!GAUGE) {
                        prm.W[row * prm.ldw + cc] = C;
                        if (rev) prm.W[(CD.rowoff + c - prm.row0) * prm.ldw + col_rev + a] = C;
                    } else {
                        const double *H = b.G + (size_t)xch * ych;
                        for (int I = 0; I < 3; ++I)
                            for (int J = 0; J < 3; ++J) {
                                // K_IJ is symmetric in I, J and in the two electrons
                                const double v = (I == J ? C : 0.0) - H[(size_t)ij_of[I][J] * xch * ych + idx];
                                prm.W[(row * 3 + I) * prm.ldw + cc * 3 + J] = v;
                                if (rev) prm.W[((CD.rowoff + c - prm.row0) * 3 + I) * prm.ldw + (col_rev + a) * 3 + J] = v;
                            }
                        if (prm.with_coulomb) {
                            prm.Wc[row * prm.ldwc + cc] = C;
                            if (rev) prm.Wc[(CD.rowoff + c - prm.row0) * prm.ldwc + col_rev + a] = C;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

WPlan eri_wplan(int maxnfp, int maxLab, bool gauge, size_t *smem) {
    WPlan p;
    p.NC = gauge ? 7 : 1;
    p.ach = p.cch = maxnfp;
    p.nhMax = nherm(maxLab);
    p.LtC = 2 * maxLab;
    p.LtR = gauge ? 2 * maxLab + 2 : -1;
    // doubles per warp: Coulomb 18 KB (3 CTAs of 4 warps per SM); the gauge
    // kernel's seven components get 24 KB so its chunks stay large enough that
    // the Hermite recursion is not repeated too often
    const int per_warp_budget = (gauge ? 24 : 18) * 1024 / 8;
    while (wplan_doubles(p.NC, p.ach, p.cch, p.nhMax, p.LtC, p.LtR) > per_warp_budget && p.ach > 4) {
        p.ach = (p.ach + 1) / 2;
        p.cch = (p.cch + 1) / 2;
    }
    p.warp_doubles = (wplan_doubles(p.NC, p.ach, p.cch, p.nhMax, p.LtC, p.LtR) + 31) & ~31;
    p.nwarps = 4;
    while (p.nwarps > 1 && (size_t)p.nwarps * p.warp_doubles * 8 > 200 * 1024) --p.nwarps;
    *smem = (size_t)p.nwarps * p.warp_doubles * 8;
    return p;
}

void launch_eri(const EriParams &prm, const EriTask *tasks, int ntasks, int maxnfp, int maxLab, int maxnpp,
                cudaStream_t s) {
    (void)maxnpp;
    if (ntasks <= 0) return;
    if (eri_gemm_fits(maxLab)) {
        const int Lt = 2 * maxLab + (prm.gauge ? 2 : 0);
        const size_t smem = (size_t)gsmem_doubles(Lt) * 8;
        if (prm.gauge) {
            QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            eri_rows_gemm_kernel<true><<<ntasks, 128, smem, s>>>(prm, tasks, Lt);
        } else {
            QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            eri_rows_gemm_kernel<false><<<ntasks, 128, smem, s>>>(prm, tasks, Lt);
        }
        QDT_CHECK_LAUNCH();
        return;
    }
    size_t smem;
    WPlan pl = eri_wplan(maxnfp, maxLab, prm.gauge != 0, &smem);
    const int threads = 32 * pl.nwarps;
    if (prm.gauge) {
        QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        eri_rows_kernel<true><<<ntasks, threads, smem, s>>>(prm, tasks, pl);
    } else {
        QDT_CUDA_TRY(cudaFuncSetAttribute(eri_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        eri_rows_kernel<false><<<ntasks, threads, smem, s>>>(prm, tasks, pl);
    }
    QDT_CHECK_LAUNCH();
}

// CTA-level plan of block_chunk (used by the Schwarz kernel).
Plan eri_plan(int maxnfp, int maxLab, int maxnpp, bool gauge, size_t *smem) {
    Plan p;
    p.NC = gauge ? 7 : 1;
    p.ach = p.cch = maxnfp;
    p.nhMax = nherm(maxLab);
    p.LtC = 2 * maxLab;
    p.LtR = gauge ? 2 * maxLab + 2 : -1;
    p.klg = maxnpp < 16 ? (maxnpp > 0 ? maxnpp : 1) : 16;
    const size_t budget = 110 * 1024;
    while (eri_smem_bytes(p) > budget && (p.ach > 16 || p.klg > 2)) {
        if (p.klg > 4) p.klg = (p.klg + 1) / 2;
        else { p.ach = (p.ach + 1) / 2; p.cch = (p.cch + 1) / 2; }
    }
    *smem = eri_smem_bytes(p);
    return p;
}

// Schwarz diagonals: Q[AB] = max over ab of sqrt(|(ab|ab)|), Coulomb kernel.
__global__ void __launch_bounds__(256) schwarz_kernel(const PrimPairDev *pp, const PairDev *pairs, const double *E,
                                                      const double *boys, Plan pl, double *Q) {
    extern __shared__ double sm[];
    const PairDev AB = pairs[blockIdx.x];
    BlockSmem b = carve(sm, pl);
    double qmax = 0.0;
    for (int a0 = 0; a0 < AB.nfp; a0 += pl.ach) {
        const int a1 = min(AB.nfp, a0 + pl.ach);
        block_chunk<false>(pp, E, boys, AB, AB, a0, a1, a0, a1, pl, b);
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
    size_t smem;
    Plan pl = eri_plan(maxnfp, maxLab, maxnpp, false, &smem);
    pl.cch = pl.ach;
    QDT_CUDA_TRY(cudaFuncSetAttribute(schwarz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    schwarz_kernel<<<npairs, 256, smem, s>>>(pp, pairs, E, boys, pl, Q);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
