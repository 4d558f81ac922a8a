// qdt_api.cu -- the C ABI of libqdt (include/qdt.h): context, basis set-up,
// coefficients and the AO-driven direct transformation driver.
//
// Pipeline of one block class (paper Sec. 2.4 and 2.5):
//   1. quaternion pair density D (Eqs. Den, QuaternionScatter), rows in bra
//      order (shell pairs by Schwarz Q descending), plus Dmax per shell pair;
//   2. ket order: w = Q * Dmax descending; every bra pair keeps a ket prefix
//      (Eq. SchwarzDen), so screening is a ragged K extent per row tile;
//   3. for bra row batches: AO integral rows of the kept quartets (stage i),
//      then V = W D_ket (first half, Eq. firsthalf);
//   4. O = D^T V over all rows (second half, Eq. secondhalf, real form);
//   5. pack the canonical Kramers quadruples.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "qdt_internal.cuh"
#include "split.cuh"

namespace qdt {
void launch_prim_pairs_map(const ShellDev *shells, const PairDev *pairs, const int *pp_pair,
                           long long npp, const double *exps, const double *coefs,
                           const double *norms, PrimPairDev *pp, double *E, cudaStream_t s);
void launch_density(bool gaunt, const PairDev *pairs, const int *bra_order, int nsp,
                    const ShellDev *shells, const double *Cq, int nK, int k0, const int *rsR,
                    const int *rsS, int nRS, double *D, double *Dmax, cudaStream_t s);
}  // namespace qdt

using namespace qdt;

namespace {

// Device buffer that only grows; freed with the context.
struct DBuf {
    void *p = nullptr;
    size_t n = 0;
    void *get(size_t bytes) {
        if (bytes <= n && p) return p;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (bytes == 0) return nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            throw Error{QDT_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
        }
        n = bytes;
        return p;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <class T>
T *dcopy(DBuf &b, const std::vector<T> &v, cudaStream_t s) {
    T *d = (T *)b.get(std::max<size_t>(1, v.size()) * sizeof(T));
    if (!v.empty()) QDT_CUDA_TRY(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return d;
}

struct ClassBufs {
    DBuf pairs, pp, E, Q, bra, pp_pair;
};

}  // namespace

struct qdt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    // basis
    bool has_basis = false;
    int nL = 0, nS = 0, nshL = 0;
    std::vector<ShellDev> h_shells;
    std::vector<double> h_exps;
    DBuf shells, exps, coefs, norms, boys;
    PairClass cls[2];
    ClassBufs cb[2];
    // coefficients (internal rows: L functions, then the distinct derivative functions)
    bool has_coef = false;
    int nK = 0;
    DBuf Cq, Craw, dsmap0, dsmap1;
    std::vector<int> smap0, smap1;
    // per-transform workspace
    DBuf Dbra, Dket, V, Vg, W, Wc, Dmax, wsort, ketsp, ketcol, prefix, ktile, tasks, O, partial,
        stage, rsR, rsS, kpos;
    SplitWorkspace split;
    cudaEvent_t ev[16];
    int launches = 0;
};

namespace {

int fail(qdt_ctx *c, const Error &e) {
    if (c) c->err = e.msg;
    return e.code;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int lcart(int l) { return (l + 1) * (l + 2) / 2; }

// FP64 multiply-adds of the E R E contraction of one shell quartet with X as
// the outer (per primitive pair) side.
double orient_cost_h(const PairDev &X, const PairDev &Y) {
    double nhx = nherm(X.Lab), nhy = nherm(Y.Lab);
    return (double)X.npp * Y.npp * nhx * Y.nfp * nhy + (double)X.npp * X.nfp * Y.nfp * nhx;
}

// Build the shell-pair tables of class `c` (0: LL+SS, 1: LS); pairs in natural
// order, primitive pairs and E offsets.
void build_class(qdt_ctx *ctx, int c) {
    PairClass &pc = ctx->cls[c];
    pc = PairClass();
    const int n = ctx->nshL;
    std::vector<std::pair<int, int>> sp;
    if (c == 0) {
        for (int off = 0; off <= n; off += n)
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b) sp.push_back({a + off, b + off});
    } else {
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) sp.push_back({a, b + n});
    }
    pc.nsp = (int)sp.size();
    std::vector<PrimPairDev> hpp;
    std::vector<int> pp_pair;
    long long eoff = 0, M = 0;
    for (int i = 0; i < pc.nsp; ++i) {
        const ShellDev &A = ctx->h_shells[sp[i].first], &B = ctx->h_shells[sp[i].second];
        PairDev pr;
        pr.sa = sp[i].first;
        pr.sb = sp[i].second;
        pr.nfp = (pr.sa == pr.sb) ? A.nfunc * (A.nfunc + 1) / 2 : A.nfunc * B.nfunc;
        pr.Lab = (A.l + A.isS) + (B.l + B.isS);
        pr.ppoff = (int)hpp.size();
        pr.rowoff = 0;
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) r2 += (A.A[d] - B.A[d]) * (A.A[d] - B.A[d]);
        for (int ia = 0; ia < A.nprim; ++ia)
            for (int ib = 0; ib < B.nprim; ++ib) {
                double a = ctx->h_exps[A.poff + ia], bb = ctx->h_exps[B.poff + ib];
                if (std::exp(-a * bb / (a + bb) * r2) < kPrimPairTol) continue;
                PrimPairDev q{};
                q.eoff = eoff;
                q.ia = ia;
                q.ib = ib;
                eoff += (long long)pr.nfp * nherm(pr.Lab);
                hpp.push_back(q);
                pp_pair.push_back(i);
            }
        pr.npp = (int)hpp.size() - pr.ppoff;
        pc.maxnpp = std::max(pc.maxnpp, pr.npp);
        M += pr.nfp;
        pc.maxnfp = std::max(pc.maxnfp, pr.nfp);
        pc.maxLab = std::max(pc.maxLab, pr.Lab);
        pc.h_pairs.push_back(pr);
    }
    pc.M = M;
    pc.npp_total = (long long)hpp.size();
    pc.e_total = eoff;
    cudaStream_t s = ctx->stream;
    ClassBufs &b = ctx->cb[c];
    pc.d_pairs = dcopy(b.pairs, pc.h_pairs, s);
    pc.d_pp = dcopy(b.pp, hpp, s);
    int *d_ppp = dcopy(b.pp_pair, pp_pair, s);
    pc.d_E = (double *)b.E.get(std::max<long long>(1, eoff) * sizeof(double));
    launch_prim_pairs_map(ctx->shells.p ? (const ShellDev *)ctx->shells.p : nullptr, pc.d_pairs, d_ppp,
                          pc.npp_total, (const double *)ctx->exps.p, (const double *)ctx->coefs.p,
                          (const double *)ctx->norms.p, pc.d_pp, pc.d_E, s);
    ctx->launches++;
    // Schwarz diagonals, then the bra order (Q descending, ties by id)
    pc.d_Q = (double *)b.Q.get(std::max(1, pc.nsp) * sizeof(double));
    launch_schwarz((const ShellDev *)ctx->shells.p, pc.d_pairs, pc.d_pp, pc.d_E,
                   (const double *)ctx->boys.p, pc.nsp, pc.maxnfp, pc.maxLab, pc.maxnpp, pc.d_Q, s);
    ctx->launches++;
    pc.h_Q.resize(pc.nsp);
    QDT_CUDA_TRY(cudaMemcpyAsync(pc.h_Q.data(), pc.d_Q, pc.nsp * sizeof(double), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
    pc.bra_order.resize(pc.nsp);
    std::iota(pc.bra_order.begin(), pc.bra_order.end(), 0);
    std::stable_sort(pc.bra_order.begin(), pc.bra_order.end(),
                     [&](int x, int y) { return pc.h_Q[x] > pc.h_Q[y]; });
    long long row = 0;
    for (int k = 0; k < pc.nsp; ++k) {
        PairDev &pr = pc.h_pairs[pc.bra_order[k]];
        pr.rowoff = row;
        row += pr.nfp;
    }
    QDT_CUDA_TRY(cudaMemcpyAsync(pc.d_pairs, pc.h_pairs.data(), pc.nsp * sizeof(PairDev),
                                 cudaMemcpyHostToDevice, s));
    pc.d_bra_order = dcopy(b.bra, pc.bra_order, s);
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
}

struct Timer {
    qdt_ctx *c;
    int n = 0;
    explicit Timer(qdt_ctx *cc) : c(cc) {}
    void mark() {
        if (n < 16) QDT_CUDA_TRY(cudaEventRecord(c->ev[n++], c->stream));
    }
    double ms(int a, int b) {
        float t = 0.f;
        if (a < n && b < n && cudaEventElapsedTime(&t, c->ev[a], c->ev[b]) != cudaSuccess) {
            cudaGetLastError();   // a timing failure must not surface as a later launch error
            t = 0.f;
        }
        return t;
    }
};

// One block class of a transformation.  Returns the device pointer of the
// packed block written into `outp`.
struct ClassRun {
    int c;                  // pair class
    bool coulomb = false, gaunt = false, gauge = false;
};

void run_class(qdt_ctx *ctx, const ClassRun &cr, int k0, int nKa, double tau, int precision,
               double *out_coul, double *out_gaunt, double *out_gauge, qdt_stats *st, Timer &tm,
               double acc_ms[6]) {
    PairClass &pc = ctx->cls[cr.c];
    cudaStream_t s = ctx->stream;
    const int nRS = nKa * (nKa + 1) / 2;
    const bool ls = cr.c == 1;
    const long long N4 = 4LL * nRS;              // columns per J component
    const long long ncolD = ls ? 3 * N4 : N4;     // density row length
    const long long M = pc.M;
    // Kramers pair list
    std::vector<int> hR, hS;
    for (int r = 0; r < nKa; ++r)
        for (int q = r; q < nKa; ++q) { hR.push_back(r); hS.push_back(q); }
    int *d_rsR = dcopy(ctx->rsR, hR, s), *d_rsS = dcopy(ctx->rsS, hS, s);
    split_invalidate(ctx->split);

    // 1. density in bra order + Dmax
    int t0 = tm.n; tm.mark();
    double *Dbra = (double *)ctx->Dbra.get(std::max<long long>(1, M * ncolD) * sizeof(double));
    double *Dmax = (double *)ctx->Dmax.get(std::max(1, pc.nsp) * sizeof(double));
    QDT_CUDA_TRY(cudaMemsetAsync(Dmax, 0, pc.nsp * sizeof(double), s));
    launch_density(ls, pc.d_pairs, pc.d_bra_order, pc.nsp, (const ShellDev *)ctx->shells.p,
                   (const double *)ctx->Cq.p, ctx->nK, k0, d_rsR, d_rsS, nRS, Dbra, Dmax, s);
    ctx->launches++;
    tm.mark();
    // 2. ket order and prefixes
    double *wsort = (double *)ctx->wsort.get(std::max(1, pc.nsp) * sizeof(double));
    int *ketsp = (int *)ctx->ketsp.get(std::max(1, pc.nsp) * sizeof(int));
    long long *ketcol = (long long *)ctx->ketcol.get((pc.nsp + 1) * sizeof(long long));
    int *prefix = (int *)ctx->prefix.get(std::max(1, pc.nsp) * sizeof(int));
    launch_ket_order(pc.d_Q, Dmax, pc.nsp, wsort, ketsp, s);
    launch_ket_columns(pc.d_pairs, ketsp, pc.nsp, ketcol, s);
    launch_prefix_lengths(pc.d_Q, wsort, pc.nsp, tau, prefix, s);
    ctx->launches += 3;
    std::vector<int> h_prefix(pc.nsp);
    std::vector<long long> h_col(pc.nsp + 1);
    QDT_CUDA_TRY(cudaMemcpyAsync(h_prefix.data(), prefix, pc.nsp * sizeof(int), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaMemcpyAsync(h_col.data(), ketcol, (pc.nsp + 1) * sizeof(long long), cudaMemcpyDeviceToHost, s));
    std::vector<int> h_ketsp(pc.nsp);
    QDT_CUDA_TRY(cudaMemcpyAsync(h_ketsp.data(), ketsp, pc.nsp * sizeof(int), cudaMemcpyDeviceToHost, s));
    // 3. ket-ordered density copy
    double *Dket = (double *)ctx->Dket.get(std::max<long long>(1, M * ncolD) * sizeof(double));
    launch_gather_rows(Dbra, pc.d_pairs, ketsp, ketcol, pc.nsp, ncolD, Dket, s);
    ctx->launches++;
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
    tm.mark();
    long long kept = 0;
    for (int i = 0; i < pc.nsp; ++i) kept += h_prefix[i];
    if (st) {
        int slot = ls ? 1 : 0;
        st->quartets_total[slot] += (long long)pc.nsp * pc.nsp;
        st->quartets_kept[slot] += kept;
        if (ls && cr.gauge) {
            st->quartets_total[2] += (long long)pc.nsp * pc.nsp;
            st->quartets_kept[2] += kept;
        }
    }

    // 4. batches of bra rows
    const int TMr = gemm_fp64_tile_m();
    // per-row K: K of its shell pair
    std::vector<long long> Krow_pair(pc.nsp);
    for (int i = 0; i < pc.nsp; ++i) Krow_pair[i] = h_col[h_prefix[i]];
    const long long NV = ls ? 3 * N4 : N4;              // V row length (Coulomb / Gaunt)
    double *Vc = nullptr, *Vg = nullptr;
    if (!ls || cr.gaunt) Vc = (double *)ctx->V.get(std::max<long long>(1, M * NV) * sizeof(double));
    if (ls && cr.gauge) Vg = (double *)ctx->Vg.get(std::max<long long>(1, 3 * M * N4) * sizeof(double));
    const long long Kfull = h_col[pc.nsp];
    const int mult = (ls && cr.gauge) ? 3 : 1;          // gauge rows/cols are (pair, I)
    // one batch (and bra-ket symmetry) when all integral rows fit comfortably,
    // else batches of at most 6 GB
    size_t wall = 0;
    {
        long long kmax_all = 0;
        for (int i = 0; i < pc.nsp; ++i) kmax_all = std::max(kmax_all, Krow_pair[i]);
        wall = (size_t)M * mult * (size_t)std::max<long long>(kmax_all, 1) * mult * sizeof(double);
    }
    // all rows at once (bra-ket symmetry) when the integral block and its digit
    // planes fit in 70 % of the device memory this context can use
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
    const size_t usable = (size_t)(0.7 * (double)(fr + ctx->W.n + ctx->Wc.n + split_held_bytes(ctx->split)));
    const double wfac = (precision == QDT_SPLIT ? 2.5 : 1.0) * ((ls && cr.gauge && cr.gaunt) ? 1.12 : 1.0);
    const bool one_batch = (double)wall * wfac <= (double)usable;
    const size_t wbudget = one_batch ? wall : ((size_t)6 << 30);
    std::vector<int> h_kpos(pc.nsp);
    for (int q = 0; q < pc.nsp; ++q) h_kpos[h_ketsp[q]] = q;
    int *d_kpos = one_batch ? dcopy(ctx->kpos, h_kpos, s) : nullptr;
    int b0 = 0;
    double ms_eri = 0, ms_h1 = 0;
    while (b0 < pc.nsp) {
        // grow the batch while the W block fits the budget
        long long rows = 0, kmax = 0;
        int b1 = b0;
        while (b1 < pc.nsp) {
            const PairDev &pr = pc.h_pairs[pc.bra_order[b1]];
            long long k = std::max(kmax, Krow_pair[pc.bra_order[b1]]);
            size_t need = (size_t)(rows + pr.nfp) * mult * (size_t)std::max<long long>(k, 1) * mult * sizeof(double);
            if (b1 > b0 && need > wbudget) break;
            rows += pr.nfp;
            kmax = k;
            ++b1;
        }
        const long long row0 = pc.h_pairs[pc.bra_order[b0]].rowoff;
        const long long ldw = std::max<long long>(kmax, 1) * mult;
        double *W = (double *)ctx->W.get((size_t)rows * mult * ldw * sizeof(double));
        double *Wc = nullptr;
        long long ldwc = std::max<long long>(kmax, 1);
        if (ls && cr.gauge && cr.gaunt) Wc = (double *)ctx->Wc.get((size_t)rows * ldwc * sizeof(double));
        int te = tm.n; tm.mark();
        launch_zero(W, rows * mult * ldw, s);
        if (Wc) launch_zero(Wc, rows * ldwc, s);
        // tasks: bra pair x chunks of its ket prefix
        std::vector<EriTask> tk;
        const int CH = 8;                  // ket positions per task
        for (int k = b0; k < b1; ++k) {
            int sp = pc.bra_order[k];
            for (int q = 0; q < h_prefix[sp]; q += CH) tk.push_back({sp, q, std::min(h_prefix[sp], q + CH)});
        }
        EriTask *d_tk = dcopy(ctx->tasks, tk, s);
        EriParams prm;
        prm.shells = (const ShellDev *)ctx->shells.p;
        prm.pairs = pc.d_pairs;
        prm.pp = pc.d_pp;
        prm.E = pc.d_E;
        prm.boys = (const double *)ctx->boys.p;
        prm.ket_sp = ketsp;
        prm.ket_col = ketcol;
        prm.W = W;
        prm.ldw = ldw;
        prm.row0 = row0;
        prm.gauge = (ls && cr.gauge) ? 1 : 0;
        prm.with_coulomb = Wc ? 1 : 0;
        prm.Wc = Wc;
        prm.ldwc = ldwc;
        prm.sym = one_batch ? 1 : 0;
        prm.ket_pos = d_kpos;
        prm.prefix = prefix;
        launch_eri(prm, d_tk, (int)tk.size(), pc.maxnfp, pc.maxLab, pc.maxnpp, s);
        ctx->launches += 2 + (Wc ? 1 : 0);
        if (st) {
            long long v = 0;
            double fl = 0.0;
            const int NC = prm.gauge ? 7 : 1;
            for (int k = b0; k < b1; ++k) {
                int sp = pc.bra_order[k];
                const PairDev &ab = pc.h_pairs[sp];
                v += (long long)ab.nfp * Krow_pair[sp];
                // E R E contraction of every kept quartet: per primitive quartet
                // 2 nha ncd nhc NC, per bra primitive pair 2 nab ncd nha NC.
                for (int q = 0; q < h_prefix[sp]; ++q) {
                    const int cid = h_ketsp[q];
                    const PairDev &cd = pc.h_pairs[cid];
                    if (one_batch && cid < sp && h_kpos[sp] < h_prefix[cid]) continue;
                    fl += 2.0 * NC * std::min(orient_cost_h(ab, cd), orient_cost_h(cd, ab));
                }
            }
            st->eri_values += v * (prm.gauge ? 6 : 1);
            st->flops_eri += fl;
        }
        int th = tm.n; tm.mark();
        // per-tile K extents (rows in units of W rows)
        long long Wrows = rows * mult;
        std::vector<long long> kt((Wrows + TMr - 1) / TMr, 0);
        for (int k = b0; k < b1; ++k) {
            const PairDev &pr = pc.h_pairs[pc.bra_order[k]];
            long long r0 = (pr.rowoff - row0) * mult, r1 = (pr.rowoff - row0 + pr.nfp) * mult;
            long long kk = Krow_pair[pc.bra_order[k]] * mult;
            for (long long t = r0 / TMr; t <= (r1 - 1) / TMr; ++t) kt[t] = std::max(kt[t], kk);
        }
        long long *d_kt = dcopy(ctx->ktile, kt, s);
        if (st) {
            double f = 0;
            for (long long t = 0; t < (long long)kt.size(); ++t) f += (double)std::min<long long>(TMr, Wrows - t * TMr) * kt[t];
            double ncols = (double)(ls ? (cr.gauge ? N4 : 0) : N4);
            st->flops_half1 += 2.0 * f * ncols;
            if (ls && cr.gaunt) {
                double fg = 0;
                for (int k = b0; k < b1; ++k) {
                    const PairDev &pr = pc.h_pairs[pc.bra_order[k]];
                    fg += (double)pr.nfp * Krow_pair[pc.bra_order[k]];
                }
                st->flops_half1 += 2.0 * fg * 3 * N4;
            }
        }
        if (!ls) {
            gemm_half1(ctx->split, precision, W, ldw, Dket, N4, Vc + row0 * N4, N4, rows, N4, d_kt, kt, s);
            ctx->launches++;
        } else {
            if (cr.gauge) {
                // gauge: rows (ab, I), K (cd, J): D_ket viewed as [(cd, J)][4 nRS]
                gemm_half1(ctx->split, precision, W, ldw, Dket, N4, Vg + row0 * 3 * N4, N4, rows * 3, N4, d_kt, kt, s);
                ctx->launches++;
            }
            if (cr.gaunt) {
                // Gaunt: Coulomb integrals over L-S pairs, N = 12 nRS
                const double *Wg = cr.gauge ? Wc : W;
                long long ldg = cr.gauge ? ldwc : ldw;
                std::vector<long long> kg((rows + TMr - 1) / TMr, 0);
                for (int k = b0; k < b1; ++k) {
                    const PairDev &pr = pc.h_pairs[pc.bra_order[k]];
                    long long r0 = pr.rowoff - row0, r1 = r0 + pr.nfp;
                    for (long long t = r0 / TMr; t <= (r1 - 1) / TMr; ++t)
                        kg[t] = std::max(kg[t], Krow_pair[pc.bra_order[k]]);
                }
                long long *d_kg = dcopy(ctx->ktile, kg, s);
                gemm_half1(ctx->split, precision, Wg, ldg, Dket, 3 * N4, Vc + row0 * 3 * N4, 3 * N4, rows, 3 * N4, d_kg, kg, s);
                ctx->launches++;
            }
        }
        int tend = tm.n; tm.mark();
        QDT_CUDA_TRY(cudaStreamSynchronize(s));
        ms_eri += tm.ms(te, th);
        ms_h1 += tm.ms(th, tend);
        tm.n = te;   // reuse the batch's events
        b0 = b1;
    }
    acc_ms[2] += ms_eri;
    acc_ms[3] += ms_h1;
    (void)Kfull;

    // 5. second half + packing, one block at a time
    const int nP = nRS;
    const long long NO = 4LL * nP;
    double *O = (double *)ctx->O.get(std::max<long long>(1, NO * NO) * sizeof(double));
    size_t pe = (size_t)std::max<long long>(1, NO * NO) * 8;
    if (pe * sizeof(double) > ((size_t)4 << 30)) pe = std::max<size_t>((size_t)NO * NO, ((size_t)4 << 30) / sizeof(double));
    double *partial = (double *)ctx->partial.get(pe * sizeof(double));
    struct Job { const double *V; long long K; double *out; };
    std::vector<Job> jobs;
    if (!ls) jobs.push_back({Vc, M, out_coul});
    if (ls && cr.gaunt) jobs.push_back({Vc, 3 * M, out_gaunt});
    if (ls && cr.gauge) jobs.push_back({Vg, 3 * M, out_gauge});
    for (const Job &j : jobs) {
        int t2 = tm.n; tm.mark();
        launch_zero(O, NO * NO, s);
        gemm_half2(ctx->split, precision, Dbra, N4, j.V, N4, O, NO, j.K, partial, pe, s);
        ctx->launches += 3;
        if (st) st->flops_half2 += 2.0 * (double)j.K * (NO * (NO + 1) / 2.0);
        int t3 = tm.n; tm.mark();
        launch_pack(O, NO, nKa, j.out, s);
        ctx->launches++;
        int t4 = tm.n; tm.mark();
        QDT_CUDA_TRY(cudaStreamSynchronize(s));
        acc_ms[4] += tm.ms(t2, t3);
        acc_ms[5] += tm.ms(t3, t4);
        tm.n = t2;   // reuse events
    }
    acc_ms[0] += tm.ms(t0, t0 + 1);
    acc_ms[1] += tm.ms(t0 + 1, t0 + 2);
    tm.n = t0;
}

}  // namespace

extern "C" {

const char *qdt_version(void) { return "qdt 0.1 (sm_103a)"; }

int qdt_create(qdt_ctx **out, int device, void *cuda_stream) {
    if (!out) return QDT_ERR_ARG;
    *out = nullptr;
    qdt_ctx *c = new (std::nothrow) qdt_ctx();
    if (!c) return QDT_ERR_OOM;
    try {
        c->device = device;
        QDT_CUDA_TRY(cudaSetDevice(device));
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            QDT_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        for (int i = 0; i < 16; ++i) QDT_CUDA_TRY(cudaEventCreate(&c->ev[i]));
        double *tab = (double *)c->boys.get((size_t)kBoysGrid * kBoysCols * sizeof(double));
        launch_boys_table(tab, c->stream);
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (const Error &e) {
        delete c;
        return e.code;
    }
    *out = c;
    return QDT_OK;
}

void qdt_destroy(qdt_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    DBuf *bufs[] = {&c->shells, &c->exps, &c->coefs, &c->norms, &c->boys, &c->Cq, &c->Craw, &c->dsmap0,
                    &c->dsmap1, &c->Dbra, &c->Dket,
                    &c->V, &c->Vg, &c->W, &c->Wc, &c->Dmax, &c->wsort, &c->ketsp, &c->ketcol,
                    &c->prefix, &c->ktile, &c->tasks, &c->O, &c->partial, &c->stage, &c->rsR, &c->rsS};
    for (DBuf *b : bufs) b->release();
    for (int k = 0; k < 2; ++k) {
        c->cb[k].pairs.release(); c->cb[k].pp.release(); c->cb[k].E.release();
        c->cb[k].Q.release(); c->cb[k].bra.release(); c->cb[k].pp_pair.release();
    }
    split_release(c->split);
    for (int i = 0; i < 16; ++i) cudaEventDestroy(c->ev[i]);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int qdt_set_basis(qdt_ctx *c, int n_centers, const double *xyz, int n_shells, const int *shell_center,
                  const int *shell_l, const int *shell_nprim, const double *exps, const double *coefs) {
    if (!c) return QDT_ERR_ARG;
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        arg_check(n_centers > 0 && n_shells > 0 && xyz && shell_center && shell_l && shell_nprim && exps && coefs,
                  "qdt_set_basis: empty or null input");
        c->has_basis = false;
        c->has_coef = false;
        // host copies (inputs may live on the device)
        auto fetch = [&](const void *p, size_t bytes, void *dst) {
            QDT_CUDA_TRY(cudaMemcpy(dst, p, bytes, cudaMemcpyDefault));
        };
        std::vector<double> hx(3 * (size_t)n_centers);
        std::vector<int> hc(n_shells), hl(n_shells), hn(n_shells);
        fetch(xyz, hx.size() * 8, hx.data());
        fetch(shell_center, n_shells * 4, hc.data());
        fetch(shell_l, n_shells * 4, hl.data());
        fetch(shell_nprim, n_shells * 4, hn.data());
        long long np = 0;
        for (int s = 0; s < n_shells; ++s) {
            arg_check(hc[s] >= 0 && hc[s] < n_centers, "qdt_set_basis: shell centre out of range");
            arg_check(hl[s] >= 0 && hl[s] <= kMaxLShell, "qdt_set_basis: shell order must be 0..QDT_MAX_L");
            arg_check(hn[s] >= 1 && hn[s] <= 64, "qdt_set_basis: 1..64 primitives per shell");
            np += hn[s];
        }
        std::vector<double> he(np), hk(np);
        fetch(exps, np * 8, he.data());
        fetch(coefs, np * 8, hk.data());
        for (long long i = 0; i < np; ++i) arg_check(he[i] > 0.0, "qdt_set_basis: exponents must be positive");
        // shells: L then derivative shells
        c->h_shells.clear();
        int foff = 0, poff = 0, noff = 0;
        for (int s = 0; s < n_shells; ++s) {
            ShellDev sh{};
            for (int d = 0; d < 3; ++d) sh.A[d] = hx[3 * hc[s] + d];
            sh.l = hl[s]; sh.isS = 0; sh.nfunc = lcart(hl[s]); sh.foff = foff; sh.nprim = hn[s];
            sh.poff = poff; sh.noff = noff;
            c->h_shells.push_back(sh);
            foff += sh.nfunc; poff += hn[s]; noff += sh.nfunc;
        }
        c->nL = foff; c->nshL = n_shells;
        // derivative shells; those of p shells keep the 6 distinct functions
        // d_K chi_i = d_i chi_K (i <= K), whose coefficient rows are merged
        c->smap0.clear(); c->smap1.clear();
        int soff = 0;
        for (int s = 0; s < n_shells; ++s) {
            ShellDev sh = c->h_shells[s];
            sh.isS = 1;
            sh.red = (sh.l == 1) ? 1 : 0;
            sh.nfunc = sh.red ? 6 : 3 * lcart(sh.l);
            const int mu0 = sh.foff;                       // first L function of the parent
            sh.foff = c->nL + soff;
            if (sh.red) {
                const int pi[6] = {0, 0, 0, 1, 1, 2}, pk[6] = {0, 1, 2, 1, 2, 2};
                for (int f = 0; f < 6; ++f) {
                    c->smap0.push_back(3 * (mu0 + pi[f]) + pk[f]);
                    c->smap1.push_back(pi[f] == pk[f] ? -1 : 3 * (mu0 + pk[f]) + pi[f]);
                }
            } else {
                for (int f = 0; f < sh.nfunc; ++f) { c->smap0.push_back(3 * mu0 + f); c->smap1.push_back(-1); }
            }
            soff += sh.nfunc;
            c->h_shells.push_back(sh);
        }
        c->nS = soff;
        dcopy(c->dsmap0, c->smap0, c->stream);
        dcopy(c->dsmap1, c->smap1, c->stream);
        cudaStream_t st = c->stream;
        dcopy(c->shells, c->h_shells, st);
        dcopy(c->exps, he, st);
        c->h_exps = he;
        dcopy(c->coefs, hk, st);
        c->norms.get(std::max(1, noff) * sizeof(double));
        launch_shell_norms((const ShellDev *)c->shells.p, n_shells, (const double *)c->exps.p,
                           (const double *)c->coefs.p, (double *)c->norms.p, st);
        build_class(c, 0);
        build_class(c, 1);
        QDT_CUDA_TRY(cudaStreamSynchronize(st));
        c->has_basis = true;
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}

int qdt_num_functions(const qdt_ctx *c) { return (c && c->has_basis) ? c->nL : 0; }

int qdt_set_coefficients(qdt_ctx *c, int nK, const double *CL, const double *CS) {
    if (!c) return QDT_ERR_ARG;
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->has_basis) throw Error{QDT_ERR_STATE, "qdt_set_coefficients: no basis"};
        arg_check(nK > 0 && CL && CS, "qdt_set_coefficients: nK must be positive");
        // CL as given; CS (3 nL rows) merged onto the internal derivative functions
        size_t nl = (size_t)c->nL * nK * 4, ns_in = (size_t)3 * c->nL * nK * 4, ns = (size_t)c->nS * nK * 4;
        double *d = (double *)c->Cq.get((nl + ns) * sizeof(double));
        double *raw = (double *)c->Craw.get(ns_in * sizeof(double));
        QDT_CUDA_TRY(cudaMemcpyAsync(d, CL, nl * sizeof(double), cudaMemcpyDefault, c->stream));
        QDT_CUDA_TRY(cudaMemcpyAsync(raw, CS, ns_in * sizeof(double), cudaMemcpyDefault, c->stream));
        launch_merge_rows(raw, (const int *)c->dsmap0.p, (const int *)c->dsmap1.p, c->nS, nK * 4, d + nl, c->stream);
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->nK = nK;
        c->has_coef = true;
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}

size_t qdt_packed_size(const qdt_ctx *c, unsigned blocks, int k_begin, int k_end) {
    (void)c;
    if (k_end <= k_begin) return 0;
    long long n = k_end - k_begin, nP = n * (n + 1) / 2;
    int nb = ((blocks & QDT_COULOMB) ? 1 : 0) + ((blocks & QDT_GAUNT) ? 1 : 0) + ((blocks & QDT_GAUGE) ? 1 : 0);
    return (size_t)(nP * (nP + 1) / 2) * 16 * sizeof(double) * nb;
}

int qdt_transform(qdt_ctx *c, unsigned blocks, int k_begin, int k_end, double tau, int precision,
                  double *out, size_t out_bytes, qdt_stats *st) {
    if (!c) return QDT_ERR_ARG;
    try {
        cudaGetLastError();      // start from a clean error state
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->has_basis || !c->has_coef) throw Error{QDT_ERR_STATE, "qdt_transform: basis or coefficients not set"};
        arg_check(blocks != 0 && (blocks & ~7u) == 0, "qdt_transform: blocks must be a non-empty subset of COULOMB|GAUNT|GAUGE");
        arg_check(k_begin >= 0 && k_end > k_begin && k_end <= c->nK, "qdt_transform: bad Kramers range");
        arg_check(tau >= 0.0, "qdt_transform: negative Schwarz threshold");
        arg_check(precision == QDT_FP64 || precision == QDT_SPLIT, "qdt_transform: bad precision");
        size_t need = qdt_packed_size(c, blocks, k_begin, k_end);
        arg_check(out != nullptr && out_bytes >= need, "qdt_transform: output buffer too small");
        const int nKa = k_end - k_begin;
        const long long nP = (long long)nKa * (nKa + 1) / 2, per = nP * (nP + 1) / 2 * 16;
        bool dev_out = is_device_ptr(out);
        double *dst = out;
        if (!dev_out) dst = (double *)c->stage.get(need);
        double *o_c = nullptr, *o_g = nullptr, *o_b = nullptr, *cur = dst;
        if (blocks & QDT_COULOMB) { o_c = cur; cur += per; }
        if (blocks & QDT_GAUNT) { o_g = cur; cur += per; }
        if (blocks & QDT_GAUGE) { o_b = cur; cur += per; }
        qdt_stats local{};
        qdt_stats *S = st ? &local : nullptr;
        if (S) { S->precision = precision; S->slices = split_slices(c->split); }
        c->launches = 0;
        Timer tm(c);
        tm.mark();
        double acc[6] = {0, 0, 0, 0, 0, 0};
        if (blocks & QDT_COULOMB) {
            ClassRun cr{0, true, false, false};
            run_class(c, cr, k_begin, nKa, tau, precision, o_c, nullptr, nullptr, S, tm, acc);
        }
        if (blocks & (QDT_GAUNT | QDT_GAUGE)) {
            ClassRun cr{1, false, (blocks & QDT_GAUNT) != 0, (blocks & QDT_GAUGE) != 0};
            run_class(c, cr, k_begin, nKa, tau, precision, nullptr, o_g, o_b, S, tm, acc);
        }
        if (!dev_out) QDT_CUDA_TRY(cudaMemcpyAsync(out, dst, need, cudaMemcpyDeviceToHost, c->stream));
        tm.mark();
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (S) {
            S->ms_total = tm.ms(0, 1);
            S->ms_density = acc[0]; S->ms_screen = acc[1]; S->ms_eri = acc[2];
            S->ms_half1 = acc[3]; S->ms_half2 = acc[4]; S->ms_pack = acc[5];
            S->kernel_launches = c->launches;
            *st = local;
        }
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}

int qdt_unpack(qdt_ctx *c, const double *packed, int n_kramers, unsigned block, double *full) {
    if (!c) return QDT_ERR_ARG;
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        arg_check(packed && full && n_kramers > 0, "qdt_unpack: bad arguments");
        arg_check(block == QDT_COULOMB || block == QDT_GAUNT || block == QDT_GAUGE, "qdt_unpack: one block");
        arg_check(is_device_ptr(packed) && is_device_ptr(full), "qdt_unpack: device pointers required");
        launch_unpack(packed, n_kramers, block != QDT_COULOMB, full, c->stream);
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}

const char *qdt_last_error(const qdt_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
