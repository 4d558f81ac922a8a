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
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "plan.h"
#include "qdt_internal.cuh"
#include "split.cuh"

namespace qdt {
void launch_prim_pairs_map(const ShellDev *shells, const PairDev *pairs, const int *pp_pair,
                           long long npp, const double *exps, const double *coefs,
                           const double *norms, PrimPairDev *pp, double *E, cudaStream_t s);
void launch_density(bool gaunt, bool ku, bool pairs_arith, const PairDev *pairs, const int *bra_order, int nsp,
                    const ShellDev *shells, int maxnf, int maxnfp, const double *Cq, int nK, int k0, const int *rsR,
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

// Page-locked staging of the uploads inside a transformation (tile extents,
// parameter sets, screening lists): each host array is copied into the arena
// and sent from there, so every upload is an asynchronous DMA instead of a
// staged copy from pageable memory.  Space is taken in order and only handed
// back by reset(), which the entry points call at their start, when the
// context's stream has drained (every transformation ends by synchronising
// it); a buffer outgrown in between is kept until then, because copies in
// flight may still read it.
struct PinnedArena {
    char *p = nullptr;
    size_t n = 0, used = 0;
    std::vector<char *> retired;
    void *take(size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        if (used + bytes > n) {
            const size_t nn = std::max(bytes, 2 * n + ((size_t)1 << 20));
            char *q = nullptr;
            if (cudaMallocHost(&q, nn) != cudaSuccess) {
                cudaGetLastError();
                throw Error{QDT_ERR_OOM, "cudaMallocHost of " + std::to_string(nn) + " bytes failed"};
            }
            if (p) retired.push_back(p);
            p = q;
            n = nn;
            used = 0;
        }
        void *r = p + used;
        used += bytes;
        return r;
    }
    void reset() {
        for (char *q : retired) cudaFreeHost(q);
        retired.clear();
        used = 0;
    }
    void release() {
        reset();
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

template <class T>
T *dcopy_pinned(PinnedArena &a, DBuf &b, const std::vector<T> &v, cudaStream_t s) {
    T *d = (T *)b.get(std::max<size_t>(1, v.size()) * sizeof(T));
    if (!v.empty()) {
        void *h = a.take(v.size() * sizeof(T));
        std::memcpy(h, v.data(), v.size() * sizeof(T));
        QDT_CUDA_TRY(cudaMemcpyAsync(d, h, v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    return d;
}

struct ClassBufs {
    DBuf pairs, pp, E, E2, E1, Q, bra, brapos, pp_pair;
};

// Instantiated graph of a batch round and the signature it was captured for.
struct GraphEntry {
    uint64_t sig = 0;
    int seen = 0;
    cudaGraphExec_t exec = nullptr;
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
    bool ku = false;            // Kramers-unrestricted coefficients (per spinor) instead of quaternions
    int nK = 0;
    DBuf Cq, Craw, dsmap0, dsmap1;
    std::vector<int> smap0, smap1;
    // per-transform workspace
    DBuf Dbra, Dket, V, Vg, W, Wc, Dmax, wsort, ketsp, ketcol, prefix, ktile, tasks, O, partial,
        stage, rsR, rsS, kpos, prms, next, ktile2;
    // row batches with bra-ket symmetry: transposed blocks for later rows, their
    // tile extents, the W2 column of each batch pair and the batch's density rows
    DBuf W2, Wc2, ktile3, ktile4, col2, ketsp2, ketcol2, Dbra2;
    // tile lists built on the device: the batch's bra pairs in tile order, their
    // first tile, and the FP32 split points of the class
    DBuf tbras, toff, dsplit;
    // ket list of a row batch with bra-ket symmetry: pairs, columns, list position,
    // kept prefix and FP32 split point per pair in list positions
    DBuf klist, kcol1, kpos1, kpre1, ksplit1;
    PinnedArena pin;            // page-locked staging of a transformation's uploads
    SplitWorkspace split;
    // first-half route of the Coulomb block: density (Eq. firsthalf) or the
    // two-quarter comparator, and the comparator's workspace
    int route = QDT_ROUTE_DENSITY;
    int mo_block = 0;           // outer MO indices per block of the MO-driven route
    DBuf qcols, qWL, qWS, qT1, qT, qVf, qCr1, qCr2, qkt[3];
    cudaEvent_t ev[16];
    int launches = 0;
    // batches owned by this context (its stream carries the fused launches)
    DBuf bprms[4], btasks[4], bnext[4];      // per kernel kind: gauge x compensated FP32
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    GraphEntry graph[2];
    long long graph_captures = 0, graph_replays = 0;
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

// Doubles of one packed block over n active units (Kramers pairs: 16 per
// canonical pair of Kramers pairs; spinors of unrestricted input: 4 per
// canonical pair of spinor pairs).
long long packed_block_elems(bool ku, long long n) {
    const long long nP = n * (n + 1) / 2;
    return nP * (nP + 1) / 2 * (ku ? 4 : 16);
}

// Rows of W per split-form first-half call: the digit planes of one call
// (6 BF16 digits per element, 12 bytes) stay within kSliceBudget, so the
// integral rows themselves decide whether a class fits one row batch.
constexpr size_t kSliceBudget = (size_t)8 << 30;
// FP64 intermediates of one row chunk of the quarter route
constexpr size_t kQuarterBudget = (size_t)4 << 30;

// FP64 multiply-adds of the E R E contraction of one shell quartet with X as
// the outer (per primitive pair) side: the ket pass over T rows (X's Hermite
// triples; gauge: also the r12 rows 2 <= |g| <= Lx + 2) and the bra pass per
// component (1 Coulomb, 7 gauge).
double orient_cost_h(const PairDev &X, const PairDev &Y, bool gauge) {
    const double nhx = nherm(X.Lab), nhy = nherm(Y.Lab);
    const double trows = nherm(X.Lab) + (gauge ? nherm(X.Lab + 2) - 4 : 0);
    return (double)X.npp * Y.npp * trows * Y.nfp * nhy + (double)X.npp * X.nfp * Y.nfp * nhx * (gauge ? 7 : 1);
}

// Cost proxy of the tiles of a bra pair: primitive pairs x Hermite terms x
// function pairs.
double bra_cost(const PairDev &p) { return (double)p.npp * nherm(p.Lab) * p.nfp; }

// Bra pairs of a list in tile order: as given (the bra order, Schwarz Q
// descending) or most expensive first, so that the tile queue ends on cheap
// tiles.
std::vector<int> tile_order(const PairClass &pc, std::vector<int> v, int order) {
    if (order == 1)
        std::stable_sort(v.begin(), v.end(),
                         [&](int a, int b) { return bra_cost(pc.h_pairs[a]) > bra_cost(pc.h_pairs[b]); });
    return v;
}

// Tiles: each bra pair's kept ket prefix cut into runs of `kets` positions.
// Tiles of `kets` sorted ket positions per bra pair; with `split`, positions
// [0, split) and [split, prefix) are tiled apart, the second set in plain FP32.
void build_tiles(const std::vector<int> &bras, const std::vector<int> &prefix, int kets, int req,
                 std::vector<EriTask> &out, const std::vector<int> *split = nullptr) {
    for (int sp : bras) {
        const int mid = split ? (*split)[sp] : prefix[sp];
        for (int q = 0; q < mid; q += kets) out.push_back({sp, q, std::min(mid, q + kets), req, 0});
        for (int q = mid; q < prefix[sp]; q += kets) out.push_back({sp, q, std::min(prefix[sp], q + kets), req, 1});
    }
}

// The same tiles written on the device, one warp per bra pair: bras[i] (tile
// order) starts at tile off[i]; its kept prefix and FP32 split point come from
// the device copies of the screening outcome (split null: no FP32 tiles).
// Only the bra list and the offsets are uploaded, not the tiles.
__global__ void build_tiles_kernel(const int *bras, const long long *off, const int *prefix, const int *split,
                                   int n, int kets, int req, EriTask *out) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int sp = bras[w];
    const int pre = prefix[sp], mid = split ? split[sp] : pre;
    const int n1 = (mid + kets - 1) / kets, n2 = (pre - mid + kets - 1) / kets;
    EriTask *o = out + off[w];
    for (int j = lane; j < n1 + n2; j += 32) {
        EriTask t;
        t.bra_sp = sp;
        t.req = req;
        if (j < n1) {
            t.k0 = j * kets;
            t.k1 = min(mid, t.k0 + kets);
            t.f32 = 0;
        } else {
            t.k0 = mid + (j - n1) * kets;
            t.k1 = min(pre, t.k0 + kets);
            t.f32 = 1;
        }
        o[j] = t;
    }
}

// Host side of build_tiles_kernel: per-bra tile offsets (from the host copy of
// the screening outcome), the uploads, the launch; returns the tile count.
int launch_build_tiles(qdt_ctx *ctx, const std::vector<int> &bras, const std::vector<int> &prefix,
                       const std::vector<int> *split, const int *d_prefix, const int *d_split, int kets,
                       EriTask *&d_tiles, cudaStream_t s) {
    std::vector<long long> off(bras.size() + 1, 0);
    for (size_t i = 0; i < bras.size(); ++i) {
        const int sp = bras[i], pre = prefix[sp], mid = split ? (*split)[sp] : pre;
        off[i + 1] = off[i] + (mid + kets - 1) / kets + (pre - mid + kets - 1) / kets;
    }
    const long long nt = off.back();
    if (nt > 0x7fffffffLL) throw Error{QDT_ERR_ARG, "integral tiles: more than 2^31 tiles in one batch"};
    d_tiles = (EriTask *)ctx->tasks.get((size_t)std::max<long long>(1, nt) * sizeof(EriTask));
    if (nt == 0) return 0;
    const int *d_bras = dcopy_pinned(ctx->pin, ctx->tbras, bras, s);
    const long long *d_off = dcopy_pinned(ctx->pin, ctx->toff, off, s);
    const long long threads = 32LL * (long long)bras.size();
    build_tiles_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(d_bras, d_off, d_prefix, split ? d_split : nullptr,
                                                                          (int)bras.size(), kets, 0, d_tiles);
    QDT_CHECK_KERNEL("build_tiles_kernel");
    ctx->launches++;
    return (int)nt;
}

// ---------------------------------------------------------------- autotuner
// Launch shape of the integral kernel per class signature (kernel kind and
// class maxima), chosen by timing on a sample of the class: every 8th bra
// pair of the bra order (an eighth of the work, so that every candidate runs
// many tiles per CTA slot).  The search is coordinate-wise from (plan threads,
// 8 kets, bra order), after one warm-up run: ket positions per tile
// {2, 4, 8, 16}, then CTA threads {128, 256}, then the tile order; each
// candidate keeps the faster of two timings.  The candidates differ only in how the work is cut and scheduled,
// never in the arithmetic of an integral, so the choice changes no result bit.
// Process-wide cache; QDT_AUTOTUNE=0 keeps the start point, QDT_AUTOTUNE_VERBOSE=1
// prints every timing to stderr, QDT_ERI_LAUNCH="threads,kets,order" pins the
// shape for every class.
struct TuneKey {
    int dev, gauge, df, maxnfp, maxLab, maxnpp;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, gauge, df, maxnfp, maxLab, maxnpp) <
               std::tie(o.dev, o.gauge, o.df, o.maxnfp, o.maxLab, o.maxnpp);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, EriLaunch> g_tune;

bool env_flag(const char *name, bool dflt) {
    const char *e = std::getenv(name);
    if (!e || !e[0]) return dflt;
    return e[0] != '0';
}

EriLaunch eri_launch_for(qdt_ctx *ctx, const PairClass &pc, const EriShape &shape, bool gauge, bool df,
                         const EriParams *d_prm, const std::vector<int> &bras, const std::vector<int> &prefix,
                         cudaStream_t s) {
    EriLaunch def;
    def.threads = eri_default_threads(shape, gauge);
    def.kets = 8;
    def.order = 0;
    if (const char *pin = std::getenv("QDT_ERI_LAUNCH")) {
        EriLaunch p = def;
        if (std::sscanf(pin, "%d,%d,%d", &p.threads, &p.kets, &p.order) == 3 && p.threads > 0 && p.kets > 0)
            return p;
        throw Error{QDT_ERR_ARG, "QDT_ERI_LAUNCH must read threads,kets,order"};
    }
    if (!env_flag("QDT_AUTOTUNE", true)) return def;
    const bool verbose = env_flag("QDT_AUTOTUNE_VERBOSE", false);
    const TuneKey key{ctx->device, gauge ? 1 : 0, df ? 1 : 0, shape.maxnfp, shape.maxLab, shape.maxnpp};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    int nsm = 0;
    QDT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    long long total = 0;
    for (int sp : bras) total += prefix[sp];
    // too little work to tell the candidates apart: fewer than ~64 tiles per CTA slot in the sample
    if (total / 8 < 64LL * 8 * 4 * nsm) return def;
    std::vector<int> sample;
    for (size_t i = 0; i < bras.size(); i += 8) sample.push_back(bras[i]);
    cudaEvent_t e0, e1;
    QDT_CUDA_TRY(cudaEventCreate(&e0));
    QDT_CUDA_TRY(cudaEventCreate(&e1));
    int *next = (int *)ctx->next.get(sizeof(int));
    // each candidate runs the sample twice and keeps the faster time: the
    // candidates differ by a few per cent, about the spread of one timing
    auto time_of = [&](const EriLaunch &how) {
        std::vector<EriTask> tk;
        build_tiles(tile_order(pc, sample, how.order), prefix, how.kets, 0, tk);
        EriTask *d_tk = dcopy(ctx->tasks, tk, s);
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            QDT_CUDA_TRY(cudaEventRecord(e0, s));
            launch_eri(d_prm, d_tk, (int)tk.size(), next, shape, gauge, df, how, s);
            QDT_CUDA_TRY(cudaEventRecord(e1, s));
            QDT_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            QDT_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            ms = rep ? std::min(ms, t) : t;
        }
        if (verbose)
            std::fprintf(stderr, "qdt autotune %s%s nfp %d L %d npp %d: threads %d kets %d order %d -> %.3f ms\n",
                         gauge ? "gauge" : "coulomb", df ? " fp32-pairs" : "", shape.maxnfp, shape.maxLab,
                         shape.maxnpp, how.threads, how.kets, how.order, ms);
        return ms;
    };
    EriLaunch best = def;
    time_of(best);                        // warm-up (module load, first-touch of the tables)
    float best_ms = time_of(best);
    auto consider = [&](EriLaunch c) {
        const float ms = time_of(c);
        if (ms < best_ms) { best_ms = ms; best = c; }
    };
    for (int k : {2, 4, 16}) { EriLaunch c = best; c.kets = k; consider(c); }
    { EriLaunch c = best; c.threads = best.threads == 128 ? 256 : 128; consider(c); }
    { EriLaunch c = best; c.order = 1; consider(c); }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return best;
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
    pc.d_E2 = (float2 *)b.E2.get(std::max<long long>(1, eoff) * sizeof(float2));
    pc.d_E1 = (float *)b.E1.get(std::max<long long>(1, eoff) * sizeof(float));
    launch_split_pairs(pc.d_E, eoff, pc.d_E2, pc.d_E1, s);
    ctx->launches += 2;
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
    pc.bra_pos.assign(pc.nsp, 0);
    for (int k = 0; k < pc.nsp; ++k) pc.bra_pos[pc.bra_order[k]] = k;
    pc.d_bra_pos = dcopy(b.brapos, pc.bra_pos, s);
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
}

struct Timer {
    qdt_ctx *c;
    int n = 0;
    bool on = true;
    explicit Timer(qdt_ctx *cc, bool enabled = true) : c(cc), on(enabled) {}
    void mark() {
        if (on && n < 16) QDT_CUDA_TRY(cudaEventRecord(c->ev[n++], c->stream));
    }
    double ms(int a, int b) {
        float t = 0.f;
        if (on && a < n && b < n && cudaEventElapsedTime(&t, c->ev[a], c->ev[b]) != cudaSuccess) {
            cudaGetLastError();   // a timing failure must not surface as a later launch error
            t = 0.f;
        }
        return t;
    }
};

// One block class of a transformation.
struct ClassRun {
    int c;                  // pair class
    bool coulomb = false, gaunt = false, gauge = false;
};

// Screening outcome and device operands of one class of a transformation.
struct ClassPlan {
    ClassRun cr{};
    int k0 = 0, nKa = 0, precision = 0, nRS = 0, mult = 1;
    double tau = 0;
    bool ls = false, one_batch = true;
    bool mirror = false;      // row batches with bra-ket symmetry (EriParams::sym 2)
    bool mo_blocks = false;   // MO-driven route in blocks: row batches without symmetry
    bool ku = false;          // columns are spinor pairs with 2 parts (Kramers-unrestricted input)
    bool quarter = false;     // Coulomb first half by two quarter steps (no ket density)
    int2 *qcols = nullptr;    // function indices of the ket-ordered integral columns
    long long N4 = 0, ncolD = 0, M = 0, NV = 0;
    double *Dbra = nullptr, *Dmax = nullptr, *Dket = nullptr, *Vc = nullptr, *Vg = nullptr;
    int *prefix = nullptr, *ketsp = nullptr, *d_kpos = nullptr;
    long long *ketcol = nullptr;
    std::vector<int> h_prefix, h_ketsp, h_kpos;
    std::vector<int> h_split;     // per bra pair: kept ket positions [h_split, h_prefix) run in plain FP32
    int *d_split = nullptr;       // its device copy (split form)
    std::vector<double> h_Dmax;
    std::vector<long long> h_col, Krow;
    size_t wbudget = 0;
};

// Steps 2-3 for the current P.Dmax: ket order and kept prefixes (copied to
// the host), then the ket-ordered density copy (density route) or the
// function indices of the ket-ordered columns (quarter route).
void order_kets(qdt_ctx *ctx, ClassPlan &P, cudaStream_t s) {
    PairClass &pc = ctx->cls[P.cr.c];
    const double tau = P.tau;
    double *wsort = (double *)ctx->wsort.get(std::max(1, pc.nsp) * sizeof(double));
    P.ketsp = (int *)ctx->ketsp.get(std::max(1, pc.nsp) * sizeof(int));
    P.ketcol = (long long *)ctx->ketcol.get((pc.nsp + 1) * sizeof(long long));
    P.prefix = (int *)ctx->prefix.get(std::max(1, pc.nsp) * sizeof(int));
    launch_ket_order(pc.d_Q, P.Dmax, pc.nsp, wsort, P.ketsp, s);
    launch_ket_columns(pc.d_pairs, P.ketsp, pc.nsp, P.ketcol, s);
    launch_prefix_lengths(pc.d_Q, wsort, pc.nsp, tau, P.prefix, s);
    ctx->launches += 3;
    P.h_prefix.resize(pc.nsp);
    P.h_col.resize(pc.nsp + 1);
    P.h_ketsp.resize(pc.nsp);
    QDT_CUDA_TRY(cudaMemcpyAsync(P.h_prefix.data(), P.prefix, pc.nsp * sizeof(int), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaMemcpyAsync(P.h_col.data(), P.ketcol, (pc.nsp + 1) * sizeof(long long), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaMemcpyAsync(P.h_ketsp.data(), P.ketsp, pc.nsp * sizeof(int), cudaMemcpyDeviceToHost, s));
    P.h_Dmax.resize(pc.nsp);
    QDT_CUDA_TRY(cudaMemcpyAsync(P.h_Dmax.data(), P.Dmax, pc.nsp * sizeof(double), cudaMemcpyDeviceToHost, s));
    // 3. ket-ordered density copy (density route) or the function indices of
    // the ket-ordered columns (quarter route)
    if (P.quarter) {
        P.qcols = (int2 *)ctx->qcols.get(std::max<long long>(1, P.M) * sizeof(int2));
        launch_ket_functions(pc.d_pairs, (const ShellDev *)ctx->shells.p, P.ketsp, P.ketcol, pc.nsp, P.qcols, s);
        const long long nX = ctx->nL + ctx->nS, Pp = P.ku ? 2 : 4;
        double *Cr1 = (double *)ctx->qCr1.get((size_t)nX * 4 * P.nKa * sizeof(double));
        double *Cr2 = (double *)ctx->qCr2.get((size_t)4 * nX * Pp * P.nKa * sizeof(double));
        launch_quarter_coefs((const double *)ctx->Cq.p, ctx->nK, P.k0, P.nKa, (int)nX, (int)Pp, Cr1, Cr2, s);
        ctx->launches++;
    } else {
        P.Dket = (double *)ctx->Dket.get(std::max<long long>(1, P.M * P.ncolD) * sizeof(double));
        launch_gather_rows(P.Dbra, pc.d_pairs, P.ketsp, P.ketcol, pc.nsp, P.ncolD, P.Dket, s);
    }
    ctx->launches++;
}

// Steps 1-3 on the context's stream: density in bra order and Dmax, ket order
// and kept prefixes (copied to the host), ket-ordered density copy.
void class_issue(qdt_ctx *ctx, const ClassRun &cr, int k0, int nKa, double tau, int precision, ClassPlan &P,
                 Timer &tm) {
    PairClass &pc = ctx->cls[cr.c];
    cudaStream_t s = ctx->stream;
    P = ClassPlan();
    P.cr = cr;
    P.k0 = k0;
    P.nKa = nKa;
    P.tau = tau;
    P.precision = precision;
    P.nRS = nKa * (nKa + 1) / 2;
    P.ls = cr.c == 1;
    P.ku = ctx->ku;
    P.quarter = !P.ls && ctx->route == QDT_ROUTE_QUARTER;
    P.N4 = (P.ku ? 2LL : 4LL) * P.nRS;          // columns per J component
    P.ncolD = P.ls ? 3 * P.N4 : P.N4;            // density row length
    P.NV = P.ls ? 3 * P.N4 : P.N4;               // V row length (Coulomb / Gaunt)
    P.M = pc.M;
    P.mult = (P.ls && cr.gauge) ? 3 : 1;         // gauge rows/cols are (pair, I)
    std::vector<int> hR, hS;
    for (int r = 0; r < nKa; ++r)
        for (int q = r; q < nKa; ++q) { hR.push_back(r); hS.push_back(q); }
    int *d_rsR = dcopy_pinned(ctx->pin, ctx->rsR, hR, s), *d_rsS = dcopy_pinned(ctx->pin, ctx->rsS, hS, s);
    split_invalidate(ctx->split);

    // 1. density in bra order + Dmax
    tm.mark();
    P.Dbra = (double *)ctx->Dbra.get(std::max<long long>(1, P.M * P.ncolD) * sizeof(double));
    P.Dmax = (double *)ctx->Dmax.get(std::max(1, pc.nsp) * sizeof(double));
    QDT_CUDA_TRY(cudaMemsetAsync(P.Dmax, 0, pc.nsp * sizeof(double), s));
    int maxnf = 1;
    for (const ShellDev &sh : ctx->h_shells) maxnf = std::max(maxnf, sh.nfunc);
    launch_density(P.ls, P.ku, precision == QDT_SPLIT, pc.d_pairs, pc.d_bra_order, pc.nsp,
                   (const ShellDev *)ctx->shells.p, maxnf, pc.maxnfp, (const double *)ctx->Cq.p, ctx->nK, k0, d_rsR,
                   d_rsS, P.nRS, P.Dbra, P.Dmax, s);
    ctx->launches++;
    if (P.quarter) {   // the quarter route screens on coefficient bounds, not on the density
        launch_coef_bound(pc.d_pairs, (const ShellDev *)ctx->shells.p, (const double *)ctx->Cq.p, ctx->nK, k0,
                          nKa, pc.nsp, P.Dmax, s);
        ctx->launches++;
    }
    tm.mark();
    order_kets(ctx, P, s);
    tm.mark();
}

// Split form: which kept quartets may have their integrals in plain FP32.
// An integral computed in FP32 from FP64 Boys values and prefactors is taken
// to be within kF32Rel Q_A Q_C of its FP64 value (kF32Rel = 256 x 2^-24,
// 23x the largest ratio measured on s/p/d quartets up to L = 12, 6.7e-7;
// `tests/test_gpu_dynprec.py` requires the measured ratio to stay 8x below it).  An error d in
// (ab|cd) moves a packed output element by at most |D_ab| d |D_cd| (times
// g: 1 Coulomb, 3 Gaunt (three J), 18 gauge (nine IJ, two terms)), so the
// FP32 quartets of a class add at most
//     sum g kF32Rel (Q_A Dmax_A nfp_A) (Q_C Dmax_C nfp_C)
// over its ordered kept pairs (A, C).  With w = Q Dmax the FP32 set is
// {w_A w_C <= t}, a suffix of every bra row's w-sorted ket list (and the
// same decision for (C, A), so bra-ket symmetry is kept); t is the largest
// threshold whose bound stays within kF32Budget.  QDT_F32_BUDGET overrides
// the budget (0 turns the FP32 quartets off).
constexpr double kF32Rel = 256.0 / 16777216.0;
// A third of the split form's 1e-10 bar against the FP64 form; the slice
// contractions add about 3e-13 on the 40-centre chain.
constexpr double kF32Budget = 3e-11;

double f32_budget() {
    if (const char *e = std::getenv("QDT_F32_BUDGET")) {
        const double v = std::atof(e);
        if (!(v >= 0.0)) throw Error{QDT_ERR_ARG, "QDT_F32_BUDGET must be >= 0"};
        return v;
    }
    return kF32Budget;
}

void f32_split(qdt_ctx *ctx, ClassPlan &P, double &bound_out) {
    PairClass &pc = ctx->cls[P.cr.c];
    const int n = pc.nsp;
    const double budget = P.precision == QDT_SPLIT ? f32_budget() : 0.0;
    const double g = !P.ls ? 1.0 : (P.cr.gauge ? 18.0 : 3.0);
    std::vector<double> w(n);
    std::vector<int> nfp(n);
    for (int i = 0; i < n; ++i) {
        w[i] = pc.h_Q[i] * P.h_Dmax[i];
        nfp[i] = pc.h_pairs[i].nfp;
    }
    f32_tail_split(w, nfp, P.h_ketsp, P.h_prefix, g * kF32Rel, budget, P.h_split, &bound_out);
}

// QDT_W_BUDGET (bytes, > 0) replaces the device-memory test of the row-batch
// decision: a class runs as one batch when its integral block fits the value,
// else in batches of at most that many bytes (without bra-ket symmetry).
// Small values exercise the batched path on small inputs.
size_t w_budget_override() {
    const char *e = std::getenv("QDT_W_BUDGET");
    if (!e || !e[0]) return 0;
    const long long v = std::atoll(e);
    if (v <= 0) throw Error{QDT_ERR_ARG, "QDT_W_BUDGET must be a positive byte count"};
    return (size_t)v;
}

// QDT_BATCH_SYM=0 runs row batches without bra-ket symmetry (every kept block
// computed in its own row's batch), for comparison.
bool batch_sym_enabled() {
    const char *e = std::getenv("QDT_BATCH_SYM");
    return !(e && e[0] == '0');
}

// Waits for class_issue; kept-quartet statistics, V buffers and the row-batch
// decision: one batch (and bra-ket symmetry) when the integral block (plus the
// split form's digit planes of one row chunk) fits in 70 % of the device
// memory this context can use, else batches of at most 6 GB.
void class_finish(qdt_ctx *ctx, ClassPlan &P, qdt_stats *st) {
    PairClass &pc = ctx->cls[P.cr.c];
    cudaStream_t s = ctx->stream;
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
    long long kept = 0, f32 = 0;
    for (int i = 0; i < pc.nsp; ++i) kept += P.h_prefix[i];
    double bound = 0.0;
    f32_split(ctx, P, bound);
    for (int i = 0; i < pc.nsp; ++i) f32 += P.h_prefix[i] - P.h_split[i];
    if (st) {
        int slot = P.ls ? 1 : 0;
        st->quartets_total[slot] += (long long)pc.nsp * pc.nsp;
        st->quartets_kept[slot] += kept;
        st->quartets_f32[slot] += f32;
        st->f32_bound = std::max(st->f32_bound, bound);
        if (P.ls && P.cr.gauge) {
            st->quartets_total[2] += (long long)pc.nsp * pc.nsp;
            st->quartets_kept[2] += kept;
            st->quartets_f32[2] += f32;
        }
    }
    P.Krow.assign(pc.nsp, 0);
    for (int i = 0; i < pc.nsp; ++i) P.Krow[i] = P.h_col[P.h_prefix[i]];
    if (!P.ls || P.cr.gaunt) P.Vc = (double *)ctx->V.get(std::max<long long>(1, P.M * P.NV) * sizeof(double));
    if (P.ls && P.cr.gauge) P.Vg = (double *)ctx->Vg.get(std::max<long long>(1, 3 * P.M * P.N4) * sizeof(double));
    long long kmax_all = 0;
    for (int i = 0; i < pc.nsp; ++i) kmax_all = std::max(kmax_all, P.Krow[i]);
    const size_t wall = (size_t)P.M * P.mult * (size_t)std::max<long long>(kmax_all, 1) * P.mult * sizeof(double);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
    const size_t usable = (size_t)(0.7 * (double)(fr + ctx->W.n + ctx->Wc.n + split_held_bytes(ctx->split)));
    const double wfac = (P.ls && P.cr.gauge && P.cr.gaunt) ? 1.12 : 1.0;
    const double slices = (P.precision == QDT_SPLIT ? 1.1 * (double)kSliceBudget : 0.0) +
                          (P.quarter ? 1.1 * (double)kQuarterBudget : 0.0);
    const size_t forced = w_budget_override();
    P.one_batch = forced ? (double)wall * wfac <= (double)forced : (double)wall * wfac + slices <= (double)usable;
    // what the decision counted as reusable is handed back first
    if (P.one_batch && (double)wall * wfac + slices > 0.7 * (double)(fr + ctx->W.n + ctx->Wc.n)) split_release(ctx->split);
    P.wbudget = P.one_batch ? wall : (forced ? forced : ((size_t)6 << 30));
    // row batches of the AO-driven density route keep bra-ket symmetry (each
    // kept pair of blocks computed once, the transpose contracted into the later
    // rows); their budget covers W and W2
    P.mirror = !P.one_batch && !P.quarter && !P.mo_blocks && batch_sym_enabled();
    if (P.mirror && !forced) {
        const double room = (double)usable - slices;
        P.wbudget = (size_t)std::max(2.0 * (1 << 30), std::min(24.0 * (1 << 30), room));
    }
    P.h_kpos.assign(pc.nsp, 0);
    for (int q = 0; q < pc.nsp; ++q) P.h_kpos[P.h_ketsp[q]] = q;
    P.d_kpos = (P.one_batch || P.mirror) ? dcopy_pinned(ctx->pin, ctx->kpos, P.h_kpos, s) : nullptr;
    P.d_split = P.precision == QDT_SPLIT ? dcopy_pinned(ctx->pin, ctx->dsplit, P.h_split, s) : nullptr;
}

// One batch of bra rows of a class.
struct RowBatch {
    int b0 = 0, b1 = 0;
    long long rows = 0, kmax = 0, row0 = 0, ldw = 1, ldwc = 1;
    double *W = nullptr, *Wc = nullptr;
    EriParams prm{};
    std::vector<int> bras;                  // the batch's bra pairs, in bra order
    std::vector<long long> kt, kg;          // K extents of the 64-row tiles (gauge/Coulomb rows, Gaunt rows)
    long long *d_kt = nullptr, *d_kg = nullptr;
    // bra-ket symmetry across batches (ClassPlan::mirror): W2 [(later rows)][(batch pairs in
    // ket order)], its Gaunt companion Wc2, their tile extents, and the batch's density rows
    // in the same order (Dbra2)
    long long row2 = 0, rows2 = 0, ld2 = 1, ldw2 = 1;
    double *W2 = nullptr, *Wc2 = nullptr, *Dbra2 = nullptr;
    std::vector<long long> kt2, kg2;
    long long *d_kt2 = nullptr, *d_kg2 = nullptr;
    // its ket list (plan.h batch_kets): per shell pair the kept prefix and the FP32
    // split point in list positions, the W columns of a batch row's kept prefix
    std::vector<int> pre1, split1;
    std::vector<long long> krow1;
    int *d_list = nullptr, *d_pos1 = nullptr, *d_pre1 = nullptr, *d_split1 = nullptr;
    long long *d_col1 = nullptr;
};

// The ket list of a row batch with bra-ket symmetry (plan.h batch_kets): the
// kets of this and later batches and the earlier ones some row keeps one way
// only, in ket order; the W columns follow the list, and the density rows of
// the list are gathered into the ket-ordered density buffer (which the
// first half of this batch reads).  Each shell pair's prefix and FP32 split
// point become list positions, which is all the integral kernel needs: for a
// batch row AB (in the list), list position < list prefix of CD exactly when
// kpos(AB) < prefix(CD).
void batch_kets_prepare(qdt_ctx *ctx, const ClassPlan &P, RowBatch &B) {
    PairClass &pc = ctx->cls[P.cr.c];
    cudaStream_t s = ctx->stream;
    const BatchKets bk = batch_kets(P.h_ketsp, P.h_kpos, P.h_prefix, pc.bra_pos, B.b0, B.bras);
    const int L = (int)bk.list.size();
    std::vector<long long> col1((size_t)L + 1, 0);
    for (int p = 0; p < L; ++p) col1[p + 1] = col1[p] + pc.h_pairs[bk.list[p]].nfp;
    B.pre1.assign(pc.nsp, 0);
    B.split1.assign(pc.nsp, 0);
    for (int sp = 0; sp < pc.nsp; ++sp) {
        B.pre1[sp] = bk.cnt[P.h_prefix[sp]];
        B.split1[sp] = bk.cnt[P.h_split[sp]];
    }
    B.krow1.assign(pc.nsp, 0);
    for (int sp : B.bras) B.krow1[sp] = col1[B.pre1[sp]];
    B.d_list = dcopy_pinned(ctx->pin, ctx->klist, bk.list, s);
    B.d_col1 = dcopy_pinned(ctx->pin, ctx->kcol1, col1, s);
    B.d_pos1 = dcopy_pinned(ctx->pin, ctx->kpos1, bk.pos, s);
    B.d_pre1 = dcopy_pinned(ctx->pin, ctx->kpre1, B.pre1, s);
    B.d_split1 = dcopy_pinned(ctx->pin, ctx->ksplit1, B.split1, s);
    launch_gather_rows(P.Dbra, pc.d_pairs, B.d_list, B.d_col1, L, P.ncolD, P.Dket, s);
    ctx->launches++;
    // the buffer's rows changed: its cached digit slices are stale
    split_forget(ctx->split, P.Dket, P.Dket + P.M * P.ncolD);
}

// Bra-ket symmetry across row batches (ClassPlan::mirror): a kept block
// (AB|CD) with CD in a later batch whose (CD|AB) is kept too is computed once,
// in AB's batch, and its transpose written into W2, whose rows are the later
// rows and whose columns are this batch's pairs in ket (w-sorted) order; the
// first half then adds W2 D(batch rows) into the later rows of V.  Row CD's
// entries are those of the batch pairs AB with kpos(AB) < prefix(CD): a prefix
// of the columns, so each 64-row tile of W2 has a K extent as W does.
void batch_prepare_mirror(qdt_ctx *ctx, const ClassPlan &P, RowBatch &B) {
    PairClass &pc = ctx->cls[P.cr.c];
    cudaStream_t s = ctx->stream;
    const int TMr = gemm_fp64_tile_m();
    const int mult = P.mult;
    B.row2 = B.row0 + B.rows;
    B.rows2 = P.M - B.row2;
    // this batch's pairs in ket order, their W2 columns
    std::vector<int> k2(B.bras);
    std::sort(k2.begin(), k2.end(), [&](int x, int y) { return P.h_kpos[x] < P.h_kpos[y]; });
    std::vector<long long> col2(pc.nsp, 0), kcol(k2.size()), kend(k2.size());
    std::vector<int> kk(k2.size());
    long long off = 0;
    for (size_t i = 0; i < k2.size(); ++i) {
        col2[k2[i]] = off;
        kcol[i] = off;
        kk[i] = P.h_kpos[k2[i]];
        off += pc.h_pairs[k2[i]].nfp;
        kend[i] = off;
    }
    B.ld2 = std::max<long long>(off, 1);
    B.ldw2 = B.ld2 * mult;
    const bool gaunt_too = P.ls && P.cr.gauge && P.cr.gaunt;
    B.W2 = (double *)ctx->W2.get((size_t)std::max<long long>(B.rows2, 1) * mult * B.ldw2 * sizeof(double));
    if (gaunt_too) B.Wc2 = (double *)ctx->Wc2.get((size_t)std::max<long long>(B.rows2, 1) * B.ld2 * sizeof(double));
    // tile extents of W2 (rows (cd, I) in units of mult) and of Wc2
    const long long Wrows2 = B.rows2 * mult;
    B.kt2.assign((size_t)((Wrows2 + TMr - 1) / TMr), 0);
    if (gaunt_too) B.kg2.assign((size_t)((B.rows2 + TMr - 1) / TMr), 0);
    for (int k = B.b1; k < pc.nsp; ++k) {
        const int cd = pc.bra_order[k];
        const PairDev &pr = pc.h_pairs[cd];
        // batch pairs AB with kpos(AB) < prefix(CD)
        const size_t n = (size_t)(std::lower_bound(kk.begin(), kk.end(), P.h_prefix[cd]) - kk.begin());
        const long long ext = n ? kend[n - 1] : 0;
        if (!ext) continue;
        const long long r0 = pr.rowoff - B.row2;
        for (long long t = r0 * mult / TMr; t <= ((r0 + pr.nfp) * mult - 1) / TMr; ++t)
            B.kt2[t] = std::max(B.kt2[t], ext * mult);
        if (gaunt_too)
            for (long long t = r0 / TMr; t <= (r0 + pr.nfp - 1) / TMr; ++t) B.kg2[t] = std::max(B.kg2[t], ext);
    }
    B.d_kt2 = dcopy_pinned(ctx->pin, ctx->ktile3, B.kt2, s);
    if (gaunt_too) B.d_kg2 = dcopy_pinned(ctx->pin, ctx->ktile4, B.kg2, s);
    else { B.kg2 = B.kt2; B.d_kg2 = B.d_kt2; }
    // the batch's density rows in W2 column order
    int *d_k2 = dcopy_pinned(ctx->pin, ctx->ketsp2, k2, s);
    long long *d_kcol = dcopy_pinned(ctx->pin, ctx->ketcol2, kcol, s);
    B.Dbra2 = (double *)ctx->Dbra2.get((size_t)B.ld2 * P.ncolD * sizeof(double));
    launch_gather_rows(P.Dbra, pc.d_pairs, d_k2, d_kcol, (int)k2.size(), P.ncolD, B.Dbra2, s);
    ctx->launches++;
    EriParams &prm = B.prm;
    prm.W2 = B.W2;
    prm.ldw2 = B.ldw2;
    prm.row2 = B.row2;
    prm.Wc2 = B.Wc2;
    prm.ldwc2 = B.ld2;
    prm.col2 = dcopy_pinned(ctx->pin, ctx->col2, col2, s);
}

// Next batch from bra position b0: sizes, integral-row buffers, the integral
// kernel's parameters and the tile extents (uploaded to the context).
void batch_prepare(qdt_ctx *ctx, const ClassPlan &P, int b0, RowBatch &B) {
    PairClass &pc = ctx->cls[P.cr.c];
    cudaStream_t s = ctx->stream;
    const int TMr = gemm_fp64_tile_m();
    const int mult = P.mult;
    B = RowBatch();
    B.b0 = b0;
    long long rows = 0, kmax = 0;
    int b1 = b0;
    const long long row_b0 = pc.h_pairs[pc.bra_order[b0]].rowoff;
    const bool gaunt_too = P.ls && P.cr.gauge && P.cr.gaunt;
    while (b1 < pc.nsp) {      // grow the batch while the W block fits the budget
        const PairDev &pr = pc.h_pairs[pc.bra_order[b1]];
        long long k = std::max(kmax, P.Krow[pc.bra_order[b1]]);
        const long long r = rows + pr.nfp;
        double need = (double)r * mult * (double)std::max<long long>(k, 1) * mult * sizeof(double);
        if (P.mirror) {      // plus W2 over the later rows, and the Gaunt companions
            need += (double)(P.M - row_b0 - r) * mult * (double)r * mult * sizeof(double);
            if (gaunt_too) need *= 10.0 / 9.0;
        }
        if (b1 > b0 && need > (double)P.wbudget) break;
        rows = r;
        kmax = k;
        ++b1;
    }
    B.b1 = b1;
    B.rows = rows;
    B.row0 = pc.h_pairs[pc.bra_order[b0]].rowoff;
    B.bras.assign(pc.bra_order.begin() + b0, pc.bra_order.begin() + b1);
    // W columns per bra row: its kept ket prefix, in the batch's own ket list
    // when the batches keep bra-ket symmetry
    const std::vector<long long> *krow = &P.Krow;
    if (P.mirror) {
        batch_kets_prepare(ctx, P, B);
        krow = &B.krow1;
        kmax = 0;
        for (int sp : B.bras) kmax = std::max(kmax, B.krow1[sp]);
    }
    B.kmax = kmax;
    B.ldw = std::max<long long>(kmax, 1) * mult;
    B.W = (double *)ctx->W.get((size_t)std::max<long long>(rows, 1) * mult * B.ldw * sizeof(double));
    B.ldwc = std::max<long long>(kmax, 1);
    if (P.ls && P.cr.gauge && P.cr.gaunt) B.Wc = (double *)ctx->Wc.get((size_t)std::max<long long>(rows, 1) * B.ldwc * sizeof(double));
    EriParams &prm = B.prm;
    prm.shells = (const ShellDev *)ctx->shells.p;
    prm.pairs = pc.d_pairs;
    prm.pp = pc.d_pp;
    prm.E = pc.d_E;
    prm.E2 = P.precision == QDT_SPLIT ? pc.d_E2 : nullptr;
    prm.E1 = P.precision == QDT_SPLIT ? pc.d_E1 : nullptr;
    prm.boys = (const double *)ctx->boys.p;
    prm.ket_sp = P.mirror ? B.d_list : P.ketsp;
    prm.ket_col = P.mirror ? B.d_col1 : P.ketcol;
    prm.W = B.W;
    prm.ldw = B.ldw;
    prm.row0 = B.row0;
    prm.gauge = (P.ls && P.cr.gauge) ? 1 : 0;
    prm.with_coulomb = B.Wc ? 1 : 0;
    prm.Wc = B.Wc;
    prm.ldwc = B.ldwc;
    prm.sym = P.one_batch ? 1 : (P.mirror ? 2 : 0);
    prm.ket_pos = P.mirror ? B.d_pos1 : P.d_kpos;
    prm.prefix = P.mirror ? B.d_pre1 : P.prefix;
    prm.bra_pos = pc.d_bra_pos;
    prm.b0 = b0;
    prm.b1 = b1;
    // per-tile K extents (rows in units of W rows)
    const long long Wrows = rows * mult;
    B.kt.assign((Wrows + TMr - 1) / TMr, 0);
    for (int k = b0; k < b1; ++k) {
        const PairDev &pr = pc.h_pairs[pc.bra_order[k]];
        long long r0 = (pr.rowoff - B.row0) * mult, r1 = (pr.rowoff - B.row0 + pr.nfp) * mult;
        long long kk = (*krow)[pc.bra_order[k]] * mult;
        for (long long t = r0 / TMr; t <= (r1 - 1) / TMr; ++t) B.kt[t] = std::max(B.kt[t], kk);
    }
    B.d_kt = dcopy_pinned(ctx->pin, ctx->ktile, B.kt, s);
    if (P.ls && P.cr.gaunt && P.cr.gauge) {
        B.kg.assign((rows + TMr - 1) / TMr, 0);
        for (int k = b0; k < b1; ++k) {
            const PairDev &pr = pc.h_pairs[pc.bra_order[k]];
            long long r0 = pr.rowoff - B.row0, r1 = r0 + pr.nfp;
            for (long long t = r0 / TMr; t <= (r1 - 1) / TMr; ++t) B.kg[t] = std::max(B.kg[t], (*krow)[pc.bra_order[k]]);
        }
        B.d_kg = dcopy_pinned(ctx->pin, ctx->ktile2, B.kg, s);
    } else {
        B.kg = B.kt;
        B.d_kg = B.d_kt;
    }
    if (P.mirror) batch_prepare_mirror(ctx, P, B);
}

// Integral values, E R E flops and first-half flops of a batch.
void batch_stats(qdt_ctx *ctx, const ClassPlan &P, const RowBatch &B, long long width, qdt_stats *st) {
    if (!st) return;
    PairClass &pc = ctx->cls[P.cr.c];
    const int TMr = gemm_fp64_tile_m();
    long long v = 0;
    double fl = 0.0, fl32 = 0.0;
    const bool gauge = B.prm.gauge != 0;
    for (int k = B.b0; k < B.b1; ++k) {
        int sp = pc.bra_order[k];
        const PairDev &ab = pc.h_pairs[sp];
        v += (long long)ab.nfp * P.Krow[sp];
        // E R E contraction of every kept quartet, cheaper orientation
        for (int q = 0; q < P.h_prefix[sp]; ++q) {
            const int cid = P.h_ketsp[q];
            const PairDev &cd = pc.h_pairs[cid];
            const bool both = cid != sp && P.h_kpos[sp] < P.h_prefix[cid];      // (CD|AB) kept too
            if (P.one_batch && both && cid < sp) continue;
            if (P.mirror && both) {
                const int bp = pc.bra_pos[cid];
                if (bp < B.b0 || (bp < B.b1 && cid < sp)) continue;
            }
            const double f = 2.0 * std::min(orient_cost_h(ab, cd, gauge), orient_cost_h(cd, ab, gauge));
            fl += f;
            if (B.prm.E2 && q >= P.h_split[sp]) fl32 += f;
        }
    }
    st->eri_values += v * (B.prm.gauge ? 6 : 1);
    st->flops_eri += fl;
    st->flops_eri_f32 += fl32;
    if (P.quarter) return;   // counted by quarter_half1
    const long long Wrows = B.rows * P.mult;
    double f = 0;
    for (long long t = 0; t < (long long)B.kt.size(); ++t) f += (double)std::min<long long>(TMr, Wrows - t * TMr) * B.kt[t];
    const double ncols = (double)(P.ls ? (P.cr.gauge ? width : 0) : width);
    st->flops_half1 += 2.0 * f * ncols;
    if (P.ls && P.cr.gaunt) {
        double fg = 0;
        const std::vector<long long> &kr = P.mirror ? B.krow1 : P.Krow;
        for (int k = B.b0; k < B.b1; ++k) fg += (double)pc.h_pairs[pc.bra_order[k]].nfp * kr[pc.bra_order[k]];
        st->flops_half1 += 2.0 * fg * 3 * width;
    }
    if (P.mirror) {         // the transposed blocks into the later rows
        double f2 = 0;
        for (long long t = 0; t < (long long)B.kt2.size(); ++t)
            f2 += (double)std::min<long long>(TMr, B.rows2 * P.mult - t * TMr) * B.kt2[t];
        st->flops_half1 += 2.0 * f2 * ncols;
        if (P.ls && P.cr.gaunt) {
            double fg2 = 0;
            for (long long t = 0; t < (long long)B.kg2.size(); ++t)
                fg2 += (double)std::min<long long>(TMr, B.rows2 - t * TMr) * B.kg2[t];
            st->flops_half1 += 2.0 * fg2 * 3 * width;
        }
    }
}

// QDT_SPLIT_CHUNK_ROWS (a positive multiple of 128) caps the rows per call.
long long split_chunk_rows(long long ldw) {
    if (const char *e = std::getenv("QDT_SPLIT_CHUNK_ROWS")) {
        const long long r = std::atoll(e);
        if (r > 0 && r % 128 == 0) return r;
        throw Error{QDT_ERR_ARG, "QDT_SPLIT_CHUNK_ROWS must be a positive multiple of 128"};
    }
    const long long per_row = 12 * std::max<long long>(ldw, 1) + 64;
    long long r = (long long)(kSliceBudget / (size_t)per_row);
    r = std::max<long long>(128, r / 128 * 128);
    return r;
}

// V rows = W D_ket over `rows` W rows from row 0 (launches only).  Split form:
// row chunks (digit planes of W within kSliceBudget) and, when the density's
// digit planes (12 bytes x longest K x N) exceed kSliceBudget too, column
// chunks outside them, so each column chunk of the density is sliced once.
void half1_rows(qdt_ctx *ctx, int precision, const double *W, long long ldw, const double *B, long long ldb,
                double *C, long long ldc, long long rows, long long N, const long long *d_kt,
                const std::vector<long long> &kt, cudaStream_t s, bool accumulate = false) {
    const int TMr = gemm_fp64_tile_m();
    const bool split = precision == QDT_SPLIT;
    const long long chunk = split ? split_chunk_rows(ldw) : std::max<long long>(rows, 1);
    long long kmax = 1;
    for (long long k : kt) kmax = std::max(kmax, k);
    long long ncols = N;
    if (split && 12.0 * (double)kmax * (double)N > (double)kSliceBudget)
        ncols = std::max<long long>(64, (long long)(kSliceBudget / (12 * (size_t)kmax)) / 64 * 64);
    if (const char *e = std::getenv("QDT_SPLIT_CHUNK_COLS")) {       // smaller chunks, to exercise this path
        const long long v = std::atoll(e);
        if (v <= 0 || v % 64) throw Error{QDT_ERR_ARG, "QDT_SPLIT_CHUNK_COLS must be a positive multiple of 64"};
        if (split) ncols = v;
    }
    for (long long n0 = 0; n0 < N; n0 += ncols) {
        const long long nw = std::min(ncols, N - n0);
        for (long long r0 = 0; r0 < rows; r0 += chunk) {
            const long long m = std::min(chunk, rows - r0);
            const size_t t0 = (size_t)(r0 / TMr), t1 = std::min(kt.size(), (size_t)((r0 + m + TMr - 1) / TMr));
            const std::vector<long long> sub(kt.begin() + t0, kt.begin() + t1);
            gemm_half1(ctx->split, precision, W + r0 * ldw, ldw, B + n0, ldb, C + r0 * ldc + n0, ldc, m, nw,
                       d_kt + t0, sub, s, accumulate);
            ctx->launches++;
        }
    }
}

// First half of a batch: V rows = W D_ket over the density columns [c0, c1)
// of each column group (launches only; the MO-driven route passes one MO
// block, the others all columns).
void batch_half1(qdt_ctx *ctx, const ClassPlan &P, const RowBatch &B, long long c0, long long c1,
                 cudaStream_t s) {
    const long long N4 = P.N4, w = c1 - c0;
    const bool acc = P.mirror;      // earlier batches' transposed blocks are already in V
    if (!P.ls) {
        half1_rows(ctx, P.precision, B.W, B.ldw, P.Dket + c0, N4, P.Vc + B.row0 * N4 + c0, N4, B.rows, w, B.d_kt,
                   B.kt, s, acc);
        return;
    }
    if (P.cr.gauge) {
        // gauge: rows (ab, I), K (cd, J): D_ket viewed as [(cd, J)][4 nRS]
        half1_rows(ctx, P.precision, B.W, B.ldw, P.Dket + c0, N4, P.Vg + B.row0 * 3 * N4 + c0, N4, B.rows * 3, w,
                   B.d_kt, B.kt, s, acc);
    }
    if (P.cr.gaunt) {
        // Gaunt: Coulomb integrals over L-S pairs, columns (J, RS, part)
        const double *Wg = P.cr.gauge ? B.Wc : B.W;
        const long long ldg = P.cr.gauge ? B.ldwc : B.ldw;
        if (w == N4) {
            half1_rows(ctx, P.precision, Wg, ldg, P.Dket, 3 * N4, P.Vc + B.row0 * 3 * N4, 3 * N4, B.rows, 3 * N4,
                       B.d_kg, B.kg, s, acc);
        } else {
            for (int J = 0; J < 3; ++J)
                half1_rows(ctx, P.precision, Wg, ldg, P.Dket + J * N4 + c0, 3 * N4,
                           P.Vc + B.row0 * 3 * N4 + J * N4 + c0, 3 * N4, B.rows, w, B.d_kg, B.kg, s, acc);
        }
    }
}

// The transposed blocks of a batch (ClassPlan::mirror): V[later rows] +=
// W2 Dbra2, with Dbra2 the batch's density rows in W2's column order (all
// density columns: the mirror path is the AO-driven route's).
void batch_half1_mirror(qdt_ctx *ctx, const ClassPlan &P, const RowBatch &B, cudaStream_t s) {
    if (B.rows2 <= 0) return;
    const long long N4 = P.N4;
    split_forget(ctx->split, B.Dbra2, B.Dbra2 + B.ld2 * P.ncolD);     // new rows in the same buffer
    if (!P.ls) {
        half1_rows(ctx, P.precision, B.W2, B.ldw2, B.Dbra2, N4, P.Vc + B.row2 * N4, N4, B.rows2, N4, B.d_kt2, B.kt2,
                   s, true);
        return;
    }
    if (P.cr.gauge)
        half1_rows(ctx, P.precision, B.W2, B.ldw2, B.Dbra2, N4, P.Vg + B.row2 * 3 * N4, N4, B.rows2 * 3, N4,
                   B.d_kt2, B.kt2, s, true);
    if (P.cr.gaunt) {
        const double *Wg = P.cr.gauge ? B.Wc2 : B.W2;
        const long long ldg = P.cr.gauge ? B.ld2 : B.ldw2;
        half1_rows(ctx, P.precision, Wg, ldg, B.Dbra2, 3 * N4, P.Vc + B.row2 * 3 * N4, 3 * N4, B.rows2, 3 * N4,
                   B.d_kg2, B.kg2, s, true);
    }
}

// Rows per chunk of the quarter route: its FP64 intermediates within
// kQuarterBudget, the split form's digit planes of the largest A operand within
// kSliceBudget, and grid rows of the contraction within range.
long long quarter_chunk_rows(const qdt_ctx *ctx, const ClassPlan &P, long long rows) {
    const long long nL = ctx->nL, nS = ctx->nS, nX = nL + nS, n = P.nKa, Pp = P.ku ? 2 : 4;
    const double per = 8.0 * (double)(nL * nL + nS * nS + 2 * nX * 4 * n + n * Pp * n);
    long long rc = (long long)((double)kQuarterBudget / per);
    if (P.precision == QDT_SPLIT) {
        const double a = 12.0 * (double)std::max(nS * ((nS + 63) / 64 * 64), n * ((4 * nX + 63) / 64 * 64));
        rc = std::min(rc, (long long)((double)kSliceBudget / a));
    }
    rc = std::min(rc, (long long)(65535LL * 64 / std::max(nX, n)));
    if (const char *e = std::getenv("QDT_QUARTER_CHUNK_ROWS")) {      // smaller chunks, to exercise them
        const long long v = std::atoll(e);
        if (v <= 0) throw Error{QDT_ERR_ARG, "QDT_QUARTER_CHUNK_ROWS must be positive"};
        rc = std::min(rc, v);
    }
    return std::max<long long>(1, std::min(rc, rows));
}

// First half of a Coulomb batch by two quarter steps (launches only): integral
// rows -> square blocks, T1 = W C (quarter 1, L and S blocks), re-lay, V =
// T1 Cr2 (quarter 2), gather of the canonical column pairs into V.
void quarter_half1(qdt_ctx *ctx, const ClassPlan &P, const RowBatch &B, qdt_stats *st, cudaStream_t s) {
    const int TMr = gemm_fp64_tile_m();
    const long long nL = ctx->nL, nS = ctx->nS, nX = nL + nS, n = P.nKa, Pp = P.ku ? 2 : 4;
    const long long rc = quarter_chunk_rows(ctx, P, B.rows);
    double *WL = (double *)ctx->qWL.get((size_t)rc * nL * nL * sizeof(double));
    double *WS = (double *)ctx->qWS.get((size_t)rc * nS * nS * sizeof(double));
    double *T1 = (double *)ctx->qT1.get((size_t)rc * nX * 4 * n * sizeof(double));
    double *T = (double *)ctx->qT.get((size_t)rc * n * 4 * nX * sizeof(double));
    double *Vf = (double *)ctx->qVf.get((size_t)rc * n * Pp * n * sizeof(double));
    double *Cr1 = (double *)ctx->qCr1.p, *Cr2 = (double *)ctx->qCr2.p;
    // K extents per 64-row tile: constant for each of the three contractions
    const long long Ks[3] = {nL, nS, 4 * nX}, Ms[3] = {rc * nL, rc * nS, rc * n};
    std::vector<long long> hk[3];
    long long *dk[3];
    for (int g = 0; g < 3; ++g) {
        hk[g].assign((size_t)((Ms[g] + TMr - 1) / TMr), Ks[g]);
        dk[g] = dcopy_pinned(ctx->pin, ctx->qkt[g], hk[g], s);
    }
    auto sub = [&](int g, long long m) {
        return std::vector<long long>(hk[g].begin(), hk[g].begin() + (m + TMr - 1) / TMr);
    };
    const long long ncols = P.M;   // every ket column of the class
    for (long long r0 = 0; r0 < B.rows; r0 += rc) {
        const long long m = std::min(rc, B.rows - r0);
        launch_square_rows(B.W + r0 * B.ldw, B.ldw, P.qcols, ncols, (int)nL, (int)nS, m, WL, WS, s);
        gemm_half1(ctx->split, P.precision, WL, nL, Cr1, 4 * n, T1, 4 * n, m * nL, 4 * n, dk[0], sub(0, m * nL), s);
        gemm_half1(ctx->split, P.precision, WS, nS, Cr1 + nL * 4 * n, 4 * n, T1 + m * nL * 4 * n, 4 * n, m * nS,
                   4 * n, dk[1], sub(1, m * nS), s);
        launch_t1_transpose(T1, T1 + m * nL * 4 * n, (int)nL, (int)nS, (int)n, m, T, s);
        gemm_half1(ctx->split, P.precision, T, 4 * nX, Cr2, Pp * n, Vf, Pp * n, m * n, Pp * n, dk[2],
                   sub(2, m * n), s);
        launch_quarter_gather(Vf, (int)n, (int)Pp, (const int *)ctx->rsR.p, (const int *)ctx->rsS.p, P.nRS, m,
                              P.Vc + (B.row0 + r0) * P.N4, s);
        ctx->launches += 6;
        if (st)
            st->flops_half1 += 2.0 * (double)m * (double)(nL * nL + nS * nS) * (double)(4 * n) +
                               2.0 * (double)(m * n) * (double)(4 * nX) * (double)(Pp * n);
    }
}

// Second-half operands of a class: the jobs (V, K, packed output) and buffers.
struct Half2 {
    struct Job { const double *V; long long K; double *out; };
    std::vector<Job> jobs;
    double *O = nullptr, *partial = nullptr;
    size_t pe = 0;
    long long NO = 0;
};

void half2_prepare(qdt_ctx *ctx, const ClassPlan &P, double *out_coul, double *out_gaunt, double *out_gauge,
                   Half2 &H) {
    H = Half2();
    H.NO = P.N4;
    H.O = (double *)ctx->O.get(std::max<long long>(1, H.NO * H.NO) * sizeof(double));
    H.pe = (size_t)std::max<long long>(1, H.NO * H.NO) * 8;
    if (H.pe * sizeof(double) > ((size_t)4 << 30))
        H.pe = std::max<size_t>((size_t)H.NO * H.NO, ((size_t)4 << 30) / sizeof(double));
    H.partial = (double *)ctx->partial.get(H.pe * sizeof(double));
    if (!P.ls) H.jobs.push_back({P.Vc, P.M, out_coul});
    if (P.ls && P.cr.gaunt) H.jobs.push_back({P.Vc, 3 * P.M, out_gaunt});
    if (P.ls && P.cr.gauge) H.jobs.push_back({P.Vg, 3 * P.M, out_gauge});
}

// O = Dq^T V and packing of one job (launches only).
void half2_job(qdt_ctx *ctx, const ClassPlan &P, const Half2 &H, const Half2::Job &j, cudaStream_t s) {
    launch_zero(H.O, H.NO * H.NO, s);
    gemm_half2(ctx->split, P.precision, P.Dbra, P.N4, j.V, P.N4, H.O, H.NO, j.K, H.partial, H.pe, s);
    ctx->launches += 3;
}

void half2_pack(qdt_ctx *ctx, const ClassPlan &P, const Half2 &H, const Half2::Job &j, cudaStream_t s) {
    launch_pack(H.O, H.NO, P.nRS, P.ku ? 2 : 4, j.out, s);
    ctx->launches++;
}

void half2_stats(const Half2 &H, qdt_stats *st) {
    if (!st) return;
    for (const Half2::Job &j : H.jobs) st->flops_half2 += 2.0 * (double)j.K * (H.NO * (H.NO + 1) / 2.0);
}

// Step 4 for the current ket order: batches of bra rows, integral rows then
// the first half over the density columns [c0, c1).
void run_batches(qdt_ctx *ctx, ClassPlan &P, long long c0, long long c1, qdt_stats *st, Timer &tm,
                 double &ms_eri, double &ms_h1) {
    PairClass &pc = ctx->cls[P.cr.c];
    cudaStream_t s = ctx->stream;
    if (P.mirror) {     // every batch adds into V (its own rows and, transposed, the later ones)
        if (P.Vc) launch_zero(P.Vc, P.M * P.NV, s);
        if (P.Vg) launch_zero(P.Vg, 3 * P.M * P.N4, s);
    }
    int b0 = 0;
    while (b0 < pc.nsp) {
        RowBatch B;
        batch_prepare(ctx, P, b0, B);
        const EriParams *d_prm = dcopy_pinned(ctx->pin, ctx->prms, std::vector<EriParams>{B.prm}, s);
        const EriShape shape{pc.maxnfp, pc.maxLab, pc.maxnpp};
        const bool df = B.prm.E2 != nullptr;
        const std::vector<int> &pre = P.mirror ? B.pre1 : P.h_prefix;       // in the kernel's ket list
        const EriLaunch how = eri_launch_for(ctx, pc, shape, B.prm.gauge != 0, df, d_prm, B.bras, pre, s);
        EriTask *d_tk = nullptr;
        const int ntiles = launch_build_tiles(ctx, tile_order(pc, B.bras, how.order), pre,
                                              df ? (P.mirror ? &B.split1 : &P.h_split) : nullptr,
                                              P.mirror ? B.d_pre1 : P.prefix, P.mirror ? B.d_split1 : P.d_split,
                                              how.kets, d_tk, s);
        int te = tm.n; tm.mark();
        if (P.quarter) {    // the quarter route lays out whole rows
            launch_zero(B.W, B.rows * P.mult * B.ldw, s);
        } else {            // the rest reads each row tile only as far as its K extent
            launch_zero_rows(B.W, B.ldw, B.rows * P.mult, B.d_kt, (long long)B.kt.size(), s);
            if (B.Wc) launch_zero_rows(B.Wc, B.ldwc, B.rows, B.d_kg, (long long)B.kg.size(), s);
        }
        if (B.W2) launch_zero_rows(B.W2, B.ldw2, B.rows2 * P.mult, B.d_kt2, (long long)B.kt2.size(), s);
        if (B.Wc2) launch_zero_rows(B.Wc2, B.ld2, B.rows2, B.d_kg2, (long long)B.kg2.size(), s);
        launch_eri(d_prm, d_tk, ntiles, (int *)ctx->next.get(sizeof(int)), shape, B.prm.gauge != 0, df, how, s);
        ctx->launches += 2 + (B.Wc ? 1 : 0);
        batch_stats(ctx, P, B, c1 - c0, st);
        int th = tm.n; tm.mark();
        if (P.quarter) {
            quarter_half1(ctx, P, B, st, s);
        } else {
            batch_half1(ctx, P, B, c0, c1, s);
            if (P.mirror) batch_half1_mirror(ctx, P, B, s);
        }
        int tend = tm.n; tm.mark();
        QDT_CUDA_TRY(cudaStreamSynchronize(s));
        ms_eri += tm.ms(te, th);
        ms_h1 += tm.ms(th, tend);
        tm.n = te;   // reuse the batch's events
        b0 = B.b1;
    }
}

void run_class(qdt_ctx *ctx, const ClassRun &cr, int k0, int nKa, double tau, int precision,
               double *out_coul, double *out_gaunt, double *out_gauge, qdt_stats *st, Timer &tm,
               double acc_ms[6]) {
    PairClass &pc = ctx->cls[cr.c];
    cudaStream_t s = ctx->stream;
    ClassPlan P;
    const int t0 = tm.n;
    class_issue(ctx, cr, k0, nKa, tau, precision, P, tm);
    double ms_eri = 0, ms_h1 = 0;
    const int parts = P.ku ? 2 : 4;
    const int nb = ctx->route == QDT_ROUTE_MO ? std::max(1, ctx->mo_block) : nKa;
    if (nb >= nKa) {
        class_finish(ctx, P, st);
        run_batches(ctx, P, 0, P.N4, st, tm, ms_eri, ms_h1);
    } else {
        // MO-driven: the outer MO index r runs in blocks; each block of density
        // columns (r, s >= r) is screened on its own Dmax and recomputes every
        // integral it keeps
        auto col = [&](int r) { return (long long)parts * (r * (long long)nKa - (long long)r * (r - 1) / 2); };
        for (int r0 = 0; r0 < nKa; r0 += nb) {
            const int r1 = std::min(nKa, r0 + nb);
            const long long c0 = col(r0), c1 = r1 < nKa ? col(r1) : P.N4;
            launch_block_dmax(pc.d_pairs, pc.nsp, P.Dbra, P.ncolD, P.ls ? 3 : 1, P.N4, c0, c1, P.Dmax, s);
            ctx->launches++;
            order_kets(ctx, P, s);
            split_invalidate(ctx->split);
            P.mo_blocks = true;
            class_finish(ctx, P, st);
            run_batches(ctx, P, c0, c1, st, tm, ms_eri, ms_h1);
        }
    }
    acc_ms[2] += ms_eri;
    acc_ms[3] += ms_h1;
    // 5. second half + packing, one block at a time
    Half2 H;
    half2_prepare(ctx, P, out_coul, out_gaunt, out_gauge, H);
    half2_stats(H, st);
    for (const Half2::Job &j : H.jobs) {
        int t2 = tm.n; tm.mark();
        half2_job(ctx, P, H, j, s);
        int t3 = tm.n; tm.mark();
        half2_pack(ctx, P, H, j, s);
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

// ------------------------------------------------------------------ batches
// Validated request of a batch: outputs split per block, host staging.
struct BatchReq {
    qdt_batch_item *it = nullptr;
    qdt_ctx *c = nullptr;
    int nKa = 0;
    bool dev_out = true;
    double *dst = nullptr, *o[3] = {nullptr, nullptr, nullptr};
    size_t need = 0;
    qdt_stats st{};
    int status = QDT_OK;
    std::string err;
    ClassPlan P;
    RowBatch B;
    Half2 H;
    bool active = false;       // has this round's class
    bool fused = false;        // this round runs in the fused sequence
};

// Everything the captured sequence of a round reads or writes, plus the
// screening outcome; equal signatures give the same launch sequence.
uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ULL; }
    return h;
}
template <class T> uint64_t fnv_v(uint64_t h, const std::vector<T> &v) {
    const size_t n = v.size();
    h = fnv(h, &n, sizeof n);
    return v.empty() ? h : fnv(h, v.data(), v.size() * sizeof(T));
}

constexpr int kKinds = 4;           // integral kernel kinds: (gauge kernel) x (compensated FP32)
inline int kind_of(const EriParams &p) { return (p.gauge ? 2 : 0) + (p.E2 ? 1 : 0); }

uint64_t round_signature(const std::vector<BatchReq *> &fz, const std::vector<EriTask> tiles[kKinds],
                         const EriLaunch how[kKinds], const EriShape shape[kKinds]) {
    uint64_t h = 1469598103934665603ULL;
    for (int k = 0; k < kKinds; ++k) {
        h = fnv_v(h, tiles[k]);
        h = fnv(h, &how[k], sizeof(EriLaunch));
        h = fnv(h, &shape[k], sizeof(EriShape));
    }
    for (BatchReq *r : fz) {
        const ClassPlan &P = r->P;
        const RowBatch &B = r->B;
        h = fnv(h, &r->c, sizeof r->c);
        h = fnv(h, &P.precision, sizeof P.precision);
        h = fnv(h, &P.nKa, sizeof P.nKa);
        const void *ptrs[] = {P.Dbra, P.Dket, P.Vc, P.Vg, P.ketsp, P.ketcol, P.prefix, P.d_kpos, B.W, B.Wc,
                              B.d_kt, B.d_kg, r->H.O, r->H.partial, r->o[0], r->o[1], r->o[2]};
        h = fnv(h, ptrs, sizeof ptrs);
        h = fnv(h, &B.prm, sizeof B.prm);
        h = fnv_v(h, B.kt);
        h = fnv_v(h, B.kg);
        const long long sz[] = {B.rows, B.ldw, B.ldwc, B.row0, r->H.NO};
        h = fnv(h, sz, sizeof sz);
        for (int i = 0; i < SplitWorkspace::kSlots; ++i) {
            h = fnv(h, &r->c->split.buf[i], sizeof(void *));
            h = fnv(h, &r->c->split.bytes[i], sizeof(size_t));
        }
    }
    return h;
}

// The launch sequence of one batch round after screening: integral rows of all
// fused requests (one persistent launch per kernel kind over the shared tile
// queue), then every request's first half, second half and packing on its own
// stream.  Allocates nothing, copies nothing from the host and never waits, so
// it can be captured into a CUDA graph.
void issue_round(qdt_ctx *owner, const std::vector<BatchReq *> &fz, const EriParams *const d_prms[kKinds],
                 const EriTask *const d_tiles[kKinds], const int ntiles[kKinds], const EriShape shape[kKinds],
                 const EriLaunch how[kKinds]) {
    cudaStream_t s0 = owner->stream;
    for (BatchReq *r : fz) {
        split_clear_status(r->c->split, s0);
        launch_zero(r->B.W, r->B.rows * r->P.mult * r->B.ldw, s0);
        if (r->B.Wc) launch_zero(r->B.Wc, r->B.rows * r->B.ldwc, s0);
        r->c->launches += 1 + (r->B.Wc ? 1 : 0);
    }
    for (int k = 0; k < kKinds; ++k)
        if (ntiles[k] > 0) {
            launch_eri(d_prms[k], d_tiles[k], ntiles[k], (int *)owner->bnext[k].p, shape[k], (k & 2) != 0,
                       (k & 1) != 0, how[k], s0);
            owner->launches++;
        }
    QDT_CUDA_TRY(cudaEventRecord(owner->fork_ev, s0));
    for (BatchReq *r : fz) {
        cudaStream_t cs = r->c->stream;
        if (cs != s0) QDT_CUDA_TRY(cudaStreamWaitEvent(cs, owner->fork_ev, 0));
        batch_half1(r->c, r->P, r->B, 0, r->P.N4, cs);
        for (const Half2::Job &j : r->H.jobs) {
            half2_job(r->c, r->P, r->H, j, cs);
            half2_pack(r->c, r->P, r->H, j, cs);
        }
        if (cs != s0) {
            QDT_CUDA_TRY(cudaEventRecord(r->c->join_ev, cs));
            QDT_CUDA_TRY(cudaStreamWaitEvent(s0, r->c->join_ev, 0));
        }
    }
}

ClassRun round_class(int round, unsigned blocks) {
    if (round == 0) return ClassRun{0, true, false, false};
    return ClassRun{1, false, (blocks & QDT_GAUNT) != 0, (blocks & QDT_GAUGE) != 0};
}

bool round_wanted(int round, unsigned blocks) {
    return round == 0 ? (blocks & QDT_COULOMB) != 0 : (blocks & (QDT_GAUNT | QDT_GAUGE)) != 0;
}

void item_fail(BatchReq &r, const Error &e) {
    if (r.status == QDT_OK) {
        r.status = e.code;
        r.err = e.msg;
    }
    r.active = false;
    r.fused = false;
}

// One round (0: Coulomb class, 1: Gaunt/gauge class) of a batch.
void batch_round(qdt_ctx *owner, std::vector<BatchReq> &R, int round, unsigned flags) {
    cudaStream_t s0 = owner->stream;
    // screening of every request, issued on all streams before the first wait
    for (BatchReq &r : R) {
        r.active = r.status == QDT_OK && round_wanted(round, r.it->blocks);
        r.fused = false;
        if (!r.active) continue;
        try {
            Timer off(r.c, false);
            class_issue(r.c, round_class(round, r.it->blocks), r.it->k_begin, r.nKa, r.it->schwarz_tau,
                        r.it->precision, r.P, off);
        } catch (const Error &e) { item_fail(r, e); }
    }
    std::vector<BatchReq *> fz;
    for (BatchReq &r : R) {
        if (!r.active) continue;
        try {
            const qdt_stats before = r.st;
            class_finish(r.c, r.P, &r.st);
            batch_prepare(r.c, r.P, 0, r.B);
            r.fused = r.B.b1 == r.c->cls[r.P.cr.c].nsp;     // the whole class in one row batch
            if (r.fused) {
                half2_prepare(r.c, r.P, r.o[0], r.o[1], r.o[2], r.H);
                batch_stats(r.c, r.P, r.B, r.P.N4, &r.st);
                half2_stats(r.H, &r.st);
                fz.push_back(&r);
            } else {
                r.st = before;       // run_class below screens again and counts
            }
        } catch (const Error &e) { item_fail(r, e); }
    }
    if (!fz.empty()) {
        // shared tile queues, one per kernel kind (Coulomb or gauge kernel, FP64 or
        // compensated FP32 contraction); tiles of all requests of the kind
        std::vector<EriParams> prms[kKinds];
        std::vector<int> req_of(fz.size());
        EriShape shape[kKinds];
        for (size_t i = 0; i < fz.size(); ++i) {
            BatchReq *r = fz[i];
            const int k = kind_of(r->B.prm);
            req_of[i] = (int)prms[k].size();
            prms[k].push_back(r->B.prm);
            const PairClass &pc = r->c->cls[r->P.cr.c];
            shape[k].merge(EriShape{pc.maxnfp, pc.maxLab, pc.maxnpp});
        }
        const EriParams *d_prms[kKinds] = {};
        const EriTask *d_tiles[kKinds] = {};
        int ntiles[kKinds] = {};
        EriLaunch how[kKinds];
        std::vector<EriTask> tiles[kKinds];
        for (int k = 0; k < kKinds; ++k) {
            if (prms[k].empty()) continue;
            d_prms[k] = dcopy_pinned(owner->pin, owner->bprms[k], prms[k], s0);
            owner->bnext[k].get(sizeof(int));
            // the tuner samples the first request of this kind
            size_t first = 0;
            while (kind_of(fz[first]->B.prm) != k) ++first;
            how[k] = eri_launch_for(owner, fz[first]->c->cls[fz[first]->P.cr.c], shape[k], (k & 2) != 0,
                                    (k & 1) != 0, d_prms[k], fz[first]->B.bras, fz[first]->P.h_prefix, s0);
            // tile order across requests: request by request in bra order, or
            // all bra pairs most expensive first
            struct Key { double cost; int i; int sp; };
            std::vector<Key> order;
            for (size_t i = 0; i < fz.size(); ++i) {
                BatchReq *r = fz[i];
                if (kind_of(r->B.prm) != k) continue;
                const PairClass &pc = r->c->cls[r->P.cr.c];
                for (int sp : r->B.bras) order.push_back({bra_cost(pc.h_pairs[sp]), (int)i, sp});
            }
            if (how[k].order == 1)
                std::stable_sort(order.begin(), order.end(), [](const Key &a, const Key &b) { return a.cost > b.cost; });
            for (const Key &o : order) {
                const std::vector<int> &pre = fz[o.i]->P.h_prefix;
                const int mid = (k & 1) ? fz[o.i]->P.h_split[o.sp] : pre[o.sp];    // FP32 tail (split form)
                for (int q = 0; q < mid; q += how[k].kets)
                    tiles[k].push_back({o.sp, q, std::min(mid, q + how[k].kets), req_of[o.i], 0});
                for (int q = mid; q < pre[o.sp]; q += how[k].kets)
                    tiles[k].push_back({o.sp, q, std::min(pre[o.sp], q + how[k].kets), req_of[o.i], 1});
            }
            d_tiles[k] = dcopy_pinned(owner->pin, owner->btasks[k], tiles[k], s0);
            ntiles[k] = (int)tiles[k].size();
        }
        for (BatchReq *r : fz) r->c->split.deferred = true;
        QDT_CUDA_TRY(cudaStreamSynchronize(s0));          // uploads done before any capture
        GraphEntry &g = owner->graph[round];
        const bool graph = (flags & QDT_BATCH_GRAPH) != 0;
        uint64_t sig = graph ? round_signature(fz, tiles, how, shape) : 0;
        const void *own[3 * kKinds];
        for (int k = 0; k < kKinds; ++k) {
            own[3 * k] = owner->bprms[k].p;
            own[3 * k + 1] = owner->btasks[k].p;
            own[3 * k + 2] = owner->bnext[k].p;
        }
        sig = fnv(sig, own, sizeof own);
        try {
            if (!graph) {
                issue_round(owner, fz, d_prms, d_tiles, ntiles, shape, how);
            } else if (g.exec && g.sig == sig) {
                QDT_CUDA_TRY(cudaGraphLaunch(g.exec, s0));
                owner->graph_replays++;
            } else if (g.seen && g.sig == sig) {
                // second sighting: every buffer already has its size, so the
                // sequence can be captured and replayed from now on
                QDT_CUDA_TRY(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
                try {
                    issue_round(owner, fz, d_prms, d_tiles, ntiles, shape, how);
                } catch (...) {
                    cudaGraph_t dead = nullptr;
                    cudaStreamEndCapture(s0, &dead);
                    if (dead) cudaGraphDestroy(dead);
                    cudaGetLastError();
                    throw;
                }
                cudaGraph_t cg = nullptr;
                QDT_CUDA_TRY(cudaStreamEndCapture(s0, &cg));
                cudaGraphExec_t ex = nullptr;
                const cudaError_t ie = cudaGraphInstantiate(&ex, cg, 0);
                cudaGraphDestroy(cg);
                QDT_CUDA_TRY(ie);
                if (g.exec) cudaGraphExecDestroy(g.exec);
                g.exec = ex;
                QDT_CUDA_TRY(cudaGraphLaunch(g.exec, s0));
                owner->graph_captures++;
            } else {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
                g.sig = sig;
                g.seen = 1;
                issue_round(owner, fz, d_prms, d_tiles, ntiles, shape, how);
            }
            QDT_CUDA_TRY(cudaStreamSynchronize(s0));
        } catch (const Error &e) {
            for (BatchReq *r : fz) {
                r->c->split.deferred = false;
                item_fail(*r, e);
            }
            fz.clear();
        }
        for (BatchReq *r : fz) {
            try {
                split_end_deferred(r->c->split, r->c->stream);
            } catch (const Error &e) { item_fail(*r, e); }
        }
    }
    // requests too large for one row batch run alone
    for (BatchReq &r : R) {
        if (!r.active || r.fused) continue;
        try {
            Timer off(r.c, false);
            double acc[6] = {0, 0, 0, 0, 0, 0};
            run_class(r.c, round_class(round, r.it->blocks), r.it->k_begin, r.nKa, r.it->schwarz_tau,
                      r.it->precision, r.o[0], r.o[1], r.o[2], &r.st, off, acc);
        } catch (const Error &e) { item_fail(r, e); }
    }
}

}  // namespace

namespace qdt {
// Frees the per-transformation workspace of a context (densities, integral
// rows, partial results, tile lists, split-form digit planes, comparator
// buffers) and drops captured batch graphs that point into it; the basis
// tables and coefficients stay.  The server calls it after every request, so
// a slot does not keep the peak buffers of its largest request.
void release_workspace(qdt_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    DBuf *bufs[] = {&c->Dbra, &c->Dket, &c->V, &c->Vg, &c->W, &c->Wc, &c->Dmax, &c->wsort, &c->ketsp, &c->ketcol,
                    &c->prefix, &c->ktile, &c->tasks, &c->O, &c->partial, &c->stage, &c->kpos, &c->prms,
                    &c->next, &c->ktile2, &c->qcols, &c->qWL, &c->qWS, &c->qT1, &c->qT, &c->qVf, &c->qkt[0],
                    &c->qkt[1], &c->qkt[2], &c->W2, &c->Wc2, &c->ktile3, &c->ktile4, &c->col2, &c->ketsp2,
                    &c->ketcol2, &c->Dbra2, &c->tbras, &c->toff, &c->dsplit, &c->klist, &c->kcol1, &c->kpos1,
                    &c->kpre1, &c->ksplit1};
    for (DBuf *b : bufs) b->release();
    split_release(c->split);
    for (GraphEntry &g : c->graph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = GraphEntry();
    }
    cudaGetLastError();
}
}  // namespace qdt

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
        QDT_CUDA_TRY(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
        QDT_CUDA_TRY(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
        // FP64 table [kBoysGrid][kBoysCols], then its FP32 and FP32-pair forms (boys_tables)
        double *tab = (double *)c->boys.get(kBoysBytes);
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
                    &c->prefix, &c->ktile, &c->tasks, &c->O, &c->partial, &c->stage, &c->rsR, &c->rsS,
                    &c->kpos, &c->prms, &c->next, &c->ktile2, &c->bprms[0], &c->bprms[1],
                    &c->bprms[2], &c->bprms[3], &c->btasks[0], &c->btasks[1], &c->btasks[2],
                    &c->btasks[3], &c->bnext[0], &c->bnext[1], &c->bnext[2], &c->bnext[3], &c->qcols,
                    &c->qWL, &c->qWS, &c->qT1, &c->qT, &c->qVf, &c->qCr1, &c->qCr2, &c->qkt[0],
                    &c->qkt[1], &c->qkt[2], &c->W2, &c->Wc2, &c->ktile3, &c->ktile4, &c->col2, &c->ketsp2,
                    &c->ketcol2, &c->Dbra2, &c->tbras, &c->toff, &c->dsplit, &c->klist, &c->kcol1, &c->kpos1,
                    &c->kpre1, &c->ksplit1};
    for (DBuf *b : bufs) b->release();
    for (int k = 0; k < 2; ++k) {
        c->cb[k].pairs.release(); c->cb[k].pp.release(); c->cb[k].E.release(); c->cb[k].E2.release(); c->cb[k].E1.release();
        c->cb[k].Q.release(); c->cb[k].bra.release(); c->cb[k].brapos.release(); c->cb[k].pp_pair.release();
    }
    split_release(c->split);
    c->pin.release();
    for (GraphEntry &g : c->graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int i = 0; i < 16; ++i) cudaEventDestroy(c->ev[i]);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
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

}  // extern "C"

namespace {
// c_light > 0: CS holds nL restricted-kinetic-balance rows (Eq. RKB), mapped
// onto the 3 nL derivative-function rows on the device first.
int set_coefficients(qdt_ctx *c, int nK, const double *CL, const double *CS, bool ku, double c_light,
                     const char *who) {
    if (!c) return QDT_ERR_ARG;
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->has_basis) throw Error{QDT_ERR_STATE, std::string(who) + ": no basis"};
        arg_check(nK > 0 && CL && CS, std::string(who) + ": the count must be positive and the arrays non-null");
        arg_check(c_light >= 0.0 && std::isfinite(c_light), std::string(who) + ": c must be positive and finite");
        c->has_coef = false;
        // CL as given; CS (3 nL rows) merged onto the internal derivative functions
        const bool rkb = c_light > 0.0;
        size_t nl = (size_t)c->nL * nK * 4, ns_in = (size_t)3 * c->nL * nK * 4, ns = (size_t)c->nS * nK * 4;
        double *d = (double *)c->Cq.get((nl + ns) * sizeof(double));
        double *raw = (double *)c->Craw.get((ns_in + (rkb ? nl : 0)) * sizeof(double));
        QDT_CUDA_TRY(cudaMemcpyAsync(d, CL, nl * sizeof(double), cudaMemcpyDefault, c->stream));
        if (rkb) {
            QDT_CUDA_TRY(cudaMemcpyAsync(raw + ns_in, CS, nl * sizeof(double), cudaMemcpyDefault, c->stream));
            launch_rkb_map(raw + ns_in, c->nL, nK, c_light, raw, c->stream);
        } else {
            QDT_CUDA_TRY(cudaMemcpyAsync(raw, CS, ns_in * sizeof(double), cudaMemcpyDefault, c->stream));
        }
        launch_merge_rows(raw, (const int *)c->dsmap0.p, (const int *)c->dsmap1.p, c->nS, nK * 4, d + nl, c->stream);
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->nK = nK;
        c->ku = ku;
        c->has_coef = true;
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}
}  // namespace

extern "C" {

int qdt_set_coefficients(qdt_ctx *c, int nK, const double *CL, const double *CS) {
    return set_coefficients(c, nK, CL, CS, false, 0.0, "qdt_set_coefficients");
}

int qdt_set_spinor_coefficients(qdt_ctx *c, int n_spinors, const double *CL, const double *CS) {
    return set_coefficients(c, n_spinors, CL, CS, true, 0.0, "qdt_set_spinor_coefficients");
}

int qdt_set_rkb_coefficients(qdt_ctx *c, int n, const double *CL, const double *CS, double c_light,
                             int spinors) {
    if (!(c_light > 0.0)) {
        if (c) c->err = "qdt_set_rkb_coefficients: c must be positive";
        return QDT_ERR_ARG;
    }
    return set_coefficients(c, n, CL, CS, spinors != 0, c_light, "qdt_set_rkb_coefficients");
}

int qdt_f32_error_ratio(qdt_ctx *c, unsigned blocks, int k_begin, int k_end, double tau, double *ratio) {
    if (!c || !ratio) return QDT_ERR_ARG;
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->has_basis || !c->has_coef) throw Error{QDT_ERR_STATE, "qdt_f32_error_ratio: basis or coefficients not set"};
        arg_check(blocks != 0 && (blocks & ~7u) == 0 && k_begin >= 0 && k_end > k_begin && k_end <= c->nK &&
                      tau >= 0.0, "qdt_f32_error_ratio: bad blocks, range or threshold");
        cudaStream_t s = c->stream;
        for (int cls = 0; cls < 2; ++cls) {
            ratio[cls] = 0.0;
            const bool want = cls == 0 ? (blocks & QDT_COULOMB) != 0 : (blocks & (QDT_GAUNT | QDT_GAUGE)) != 0;
            if (!want) continue;
            ClassRun cr{cls, cls == 0, cls == 1 && (blocks & QDT_GAUNT), cls == 1 && (blocks & QDT_GAUGE)};
            PairClass &pc = c->cls[cls];
            ClassPlan P;
            Timer tm(c, false);
            class_issue(c, cr, k_begin, k_end - k_begin, tau, QDT_SPLIT, P, tm);
            class_finish(c, P, nullptr);
            RowBatch B;
            batch_prepare(c, P, 0, B);
            arg_check(P.one_batch && B.b1 == pc.nsp, "qdt_f32_error_ratio: the class must fit one row batch");
            const EriParams *d_prm = dcopy(c->prms, std::vector<EriParams>{B.prm}, s);
            const EriShape shape{pc.maxnfp, pc.maxLab, pc.maxnpp};
            EriLaunch how;
            how.threads = eri_default_threads(shape, B.prm.gauge != 0);
            const size_t n = (size_t)B.rows * P.mult * B.ldw;
            struct Bufs {         // released on every exit path
                DBuf ref, rp, cp, out;
                ~Bufs() { ref.release(); rp.release(); cp.release(); out.release(); }
            } tmp;
            double *W2 = (double *)tmp.ref.get(std::max<size_t>(1, n) * sizeof(double));
            std::vector<int> none(pc.nsp, 0);
            for (int pass = 0; pass < 2; ++pass) {      // compensated FP32, then plain FP32
                std::vector<EriTask> tk;
                build_tiles(B.bras, P.h_prefix, how.kets, 0, tk, pass ? &none : nullptr);
                EriTask *d_tk = dcopy(c->tasks, tk, s);
                launch_zero(B.W, (long long)n, s);
                launch_eri(d_prm, d_tk, (int)tk.size(), (int *)c->next.get(sizeof(int)), shape, B.prm.gauge != 0, true,
                           how, s);
                if (pass == 0) QDT_CUDA_TRY(cudaMemcpyAsync(W2, B.W, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            }
            std::vector<int> rp(P.M), cp(P.M);
            for (int k = 0; k < pc.nsp; ++k) {
                const PairDev &pr = pc.h_pairs[pc.bra_order[k]];
                for (int f = 0; f < pr.nfp; ++f) rp[pr.rowoff + f] = pc.bra_order[k];
            }
            for (int q = 0; q < pc.nsp; ++q)
                for (long long j = P.h_col[q]; j < P.h_col[q + 1]; ++j) cp[j] = P.h_ketsp[q];
            const int *d_rp = dcopy(tmp.rp, rp, s), *d_cp = dcopy(tmp.cp, cp, s);
            double *d_out = (double *)tmp.out.get(sizeof(double));
            QDT_CUDA_TRY(cudaMemsetAsync(d_out, 0, sizeof(double), s));
            launch_ratio(B.W, W2, B.rows * P.mult, B.ldw, P.mult, d_rp, d_cp, P.M, pc.d_Q, d_out, s);
            QDT_CUDA_TRY(cudaMemcpyAsync(&ratio[cls], d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
            QDT_CUDA_TRY(cudaStreamSynchronize(s));
        }
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}

int qdt_check_bounded_wait(qdt_ctx *c, double limit_s) {
    if (!c) return QDT_ERR_ARG;
    if (!(limit_s > 0.0 && limit_s <= 2.0)) {
        c->err = "qdt_check_bounded_wait: the limit must be in (0, 2] seconds";
        return QDT_ERR_ARG;
    }
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        if (split_wait_probe(c->split, limit_s, c->stream)) {
            c->err = "qdt_check_bounded_wait: the wait gave up after its limit, as it should";
            return QDT_ERR_TIMEOUT;
        }
        throw Error{QDT_ERR_CUDA, "qdt_check_bounded_wait: a wait on an mbarrier nothing arrives at completed"};
    } catch (const Error &e) {
        return fail(c, e);
    }
}

int qdt_set_route(qdt_ctx *c, int route, int mo_block) {
    if (!c) return QDT_ERR_ARG;
    if (route != QDT_ROUTE_DENSITY && route != QDT_ROUTE_QUARTER && route != QDT_ROUTE_MO) {
        c->err = "qdt_set_route: route must be QDT_ROUTE_DENSITY, QDT_ROUTE_QUARTER or QDT_ROUTE_MO";
        return QDT_ERR_ARG;
    }
    if (route == QDT_ROUTE_MO && mo_block <= 0) {
        c->err = "qdt_set_route: the MO-driven route needs a positive block size";
        return QDT_ERR_ARG;
    }
    c->route = route;
    c->mo_block = route == QDT_ROUTE_MO ? mo_block : 0;
    c->err.clear();
    return QDT_OK;
}

size_t qdt_packed_size(const qdt_ctx *c, unsigned blocks, int k_begin, int k_end) {
    if (k_end <= k_begin) return 0;
    const bool ku = c && c->has_coef && c->ku;
    int nb = ((blocks & QDT_COULOMB) ? 1 : 0) + ((blocks & QDT_GAUNT) ? 1 : 0) + ((blocks & QDT_GAUGE) ? 1 : 0);
    return (size_t)packed_block_elems(ku, k_end - k_begin) * sizeof(double) * nb;
}

int qdt_transform(qdt_ctx *c, unsigned blocks, int k_begin, int k_end, double tau, int precision,
                  double *out, size_t out_bytes, qdt_stats *st) {
    if (!c) return QDT_ERR_ARG;
    try {
        cudaGetLastError();      // start from a clean error state
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        if (!c->has_basis || !c->has_coef) throw Error{QDT_ERR_STATE, "qdt_transform: basis or coefficients not set"};
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));      // staged uploads of earlier calls have landed
        c->pin.reset();
        arg_check(blocks != 0 && (blocks & ~7u) == 0, "qdt_transform: blocks must be a non-empty subset of COULOMB|GAUNT|GAUGE");
        arg_check(k_begin >= 0 && k_end > k_begin && k_end <= c->nK, "qdt_transform: bad Kramers-pair (or spinor) range");
        arg_check(tau >= 0.0, "qdt_transform: negative Schwarz threshold");
        arg_check(precision == QDT_FP64 || precision == QDT_SPLIT, "qdt_transform: bad precision");
        size_t need = qdt_packed_size(c, blocks, k_begin, k_end);
        arg_check(out != nullptr && out_bytes >= need, "qdt_transform: output buffer too small");
        const int nKa = k_end - k_begin;
        const long long per = packed_block_elems(c->ku, nKa);
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

int qdt_transform_batch(qdt_batch_item *items, int n, unsigned flags) {
    if (!items || n <= 0 || (flags & ~QDT_BATCH_GRAPH)) return QDT_ERR_ARG;
    std::vector<BatchReq> R(n);
    qdt_ctx *owner = nullptr;
    for (int i = 0; i < n; ++i) {
        BatchReq &r = R[i];
        r.it = &items[i];
        r.c = items[i].ctx;
        try {
            arg_check(r.c != nullptr, "qdt_transform_batch: null context");
            for (int j = 0; j < i; ++j) arg_check(items[j].ctx != r.c, "qdt_transform_batch: a context appears twice");
            if (!owner) owner = r.c;
            arg_check(r.c->device == owner->device, "qdt_transform_batch: contexts on different devices");
            QDT_CUDA_TRY(cudaSetDevice(r.c->device));
            cudaGetLastError();
            if (!r.c->has_basis || !r.c->has_coef) throw Error{QDT_ERR_STATE, "qdt_transform_batch: basis or coefficients not set"};
            if (r.c->route != QDT_ROUTE_DENSITY)
                throw Error{QDT_ERR_UNIMPLEMENTED, "qdt_transform_batch: the quarter and MO-driven routes run through qdt_transform only"};
            const qdt_batch_item &it = items[i];
            arg_check(it.blocks != 0 && (it.blocks & ~7u) == 0, "qdt_transform_batch: blocks must be a non-empty subset of COULOMB|GAUNT|GAUGE");
            arg_check(it.k_begin >= 0 && it.k_end > it.k_begin && it.k_end <= r.c->nK, "qdt_transform_batch: bad Kramers range");
            arg_check(it.schwarz_tau >= 0.0, "qdt_transform_batch: negative Schwarz threshold");
            arg_check(it.precision == QDT_FP64 || it.precision == QDT_SPLIT, "qdt_transform_batch: bad precision");
            r.need = qdt_packed_size(r.c, it.blocks, it.k_begin, it.k_end);
            arg_check(it.out != nullptr && it.out_bytes >= r.need, "qdt_transform_batch: output buffer too small");
            r.nKa = it.k_end - it.k_begin;
            const long long per = packed_block_elems(r.c->ku, r.nKa);
            r.dev_out = is_device_ptr(it.out);
            r.dst = r.dev_out ? it.out : (double *)r.c->stage.get(r.need);
            double *cur = r.dst;
            if (it.blocks & QDT_COULOMB) { r.o[0] = cur; cur += per; }
            if (it.blocks & QDT_GAUNT) { r.o[1] = cur; cur += per; }
            if (it.blocks & QDT_GAUGE) { r.o[2] = cur; cur += per; }
            r.st.precision = it.precision;
            r.st.slices = split_slices(r.c->split);
            r.c->launches = 0;
            QDT_CUDA_TRY(cudaStreamSynchronize(r.c->stream));  // staged uploads of earlier calls have landed
            r.c->pin.reset();
        } catch (const Error &e) {
            r.status = e.code;
            r.err = e.msg;
        }
    }
    if (owner) {
        try {
            QDT_CUDA_TRY(cudaSetDevice(owner->device));
            QDT_CUDA_TRY(cudaEventRecord(owner->ev[14], owner->stream));
            for (int round = 0; round < 2; ++round) batch_round(owner, R, round, flags);
            for (BatchReq &r : R)
                if (r.status == QDT_OK && !r.dev_out)
                    QDT_CUDA_TRY(cudaMemcpyAsync(r.it->out, r.dst, r.need, cudaMemcpyDeviceToHost, r.c->stream));
            for (BatchReq &r : R)
                if (r.status == QDT_OK) {
                    QDT_CUDA_TRY(cudaEventRecord(r.c->join_ev, r.c->stream));
                    QDT_CUDA_TRY(cudaStreamWaitEvent(owner->stream, r.c->join_ev, 0));
                }
            QDT_CUDA_TRY(cudaEventRecord(owner->ev[15], owner->stream));
            QDT_CUDA_TRY(cudaStreamSynchronize(owner->stream));
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, owner->ev[14], owner->ev[15]) != cudaSuccess) { cudaGetLastError(); ms = 0.f; }
            for (BatchReq &r : R) r.st.ms_total = ms;
        } catch (const Error &e) {
            for (BatchReq &r : R)
                if (r.status == QDT_OK) { r.status = e.code; r.err = e.msg; }
        }
    }
    int first = QDT_OK;
    for (int i = 0; i < n; ++i) {
        BatchReq &r = R[i];
        items[i].status = r.status;
        if (r.c) {
            if (r.status == QDT_OK) r.c->err.clear();
            else r.c->err = r.err;
        }
        if (items[i].stats && r.status == QDT_OK) {
            r.st.kernel_launches = r.c->launches;
            *items[i].stats = r.st;
        }
        if (first == QDT_OK && r.status != QDT_OK) first = r.status;
    }
    return first;
}

int qdt_graph_counts(const qdt_ctx *c, long long *captures, long long *replays) {
    if (!c) return QDT_ERR_ARG;
    if (captures) *captures = c->graph_captures;
    if (replays) *replays = c->graph_replays;
    return QDT_OK;
}

int qdt_unpack(qdt_ctx *c, const double *packed, int n_kramers, unsigned block, double *full) {
    if (!c) return QDT_ERR_ARG;
    try {
        QDT_CUDA_TRY(cudaSetDevice(c->device));
        arg_check(packed && full && n_kramers > 0, "qdt_unpack: bad arguments");
        arg_check(block == QDT_COULOMB || block == QDT_GAUNT || block == QDT_GAUGE, "qdt_unpack: one block");
        arg_check(is_device_ptr(packed) && is_device_ptr(full), "qdt_unpack: device pointers required");
        launch_unpack(packed, n_kramers, block != QDT_COULOMB, c->ku, full, c->stream);
        QDT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (const Error &e) {
        return fail(c, e);
    }
    c->err.clear();
    return QDT_OK;
}

const char *qdt_last_error(const qdt_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
