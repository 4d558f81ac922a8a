// qdt_internal.cuh -- internal types and helpers of libqdt (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/qdt.h"

namespace qdt {

// ------------------------------------------------------------------ limits
constexpr int kMaxLShell = QDT_MAX_L;              // large-component shell order
constexpr int kMaxLFunc = kMaxLShell + 1;          // derivative functions reach l+1
constexpr int kMaxLPair = 2 * kMaxLFunc;           // Hermite order of a pair
constexpr int kMaxLTot = 2 * kMaxLPair + 2;        // + 2 for the gauge kernel
constexpr int kBoysNMax = kMaxLTot + 1;            // orders needed
constexpr int kBoysTaylor = 7;                     // Taylor terms of the table
constexpr double kBoysDelta = 0.05;                // table spacing in T
constexpr double kBoysTMax = 36.0;                 // table range; asymptotic beyond
constexpr int kBoysGrid = 721;                     // 36 / 0.05 + 1
constexpr int kBoysCols = kBoysNMax + kBoysTaylor + 1;

__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

// The Boys tables in one device buffer: the FP64 table [kBoysGrid][kBoysCols],
// then its FP32 copy, its split into FP32 pairs (hi, lo), and per grid point
// exp(-T_i) and T_i = i kBoysDelta as pairs.
// floats of the FP32 copy, rounded up to an even count so the pairs after it are 8-byte aligned
constexpr size_t kBoysF32Slots = ((size_t)kBoysGrid * kBoysCols + 1) / 2 * 2;
struct BoysTables {
    const double *f64;
    float *f32;
    float2 *pair;
    float2 *exp_pair;
    float2 *t_pair;
};
__host__ __device__ inline BoysTables boys_tables(const double *tab) {
    BoysTables t;
    t.f64 = tab;
    t.f32 = reinterpret_cast<float *>(const_cast<double *>(tab) + (size_t)kBoysGrid * kBoysCols);
    t.pair = reinterpret_cast<float2 *>(t.f32 + kBoysF32Slots);         // 8-byte aligned
    t.exp_pair = t.pair + (size_t)kBoysGrid * kBoysCols;
    t.t_pair = t.exp_pair + kBoysGrid;
    return t;
}
constexpr size_t kBoysBytes = (size_t)kBoysGrid * kBoysCols * (sizeof(double) + sizeof(float2)) +
                              kBoysF32Slots * sizeof(float) + 2 * (size_t)kBoysGrid * sizeof(float2);

#ifdef __CUDACC__
// x = hi + lo with hi = fl32(x) and lo = fl32(x - hi) (an FP32 pair, ~48 bits)
__device__ inline float2 split_pair(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}
#endif
__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Hermite / Cartesian triple index: all triples of order <= L, ordered by
// order, then x-major inside one order.
__host__ __device__ inline int hidx(int t, int u, int v) {
    int s = t + u + v, uv = u + v;
    return s * (s + 1) * (s + 2) / 6 + uv * (uv + 1) / 2 + v;
}

// ------------------------------------------------------------------ errors
struct Error {
    int code;
    std::string msg;
};

#define QDT_CUDA_TRY(expr)                                                             \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess)                                                         \
            throw ::qdt::Error{QDT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
    } while (0)

#define QDT_STR2(x) #x
#define QDT_STR(x) QDT_STR2(x)
#define QDT_CHECK_LAUNCH() QDT_CHECK_KERNEL(__FILE__ ":" QDT_STR(__LINE__))
// launch check naming the kernel
#define QDT_CHECK_KERNEL(name)                                                         \
    do {                                                                               \
        cudaError_t _e = cudaGetLastError();                                           \
        if (_e != cudaSuccess)                                                         \
            throw ::qdt::Error{QDT_ERR_CUDA, std::string("launch of ") + (name) + ": " + cudaGetErrorString(_e)}; \
    } while (0)

inline void arg_check(bool ok, const std::string &m) {
    if (!ok) throw Error{QDT_ERR_ARG, m};
}

// ------------------------------------------------------------- device data
// One shell of the combined list: L shells 0..n-1, derivative (S) shells n..2n-1.
struct ShellDev {
    double A[3];
    int l;          // order of the parent large-component shell
    int isS;        // 1 for a derivative shell
    int nfunc;      // ncart(l) or 3 ncart(l)
    int foff;       // first function in the combined list F = L (0..nL-1), S (nL..)
    int nprim;
    int poff;       // first primitive in the exponent/coefficient arrays
    int noff;       // first normalisation constant (per Cartesian component)
    int red;        // derivative shell of a p shell kept as its 6 distinct functions
};

// Shell pair of a class.  Class 0 (Coulomb): LL pairs A<=B then SS pairs A<=B;
// class 1 (Gaunt and gauge): L x S pairs.
struct PairDev {
    int sa, sb;     // combined shell indices
    int nfp;        // function pairs stored (upper triangle if sa == sb)
    int Lab;        // Hermite order of the pair
    int npp;        // primitive pairs
    int ppoff;      // first primitive pair
    long long rowoff;   // first row in the bra (Q-sorted) order
};

struct PrimPairDev {
    double p;
    double inv_p;   // 1 / p
    double P[3];
    long long eoff; // offset of this primitive pair's E matrix [nherm(Lab)][nfp]
    int ia, ib;     // primitives of the two shells
};

// Primitive pairs with exp(-a b / (a+b) |A-B|^2) below this are dropped at
// set-up (their integrals are below 1e-24 of the pair's leading terms).
constexpr double kPrimPairTol = 1e-24;

// Host + device tables of one pair class.
struct PairClass {
    int nsp = 0;
    long long M = 0;            // function pairs (rows)
    std::vector<PairDev> h_pairs;
    std::vector<int> bra_order; // shell pair ids, Q descending
    std::vector<double> h_Q;
    PairDev *d_pairs = nullptr;
    PrimPairDev *d_pp = nullptr;
    double *d_E = nullptr;
    float2 *d_E2 = nullptr;     // E split into FP32 pairs (hi, lo) for the split form's integrals
    float *d_E1 = nullptr;      // the high parts alone, for the quartets run in plain FP32
    double *d_Q = nullptr;
    int *d_bra_order = nullptr;
    std::vector<int> bra_pos;   // bra position of every shell pair (inverse of bra_order)
    int *d_bra_pos = nullptr;
    long long npp_total = 0, e_total = 0;
    int maxnfp = 0, maxLab = 0, maxnpp = 0;
};

// ------------------------------------------------------------------ kernels
struct EriParams {
    const ShellDev *shells;
    const PairDev *pairs;
    const PrimPairDev *pp;
    const double *E;
    const float2 *E2;           // E as FP32 pairs: non-null selects the compensated FP32 contraction
    const float *E1;            // fl32(E), read by the tiles run in plain FP32
    const double *boys;         // [kBoysGrid][kBoysCols], followed by the same as floats
    // the ket list the tiles index: the w-sorted ket order of the class, or in
    // row batches with bra-ket symmetry the batch's own list (plan.h
    // batch_kets); positions, prefixes and columns below are in that list
    const int *ket_sp;          // shell pair id at each ket position
    const long long *ket_col;   // first column of each ket position
    double *W;                  // output rows
    long long ldw;
    long long row0;             // bra-order row of W's first row
    int gauge;                  // 0: Coulomb kernel; 1: gauge kernel (9 components)
    int with_coulomb;           // gauge mode: also write the plain Coulomb block
    double *Wc;                 // gauge mode: Coulomb block output (may be null)
    long long ldwc;
    // bra-ket symmetry: when (AB|CD) and (CD|AB) both survive, one block
    // serves both.  sym 1 (all rows in one batch): the task of the lower pair
    // id computes it and writes both.  sym 2 (row batches b0 <= bra position <
    // b1): a ket pair CD of the same batch as in sym 1; of a later batch, the
    // block is computed here and its transpose written into W2 (rows of the
    // later pairs, columns of this batch's pairs), which the first half
    // contracts into the later rows; of an earlier batch, skipped (its
    // transpose came from W2 of that batch).
    int sym;
    const int *ket_pos;         // ket position of every pair id in the list (sym 2: of the batch's pairs)
    const int *prefix;          // kept ket prefix length of every pair id, in list positions
    const int *bra_pos;         // sym 2: bra position of every pair id
    int b0, b1;                 // sym 2: this batch's bra positions
    double *W2;                 // sym 2: transposed blocks for later rows (gauge: 9 components)
    long long ldw2;
    long long row2;             // bra-order row of W2's first row (the first row after the batch)
    double *Wc2;                // sym 2, gauge mode: transposed plain Coulomb blocks (may be null)
    long long ldwc2;
    const long long *col2;      // sym 2: W2 column of every pair id of the batch
};

struct EriTask {                // one tile: bra shell pair x range of sorted ket positions
    int bra_sp;
    int k0, k1;
    int req;                    // index into the EriParams array of the launch
    int f32 = 0;                // compensated-FP32 kernels: 1 = these quartets in plain FP32
};

// Class maxima that fix the integral kernel's shared-memory plan.
struct EriShape {
    int maxnfp = 0, maxLab = 0, maxnpp = 0;
    void merge(const EriShape &o) {
        maxnfp = maxnfp > o.maxnfp ? maxnfp : o.maxnfp;
        maxLab = maxLab > o.maxLab ? maxLab : o.maxLab;
        maxnpp = maxnpp > o.maxnpp ? maxnpp : o.maxnpp;
    }
};

// Launch shape of the integral kernel (the autotuned part): CTA threads and
// ket positions per tile.  Neither changes the arithmetic of an integral.
struct EriLaunch {
    int threads = 0;            // 0: the plan's default
    int kets = 8;
    int order = 0;              // tile order: 0 bra pairs by Schwarz Q (bra order), 1 most expensive first
};

void launch_boys_table(double *d_tab, cudaStream_t s);
void launch_shell_norms(const ShellDev *shells, int nL_shells, const double *exps,
                        const double *coefs, double *norms, cudaStream_t s);
// Persistent integral kernel over a shared tile queue: `next` (device int,
// zeroed by this call) hands out the tiles in array order.  prms: device array
// of the parameter sets the tiles' `req` index.
// df: every parameter set carries E2 and the contractions run in compensated
// FP32 pairs (the split form); otherwise in FP64.
void launch_eri(const EriParams *prms, const EriTask *tasks, int ntasks, int *next, const EriShape &shape,
                bool gauge, bool df, const EriLaunch &how, cudaStream_t s);
// E2[i] = (hi, lo) with hi = fl32(E[i]), lo = fl32(E[i] - hi).
// max |A - B| / (Q_row Q_col) over integral rows (FP32 error model check).
void launch_ratio(const double *A, const double *B, long long rows, long long ldw, int mult, const int *row_pair,
                  const int *col_pair, long long ncols, const double *Q, double *out, cudaStream_t s);
void launch_split_pairs(const double *E, long long n, float2 *E2, float *E1, cudaStream_t s);
int eri_default_threads(const EriShape &shape, bool gauge);
void launch_schwarz(const ShellDev *shells, const PairDev *pairs, const PrimPairDev *pp,
                    const double *E, const double *boys, int npairs, int maxnfp, int maxLab,
                    int maxnpp, double *Q, cudaStream_t s);

void launch_ket_order(const double *Q, const double *Dmax, int nsp, double *w, int *ket_sp,
                      cudaStream_t s);
void launch_ket_columns(const PairDev *pairs, const int *ket_sp, int nsp, long long *ket_col,
                        cudaStream_t s);
void launch_prefix_lengths(const double *Q, const double *w_sorted, int nsp, double tau,
                           int *prefix, cudaStream_t s);
void launch_gather_rows(const double *src, const PairDev *pairs, const int *ket_sp,
                        const long long *ket_col, int nsp, long long rowlen, double *dst,
                        cudaStream_t s);

// GEMMs
// C (=, or += with accumulate) A B, K per 64-row tile from ktile.
void gemm_fp64_nn_ragged(const double *A, long long lda, const double *B, long long ldb,
                         double *C, long long ldc, long long M, long long N,
                         const long long *ktile, int tileM, cudaStream_t s, bool accumulate = false);
void gemm_fp64_tn_sym(const double *A, long long lda, const double *B, long long ldb, double *C,
                      long long N, long long K, double *partial, size_t partial_elems,
                      cudaStream_t s);
int gemm_fp64_tile_m();

// packing
// parts: 4 (Kramers pairs) or 2 (spinor pairs, Kramers-unrestricted input); nP units
void launch_pack(const double *O, long long ldo, int nP, int parts, double *out, cudaStream_t s);
// n_units: Kramers pairs (ku false, 2 n spinors) or spinors (ku true)
void launch_unpack(const double *packed, int n_units, int gaunt_like, bool ku, double *full, cudaStream_t s);
void launch_zero(double *p, long long n, cudaStream_t s);
// rows x ld integral rows, zeroed as far as the contractions read them (the
// K extents kt64 of its 64-row tiles, nt64 of them)
void launch_zero_rows(double *W, long long ld, long long rows, const long long *kt64, long long nt64,
                      cudaStream_t s);
// coefficient rows of the internal small-component basis: row r = in[m0[r]] (+ in[m1[r]])
// Eq. RKB: c^S[nL][n][4] -> derivative-function coefficients [3 nL][n][4].
void launch_rkb_map(const double *in, long long nL, long long n, double c_light, double *out,
                    cudaStream_t s);
// Dmax over the columns [c0, c1) of each of nJ column groups (MO-driven route).
void launch_block_dmax(const PairDev *pairs, int nsp, const double *D, long long ld, int nJ, long long N4,
                       long long c0, long long c1, double *Dmax, cudaStream_t s);
// Quarter-transform comparator of the Coulomb first half (quarter_kernels.cu).
void launch_ket_functions(const PairDev *pairs, const ShellDev *shells, const int *ket_sp,
                          const long long *ket_col, int nsp, int2 *cols, cudaStream_t s);
void launch_coef_bound(const PairDev *pairs, const ShellDev *shells, const double *Cq, int nK, int k0,
                       int nKa, int nsp, double *Dmax, cudaStream_t s);
void launch_quarter_coefs(const double *Cq, int nK, int k0, int n, int nX, int P, double *Cr1, double *Cr2,
                          cudaStream_t s);
void launch_square_rows(const double *W, long long ldw, const int2 *cols, long long ncols, int nL, int nS,
                        long long rows, double *WL, double *WS, cudaStream_t s);
void launch_t1_transpose(const double *TL, const double *TS, int nL, int nS, int n, long long rows, double *T,
                         cudaStream_t s);
void launch_quarter_gather(const double *Vf, int n, int P, const int *rsR, const int *rsS, int nRS,
                           long long rows, double *V, cudaStream_t s);
void launch_merge_rows(const double *in, const int *m0, const int *m1, int nrows, int rowlen, double *out,
                       cudaStream_t s);

// Frees a context's per-transformation workspace (basis tables and
// coefficients stay); the request server calls it after every request.
void release_workspace(qdt_ctx *c);

}  // namespace qdt
