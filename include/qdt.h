/*
 * qdt.h -- C ABI of the GB300 quaternion Dirac-Coulomb-Breit AO->MO integral
 * transformation library (libqdt.so).
 *
 * The library computes the four-index spinor MO integrals (pq|rs) of
 * arXiv 2606.04316 (Eqs. AOtoMO, DCInt, GauntInt, gaugeInt) by the AO-driven
 * direct quaternion-density route (Sec. 2.4, Eqs. Den, QuaternionScatter,
 * firsthalf, secondhalf) with density-weighted Cauchy-Schwarz screening
 * (Sec. 2.5, Eq. SchwarzDen).  Every arithmetic step of a transformation runs
 * in the library's own CUDA kernels on one sm_103a GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units: atomic units (bohr, hartree).
 *  - Large-component basis: contracted Cartesian Gaussians
 *      chi_mu = N_mu sum_p d_p (x-A_x)^i (y-A_y)^j (z-A_z)^k exp(-alpha_p |r-A|^2),
 *    every Cartesian component normalised to <chi|chi> = 1 by the library;
 *    components of a shell of order l in the order i = l..0, j = l-i..0.
 *  - Small-component basis: the derivative functions d/dr_K chi_mu, K = x,y,z,
 *    stored at index 3 mu + K (nS = 3 nL; restricted kinetic balance, Eq. RKB,
 *    with the factor sigma.p/(2c) carried by the coefficients).
 *  - MO coefficients are Kramers-restricted quaternions q = q0 + q1 i + q2 j + q3 k
 *    per basis row and Kramers pair k.  Spinor 2k has two-spinor coefficients
 *    (alpha, beta) = (q0 + i q1, q2 + i q3); spinor 2k+1 is its Kramers partner
 *    (-conj(beta), conj(alpha)).
 *  - Mulliken order: (pq|rs) = int int psi_p^+ O psi_q (1) K(r12) psi_r^+ O psi_s (2).
 *      QDT_COULOMB: O = 1, K = 1/r12                          (Eqs. Coulomb, DCInt)
 *      QDT_GAUNT:   sum_J O = alpha_J on both sides, K = 1/r12 (Eq. GauntInt)
 *      QDT_GAUGE:   sum_IJ alpha_I (1), alpha_J (2), K = r_I r_J / r^3 (Eq. gaugeInt)
 *    The Breit operator of Eq. breit is -1/2 GAUNT - 1/2 GAUGE; blocks are
 *    returned unsigned and separately.
 *  - Screening: shell quartet (AB|CD) is skipped iff Q_AB * (Q_CD * Dmax_CD) < tau,
 *    Q = max sqrt((ab|ab)) over the shell pair (Coulomb kernel, also for the
 *    gauge block), Dmax = max |real part| of the symmetrised quaternion density
 *    of the ket pair over its functions and all active Kramers-pair columns.
 *    tau = 0 keeps every quartet.
 *
 * Packed output layout (one block after another, COULOMB, GAUNT, GAUGE order
 * of the bits set in `blocks`): let n = k_end - k_begin active Kramers pairs,
 * pair index pq = P n - P (P-1)/2 + (Q - P) for P <= Q (nP = n(n+1)/2 pairs), and
 * quadruple index t = pq nP - pq (pq-1)/2 + (rs - pq) for pq <= rs.  Entry t holds
 * 16 doubles O[i][j] (i, j = 0..3) = sum_ab,cd Dq_i^{PQ}(ab) (ab|K|cd) Dq_j^{RS}(cd),
 * where Dq_0..3 are Re A, Im A, Re B, Im B of the symmetrised spinor densities
 * A = D^{2P,2Q}, B = D^{2P+1,2Q} (Eq. QuaternionScatter in real form).
 * qdt_unpack() expands it to the full complex (pq|rs).
 *
 * Errors: every int-returning call returns QDT_OK (0) or a negative QDT_ERR_*;
 * qdt_last_error() then describes the failure.  No call aborts the process
 * and no exception crosses the ABI.  A context is not thread-safe: use one
 * context per host thread.
 *
 * Pointers: inputs of qdt_set_basis / qdt_set_coefficients and the output of
 * qdt_transform may be host or device pointers (the library checks with
 * cudaPointerGetAttributes); the library copies inputs and never keeps a
 * caller pointer after the call returns.  All work is ordered on the
 * context's stream; qdt_transform returns after the output is complete.
 */
#ifndef QDT_H
#define QDT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QDT_OK 0
#define QDT_ERR_ARG (-1)            /* invalid argument or size                    */
#define QDT_ERR_OOM (-2)            /* device allocation failed                    */
#define QDT_ERR_CUDA (-3)           /* a CUDA runtime call or kernel failed        */
#define QDT_ERR_STATE (-4)          /* basis or coefficients not set               */
#define QDT_ERR_UNIMPLEMENTED (-5)  /* option not built                            */
#define QDT_ERR_TIMEOUT (-6)        /* a bounded device wait gave up               */
#define QDT_ERR_ADMISSION (-7)      /* request does not fit the memory pool        */

#define QDT_COULOMB 1u
#define QDT_GAUNT 2u
#define QDT_GAUGE 4u

#define QDT_FP64 0                  /* all-FP64 contractions                        */
#define QDT_SPLIT 1                 /* Ozaki BF16 slices, exact FP32 chunks, FP64 recombination */

#define QDT_ROUTE_DENSITY 0         /* first half through the pair density (Eq. firsthalf) */
#define QDT_ROUTE_QUARTER 1         /* Coulomb first half by two O(N^5) quarter steps      */
#define QDT_ROUTE_MO 2              /* MO-driven: integrals recomputed per outer-MO block   */
#define QDT_MAX_L 2                 /* largest large-component shell order accepted */

typedef struct qdt_ctx qdt_ctx;

/* Per-call statistics (filled when the pointer is non-NULL). */
typedef struct {
    double ms_total;            /* wall time of the call on the stream (CUDA events) */
    double ms_density;          /* quaternion pair density (Eq. Den)                  */
    double ms_screen;           /* screening: ket ordering and survivor counts        */
    double ms_eri;              /* AO integral tiles (stage i)                        */
    double ms_half1;            /* first half-transform GEMMs (Eq. firsthalf)         */
    double ms_half2;            /* second half-transform GEMMs (Eq. secondhalf)       */
    double ms_pack;             /* packing of the canonical quadruples                */
    double flops_half1;         /* algorithmic FP64-equivalent flops, first half      */
    double flops_half2;         /* algorithmic FP64-equivalent flops, second half     */
    long long quartets_total[3];/* shell quartets per block (Coulomb, Gaunt, gauge)   */
    long long quartets_kept[3]; /* shell quartets surviving the screening             */
    long long eri_values;       /* AO integral values produced                        */
    int kernel_launches;        /* library kernels launched by the call               */
    int precision;              /* QDT_FP64 or QDT_SPLIT                              */
    int slices;                 /* BF16 slices per operand in the split form          */
    double flops_eri;           /* FP64 flops of the integral contractions (E R E)    */
    long long quartets_f32[3];  /* split form: kept quartets whose integrals ran in   */
                                /* plain FP32 under the error budget                  */
    double f32_bound;           /* bound on their summed effect on any output element */
    double flops_eri_f32;       /* the part of flops_eri that ran in plain FP32       */
} qdt_stats;

/*
 * Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to
 * order all work on, or NULL for a stream the context creates and owns.
 * Returns QDT_OK and *ctx, or QDT_ERR_CUDA / QDT_ERR_OOM (then *ctx = NULL).
 */
int qdt_create(qdt_ctx **ctx, int device, void *cuda_stream);

/* Release every device and host resource of the context (NULL is allowed). */
void qdt_destroy(qdt_ctx *ctx);

/*
 * Set the large-component basis (the small-component derivative basis follows
 * from it).  xyz[n_centers][3]; per shell: centre index, order l (0..QDT_MAX_L),
 * number of primitives; exps/coefs hold sum(shell_nprim) exponents and raw
 * contraction coefficients, shell after shell.  Builds the shell-pair tables,
 * the Hermite expansion coefficients and the Schwarz diagonals on the GPU
 * (Eq. SchwarzDen).  Invalidates the coefficients.  QDT_ERR_ARG on bad sizes.
 */
int qdt_set_basis(qdt_ctx *ctx, int n_centers, const double *xyz, int n_shells,
                  const int *shell_center, const int *shell_l, const int *shell_nprim,
                  const double *exps, const double *coefs);

/* Number of large-component functions nL of the current basis (0 if none). */
int qdt_num_functions(const qdt_ctx *ctx);

/*
 * Set the quaternion MO coefficients: CL[nL][nK][4] and CS[3 nL][nK][4],
 * row-major doubles (host or device).  QDT_ERR_STATE without a basis.
 */
int qdt_set_coefficients(qdt_ctx *ctx, int nK, const double *CL, const double *CS);

/*
 * Kramers-unrestricted coefficients (the paper's own setting, Sec. 3): n
 * spinors, each with its own two-spinor coefficients, no Kramers partner.
 * CL: [nL][n][4], CS: [3 nL][n][4] doubles per row and spinor (Re alpha,
 * Im alpha, Re beta, Im beta), row order as for qdt_set_coefficients; host or
 * device, copied.  Replaces any coefficients set before.  qdt_transform then
 * takes [k_begin, k_end) as a spinor range and writes, per block, 4 reals
 * O[pq,i][rs,j] (i, j = Re, Im of the symmetrised spinor-pair densities
 * D^{pq}, p <= q, Eq. Den) for every canonical pair of pairs pq <= rs,
 * row-major over (pq, rs); D^{qp} = conj D^{pq} gives the rest (qdt_unpack).
 * qdt_set_coefficients switches back to quaternion input.
 */
int qdt_set_spinor_coefficients(qdt_ctx *ctx, int n_spinors, const double *CL, const double *CS);

/*
 * Restricted-kinetic-balance input (Eq. RKB, Sec. 2): the small component of
 * each spinor is (1/2c) sigma.p applied to large-component functions, so CS
 * has nL rows, CS[nL][n][4], like CL.  The library expands it over the
 * derivative functions d_K chi_mu (p = -i grad) with coefficients
 * (-i/2c) sigma_K c^S_mu on the device; the transform is then the same as
 * for the expanded coefficients.  spinors = 0: quaternion columns (as
 * qdt_set_coefficients, n = nK Kramers pairs); spinors != 0: unrestricted
 * spinors (as qdt_set_spinor_coefficients).  c_light > 0 (atomic units:
 * 137.035999084 by CODATA 2018; the paper's runs use 137.035999074).  QDT_ERR_ARG
 * on bad sizes or c; host or device, copied.
 */
int qdt_set_rkb_coefficients(qdt_ctx *ctx, int n, const double *CL, const double *CS, double c_light,
                             int spinors);

/*
 * Transformation route for later qdt_transform calls (Sec. 2.2, Sec. 3.3 and
 * the appendix's operation counts):
 *   QDT_ROUTE_DENSITY (default): AO-driven; every kept integral is computed
 *     once and contracted with the pair density (Eq. firsthalf).
 *   QDT_ROUTE_QUARTER, a comparator for the Coulomb block: the first half
 *     contracts one AO index at a time with the coefficients, T1 = sum_d
 *     (ab|cd) C_d then V = sum_c C*_c T1, and screens on coefficient bounds
 *     (2 max|C_c| max|C_d| per ket shell pair) since it forms no density.
 *     The Gaunt and gauge blocks take the density route.
 *   QDT_ROUTE_MO, a comparator for every block: MO-driven; the outer MO index
 *     r (Kramers pair or spinor of the active range) runs in blocks of
 *     mo_block, and each block screens on the density of its own columns
 *     (r, s >= r) and recomputes every integral it keeps.
 * The output layout and the second half are the same on every route.
 * mo_block is read for QDT_ROUTE_MO only (> 0).  qdt_transform_batch rejects
 * contexts on the comparator routes (QDT_ERR_UNIMPLEMENTED).  QDT_ERR_ARG on
 * an unknown route or a bad block size.
 */
int qdt_set_route(qdt_ctx *ctx, int route, int mo_block);

/*
 * Check of the split form's FP32 error model: for each requested class
 * (ratio[0] Coulomb, ratio[1] the L-S class of Gaunt/gauge) the kept
 * integral rows are computed twice, in compensated FP32 pairs and in plain
 * FP32, and ratio[c] = max |difference| / (Q_A Q_C) over all entries (Q the
 * Schwarz factors of the bra and ket shell pairs).  The split form lets a
 * quartet run in plain FP32 assuming this ratio stays below 256 x 2^-24.
 * Small inputs only: each class must fit one row batch (QDT_ERR_ARG).
 */
int qdt_f32_error_ratio(qdt_ctx *ctx, unsigned blocks, int k_begin, int k_end, double tau, double ratio[2]);

/*
 * Failure-detection self-check: runs the bounded wait that guards every
 * tensor-core pipeline wait on an mbarrier that nothing arrives at, with the
 * given limit (0 < limit_s <= 2).  Returns QDT_ERR_TIMEOUT when the wait gave
 * up and reported it through the device status word (the expected outcome;
 * the context stays usable), QDT_ERR_CUDA if it did not, QDT_ERR_ARG on a bad
 * limit.
 */
int qdt_check_bounded_wait(qdt_ctx *ctx, double limit_s);

/* Bytes of the packed output of qdt_transform for these blocks and range
   (for the input kind last set: quaternion or Kramers-unrestricted). */
size_t qdt_packed_size(const qdt_ctx *ctx, unsigned blocks, int k_begin, int k_end);

/*
 * Transform: packed (pq|rs) for the Kramers pairs [k_begin, k_end) of the
 * current coefficients, for every block bit set in `blocks`, with Schwarz
 * threshold `schwarz_tau` >= 0 and `precision` QDT_FP64 or QDT_SPLIT.
 * QDT_FP64: integrals and contractions in FP64.  QDT_SPLIT: contractions as
 * Ozaki BF16 slices on the tensor cores with FP64 recombination; integrals in
 * compensated FP32 pairs, except the quartets whose error bound fits a 3e-11
 * budget on every output element, which run in plain FP32 (the environment
 * variable QDT_F32_BUDGET sets the budget, 0 turns it off; stats report the
 * quartets and the bound).  Held to 1e-10 Eh of the FP64 form.
 * `out` (host or device, caller-owned) receives qdt_packed_size() bytes;
 * `out_bytes` must be at least that.  Device scratch, and page-locked host
 * memory that stages the call's uploads, are allocated and kept by the
 * context between calls; the call starts by synchronising the context's
 * stream.  A class whose integral rows do not fit the device runs in row
 * batches that keep bra-ket symmetry (environment: QDT_W_BUDGET=bytes forces
 * batches of at most that size, QDT_BATCH_SYM=0 turns the symmetry across
 * batches off).  `stats` may be NULL.
 */
int qdt_transform(qdt_ctx *ctx, unsigned blocks, int k_begin, int k_end, double schwarz_tau,
                  int precision, double *out, size_t out_bytes, qdt_stats *stats);

/*
 * Expand one packed block (`block` = QDT_COULOMB, QDT_GAUNT or QDT_GAUGE) of n
 * Kramers pairs to the full complex array full[2n][2n][2n][2n] of
 * interleaved (re, im) doubles, on the context's GPU.  After
 * qdt_set_spinor_coefficients n counts spinors and full is [n][n][n][n].
 * Both pointers are device pointers.
 */
int qdt_unpack(qdt_ctx *ctx, const double *packed, int n_kramers, unsigned block, double *full);

/* ------------------------------------------------------------------ batches
 * Several transformations as one batch: after each request's screening (run
 * on its own context's stream), the kept shell-quartet tiles of all requests
 * are fused into one persistent launch of the integral kernel per kernel kind
 * (Coulomb kernel; gauge kernel) over a shared tile queue, most expensive
 * tiles first, and every request's first half, second half and packing then
 * run concurrently on its own stream.  The result of each item equals that of
 * qdt_transform with the same arguments to rounding (the fused launch sizes
 * its shared-memory plan for the largest request, which can regroup the
 * primitive sums).  A request whose integral rows do not fit in one row batch
 * runs alone after the fused ones.  The paper computes one system at a time;
 * batching is this library's addition.
 *
 * flags: 0, or QDT_BATCH_GRAPH: the launch sequence after screening is
 * captured into a CUDA graph the second time the same batch is seen (same
 * contexts, arguments, device buffers and screening outcome) and the graph is
 * replayed from the third time on; the first sighting runs the sequence
 * directly so that every buffer reaches its size before capture.  The graph
 * belongs to the first item's context (its stream carries the fused launches)
 * and is replaced when a different batch is seen.
 *
 * items: n >= 1 entries; every ctx distinct, non-NULL, on the same device, with
 * basis and coefficients set.  Each item's fields mean what qdt_transform's
 * arguments mean; `status` receives that item's own result and `stats`
 * (nullable) its statistics, whose ms_total is the whole batch's time and
 * whose per-phase times are 0 for fused items.  Returns QDT_OK when every
 * item succeeded, else the first failing item's code; qdt_last_error(item
 * ctx) describes that item's failure.  Synchronises every item's stream.
 */
#define QDT_BATCH_GRAPH 1u

typedef struct {
    qdt_ctx *ctx;
    unsigned blocks;
    int k_begin, k_end;
    double schwarz_tau;
    int precision;
    double *out;                    /* host or device, qdt_packed_size bytes */
    size_t out_bytes;
    qdt_stats *stats;               /* nullable                              */
    int status;                     /* written by the call                   */
} qdt_batch_item;

int qdt_transform_batch(qdt_batch_item *items, int n, unsigned flags);

/* Graphs captured and replayed by batches this context owned (diagnostics). */
int qdt_graph_counts(const qdt_ctx *ctx, long long *captures, long long *replays);

/* ------------------------------------------------------------------ serving
 * A server runs transformation requests of different basis and active-space
 * sizes on one GPU with continuous batching: `n_slots` contexts, each with its
 * own stream, execute admitted requests concurrently (their kernels overlap on
 * the device); a request waiting in the queue is admitted as soon as a slot is
 * free and its estimated device footprint (qdt_footprint) fits in what is left
 * of `pool_bytes`.  A slot keeps its basis tables resident and reuses them when
 * the next request carries the same basis.  All pointers of a request are
 * caller-owned and must stay valid until qdt_wait/qdt_poll reports it done.
 */
typedef struct qdt_server qdt_server;

typedef struct {
    int n_centers;                  /* basis, as for qdt_set_basis            */
    const double *xyz;
    int n_shells;
    const int *shell_center, *shell_l, *shell_nprim;
    const double *exps, *coefs;
    int nK;                         /* coefficients, as qdt_set_coefficients  */
    const double *CL, *CS;
    unsigned blocks;                /* as qdt_transform                       */
    int k_begin, k_end;
    double schwarz_tau;
    int precision;
    double *out;                    /* host or device, qdt_packed_size bytes  */
    size_t out_bytes;
} qdt_request;

/* Estimated peak device bytes of one request (integrals, densities, partial
   results, split-form digit planes); used for admission. */
size_t qdt_footprint(const qdt_request *req);

/* Create a server on `device` with `n_slots` (1..16) concurrent contexts and a
   device memory budget of `pool_bytes` (0: 80 % of the free memory). */
int qdt_server_create(qdt_server **srv, int device, int n_slots, size_t pool_bytes);

/* Finish queued and running requests, then release everything (NULL allowed). */
void qdt_server_destroy(qdt_server *srv);

/* Queue a request (copied; its arrays are not).  QDT_ERR_ADMISSION if its
   footprint exceeds the whole pool; QDT_ERR_ARG on bad sizes. */
int qdt_submit(qdt_server *srv, const qdt_request *req, uint64_t *handle);

/* *done = 1 once the request has finished (successfully or not). */
int qdt_poll(qdt_server *srv, uint64_t handle, int *done);

/* Wait up to timeout_s seconds (< 0: forever).  Returns the request's own
   status (QDT_OK or its error), or QDT_ERR_TIMEOUT.  latency_s (nullable)
   receives completion minus submission time; stats (nullable) the call's
   statistics.  A finished request's record is released by this call. */
int qdt_wait(qdt_server *srv, uint64_t handle, double timeout_s, double *latency_s, qdt_stats *stats);

/* ------------------------------------------------------------ no allocation
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory -- a host framework that owns all device memory
 * through its own pool allocator, or a latency-critical service that must not
 * take the implicit synchronisation of a fresh cudaMalloc.  It computes the
 * FP64 second-half contraction O = Dq^T V like qdt_transform does
 * internally, but keeps its split-K partial sums
 * in a fixed device array of the library (32 MiB of doubles, held on every GPU
 * that loads the library until the process exits) and calls no allocator.
 *
 *   Dq, V  device pointers, [K][N] row-major doubles (rows: AO pairs, in any
 *          order as long as both use the same; columns: Kramers-pair column x
 *          quaternion part); K >= 0.
 *   O      device pointer, [N][N] row-major; receives Dq^T V in every 64 x 64
 *          tile on or above the diagonal (tile row <= tile column); entries of
 *          the tiles below hold unspecified values.  Caller-owned.
 *   N      1 <= N and N * N <= 4 * 2^20 (N <= 2048); larger N returns
 *          QDT_ERR_ARG without launching anything.
 *   cuda_stream  cudaStream_t to order the work on (NULL: legacy stream); the
 *          call returns after queueing, without synchronising.
 *   msg    optional buffer (msg_len bytes) for an error description.
 *
 * The first call on a device looks up the array's device address on that
 * device (it must be the current device) and caches it for the process; make
 * that first call before any stream capture.  After cudaDeviceReset on that
 * device the cached address is stale: do not call this entry point again in
 * that process.  Every call shares the one array: calls whose work overlaps
 * on the GPU (different streams, or host threads) race and must be serialised
 * by the caller.  Returns QDT_OK, QDT_ERR_ARG or QDT_ERR_CUDA.
 */
int qdt_second_half_noalloc(const double *Dq, const double *V, long long K, long long N, double *O,
                            void *cuda_stream, char *msg, size_t msg_len);

/*
 * Measured FMA throughput of the CUDA cores of `device`, the peak that the AO
 * integral kernel's roofline divides by (that kernel runs on the CUDA cores:
 * FP64 FMAs in the FP64 form, FP32 FMAs in the split form).  The paper has no
 * counterpart; it is a diagnostic.  kind 0: FP32 FMA, kind 1: FP64 FMA;
 * *tflops receives 2 x FMAs per second / 1e12 of a kernel of eight
 * independent FMA chains per thread on every SM (best of three timed runs
 * after a warm-up).  Runs on a stream of its own and synchronises it.
 * Returns QDT_OK, QDT_ERR_ARG (bad kind or NULL) or QDT_ERR_CUDA.
 */
int qdt_alu_peak(int device, int kind, double *tflops);

/* Text of the last error of this context ("" if none); valid until the next call. */
const char *qdt_last_error(const qdt_ctx *ctx);

/* Library version string. */
const char *qdt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QDT_H */
