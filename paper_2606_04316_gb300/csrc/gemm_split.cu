// gemm_split.cu -- the half-transform contractions (paper Eqs. firsthalf and
// secondhalf) in two forms:
//
//  QDT_FP64:  plain FP64 GEMMs (gemm_fp64.cu).
//  QDT_SPLIT: Ozaki-style split precision on the 5th-generation tensor cores.
//    Every FP64 operand row (A) or column (B) gets a power-of-two scale 2^e
//    with 2^e > max |x|; x 2^{42-e} is rounded to an integer X and written as
//    six balanced 7-bit digits, x = 2^e sum_{i=1..6} d_i 2^{-7 i} with d_1 in
//    [-128, 128] and d_2..d_6 in [-64, 64] (all exact in BF16; rounding halves
//    the representation error of truncated digits).  C = 2^{e_r + f_c}
//    sum_{i+j<=7} 2^{-7(i+j)} sum_k a_i b_j.  Per K index the digit products
//    of the diagonals i+j = 2, 3, 4 sum to at most 128^2, 2 * 128 * 64 and
//    2 * 128 * 64 + 64^2 (20 480), so over a K chunk of 768 their sums stay
//    within 2^24 and are exact in the FP32 TMEM accumulators; after each chunk
//    they are converted to integers and folded into a 64-bit integer
//    accumulator.  The lighter diagonals 5, 6, 7 (weights <= 2^{-35})
//    accumulate in FP32 over the whole K.  The result is recombined in FP64.
//
//  Tensor-core kernel: tcgen05.mma kind::f16 (BF16 x BF16 -> FP32), M = 128,
//  N = 80, operands K-major in shared memory with the 128-byte swizzle, staged
//  by TMA (cp.async.bulk.tensor): per K subtile of 64 the six B planes are
//  loaded once into one of two panels and the six A planes into one stage
//  each, all tracked by mbarriers; six FP32 accumulators (480 of the 512 TMEM
//  columns) per CTA.  N = 80 is the widest tile whose six accumulators fit the
//  TMEM; each MMA then reads 6.5 KB of operands per 46 cycles instead of 6 KB
//  per 37 (N = 64), which eases the shared-memory bandwidth the tensor pipe
//  waits on.  Roles: one thread issues the TMA loads, one the MMAs (its loops
//  unrolled over the digit pairs, so A stage, barrier phase, accumulator and
//  descriptors are compile-time constants), eight warps (two per TMEM lane
//  quadrant, 40 columns each) fold the exact diagonals and write the result.
//  Every wait is bounded and reports a timeout through a device status word
//  instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "split.cuh"

namespace qdt {

constexpr int kSlices = 6;
constexpr int kBits = 7;
constexpr int kFrac = kSlices * kBits;       // 42 fractional bits
constexpr int SBM = 128, SBN = 80, SBK = 64;
constexpr int kChunkSub = 12;                 // 12 x 64 = 768 K per exact chunk
constexpr size_t kPlaneBudget = (size_t)16 << 30;   // digit planes of one second-half K chunk
constexpr int kATile = SBM * SBK * 2;         // 16 KB: one A digit plane of a K subtile
constexpr int kBTile = SBN * SBK * 2;         // 10 KB: one B digit plane
constexpr int kBPanel = kSlices * kBTile;     // 60 KB: the six B planes of a K subtile
// shared memory: one stage per A plane (6 x 16 KB) and two B panels (2 x 48 KB)
constexpr int kSmemBytes = kSlices * kATile + 2 * kBPanel + 1024 + 256;
constexpr long long kWaitNs = 2000000000LL;   // 2 s bound on every wait

// ------------------------------------------------------------ workspace
enum { WS_A = 0, WS_B0 = 1, WS_B1 = 2, WS_EXP = 3, WS_KT = 4, WS_ERR = 5, WS_A2 = 6, WS_B2 = 7, WS_STAT = 8 };

static void *ws_get(SplitWorkspace &w, int slot, size_t bytes) {
    if (w.bytes[slot] >= bytes && w.buf[slot]) return w.buf[slot];
    if (w.buf[slot]) cudaFree(w.buf[slot]);
    w.buf[slot] = nullptr;
    w.bytes[slot] = 0;
    if (cudaMalloc(&w.buf[slot], bytes) != cudaSuccess) {
        cudaGetLastError();
        w.buf[slot] = nullptr;
        throw Error{QDT_ERR_OOM, "split workspace allocation failed"};
    }
    w.bytes[slot] = bytes;
    return w.buf[slot];
}

void split_release(SplitWorkspace &w) {
    for (int i = 0; i < SplitWorkspace::kSlots; ++i) {
        if (w.buf[i]) cudaFree(w.buf[i]);
        w.buf[i] = nullptr;
        w.bytes[i] = 0;
    }
    w.bkey[0] = w.bkey[1] = SplitKey();
    w.bnext = 0;
}

int split_slices(const SplitWorkspace &w) { return w.slices; }

size_t split_held_bytes(const SplitWorkspace &w) {
    size_t b = 0;
    for (int i = 0; i < SplitWorkspace::kSlots; ++i) b += w.bytes[i];
    return b;
}

void split_clear_status(SplitWorkspace &w, cudaStream_t s) {
    QDT_CUDA_TRY(cudaMemsetAsync(ws_get(w, WS_STAT, 256), 0, 256, s));
}

void split_begin_deferred(SplitWorkspace &w, cudaStream_t s) {
    split_clear_status(w, s);
    w.deferred = true;
}

void split_end_deferred(SplitWorkspace &w, cudaStream_t s) {
    w.deferred = false;
    int h = 0;
    QDT_CUDA_TRY(cudaMemcpyAsync(&h, ws_get(w, WS_STAT, 256), sizeof(int), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) throw Error{QDT_ERR_TIMEOUT, "split contraction: a bounded tensor-core wait gave up"};
}

void split_invalidate(SplitWorkspace &w) {
    w.bkey[0] = w.bkey[1] = SplitKey();
    w.bnext = 0;      // every class fills the slots in the same order, call after call
}

void split_forget(SplitWorkspace &w, const void *lo, const void *hi) {
    for (int q = 0; q < 2; ++q)
        if (w.bkey[q].ptr >= lo && w.bkey[q].ptr < hi) w.bkey[q] = SplitKey();
}

static inline long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

// ------------------------------------------------------------ digits
__device__ inline int exp_of_max(double m) {
    // smallest e with 2^e > m (m >= 0); 0 for m == 0
    if (!(m > 0.0)) return 0;
    long long bits = __double_as_longlong(m);
    int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return -1022;
    return ex - 1023 + 1;
}

// x 2^{42-e} rounded to the nearest integer X (|X| <= 2^42 when |x| < 2^e), by
// integer operations on the bits, then its balanced digits: d_1 = round(X /
// 2^35) in [-128, 128], X -= d_1 2^35, and so on down to d_6 = X in [-64, 63].
__device__ inline void digits7(double x, int e, __nv_bfloat16 *d, size_t plane) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    long long X = 0;
    if (ex != 0) {
        const unsigned long long mant = (bits & ((1ULL << 52) - 1)) | (1ULL << 52);
        const int sh = ex - 1075 + kFrac - e;         // |x| 2^{42-e} = mant 2^sh
        unsigned long long M;
        if (sh >= 0) M = 1ULL << kFrac;               // cannot happen when 2^e > |x|
        else if (sh > -63) M = (mant + (1ULL << (-sh - 1))) >> (-sh);
        else M = 0;
        if (M > (1ULL << kFrac)) M = 1ULL << kFrac;
        X = (bits >> 63) ? -(long long)M : (long long)M;
    }
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
        const int shift = kBits * (kSlices - 1 - i);
        // floor((X + 2^{shift-1}) / 2^shift): arithmetic shift of a signed value
        const long long di = shift ? (X + (1LL << (shift - 1))) >> shift : X;
        X -= di * (1LL << shift);
        d[i * plane] = __float2bfloat16_rn((float)di);
    }
}

// A operand: rows of X (row-major, ld) scaled per row; out[i][r][k] for
// r < Mpad, k < Kpad (zeros outside the matrix).  One CTA per row.  With the
// K extents of the 128-row tiles (kt128), a row is sliced only as far as the
// contraction reads it, its tile's extent rounded up to the 64-wide K
// subtile (the digits past it are never loaded).
__global__ void slice_rows_kernel(const double *X, long long ld, long long M, long long K,
                                  long long Mpad, long long Kpad, __nv_bfloat16 *out, int *rowexp,
                                  const long long *kt128) {
    long long r = blockIdx.x;
    __shared__ double wm[32];
    __shared__ int e_sh;
    const long long Kr = kt128 ? min(Kpad, (kt128[r / SBM] + SBK - 1) / SBK * SBK) : Kpad;
    const long long Kx = min(K, Kr);
    double m = 0.0;
    if (r < M)
        for (long long k = threadIdx.x; k < Kx; k += blockDim.x) m = fmax(m, fabs(X[r * ld + k]));
    // row maximum: warp shuffles, then the warps' maxima in the first warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) e_sh = exp_of_max(m);
    }
    __syncthreads();
    const int e = e_sh;
    if (threadIdx.x == 0) rowexp[r] = e;
    size_t plane = (size_t)Mpad * Kpad;
    for (long long k = threadIdx.x; k < Kr; k += blockDim.x) {
        double x = (r < M && k < Kx) ? X[r * ld + k] : 0.0;
        digits7(x, e, out + (size_t)r * Kpad + k, plane);
    }
}

// column maxima (as exponents) of X[rows][cols]
__global__ void col_max_kernel(const double *X, long long ld, long long rows, long long cols,
                               long long rows_per_block, unsigned long long *cmax) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= cols) return;
    long long r0 = blockIdx.y * rows_per_block, r1 = min(rows, r0 + rows_per_block);
    double m = 0.0;
    for (long long r = r0; r < r1; ++r) m = fmax(m, fabs(X[r * ld + c]));
    atomicMax(cmax + c, (unsigned long long)__double_as_longlong(m));
}

__global__ void col_exp_kernel(const unsigned long long *cmax, long long cols, long long cols_pad, int *colexp) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= cols_pad) return;
    colexp[c] = (c < cols) ? exp_of_max(__longlong_as_double((long long)cmax[c])) : 0;
}

// B operand (or a transposed A): columns of X scaled per column, written
// transposed: out[i][c][r] for c < Cpad, r < Rpad.  Tile 64 rows x 32 cols.
__global__ void slice_cols_t_kernel(const double *X, long long ld, long long rows, long long cols,
                                    long long Rpad, long long Cpad, const int *colexp,
                                    __nv_bfloat16 *out) {
    __shared__ double t[64][33];
    long long r0 = blockIdx.x * 64LL, c0 = blockIdx.y * 32LL;
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
        int rr = i / 32, cc = i % 32;
        long long r = r0 + rr, c = c0 + cc;
        t[rr][cc] = (r < rows && c < cols) ? X[r * ld + c] : 0.0;
    }
    __syncthreads();
    size_t plane = (size_t)Cpad * Rpad;
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
        int cc = i / 64, rr = i % 64;
        long long r = r0 + rr, c = c0 + cc;
        if (r < Rpad && c < Cpad) digits7(t[rr][cc], colexp[c], out + (size_t)c * Rpad + r, plane);
    }
}

// ------------------------------------------------------------ PTX helpers
__device__ inline uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void mbar_init(uint64_t *b, int cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(cnt) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

// bounded wait for phase `parity` of an mbarrier; false after limit_ns
__device__ inline bool mbar_wait_for(uint64_t *b, uint32_t parity, long long limit_ns) {
    uint32_t a = su32(b);
    unsigned long long t0 = gtimer();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((long long)(gtimer() - t0) > limit_ns) return false;
    }
}

__device__ inline bool mbar_wait(uint64_t *b, uint32_t parity) { return mbar_wait_for(b, parity, kWaitNs); }

// Self-check of the bounded wait: one thread waits on an mbarrier that
// nothing arrives at; the wait must give up after limit_ns and record it.
__global__ void wait_probe_kernel(long long limit_ns, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_for(&bar, 0, limit_ns)) atomicExch(status, 1);
}

__device__ inline void tma_load(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ inline uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// instruction descriptor: D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SBN >> 3) << 17) |
                            ((uint32_t)(SBM >> 4) << 24);

__device__ inline void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ inline void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ GEMM kernel
__device__ inline void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

// warps 0-7 fold and write (warp w: TMEM lanes 32 (w % 4) .. + 31, columns
// 40 (w / 4) .. + 39), warp 8 loads, warp 9 issues MMAs
constexpr int kFoldWarps = 8, kFoldCols = SBN / 2;
constexpr int kThreads = 32 * (kFoldWarps + 2);

// C[M x N] (FP64, ld ldc) = sum of digit products of A slices (tmA rows
// i*Mpad + m) and B slices (tmB rows j*Npad + n), K extent per 128-row tile.
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_umma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      long long Mpad, long long Npad, const long long *__restrict__ ktile,
                      const int *__restrict__ rowexp, const int *__restrict__ colexp, double *C, long long ldc,
                      long long Mvalid, long long Nvalid, int flags, int *status) {
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.y * SBM, n0 = (long long)blockIdx.x * SBN;
    const bool upper_only = (flags & 1) != 0, accumulate = (flags & 2) != 0;   // C += instead of C =
    if (upper_only && (m0 / 4) > (n0 + SBN - 1) / 4) return;   // below the block diagonal: unused
    if (*(volatile int *)status) return;                       // an earlier CTA gave up: skip the work
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bpanel = base + kSlices * kATile;                  // two B panels after the six A stages
    uint64_t *afull = (uint64_t *)(bpanel + 2 * kBPanel);
    uint64_t *aempty = afull + kSlices;
    uint64_t *bfull = aempty + kSlices;        // [2]
    uint64_t *bempty = bfull + 2;              // [2]
    uint64_t *chunk_bar = bempty + 2;          // a chunk's MMAs finished
    uint64_t *folded = chunk_bar + 1;          // the exact accumulators were read (4 warps)
    uint64_t *done = folded + 1;               // every MMA finished
    uint32_t *tslot = (uint32_t *)(done + 1);
    __shared__ int abort_flag;

    const long long K = ktile[blockIdx.y];
    const int nk = (int)((K + SBK - 1) / SBK);
    const int nchunks = (nk + kChunkSub - 1) / kChunkSub;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < kSlices; ++i) { mbar_init(afull + i, 1); mbar_init(aempty + i, 1); }
        for (int p = 0; p < 2; ++p) { mbar_init(bfull + p, 1); mbar_init(bempty + p, 1); }
        mbar_init(chunk_bar, 1);
        mbar_init(folded, kFoldWarps);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == kFoldWarps) {
        if (lane == 0) {                               // TMA producer
            bool ok = true;
            for (int kt = 0; kt < nk && ok; ++kt) {
                const int p = kt & 1;
                // B panel of subtile kt: the panel's previous user is subtile kt - 2
                if (kt >= 2 && !mbar_wait(bempty + p, (uint32_t)(((kt >> 1) - 1) & 1))) { ok = false; break; }
                mbar_expect_tx(bfull + p, kBPanel);
                for (int j = 0; j < kSlices; ++j)
                    tma_load(bpanel + p * kBPanel + j * kBTile, &tmB, kt * SBK, (int)(j * Npad + n0), bfull + p);
                // A planes: stage i's previous user is subtile kt - 1
                for (int i = 0; i < kSlices; ++i) {
                    if (kt >= 1 && !mbar_wait(aempty + i, (uint32_t)((kt - 1) & 1))) { ok = false; break; }
                    if (*(volatile int *)&abort_flag) { ok = false; break; }
                    mbar_expect_tx(afull + i, kATile);
                    tma_load(base + i * kATile, &tmA, kt * SBK, (int)(i * Mpad + m0), afull + i);
                }
            }
            if (!ok) abort_flag = 1;
        }
    } else if (warp == kFoldWarps + 1) {
        if (lane == 0) {                               // MMA issuer
            bool ok = true;
            const uint64_t da0 = sdesc(su32(base)), db0 = sdesc(su32(bpanel));
            for (int c = 0; c < nchunks && ok; ++c) {
                // the exact accumulators of chunk c - 1 must be folded before they are overwritten
                if (c > 0 && !mbar_wait(folded, (uint32_t)((c - 1) & 1))) { ok = false; break; }
                tc_fence_after();
                const int kt1 = min(nk, (c + 1) * kChunkSub);
                for (int kt = c * kChunkSub; kt < kt1 && ok; ++kt) {
                    const bool chunk_first = kt == c * kChunkSub, first_kt = kt == 0;
                    const int p = kt & 1;
                    if (!mbar_wait(bfull + p, (uint32_t)((kt >> 1) & 1))) { ok = false; break; }
                    const uint64_t db = db0 + (uint64_t)((p * kBPanel) >> 4);
#pragma unroll
                    for (int i = 0; i < kSlices; ++i) {
                        if (!mbar_wait(afull + i, (uint32_t)(kt & 1)) || *(volatile int *)&abort_flag) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t da = da0 + (uint64_t)((i * kATile) >> 4);
#pragma unroll
                        for (int j = 0; j < kSlices - i; ++j) {
                            const int a = i + j;
                            const bool fresh_i = i == 0 && (a <= 2 ? chunk_first : first_kt);
#pragma unroll
                            for (int k16 = 0; k16 < SBK / 16; ++k16)
                                umma(tmem + (uint32_t)(a * SBN), da + (uint64_t)(2 * k16),
                                     db + (uint64_t)(j * (kBTile >> 4) + 2 * k16), (fresh_i && k16 == 0) ? 0u : 1u);
                        }
                        umma_commit(aempty + i);
                    }
                    if (ok) umma_commit(bempty + p);
                }
                if (ok) umma_commit(chunk_bar);
            }
            umma_commit(done);                         // also on abort: lets issued MMAs be awaited
            if (!ok) abort_flag = 1;
        }
    } else {                                           // fold warps: 32 rows x 40 columns each
        long long acc[kFoldCols];
#pragma unroll
        for (int j = 0; j < kFoldCols; ++j) acc[j] = 0;
        const int quad = warp & 3, cbase = (warp >> 2) * kFoldCols;
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)cbase;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            if (!mbar_wait(chunk_bar, (uint32_t)(c & 1)) || *(volatile int *)&abort_flag) {
                ok = false;
                break;
            }
            tc_fence_after();
            // fold the exact diagonals (accumulators 0, 1, 2) into the integer accumulator;
            // |sums| <= 20 480 * 768 < 2^24: integers exact in FP32 and in 32-bit ints,
            // 32-bit conversions and 64-bit integer adds keep the FP64 pipe free
#pragma unroll
            for (int q = 0; q < kFoldCols / 8; ++q) {
                float v0[8], v1[8], v2[8];
                tmem_ld8(trow + 0 * SBN + q * 8, v0);
                tmem_ld8(trow + 1 * SBN + q * 8, v1);
                tmem_ld8(trow + 2 * SBN + q * 8, v2);
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    acc[q * 8 + t] += (long long)__float2int_rn(v0[t]) * 16384 +
                                      (long long)__float2int_rn(v1[t]) * 128 + (long long)__float2int_rn(v2[t]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(folded);
        }
        const long long m = m0 + quad * 32 + lane;
        if (ok && nk > 0 && !mbar_wait(done, 0)) ok = false;
        if (!ok) {
            abort_flag = 1;
        } else if (nk > 0) {
            tc_fence_after();
            const int er = (m < Mpad) ? rowexp[m] : 0;
#pragma unroll
            for (int q = 0; q < kFoldCols / 8; ++q) {
                float v3[8], v4[8], v5[8];
                tmem_ld8(trow + 3 * SBN + q * 8, v3);
                tmem_ld8(trow + 4 * SBN + q * 8, v4);
                tmem_ld8(trow + 5 * SBN + q * 8, v5);
                if (m < Mvalid) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const long long n = n0 + cbase + q * 8 + t;
                        if (n < Nvalid) {
                            // diagonals 5, 6, 7 (weights 2^-35, -42, -49) folded in FP32, whose
                            // rounding is ~2^-59 of the result; then acc (weight 2^-28) in FP64
                            const float w = fmaf(v5[t], 0x1p-14f, fmaf(v4[t], 0x1p-7f, v3[t]));
                            const double v = fma((double)w, 0x1p-7, (double)acc[q * 8 + t]);
                            const int k = er + colexp[n] - 28;
                            const double r = (k > -1022 && k < 1023)
                                                 ? v * __longlong_as_double((long long)(k + 1023) << 52)
                                                 : ldexp(v, k);
                            C[m * ldc + n] = accumulate ? C[m * ldc + n] + r : r;
                        }
                    }
                }
            }
        } else if (m < Mvalid && !accumulate) {
            for (int t = 0; t < kFoldCols; ++t)
                if (n0 + cbase + t < Nvalid) C[m * ldc + n0 + cbase + t] = 0.0;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && tid == 0) {
        atomicExch(status, 1);
        // let copies and MMAs in flight land before the CTA exits (bounded)
        mbar_wait(done, 0);
        for (int i = 0; i < kSlices; ++i) { mbar_wait(afull + i, 0); mbar_wait(afull + i, 1); }
        for (int q = 0; q < 2; ++q) { mbar_wait(bfull + q, 0); mbar_wait(bfull + q, 1); }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        QDT_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) throw Error{QDT_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"};
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2D BF16 map over [rows][cols] (row pitch cols*2 bytes), box {64, box_rows}, 128B swizzle
static CUtensorMap make_map(void *ptr, long long rows, long long cols, int box_rows) {
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)SBK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{QDT_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    return m;
}

// Column-scaled, transposed slices of X[rows][cols] into slot; returns (Cpad, Rpad).
static void slice_cols(SplitWorkspace &w, int slot, const double *X, long long ld, long long rows, long long cols,
                       long long Rpad, long long Cpad, int *colexp, cudaStream_t s) {
    unsigned long long *cmax = (unsigned long long *)ws_get(w, WS_ERR, std::max<size_t>(4096, (size_t)Cpad * 8 + 64));
    QDT_CUDA_TRY(cudaMemsetAsync(cmax, 0, (size_t)Cpad * 8, s));
    long long rpb = std::max<long long>(64, (rows + 1023) / 1024);
    dim3 g1((unsigned)((cols + 255) / 256), (unsigned)((rows + rpb - 1) / rpb));
    if (rows > 0 && cols > 0) col_max_kernel<<<g1, 256, 0, s>>>(X, ld, rows, cols, rpb, cmax);
    QDT_CHECK_KERNEL("col_max_kernel");
    col_exp_kernel<<<(unsigned)((Cpad + 255) / 256), 256, 0, s>>>(cmax, cols, Cpad, colexp);
    QDT_CHECK_KERNEL("col_exp_kernel");
    __nv_bfloat16 *out = (__nv_bfloat16 *)ws_get(w, slot, (size_t)kSlices * Cpad * Rpad * 2 + (size_t)Cpad * sizeof(int));
    dim3 g2((unsigned)(Rpad / 64), (unsigned)((Cpad + 31) / 32));
    slice_cols_t_kernel<<<g2, 256, 0, s>>>(X, ld, rows, cols, Rpad, Cpad, colexp, out);
    QDT_CHECK_KERNEL("slice_cols_t_kernel");
}

static void run_umma(SplitWorkspace &w, void *Asl, long long Mpad, long long KpadA, void *Bsl, long long Npad,
                     long long KpadB, const long long *d_kt128, const int *rowexp, const int *colexp, double *C,
                     long long ldc, long long M, long long N, int flags, cudaStream_t s) {
    CUtensorMap ta = make_map(Asl, kSlices * Mpad, KpadA, SBM);
    CUtensorMap tb = make_map(Bsl, kSlices * Npad, KpadB, SBN);
    int *status = (int *)ws_get(w, WS_STAT, 256);
    if (!w.deferred) QDT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    QDT_CUDA_TRY(cudaFuncSetAttribute(ozaki_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    dim3 grid((unsigned)(Npad / SBN), (unsigned)(Mpad / SBM));
    ozaki_umma_kernel<<<grid, kThreads, kSmemBytes, s>>>(ta, tb, Mpad, Npad, d_kt128, rowexp, colexp, C, ldc, M, N,
                                                    flags, status);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, ozaki_umma_kernel);
        int dev = 0, optin = 0, perblock = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&perblock, cudaDevAttrMaxSharedMemoryPerBlock, dev);
        cudaGetLastError();
        char msg[512];
        snprintf(msg, sizeof msg,
                 "launch of ozaki_umma_kernel: %s (grid %u x %u, dyn smem %d, static %zu, max dyn attr %d, "
                 "regs %d, max threads %d, optin %d, per block %d, param %zu)",
                 cudaGetErrorString(le), grid.x, grid.y, kSmemBytes, fa.sharedSizeBytes, fa.maxDynamicSharedSizeBytes,
                 fa.numRegs, fa.maxThreadsPerBlock, optin, perblock, sizeof(CUtensorMap));
        throw Error{QDT_ERR_CUDA, msg};
    }
    if (w.deferred) return;
    int h = 0;
    QDT_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) throw Error{QDT_ERR_TIMEOUT, "split contraction: a bounded tensor-core wait gave up"};
}

bool split_wait_probe(SplitWorkspace &w, double limit_s, cudaStream_t s) {
    int *status = (int *)ws_get(w, WS_STAT, 256);
    QDT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    wait_probe_kernel<<<1, 32, 0, s>>>((long long)(limit_s * 1e9), status);
    QDT_CHECK_KERNEL("wait_probe_kernel");
    int h = 0;
    QDT_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    QDT_CUDA_TRY(cudaStreamSynchronize(s));
    QDT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    return h != 0;
}

// Extents of the 128-row tensor-core tiles: the maximum over the 64-row tiles
// they cover, or one constant extent when kt64 is null.  Kept on the device so
// that the contraction needs no host-to-device copy.
__global__ void tile_extent_kernel(const long long *kt64, long long n64, int ratio, long long *kt, long long n,
                                   long long constant) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (!kt64) {
        kt[t] = constant;
        return;
    }
    long long m = 0;
    for (int r = 0; r < ratio; ++r) {
        const long long i = t * ratio + r;
        if (i < n64) m = max(m, kt64[i]);
    }
    kt[t] = m;
}

void gemm_half1(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B, long long ldb,
                double *C, long long ldc, long long M, long long N, const long long *d_ktile,
                const std::vector<long long> &h_ktile, cudaStream_t s, bool accumulate) {
    if (precision != QDT_SPLIT) {
        gemm_fp64_nn_ragged(A, lda, B, ldb, C, ldc, M, N, d_ktile, gemm_fp64_tile_m(), s, accumulate);
        return;
    }
    if (M <= 0 || N <= 0) return;
    const int TMr = gemm_fp64_tile_m();
    const long long Mpad = rup(M, SBM), Npad = rup(N, SBN);
    std::vector<long long> kt((size_t)(Mpad / SBM), 0);
    long long kmax = 0;
    for (size_t t = 0; t < h_ktile.size(); ++t) {
        long long r = (long long)t * TMr / SBM;
        if (r < (long long)kt.size()) kt[r] = std::max(kt[r], h_ktile[t]);
        kmax = std::max(kmax, h_ktile[t]);
    }
    const long long KpadA = std::max<long long>(SBK, rup(std::min(kmax, lda), SBK));
    // tile extents of the 128-row tiles, from the 64-row ones on the device
    static_assert(SBM % 64 == 0, "tensor-core row tile must cover whole 64-row tiles");
    long long *d_kt = (long long *)ws_get(w, WS_KT, std::max<size_t>(256, kt.size() * sizeof(long long)));
    tile_extent_kernel<<<(unsigned)((kt.size() + 127) / 128), 128, 0, s>>>(d_ktile, (long long)h_ktile.size(),
                                                                          SBM / TMr, d_kt, (long long)kt.size(), 0);
    QDT_CHECK_KERNEL("tile_extent_kernel");
    // A slices (row scaled)
    int *rowexp = (int *)ws_get(w, WS_EXP, (size_t)(Mpad + Npad + 64) * sizeof(int) * 2);
    __nv_bfloat16 *Asl = (__nv_bfloat16 *)ws_get(w, WS_A, (size_t)kSlices * Mpad * KpadA * 2);
    slice_rows_kernel<<<(unsigned)Mpad, 256, 0, s>>>(A, lda, M, std::min(kmax, lda), Mpad, KpadA, Asl, rowexp, d_kt);
    QDT_CHECK_KERNEL("slice_rows_kernel");
    // B slices (column scaled, transposed), cached per (pointer, shape) until
    // split_invalidate(): the densities are the same for every row batch.
    const long long Krows = kmax;
    long long KpadB = std::max<long long>(SBK, rup(Krows, SBK));
    SplitKey key{B, ldb, N, KpadB};
    int slot = -1;
    for (int q = 0; q < 2; ++q)
        if (w.bkey[q].ptr == B && w.bkey[q].ld == ldb && w.bkey[q].n == N && w.bkey[q].k >= KpadB) slot = q;
    // the first (highest-Q) row batch has the longest ket prefix; later
    // batches reuse its slices with the cached row pitch
    if (slot >= 0) KpadB = w.bkey[slot].k;
    const size_t bslice = (size_t)kSlices * Npad * KpadB * 2;
    if (slot < 0) {
        slot = w.bnext;
        w.bnext ^= 1;
        w.bkey[slot] = SplitKey();
        char *bb = (char *)ws_get(w, WS_B0 + slot, bslice + (size_t)Npad * sizeof(int));
        slice_cols(w, WS_B0 + slot, B, ldb, Krows, N, KpadB, Npad, (int *)(bb + bslice), s);
        w.bkey[slot] = key;
    }
    char *bb = (char *)w.buf[WS_B0 + slot];
    run_umma(w, Asl, Mpad, KpadA, bb, Npad, KpadB, d_kt, rowexp, (const int *)(bb + bslice), C, ldc, M, N,
             accumulate ? 2 : 0, s);
}

void gemm_half2(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B, long long ldb,
                double *C, long long N, long long K, double *partial, size_t partial_elems, cudaStream_t s) {
    if (precision != QDT_SPLIT) {
        gemm_fp64_tn_sym(A, lda, B, ldb, C, N, K, partial, partial_elems, s);
        return;
    }
    if (N <= 0) return;
    const long long Mpad = rup(N, SBM), Npad = rup(N, SBN);
    // K in chunks whose digit planes (12 bytes per element of A and B) stay within
    // kPlaneBudget; the chunks' products are summed in FP64 into C
    long long kc_max = std::max<long long>(SBK, (long long)(kPlaneBudget / (12 * (size_t)(Mpad + Npad))) / SBK * SBK);
    if (const char *e = std::getenv("QDT_SPLIT_KCHUNK")) {          // smaller chunks, to exercise this path
        const long long v = std::atoll(e);
        if (v <= 0 || v % SBK) throw Error{QDT_ERR_ARG, "QDT_SPLIT_KCHUNK must be a positive multiple of 64"};
        kc_max = v;
    }
    int *exps = (int *)ws_get(w, WS_EXP, (size_t)(Mpad + Npad + 64) * sizeof(int) * 2);
    int *aexp = exps, *bexp = exps + Mpad + 32;
    const long long nkt = Mpad / SBM;
    for (long long k0 = 0; k0 < std::max<long long>(K, 1); k0 += kc_max) {
        const long long kc = std::min(kc_max, K - k0), Kpad = std::max<long long>(SBK, rup(kc, SBK));
        slice_cols(w, WS_A2, A + k0 * lda, lda, kc, N, Kpad, Mpad, aexp, s);
        slice_cols(w, WS_B2, B + k0 * ldb, ldb, kc, N, Kpad, Npad, bexp, s);
        long long *d_kt = (long long *)ws_get(w, WS_KT, std::max<size_t>(256, (size_t)nkt * sizeof(long long)));
        tile_extent_kernel<<<(unsigned)((nkt + 127) / 128), 128, 0, s>>>(nullptr, 0, 1, d_kt, nkt, kc);
        QDT_CHECK_KERNEL("tile_extent_kernel");
        // upper block tiles; the first chunk writes C, later ones add to it
        run_umma(w, w.buf[WS_A2], Mpad, Kpad, w.buf[WS_B2], Npad, Kpad, d_kt, aexp, bexp, C, N, N, N,
                 1 | (k0 > 0 ? 2 : 0), s);
        if (K <= 0) break;
    }
}

}  // namespace qdt
