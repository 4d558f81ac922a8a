// split.cuh -- contraction dispatch: plain FP64 form or the split-precision
// (Ozaki) form of the first and second half-transforms.
#pragma once

#include <vector>

#include "qdt_internal.cuh"

namespace qdt {

struct SplitKey {
    const void *ptr = nullptr;
    long long ld = 0, n = 0, k = 0;
    bool operator==(const SplitKey &o) const { return ptr == o.ptr && ld == o.ld && n == o.n && k == o.k; }
};

struct SplitWorkspace {
    static constexpr int kSlots = 9;
    void *buf[kSlots] = {};
    size_t bytes[kSlots] = {};
    int slices = 6;            // 7-bit digits per operand
    SplitKey bkey[2];          // cached first-half B operands (density slices)
    int bnext = 0;
    bool deferred = false;     // status of the tensor-core waits read once at the end
};

void split_release(SplitWorkspace &w);
int split_slices(const SplitWorkspace &w);
// Device bytes currently held by the workspace.
size_t split_held_bytes(const SplitWorkspace &w);
// Drop cached operand slices (call whenever the densities change).
void split_invalidate(SplitWorkspace &w);
// Deferred status: begin clears the status word (a stream operation, so it
// can be part of a captured graph) and stops the per-launch status reads;
// end reads the word once (synchronising `s`) and throws QDT_ERR_TIMEOUT if a
// bounded wait gave up in any contraction since begin.
// split_clear_status alone clears the word without changing the mode.
void split_begin_deferred(SplitWorkspace &w, cudaStream_t s);
void split_clear_status(SplitWorkspace &w, cudaStream_t s);
void split_end_deferred(SplitWorkspace &w, cudaStream_t s);
// Runs one bounded wait on an mbarrier that nothing arrives at, with the
// given limit; true when the wait gave up and reported it (the expected case).
bool split_wait_probe(SplitWorkspace &w, double limit_s, cudaStream_t s);

// Drop the cached slices of the first-half B operands inside [lo, hi)
// (a buffer whose contents change).
void split_forget(SplitWorkspace &w, const void *lo, const void *hi);

// C[M x N] = A[M x K_t] B[K_t x N] (+= with accumulate), K_t from the
// per-64-row-tile extents.
void gemm_half1(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B,
                long long ldb, double *C, long long ldc, long long M, long long N,
                const long long *d_ktile, const std::vector<long long> &h_ktile, cudaStream_t s,
                bool accumulate = false);

// C[N x N] += A^T B over K rows (upper block tiles valid).
void gemm_half2(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B,
                long long ldb, double *C, long long N, long long K, double *partial,
                size_t partial_elems, cudaStream_t s);

}  // namespace qdt
