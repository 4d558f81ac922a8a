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
    void *buf[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t bytes[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int slices = 6;            // 7-bit digits per operand
    SplitKey bkey[2];          // cached first-half B operands (density slices)
    int bnext = 0;
};

void split_release(SplitWorkspace &w);
int split_slices(const SplitWorkspace &w);
// Device bytes currently held by the workspace.
size_t split_held_bytes(const SplitWorkspace &w);
// Drop cached operand slices (call whenever the densities change).
void split_invalidate(SplitWorkspace &w);

// C[M x N] = A[M x K_t] B[K_t x N], K_t from the per-64-row-tile extents.
void gemm_half1(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B,
                long long ldb, double *C, long long ldc, long long M, long long N,
                const long long *d_ktile, const std::vector<long long> &h_ktile, cudaStream_t s);

// C[N x N] += A^T B over K rows (upper block tiles valid).
void gemm_half2(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B,
                long long ldb, double *C, long long N, long long K, double *partial,
                size_t partial_elems, cudaStream_t s);

}  // namespace qdt
