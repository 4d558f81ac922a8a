// gemm_split.cu -- dispatch of the half-transform contractions.
#include "split.cuh"

namespace qdt {

void split_release(SplitWorkspace &w) {
    for (int i = 0; i < 8; ++i) {
        if (w.buf[i]) cudaFree(w.buf[i]);
        w.buf[i] = nullptr;
        w.bytes[i] = 0;
    }
}

int split_slices(const SplitWorkspace &w) { return w.slices; }

void gemm_half1(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B,
                long long ldb, double *C, long long ldc, long long M, long long N,
                const long long *d_ktile, const std::vector<long long> &h_ktile, cudaStream_t s) {
    (void)w; (void)h_ktile;
    if (precision == QDT_SPLIT) throw Error{QDT_ERR_UNIMPLEMENTED, "split form not built yet"};
    gemm_fp64_nn_ragged(A, lda, B, ldb, C, ldc, M, N, d_ktile, gemm_fp64_tile_m(), s);
}

void gemm_half2(SplitWorkspace &w, int precision, const double *A, long long lda, const double *B,
                long long ldb, double *C, long long N, long long K, double *partial,
                size_t partial_elems, cudaStream_t s) {
    (void)w;
    if (precision == QDT_SPLIT) throw Error{QDT_ERR_UNIMPLEMENTED, "split form not built yet"};
    gemm_fp64_tn_sym(A, lda, B, ldb, C, N, K, partial, partial_elems, s);
}

}  // namespace qdt
