// gemm_fp64.cu -- the plain-form (all FP64) contractions.
//   first half  (Eq. firsthalf):  V[ab, (rs,i)] = sum_cd (ab|cd) Dq[cd, (rs,i)]
//       -> C = A B with a ragged K per 64-row tile (the screened ket prefix);
//   second half (Eq. secondhalf with the quaternion->two-spinor conversion of
//   the paper's Sec. 2.4.2 folded into real parts):
//       O[(pq,i), (rs,j)] = sum_ab Dq[ab, (pq,i)] V[ab, (rs,j)]
//       -> C = A^T B, symmetric, upper block tiles only, deterministic split-K.
#include "qdt_internal.cuh"

namespace qdt {

constexpr int TM = 64, TN = 64, TK = 16;

int gemm_fp64_tile_m() { return TM; }

// 256 threads, 4x4 outputs each, register-blocked DFMA.
__global__ void __launch_bounds__(256) dgemm_nn_ragged(const double *__restrict__ A, long long lda,
                                                       const double *__restrict__ B, long long ldb,
                                                       double *__restrict__ C, long long ldc,
                                                       long long M, long long N,
                                                       const long long *__restrict__ ktile, int accumulate) {
    __shared__ double As[TK][TM + 1];
    __shared__ double Bs[TK][TN];
    const long long m0 = (long long)blockIdx.y * TM, n0 = (long long)blockIdx.x * TN;
    const long long K = ktile[blockIdx.y];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (long long k0 = 0; k0 < K; k0 += TK) {
        for (int i = threadIdx.x; i < TM * TK; i += 256) {
            int r = i / TK, c = i % TK;
            long long gr = m0 + r, gc = k0 + c;
            As[c][r] = (gr < M && gc < K) ? A[gr * lda + gc] : 0.0;
        }
        for (int i = threadIdx.x; i < TK * TN; i += 256) {
            int r = i / TN, c = i % TN;
            long long gr = k0 + r, gc = n0 + c;
            Bs[r][c] = (gr < K && gc < N) ? B[gr * ldb + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
            if (r < M && c < N) C[r * ldc + c] = accumulate ? C[r * ldc + c] + acc[i][j] : acc[i][j];
        }
}

void gemm_fp64_nn_ragged(const double *A, long long lda, const double *B, long long ldb, double *C,
                         long long ldc, long long M, long long N, const long long *ktile, int tileM,
                         cudaStream_t s, bool accumulate) {
    if (M <= 0 || N <= 0) return;
    if (tileM != TM) throw Error{QDT_ERR_ARG, "ragged GEMM tile mismatch"};
    dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM));
    dgemm_nn_ragged<<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, ktile, accumulate ? 1 : 0);
    QDT_CHECK_LAUNCH();
}

// C (N x N) = A^T B over K rows; upper block tiles (bi <= bj); split-K slices
// write partial[slice][N][N]; a second kernel sums slices in fixed order and
// mirrors nothing (only the upper tiles are consumed by the packer).
__global__ void __launch_bounds__(256) dgemm_tn_upper(const double *__restrict__ A, long long lda,
                                                      const double *__restrict__ B, long long ldb,
                                                      double *__restrict__ P, long long N, long long K,
                                                      long long kchunk, int ntb) {
    __shared__ double As[TK][TM];
    __shared__ double Bs[TK][TN];
    // decode the upper tile index
    int t = blockIdx.x, bi = 0;
    while (t >= ntb - bi) { t -= ntb - bi; ++bi; }
    int bj = bi + t;
    const long long m0 = (long long)bi * TM, n0 = (long long)bj * TN;
    const long long kb = (long long)blockIdx.y * kchunk, ke = min(K, kb + kchunk);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (long long k0 = kb; k0 < ke; k0 += TK) {
        for (int i = threadIdx.x; i < TK * TM; i += 256) {
            int r = i / TM, c = i % TM;
            long long gk = k0 + r;
            As[r][c] = (gk < ke && m0 + c < N) ? A[gk * lda + m0 + c] : 0.0;
            Bs[r][c] = (gk < ke && n0 + c < N) ? B[gk * ldb + n0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *Ps = P + (long long)blockIdx.y * N * N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long long r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
            if (r < N && c < N) Ps[r * N + c] = acc[i][j];
        }
}

__global__ void reduce_slices(const double *P, int nslice, long long NN, double *C, int accumulate) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NN;
         i += (long long)gridDim.x * blockDim.x) {
        double s = accumulate ? C[i] : 0.0;
        for (int k = 0; k < nslice; ++k) s += P[k * NN + i];
        C[i] = s;
    }
}

// C = A^T B (upper tiles valid).  `partial` must hold nslice * N * N doubles,
// nslice = partial_elems / (N*N) at most.
void gemm_fp64_tn_sym(const double *A, long long lda, const double *B, long long ldb, double *C,
                      long long N, long long K, double *partial, size_t partial_elems,
                      cudaStream_t s) {
    if (N <= 0) return;
    int ntb = (int)((N + TM - 1) / TM);
    int ntiles = ntb * (ntb + 1) / 2;
    long long maxslice = (long long)(partial_elems / (size_t)(N * N));
    long long want = (2 * 152 + ntiles - 1) / ntiles;
    if (want < 1) want = 1;
    if (want > 64) want = 64;
    if (want > maxslice) want = maxslice;
    if (want < 1) throw Error{QDT_ERR_OOM, "no room for the second-half partial sums"};
    long long kchunk = (K + want - 1) / want;
    kchunk = ((kchunk + TK - 1) / TK) * TK;
    if (kchunk < TK) kchunk = TK;
    int nslice = (int)((K + kchunk - 1) / kchunk);
    if (nslice < 1) nslice = 1;
    dim3 grid(ntiles, nslice);
    if (K > 0) {
        dgemm_tn_upper<<<grid, 256, 0, s>>>(A, lda, B, ldb, partial, N, K, kchunk, ntb);
        QDT_CHECK_LAUNCH();
    } else {
        launch_zero(partial, N * N, s);
        nslice = 1;
    }
    long long NN = N * N;
    long long blocks = (NN + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    reduce_slices<<<(unsigned)blocks, 256, 0, s>>>(partial, nslice, NN, C, 1);
    QDT_CHECK_LAUNCH();
}

}  // namespace qdt
