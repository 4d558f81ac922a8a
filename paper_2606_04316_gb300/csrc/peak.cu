// peak.cu -- measured FMA throughput of the CUDA cores (FP32 and FP64), the
// peak that the integral kernel's roofline divides by.  The integral engine
// runs on the CUDA cores (FP64 FMAs in the FP64 form, FP32 FMAs and
// compensated FP32 pairs in the split form), so its bound is the FMA issue
// rate of this part; this entry point measures that rate instead of deriving
// it from unit counts and clocks.
#include "qdt_internal.cuh"

namespace {

__device__ float g_sink_f;
__device__ double g_sink_d;

// Eight independent FMA chains per thread (enough to cover the FMA latency at
// full occupancy); the result is stored only when it equals an impossible
// value, so the chains stay live without a store per thread.
template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T a, T b, int iters) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)-12345.678) {
        if constexpr (sizeof(T) == 4) g_sink_f = (float)s;
        else g_sink_d = (double)s;
    }
}

template <class T>
double probe(int iters, cudaStream_t s) {
    int dev = 0, nsm = 0;
    QDT_CUDA_TRY(cudaGetDevice(&dev));
    QDT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = nsm * 8;        // 2048 threads per SM
    cudaEvent_t e0, e1;
    QDT_CUDA_TRY(cudaEventCreate(&e0));
    QDT_CUDA_TRY(cudaEventCreate(&e1));
    float best = 0.f;
    const T a = (T)0.999999, b = (T)1e-7;
    for (int rep = 0; rep < 4; ++rep) {                  // the first run is a warm-up
        QDT_CUDA_TRY(cudaEventRecord(e0, s));
        fma_probe_kernel<T><<<blocks, threads, 0, s>>>(a, b, iters);
        QDT_CUDA_TRY(cudaEventRecord(e1, s));
        QDT_CUDA_TRY(cudaEventSynchronize(e1));
        QDT_CHECK_KERNEL("fma_probe_kernel");
        float ms = 0.f;
        QDT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * (double)iters * threads * blocks;
    return flops / (best * 1e-3) / 1e12;
}

}  // namespace

extern "C" int qdt_alu_peak(int device, int kind, double *tflops) {
    if (!tflops || (kind != 0 && kind != 1)) return QDT_ERR_ARG;
    *tflops = 0.0;
    try {
        int cur = 0;
        QDT_CUDA_TRY(cudaGetDevice(&cur));
        QDT_CUDA_TRY(cudaSetDevice(device));
        cudaStream_t s = nullptr;
        QDT_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        try {
            *tflops = kind == 0 ? probe<float>(1 << 16, s) : probe<double>(1 << 11, s);
        } catch (...) {
            cudaStreamDestroy(s);
            cudaSetDevice(cur);
            throw;
        }
        cudaStreamDestroy(s);
        QDT_CUDA_TRY(cudaSetDevice(cur));
    } catch (const qdt::Error &e) {
        return e.code;
    }
    return QDT_OK;
}
