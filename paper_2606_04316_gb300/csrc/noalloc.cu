// noalloc.cu -- the second-half contraction O = Dq^T V (FP64) for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns every byte
// of device memory through its own pool allocator (an extra cudaMalloc would
// exceed or fragment its budget), or a latency-critical service that must not
// take the implicit device synchronisation a fresh allocation can cause.  This
// entry point gives them the split-K contraction with its partial sums held in
// a fixed, file-scope device array instead of context scratch.
//
// The array is g_second_half_scratch below: kNoAllocScratchDoubles doubles
// (32 MiB), held on every GPU that loads the library until the process exits.
// Host code never dereferences or passes the array's name to a kernel (on the
// host it is only a stand-in symbol); its device address is obtained once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device, and cached for the life of the process; a
// cudaDeviceReset on that device invalidates the cached address.
#include <mutex>
#include <string>

#include "qdt_internal.cuh"

namespace {

constexpr long long kNoAllocScratchDoubles = 4LL << 20;   // 32 MiB

static __device__ __align__(256) double g_second_half_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

void put_msg(char *msg, size_t len, const std::string &s) {
    if (!msg || len == 0) return;
    size_t n = s.size() < len - 1 ? s.size() : len - 1;
    s.copy(msg, n);
    msg[n] = '\0';
}

}  // namespace

extern "C" int qdt_second_half_noalloc(const double *Dq, const double *V, long long K, long long N, double *O,
                                       void *cuda_stream, char *msg, size_t msg_len) {
    put_msg(msg, msg_len, "");
    if (!Dq || !V || !O || K < 0 || N <= 0) {
        put_msg(msg, msg_len, "qdt_second_half_noalloc: null pointer or non-positive size");
        return QDT_ERR_ARG;
    }
    // N > max / N, not N * N > max: the product overflows for N above ~3e9
    if (N > kNoAllocScratchDoubles / N) {
        put_msg(msg, msg_len, "qdt_second_half_noalloc: N = " + std::to_string(N) +
                                  " needs N*N doubles, more than the fixed scratch of " +
                                  std::to_string(kNoAllocScratchDoubles) + " doubles (N <= 2048)");
        return QDT_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        put_msg(msg, msg_len, "qdt_second_half_noalloc: no current CUDA device");
        return QDT_ERR_CUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_second_half_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                put_msg(msg, msg_len, std::string("qdt_second_half_noalloc: cudaGetSymbolAddress failed: ") +
                                          cudaGetErrorString(e));
                return QDT_ERR_CUDA;
            }
            g_scratch_ptr[dev] = (double *)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    try {
        // the reduction accumulates into O, so start from zero; the partial
        // sums of the previous call are overwritten slice by slice
        qdt::launch_zero(O, N * N, s);
        qdt::gemm_fp64_tn_sym(Dq, N, V, N, O, N, K, scratch, (size_t)kNoAllocScratchDoubles, s);
    } catch (const qdt::Error &e) {
        put_msg(msg, msg_len, e.msg);
        return e.code;
    }
    return QDT_OK;
}
