// Allocation-free variant of the coreset sampler (csgs_sample_coreset_noalloc in
// include/csgs.h).  Some callers cannot allocate device memory at all: code that
// runs inside a host framework which owns every byte of the GPU through its own pool
// (so a cudaMalloc would fail or break its accounting), real-time or embedded
// runtimes that forbid allocation after start-up, and callers without a context
// object (creating a csgs_ctx allocates its work buffers).  For them the sampler's
// scratch - the integer CDF, the per-Gaussian draw counts and the scan partials -
// lives in one file-scope device array of fixed size, and the entry point takes
// only the caller's inputs, outputs and stream.
#include <mutex>

#include "csgs_internal.cuh"

namespace {

constexpr int64_t kMaxN = CSGS_NOALLOC_MAX_N;
constexpr int64_t kParts = (kMaxN + 2047) / 2048 + 64;  // scan partials per level

// Layout: C[kMaxN] u64 | C_tmp[kParts] u64 | counts[kMaxN] u32 | scan_tmp[kParts] u32 | n_out[2] u32
constexpr size_t kOffC = 0;
constexpr size_t kOffCtmp = kOffC + sizeof(unsigned long long) * kMaxN;
constexpr size_t kOffCounts = kOffCtmp + sizeof(unsigned long long) * kParts;
constexpr size_t kOffStmp = kOffCounts + sizeof(uint32_t) * kMaxN;
constexpr size_t kOffNout = kOffStmp + sizeof(uint32_t) * kParts;
constexpr size_t kScratchBytes = kOffNout + 2 * sizeof(uint32_t);

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_sample_scratch[kScratchBytes];

// Device address of the array, looked up once per device (the name is only a
// host-side stand-in for it in host code).
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" csgs_status csgs_sample_coreset_noalloc(const double* p_dev, int64_t n, int64_t m, uint64_t seed,
                                                   int32_t* idx_dev, float* w_dev, int64_t* n_distinct,
                                                   void* cuda_stream) {
    if (!p_dev || !idx_dev || !w_dev || !n_distinct) return CSGS_E_INVAL;
    if (n <= 0 || n > kMaxN) return CSGS_E_INVAL;
    if (m <= 0 || m >= (1ll << 31)) return CSGS_E_INVAL;
    // An error left pending by earlier work on this thread is not this call's: report
    // it without launching and leave it in place for its owner.
    if (cudaPeekAtLastError() != cudaSuccess) return CSGS_E_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CSGS_E_CUDA;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_sample_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return CSGS_E_CUDA;
            }
            g_addr[dev] = ptr;
        }
        base = g_addr[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    csgs::SampleTemp t;
    t.partial = nullptr;
    t.S = nullptr;
    t.C = reinterpret_cast<unsigned long long*>(b + kOffC);
    t.C_tmp = reinterpret_cast<unsigned long long*>(b + kOffCtmp);
    t.counts = reinterpret_cast<uint32_t*>(b + kOffCounts);
    t.scan_tmp = reinterpret_cast<uint32_t*>(b + kOffStmp);
    t.n_out = reinterpret_cast<uint32_t*>(b + kOffNout);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // sample_draws clears the counts it accumulates; every other scratch word is
    // written before it is read
    csgs::sample_draws(p_dev, n, m, seed, t, nullptr, idx_dev, w_dev, st);
    if (cudaGetLastError() != cudaSuccess) return CSGS_E_CUDA;
    uint32_t nd = 0;
    if (cudaMemcpyAsync(&nd, t.n_out, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CSGS_E_CUDA;
    }
    *n_distinct = (int64_t)nd;
    return CSGS_OK;
}
