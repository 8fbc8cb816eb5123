// gbx_mxv_pull_noalloc: the masked row-based matvec without any allocation.
//
// Some callers cannot allocate device memory when they call into this library:
// a serving process whose device memory is all handed out up front by its own
// pool, a latency-bound loop that must not pay for the device-wide
// synchronisation cudaMalloc / cudaFree can cause, or an embedding that forbids
// allocation after start-up.  This entry point takes the matrix as CSR arrays
// the caller already owns and keeps its scratch (four n-bit bitmaps) in one
// fixed file-scope device array instead of a graph's scratch, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
#include <mutex>

#include "gbx_internal.cuh"

namespace gbx {

// Largest n the allocation-free path accepts, and its scratch: u, pass, nonempty
// rows and result bitmaps of kNoAllocWords words each (8 MiB + 512 B in total).
// Every GPU that loads this library holds the array until the process exits.
constexpr int32_t kNoAllocMaxN = 1 << 24;
constexpr int64_t kNoAllocWords = (int64_t)kNoAllocMaxN / 32 + 32;
static __device__ __align__(256) uint32_t g_noalloc_scratch[4 * kNoAllocWords];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static uint32_t* g_noalloc_addr[kNoAllocMaxDevices] = {};
static int g_noalloc_sms[kNoAllocMaxDevices] = {};

__global__ void noalloc_nonempty_rows_kernel(const int32_t* __restrict__ row_ptr, int32_t n, uint32_t* __restrict__ bm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw32 = ((int64_t)n + 31) & ~(int64_t)31;
    if (i - (threadIdx.x & 31) >= nw32) return;
    const bool nz = i < n && row_ptr[i + 1] > row_ptr[i];
    const uint32_t word = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0) bm[i >> 5] = word;
}

// Device address of the scratch array on the current device.  The first call on a
// device looks it up (cudaGetSymbolAddress, with that device current) and caches
// it; host code never hands the array's host-side name to a kernel.  The cached
// address belongs to the device's context of that moment: after cudaDeviceReset
// the module may be loaded elsewhere, so this entry point must not be called
// again in a process that reset a device it used.
static gbx_status noalloc_scratch(uint32_t** out, int* sms) {
    int dev = 0;
    GBX_CUDA_TRY(cudaGetDevice(&dev));
    GBX_CHECK(dev >= 0 && dev < kNoAllocMaxDevices, GBX_ERR_NOT_SUPPORTED,
              "gbx_mxv_pull_noalloc supports device indices below 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        // With lazy module loading (CUDA's default) this is where the library's module,
        // and with it the array, is put on the device: it can allocate and fail.
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error(std::string("gbx_mxv_pull_noalloc: could not place its fixed scratch array on device ") +
                      std::to_string(dev) + " (" + cudaGetErrorString(e) + ")");
            return e == cudaErrorMemoryAllocation ? GBX_ERR_OUT_OF_MEMORY : GBX_ERR_CUDA;
        }
        int nsm = 0;
        GBX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        g_noalloc_addr[dev] = static_cast<uint32_t*>(p);
        g_noalloc_sms[dev] = nsm;
    }
    *out = g_noalloc_addr[dev];
    *sms = g_noalloc_sms[dev];
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_mxv_pull_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col, const uint8_t* u,
                                           const uint8_t* mask, int32_t mask_complement, int32_t early_exit,
                                           uint8_t* w, void* stream) {
    clear_error();
    GBX_CHECK(n >= 1, GBX_ERR_INVALID_VALUE, "n must be >= 1");
    GBX_CHECK(n <= kNoAllocMaxN, GBX_ERR_INVALID_VALUE,
              "gbx_mxv_pull_noalloc: n exceeds its fixed scratch (at most 16777216 rows)");
    GBX_CHECK(row_ptr && col && u && w, GBX_ERR_NULL_POINTER, "row_ptr, col, u or w is NULL");
    GBX_CHECK(static_cast<const void*>(w) != static_cast<const void*>(u) &&
                  static_cast<const void*>(w) != static_cast<const void*>(mask),
              GBX_ERR_INVALID_VALUE, "w must not alias u or mask");
    uint32_t* scratch = nullptr;
    int sms = 0;
    GBX_TRY(noalloc_scratch(&scratch, &sms));
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* ubm = scratch;
    uint32_t* pass = scratch + kNoAllocWords;
    uint32_t* nzrows = scratch + 2 * kNoAllocWords;
    uint32_t* R = scratch + 3 * kNoAllocWords;
    const int32_t nwords = (n + 31) / 32;
    // every bitmap below is fully rewritten by this call; nothing from an earlier call is read
    if (!mask && mask_complement) {
        GBX_TRY(fill_bitmap(R, n, 0u, s));  // the complement of "no mask" passes nothing
    } else {
        GBX_TRY(pack_dense_to_bitmap(u, n, 0u, ubm, s));
        if (mask) GBX_TRY(pack_dense_to_bitmap(mask, n, mask_complement ? 1u : 0u, pass, s));
        const int64_t nw32 = ((int64_t)n + 31) & ~(int64_t)31;
        noalloc_nonempty_rows_kernel<<<div_up(nw32, 256), 256, 0, s>>>(row_ptr, n, nzrows);
        mxv_pull_kernel<<<sms * 8, kMxvThreads, 0, s>>>(row_ptr, col, nullptr, nullptr, nzrows, nullptr, ubm, mask ? pass : nullptr, R, nwords,
                                                early_exit ? 1 : 0, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    GBX_TRY(bitmap_to_dense(R, n, nullptr, w, s));
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}
