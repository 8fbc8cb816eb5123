// Column-based masked matvec laid out as Algorithm 3 and Section 6.2 describe it:
// the lengths of the columns that u selects are scanned, those columns' row
// indices are gathered into one list (the IntervalGather step), the list is
// sorted by a key-only LSD radix sort (the multiway merge), and a segmented
// reduction over runs of equal keys -- for the Boolean semiring, keeping one --
// followed by the mask test leaves w as a sorted, duplicate-free index list
// (Eq 5).  The bitmap push of mxv.cu computes the same w in one pass with an
// atomicOr claim per entry; this path is the paper's own design, kept as a
// selectable alternative (desc.push_sort) to compare against it.
#include "gbx_internal.cuh"

namespace gbx {

constexpr int kGatherThreads = 256;
constexpr int kGatherTile = kGatherThreads * 8;  // gathered entries per block
constexpr int kSelectThreads = 256;

// Largest k in [lo, hi) with pre[k] <= e, given pre[lo] <= e (pre ascending).
__device__ __forceinline__ int32_t last_le(const int32_t* __restrict__ pre, int32_t lo, int32_t hi, int32_t e) {
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (pre[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// keys[e] = col[ptr[u_k] + e - pre[k]] for e in [0, E), k the entry of u whose
// column holds gathered position e.  Each block first bounds the entries its
// tile spans (two searches), then each thread searches inside that range.
// Entries with an empty column (pre[k] == pre[k + 1]) are never selected: the
// largest k with pre[k] <= e always has e < pre[k + 1].
__global__ void __launch_bounds__(kGatherThreads)
    sort_gather_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                       const int32_t* __restrict__ ulist, int32_t count, const int32_t* __restrict__ pre, int32_t E,
                       uint32_t* __restrict__ keys) {
    __shared__ int32_t range[2];
    const int64_t e0 = (int64_t)blockIdx.x * kGatherTile;
    if (e0 >= E) return;
    const int64_t e1 = (int64_t)E - e0 < kGatherTile ? (int64_t)E : e0 + kGatherTile;
    if (threadIdx.x < 2) {
        const int32_t e = threadIdx.x == 0 ? (int32_t)e0 : (int32_t)(e1 - 1);
        range[threadIdx.x] = last_le(pre, 0, count, e);
    }
    __syncthreads();
    const int32_t klo = range[0], khi = range[1] + 1;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kGatherThreads) {
        const int32_t k = last_le(pre, klo, khi, (int32_t)e);
        const int32_t u = ulist[k];
        keys[e] = (uint32_t)__ldg(col + __ldg(ptr + u) + ((int32_t)e - pre[k]));
    }
}

// Segmented reduction + mask: flag[e] = 1 iff keys[e] opens a run of equal keys
// (the OR of a run of ones is one entry) and its row passes the mask.
__global__ void __launch_bounds__(kSelectThreads)
    sort_select_kernel(const uint32_t* __restrict__ keys, int32_t E, const uint32_t* __restrict__ pass,
                       int32_t* __restrict__ flag) {
    for (int64_t e = (int64_t)blockIdx.x * kSelectThreads + threadIdx.x; e < E; e += (int64_t)gridDim.x * kSelectThreads) {
        const uint32_t k = keys[e];
        const bool first = e == 0 || keys[e - 1] != k;
        const bool passes = !pass || ((pass[k >> 5] >> (k & 31)) & 1u);
        flag[e] = (first && passes) ? 1 : 0;
    }
}

// Compaction of the selected keys: into a sorted list, or into a result bitmap.
__global__ void __launch_bounds__(kSelectThreads)
    sort_emit_kernel(const uint32_t* __restrict__ keys, int32_t E, const int32_t* __restrict__ flag,
                     const int32_t* __restrict__ pos, int32_t* __restrict__ out_list, uint32_t* __restrict__ R) {
    for (int64_t e = (int64_t)blockIdx.x * kSelectThreads + threadIdx.x; e < E; e += (int64_t)gridDim.x * kSelectThreads) {
        if (!flag[e]) continue;
        const uint32_t k = keys[e];
        if (out_list)
            out_list[pos[e]] = (int32_t)k;
        else
            atomicOr(R + (k >> 5), 1u << (k & 31));
    }
}

__global__ void sort_degrees_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ list, int32_t count,
                                    int32_t cap, int32_t n, int32_t* __restrict__ deg) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int32_t u = k < cap ? list[k] : -1;
        deg[k] = (u >= 0 && u < n) ? ptr[u + 1] - ptr[u] : 0;
    }
}

static int key_bits(int32_t n) {  // bits that tell apart 0 .. n - 1
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
    return b;
}

// Scratch of one call, released on every exit path.
struct SortScratch {
    cudaStream_t s = nullptr;
    void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    ~SortScratch() {
        for (void* q : p)
            if (q) cudaFreeAsync(q, s);
    }
};

gbx_status mxv_push_sorted(Graph* G, const int32_t* push_ptr, const int32_t* push_col, const int32_t* ulist,
                           int32_t count, int32_t cap, const uint32_t* pass_bm, uint32_t* R, int32_t* out_list,
                           int32_t* out_count, int64_t* edges, cudaStream_t s) {
    const int32_t n = G->n;
    int32_t* deg = G->ws.q[0];
    int32_t* pre = G->ws.qp[0];
    *edges = 0;
    if (count > 0) {
        sort_degrees_kernel<<<div_up(count, 256), 256, 0, s>>>(push_ptr, ulist, count, cap, n, deg);
        GBX_TRY(exclusive_scan_i32(deg, pre, count, nullptr, G->ws.scan_tmp, s));
    }
    int32_t E = 0;
    if (count > 0) {
        GBX_CUDA_TRY(cudaMemcpyAsync(&E, pre + count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GBX_CUDA_TRY(cudaStreamSynchronize(s));
    }
    *edges = E;
    if (E == 0) {
        if (out_list) GBX_CUDA_TRY(cudaMemsetAsync(out_count, 0, sizeof(int32_t), s));
        return GBX_OK;
    }
    SortScratch sc;
    sc.s = s;
    const size_t eb = sizeof(uint32_t) * (size_t)E;
    GBX_CUDA_TRY(cudaMallocAsync(&sc.p[0], eb, s));
    GBX_CUDA_TRY(cudaMallocAsync(&sc.p[1], eb, s));
    GBX_CUDA_TRY(cudaMallocAsync(&sc.p[2], sizeof(int32_t) * ((size_t)E + 1), s));
    GBX_CUDA_TRY(cudaMallocAsync(&sc.p[3], sizeof(int32_t) * ((size_t)E + 1), s));
    GBX_CUDA_TRY(cudaMallocAsync(&sc.p[4], sizeof(int32_t) * scan_tmp_ints((int64_t)E), s));
    uint32_t* keys = static_cast<uint32_t*>(sc.p[0]);
    uint32_t* alt = static_cast<uint32_t*>(sc.p[1]);
    int32_t* flag = static_cast<int32_t*>(sc.p[2]);
    int32_t* pos = static_cast<int32_t*>(sc.p[3]);
    sort_gather_kernel<<<div_up(E, kGatherTile), kGatherThreads, 0, s>>>(push_ptr, push_col, ulist, count, pre, E,
                                                                          keys);
    GBX_TRY(radix_sort_u32(&keys, &alt, E, key_bits(n), s));
    const unsigned int grid = div_up(E, kSelectThreads) < 152u * 32 ? div_up(E, kSelectThreads) : 152u * 32;
    sort_select_kernel<<<grid, kSelectThreads, 0, s>>>(keys, E, pass_bm, flag);
    GBX_TRY(exclusive_scan_i32(flag, pos, E, nullptr, static_cast<int32_t*>(sc.p[4]), s));
    sort_emit_kernel<<<grid, kSelectThreads, 0, s>>>(keys, E, flag, pos, out_list, R);
    if (out_list) GBX_CUDA_TRY(cudaMemcpyAsync(out_count, pos + E, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

}  // namespace gbx
