// Device primitives used by the graph build and the matvec operators:
// a three-phase exclusive scan, a stable LSD radix sort of 64- or 32-bit keys, and
// bitmap <-> dense / sorted-list conversions (the DENSE2SPARSE / SPARSE2DENSE
// vector conversions of Section 6.3, on bit-packed vectors).
#include "gbx_internal.cuh"

namespace gbx {

// ---------------------------------------------------------------- block scan

// Exclusive sum over the block; *total receives the block total.  All threads call it.
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t x, uint32_t* total) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t block_tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    const uint32_t inc = warp_inclusive_sum(x);
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t v = lane < nw ? warp_tot[lane] : 0u;
        const uint32_t vi = warp_inclusive_sum(v);
        warp_tot[lane] = vi - v;
        if (lane == 31) block_tot = vi;
    }
    __syncthreads();
    const uint32_t r = warp_tot[wid] + inc - x;
    *total = block_tot;
    __syncthreads();
    return r;
}

__device__ __forceinline__ int64_t resolve_count(const int32_t* count_dev, int64_t count_max) {
    if (!count_dev) return count_max;
    const int64_t c = *count_dev;
    return c < 0 ? 0 : (c > count_max ? count_max : c);
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const int32_t* __restrict__ in, int64_t count_max,
                                                                  const int32_t* count_dev, int32_t* __restrict__ sums) {
    const int64_t count = resolve_count(count_dev, count_max);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= count && blockIdx.x > 0) return;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanBlock + threadIdx.x;
        if (i < count) acc += (uint32_t)in[i];
    }
    uint32_t tot;
    block_exclusive_sum(acc, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = (int32_t)tot;
}

// One block: exclusive scan of the block sums in place; writes out[count] = total.
__global__ void __launch_bounds__(kScanBlock) scan_sums_kernel(int32_t* sums, int64_t nblocks_max, int64_t count_max,
                                                                const int32_t* count_dev, int32_t* out) {
    const int64_t count = resolve_count(count_dev, count_max);
    const int64_t nb = count == 0 ? 1 : (count + kScanTile - 1) / kScanTile;
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? (uint32_t)sums[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_sum(v, &tot);
        if (i < nb) sums[i] = (int32_t)(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) out[count] = (int32_t)carry;
    (void)nblocks_max;
}

__global__ void __launch_bounds__(kScanBlock) scan_apply_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                                 int64_t count_max, const int32_t* count_dev,
                                                                 const int32_t* __restrict__ sums) {
    const int64_t count = resolve_count(count_dev, count_max);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= count) return;
    // each thread owns kScanItems consecutive items
    const int64_t t0 = base + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (t0 + k < count) ? (uint32_t)in[t0 + k] : 0u;
        acc += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_sum(acc, &tot) + (uint32_t)sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (t0 + k < count) out[t0 + k] = (int32_t)ex;
        ex += v[k];
    }
}

size_t scan_tmp_ints(int64_t count_max) { return (size_t)((count_max + kScanTile - 1) / kScanTile) + 2; }

gbx_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t count_max, const int32_t* count_dev,
                              int32_t* tmp, cudaStream_t s) {
    const int64_t nb = count_max <= 0 ? 1 : (count_max + kScanTile - 1) / kScanTile;
    scan_reduce_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, count_max, count_dev, tmp);
    scan_sums_kernel<<<1, kScanBlock, 0, s>>>(tmp, nb, count_max, count_dev, out);
    scan_apply_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, count_max, count_dev, tmp);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

// ---------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // keys per block

template <typename K>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                                                                   int32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = (int32_t)cnt[threadIdx.x];
}

// Stable scatter: keys are ranked by (round, warp, lane), i.e. by input order.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const K* __restrict__ in, K* __restrict__ out,
                                                                      int64_t n, int shift,
                                                                      const int32_t* __restrict__ offs_all, int nblocks) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t offs[256];
    __shared__ uint32_t wcnt[kWarps][256];
    const int wid = threadIdx.x >> 5;
    offs[threadIdx.x] = (uint32_t)offs_all[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        K key = 0;
        uint32_t d = 0, rank = 0;
        const uint32_t act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            key = in[i];
            d = (uint32_t)(key >> shift) & 255u;
            const uint32_t peers = __match_any_sync(act, d);
            rank = __popc(peers & lanemask_lt());
            if ((peers & lanemask_lt()) == 0) wcnt[wid][d] = __popc(peers);
        }
        __syncthreads();
        if (valid) {
            uint32_t before = 0;
            for (int w = 0; w < wid; ++w) before += wcnt[w][d];
            out[offs[d] + before + rank] = key;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) tot += wcnt[w][threadIdx.x];
        offs[threadIdx.x] += tot;
        __syncthreads();
    }
}

template <typename K>
static gbx_status radix_sort(K** keys, K** alt, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return GBX_OK;
    const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t hn = (int64_t)nblocks * 256;
    int32_t* hist = nullptr;
    int32_t* tmp = nullptr;
    GBX_CUDA_TRY(cudaMallocAsync((void**)&hist, sizeof(int32_t) * (size_t)(hn + 1), s));
    const cudaError_t e2 = cudaMallocAsync((void**)&tmp, sizeof(int32_t) * scan_tmp_ints(hn), s);
    if (e2 != cudaSuccess) {
        cudaFreeAsync(hist, s);
        GBX_CUDA_TRY(e2);
    }
    gbx_status st = GBX_OK;
    for (int shift = 0; shift < bits && st == GBX_OK; shift += 8) {
        radix_hist_kernel<K><<<nblocks, kSortThreads, 0, s>>>(*keys, n, shift, hist, nblocks);
        st = exclusive_scan_i32(hist, hist, hn, nullptr, tmp, s);
        if (st != GBX_OK) break;
        radix_scatter_kernel<K><<<nblocks, kSortThreads, 0, s>>>(*keys, *alt, n, shift, hist, nblocks);
        K* t = *keys;
        *keys = *alt;
        *alt = t;
    }
    const cudaError_t le = cudaGetLastError();
    cudaFreeAsync(tmp, s);
    cudaFreeAsync(hist, s);
    if (st != GBX_OK) return st;
    GBX_CUDA_TRY(le);
    return GBX_OK;
}

gbx_status radix_sort_u64(unsigned long long** keys, unsigned long long** alt, int64_t n, int bits, cudaStream_t s) {
    return radix_sort<unsigned long long>(keys, alt, n, bits, s);
}

gbx_status radix_sort_u32(uint32_t** keys, uint32_t** alt, int64_t n, int bits, cudaStream_t s) {
    return radix_sort<uint32_t>(keys, alt, n, bits, s);
}

// ---------------------------------------------------------------- bitmaps

__device__ __forceinline__ uint32_t tail_mask(int32_t n, int32_t w) {
    const int32_t rem = n - (w << 5);
    return rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
}

// One thread per bitmap word: reads the word's 32 bytes (two 16-byte loads when
// the vector is 16-byte aligned), writes the word.
__global__ void pack_dense_kernel(const uint8_t* __restrict__ dense, int32_t n, uint32_t invert, uint32_t* __restrict__ bm) {
    const int32_t nw = (n + 31) >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(dense) & 15u) == 0;
    for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const int64_t base = (int64_t)w << 5;
        uint32_t word = 0;
        if (vec && base + 32 <= n) {
            const uint4 a = reinterpret_cast<const uint4*>(dense + base)[0];
            const uint4 b = reinterpret_cast<const uint4*>(dense + base)[1];
            const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int t = 0; t < 4; ++t) word |= (((v[q] >> (8 * t)) & 0xffu) != 0u ? 1u : 0u) << (4 * q + t);
        } else {
            for (int t = 0; t < 32 && base + t < n; ++t) word |= (dense[base + t] != 0 ? 1u : 0u) << t;
        }
        if (invert) {
            const int64_t rem = n - base;
            word = ~word & (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
        }
        bm[w] = word;
    }
}

gbx_status pack_dense_to_bitmap(const uint8_t* dense, int32_t n, uint32_t invert, uint32_t* bm, cudaStream_t s) {
    const int32_t nw = (n + 31) >> 5;
    pack_dense_kernel<<<max(1u, min(div_up(nw, 256), 152u * 16)), 256, 0, s>>>(dense, n, invert ? 1u : 0u, bm);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

__global__ void scatter_list_kernel(const int32_t* __restrict__ list, const int32_t* count_dev, int32_t cap,
                                    int32_t n_bound, uint32_t* __restrict__ bm) {
    const int32_t count = min(*count_dev, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[i];
        if (v >= 0 && v < n_bound) atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
}

gbx_status scatter_list_to_bitmap(const int32_t* list, const int32_t* count_dev, int32_t cap, int32_t n, uint32_t* bm,
                                  cudaStream_t s) {
    const unsigned blocks = cap <= 0 ? 1 : min(div_up(cap, 256), 65535u * 4);
    scatter_list_kernel<<<blocks, 256, 0, s>>>(list, count_dev, cap, n, bm);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

__global__ void fill_bitmap_kernel(uint32_t* bm, int32_t n, uint32_t value) {
    const int32_t nw = (n + 31) >> 5;
    for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x)
        bm[w] = value & tail_mask(n, w);
}

gbx_status fill_bitmap(uint32_t* bm, int32_t n, uint32_t value, cudaStream_t s) {
    const int32_t nw = (n + 31) >> 5;
    fill_bitmap_kernel<<<max(1u, min(div_up(nw, 256), 4096u)), 256, 0, s>>>(bm, n, value);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

__global__ void invert_bitmap_kernel(uint32_t* bm, int32_t n) {
    const int32_t nw = (n + 31) >> 5;
    for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x)
        bm[w] = ~bm[w] & tail_mask(n, w);
}

gbx_status invert_bitmap(uint32_t* bm, int32_t n, cudaStream_t s) {
    const int32_t nw = (n + 31) >> 5;
    invert_bitmap_kernel<<<max(1u, min(div_up(nw, 256), 4096u)), 256, 0, s>>>(bm, n);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

__global__ void popc_words_kernel(const uint32_t* __restrict__ bm, int32_t nw, int32_t* __restrict__ cnt) {
    const int32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) cnt[w] = __popc(bm[w]);
}

__global__ void emit_list_kernel(const uint32_t* __restrict__ bm, int32_t nw, const int32_t* __restrict__ pos,
                                 int32_t* __restrict__ list, int32_t* count_dev) {
    const int32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) {
        uint32_t word = bm[w];
        int32_t p = pos[w];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            list[p++] = (w << 5) + b;
        }
    }
    if (w == 0) *count_dev = pos[nw];
}

gbx_status bitmap_to_list(const uint32_t* bm, int32_t n, int32_t* list, int32_t* count_dev, int32_t* scan_out,
                          int32_t* tmp, cudaStream_t s) {
    const int32_t nw = (n + 31) >> 5;
    popc_words_kernel<<<div_up(nw, 256), 256, 0, s>>>(bm, nw, scan_out);
    GBX_TRY(exclusive_scan_i32(scan_out, scan_out, nw, nullptr, tmp, s));
    emit_list_kernel<<<div_up(nw, 256), 256, 0, s>>>(bm, nw, scan_out, list, count_dev);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

// One thread per bitmap word: writes the word's 32 bytes (two 16-byte stores when
// aligned), OR-ing in the old dense value when accumulating.
__global__ void bitmap_to_dense_kernel(const uint32_t* __restrict__ bm, int32_t n, const uint8_t* old_dense,
                                       uint8_t* out) {
    const int32_t nw = (n + 31) >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 &&
                     (old_dense == nullptr || (reinterpret_cast<uintptr_t>(old_dense) & 15u) == 0);
    for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const uint32_t word = bm[w];
        const int64_t base = (int64_t)w << 5;
        if (vec && base + 32 <= n) {
            uint32_t v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t x = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) x |= ((word >> (4 * q + t)) & 1u) << (8 * t);
                v[q] = x;
            }
            if (old_dense) {
                const uint4 a = reinterpret_cast<const uint4*>(old_dense + base)[0];
                const uint4 b = reinterpret_cast<const uint4*>(old_dense + base)[1];
                const uint32_t o[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[q] |= (((o[q] >> (8 * t)) & 0xffu) != 0u ? 1u : 0u) << (8 * t);
            }
            reinterpret_cast<uint4*>(out + base)[0] = make_uint4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<uint4*>(out + base)[1] = make_uint4(v[4], v[5], v[6], v[7]);
        } else {
            for (int t = 0; t < 32 && base + t < n; ++t) {
                uint8_t x = (uint8_t)((word >> t) & 1u);
                if (old_dense) x |= old_dense[base + t] != 0 ? 1 : 0;
                out[base + t] = x;
            }
        }
    }
}

gbx_status bitmap_to_dense(const uint32_t* bm, int32_t n, const uint8_t* old_dense, uint8_t* out, cudaStream_t s) {
    const int32_t nw = (n + 31) >> 5;
    bitmap_to_dense_kernel<<<max(1u, min(div_up(nw, 256), 152u * 16)), 256, 0, s>>>(bm, n, old_dense, out);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

}  // namespace gbx
