// Masked matvec over the (min, +) semiring (R u {+inf}, +, min, +inf) that
// Section 5.6 names for SSSP: the generalised-semiring form of Eq 2-5 with
// x = + and + = min, no early exit (it exists only for Boolean semirings) and no
// structure-only shortcut (the values are read).  Same two directions as the
// Boolean operator: pull computes each passing row's minimum over its entries
// (Algorithm 2 without the break), push expands the columns of u's finite
// entries and folds them into w with an atomic minimum (Eq 5 / Algorithm 3's
// reduction, done in place).  All sums are binary32.
#include <cmath>

#include "gbx_internal.cuh"

namespace gbx {

constexpr int kMpThreads = 256;

__device__ __forceinline__ bool mp_enabled(const int32_t* flag, int want) { return !flag || *flag == want; }

__device__ __forceinline__ bool mp_pass(const uint32_t* pass, int32_t i) {
    return !pass || ((pass[i >> 5] >> (i & 31)) & 1u);
}

// bm bit i = u[i] is finite (an entry of u)
__global__ void mp_finite_bitmap_kernel(const float* __restrict__ u, int32_t n, uint32_t* __restrict__ bm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n32 = ((int64_t)n + 31) & ~(int64_t)31;
    if (i - (threadIdx.x & 31) >= n32) return;
    const bool fin = i < n && u[i] < INFINITY;
    const uint32_t word = __ballot_sync(0xffffffffu, fin);
    if ((threadIdx.x & 31) == 0) bm[i >> 5] = word;
}

__global__ void mp_degrees_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ list,
                                  const int32_t* count_dev, int32_t n, int32_t* __restrict__ deg, const int32_t* flag) {
    if (!mp_enabled(flag, GBX_DIR_PUSH)) return;
    const int32_t count = min(*count_dev, n);
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int32_t u = list[k];
        deg[k] = ptr[u + 1] - ptr[u];
    }
}

// Push: w(i) <- min(w(i), a(j, i) + u(j)) for every entry of the columns of u's
// finite entries j, rows that pass the mask only.  w was set to +inf (or keeps
// w_old with accumulate) beforehand.  Each thread takes gathered positions
// grid-stride and finds its column by binary search of the degree prefix.
__global__ void __launch_bounds__(kMpThreads)
    mp_push_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const float* __restrict__ val,
                   const int32_t* __restrict__ list, const int32_t* count_dev, int32_t n,
                   const int32_t* __restrict__ pre, const float* __restrict__ u, const uint32_t* __restrict__ pass,
                   float* w, const int32_t* flag) {
    if (!mp_enabled(flag, GBX_DIR_PUSH)) return;
    const int32_t count = min(*count_dev, n);
    if (count <= 0) return;
    const int64_t E = pre[count];
    for (int64_t e = (int64_t)blockIdx.x * kMpThreads + threadIdx.x; e < E; e += (int64_t)gridDim.x * kMpThreads) {
        int32_t lo = 0, hi = count;  // largest k with pre[k] <= e (pre[0] = 0)
        while (hi - lo > 1) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (pre[mid] <= e)
                lo = mid;
            else
                hi = mid;
        }
        const int32_t j = list[lo];
        const int64_t idx = (int64_t)ptr[j] + (e - pre[lo]);
        const int32_t i = col[idx];
        if (!mp_pass(pass, i)) continue;
        const float x = u[j] + val[idx];
        if (x < w[i]) atomic_min_f32(w + i, x);
    }
}

__global__ void mp_prepare_kernel(float* __restrict__ w, int32_t n, int accum, const int32_t* flag) {
    if (!mp_enabled(flag, GBX_DIR_PUSH) || accum) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = INFINITY;
}

// Pull: a warp takes 32 consecutive rows, a lane each; rows with more than 32
// entries are then reduced by the whole warp, one after another.
__global__ void __launch_bounds__(kMpThreads)
    mp_pull_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const float* __restrict__ val,
                   int32_t n, const float* __restrict__ u, const uint32_t* __restrict__ pass, float* __restrict__ w,
                   int accum, const int32_t* flag) {
    if (!mp_enabled(flag, GBX_DIR_PULL)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * kMpThreads) >> 5;
    const int64_t ntiles = ((int64_t)n + 31) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * kMpThreads + threadIdx.x) >> 5; tile < ntiles; tile += nwarps) {
        const int64_t i64 = (tile << 5) + lane;
        const bool in_range = i64 < n;
        const int32_t i = (int32_t)i64;
        const bool ps = in_range && mp_pass(pass, i);
        int32_t beg = 0, end = 0;
        if (ps) {
            beg = ptr[i];
            end = ptr[i + 1];
        }
        float t = INFINITY;
        const bool longrow = end - beg > 32;
        if (!longrow)
            for (int32_t k = beg; k < end; ++k) t = fminf(t, val[k] + u[col[k]]);
        uint32_t pend = __ballot_sync(0xffffffffu, longrow);
        while (pend) {
            const int owner = __ffs(pend) - 1;
            pend &= pend - 1;
            const int32_t b = __shfl_sync(0xffffffffu, beg, owner);
            const int32_t e = __shfl_sync(0xffffffffu, end, owner);
            float m = INFINITY;
            for (int32_t k = b + lane; k < e; k += 32) m = fminf(m, val[k] + u[col[k]]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == owner) t = m;
        }
        if (in_range) {
            const float old = accum ? w[i] : INFINITY;
            w[i] = ps ? fminf(old, t) : old;
        }
    }
}

__global__ void mp_decide_kernel(const int32_t* count_dev, int32_t n, float alpha, int32_t* flag) {
    const double r = (double)(*count_dev) / (double)n;
    *flag = r <= (double)alpha ? GBX_DIR_PUSH : GBX_DIR_PULL;
}

gbx_status mxv_minplus(Graph* G, float* w, const uint32_t* pass_bm, bool nothing_passes, const float* u,
                       const gbx_desc& d, cudaStream_t s) {
    const int32_t n = G->n;
    GBX_CHECK(G->out_val != nullptr, GBX_ERR_INVALID_VALUE,
              "the (min, +) semiring needs edge weights (gbx_graph_set_weights)");
    const int32_t* pull_ptr = d.transpose ? G->in_ptr : G->out_ptr;
    const int32_t* pull_col = d.transpose ? G->in_col : G->out_col;
    const float* pull_val = d.transpose ? G->in_val : G->out_val;
    const int32_t* push_ptr = d.transpose ? G->out_ptr : G->in_ptr;
    const int32_t* push_col = d.transpose ? G->out_col : G->in_col;
    const float* push_val = d.transpose ? G->out_val : G->in_val;
    const unsigned int grid = (unsigned)G->num_sms * 8u;
    if (nothing_passes) {
        // every row fails the mask: w keeps w_old (accumulate) or becomes +inf
        if (!d.accum) mp_prepare_kernel<<<grid, kMpThreads, 0, s>>>(w, n, 0, nullptr);
        GBX_CUDA_TRY(cudaGetLastError());
        return GBX_OK;
    }
    const int dir = d.direction;
    const bool want_push = dir != GBX_DIR_PULL;
    const bool want_pull = dir != GBX_DIR_PUSH;
    uint32_t* ubm = G->ws.bm[0];
    int32_t* list = G->ws.list;
    int32_t* count = G->ws.flag + 0;
    int32_t* dflag = G->ws.flag + 1;
    const int32_t* flag = nullptr;
    if (want_push) {
        const int64_t n32 = ((int64_t)n + 31) & ~(int64_t)31;
        mp_finite_bitmap_kernel<<<div_up(n32, 256), 256, 0, s>>>(u, n, ubm);
        GBX_TRY(bitmap_to_list(ubm, n, list, count, G->ws.qd[0], G->ws.scan_tmp, s));
        if (dir == GBX_DIR_AUTO) {
            mp_decide_kernel<<<1, 1, 0, s>>>(count, n, d.alpha, dflag);
            flag = dflag;
        }
        int32_t* deg = G->ws.q[0];
        int32_t* pre = G->ws.qp[0];
        mp_degrees_kernel<<<grid, 256, 0, s>>>(push_ptr, list, count, n, deg, flag);
        GBX_TRY(exclusive_scan_i32(deg, pre, n, count, G->ws.scan_tmp, s));
        mp_prepare_kernel<<<grid, kMpThreads, 0, s>>>(w, n, d.accum ? 1 : 0, flag);
        mp_push_kernel<<<grid, kMpThreads, 0, s>>>(push_ptr, push_col, push_val, list, count, n, pre, u, pass_bm, w,
                                                   flag);
    }
    if (want_pull)
        mp_pull_kernel<<<grid, kMpThreads, 0, s>>>(pull_ptr, pull_col, pull_val, n, u, pass_bm, w, d.accum ? 1 : 0,
                                                   flag);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_OK;
}

}  // namespace gbx
