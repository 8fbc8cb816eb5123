// Edge weights for the (min, +) semiring that Section 5.6 names for SSSP: the
// Boolean path needs only the structure of A (Section 5.5), the tropical one a
// value per stored entry.  Weights are attached after the build: every input
// pair finds its CSR entry (and its reverse, or its CSC entry) by binary search
// in the sorted row, and parallel pairs keep the smallest weight.
#include <cmath>

#include "gbx_internal.cuh"

namespace gbx {

__global__ void fill_f32_kernel(float* __restrict__ a, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// Index of c in the ascending col[beg, end), or -1.
__device__ __forceinline__ int64_t find_in_row(const int32_t* __restrict__ col, int64_t beg, int64_t end, int32_t c) {
    while (beg < end) {
        const int64_t mid = beg + ((end - beg) >> 1);
        const int32_t x = col[mid];
        if (x == c) return mid;
        if (x < c)
            beg = mid + 1;
        else
            end = mid;
    }
    return -1;
}

// bad: 1 = vertex out of range or a weight that is not finite, 2 = a pair the
// graph does not store (the graph was built from another edge list).
__global__ void set_weights_kernel(int64_t m, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                   const float* __restrict__ w, int32_t n, int sym, int drop,
                                   const int32_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col,
                                   float* out_val, const int32_t* __restrict__ in_ptr,
                                   const int32_t* __restrict__ in_col, float* in_val, int32_t* bad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = src[e], c = dst[e];
        const float x = w[e];
        if (r < 0 || r >= n || c < 0 || c >= n || !isfinite(x)) {
            atomicCAS(bad, 0, 1);
            continue;
        }
        if (drop && r == c) continue;
        const int64_t k = find_in_row(out_col, out_ptr[r], out_ptr[r + 1], c);
        if (k < 0) {
            atomicCAS(bad, 0, 2);
            continue;
        }
        atomic_min_f32(out_val + k, x);
        if (sym) {
            const int64_t k2 = find_in_row(out_col, out_ptr[c], out_ptr[c + 1], r);
            if (k2 < 0) {
                atomicCAS(bad, 0, 2);
                continue;
            }
            if (k2 != k) atomic_min_f32(out_val + k2, x);
        } else {
            const int64_t k3 = find_in_row(in_col, in_ptr[c], in_ptr[c + 1], r);
            if (k3 < 0) {
                atomicCAS(bad, 0, 2);
                continue;
            }
            atomic_min_f32(in_val + k3, x);
        }
    }
}

__global__ void nzr_ptr_kernel(const int32_t* __restrict__ rows, int32_t count, const int32_t* __restrict__ row_ptr,
                               int32_t n, int32_t* __restrict__ ptr) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= count; j += gridDim.x * blockDim.x)
        ptr[j] = row_ptr[j < count ? rows[j] : n];
}

// The compact list of rows with in-edges and their in-edge starts (Graph::nzr_in).
static gbx_status build_nzr_in(Graph* G, cudaStream_t s) {
    int32_t* count_dev = G->ws.flag + 9;
    GBX_TRY(bitmap_to_list(G->nz_in, G->n, G->ws.list, count_dev, G->ws.qd[0], G->ws.scan_tmp, s));
    int32_t count = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&count, count_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GBX_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t* buf = nullptr;
    GBX_CUDA_TRY(cudaMalloc((void**)&buf, sizeof(int32_t) * (2 * (size_t)count + 1)));
    cudaError_t e = cudaMemcpyAsync(buf, G->ws.list, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        const unsigned grid = div_up((int64_t)count + 1, 256) < 4096u ? div_up((int64_t)count + 1, 256) : 4096u;
        nzr_ptr_kernel<<<grid, 256, 0, s>>>(buf, count, G->in_ptr, G->n, buf + count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(buf);
        GBX_CUDA_TRY(e);
    }
    G->nzr_in = buf;
    G->nzr_in_ptr = buf + count;
    G->nnzr_in = count;
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_graph_set_weights(gbx_graph* g, int64_t m, const int32_t* src, const int32_t* dst,
                                            const float* w, uint32_t flags, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(m >= 0, GBX_ERR_INVALID_VALUE, "m must be >= 0");
    GBX_CHECK((flags & ~GBX_DEVICE_EDGES) == 0, GBX_ERR_INVALID_VALUE, "only GBX_DEVICE_EDGES is accepted");
    GBX_CHECK(m == 0 || (src != nullptr && dst != nullptr && w != nullptr), GBX_ERR_NULL_POINTER,
              "src, dst or w is NULL");
    Graph* G = as_impl(g);
    cudaStream_t s = (cudaStream_t)stream;
    const bool on_device = (flags & GBX_DEVICE_EDGES) != 0;
    if (!on_device)
        for (int64_t e = 0; e < m; ++e) GBX_CHECK(std::isfinite(w[e]), GBX_ERR_INVALID_VALUE, "weights must be finite");
    const int64_t nnz = G->nnz;
    if (!G->out_val) {  // both orientations or neither: a half-made pair would leave in_val null
        const size_t bytes = sizeof(float) * (size_t)(nnz > 0 ? nnz : 1);
        float* ov = nullptr;
        float* iv = nullptr;
        cudaError_t e = cudaMalloc((void**)&ov, bytes);
        if (e == cudaSuccess && !G->symmetric) e = cudaMalloc((void**)&iv, bytes);
        if (e != cudaSuccess) {
            if (ov) cudaFree(ov);
            GBX_CUDA_TRY(e);
        }
        G->out_val = ov;
        G->in_val = G->symmetric ? ov : iv;
    }
    if (!G->nzr_in) GBX_TRY(build_nzr_in(G, s));
    const float inf = INFINITY;
    if (nnz > 0) {
        fill_f32_kernel<<<div_up(nnz, 256) < 4096u ? div_up(nnz, 256) : 4096u, 256, 0, s>>>(G->out_val, nnz, inf);
        if (!G->symmetric)
            fill_f32_kernel<<<div_up(nnz, 256) < 4096u ? div_up(nnz, 256) : 4096u, 256, 0, s>>>(G->in_val, nnz, inf);
    }
    if (m == 0) {
        GBX_CUDA_TRY(cudaGetLastError());
        return GBX_OK;
    }
    // host inputs are staged on the device
    const int32_t* dsrc = src;
    const int32_t* ddst = dst;
    const float* dw = w;
    void* stage = nullptr;
    if (!on_device) {
        const size_t bytes = (sizeof(int32_t) * 2 + sizeof(float)) * (size_t)m;
        GBX_CUDA_TRY(cudaMallocAsync(&stage, bytes, s));
        int32_t* ps = static_cast<int32_t*>(stage);
        int32_t* pd = ps + m;
        float* pw = reinterpret_cast<float*>(pd + m);
        cudaError_t ce = cudaMemcpyAsync(ps, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(pd, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(pw, w, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, s);
        if (ce != cudaSuccess) {
            cudaFreeAsync(stage, s);
            GBX_CUDA_TRY(ce);
        }
        dsrc = ps;
        ddst = pd;
        dw = pw;
    }
    int32_t* bad = G->ws.flag + 8;
    GBX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
    const unsigned int grid = div_up(m, 256) < (unsigned)G->num_sms * 16u ? div_up(m, 256) : (unsigned)G->num_sms * 16u;
    set_weights_kernel<<<grid, 256, 0, s>>>(m, dsrc, ddst, dw, G->n, G->symmetric, G->drop_self_loops, G->out_ptr,
                                            G->out_col, G->out_val, G->in_ptr, G->in_col,
                                            G->symmetric ? nullptr : G->in_val, bad);
    const cudaError_t le = cudaGetLastError();
    if (stage) cudaFreeAsync(stage, s);
    GBX_CUDA_TRY(le);
    int32_t hbad = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GBX_CUDA_TRY(cudaStreamSynchronize(s));
    GBX_CHECK(hbad != 1, GBX_ERR_INVALID_INDEX, "a vertex outside [0, n) or a weight that is not finite");
    GBX_CHECK(hbad != 2, GBX_ERR_INVALID_VALUE, "a pair that the graph does not store (built from another edge list?)");
    return GBX_OK;
}

extern "C" gbx_status gbx_graph_copy_weights(const gbx_graph* g, int32_t transpose, float* dst) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(dst != nullptr, GBX_ERR_NULL_POINTER, "dst is NULL");
    const Graph* G = as_impl(g);
    GBX_CHECK(G->out_val != nullptr, GBX_ERR_INVALID_VALUE, "the graph has no weights");
    if (G->nnz > 0) {
        GBX_CUDA_TRY(cudaDeviceSynchronize());
        GBX_CUDA_TRY(cudaMemcpy(dst, transpose ? G->in_val : G->out_val, sizeof(float) * (size_t)G->nnz,
                                cudaMemcpyDefault));
    }
    return GBX_OK;
}
