// Graph construction on the device: edge list -> CSR of A and CSR of A^T.
//
// Section 7.1: every dataset is made undirected and has self-loops and
// duplicate edges removed.  The build packs each directed entry (row, col)
// into one 64-bit key row << b | col (b = bits of n), radix-sorts the keys,
// drops repeats, and derives row offsets from the sorted rows.  Neighbour lists
// therefore come out ascending (Section 3 assumes sorted index lists).
#include <algorithm>
#include <new>

#include "gbx_internal.cuh"

namespace gbx {

static int bits_for(int64_t v) {  // smallest b with 2^b > v
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) <= v) ++b;
    return b;
}

__global__ void make_keys_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                 int32_t n, int b, int symmetrize, int drop_self, int reverse,
                                 unsigned long long* __restrict__ keys, int32_t* status) {
    const unsigned long long sentinel = ~0ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = src[e], v = dst[e];
        if (reverse) {
            const int32_t t = u;
            u = v;
            v = t;
        }
        unsigned long long k0 = sentinel, k1 = sentinel;
        if (u < 0 || u >= n || v < 0 || v >= n) {
            atomicCAS(status + ST_BADINDEX, -1, (int)(e < INT32_MAX ? e : INT32_MAX));
        } else if (!(drop_self && u == v)) {
            k0 = ((unsigned long long)u << b) | (unsigned long long)v;
            k1 = ((unsigned long long)v << b) | (unsigned long long)u;
        }
        keys[e] = k0;
        if (symmetrize) keys[m + e] = k1;
    }
}

// keep[k] = 1 if key k is valid and differs from key k-1.
__global__ void mark_unique_kernel(const unsigned long long* __restrict__ keys, int64_t K, int32_t* __restrict__ keep) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = keys[k];
        keep[k] = (x != ~0ull) && (k == 0 || keys[k - 1] != x) ? 1 : 0;
    }
}

__global__ void emit_csr_kernel(const unsigned long long* __restrict__ keys, int64_t K, const int32_t* __restrict__ keep,
                                const int32_t* __restrict__ pos, int b, int32_t* __restrict__ col,
                                int32_t* __restrict__ rows) {
    const unsigned long long mask = (1ull << b) - 1ull;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[k]) continue;
        const unsigned long long x = keys[k];
        col[pos[k]] = (int32_t)(x & mask);
        rows[pos[k]] = (int32_t)(x >> b);
    }
}

// row_ptr[r] = first position whose row is >= r (rows are sorted).
__global__ void row_ptr_kernel(const int32_t* __restrict__ rows, int64_t nnz, int32_t n, int32_t* __restrict__ row_ptr) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t hi = p < nnz ? rows[p] : n;
        const int32_t lo = p == 0 ? -1 : rows[p - 1];
        for (int32_t r = lo + 1; r <= hi; ++r) row_ptr[r] = (int32_t)p;
    }
}

__global__ void first_neighbour_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                       int32_t n, int32_t* __restrict__ first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        first[i] = row_ptr[i + 1] > row_ptr[i] ? col[row_ptr[i]] : -1;
}

// next[i] = entries 1..4 of row i (-1 past the row's end).
__global__ void next_neighbours_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                       int32_t n, int4* __restrict__ next) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = row_ptr[i], d = row_ptr[i + 1] - b;
        next[i] = make_int4(d > 1 ? col[b + 1] : -1, d > 2 ? col[b + 2] : -1, d > 3 ? col[b + 3] : -1,
                            d > 4 ? col[b + 4] : -1);
    }
}

// bm bit i set iff row i has at least min_len entries.
__global__ void nonzero_rows_kernel(const int32_t* __restrict__ row_ptr, int32_t n, int32_t min_len,
                                    uint32_t* __restrict__ bm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw32 = ((int64_t)n + 31) & ~(int64_t)31;
    if (i - (threadIdx.x & 31) >= nw32) return;
    const bool nz = i < n && row_ptr[i + 1] - row_ptr[i] >= min_len;
    const uint32_t word = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0) bm[i >> 5] = word;
}

static unsigned grid_for(int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 32)); }

// Sort the K keys and produce CSR (row_ptr, col) in freshly allocated device memory.
static gbx_status keys_to_csr(unsigned long long* keys, unsigned long long* alt, int64_t K, int32_t n, int b,
                              int32_t** row_ptr_out, int32_t** col_out, int64_t* nnz_out, cudaStream_t s) {
    unsigned long long* k1 = keys;
    unsigned long long* k2 = alt;
    GBX_TRY(radix_sort_u64(&k1, &k2, K, 2 * b, s));
    // k2 is free now; reuse it as keep flags + positions (2K + 1 int32 fit in K + 1 uint64)
    int32_t* keep = reinterpret_cast<int32_t*>(k2);
    int32_t* pos = keep + K;
    int32_t* tmp = nullptr;
    GBX_CUDA_TRY(cudaMallocAsync((void**)&tmp, sizeof(int32_t) * scan_tmp_ints(K), s));
    mark_unique_kernel<<<grid_for(K), 256, 0, s>>>(k1, K, keep);
    gbx_status st = exclusive_scan_i32(keep, pos, K, nullptr, tmp, s);
    int32_t nnz32 = 0;
    if (st == GBX_OK) {
        const cudaError_t e1 = cudaMemcpyAsync(&nnz32, pos + K, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        const cudaError_t e2 = cudaStreamSynchronize(s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cudaFreeAsync(tmp, s);
            GBX_CUDA_TRY(e1 != cudaSuccess ? e1 : e2);
        }
    }
    cudaFreeAsync(tmp, s);
    if (st != GBX_OK) return st;
    const int64_t nnz = (uint32_t)nnz32;  // K < 2^32 entries; counts below 2^31 checked below
    GBX_CHECK(nnz < ((int64_t)1 << 31), GBX_ERR_OVERFLOW, "graph has 2^31 or more stored edges");
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    int32_t* rows = nullptr;
    GBX_CUDA_TRY(cudaMalloc((void**)&row_ptr, sizeof(int32_t) * ((size_t)n + 1)));
    cudaError_t e = cudaMalloc((void**)&col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&rows, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1), s);
    if (e != cudaSuccess) {
        cudaFree(row_ptr);
        if (col) cudaFree(col);
        GBX_CUDA_TRY(e);
    }
    emit_csr_kernel<<<grid_for(K), 256, 0, s>>>(k1, K, keep, pos, b, col, rows);
    row_ptr_kernel<<<grid_for(nnz + 1), 256, 0, s>>>(rows, nnz, n, row_ptr);
    cudaFreeAsync(rows, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(row_ptr);
        cudaFree(col);
        GBX_CUDA_TRY(e);
    }
    *row_ptr_out = row_ptr;
    *col_out = col;
    *nnz_out = nnz;
    return GBX_OK;
}

void workspace_release(Workspace& w) {
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    for (auto& p : w.bm) f(p);
    for (int i = 0; i < 2; ++i) {
        f(w.q[i]);
        f(w.qp[i]);
        f(w.qd[i]);
    }
    f(w.list);
    f(w.scan_tmp);
    f(w.ctr);
    f(w.bar);
    f(w.trace);
    f(w.status);
    f(w.flag);
    f(w.msV);
    for (auto& p : w.msF) f(p);
    f(w.msP);
    f(w.msT);
    f(w.ms_src);
    if (w.ms_src_pinned) cudaFreeHost(w.ms_src_pinned);
    if (w.ms_src_ready) cudaEventDestroy(w.ms_src_ready);
    w = Workspace{};
}

static void graph_release(Graph* g) {
    if (!g) return;
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    if (g->in_ptr != g->out_ptr) f(g->in_ptr);
    if (g->in_col != g->out_col) f(g->in_col);
    f(g->out_ptr);
    f(g->out_col);
    f(g->nz_in);
    if (g->multi_out != g->multi_in) f(g->multi_out);
    f(g->multi_in);
    if (g->nz_out != g->nz_in) f(g->nz_out);
    if (g->first_out != g->first_in) f(g->first_out);
    f(g->first_in);
    if (g->next_out != g->next_in) f(g->next_out);
    f(g->next_in);
    if (g->in_val != g->out_val) f(g->in_val);
    f(g->out_val);
    f(g->nzr_in);
    workspace_release(g->ws);
    for (int i = 0; i < 2; ++i) {
        f(g->hdepth[i]);
        f(g->hparent[i]);
        if (g->ev_done[i]) cudaEventDestroy(g->ev_done[i]);
        if (g->ev_copied[i]) cudaEventDestroy(g->ev_copied[i]);
    }
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    mxv_cache_release(g);
    delete g;
}

static gbx_status workspace_alloc_all(Workspace& w, int32_t n) {
    const size_t nw = (size_t)(n + 31) / 32 + 1;
    const size_t nn = (size_t)n + 1;
    for (auto& p : w.bm) GBX_CUDA_TRY(cudaMalloc((void**)&p, sizeof(uint32_t) * nw));
    for (int i = 0; i < 2; ++i) {
        GBX_CUDA_TRY(cudaMalloc((void**)&w.q[i], sizeof(int32_t) * nn));
        GBX_CUDA_TRY(cudaMalloc((void**)&w.qp[i], sizeof(int32_t) * nn));
        GBX_CUDA_TRY(cudaMalloc((void**)&w.qd[i], sizeof(int32_t) * nn));
    }
    GBX_CUDA_TRY(cudaMalloc((void**)&w.list, sizeof(int32_t) * nn));
    GBX_CUDA_TRY(cudaMalloc((void**)&w.scan_tmp, sizeof(int32_t) * scan_tmp_ints((int64_t)nn)));
    GBX_CUDA_TRY(cudaMalloc((void**)&w.ctr, sizeof(LevelCtr) * 4));
    GBX_CUDA_TRY(cudaMalloc((void**)&w.bar, sizeof(GridBar)));
    GBX_CUDA_TRY(cudaMemset(w.bar, 0, sizeof(GridBar)));
    GBX_CUDA_TRY(cudaMalloc((void**)&w.trace, sizeof(LevelRec) * kTraceCap));
    GBX_CUDA_TRY(cudaMalloc((void**)&w.status, sizeof(int32_t) * ST_WORDS));
    GBX_CUDA_TRY(cudaMemset(w.status, 0, sizeof(int32_t) * ST_WORDS));
    GBX_CUDA_TRY(cudaMalloc((void**)&w.flag, sizeof(int32_t) * 64));
    GBX_CUDA_TRY(cudaMemset(w.flag, 0, sizeof(int32_t) * 64));
    w.n_cap = n;  // only once every buffer exists
    return GBX_OK;
}

// All or nothing: a failed allocation releases what was allocated, so no half-built
// workspace (one that claims capacity n but holds null buffers) is ever left behind.
gbx_status workspace_alloc(Workspace& w, int32_t n) {
    const gbx_status st = workspace_alloc_all(w, n);
    if (st != GBX_OK) workspace_release(w);
    return st;
}

static gbx_status build_impl(Graph* g, int32_t n, int64_t m, const int32_t* src, const int32_t* dst, uint32_t flags,
                             cudaStream_t s) {
    const int sym = (flags & GBX_SYMMETRIZE) ? 1 : 0;
    const int drop = (flags & GBX_DROP_SELF_LOOPS) ? 1 : 0;
    GBX_CUDA_TRY(cudaGetDevice(&g->device));
    GBX_CUDA_TRY(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    g->n = n;
    g->nwords = (n + 31) / 32;
    g->symmetric = sym;
    g->drop_self_loops = drop;
    GBX_TRY(workspace_alloc(g->ws, n));

    const int64_t K = sym ? 2 * m : m;
    GBX_CHECK(K < ((int64_t)1 << 32), GBX_ERR_OVERFLOW, "too many edge entries (2^32 or more)");
    const int b = bits_for(n);  // 2^b > n - 1 and the all-ones pattern is never a vertex pair

    // device copies of the edge list
    const int32_t* dsrc = src;
    const int32_t* ddst = dst;
    int32_t* own = nullptr;
    if (!(flags & GBX_DEVICE_EDGES) && m > 0) {
        GBX_CUDA_TRY(cudaMallocAsync((void**)&own, sizeof(int32_t) * 2 * (size_t)m, s));
        GBX_CUDA_TRY(cudaMemcpyAsync(own, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        GBX_CUDA_TRY(cudaMemcpyAsync(own + m, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        dsrc = own;
        ddst = own + m;
    }
    unsigned long long* keys = nullptr;
    unsigned long long* alt = nullptr;
    const size_t kbytes = sizeof(unsigned long long) * (size_t)(K + 1);  // + 1: keep flags and positions reuse it
    cudaError_t e = cudaMallocAsync((void**)&keys, kbytes, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&alt, kbytes, s);
    if (e != cudaSuccess) {
        if (own) cudaFreeAsync(own, s);
        if (keys) cudaFreeAsync(keys, s);
        GBX_CUDA_TRY(e);
    }
    gbx_status st = GBX_OK;
    int32_t bad = -1;
    auto cleanup = [&]() {
        cudaFreeAsync(keys, s);
        cudaFreeAsync(alt, s);
        if (own) cudaFreeAsync(own, s);
    };
    GBX_CUDA_TRY(cudaMemsetAsync(g->ws.status + ST_BADINDEX, 0xff, sizeof(int32_t), s));
    if (m > 0) make_keys_kernel<<<grid_for(m), 256, 0, s>>>(dsrc, ddst, m, n, b, sym, drop, 0, keys, g->ws.status);
    e = cudaMemcpyAsync(&bad, g->ws.status + ST_BADINDEX, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        GBX_CUDA_TRY(e);
    }
    if (bad >= 0) {
        cleanup();
        set_error("edge " + std::to_string(bad) + " has an endpoint outside [0, n)");
        return GBX_ERR_INVALID_INDEX;
    }
    st = keys_to_csr(keys, alt, K, n, b, &g->out_ptr, &g->out_col, &g->nnz, s);
    if (st == GBX_OK && !sym) {
        // A^T: the same entries with row and column exchanged
        if (m > 0) make_keys_kernel<<<grid_for(m), 256, 0, s>>>(dsrc, ddst, m, n, b, 0, drop, 1, keys, g->ws.status);
        int64_t nnz_t = 0;
        st = keys_to_csr(keys, alt, K, n, b, &g->in_ptr, &g->in_col, &nnz_t, s);
        if (st == GBX_OK && nnz_t != g->nnz) {
            set_error("internal: transpose has a different edge count");
            st = GBX_ERR_CUDA;
        }
    } else if (st == GBX_OK) {
        g->in_ptr = g->out_ptr;
        g->in_col = g->out_col;
    }
    cleanup();
    if (st != GBX_OK) return st;
    GBX_CUDA_TRY(cudaMalloc((void**)&g->nz_in, sizeof(uint32_t) * ((size_t)g->nwords + 1)));
    const int64_t nw32 = ((int64_t)n + 31) & ~(int64_t)31;
    nonzero_rows_kernel<<<div_up(nw32, 256), 256, 0, s>>>(g->in_ptr, n, 1, g->nz_in);
    GBX_CUDA_TRY(cudaMalloc((void**)&g->multi_in, sizeof(uint32_t) * ((size_t)g->nwords + 1)));
    nonzero_rows_kernel<<<div_up(nw32, 256), 256, 0, s>>>(g->in_ptr, n, 2, g->multi_in);
    if (sym) {
        g->nz_out = g->nz_in;
        g->multi_out = g->multi_in;
    } else {
        GBX_CUDA_TRY(cudaMalloc((void**)&g->multi_out, sizeof(uint32_t) * ((size_t)g->nwords + 1)));
        nonzero_rows_kernel<<<div_up(nw32, 256), 256, 0, s>>>(g->out_ptr, n, 2, g->multi_out);
        GBX_CUDA_TRY(cudaMalloc((void**)&g->nz_out, sizeof(uint32_t) * ((size_t)g->nwords + 1)));
        nonzero_rows_kernel<<<div_up(nw32, 256), 256, 0, s>>>(g->out_ptr, n, 1, g->nz_out);
    }
    GBX_CUDA_TRY(cudaMalloc((void**)&g->first_in, sizeof(int32_t) * ((size_t)n + 1)));
    first_neighbour_kernel<<<grid_for(n), 256, 0, s>>>(g->in_ptr, g->in_col, n, g->first_in);
    if (sym) {
        g->first_out = g->first_in;
    } else {
        GBX_CUDA_TRY(cudaMalloc((void**)&g->first_out, sizeof(int32_t) * ((size_t)n + 1)));
        first_neighbour_kernel<<<grid_for(n), 256, 0, s>>>(g->out_ptr, g->out_col, n, g->first_out);
    }
    GBX_CUDA_TRY(cudaMalloc((void**)&g->next_in, sizeof(int4) * ((size_t)n + 1)));
    next_neighbours_kernel<<<grid_for(n), 256, 0, s>>>(g->in_ptr, g->in_col, n, g->next_in);
    if (sym) {
        g->next_out = g->next_in;
    } else {
        GBX_CUDA_TRY(cudaMalloc((void**)&g->next_out, sizeof(int4) * ((size_t)n + 1)));
        next_neighbours_kernel<<<grid_for(n), 256, 0, s>>>(g->out_ptr, g->out_col, n, g->next_out);
    }
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaStreamSynchronize(s));
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_graph_build(gbx_graph** out, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                      uint32_t flags, void* stream) {
    clear_error();
    GBX_CHECK(out != nullptr, GBX_ERR_NULL_POINTER, "out is NULL");
    *out = nullptr;
    GBX_CHECK(n >= 1, GBX_ERR_INVALID_VALUE, "n must be >= 1");
    GBX_CHECK(m >= 0, GBX_ERR_INVALID_VALUE, "m must be >= 0");
    GBX_CHECK((flags & ~(GBX_SYMMETRIZE | GBX_DROP_SELF_LOOPS | GBX_DEVICE_EDGES)) == 0, GBX_ERR_INVALID_VALUE,
              "unknown flag bits");
    GBX_CHECK(m == 0 || (src != nullptr && dst != nullptr), GBX_ERR_NULL_POINTER, "src or dst is NULL");
    Graph* g = new (std::nothrow) Graph();
    GBX_CHECK(g != nullptr, GBX_ERR_OUT_OF_MEMORY, "host allocation failed");
    const gbx_status st = build_impl(g, n, m, src, dst, flags, (cudaStream_t)stream);
    if (st != GBX_OK) {
        graph_release(g);
        return st;
    }
    *out = reinterpret_cast<gbx_graph*>(g);
    return GBX_OK;
}

extern "C" gbx_status gbx_graph_free(gbx_graph* g) {
    clear_error();
    if (!g) return GBX_OK;
    Graph* G = as_impl(g);
    cudaDeviceSynchronize();
    graph_release(G);
    return GBX_OK;
}

extern "C" gbx_status gbx_graph_info(const gbx_graph* g, int32_t* n, int64_t* nnz, int32_t* symmetric) {
    clear_error();
    GBX_TRY(check_graph(g));
    const Graph* G = as_impl(g);
    if (n) *n = G->n;
    if (nnz) *nnz = G->nnz;
    if (symmetric) *symmetric = G->symmetric;
    return GBX_OK;
}

extern "C" gbx_status gbx_graph_csr(const gbx_graph* g, int32_t transpose, const int32_t** row_ptr,
                                    const int32_t** col) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(row_ptr != nullptr && col != nullptr, GBX_ERR_NULL_POINTER, "row_ptr or col is NULL");
    const Graph* G = as_impl(g);
    *row_ptr = transpose ? G->in_ptr : G->out_ptr;
    *col = transpose ? G->in_col : G->out_col;
    return GBX_OK;
}

extern "C" gbx_status gbx_graph_copy_csr(const gbx_graph* g, int32_t transpose, int32_t* row_ptr_dst,
                                         int32_t* col_dst) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(row_ptr_dst != nullptr && col_dst != nullptr, GBX_ERR_NULL_POINTER, "destination is NULL");
    const Graph* G = as_impl(g);
    GBX_CUDA_TRY(cudaDeviceSynchronize());
    GBX_CUDA_TRY(cudaMemcpy(row_ptr_dst, transpose ? G->in_ptr : G->out_ptr, sizeof(int32_t) * ((size_t)G->n + 1),
                            cudaMemcpyDefault));
    if (G->nnz > 0)
        GBX_CUDA_TRY(cudaMemcpy(col_dst, transpose ? G->in_col : G->out_col, sizeof(int32_t) * (size_t)G->nnz,
                                cudaMemcpyDefault));
    return GBX_OK;
}

extern "C" gbx_status gbx_graph_sync(gbx_graph* g, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    cudaStream_t s = (cudaStream_t)stream;
    GBX_CUDA_TRY(cudaStreamSynchronize(s));
    if (G->ws.last_stream && G->ws.last_stream != s) GBX_CUDA_TRY(cudaStreamSynchronize(G->ws.last_stream));
    int32_t err = 0;
    GBX_CUDA_TRY(cudaMemcpy(&err, G->ws.status + ST_ERROR, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (err != 0) {
        // a kernel gave up: clear the error and the barrier it may have left half-arrived
        GBX_CUDA_TRY(cudaMemset(G->ws.status + ST_ERROR, 0, sizeof(int32_t)));
        GBX_CUDA_TRY(cudaMemset(G->ws.bar, 0, sizeof(GridBar)));
        set_error(err == GBX_ERR_TIMEOUT ? "a bounded device-side wait ran out" : "device-side error");
        return (gbx_status)err;
    }
    return GBX_OK;
}
