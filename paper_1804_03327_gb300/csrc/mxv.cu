// GrB_mxv over the Boolean semiring: the four matvec variants of Table 1.
//
//   row-based (pull, Eq 2 / Eq 4, Algorithm 2): one warp per 32 output rows;
//     only rows whose mask test passes are computed; each row ORs u over its
//     entries, stopping at the first hit when early exit is on (Section 5.3).
//   column-based (push, Eq 3 / Eq 5): the columns selected by u's nonzeros
//     are expanded with their edges split evenly over warps (exclusive prefix
//     of the selected columns' lengths); every hit that passes the mask sets
//     its bit in a result bitmap with atomicOr, which merges the columns
//     exactly (the multiway merge of Section 3.1, done by a bitmap instead of
//     the radix sort of Algorithm 3).
// The result bitmap is then written out as a dense byte vector or as a sorted
// index list (Section 3: sparse vectors are sorted lists).
#include <cstring>
#include <new>
#include <vector>

#include "gbx_internal.cuh"

namespace gbx {

constexpr int kMxvProbe = 16;
constexpr int kMxvLaneRow = 32;
constexpr int kMxvHugeRow = 4096;  // rows longer than this are spread over every warp
constexpr int kMxvChunk = 1024;

__device__ __forceinline__ bool dir_enabled(const int32_t* flag, int want) { return !flag || *flag == want; }

// Row-based matvec over the rows the mask lets through (Eq 2 / Eq 4).  A warp
// takes a tile of 32 result words (1024 rows), lists the passing nonempty rows in
// shared memory (each lane its word's rows, at its prefix of the words' counts)
// and computes them 64 per round, two rows per lane probing in lockstep: the
// first entry of a row comes from the dense first-entry array when one is given
// (one coalesced read instead of a random sector), entries 1..4 from the dense
// next-entries array (one 16-byte read), then up to kMxvProbe entries four at a
// time; longer rows are finished by the whole warp 32 entries at a time.  With
// early exit a row stops at its first hit (Section 5.3); the result is the same
// either way.
constexpr int kMxvIlp = 2;
constexpr int kMxvP1 = 4;  // first-pass rows per lane per round

// The rows of a tile whose bits are set in the lane words m (lane l: word l), in
// row order, as offsets in the tile, written at the lane's prefix excl.
__device__ __forceinline__ void mxv_tile_list(uint16_t* list, uint32_t m, uint32_t excl) {
    __syncwarp();
    const uint32_t rowbase = (threadIdx.x & 31) << 5;
    while (m) {
        const uint32_t b = __ffs(m) - 1;
        m &= m - 1;
        list[excl++] = (uint16_t)(rowbase + b);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kMxvThreads) mxv_pull_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                                const int32_t* __restrict__ first,
                                                                const int4* __restrict__ next,
                                                                const uint32_t* __restrict__ nzrows,
                                                                const uint32_t* __restrict__ multi,
                                                                const uint32_t* __restrict__ ubm,
                                                                const uint32_t* __restrict__ pass, uint32_t* __restrict__ R,
                                                                int32_t nwords, int early_exit, const int32_t* flag,
                                                                MxvStats* stats, int32_t* huge, int32_t* huge_next,
                                                                int32_t* huge_count) {
    if (!dir_enabled(flag, GBX_DIR_PULL)) return;
    __shared__ uint32_t tile_hits[kMxvThreads / 32][32];
    __shared__ uint16_t tile_rows[kMxvThreads / 32][1024];
    uint32_t* hits = tile_hits[threadIdx.x >> 5];
    uint16_t* list = tile_rows[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int32_t ntiles = (nwords + 31) >> 5;
    unsigned long long rows = 0, exam = 0;
    for (int32_t tile = gwarp; tile < ntiles; tile += nwarps) {
        const int32_t w = (tile << 5) + lane;
        const bool wok = w < nwords;
        const uint32_t cand0 = wok ? ((pass ? pass[w] : 0xffffffffu) & nzrows[w]) : 0u;
        hits[lane] = 0u;
        __syncwarp();
        // a tile with more candidates than one round first tests every candidate's first entry
        // (the dense first-entry array: no row offsets loaded); the rest goes on with the rows it
        // left open that have more entries
        const uint32_t cnt0 = __popc(cand0);
        const uint32_t incl0 = warp_inclusive_sum(cnt0);
        const uint32_t total0 = __shfl_sync(0xffffffffu, incl0, 31);
        const bool two_pass = first != nullptr && total0 > 32u * kMxvIlp;
        if (two_pass) {
            mxv_tile_list(list, cand0, incl0 - cnt0);
            for (uint32_t base = 0; base < total0; base += 32 * kMxvP1) {
                int32_t i[kMxvP1], f0[kMxvP1];
#pragma unroll
                for (int r = 0; r < kMxvP1; ++r) {
                    const uint32_t c = base + 32 * r + lane;
                    i[r] = c < total0 ? (tile << 10) + (int)list[c] : -1;
                }
#pragma unroll
                for (int r = 0; r < kMxvP1; ++r) f0[r] = i[r] >= 0 ? first[i[r]] : -1;
#pragma unroll
                for (int r = 0; r < kMxvP1; ++r) {
                    if (i[r] < 0) continue;
                    rows += 1;
                    exam += 1;
                    if (bit_test(ubm, f0[r])) atomicOr(hits + ((i[r] >> 5) - (tile << 5)), 1u << (i[r] & 31));
                }
            }
            __syncwarp();
        }
        const uint32_t f1 = hits[lane];  // rows the first pass found
        const uint32_t cand =
            two_pass ? cand0 & (multi ? (wok ? multi[w] : 0u) : 0xffffffffu) & (early_exit ? ~f1 : 0xffffffffu) : cand0;
        const uint32_t cntw = __popc(cand);
        const uint32_t incl = warp_inclusive_sum(cntw);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) mxv_tile_list(list, cand, incl - cntw);
        for (uint32_t base = 0; base < total; base += 32 * kMxvIlp) {
            bool mine[kMxvIlp], found[kMxvIlp], done[kMxvIlp];
            int jw[kMxvIlp], bitpos[kMxvIlp];
            uint32_t f1w[kMxvIlp];
            int32_t k[kMxvIlp], end[kMxvIlp], beg[kMxvIlp], f0[kMxvIlp];
#pragma unroll
            for (int r = 0; r < kMxvIlp; ++r) {
                const uint32_t c = base + 32 * r + lane;
                mine[r] = c < total;
                const int off = mine[r] ? (int)list[c] : 0;
                const int j = off >> 5;
                jw[r] = j;
                f1w[r] = __shfl_sync(0xffffffffu, f1, j);
                bitpos[r] = off & 31;
                found[r] = false;
                done[r] = false;
            }
            int4 nx[kMxvIlp];
#pragma unroll
            for (int r = 0; r < kMxvIlp; ++r) {
                const int32_t i = (((tile << 5) + jw[r]) << 5) + bitpos[r];
                beg[r] = mine[r] ? ptr[i] : 0;
                end[r] = mine[r] ? ptr[i + 1] : 0;
                f0[r] = (mine[r] && !two_pass) ? (first ? first[i] : -2) : -1;
                nx[r] = (mine[r] && next) ? next[i] : make_int4(-1, -1, -1, -1);
            }
#pragma unroll
            for (int r = 0; r < kMxvIlp; ++r) {
                if (!mine[r]) continue;
                k[r] = beg[r] + 1;
                if (two_pass) {  // the first entry was examined (and counted) by the first pass
                    found[r] = (f1w[r] >> bitpos[r]) & 1u;  // only without early exit can it be set here
                    continue;
                }
                rows += 1;
                if (f0[r] == -2) f0[r] = col[beg[r]];  // no first-entry array: read the row's first entry
                exam += 1;
                if (bit_test(ubm, f0[r])) {
                    found[r] = true;
                    done[r] = early_exit != 0;
                }
            }
            // entries 1..4 from the dense next-entries array (one 16-byte read, four probes in flight)
#pragma unroll
            for (int r = 0; r < kMxvIlp; ++r) {
                if (!mine[r] || done[r] || !next) continue;
                const bool h0 = nx[r].x >= 0 && bit_test(ubm, nx[r].x);
                const bool h1 = nx[r].y >= 0 && bit_test(ubm, nx[r].y);
                const bool h2 = nx[r].z >= 0 && bit_test(ubm, nx[r].z);
                const bool h3 = nx[r].w >= 0 && bit_test(ubm, nx[r].w);
                const int nv = (nx[r].x >= 0) + (nx[r].y >= 0) + (nx[r].z >= 0) + (nx[r].w >= 0);
                const int hit = h0 ? 0 : (h1 ? 1 : (h2 ? 2 : (h3 ? 3 : -1)));
                if (hit >= 0) found[r] = true;
                const bool stop = hit >= 0 && early_exit;
                const int used = stop ? hit + 1 : nv;
                exam += (unsigned long long)used;
                k[r] += used;
                done[r] = stop;
            }
            // a lane scans rows of up to kMxvLaneRow entries itself; longer rows get kMxvProbe
            // entries here and the rest from the whole warp below
            while (true) {
                int32_t jj[kMxvIlp][4];
                int32_t cnt[kMxvIlp];
                bool act[kMxvIlp];
#pragma unroll
                for (int r = 0; r < kMxvIlp; ++r) {
                    const int32_t span = end[r] - beg[r] <= kMxvLaneRow ? kMxvLaneRow : kMxvProbe;
                    const int32_t lim = end[r] < beg[r] + span ? end[r] : beg[r] + span;
                    act[r] = mine[r] && !done[r] && k[r] < lim;
                    cnt[r] = act[r] ? (lim - k[r] < 4 ? lim - k[r] : 4) : 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) jj[r][t] = t < cnt[r] ? col[k[r] + t] : 0;
                }
                if (!__any_sync(0xffffffffu, act[0] || act[1])) break;
#pragma unroll
                for (int r = 0; r < kMxvIlp; ++r) {
                    if (!act[r]) continue;
                    int hit = -1;
#pragma unroll
                    for (int t = 3; t >= 0; --t)
                        if (t < cnt[r] && bit_test(ubm, jj[r][t])) hit = t;
                    if (hit >= 0) {
                        found[r] = true;
                        if (early_exit) {
                            exam += (unsigned long long)(hit + 1);
                            k[r] += hit + 1;
                            done[r] = true;
                            continue;
                        }
                    }
                    exam += (unsigned long long)cnt[r];
                    k[r] += cnt[r];
                }
            }
#pragma unroll
            for (int r = 0; r < kMxvIlp; ++r) {
                if (huge && mine[r] && !done[r] && end[r] - beg[r] > kMxvHugeRow) {
                    // still unresolved after the lane probe: mxv_pull_huge_kernel scans the rest of
                    // the row with a whole block (a found row keeps its bit from the probe)
                    const int32_t i = (((tile << 5) + jw[r]) << 5) + bitpos[r];
                    const int32_t slot = atomicAdd(huge_count, 1);  // fewer than n rows: fits
                    huge[slot] = i;
                    huge_next[slot] = k[r];
                    done[r] = true;
                }
                uint32_t pend = __ballot_sync(0xffffffffu, mine[r] && !done[r] && k[r] < end[r]);
                while (pend) {
                    const int t = __ffs(pend) - 1;
                    pend &= pend - 1;
                    int32_t kk = __shfl_sync(0xffffffffu, k[r], t);
                    const int32_t ee = __shfl_sync(0xffffffffu, end[r], t);
                    bool tf = __shfl_sync(0xffffffffu, found[r], t);
                    unsigned long long tx = 0;
                    // 128 entries per round (four independent loads per lane)
                    for (; kk < ee; kk += 128) {
                        int32_t jq[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int32_t idx = kk + 32 * q + lane;
                            jq[q] = idx < ee ? col[idx] : -1;
                        }
                        bool stop = false;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (stop) break;
                            const uint32_t hb = __ballot_sync(0xffffffffu, jq[q] >= 0 && bit_test(ubm, jq[q]));
                            const int32_t left = ee - (kk + 32 * q);
                            if (left <= 0) break;
                            if (hb) {
                                tf = true;
                                if (early_exit) {
                                    tx += (unsigned long long)__ffs(hb);
                                    stop = true;
                                    break;
                                }
                            }
                            tx += (unsigned long long)(left < 32 ? left : 32);
                        }
                        if (stop) break;
                    }
                    if (lane == t) {
                        found[r] = tf;
                        exam += tx;
                    }
                }
                if (found[r]) atomicOr(hits + jw[r], 1u << bitpos[r]);
            }
        }
        __syncwarp();
        if (wok) R[w] = hits[lane];
        __syncwarp();
    }
    if (stats) {
        rows = warp_sum_u64(rows);
        exam = warp_sum_u64(exam);
        if (lane == 0) {
            if (rows) atomicAdd(&stats->rows, rows);
            if (exam) atomicAdd(&stats->exam, exam);
        }
    }
}

// Rows longer than kMxvHugeRow that the lane probe left unresolved: block b takes
// rows b, b + gridDim.x, ... of the deferred list (row, next entry) and its warps
// split the rest of the row into 1024-entry chunks, so a power-law hub is not
// scanned by one warp.  A hit sets the row's result bit; with early exit, chunks
// of a row already found are skipped.
__global__ void __launch_bounds__(kMxvThreads) mxv_pull_huge_kernel(const int32_t* __restrict__ ptr,
                                                                     const int32_t* __restrict__ col,
                                                                     const uint32_t* __restrict__ ubm, uint32_t* R,
                                                                     const int32_t* huge, const int32_t* huge_next,
                                                                     const int32_t* huge_count,
                                                                     int early_exit, const int32_t* flag, MxvStats* stats) {
    if (!dir_enabled(flag, GBX_DIR_PULL)) return;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int32_t count = *huge_count;
    unsigned long long exam = 0;
    for (int32_t h = blockIdx.x; h < count; h += gridDim.x) {
        const int32_t i = huge[h];
        const int32_t beg = huge_next[h], end = ptr[i + 1];
        for (int32_t c0 = beg + wib * kMxvChunk; c0 < end; c0 += nw * kMxvChunk) {
            if (early_exit && ((__ldcg(R + (i >> 5)) >> (i & 31)) & 1u)) break;
            const int32_t c1 = end - c0 > kMxvChunk ? c0 + kMxvChunk : end;
            bool hit = false;
            for (int32_t k = c0 + lane; k < c1; k += 32) hit |= bit_test(ubm, col[k]);
            exam += (unsigned long long)((c1 - c0) / 32 + (lane < (c1 - c0) % 32 ? 1 : 0));
            if (__any_sync(0xffffffffu, hit)) {
                if (lane == 0) atomicOr(R + (i >> 5), 1u << (i & 31));
                if (early_exit) break;
            }
        }
    }
    if (stats) {
        exam = warp_sum_u64(exam);
        if (lane == 0 && exam) atomicAdd(&stats->exam, exam);
    }
}

__global__ void mxv_degrees_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ list,
                                   const int32_t* count_dev, int32_t cap, int32_t n, int32_t* __restrict__ deg,
                                   const int32_t* flag) {
    if (!dir_enabled(flag, GBX_DIR_PUSH)) return;
    // same count as the scan that follows (clamped to n); entries past the
    // capacity or outside [0, n) expand nothing
    const int32_t count = min(*count_dev, n);
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int32_t u = k < cap ? list[k] : -1;
        deg[k] = (u >= 0 && u < n) ? ptr[u + 1] - ptr[u] : 0;
    }
}

// Number of entries of the warp-held sorted window (one value per lane) that are <= e.
__device__ __forceinline__ int window_rank(long long win, long long e) {
    int c = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) c += (__shfl_sync(0xffffffffu, win, j) <= e) ? 1 : 0;
    return c;
}

__device__ __forceinline__ int32_t last_le(const int32_t* pre, int32_t lo, int32_t hi, long long e) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((long long)pre[mid] <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kMxvThreads) mxv_push_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                                                const int32_t* __restrict__ list, const int32_t* count_dev,
                                                                int32_t cap, const int32_t* __restrict__ pre,
                                                                const uint32_t* __restrict__ pass, uint32_t* R,
                                                                const int32_t* flag, MxvStats* stats) {
    if (!dir_enabled(flag, GBX_DIR_PUSH)) return;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int32_t count = min(*count_dev, cap);  // cap = n here: matches the scan's count
    if (count <= 0) return;
    const long long E = pre[count];
    if (stats && gwarp == 0 && lane == 0) {
        atomicAdd(&stats->ucount, (unsigned long long)count);
        atomicAdd(&stats->edges, (unsigned long long)E);
    }
    long long chunk = (E + nwarps - 1) / nwarps;
    chunk = chunk < 64 ? 64 : ((chunk + 31) & ~31ll);
    for (long long e0 = (long long)gwarp * chunk; e0 < E; e0 += (long long)nwarps * chunk) {
        const long long e1 = e0 + chunk < E ? e0 + chunk : E;
        int32_t k = 0;
        if (lane == 0) k = last_le(pre, 0, count - 1, e0);
        k = __shfl_sync(0xffffffffu, k, 0);
        for (long long base = e0; base < e1; base += 32) {
            const int32_t wi = k + 1 + lane;
            const long long win = wi < count ? (long long)pre[wi] : (long long)INT64_MAX;
            const long long e = base + lane;
            const int c = window_rank(win, e);
            int32_t kk = k + c;
            if (c == 32) kk = last_le(pre, k + 32, count - 1, e);  // many empty columns in a row
            if (e < e1) {
                const int32_t u = list[kk];
                const int32_t v = col[ptr[u] + (int32_t)(e - pre[kk])];
                if (!pass || bit_test(pass, v)) {
                    const uint32_t bit = 1u << (v & 31);
                    if (!(__ldcg(R + (v >> 5)) & bit)) atomicOr(R + (v >> 5), bit);
                }
            }
            k = __shfl_sync(0xffffffffu, kk, 31);
        }
    }
}

// AUTO: push when nnz(u)/n <= alpha (input sparsity), else pull (Section 6.3).
__global__ void mxv_decide_kernel(const int32_t* count_dev, int32_t n, float alpha, int32_t* flag) {
    const double r = (double)(*count_dev) / (double)n;
    *flag = r <= (double)alpha ? GBX_DIR_PUSH : GBX_DIR_PULL;
}

__global__ void zero_stats_kernel(MxvStats* s) {
    MxvStats z = {};
    *s = z;
}

__global__ void set_push_stats_kernel(MxvStats* s, int32_t ucount, int64_t edges) {
    s->ucount = (unsigned long long)ucount;
    s->edges = (unsigned long long)edges;
}

static gbx_status check_vec(const gbx_vector* v, int32_t n, const char* name, bool output) {
    GBX_CHECK(v->format == GBX_DENSE || v->format == GBX_SPARSE || v->format == GBX_DENSE_F32, GBX_ERR_INVALID_VALUE,
              std::string(name) + ": unknown format");
    GBX_CHECK(v->size == n, GBX_ERR_DIMENSION_MISMATCH, std::string(name) + ": size differs from the graph's n");
    GBX_CHECK(v->data != nullptr, GBX_ERR_NULL_POINTER, std::string(name) + ": data is NULL");
    if (v->format == GBX_SPARSE) {
        GBX_CHECK(v->nnz != nullptr, GBX_ERR_NULL_POINTER, std::string(name) + ": nnz is NULL");
        GBX_CHECK(v->capacity >= 0, GBX_ERR_INVALID_VALUE, std::string(name) + ": capacity < 0");
        if (output)
            GBX_CHECK(v->capacity >= v->size, GBX_ERR_INVALID_VALUE,
                      std::string(name) + ": a sparse output needs capacity >= size");
    }
    return GBX_OK;
}

// mask -> bitmap of passing rows; pass = m XOR complement (Algorithm 2, line 3).
// No mask: every row passes (*pass_bm = NULL), or none with the complement.
static gbx_status build_pass(Graph* G, const gbx_vector* mask, int complement, const uint32_t** pass_bm,
                             bool* nothing_passes, cudaStream_t s) {
    const int32_t n = G->n;
    uint32_t* pass = G->ws.bm[1];
    *pass_bm = nullptr;
    *nothing_passes = false;
    if (!mask) {
        *nothing_passes = complement != 0;
    } else if (mask->format == GBX_DENSE) {
        GBX_TRY(pack_dense_to_bitmap((const uint8_t*)mask->data, n, complement ? 1u : 0u, pass, s));
        *pass_bm = pass;
    } else {
        GBX_TRY(fill_bitmap(pass, n, 0u, s));
        GBX_TRY(scatter_list_to_bitmap((const int32_t*)mask->data, mask->nnz, mask->capacity, n, pass, s));
        if (complement) GBX_TRY(invert_bitmap(pass, n, s));
        *pass_bm = pass;
    }
    return GBX_OK;
}

gbx_status mxv_minplus(Graph* G, float* w, const uint32_t* pass_bm, bool nothing_passes, const float* u,
                       const gbx_desc& d, cudaStream_t s);
gbx_status mxv_issue(Graph* G, gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_vector* u,
                     const gbx_desc& d, cudaStream_t s);
gbx_status mxv_replay(Graph* G, gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_vector* u,
                      const gbx_desc& d, cudaStream_t s);

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_mxv(gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_graph* A,
                              const gbx_vector* u, const gbx_desc* desc, void* stream) {
    clear_error();
    GBX_TRY(check_graph(A));
    GBX_CHECK(w != nullptr && u != nullptr, GBX_ERR_NULL_POINTER, "w or u is NULL");
    GBX_CHECK(semiring == GBX_LOR_LAND || semiring == GBX_MIN_PLUS_F32, GBX_ERR_NOT_SUPPORTED,
              "semiring must be GBX_LOR_LAND or GBX_MIN_PLUS_F32");
    Graph* G = const_cast<Graph*>(as_impl(A));
    const int32_t n = G->n;
    GBX_TRY(check_vec(u, n, "u", false));
    GBX_TRY(check_vec(w, n, "w", true));
    if (mask) GBX_TRY(check_vec(mask, n, "mask", false));
    GBX_CHECK(w->data != u->data && (!mask || w->data != mask->data), GBX_ERR_INVALID_VALUE,
              "w must not alias u or mask");
    gbx_desc d;
    if (desc)
        d = *desc;
    else
        gbx_desc_init(&d);
    GBX_CHECK(d.direction >= GBX_DIR_AUTO && d.direction <= GBX_DIR_PULL, GBX_ERR_INVALID_VALUE, "desc.direction");
    GBX_CHECK(d.alpha >= 0.0f && d.alpha == d.alpha, GBX_ERR_INVALID_VALUE, "desc.alpha must be >= 0");
    GBX_CHECK(d.push_sort == 0 || d.push_sort == 1, GBX_ERR_INVALID_VALUE, "desc.push_sort must be 0 or 1");
    for (int k = 0; k < 2; ++k) GBX_CHECK(d.reserved[k] == 0, GBX_ERR_INVALID_VALUE, "desc.reserved must be 0");
    GBX_CHECK(!mask || mask->format != GBX_DENSE_F32, GBX_ERR_INVALID_VALUE, "mask: GBX_DENSE or GBX_SPARSE");
    if (semiring == GBX_MIN_PLUS_F32) {
        GBX_CHECK(u->format == GBX_DENSE_F32 && w->format == GBX_DENSE_F32, GBX_ERR_INVALID_VALUE,
                  "the (min, +) semiring takes GBX_DENSE_F32 u and w");
        GBX_CHECK(d.push_sort == 0, GBX_ERR_NOT_SUPPORTED, "desc.push_sort is for the Boolean semiring");
        GBX_CHECK(G->out_val != nullptr, GBX_ERR_INVALID_VALUE,
                  "the (min, +) semiring needs edge weights (gbx_graph_set_weights)");
    } else {
        GBX_CHECK(u->format != GBX_DENSE_F32 && w->format != GBX_DENSE_F32, GBX_ERR_INVALID_VALUE,
                  "GBX_DENSE_F32 vectors belong to the (min, +) semiring");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the sorted push reads the frontier size on the host: issued directly; every
    // other call is one fixed launch sequence, replayed from a captured graph
    if (d.push_sort) return mxv_issue(G, w, mask, semiring, u, d, s);
    return mxv_replay(G, w, mask, semiring, u, d, s);
}

namespace gbx {

gbx_status mxv_issue(Graph* G, gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_vector* u,
                     const gbx_desc& d, cudaStream_t s) {
    const int32_t n = G->n;
    if (semiring == GBX_MIN_PLUS_F32) {
        const uint32_t* pbm = nullptr;
        bool none = false;
        GBX_TRY(build_pass(G, mask, d.mask_complement, &pbm, &none, s));
        GBX_TRY(mxv_minplus(G, (float*)w->data, pbm, none, (const float*)u->data, d, s));
        G->ws.last_stream = s;
        return GBX_OK;
    }

    // w = A' u with A' = A^T (transpose) or A.  Pull reads rows of A' (CSR of A'),
    // push reads the columns of A' selected by u, i.e. rows of (A')^T.
    const int32_t* pull_ptr = d.transpose ? G->in_ptr : G->out_ptr;
    const int32_t* pull_col = d.transpose ? G->in_col : G->out_col;
    const uint32_t* pull_nz = d.transpose ? G->nz_in : G->nz_out;
    const int32_t* pull_first = d.transpose ? G->first_in : G->first_out;
    const int4* pull_next = d.transpose ? G->next_in : G->next_out;
    const int32_t* push_ptr = d.transpose ? G->out_ptr : G->in_ptr;
    const int32_t* push_col = d.transpose ? G->out_col : G->in_col;

    uint32_t* ubm = G->ws.bm[0];
    uint32_t* R = G->ws.bm[2];
    int32_t* list_count = G->ws.flag + 0;
    int32_t* dflag = G->ws.flag + 1;
    MxvStats* stats = d.trace ? reinterpret_cast<MxvStats*>(G->ws.ctr + 3) : nullptr;
    if (stats) zero_stats_kernel<<<1, 1, 0, s>>>(stats);

    int dir = d.direction;
    bool want_pull = dir != GBX_DIR_PUSH;
    bool want_push = dir != GBX_DIR_PULL;

    // u as a bitmap (pull) and as a sorted list (push)
    const int32_t* ulist = nullptr;
    const int32_t* ucount = nullptr;
    int32_t ucap = n;
    if (u->format == GBX_DENSE) {
        GBX_TRY(pack_dense_to_bitmap((const uint8_t*)u->data, n, 0, ubm, s));
        if (want_push) {
            GBX_TRY(bitmap_to_list(ubm, n, G->ws.list, list_count, G->ws.qd[0], G->ws.scan_tmp, s));
            ulist = G->ws.list;
            ucount = list_count;
        }
    } else {
        ulist = (const int32_t*)u->data;
        ucount = u->nnz;
        ucap = u->capacity < n ? u->capacity : n;
        if (want_pull) {
            GBX_TRY(fill_bitmap(ubm, n, 0u, s));
            GBX_TRY(scatter_list_to_bitmap(ulist, ucount, ucap, n, ubm, s));
        }
    }
    const uint32_t* pass_bm = nullptr;
    bool nothing_passes = false;
    GBX_TRY(build_pass(G, mask, d.mask_complement, &pass_bm, &nothing_passes, s));
    // Algorithm 3 (desc.push_sort): sizes its scratch from the frontier, so the
    // frontier size and the AUTO decision are taken on the host
    bool sorted_done = false;
    if (d.push_sort && want_push && !nothing_passes) {
        int32_t hc = 0;
        GBX_CUDA_TRY(cudaMemcpyAsync(&hc, ucount, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GBX_CUDA_TRY(cudaStreamSynchronize(s));
        if (dir == GBX_DIR_PUSH || (double)hc / (double)n <= (double)d.alpha) {
            const int32_t count = hc < 0 ? 0 : (hc > n ? n : hc);
            const bool direct = w->format == GBX_SPARSE && !d.accum;  // the sorted list is w itself
            if (!direct) GBX_TRY(fill_bitmap(R, n, 0u, s));
            int64_t edges = 0;
            GBX_TRY(mxv_push_sorted(G, push_ptr, push_col, ulist, count, ucap, pass_bm, direct ? nullptr : R,
                                    direct ? (int32_t*)w->data : nullptr, direct ? w->nnz : nullptr, &edges, s));
            if (stats) set_push_stats_kernel<<<1, 1, 0, s>>>(stats, count, edges);
            if (direct) {
                GBX_CUDA_TRY(cudaGetLastError());
                G->ws.last_stream = s;
                return GBX_OK;
            }
            sorted_done = true;
        } else {
            dir = GBX_DIR_PULL;
            want_push = false;
        }
    }
    // a pull writes every result word; push accumulates into a cleared bitmap
    if (!sorted_done && (want_push || nothing_passes)) GBX_TRY(fill_bitmap(R, n, 0u, s));
    if (!nothing_passes && !sorted_done) {
        const int32_t* flag = nullptr;
        if (dir == GBX_DIR_AUTO) {
            mxv_decide_kernel<<<1, 1, 0, s>>>(ucount, n, d.alpha, dflag);
            flag = dflag;
        }
        if (want_push) {
            int32_t* deg = G->ws.q[0];
            int32_t* pre = G->ws.qp[0];
            mxv_degrees_kernel<<<max(1u, min(div_up(n, 256), 152u * 16)), 256, 0, s>>>(push_ptr, ulist, ucount, ucap,
                                                                                    n, deg, flag);
            GBX_TRY(exclusive_scan_i32(deg, pre, n, ucount, G->ws.scan_tmp, s));
            mxv_push_kernel<<<G->num_sms * 8, kMxvThreads, 0, s>>>(push_ptr, push_col,
                                                                    ulist, ucount, n, pre, pass_bm, R, flag, stats);
        }
        if (want_pull) {
            int32_t* huge = G->ws.q[1];
            int32_t* huge_next = G->ws.qp[1];
            int32_t* huge_count = G->ws.flag + 2;
            GBX_CUDA_TRY(cudaMemsetAsync(huge_count, 0, sizeof(int32_t), s));
            mxv_pull_kernel<<<G->num_sms * 8, kMxvThreads, 0, s>>>(pull_ptr, pull_col, pull_first, pull_next, pull_nz,
                                                                    d.transpose ? G->multi_in : G->multi_out, ubm,
                                                                    pass_bm, R, G->nwords, d.early_exit ? 1 : 0, flag,
                                                                    stats, huge, huge_next, huge_count);
            mxv_pull_huge_kernel<<<G->num_sms * 8, kMxvThreads, 0, s>>>(pull_ptr, pull_col, ubm, R, huge, huge_next,
                                                                         huge_count, d.early_exit ? 1 : 0, flag, stats);
        }
    }
    // output
    if (w->format == GBX_DENSE) {
        GBX_TRY(bitmap_to_dense(R, n, d.accum ? (const uint8_t*)w->data : nullptr, (uint8_t*)w->data, s));
    } else {
        if (d.accum) GBX_TRY(scatter_list_to_bitmap((const int32_t*)w->data, w->nnz, w->capacity, n, R, s));
        GBX_TRY(bitmap_to_list(R, n, (int32_t*)w->data, w->nnz, G->ws.qd[1], G->ws.scan_tmp, s));
    }
    GBX_CUDA_TRY(cudaGetLastError());
    G->ws.last_stream = s;
    return GBX_OK;
}

// ---------------------------------------------------------------- captured launch sequences

// A gbx_mxv call with the same graph, buffers, counts' addresses, semiring and
// descriptor issues the same kernels with the same arguments (counts and
// contents are read on the device), so its launch sequence is captured once, on
// a private stream, into a CUDA graph and replayed on the caller's stream.  The
// most recently used kMxvGraphs sequences are kept per graph.
constexpr size_t kMxvGraphs = 32;

struct MxvKey {
    const void* wd;
    const void* wn;
    const void* md;
    const void* mn;
    const void* ud;
    const void* un;
    int32_t wf, wc, mf, mc, uf, uc, has_mask, semiring;
    gbx_desc d;
};

struct MxvCache {
    struct Entry {
        MxvKey key;
        cudaGraphExec_t exec;
        uint64_t used;
    };
    std::vector<Entry> entries;
    uint64_t clock = 0;
};

static MxvKey make_key(const gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_vector* u,
                       const gbx_desc& d) {
    MxvKey k;
    std::memset(&k, 0, sizeof(k));
    k.wd = w->data;
    k.wn = w->format == GBX_SPARSE ? w->nnz : nullptr;
    k.wf = w->format;
    k.wc = w->format == GBX_SPARSE ? w->capacity : 0;
    if (mask) {
        k.has_mask = 1;
        k.md = mask->data;
        k.mn = mask->format == GBX_SPARSE ? mask->nnz : nullptr;
        k.mf = mask->format;
        k.mc = mask->format == GBX_SPARSE ? mask->capacity : 0;
    }
    k.ud = u->data;
    k.un = u->format == GBX_SPARSE ? u->nnz : nullptr;
    k.uf = u->format;
    k.uc = u->format == GBX_SPARSE ? u->capacity : 0;
    k.semiring = semiring;
    k.d = d;
    return k;
}

void mxv_cache_release(Graph* G) {
    if (G->mxv_cache) {
        for (auto& e : G->mxv_cache->entries) cudaGraphExecDestroy(e.exec);
        delete G->mxv_cache;
        G->mxv_cache = nullptr;
    }
    if (G->mxv_cap_stream) {
        cudaStreamDestroy(G->mxv_cap_stream);
        G->mxv_cap_stream = nullptr;
    }
}

gbx_status mxv_replay(Graph* G, gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_vector* u,
                      const gbx_desc& d, cudaStream_t s) {
    if (!G->mxv_cache) {
        G->mxv_cache = new (std::nothrow) MxvCache();
        GBX_CHECK(G->mxv_cache != nullptr, GBX_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    MxvCache& C = *G->mxv_cache;
    const MxvKey key = make_key(w, mask, semiring, u, d);
    for (auto& e : C.entries)
        if (std::memcmp(&e.key, &key, sizeof(key)) == 0) {
            e.used = ++C.clock;
            GBX_CUDA_TRY(cudaGraphLaunch(e.exec, s));
            G->ws.last_stream = s;
            return GBX_OK;
        }
    if (!G->mxv_cap_stream) GBX_CUDA_TRY(cudaStreamCreateWithFlags(&G->mxv_cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = G->mxv_cap_stream;
    GBX_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const gbx_status st = mxv_issue(G, w, mask, semiring, u, d, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaErrorUnknown;
    if (st == GBX_OK && ce == cudaSuccess && graph) ie = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != GBX_OK || ce != cudaSuccess || ie != cudaSuccess) {
        // not capturable here: issue the sequence directly on the caller's stream
        if (exec) cudaGraphExecDestroy(exec);
        cudaGetLastError();
        return mxv_issue(G, w, mask, semiring, u, d, s);
    }
    if (C.entries.size() >= kMxvGraphs) {
        size_t lru = 0;
        for (size_t i = 1; i < C.entries.size(); ++i)
            if (C.entries[i].used < C.entries[lru].used) lru = i;
        cudaGraphExecDestroy(C.entries[lru].exec);
        C.entries.erase(C.entries.begin() + (long)lru);
    }
    C.entries.push_back({key, exec, ++C.clock});
    GBX_CUDA_TRY(cudaGraphLaunch(exec, s));
    G->ws.last_stream = s;
    return GBX_OK;
}

}  // namespace gbx

extern "C" gbx_status gbx_mxv_stats(const gbx_graph* A, int64_t* rows, int64_t* examined, int64_t* u_nnz,
                                    int64_t* edges) {
    clear_error();
    GBX_TRY(check_graph(A));
    const Graph* G = as_impl(A);
    if (G->ws.last_stream) GBX_CUDA_TRY(cudaStreamSynchronize(G->ws.last_stream));
    MxvStats st;
    GBX_CUDA_TRY(cudaMemcpy(&st, G->ws.ctr + 3, sizeof(st), cudaMemcpyDeviceToHost));
    if (rows) *rows = (int64_t)st.rows;
    if (examined) *examined = (int64_t)st.exam;
    if (u_nnz) *u_nnz = (int64_t)st.ucount;
    if (edges) *edges = (int64_t)st.edges;
    return GBX_OK;
}
