// Internal declarations shared by the libgbx translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gbx.h"

namespace gbx {

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);
void clear_error();
uint64_t wait_timeout_ns();

#define GBX_CUDA_TRY(expr)                                                                                \
    do {                                                                                                  \
        cudaError_t err__ = (expr);                                                                       \
        if (err__ != cudaSuccess) {                                                                       \
            ::gbx::set_error(std::string(#expr) + ": " + cudaGetErrorString(err__) + " (" + __FILE__ + ":" + \
                             std::to_string(__LINE__) + ")");                                             \
            return err__ == cudaErrorMemoryAllocation ? GBX_ERR_OUT_OF_MEMORY : GBX_ERR_CUDA;             \
        }                                                                                                 \
    } while (0)

#define GBX_CHECK(cond, status, msg)       \
    do {                                   \
        if (!(cond)) {                     \
            ::gbx::set_error(msg);         \
            return (status);               \
        }                                  \
    } while (0)

#define GBX_TRY(expr)                      \
    do {                                   \
        gbx_status st__ = (expr);          \
        if (st__ != GBX_OK) return st__;   \
    } while (0)

// ---------------------------------------------------------------- device status words

// Device-side status: [0] error code recorded by kernels (GBX_ERR_TIMEOUT ...),
// [1] levels of the last BFS, [2] index of the first bad vertex (graph build).
enum { ST_ERROR = 0, ST_LEVELS = 1, ST_BADINDEX = 2, ST_WORDS = 8 };

// ---------------------------------------------------------------- level counters

// One BFS level's counters, written with atomics by the level's producers.
struct LevelCtr {
    unsigned long long q;          // low 32 bits: queue entries, high 32: their out-degree sum
    unsigned long long n_new;      // vertices discovered (all)
    unsigned long long mf_new;     // out-degree sum of the discovered vertices
    unsigned long long indeg_new;  // in-degree sum of the discovered vertices
    unsigned long long e_exam;     // pull: in-edges examined
    unsigned long long list;       // batched BFS: entries of the level's row list
    unsigned long long huge;       // pull: deferred long rows (low 32 bits) and their edge chunks (high 32)
    unsigned long long pad[1];
};

// Arrival counters of the persistent kernels' grid barrier.  Within one launch a
// counter only grows (barrier r completes when it reaches r * nblocks); launches
// alternate between the two counters and each launch zeroes the one it does not
// use, so a launch that gave up half-way leaves nothing behind for the next.
struct GridBar {
    unsigned int count[2];
    unsigned int pad[30];
};

// Device-side trace record (mirrors gbx_level; nu / nu_nz filled on the host).
struct LevelRec {
    int32_t direction;
    int32_t level;
    long long nf, mf, mu, e_exam, n_new, mf_new, t_ns;
};

constexpr int kTraceCap = 1 << 16;

// ---------------------------------------------------------------- graph

// Per-run scratch of the persistent kernels and of gbx_mxv.  A graph owns one
// (used by gbx_bfs, gbx_mxv, gbx_bfs_batch); the server gives each of its slots
// another, so several batches of the same graph can run at once.
struct Workspace {
    int32_t n_cap = 0;  // vertices the buffers below hold
    uint32_t* bm[4] = {nullptr, nullptr, nullptr, nullptr};  // n-bit bitmaps
    int32_t* q[2] = {nullptr, nullptr};                       // frontier queues
    int32_t* qp[2] = {nullptr, nullptr};                      // out-degree prefix per entry
    int32_t* qd[2] = {nullptr, nullptr};                      // row start minus prefix per entry
    int32_t* list = nullptr;                                  // n ints (mxv lists, touched lists)
    int32_t* scan_tmp = nullptr;                              // block sums for scans
    LevelCtr* ctr = nullptr;                                  // 4 entries
    GridBar* bar = nullptr;
    LevelRec* trace = nullptr;                                // kTraceCap records
    int32_t* status = nullptr;                                // ST_WORDS ints
    int32_t* flag = nullptr;                                  // small device scratch (mxv decisions)
    unsigned int bar_parity = 0;  // counter of GridBar the next persistent launch uses
    // batched multi-source BFS scratch (allocated on first use, grown as needed)
    unsigned long long* msV = nullptr;                     // visited lanes [n][W]
    unsigned long long* msF[3] = {nullptr, nullptr, nullptr};  // lanes found per level, rotating [n][W]
    unsigned long long* msP = nullptr;  // depth bit planes: 5 x [n][W] (bits 0-3 of depths below 16, overflow)
    int32_t* msT = nullptr;                                    // vertices a wide push level touched [n]
    int64_t ms_t_cap = 0;                                      // entries msT holds
    int64_t ms_cap_words = 0;
    int32_t* ms_src = nullptr;  // device copy of the sources
    int32_t* ms_src_pinned = nullptr;
    int32_t ms_src_cap = 0;
    cudaEvent_t ms_src_ready = nullptr;
    cudaStream_t last_stream = nullptr;
    int last_traced = 0;
};

gbx_status workspace_alloc(Workspace& w, int32_t n);
void workspace_release(Workspace& w);

struct Graph {
    int32_t n = 0;
    int32_t nwords = 0;  // ceil(n / 32)
    int64_t nnz = 0;
    int32_t symmetric = 0;
    int device = 0;
    int num_sms = 0;
    // CSR of A (out-edges) and of A^T (in-edges); in_* alias out_* when symmetric.
    int32_t* out_ptr = nullptr;
    int32_t* out_col = nullptr;
    int32_t* in_ptr = nullptr;
    int32_t* in_col = nullptr;
    uint32_t* nz_in = nullptr;   // bit v set iff in-degree(v) > 0
    uint32_t* nz_out = nullptr;  // bit v set iff out-degree(v) > 0
    uint32_t* multi_in = nullptr;   // bit v set iff in-degree(v) > 1
    uint32_t* multi_out = nullptr;  // bit v set iff out-degree(v) > 1 (aliases multi_in when symmetric)
    // first (smallest) in-neighbour of each row, -1 if none: the first probe of a
    // pull row reads this dense array instead of a random sector of in_col
    int32_t* first_in = nullptr;
    int32_t* first_out = nullptr;
    // entries 1..4 of each row (-1 past its end), one 16-byte load: a pull row that the
    // first entry did not settle probes these before it reads the row offsets and in_col
    int4* next_in = nullptr;
    int4* next_out = nullptr;
    // binary32 edge weights (gbx_graph_set_weights): out_val[k] belongs to out_col[k],
    // in_val[k] to in_col[k] (aliases out_val when symmetric); NULL until set
    float* out_val = nullptr;
    float* in_val = nullptr;
    // the rows with in-edges, ascending (nzr_in), and where their in-edges start
    // (nzr_in_ptr, nnzr_in + 1 entries, the last = nnz): the edge-balanced (min, +)
    // pull walks these.  One allocation, made with the weights.
    int32_t* nzr_in = nullptr;
    int32_t* nzr_in_ptr = nullptr;
    int32_t nnzr_in = 0;
    int32_t drop_self_loops = 0;  // as built
    Workspace ws;  // scratch of the operations called on this graph (ordered on one stream)
    // host-side copies for gbx_bfs_host (allocated on first use)
    int32_t* hdepth[2] = {nullptr, nullptr};
    int32_t* hparent[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    int bfs_blocks = 0;  // BFS launch geometry
    // gbx_mxv launch sequences captured as CUDA graphs (keyed by the call's buffers and descriptor)
    cudaStream_t mxv_cap_stream = nullptr;
    struct MxvCache* mxv_cache = nullptr;
};

// Releases the captured gbx_mxv graphs of G (mxv.cu).
void mxv_cache_release(Graph* G);

// ---------------------------------------------------------------- primitives (prims.cu)

constexpr int kScanBlock = 1024;      // threads per scan block
constexpr int kScanItems = 4;         // items per thread
constexpr int kScanTile = kScanBlock * kScanItems;

// Exclusive scan of in[0 .. *count_dev) (or [0, count_max) when count_dev is NULL) into
// out[0 .. count], with out[count] = total.  tmp needs scan_tmp_ints(count_max) ints.
size_t scan_tmp_ints(int64_t count_max);
gbx_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t count_max, const int32_t* count_dev,
                              int32_t* tmp, cudaStream_t s);

// Stable LSD radix sort of 64-bit keys on the low `bits` bits; result in *keys (buffers swapped as needed).
gbx_status radix_sort_u64(unsigned long long** keys, unsigned long long** alt, int64_t n, int bits, cudaStream_t s);
// The same for 32-bit keys (the key-only sort of Algorithm 3's multiway merge).
gbx_status radix_sort_u32(uint32_t** keys, uint32_t** alt, int64_t n, int bits, cudaStream_t s);

struct Graph;
// Column-based matvec as Algorithm 3 (mxv_sort.cu): the columns of u's `count`
// entries (ulist, entries at or past `cap` expand nothing) are gathered, sorted,
// reduced and masked by pass_bm (NULL: all pass).  Output either as a sorted list
// (out_list + device count out_count) or as bits set in R (out_list NULL).
// *edges receives the number of gathered entries.  Synchronises `s` once.
gbx_status mxv_push_sorted(Graph* G, const int32_t* push_ptr, const int32_t* push_col, const int32_t* ulist,
                           int32_t count, int32_t cap, const uint32_t* pass_bm, uint32_t* R, int32_t* out_list,
                           int32_t* out_count, int64_t* edges, cudaStream_t s);

// Bitmap helpers.
gbx_status pack_dense_to_bitmap(const uint8_t* dense, int32_t n, uint32_t invert, uint32_t* bm, cudaStream_t s);
// Entries outside [0, n) are ignored.
gbx_status scatter_list_to_bitmap(const int32_t* list, const int32_t* count_dev, int32_t cap, int32_t n, uint32_t* bm,
                                  cudaStream_t s);
gbx_status fill_bitmap(uint32_t* bm, int32_t n, uint32_t value, cudaStream_t s);
gbx_status invert_bitmap(uint32_t* bm, int32_t n, cudaStream_t s);
gbx_status bitmap_to_list(const uint32_t* bm, int32_t n, int32_t* list, int32_t* count_dev, int32_t* scan_out,
                          int32_t* tmp, cudaStream_t s);
gbx_status bitmap_to_dense(const uint32_t* bm, int32_t n, const uint8_t* old_dense, uint8_t* out, cudaStream_t s);

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) { return *(const volatile int32_t*)p; }

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// atomic min of a binary32 value: non-negative floats order like their int bits
// and negative ones in reverse of their unsigned bits, so the two halves use
// atomicMin (int) and atomicMax (unsigned).  Returns the previous value.  NaN is
// never stored (callers keep it out).
__device__ __forceinline__ float atomic_min_f32(float* a, float v) {
    if (v >= 0.0f) return __int_as_float(atomicMin(reinterpret_cast<int*>(a), __float_as_int(v)));
    return __uint_as_float(atomicMax(reinterpret_cast<unsigned int*>(a), __float_as_uint(v)));
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ bool bit_test(const uint32_t* bm, int32_t v) { return (bm[v >> 5] >> (v & 31)) & 1u; }

// Inclusive warp scan (sum) of a 32-bit value.
__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Grid-wide barrier for persistent cooperative kernels.  Thread 0 of each block
// arrives with a release reduction and polls with relaxed loads until all
// nblocks blocks of this round have arrived, then takes one acquire load of the
// counter; nothing else is on that path.  Bounded: every 16th poll also reads the
// status word and the clock; a block that sees an error recorded by another block,
// or that has waited longer than timeout_ns (it then records GBX_ERR_TIMEOUT in
// status[ST_ERROR]), returns false, and so does every block still waiting once an
// error is recorded.  Blocks decide to stop for other reasons (a level cap) all
// alike, so a completed barrier needs no status check.  `round` is thread 0's
// count of barriers passed in this launch.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int nblocks, unsigned int& round,
                                             int32_t* status, unsigned long long timeout_ns) {
    __shared__ int ok_shared;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        round += 1;
        const unsigned int target = round * nblocks;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        unsigned int spins = 0;
        unsigned long long t0 = 0ull;
        // relaxed polls (an acquire on every poll would cost more per iteration), then one
        // acquire load once the count is reached, which orders everything after the barrier
        while ((int)(ld_relaxed_u32(count) - target) < 0) {
            if ((++spins & 15u) == 0u) {
                if (ld_volatile_i32(status + ST_ERROR) != 0) {
                    ok = 0;
                    break;
                }
                const unsigned long long now = global_timer_ns();
                if (t0 == 0ull) {
                    t0 = now;
                } else if (now - t0 > timeout_ns) {
                    atomicCAS(status + ST_ERROR, 0, (int)GBX_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok) (void)ld_acquire_u32(count);
        ok_shared = ok;
    }
    __syncthreads();
    return ok_shared != 0;
}

inline unsigned int div_up(int64_t a, int64_t b) { return (unsigned int)((a + b - 1) / b); }

inline gbx_status check_graph(const gbx_graph* g) {
    GBX_CHECK(g != nullptr, GBX_ERR_NULL_POINTER, "graph handle is NULL");
    return GBX_OK;
}

inline Graph* as_impl(gbx_graph* g) { return reinterpret_cast<Graph*>(g); }
inline const Graph* as_impl(const gbx_graph* g) { return reinterpret_cast<const Graph*>(g); }

// The row-based masked matvec of gbx_mxv (mxv.cu), also launched by the
// allocation-free entry point (noalloc.cu).  It must be launched with
// kMxvThreads threads per block: its shared tile is sized from that constant.
constexpr int kMxvThreads = 256;

// Per-call counters of gbx_mxv (desc.trace): [0] rows computed by pull, [1]
// entries examined by pull, [2] nonzeros of u expanded by push, [3] edges expanded.
struct MxvStats {
    unsigned long long rows, exam, ucount, edges, pad[4];
};

__global__ void __launch_bounds__(kMxvThreads)
    mxv_pull_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col, const int32_t* __restrict__ first,
                    const int4* __restrict__ next, const uint32_t* __restrict__ nzrows, const uint32_t* __restrict__ multi,
                    const uint32_t* __restrict__ ubm,
                    const uint32_t* __restrict__ pass, uint32_t* __restrict__ R, int32_t nwords, int early_exit,
                    const int32_t* flag, MxvStats* stats, int32_t* huge, int32_t* huge_next, int32_t* huge_count);

// Batched BFS internals (msbfs.cu), shared with the server.
gbx_status ms_reserve(Workspace& w, int32_t n, int32_t S, cudaStream_t s);
int64_t ms_scratch_bytes(int32_t n, int32_t S);
gbx_status ms_run(Graph* G, Workspace& w, int32_t S, const int32_t* src_dev, void* depth, void* const* rows,
                  int depth16, const gbx_desc& d, int blocks, cudaStream_t s);

}  // namespace gbx
