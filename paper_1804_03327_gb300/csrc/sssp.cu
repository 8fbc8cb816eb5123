// Single-source shortest paths as the two-phase direction-optimised traversal
// Section 5.6 sketches: Bellman-Ford over the (min, +) semiring, starting with
// the column-based (push) matvec of the vertices whose distance improved in the
// last iteration, and switching to the row-based (pull) matvec over every row
// once that set grows (Section 6.3's rule, with beta = 0 keeping the two phases
// of Section 5.6).  No mask: a reached vertex can still improve, and early exit
// does not exist for this semiring.  One persistent cooperative launch, the
// same level loop and queue machinery as the BFS kernel.
//
// Distances are binary32 and every relaxation is one binary32 addition.  For
// non-negative weights the fixpoint is, for each vertex, the smallest rounded
// left-to-right path sum from the source, whichever order relaxations run in
// (rounding is monotonic), so the result does not depend on the schedule.
#include "frontier.cuh"
#include "gbx_internal.cuh"

namespace gbx {

constexpr int kSsspThreads = 512;
// Register budgets: the default build fits two 512-thread blocks on an SM (64
// registers, no spills), the lean build three (40 registers, ~200 bytes of spills).
// Lean hides more gather latency on push iterations over a skewed graph (RMAT-22
// push only: 2.61 -> 2.28 ms) and loses where pull iterations or many small ones
// dominate (the direction rule on RMAT-22 3.27 -> 4.89 ms, a 1024x1024 grid +16 %),
// so a descriptor chooses it (blocks_per_sm >= 3) and the autotuner times it.
constexpr int kSsspOcc = 2;
constexpr int kSsspOccLean = 3;

struct SsspArgs {
    int32_t n, nwords, source;
    const int32_t* out_ptr;
    const int32_t* out_col;
    const float* out_val;
    const int32_t* in_ptr;
    const int32_t* in_col;
    const float* in_val;
    const uint32_t* nz_in;
    float* dist;
    int32_t* stamp;  // iteration + 1 at which the vertex was last queued (dedup of the push queue)
    uint32_t* chg;   // pull: bit v = dist[v] improved in this iteration
    int32_t* q[2];
    int32_t* qp[2];
    int32_t* qd[2];
    LevelCtr* ctr;
    GridBar* bar;
    LevelRec* trace;
    int32_t* status;
    float alpha, beta;
    int32_t mode, trace_cap;
    unsigned long long timeout_ns;
    unsigned int bar_parity;
};

// Push: relax the out-edges of the queued vertices, edge-balanced over warps.
// A vertex whose distance drops is queued once for the next iteration.
__device__ __forceinline__ void sssp_push(const SsspArgs& a, int32_t L, int cur, uint32_t qcount, uint32_t qedges,
                                          Stage& stg, Acc& acc) {
    const int gwarp = (int)((blockIdx.x * kSsspThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kSsspThreads) >> 5);
    const int32_t* q = a.q[cur];
    const int32_t* qp = a.qp[cur];
    const int32_t* qd = a.qd[cur];
    const int32_t E = (int32_t)qedges;
    int32_t chunk = (int32_t)(((long long)E + nwarps - 1) / nwarps);
    chunk = chunk < kPushStep ? kPushStep : ((chunk + kPushStep - 1) / kPushStep) * kPushStep;
    for (long long e0l = (long long)gwarp * chunk; e0l < E; e0l += (long long)nwarps * chunk) {
        const int32_t e0 = (int32_t)e0l;
        const int32_t e1 = E - e0 > chunk ? e0 + chunk : E;
        PushCursor cur_;
        cur_.k = warp_find_entry(qp, (int32_t)qcount, e0);
        cur_.wlast = -1;
        for (int32_t base = e0; base < e1; base += kPushStep) {
            const PushStep st = cur_.gather(a.out_col, q, qp, qd, qcount, base, e1);
            bool queued[kPushIlp];
#pragma unroll
            for (int t = 0; t < kPushIlp; ++t) {
                queued[t] = false;
                if (st.u[t] < 0) continue;
                const float x = a.dist[st.u[t]] + __ldg(a.out_val + st.k[t]);
                if (x < a.dist[st.v[t]]) {
                    const float old = atomic_min_f32(a.dist + st.v[t], x);
                    if (x < old) queued[t] = atomicMax(a.stamp + st.v[t], L + 1) < L + 1;
                }
            }
#pragma unroll
            for (int t = 0; t < kPushIlp; ++t) {
                acc.exam += st.u[t] >= 0 ? 1u : 0u;
                if (queued[t]) acc.n_new += 1;
                stg.put(queued[t], st.v[t]);
            }
        }
    }
    stg.flush();
}

// Pull: every row with in-edges takes the minimum over them; a lane per row,
// rows with more than 32 in-edges reduced by the whole warp.  Improved rows
// set their bit in chg (one word per warp and tile, written whole).
__device__ __forceinline__ void sssp_pull(const SsspArgs& a, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kSsspThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kSsspThreads) >> 5);
    for (int32_t wd = gwarp; wd < a.nwords; wd += nwarps) {
        const int32_t i = (wd << 5) + lane;
        const bool has = (a.nz_in[wd] >> lane) & 1u;
        int32_t beg = 0, end = 0;
        if (has) {
            beg = __ldg(a.in_ptr + i);
            end = __ldg(a.in_ptr + i + 1);
        }
        float t = INFINITY;
        const bool longrow = end - beg > 32;
        if (!longrow)
            for (int32_t k = beg; k < end; ++k) t = fminf(t, a.dist[__ldg(a.in_col + k)] + __ldg(a.in_val + k));
        uint32_t pend = __ballot_sync(0xffffffffu, longrow);
        while (pend) {
            const int owner = __ffs(pend) - 1;
            pend &= pend - 1;
            const int32_t b = __shfl_sync(0xffffffffu, beg, owner);
            const int32_t e = __shfl_sync(0xffffffffu, end, owner);
            float m = INFINITY;
            for (int32_t k = b + lane; k < e; k += 32) m = fminf(m, a.dist[__ldg(a.in_col + k)] + __ldg(a.in_val + k));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == owner) t = m;
        }
        bool better = false;
        if (has && t < a.dist[i]) {
            a.dist[i] = t;  // this lane owns row i
            better = true;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, better);
        if (lane == 0) a.chg[wd] = word;
        acc.exam += (uint32_t)(end - beg);
        if (better) acc.n_new += 1;
    }
}

// The improved set of a pull iteration as the next push queue.
__device__ __forceinline__ void sssp_chg_to_queue(const SsspArgs& a, Stage& st) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kSsspThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kSsspThreads) >> 5);
    const int32_t ntiles = (a.nwords + 31) >> 5;
    for (int32_t tile = gwarp; tile < ntiles; tile += nwarps) {
        const int32_t wl = (tile << 5) + lane;
        const uint32_t mine = wl < a.nwords ? a.chg[wl] : 0u;
        uint32_t todo = __ballot_sync(0xffffffffu, mine != 0u);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t nw = __shfl_sync(0xffffffffu, mine, j);
            st.put((nw >> lane) & 1u, (((tile << 5) + j) << 5) + lane);
        }
    }
    st.flush();
}

template <bool kTrace, int kOcc>
__global__ void __launch_bounds__(kSsspThreads, kOcc) sssp_kernel(SsspArgs a) {
    const long long gtid = (long long)blockIdx.x * kSsspThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kSsspThreads;
    const int32_t s = a.source;
    const int pending = threadIdx.x == 0 ? ld_volatile_i32(a.status + ST_ERROR) : 0;
    unsigned long long t_mark = kTrace && gtid == 0 ? global_timer_ns() : 0ull;
    for (long long i = gtid; i < a.n; i += gstride) {
        a.dist[i] = i == s ? 0.0f : INFINITY;
        a.stamp[i] = 0;
    }
    const int32_t s_rs = __ldg(a.out_ptr + s);
    const int32_t s_od = __ldg(a.out_ptr + s + 1) - s_rs;
    if (gtid == 0) {
        if (s_od > 0) {
            a.q[0][0] = s;
            a.qp[0][0] = 0;
            a.qd[0][0] = s_rs;
        }
        LevelCtr z = {};
        a.ctr[1] = z;
        a.ctr[2] = z;
        z.q = s_od > 0 ? (((unsigned long long)s_od << 32) | 1ull) : 0ull;
        a.ctr[0] = z;
        a.status[ST_LEVELS] = 0;
        a.bar->count[a.bar_parity ^ 1u] = 0u;
    }
    unsigned int* barc = a.bar->count + a.bar_parity;
    unsigned int bar_round = 0;
    if (__syncthreads_or(pending)) return;
    if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;

    __shared__ StageBuf stage_mem[kSsspThreads / 32];
    __shared__ unsigned long long lvl[4];
    __shared__ unsigned long long acc_mem[kSsspThreads / 32][4];
    const int wib = threadIdx.x >> 5;
    unsigned long long qv = s_od > 0 ? (((unsigned long long)s_od << 32) | 1ull) : 0ull;
    int dir = a.mode == GBX_DIR_PULL ? GBX_DIR_PULL : GBX_DIR_PUSH;
    int cur = 0;
    long long nf = 1, mf = s_od;
    for (int32_t L = 0;; ++L) {
        LevelCtr* cout = a.ctr + ((L + 1) % 3);
        if (gtid == 0) {
            LevelCtr z = {};
            a.ctr[(L + 2) % 3] = z;
        }
        const uint32_t qcount = (uint32_t)qv, qedges = (uint32_t)(qv >> 32);
        Acc acc;
        Stage st{stage_mem + wib, 0, cout, a.q[cur ^ 1], a.qp[cur ^ 1], a.qd[cur ^ 1],
                 a.out_ptr, a.in_ptr, 1, 0, &acc};
        if (dir == GBX_DIR_PUSH)
            sssp_push(a, L, cur, qcount, qedges, st, acc);
        else
            sssp_pull(a, acc);
        // counts: n_new, mf_new (push: from the staged degrees), examined edges
        block_add_counts<kSsspThreads / 32>(acc_mem, acc.n_new, acc.mf, acc.exam, 0ull, &cout->n_new, &cout->mf_new,
                                            &cout->e_exam, nullptr);
        if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
        if (threadIdx.x == 0) {
            lvl[0] = ld_volatile_u64(&cout->n_new);
            lvl[1] = ld_volatile_u64(&cout->mf_new);
            lvl[2] = ld_volatile_u64(&cout->e_exam);
            lvl[3] = ld_volatile_u64(&cout->q);
        }
        __syncthreads();
        const long long n_new = (long long)lvl[0];
        long long mf_new = (long long)lvl[1];
        qv = lvl[3];
        int next = dir;
        if (a.mode == GBX_DIR_AUTO && n_new > 0) {
            const double r_new = (double)n_new / (double)a.n;
            if (dir == GBX_DIR_PUSH) {
                if (r_new > (double)a.alpha && n_new > nf) next = GBX_DIR_PULL;
            } else {
                if (r_new < (double)a.beta && n_new < nf) next = GBX_DIR_PUSH;
            }
        }
        if (dir == GBX_DIR_PULL && next == GBX_DIR_PUSH) {
            // the improved set becomes the queue (with its degree prefix)
            sssp_chg_to_queue(a, st);
            if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
            if (threadIdx.x == 0) lvl[3] = ld_volatile_u64(&cout->q);
            __syncthreads();
            qv = lvl[3];
            mf_new = (long long)(qv >> 32);
        }
        if (kTrace && gtid == 0 && L < a.trace_cap) {
            LevelRec r;
            r.direction = dir;
            r.level = L;
            r.nf = nf;
            r.mf = dir == GBX_DIR_PUSH ? mf : -1;
            r.mu = -1;
            r.e_exam = (long long)lvl[2];
            r.n_new = n_new;
            r.mf_new = dir == GBX_DIR_PUSH || next == GBX_DIR_PUSH ? mf_new : -1;
            const unsigned long long now = global_timer_ns();
            r.t_ns = (long long)(now - t_mark);
            t_mark = now;
            a.trace[L] = r;
        }
        if (n_new == 0) {
            if (gtid == 0) a.status[ST_LEVELS] = L + 1;
            return;
        }
        if (L + 1 > a.n) {  // non-negative weights settle within n iterations; a negative cycle does not
            if (gtid == 0) atomicCAS(a.status + ST_ERROR, 0, (int)GBX_ERR_OVERFLOW);
            return;
        }
        nf = n_new;
        mf = mf_new;
        cur ^= 1;
        dir = next;
    }
}

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_sssp(gbx_graph* g, int32_t source, float* dist, const gbx_desc* desc, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(dist != nullptr, GBX_ERR_NULL_POINTER, "dist is NULL");
    Graph* G = as_impl(g);
    GBX_CHECK(source >= 0 && source < G->n, GBX_ERR_INVALID_INDEX, "source outside [0, n)");
    GBX_CHECK(G->out_val != nullptr, GBX_ERR_INVALID_VALUE, "gbx_sssp needs edge weights (gbx_graph_set_weights)");
    gbx_desc d;
    if (desc)
        d = *desc;
    else
        gbx_desc_init(&d);
    GBX_CHECK(d.direction >= GBX_DIR_AUTO && d.direction <= GBX_DIR_PULL, GBX_ERR_INVALID_VALUE, "desc.direction");
    GBX_CHECK(d.alpha >= 0.0f && d.beta >= 0.0f && d.alpha == d.alpha && d.beta == d.beta, GBX_ERR_INVALID_VALUE,
              "desc.alpha / desc.beta must be >= 0");
    GBX_CHECK(d.push_sort == 0, GBX_ERR_NOT_SUPPORTED, "desc.push_sort applies to gbx_mxv only");
    GBX_CHECK(d.blocks_per_sm >= 0, GBX_ERR_INVALID_VALUE, "desc.blocks_per_sm must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    Workspace& w = G->ws;
    SsspArgs a;
    a.n = G->n;
    a.nwords = G->nwords;
    a.source = source;
    a.out_ptr = G->out_ptr;
    a.out_col = G->out_col;
    a.out_val = G->out_val;
    a.in_ptr = G->in_ptr;
    a.in_col = G->in_col;
    a.in_val = G->in_val;
    a.nz_in = G->nz_in;
    a.dist = dist;
    a.stamp = w.list;  // n ints
    a.chg = w.bm[2];
    for (int i = 0; i < 2; ++i) {
        a.q[i] = w.q[i];
        a.qp[i] = w.qp[i];
        a.qd[i] = w.qd[i];
    }
    a.ctr = w.ctr;
    a.bar = w.bar;
    a.trace = w.trace;
    a.status = w.status;
    a.alpha = d.alpha;
    a.beta = d.beta;
    a.mode = d.direction;
    a.trace_cap = kTraceCap;
    a.timeout_ns = wait_timeout_ns();
    a.bar_parity = w.bar_parity;
    const bool lean = d.blocks_per_sm >= kSsspOccLean;
    const void* fn = lean ? (d.trace ? (const void*)sssp_kernel<true, kSsspOccLean>
                                     : (const void*)sssp_kernel<false, kSsspOccLean>)
                          : (d.trace ? (const void*)sssp_kernel<true, kSsspOcc> : (const void*)sssp_kernel<false, kSsspOcc>);
    int per_sm = 0;
    GBX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSsspThreads, 0));
    GBX_CHECK(per_sm >= 1, GBX_ERR_CUDA, "SSSP kernel cannot be resident");
    if (!lean && d.blocks_per_sm > 0 && d.blocks_per_sm < per_sm) per_sm = d.blocks_per_sm;
    void* args[] = {&a};
    GBX_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(per_sm * G->num_sms), dim3(kSsspThreads), args, 0, s));
    w.bar_parity ^= 1u;
    w.last_stream = s;
    w.last_traced = d.trace ? 1 : 0;
    return GBX_OK;
}

extern "C" gbx_status gbx_sssp_trace(gbx_graph* g, gbx_level* levels, int32_t cap, int32_t* nlevels) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(nlevels != nullptr && (cap == 0 || levels != nullptr), GBX_ERR_NULL_POINTER, "levels or nlevels is NULL");
    Graph* G = as_impl(g);
    if (G->ws.last_stream) GBX_CUDA_TRY(cudaStreamSynchronize(G->ws.last_stream));
    int32_t st[ST_WORDS];
    GBX_CUDA_TRY(cudaMemcpy(st, G->ws.status, sizeof(st), cudaMemcpyDeviceToHost));
    GBX_CHECK(st[ST_ERROR] == 0, (gbx_status)st[ST_ERROR], "the last SSSP recorded a device-side error");
    GBX_CHECK(G->ws.last_traced, GBX_ERR_INVALID_VALUE, "the last run was not traced (desc.trace = 0)");
    const int32_t nl = st[ST_LEVELS] < kTraceCap ? st[ST_LEVELS] : kTraceCap;
    *nlevels = nl;
    const int32_t k = nl < cap ? nl : cap;
    if (k > 0) {
        LevelRec* tmp = new LevelRec[k];
        const cudaError_t ce = cudaMemcpy(tmp, G->ws.trace, sizeof(LevelRec) * (size_t)k, cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess)
            for (int32_t i = 0; i < k; ++i) {
                gbx_level& o = levels[i];
                o.direction = tmp[i].direction == GBX_DIR_PUSH ? GBX_DIR_PUSH : GBX_DIR_PULL;
                o.level = tmp[i].level;
                o.nf = tmp[i].nf;
                o.mf = tmp[i].mf;
                o.nu = -1;
                o.nu_nz = -1;
                o.mu = -1;
                o.e_exam = tmp[i].e_exam;
                o.n_new = tmp[i].n_new;
                o.mf_new = tmp[i].mf_new;
                o.time_ns = tmp[i].t_ns;
            }
        delete[] tmp;
        GBX_CUDA_TRY(ce);
    }
    return GBX_OK;
}
