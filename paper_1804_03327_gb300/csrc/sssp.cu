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
// registers), the lean build three (40 registers, ~230 bytes of spills).  Lean
// once hid gather latency on push iterations that waited on one load at a time;
// with the pipelined push and the edge-balanced pull it spills on the hot loops
// and loses (RMAT-22 push only 1.70 -> 3.38 ms, pull only 4.09 -> 4.62 ms), but a
// descriptor can still choose it (blocks_per_sm >= 3) and the autotuner times it.
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
    const int32_t* nzr;      // rows with in-edges, ascending
    const int32_t* nzr_ptr;  // their first in-edge (nnzr + 1 entries)
    int32_t nnzr, nnz;
    float* dist;
    int32_t* stamp;  // iteration + 1 at which the vertex last improved (dedup of the push queue)
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
// A vertex whose distance drops is queued once for the next iteration.  A warp
// range of more than one step is walked as a software pipeline of five stages,
// each on a different step of 32 edges: (1) map the edges to queue entries and
// load their vertex u and row offset, (2) load the child v, the weight and d[u],
// (3) load d[v], (4) lower d[v] with an atomic minimum where d[u] + w is below
// it, (5) claim the lowered children for the next queue (atomicMax on stamp).
// One iteration issues the memory operations of all five stages before it waits
// for any of them.
__device__ __forceinline__ void sssp_push(const SsspArgs& a, int32_t L, int cur, uint32_t qcount, uint32_t qedges,
                                          Stage& stg, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kSsspThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kSsspThreads) >> 5);
    const int32_t* q = a.q[cur];
    const int32_t* qp = a.qp[cur];
    const int32_t* qd = a.qd[cur];
    const int32_t E = (int32_t)qedges;
    int32_t chunk = (int32_t)(((long long)E + nwarps - 1) / nwarps);
    chunk = chunk < 32 ? 32 : ((chunk + 31) / 32) * 32;
    for (long long e0l = (long long)gwarp * chunk; e0l < E; e0l += (long long)nwarps * chunk) {
        const int32_t e0 = (int32_t)e0l;
        const int32_t e1 = E - e0 > chunk ? e0 + chunk : E;
        const int32_t nsteps = (e1 - e0 + 31) / 32;
        PushCursorT<1> cur_;
        cur_.k = warp_find_entry(qp, (int32_t)qcount, e0);
        cur_.wlast = -1;
        if (nsteps == 1) {
            // a single step (a small queue): no pipeline fill and drain
            const PushStepT<1> st = cur_.gather(a.out_col, q, qp, qd, qcount, e0, e1);
            bool queued = false;
            if (st.u[0] >= 0) {
                const float x = a.dist[st.u[0]] + __ldg(a.out_val + st.k[0]);
                if (x < a.dist[st.v[0]]) {
                    const float old = atomic_min_f32(a.dist + st.v[0], x);
                    if (x < old) queued = atomicMax(a.stamp + st.v[0], L + 1) < L + 1;
                }
            }
            acc.exam += st.u[0] >= 0 ? 1u : 0u;
            if (queued) acc.n_new += 1;
            stg.put(queued, st.v[0]);
            continue;
        }
        // stage registers (a child < 0 marks an empty slot: past e1, pipeline fill or drain)
        int32_t u1 = -1, d1 = 0;               // after stage 1: vertex, row start - prefix
        int32_t v2 = -1;                       // after stage 2: child, weight, d[u]
        float w2 = 0.0f, du2 = 0.0f;
        int32_t v3 = -1;                       // after stage 3: child, candidate, d[v]
        float x3 = 0.0f, dv3 = 0.0f;
        int32_t v4 = -1;                       // after stage 4: child, candidate, d[v] before the minimum
        float x4 = 0.0f, old4 = 0.0f;
        for (int32_t it = 0; it < nsteps + 4; ++it) {
            // stage 5 (step it - 4): claim the children whose distance the candidate lowered
            const bool lowered = v4 >= 0 && x4 < old4;
            const int32_t prev = lowered ? atomicMax(a.stamp + v4, L + 1) : L + 1;
            // stage 4 (step it - 3): lower d[v] where the candidate is below the d[v] read
            const float old3 = v3 >= 0 && x3 < dv3 ? atomic_min_f32(a.dist + v3, x3) : x3;
            // stage 3 (step it - 2): d[v]
            const float dv2 = v2 >= 0 ? a.dist[v2] : 0.0f;
            // stage 2 (step it - 1): child, weight, d[u]
            int32_t v1 = -1;
            float w1 = 0.0f, du1 = 0.0f;
            if (u1 >= 0) {
                const int32_t kpos = e0 + (it - 1) * 32 + lane + d1;
                v1 = __ldg(a.out_col + kpos);
                w1 = __ldg(a.out_val + kpos);
                du1 = a.dist[u1];
            }
            // stage 1 (step it): queue entries
            int32_t u0[1] = {-1}, d0[1] = {0};
            if (it == 0) {
                cur_.map(q, qp, qd, qcount, e0, e1, u0, d0);
            } else if (it < nsteps) {
                const int32_t ul = __shfl_sync(0xffffffffu, u1, 31);
                const int32_t dl = __shfl_sync(0xffffffffu, d1, 31);
                cur_.map_after(q, qp, qd, qcount, e0 + it * 32, e1, ul, dl, u0, d0);
            }
            // stage 5, continued: queue the claimed children
            const bool queued = lowered && prev < L + 1;
            acc.exam += u1 >= 0 ? 1u : 0u;
            if (queued) acc.n_new += 1;
            stg.put(queued, v4);
            // advance the pipeline
            v4 = v3;
            x4 = x3;
            old4 = old3;
            v3 = v2;
            x3 = du2 + w2;
            dv3 = dv2;
            v2 = v1;
            w2 = w1;
            du2 = du1;
            u1 = u0[0];
            d1 = d0[0];
        }
    }
    stg.flush();
}

// Pull: every row with in-edges takes the minimum of d[j] + w(j, i) over them.
// The in-edges of the rows that have any (the compact list nzr, with nzr_ptr
// where each row's in-edges start) are cut into equal chunks, one per warp, so a
// hub row costs no more than its edges.  A warp walks its chunk kSpullStep edges
// at a time, each lane kSpullVec consecutive edges (one 16-byte load of columns
// and one of weights, issued a step ahead): the lane takes the minimum over each
// row's run of its edges, a group minimum over the lanes whose last run belongs
// to one row joins the rows that cross lanes, and the row still open at the end
// of a step is carried into the next.  Finished rows are queued in a per-warp
// ring in shared memory and written 32 at a time, one per lane, so no step waits
// for the loads of a write.  A row whose in-edges all lie inside the chunk is
// written by this warp alone; the chunk's first and last row may be shared with
// the neighbouring chunks and are lowered with an atomic minimum.  An improved
// row records the iteration in stamp, the set a following push iteration starts
// from.
constexpr int kSpullVec = 4;                   // consecutive in-edges per lane and step
constexpr int kSpullStep = 32 * kSpullVec;     // in-edges per warp and step
static_assert(kSpullStep == 128, "a step's row starts fit four 32-bit words, one per group of eight lanes");
// Finished rows wait in a ring of kSpullRing (row entry, minimum) pairs: fewer than
// 32 are left after a write-out and one step adds at most kSpullStep.
constexpr int kSpullRing = 256;
static_assert(kSpullRing >= 31 + kSpullStep && (kSpullRing & (kSpullRing - 1)) == 0, "pull ring size");

struct SpullSmem {
    uint32_t occ[4];            // row starts of the step, one bit per edge
    int2 ring[kSpullRing];      // finished rows: (entry, or ~entry when shared; minimum's bits)
};

// Lowers the distance of row entry kr to m, the row's minimum over this warp's
// part of its in-edges.  own: no other thread writes that row.
__device__ __forceinline__ void sssp_pull_commit(const SsspArgs& a, int32_t L, int32_t kr, float m, bool own,
                                                 Acc& acc) {
    const int32_t row = __ldg(a.nzr + kr);
    if (!(m < a.dist[row])) return;  // distances only fall: nothing to lower
    if (own) {
        a.dist[row] = m;
        a.stamp[row] = L + 1;
        acc.n_new += 1;
    } else {
        const float prev = atomic_min_f32(a.dist + row, m);
        if (m < prev && atomicMax(a.stamp + row, L + 1) < L + 1) acc.n_new += 1;
    }
}

// binary32 <-> an unsigned key with the same order (for a warp-wide integer minimum)
__device__ __forceinline__ uint32_t f32_order_key(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float f32_from_order_key(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The in-edge columns and weights of a lane's kSpullVec edges from es (none at or past e1).
__device__ __forceinline__ void sssp_pull_load(const SsspArgs& a, int32_t es, int32_t e1, bool full, int4& c4,
                                               float4& w4) {
    if (full) {
        c4 = __ldcs(reinterpret_cast<const int4*>(a.in_col + es));
        w4 = __ldcs(reinterpret_cast<const float4*>(a.in_val + es));
    } else {
        c4.x = es + 0 < e1 ? __ldcs(a.in_col + es + 0) : 0;
        c4.y = es + 1 < e1 ? __ldcs(a.in_col + es + 1) : 0;
        c4.z = es + 2 < e1 ? __ldcs(a.in_col + es + 2) : 0;
        c4.w = es + 3 < e1 ? __ldcs(a.in_col + es + 3) : 0;
        w4.x = es + 0 < e1 ? __ldcs(a.in_val + es + 0) : 0.0f;
        w4.y = es + 1 < e1 ? __ldcs(a.in_val + es + 1) : 0.0f;
        w4.z = es + 2 < e1 ? __ldcs(a.in_val + es + 2) : 0.0f;
        w4.w = es + 3 < e1 ? __ldcs(a.in_val + es + 3) : 0.0f;
    }
}

// Queues the finished row (entry kr, minimum m) of each lane with `take` (all lanes call).
__device__ __forceinline__ void sssp_pull_queue(SpullSmem& sm, uint32_t& tail, bool take, int32_t kr, bool own,
                                                float m) {
    const uint32_t b = __ballot_sync(0xffffffffu, take);
    if (take)
        sm.ring[(tail + __popc(b & lanemask_lt())) & (kSpullRing - 1)] =
            make_int2(own ? kr : ~kr, __float_as_int(m));
    tail += __popc(b);
}

// Writes the queued rows out, 32 at a time, while at least `least` are queued
// (least = 1: all of them).
__device__ __forceinline__ void sssp_pull_drain(const SsspArgs& a, int32_t L, SpullSmem& sm, uint32_t& head,
                                                uint32_t tail, uint32_t least, Acc& acc) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    while (tail - head >= least) {
        if ((uint32_t)lane < tail - head) {
            const int2 e = sm.ring[(head + lane) & (kSpullRing - 1)];
            sssp_pull_commit(a, L, e.x >= 0 ? e.x : ~e.x, __int_as_float(e.y), e.x >= 0, acc);
        }
        head += tail - head < 32u ? tail - head : 32u;
    }
    __syncwarp();
}

// sm: this warp's shared scratch, occ zero on entry and on return.
__device__ __forceinline__ void sssp_pull(const SsspArgs& a, int32_t L, SpullSmem& sm, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kSsspThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kSsspThreads) >> 5);
    const int32_t E = a.nnz;
    int32_t chunk = (int32_t)(((long long)E + nwarps - 1) / nwarps);
    chunk = chunk < kSpullStep ? kSpullStep : ((chunk + kSpullStep - 1) / kSpullStep) * kSpullStep;
    for (long long e0l = (long long)gwarp * chunk; e0l < E; e0l += (long long)nwarps * chunk) {
        const int32_t e0 = (int32_t)e0l;
        const int32_t e1 = E - e0 > chunk ? e0 + chunk : E;
        PushCursorT<kSpullVec> cur_;
        cur_.k = warp_find_entry(a.nzr_ptr, a.nnzr, e0);
        cur_.wlast = -1;
        const int32_t k_first = cur_.k;  // the chunk's first row: may have in-edges before e0
        int32_t ckey = -1;               // the open row carried from the last step (entry), its minimum
        float cmin = INFINITY;
        uint32_t head = 0, tail = 0;     // ring positions (same in every lane)
        int4 c4;
        float4 w4;
        sssp_pull_load(a, e0 + kSpullVec * lane, e1, e1 - e0 >= kSpullStep, c4, w4);
        for (int32_t base = e0; base < e1; base += kSpullStep) {
            const int32_t k0 = cur_.k;  // entry of edge base - 1 (of e0 in the first step)
            const int32_t es = base + kSpullVec * lane;  // this lane's first edge
            // candidates d[j] + w(j, i) of this step; the next step's edges are loaded meanwhile
            float x0 = es + 0 < e1 ? a.dist[c4.x] + w4.x : INFINITY;
            const float x1 = es + 1 < e1 ? a.dist[c4.y] + w4.y : INFINITY;
            const float x2 = es + 2 < e1 ? a.dist[c4.z] + w4.z : INFINITY;
            const float x3 = es + 3 < e1 ? a.dist[c4.w] + w4.w : INFINITY;
            if (base + kSpullStep < e1)
                sssp_pull_load(a, es + kSpullStep, e1, e1 - base - kSpullStep >= kSpullStep, c4, w4);
            // row starts in the step: bit j of word m set iff a row starts at edge base + 32 m + j
            // (none at or past e1, so that slots past e1 stay in the chunk's last row)
            if (cur_.wlast <= base + kSpullStep - 1) {
#pragma unroll
                for (int t = 0; t < kSpullVec; ++t) {
                    const int32_t wi = cur_.k + 1 + lane + 32 * t;
                    cur_.wv[t] = wi < a.nnzr ? __ldg(a.nzr_ptr + wi) : INT32_MAX;
                }
                cur_.wlast = __shfl_sync(0xffffffffu, cur_.wv[kSpullVec - 1], 31);
            }
#pragma unroll
            for (int t = 0; t < kSpullVec; ++t) {
                const int32_t rel = cur_.wv[t] - base;  // wv <= INT32_MAX, base >= 0: no overflow
                if (rel >= 0 && rel < kSpullStep && base + rel < e1) atomicOr(sm.occ + (rel >> 5), 1u << (rel & 31));
            }
            __syncwarp();
            const uint4 o4 = *reinterpret_cast<const uint4*>(sm.occ);
            __syncwarp();
            if (lane < 4) sm.occ[lane] = 0u;
            __syncwarp();  // the words are clear before any lane's next step sets bits in them
            const uint32_t p0 = __popc(o4.x), p1 = __popc(o4.y), p2 = __popc(o4.z), p3 = __popc(o4.w);
            cur_.k = k0 + (int32_t)(p0 + p1 + p2 + p3);
            // this lane's edges es .. es + 3: where rows start among them, the rows before them
            const int grp = lane >> 3;
            const int sh = (lane & 7) * kSpullVec;
            const uint32_t before_grp = grp == 0 ? 0u : (grp == 1 ? p0 : (grp == 2 ? p0 + p1 : p0 + p1 + p2));
            const uint32_t word = (grp & 2) ? ((grp & 1) ? o4.w : o4.z) : ((grp & 1) ? o4.y : o4.x);
            const uint32_t bits = (word >> sh) & ((1u << kSpullVec) - 1u);
            const bool b0 = bits & 1u, b1 = (bits >> 1) & 1u, b2 = (bits >> 2) & 1u, b3 = (bits >> 3) & 1u;
            const int32_t kk_s = k0 + (int32_t)(before_grp + __popc(word & ((1u << sh) - 1u)) + (b0 ? 1u : 0u));
            const int32_t kk_e = kk_s + (int32_t)b1 + (int32_t)b2 + (int32_t)b3;  // row of the lane's last edge
            const int32_t nv = e1 - es;
            acc.exam += nv <= 0 ? 0u : (nv >= kSpullVec ? (uint32_t)kSpullVec : (uint32_t)nv);
            // minimum of the run ending at each edge (lane 0 continues the carried row)
            if (lane == 0 && ckey >= 0 && !b0) x0 = fminf(x0, cmin);
            const float s0 = x0;
            const float s1 = b1 ? x1 : fminf(s0, x1);
            const float s2 = b2 ? x2 : fminf(s1, x2);
            const float s3 = b3 ? x3 : fminf(s2, x3);
            // the minimum of each row's open runs over the lanes that end in it (they are adjacent)
            const uint32_t same = __match_any_sync(0xffffffffu, kk_e);
            const float gmin = f32_from_order_key(__reduce_min_sync(same, f32_order_key(s3)));
            float in_min = __shfl_up_sync(0xffffffffu, gmin, 1);
            if (lane == 0) in_min = cmin;
            // rows finished here: the row before the lane (it ended at the border), and the rows
            // ending at edges 0, 1, 2; the first of those takes the earlier lanes' runs when it
            // entered from them
            const bool enter = lane > 0 && !b0;
            sssp_pull_queue(sm, tail, b0 && (lane > 0 || ckey >= 0), kk_s - 1, kk_s - 1 != k_first, in_min);
            sssp_pull_queue(sm, tail, b1, kk_s, kk_s != k_first, enter ? fminf(s0, in_min) : s0);
            const int32_t k1 = kk_s + (int32_t)b1;
            sssp_pull_queue(sm, tail, b2, k1, k1 != k_first, enter && !b1 ? fminf(s1, in_min) : s1);
            const int32_t k2 = k1 + (int32_t)b2;
            sssp_pull_queue(sm, tail, b3, k2, k2 != k_first, enter && !b1 && !b2 ? fminf(s2, in_min) : s2);
            ckey = __shfl_sync(0xffffffffu, kk_e, 31);
            cmin = __shfl_sync(0xffffffffu, gmin, 31);
            if (tail - head >= 32u) sssp_pull_drain(a, L, sm, head, tail, 32u, acc);
        }
        // the chunk's last row: its in-edges may continue in the next chunk
        sssp_pull_queue(sm, tail, lane == 0 && ckey >= 0, ckey, false, cmin);
        sssp_pull_drain(a, L, sm, head, tail, 1u, acc);
    }
}

// The rows a pull iteration improved (stamp = iteration + 1) as the next push queue.
__device__ __forceinline__ void sssp_stamp_to_queue(const SsspArgs& a, int32_t L, Stage& st) {
    const int lane = threadIdx.x & 31;
    const long long gwarp = (long long)((blockIdx.x * kSsspThreads + threadIdx.x) >> 5);
    const long long nwarps = (long long)((gridDim.x * kSsspThreads) >> 5);
    for (long long b = gwarp * 32; b < a.n; b += nwarps * 32) {
        const int32_t v = (int32_t)b + lane;
        st.put(v < a.n && a.stamp[v] == L + 1, v);
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
    __shared__ __align__(16) SpullSmem pull_sm[kSsspThreads / 32];
    const int wib = threadIdx.x >> 5;
    if ((threadIdx.x & 31) < 4) pull_sm[wib].occ[threadIdx.x & 31] = 0u;
    __syncwarp();
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
            sssp_pull(a, L, pull_sm[wib], acc);
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
            sssp_stamp_to_queue(a, L, st);
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
    a.nzr = G->nzr_in;
    a.nzr_ptr = G->nzr_in_ptr;
    a.nnzr = G->nnzr_in;
    a.nnz = (int32_t)G->nnz;
    a.dist = dist;
    a.stamp = w.list;  // n ints
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
