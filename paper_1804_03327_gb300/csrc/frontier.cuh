// Frontier machinery shared by the single-source and the batched BFS kernels:
// per-level counters, the staged frontier queue with its out-degree prefix, and
// the edge-balanced cursor that walks a queue's edges.
#pragma once

#include "gbx_internal.cuh"

#ifndef GBX_PUSH_ILP
#define GBX_PUSH_ILP 2
#endif

namespace gbx {

constexpr int kPushIlp = GBX_PUSH_ILP;  // edges per lane per push step (independent chains)
constexpr int kPushStep = 32 * kPushIlp;

// One thread's counts of a level (each stays below 2^32: a level finds at most n
// vertices and examines at most nnz < 2^31 entries); blocks add them up in 64 bits.
struct Acc {
    uint32_t n_new = 0, mf = 0, indeg = 0, exam = 0;
};

// Next-frontier appends are staged per warp in shared memory and published
// kStage at a time: one packed 64-bit atomic reserves both the queue slots
// (low 32 bits) and the matching range of the out-degree prefix (high 32
// bits), so the prefix stays ascending in queue order and the queue needs no
// separate scan.  Staging keeps same-address atomics on the level counter to
// one per kStage discovered vertices.
constexpr int kStage = 128;
struct StageBuf {
    int32_t v[kStage];
};

struct Stage {
    StageBuf* sb;
    int cnt;  // warp-uniform
    LevelCtr* cout;
    int32_t* nq;
    int32_t* nqp;
    int32_t* nqd;
    const int32_t* out_ptr;
    const int32_t* in_ptr;
    int count_degrees;  // add the staged vertices' degrees to acc (push levels)
    int need_indeg;
    Acc* acc;

    // Publish the staged vertices: their row offsets are loaded here, all at once
    // (off the per-edge critical path); vertices without out-edges are counted
    // but not queued, so every queue entry owns at least one edge.
    __device__ __forceinline__ void flush() {
        if (cnt == 0) return;
        __syncwarp();
        const int lane = threadIdx.x & 31;
        constexpr int R = kStage / 32;
        int32_t v[R], rs[R], od[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int idx = t * 32 + lane;
            v[t] = idx < cnt ? sb->v[idx] : -1;
        }
#pragma unroll
        for (int t = 0; t < R; ++t) {
            rs[t] = v[t] >= 0 ? __ldg(out_ptr + v[t]) : 0;
            od[t] = v[t] >= 0 ? __ldg(out_ptr + v[t] + 1) - rs[t] : 0;
        }
        if (count_degrees) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                acc->mf += (uint32_t)od[t];
                if (need_indeg)
                    acc->indeg += v[t] >= 0 ? (uint32_t)(__ldg(in_ptr + v[t] + 1) - __ldg(in_ptr + v[t])) : 0u;
                else
                    acc->indeg += (uint32_t)od[t];
            }
        }
        uint32_t keep[R];
        uint32_t nkeep = 0, sum = 0;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            keep[t] = __ballot_sync(0xffffffffu, od[t] > 0);
            nkeep += __popc(keep[t]);
            sum += (uint32_t)od[t];
        }
        if (nkeep > 0) {
            const uint32_t tot = __reduce_add_sync(0xffffffffu, sum);
            unsigned long long old = 0;
            if (lane == 0) old = atomicAdd(&cout->q, ((unsigned long long)tot << 32) | (unsigned long long)nkeep);
            old = __shfl_sync(0xffffffffu, old, 0);
            int32_t pos = (int32_t)(uint32_t)old;
            uint32_t pre_base = (uint32_t)(old >> 32);
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const uint32_t inc = warp_inclusive_sum((uint32_t)od[t]);
                if (od[t] > 0) {
                    const int32_t p = pos + __popc(keep[t] & lanemask_lt());
                    const int32_t pre = (int32_t)(pre_base + inc - (uint32_t)od[t]);
                    nq[p] = v[t];
                    nqp[p] = pre;
                    nqd[p] = rs[t] - pre;
                }
                pos += __popc(keep[t]);
                pre_base += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        cnt = 0;
        __syncwarp();
    }

    // End-of-level publish by the whole block (every thread of the block calls it):
    // the warps' staged vertices go out with one packed atomic for the block instead
    // of one per warp, the warps' ranges placed by a scan over the block in bsm
    // (kWarps shared words that no other code touches until the next block barrier).
    template <int kWarps>
    __device__ __forceinline__ void flush_block(unsigned long long* bsm) {
        __syncwarp();
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        constexpr int R = kStage / 32;
        int32_t v[R], rs[R], od[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int idx = t * 32 + lane;
            v[t] = idx < cnt ? sb->v[idx] : -1;
        }
#pragma unroll
        for (int t = 0; t < R; ++t) {
            rs[t] = v[t] >= 0 ? __ldg(out_ptr + v[t]) : 0;
            od[t] = v[t] >= 0 ? __ldg(out_ptr + v[t] + 1) - rs[t] : 0;
        }
        if (count_degrees) {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                acc->mf += (uint32_t)od[t];
                if (need_indeg)
                    acc->indeg += v[t] >= 0 ? (uint32_t)(__ldg(in_ptr + v[t] + 1) - __ldg(in_ptr + v[t])) : 0u;
                else
                    acc->indeg += (uint32_t)od[t];
            }
        }
        uint32_t keep[R];
        uint32_t nkeep = 0, sum = 0;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            keep[t] = __ballot_sync(0xffffffffu, od[t] > 0);
            nkeep += __popc(keep[t]);
            sum += (uint32_t)od[t];
        }
        const uint32_t tot = __reduce_add_sync(0xffffffffu, sum);
        if (lane == 0) bsm[w] = ((unsigned long long)tot << 32) | (unsigned long long)nkeep;
        __syncthreads();
        if (w == 0) {
            // packed (degree sum, count) pairs add without carries: both halves stay below 2^32
            const unsigned long long own = lane < kWarps ? bsm[lane] : 0ull;
            unsigned long long x = own;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const unsigned long long total = __shfl_sync(0xffffffffu, x, 31);
            unsigned long long old = 0;
            if (lane == 0 && total) old = atomicAdd(&cout->q, total);
            old = __shfl_sync(0xffffffffu, old, 0);
            __syncwarp();
            if (lane < kWarps) bsm[lane] = old + x - own;
        }
        __syncthreads();
        const unsigned long long base = bsm[w];
        int32_t pos = (int32_t)(uint32_t)base;
        uint32_t pre_base = (uint32_t)(base >> 32);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const uint32_t inc = warp_inclusive_sum((uint32_t)od[t]);
            if (od[t] > 0) {
                const int32_t p = pos + __popc(keep[t] & lanemask_lt());
                const int32_t pre = (int32_t)(pre_base + inc - (uint32_t)od[t]);
                nq[p] = v[t];
                nqp[p] = pre;
                nqd[p] = rs[t] - pre;
            }
            pos += __popc(keep[t]);
            pre_base += __shfl_sync(0xffffffffu, inc, 31);
        }
        cnt = 0;
        __syncwarp();
    }

    // Stage the lanes with `take` (all 32 lanes call this).
    __device__ __forceinline__ void put(bool take, int32_t v) {
        const uint32_t app = __ballot_sync(0xffffffffu, take);
        if (!app) return;
        if (cnt + __popc(app) > kStage) flush();
        if (take) sb->v[cnt + __popc(app & lanemask_lt())] = v;
        cnt += __popc(app);
        __syncwarp();
    }
};

// A level's counters, added once per block.  Each warp leaves its sums in shared
// memory; after a block barrier warp 0 adds them up and thread 0 adds the block's
// totals to the global counters, one atomic per counter and block.  The counters
// of a level share one cache line, and same-line atomics serialise at one L2 slice,
// so one atomic per warp from a grid of thousands of warps costs microseconds per
// level.  Every thread of the block calls this; a null counter is skipped.  Thread
// 0 issues the atomics, so its arrival at the next grid barrier (a release) orders
// them before the barrier completes.
template <int kWarps>
__device__ __forceinline__ void block_add_counts(unsigned long long (*sm)[4], unsigned long long x0,
                                                 unsigned long long x1, unsigned long long x2, unsigned long long x3,
                                                 unsigned long long* c0, unsigned long long* c1,
                                                 unsigned long long* c2, unsigned long long* c3) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x0 = warp_sum_u64(x0);
    x1 = warp_sum_u64(x1);
    x2 = warp_sum_u64(x2);
    x3 = warp_sum_u64(x3);
    if (lane == 0) {
        sm[w][0] = x0;
        sm[w][1] = x1;
        sm[w][2] = x2;
        sm[w][3] = x3;
    }
    __syncthreads();
    if (w == 0) {
        unsigned long long y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) y[k] = warp_sum_u64(lane < kWarps ? sm[lane][k] : 0ull);
        if (lane == 0) {
            if (c0 && y[0]) atomicAdd(c0, y[0]);
            if (c1 && y[1]) atomicAdd(c1, y[1]);
            if (c2 && y[2]) atomicAdd(c2, y[2]);
            if (c3 && y[3]) atomicAdd(c3, y[3]);
        }
    }
}

// Largest k in [0, count) with qp[k] <= e (qp ascending, qp[0] = 0), found by the
// whole warp: 32 samples per round shrink the range 32-fold.
__device__ __forceinline__ int32_t warp_find_entry(const int32_t* qp, int32_t count, long long e) {
    const int lane = threadIdx.x & 31;
    int32_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const long long span = hi - lo;
        const int32_t idx = lo + (int32_t)((span * lane) >> 5);
        const uint32_t m = __ballot_sync(0xffffffffu, (long long)qp[idx] <= e);
        const int last = 31 - __clz(m);
        const int32_t nlo = lo + (int32_t)((span * last) >> 5);
        const int32_t nhi = last == 31 ? hi : lo + (int32_t)((span * (last + 1)) >> 5);
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Edges of one push step of I edges per lane: the frontier vertex u, child v and
// CSR position k (for edge values) of each lane's edges.
template <int I>
struct PushStepT {
    int32_t u[I];
    int32_t v[I];
    int32_t k[I];
};

// Walks a warp's edge range: maps edge ids to (queue entry, child) with a window
// of the next 32 * kPushIlp entry boundaries (lane holds entries k+1+lane+32t).
// Every entry has at least one edge, so the boundaries inside one step are all in
// the window; it is reloaded only once a step could reach past its last boundary.
template <int I>
struct PushCursorT {
    static constexpr int kStep = 32 * I;  // edges of one step
    int32_t k;
    int32_t wlast;
    int32_t wv[I];

    // Occupancy of the step [base, base + kStep) by entry boundaries: bit j of
    // occ[m] is set iff an entry after the cursor's starts at edge base + 32 m + j
    // (the window is reloaded first if the step could reach past it).
    __device__ __forceinline__ void occupancy(const int32_t* qp, uint32_t qcount, int32_t base, uint32_t (&occ)[I]) {
        const int lane = threadIdx.x & 31;
        if (wlast <= base + kStep - 1) {
#pragma unroll
            for (int t = 0; t < I; ++t) {
                const int32_t wi = k + 1 + lane + 32 * t;
                wv[t] = wi < (int32_t)qcount ? qp[wi] : INT32_MAX;
            }
            wlast = __shfl_sync(0xffffffffu, wv[I - 1], 31);
        }
#pragma unroll
        for (int m = 0; m < I; ++m) {
            uint32_t c = 0;
#pragma unroll
            for (int t = 0; t < I; ++t) {
                const int32_t rel = wv[t] - base;  // wv <= INT32_MAX, base >= 0: no overflow
                c |= (rel >= 32 * m && rel < 32 * (m + 1)) ? (1u << (rel - 32 * m)) : 0u;
            }
            occ[m] = __reduce_or_sync(0xffffffffu, c);
        }
    }

    // Maps the edges [base, base + kStep) of one step (lane t-th slot: edge
    // base + 32 t + lane) to their queue entries and loads each edge's frontier
    // vertex u (-1 at or past e1) and d = (row start - prefix) of its entry, so that
    // the edge's CSR position is e + d.  The loads are issued, not waited for.
    __device__ __forceinline__ void map(const int32_t* q, const int32_t* qp, const int32_t* qd, uint32_t qcount,
                                        int32_t base, int32_t e1, int32_t (&u)[I], int32_t (&d)[I]) {
        const int lane = threadIdx.x & 31;
        uint32_t occ[I];
        occupancy(qp, qcount, base, occ);
        uint32_t before = 0;
#pragma unroll
        for (int t = 0; t < I; ++t) {
            const int32_t kk = k + (int32_t)(before + __popc(occ[t] & (0xffffffffu >> (31 - lane))));
            before += __popc(occ[t]);
            const int32_t e = base + 32 * t + lane;
            u[t] = -1;
            d[t] = 0;
            if (e < e1) {
                u[t] = q[kk];
                d[t] = qd[kk];
            }
        }
        k += (int32_t)before;
    }

    // As map, for the step right after another step of the same walk whose last
    // slot (lane 31, slot I - 1) held entry values (u_last, d_last): a step with no
    // entry boundary in it belongs wholly to that entry and needs no loads (the
    // heavy push levels of a power-law graph walk a few long rows).
    __device__ __forceinline__ void map_after(const int32_t* q, const int32_t* qp, const int32_t* qd, uint32_t qcount,
                                              int32_t base, int32_t e1, int32_t u_last, int32_t d_last,
                                              int32_t (&u)[I], int32_t (&d)[I]) {
        const int lane = threadIdx.x & 31;
        uint32_t occ[I];
        occupancy(qp, qcount, base, occ);
        uint32_t any = 0u;
#pragma unroll
        for (int t = 0; t < I; ++t) any |= occ[t];
        if (any == 0u) {
#pragma unroll
            for (int t = 0; t < I; ++t) {
                const bool ok = base + 32 * t + lane < e1;
                u[t] = ok ? u_last : -1;
                d[t] = ok ? d_last : 0;
            }
            return;
        }
        uint32_t before = 0;
#pragma unroll
        for (int t = 0; t < I; ++t) {
            const int32_t kk = k + (int32_t)(before + __popc(occ[t] & (0xffffffffu >> (31 - lane))));
            before += __popc(occ[t]);
            const int32_t e = base + 32 * t + lane;
            u[t] = -1;
            d[t] = 0;
            if (e < e1) {
                u[t] = q[kk];
                d[t] = qd[kk];
            }
        }
        k += (int32_t)before;
    }

    // The entry of each lane's edge slots of the step [base, base + kStep) (qp must
    // be strictly ascending: no entry without edges); the cursor moves on to the
    // entry of the step's last edge.  A slot at or past the end of the last entry's
    // edges maps to the last entry.
    __device__ __forceinline__ void locate(const int32_t* qp, uint32_t qcount, int32_t base, int32_t (&kk)[I]) {
        const int lane = threadIdx.x & 31;
        uint32_t occ[I];
        occupancy(qp, qcount, base, occ);
        uint32_t before = 0;
#pragma unroll
        for (int t = 0; t < I; ++t) {
            kk[t] = k + (int32_t)(before + __popc(occ[t] & (0xffffffffu >> (31 - lane))));
            before += __popc(occ[t]);
        }
        k += (int32_t)before;
    }

    __device__ __forceinline__ PushStepT<I> gather(const int32_t* out_col, const int32_t* q, const int32_t* qp,
                                               const int32_t* qd, uint32_t qcount, int32_t base, int32_t e1) {
        const int lane = threadIdx.x & 31;
        int32_t u[I], d[I];
        map(q, qp, qd, qcount, base, e1, u, d);
        PushStepT<I> st;
#pragma unroll
        for (int t = 0; t < I; ++t) {
            st.u[t] = u[t];
            st.k[t] = u[t] >= 0 ? base + 32 * t + lane + d[t] : 0;
            st.v[t] = u[t] >= 0 ? __ldg(out_col + st.k[t]) : 0;
        }
        return st;
    }
};


using PushStep = PushStepT<kPushIlp>;
using PushCursor = PushCursorT<kPushIlp>;

}  // namespace gbx
