// Batched multi-source BFS: S sources at once as bit lanes (Algorithm 1 run for
// S frontier vectors together), with the Boolean semiring acting lane-wise on
// uint64 words (OR = bitwise OR, AND = bitwise AND).  Lane b of vertex v is
// bit b % 64 of word b / 64 of v's W-word row.
//
// State (vertex-major, W words per vertex, W padded to a multiple of the chunk):
//   V[v]      lanes in which v has been visited,
//   F_k[v]    lanes in which v was found at level L (k = L mod 3): level L reads
//             F_{L mod 3} of its active list, writes F_{(L+1) mod 3}, and clears
//             F_{(L+2) mod 3} for the list of level L - 1 (read one level earlier,
//             written again one level later), so no extra barrier is needed;
//   D         one bit per vertex: every lane visited (pull skips it without loads);
//   T_k       one bit per vertex: listed for level L + 1 (W > 1), rotating like F.
// Each level runs in the direction chosen for the whole batch:
//   push (Eq 5 lane-wise): the active list's edges are split evenly over warps.
//     One word per vertex (S <= 64): each edge claims the lanes F[u] & ~V[v] with a
//     64-bit atomicOr on V[v]; the lanes it gained are new (unique claimant): their
//     depth is written, they are ORed into F_next[v], and the first claimant of v
//     lists it -- one phase.  Wider batches: each edge ORs F[u] & ~V[v] into
//     F_next[v] with reductions and lists v once; after a grid barrier a finalising
//     pass over the touched vertices keeps new = F_next & ~V, sets V |= new and
//     writes the depths (one returning atomic per word and edge would cost more).
//   pull (Eq 4 lane-wise, masking + early exit + operand reuse): every vertex with
//     an unvisited lane ORs V of its in-neighbours (V is the state before this
//     level) and stops as soon as every unvisited lane is covered; new = acc & ~V.
// New lanes get depth L + 1.  Depths are not stored as they are found (2-byte
// stores scattered over S rows leave partial sectors that are evicted and merged
// again level after level): a depth below 16 is recorded as bits in four per-vertex
// planes of lane words (plane p holds bit p), larger ones are stored at once, and
// after the last level one pass emits every other entry of the S rows exactly once,
// coalesced along the vertices (-1 where a lane never arrived).
#include "frontier.cuh"
#include "gbx_internal.cuh"

namespace gbx {

constexpr int kMsThreads = 512;
// Register budgets of the persistent batched kernel: the default build fits two
// 512-thread blocks on an SM (64 registers a thread: twice the resident warps of an
// unbounded build at 114, for 24-222 bytes of spills), the lean build three (40
// registers, more spills; lane words 1 and 2 only).  Lean pays on graphs with few
// wide levels and loses on long chains of small ones (a grid), so a descriptor
// chooses it (blocks_per_sm >= 3) and the autotuner times both.
constexpr int kMsOcc = 2;
constexpr int kMsOccLean = 3;
constexpr int kMsProbe = 8;  // default in-neighbours a lane scans alone before the warp takes over
constexpr int kMsPlanes = 4;  // depth bit planes: bit p of depths below 16

struct MsArgs {
    int32_t n, S, W, nwords;
    long long nnz;
    const int32_t* out_ptr;
    const int32_t* out_col;
    const int32_t* in_ptr;
    const int32_t* in_col;
    const uint32_t* nz_in;
    unsigned long long* V;
    unsigned long long* Fb[3];  // rotating found-lane buffers
    unsigned long long* P[4];   // depth bit planes (see record_depth)
    uint32_t* D;                // all lanes visited
    uint32_t* Tb[3];            // rotating "listed" bitmaps
    int32_t* tlist;             // vertices touched by a wide push level
    void* depth;        // [S][n], used when rows is NULL
    void* const* rows;  // optional: lane b writes its n depths to rows[b]
    int depth16;
    const int32_t* src;
    int32_t* ids[3];  // active lists, rotating like Fb
    int32_t* qp[2];
    int32_t* qd[2];
    LevelCtr* ctr;
    GridBar* bar;
    unsigned int bar_parity;
    LevelRec* trace;
    int32_t* status;
    float alpha;
    int32_t mode, trace_cap, symmetric, probe;
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long lane_mask(int32_t S, int32_t w) {
    const int32_t lo = w * 64;
    if (lo + 64 <= S) return ~0ull;
    if (lo >= S) return 0ull;
    return (1ull << (S - lo)) - 1ull;
}

__device__ __forceinline__ void store_depth(const MsArgs& a, int32_t lane_b, int32_t v, int32_t d) {
    if (a.rows) {
        if (a.depth16)
            static_cast<int16_t*>(a.rows[lane_b])[v] = (int16_t)d;
        else
            static_cast<int32_t*>(a.rows[lane_b])[v] = d;
        return;
    }
    const size_t idx = (size_t)lane_b * (size_t)a.n + (size_t)v;
    if (a.depth16)
        static_cast<int16_t*>(a.depth)[idx] = (int16_t)d;
    else
        static_cast<int32_t*>(a.depth)[idx] = d;
}

// Records depth d for the lanes nw of word w of vertex v.  Depths below 16 go to
// the bit planes (atomically when several edges may record lanes of one word in the
// same level, as the one-phase push does); larger ones are stored now.  A visited
// lane with no plane bit is either its own source (depth 0) or such a deep one,
// which the emission pass tells apart by the source.
__device__ __forceinline__ void record_depth(const MsArgs& a, int32_t v, int32_t w, unsigned long long nw, int32_t d,
                                             bool atomic) {
    if (!nw) return;
    if (d < 16) {
        const size_t iv = (size_t)v * a.W + w;
#pragma unroll
        for (int p = 0; p < kMsPlanes; ++p) {
            if (!((d >> p) & 1)) continue;
            if (atomic)
                atomicOr(a.P[p] + iv, nw);
            else
                a.P[p][iv] |= nw;
        }
        return;
    }
    unsigned long long m = nw;
    while (m) {
        const int b = __ffsll((long long)m) - 1;
        m &= m - 1;
        store_depth(a, w * 64 + b, v, d);
    }
}

// After the last level: every (lane, vertex) entry of the output rows, once.  A warp
// takes 32 consecutive vertices and one lane word; for each of the word's lanes the 32
// entries are one coalesced store.  Lanes never visited get -1; lanes found at depth
// 16 or more were stored when found and are left alone.
__device__ __forceinline__ void emit_depths(const MsArgs& a) {
    const int lane = threadIdx.x & 31;
    const long long gwarp = ((long long)blockIdx.x * kMsThreads + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * kMsThreads) >> 5;
    const int32_t nvb = (a.n + 31) >> 5;
    const int32_t wl = (a.S + 63) >> 6;  // words holding real lanes
    const long long items = (long long)nvb * wl;
    for (long long it = gwarp; it < items; it += nwarps) {
        const int32_t vb = (int32_t)(it / wl), w = (int32_t)(it - (long long)vb * wl);
        const int32_t v = (vb << 5) + lane;
        const bool ok = v < a.n;
        const size_t iv = (size_t)(ok ? v : 0) * a.W + w;
        const unsigned long long vis = ok ? a.V[iv] : 0ull;
        const unsigned long long p0 = ok ? a.P[0][iv] : 0ull, p1 = ok ? a.P[1][iv] : 0ull;
        const unsigned long long p2 = ok ? a.P[2][iv] : 0ull, p3 = ok ? a.P[3][iv] : 0ull;
        const unsigned long long any = p0 | p1 | p2 | p3;
        const int nb = a.S - w * 64 < 64 ? a.S - w * 64 : 64;
        for (int b = 0; b < nb; ++b) {
            if (!ok) continue;
            int32_t d = -1;
            if ((vis >> b) & 1ull) {
                if (!((any >> b) & 1ull) && __ldg(a.src + w * 64 + b) != v) continue;  // deep: already stored
                d = (int32_t)(((p0 >> b) & 1ull) | (((p1 >> b) & 1ull) << 1) | (((p2 >> b) & 1ull) << 2) |
                              (((p3 >> b) & 1ull) << 3));
            }
            store_depth(a, w * 64 + b, v, d);
        }
    }
}

// ---------------------------------------------------------------- pull level

template <int CW>
__device__ __forceinline__ void ms_pull(const MsArgs& a, int32_t L, unsigned long long* Fn, Stage& st, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kMsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kMsThreads) >> 5);
    const int32_t ntiles = (a.n + 31) >> 5;
    for (int32_t tile = gwarp; tile < ntiles; tile += nwarps) {
        const int32_t v = (tile << 5) + lane;
        const uint32_t todo = v < a.n ? (a.nz_in[tile] & ~a.D[tile]) : 0u;
        if (__ballot_sync(0xffffffffu, (todo >> lane) & 1u) == 0u) continue;
        const bool mine = (todo >> lane) & 1u;
        int32_t beg = 0, end = 0;
        bool sink = false;
        if (mine) {
            beg = __ldg(a.in_ptr + v);
            end = __ldg(a.in_ptr + v + 1);
            sink = !a.symmetric && __ldg(a.out_ptr + v + 1) == __ldg(a.out_ptr + v);
        }
        // A vertex without out-edges is nobody's in-neighbour, so no other row reads
        // its V during this level: its new lanes are committed in place (it never
        // joins the active list, which holds vertices with out-edges only).
        bool any_new = false, full = true;
        for (int32_t c = 0; c < a.W; c += CW) {
            unsigned long long unv[CW], accw[CW];
            bool pend = false;
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                unv[j] = mine ? (~a.V[(size_t)v * a.W + c + j] & lane_mask(a.S, c + j)) : 0ull;
                accw[j] = 0ull;
                pend |= unv[j] != 0ull;
            }
            unsigned long long exam = 0;
            // lane probes: up to a.probe in-neighbours, two loads in flight
            int32_t k = beg;
            bool covered = !pend;
            const int32_t lim = end < beg + a.probe ? end : beg + a.probe;
            while (!covered && k < lim) {
                const bool two = k + 1 < lim;
                const int32_t u0 = __ldg(a.in_col + k);
                const int32_t u1 = two ? __ldg(a.in_col + k + 1) : u0;
                covered = true;
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    accw[j] |= a.V[(size_t)u0 * a.W + c + j] | a.V[(size_t)u1 * a.W + c + j];
                    covered &= (accw[j] & unv[j]) == unv[j];
                }
                k += two ? 2 : 1;
                exam += two ? 2u : 1u;
            }
            // long rows: the whole warp ORs 32 in-neighbours at a time and stops once
            // every unvisited lane of the chunk is covered (warp OR-reduction)
            uint32_t wpend = __ballot_sync(0xffffffffu, !covered && k < end);
            while (wpend) {
                const int t = __ffs(wpend) - 1;
                wpend &= wpend - 1;
                const int32_t kt = __shfl_sync(0xffffffffu, k, t);
                const int32_t et = __shfl_sync(0xffffffffu, end, t);
                unsigned long long ut[CW], wa[CW];
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    ut[j] = __shfl_sync(0xffffffffu, unv[j], t);
                    wa[j] = __shfl_sync(0xffffffffu, accw[j], t);
                }
                unsigned long long tx = 0;
                for (int32_t kk = kt; kk < et; kk += 32) {
                    const int32_t idx = kk + lane;
                    unsigned long long x[CW];
                    if (idx < et) {
                        const int32_t u = __ldg(a.in_col + idx);
#pragma unroll
                        for (int j = 0; j < CW; ++j) x[j] = a.V[(size_t)u * a.W + c + j];
                    } else {
#pragma unroll
                        for (int j = 0; j < CW; ++j) x[j] = 0ull;
                    }
                    bool cov = true;
#pragma unroll
                    for (int j = 0; j < CW; ++j) {
                        const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)x[j]);
                        const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(x[j] >> 32));
                        wa[j] |= ((unsigned long long)hi << 32) | lo;
                        cov &= (wa[j] & ut[j]) == ut[j];
                    }
                    tx += (unsigned long long)(et - kk < 32 ? et - kk : 32);
                    if (cov) break;
                }
                if (lane == t) {
#pragma unroll
                    for (int j = 0; j < CW; ++j) accw[j] = wa[j];
                    exam += tx;
                }
            }
            acc.exam += exam;
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const unsigned long long nw = accw[j] & unv[j];
                if (mine) Fn[(size_t)v * a.W + c + j] = nw;
                if (sink) {
                    a.V[(size_t)v * a.W + c + j] |= nw;
                    full &= unv[j] == nw;
                }
                any_new |= nw != 0ull;
                acc.n_new += (uint32_t)__popcll(nw);
                if (mine) record_depth(a, v, c + j, nw, L + 1, false);
            }
        }
        if (sink && full) atomicOr(a.D + (v >> 5), 1u << (v & 31));
        st.put(any_new && !sink, v);
    }
    st.flush();
}

// V |= F for the vertices found by the pull level; mark vertices with all lanes visited.
template <int CW>
__device__ __forceinline__ void ms_pull_commit(const MsArgs& a, const int32_t* list, uint32_t count,
                                               const unsigned long long* Fn) {
    const long long gtid = (long long)blockIdx.x * kMsThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kMsThreads;
    for (long long k = gtid; k < count; k += gstride) {
        const int32_t v = list[k];
        bool full = true;
        for (int32_t w = 0; w < a.W; ++w) {
            const unsigned long long x = a.V[(size_t)v * a.W + w] | Fn[(size_t)v * a.W + w];
            a.V[(size_t)v * a.W + w] = x;
            full &= (x & lane_mask(a.S, w)) == lane_mask(a.S, w);
        }
        if (full) atomicOr(a.D + (v >> 5), 1u << (v & 31));
    }
}

// ---------------------------------------------------------------- push level

// One phase: each edge (u, v) of the active list claims the lanes F_cur[u] & ~V[v]
// with an atomicOr on V[v]; the lanes it gained (not set before) are new at level
// L + 1 and this edge is their only claimant, so it writes their depth and ORs them
// into F_next[v]; the first edge to gain anything at v lists v (for W == 1 the
// previous F_next word tells, otherwise the T_next bit).  One-word batches claim
// without probing V[v] first (a dependent load per edge costs more than the extra
// atomics); wider ones probe, which only saves reductions (bits are only ever set).
template <int CW>
__device__ __forceinline__ void ms_push(const MsArgs& a, int32_t L, const int32_t* q, const int32_t* qp,
                                        const int32_t* qd, uint32_t qcount, uint32_t qedges,
                                        const unsigned long long* Fc, unsigned long long* Fn, uint32_t* Tn, Stage& st,
                                        Acc& acc) {
    const int gwarp = (int)((blockIdx.x * kMsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kMsThreads) >> 5);
    const int32_t E = (int32_t)qedges;
    const unsigned long long full0 = lane_mask(a.S, 0);
    int32_t chunk = (int32_t)(((long long)E + nwarps - 1) / nwarps);
    chunk = chunk < kPushStep ? kPushStep : ((chunk + kPushStep - 1) / kPushStep) * kPushStep;
    for (long long e0l = (long long)gwarp * chunk; e0l < E; e0l += (long long)nwarps * chunk) {
        const int32_t e0 = (int32_t)e0l;
        const int32_t e1 = E - e0 > chunk ? e0 + chunk : E;
        PushCursor cur_;
        cur_.k = warp_find_entry(qp, (int32_t)qcount, e0);
        cur_.wlast = -1;
        for (int32_t base = e0; base < e1; base += kPushStep) {
            const PushStep ps = cur_.gather(a.out_col, q, qp, qd, qcount, base, e1);
#pragma unroll
            for (int t = 0; t < kPushIlp; ++t) {
                const int32_t u = ps.u[t], v = ps.v[t];
                bool first = false;
                if (CW > 1 && u >= 0 && !((a.D[v >> 5] >> (v & 31)) & 1u)) {
                    // wide batch: accumulate, finalised after the barrier
                    bool touched = false;
                    for (int32_t c = 0; c < a.W; c += CW) {
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            const size_t iu = (size_t)u * a.W + c + j, iv = (size_t)v * a.W + c + j;
                            const unsigned long long cand = Fc[iu] & ~a.V[iv];
                            if (cand) {
                                atomicOr(Fn + iv, cand);  // result unused: a reduction
                                touched = true;
                            }
                        }
                    }
                    if (touched) first = !(atomicOr(Tn + (v >> 5), 1u << (v & 31)) & (1u << (v & 31)));
                } else if (CW == 1 && u >= 0 && !((a.D[v >> 5] >> (v & 31)) & 1u)) {
                    bool any = false;
                    for (int32_t c = 0; c < a.W; c += CW) {
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            const size_t iu = (size_t)u * a.W + c + j, iv = (size_t)v * a.W + c + j;
                            const unsigned long long cand = Fc[iu];
                            if (!cand) continue;
                            const unsigned long long old = atomicOr(a.V + iv, cand);
                            const unsigned long long gained = cand & ~old;
                            if (!gained) continue;
                            if (a.W == 1) {
                                first |= atomicOr(Fn + iv, gained) == 0ull;
                                if (((old | cand) & full0) == full0) atomicOr(a.D + (v >> 5), 1u << (v & 31));
                            } else {
                                atomicOr(Fn + iv, gained);  // result unused: a reduction; T_next lists v
                            }
                            any = true;
                            acc.n_new += (uint32_t)__popcll(gained);
                            record_depth(a, v, c + j, gained, L + 1, true);
                        }
                    }
                    (void)any;
                }
                if (CW == 1) {
                    st.put(first, v);
                } else {
                    // warp-aggregated append to the touched list
                    const int lane = threadIdx.x & 31;
                    const uint32_t m = __ballot_sync(0xffffffffu, first);
                    if (m) {
                        unsigned long long base_pos = 0;
                        if (lane == 0) base_pos = atomicAdd(&st.cout->list, (unsigned long long)__popc(m));
                        base_pos = __shfl_sync(0xffffffffu, base_pos, 0);
                        if (first) a.tlist[base_pos + __popc(m & lanemask_lt())] = v;
                    }
                }
            }
        }
    }
    if (CW == 1) st.flush();
}

// Wide push levels, after the barrier: new = F_next & ~V for the touched vertices;
// V |= new, F_next = new, depth, "all lanes" map; the touched ones with new lanes
// form the next active list.  Every T_next bit belongs to a touched vertex, so the
// words are cleared whole (racing writers all store zero).
template <int CW>
__device__ __forceinline__ void ms_push_finalize(const MsArgs& a, int32_t L, uint32_t count, unsigned long long* Fn,
                                                 uint32_t* Tn, Stage& st, Acc& acc) {
    const long long gtid = (long long)blockIdx.x * kMsThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kMsThreads;
    const long long rounds = ((long long)count + gstride - 1) / gstride;
    for (long long r = 0; r < rounds; ++r) {  // warp-uniform trip count: st.put needs all lanes
        const long long k = r * gstride + gtid;
        const bool mine = k < count;
        const int32_t v = mine ? a.tlist[k] : 0;
        bool any_new = false, full = true;
        if (mine) {
            for (int32_t w = 0; w < a.W; ++w) {
                const size_t idx = (size_t)v * a.W + w;
                const unsigned long long vv = a.V[idx];
                const unsigned long long nw = Fn[idx] & ~vv & lane_mask(a.S, w);
                a.V[idx] = vv | nw;
                Fn[idx] = nw;
                full &= ((vv | nw) & lane_mask(a.S, w)) == lane_mask(a.S, w);
                acc.n_new += (uint32_t)__popcll(nw);
                any_new |= nw != 0ull;
                record_depth(a, v, w, nw, L + 1, false);
            }
            Tn[v >> 5] = 0u;
            if (full) atomicOr(a.D + (v >> 5), 1u << (v & 31));
        }
        st.put(mine && any_new, v);
    }
    st.flush();
}

// Clear F_{(L+2) mod 3} and T_{(L+2) mod 3} for the active list of level L - 1:
// those buffers were last read at level L - 1 and are written again at level L + 1.
__device__ __forceinline__ void ms_clear_prev(const MsArgs& a, const int32_t* ids, uint32_t count,
                                              unsigned long long* F, uint32_t* T) {
    const long long gtid = (long long)blockIdx.x * kMsThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kMsThreads;
    for (long long k = gtid; k < count; k += gstride) {
        const int32_t v = ids[k];
        for (int32_t w = 0; w < a.W; ++w) F[(size_t)v * a.W + w] = 0ull;
        T[v >> 5] = 0u;  // every bit of T_{(L+2) mod 3} belongs to that list: racing writers all store zero
    }
}

// ---------------------------------------------------------------- kernel

template <int CW, int kOcc>
__global__ void __launch_bounds__(kMsThreads, kOcc) ms_bfs_kernel(MsArgs a) {
    const long long gtid = (long long)blockIdx.x * kMsThreads + threadIdx.x;
    // an error of an earlier launch not yet read by the host: this launch does nothing
    const int pending = threadIdx.x == 0 ? ld_volatile_i32(a.status + ST_ERROR) : 0;
    const long long gstride = (long long)gridDim.x * kMsThreads;
    __shared__ StageBuf stage_mem[kMsThreads / 32];
    __shared__ unsigned long long lvl[6];
    __shared__ unsigned long long acc_mem[kMsThreads / 32][4];
    const int wib = threadIdx.x >> 5;
    unsigned int* barc = a.bar->count + a.bar_parity;
    unsigned int bar_round = 0;
    unsigned long long t_mark = gtid == 0 ? global_timer_ns() : 0ull;
    // ---- init: V = F_k = 0, depth planes = 0, D = T_k = 0 (the output rows are written at the end)
    const size_t nw_total = (size_t)a.n * (size_t)a.W;
    for (size_t i = gtid; i < nw_total; i += gstride) {
        a.V[i] = 0ull;
        a.Fb[0][i] = 0ull;
        a.Fb[1][i] = 0ull;
        a.Fb[2][i] = 0ull;
#pragma unroll
        for (int p = 0; p < kMsPlanes; ++p) a.P[p][i] = 0ull;
    }
    for (long long w = gtid; w < a.nwords; w += gstride) {
        a.D[w] = 0u;
        a.Tb[0][w] = 0u;
        a.Tb[1][w] = 0u;
        a.Tb[2][w] = 0u;
    }
    if (gtid == 0) {
        LevelCtr z = {};
        a.ctr[0] = z;
        a.ctr[1] = z;
        a.ctr[2] = z;
        a.status[ST_LEVELS] = 0;
        a.bar->count[a.bar_parity ^ 1u] = 0u;
    }
    if (__syncthreads_or(pending)) return;
    if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
    // ---- sources: lane b starts at src[b] with depth 0
    for (long long b = gtid; b < a.S; b += gstride) {
        const int32_t s = a.src[b];
        atomicOr(a.V + (size_t)s * a.W + (b >> 6), 1ull << (b & 63));  // depth 0: no plane bit
    }
    if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
    // F = V for the (distinct) source vertices; they form the first active list
    {
        Acc acc0;
        Stage st{stage_mem + wib, 0, a.ctr + 0, a.ids[0], a.qp[0], a.qd[0], a.out_ptr, a.in_ptr, 1, 0, &acc0};
        const long long rounds = ((long long)a.S + gstride - 1) / gstride;
        for (long long r = 0; r < rounds; ++r) {
            const long long b = r * gstride + gtid;
            bool take = false;
            int32_t s = 0;
            if (b < a.S) {
                s = a.src[b];
                take = !(atomicOr(a.Tb[0] + (s >> 5), 1u << (s & 31)) & (1u << (s & 31)));
                if (take)
                    for (int32_t w = 0; w < a.W; ++w) a.Fb[0][(size_t)s * a.W + w] = a.V[(size_t)s * a.W + w];
            }
            st.put(take, s);
        }
        st.flush();
        const unsigned long long m = warp_sum_u64(acc0.mf);
        if ((threadIdx.x & 31) == 0 && m) atomicAdd(&a.ctr[0].mf_new, m);
    }
    if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
    for (long long b = gtid; b < a.S; b += gstride) {
        const int32_t s = a.src[b];
        a.Tb[0][s >> 5] = 0u;  // racing writers all store zero
    }
    if (threadIdx.x == 0) lvl[4] = ld_volatile_u64(&a.ctr[0].q);
    if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
    unsigned long long qv = lvl[4];
    uint32_t prev_count = 0;  // size of the active list of level L - 1
    long long pairs = a.S;
    for (int32_t L = 0;; ++L) {
        const int r0 = L % 3, r1 = (L + 1) % 3, r2 = (L + 2) % 3, p0 = L & 1, p1 = p0 ^ 1;
        LevelCtr* cout = a.ctr + ((L + 1) % 3);
        if (gtid == 0) {
            LevelCtr z = {};
            a.ctr[(L + 2) % 3] = z;
        }
        const uint32_t qcount = (uint32_t)qv, qedges = (uint32_t)(qv >> 32);
        // direction for the whole batch: pull once the active edges exceed alpha * nnz
        int dir = a.mode;
        if (dir == GBX_DIR_AUTO) dir = (double)qedges > (double)a.alpha * (double)a.nnz ? GBX_DIR_PULL : GBX_DIR_PUSH;
        if (a.depth16 && L + 1 > 32767) {
            if (gtid == 0) atomicCAS(a.status + ST_ERROR, 0, (int)GBX_ERR_OVERFLOW);
            return;
        }
        Acc acc;
        Stage st{stage_mem + wib, 0, cout, a.ids[r1], a.qp[p1], a.qd[p1], a.out_ptr, a.in_ptr, 1, 0, &acc};
        ms_clear_prev(a, a.ids[r2], prev_count, a.Fb[r2], a.Tb[r2]);
        if (dir == GBX_DIR_PUSH) {
            ms_push<CW>(a, L, a.ids[r0], a.qp[p0], a.qd[p0], qcount, qedges, a.Fb[r0], a.Fb[r1], a.Tb[r1], st, acc);
            if (CW > 1) {
                if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
                if (threadIdx.x == 0) lvl[5] = ld_volatile_u64(&cout->list);
                __syncthreads();
                ms_push_finalize<CW>(a, L, (uint32_t)lvl[5], a.Fb[r1], a.Tb[r1], st, acc);
            }
        } else {
            ms_pull<CW>(a, L, a.Fb[r1], st, acc);
        }
        block_add_counts<kMsThreads / 32>(acc_mem, acc.n_new, acc.mf, acc.exam, 0ull, &cout->n_new, &cout->mf_new,
                                          &cout->e_exam, nullptr);
        if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
        if (threadIdx.x == 0) {
            lvl[0] = ld_volatile_u64(&cout->n_new);
            lvl[1] = ld_volatile_u64(&cout->mf_new);
            lvl[3] = ld_volatile_u64(&cout->e_exam);
            lvl[4] = ld_volatile_u64(&cout->q);
        }
        __syncthreads();
        qv = lvl[4];
        if (dir == GBX_DIR_PULL) {
            // V |= F for the vertices the pull found (their new lanes were kept apart so the
            // level read V as it was before it started)
            ms_pull_commit<CW>(a, a.ids[r1], (uint32_t)qv, a.Fb[r1]);
            if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
        }
        const long long n_new = (long long)lvl[0];
        if (gtid == 0 && L < a.trace_cap) {
            LevelRec r;
            r.direction = dir;
            r.level = L;
            r.nf = (long long)qcount;
            r.mf = (long long)qedges;
            r.mu = pairs;
            r.e_exam = dir == GBX_DIR_PULL ? (long long)lvl[3] : -1;
            r.n_new = n_new;
            r.mf_new = (long long)lvl[1];
            const unsigned long long now = global_timer_ns();
            r.t_ns = (long long)(now - t_mark);
            t_mark = now;
            a.trace[L] = r;
        }
        if (n_new == 0) {
            if (gtid == 0) a.status[ST_LEVELS] = L + 1;
            emit_depths(a);
            return;
        }
        if (L + 1 >= a.n) {
            if (gtid == 0) atomicCAS(a.status + ST_ERROR, 0, (int)GBX_ERR_OVERFLOW);
            return;
        }
        pairs = n_new;
        prev_count = qcount;
    }
}

gbx_status ms_reserve(Workspace& w, int32_t n, int32_t S, cudaStream_t s) {
    const int32_t w_raw = (S + 63) / 64;
    const int cw = w_raw >= 4 ? 4 : (w_raw >= 2 ? 2 : 1);
    const int64_t need = (int64_t)n * ((w_raw + cw - 1) / cw * cw);
    if (w.ms_cap_words < need) {
        if (w.msV || w.msP || w.msF[0] || w.msF[1] || w.msF[2]) {
            GBX_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(w.msV);
            w.msV = nullptr;
            for (auto& p : w.msF) {
                cudaFree(p);
                p = nullptr;
            }
            cudaFree(w.msP);
            w.msP = nullptr;
            w.ms_cap_words = 0;
        }
        GBX_CUDA_TRY(cudaMalloc((void**)&w.msV, sizeof(unsigned long long) * (size_t)need));
        for (auto& p : w.msF) GBX_CUDA_TRY(cudaMalloc((void**)&p, sizeof(unsigned long long) * (size_t)need));
        GBX_CUDA_TRY(cudaMalloc((void**)&w.msP, sizeof(unsigned long long) * (size_t)need * kMsPlanes));
        w.ms_cap_words = need;  // only once every buffer exists
    }
    if (w.ms_t_cap < (int64_t)n + 1) {
        if (w.msT) {
            GBX_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(w.msT);
            w.msT = nullptr;
            w.ms_t_cap = 0;
        }
        GBX_CUDA_TRY(cudaMalloc((void**)&w.msT, sizeof(int32_t) * ((size_t)n + 1)));
        w.ms_t_cap = (int64_t)n + 1;
    }
    return GBX_OK;
}

int64_t ms_scratch_bytes(int32_t n, int32_t S) {
    const int32_t w_raw = (S + 63) / 64;
    const int cw = w_raw >= 4 ? 4 : (w_raw >= 2 ? 2 : 1);
    return (4ll + kMsPlanes) * 8ll * (int64_t)n * ((w_raw + cw - 1) / cw * cw) + 4ll * ((int64_t)n + 1);
}

template <int CW, int kOcc>
static gbx_status ms_launch(Graph* G, const MsArgs& a0, int blocks, int per_sm_cap, cudaStream_t s) {
    int per_sm = 0;
    GBX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ms_bfs_kernel<CW, kOcc>, kMsThreads, 0));
    GBX_CHECK(per_sm >= 1, GBX_ERR_CUDA, "batched BFS kernel cannot be resident");
    if (per_sm_cap > 0 && per_sm_cap < per_sm) per_sm = per_sm_cap;
    const int full = per_sm * G->num_sms;
    const int nb = blocks > 1 ? (full / blocks > 0 ? full / blocks : 1) : full;  // a 1/blocks share of the GPU
    MsArgs a = a0;
    void* args[] = {&a};
    GBX_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)ms_bfs_kernel<CW, kOcc>, dim3(nb), dim3(kMsThreads), args, 0,
                                             s));
    return GBX_OK;
}

// One batched BFS on G: sources already on the device (src_dev), depth either a
// [S][n] buffer or a device table of S row pointers.  `blocks` > 1 runs the
// persistent kernel on 1/blocks of the GPU's resident blocks (so that many
// batches of other graphs fit alongside); scratch must be reserved for S lanes.
gbx_status ms_run(Graph* G, Workspace& w, int32_t S, const int32_t* src_dev, void* depth, void* const* rows,
                  int depth16, const gbx_desc& d, int blocks, cudaStream_t s) {
    const int32_t w_raw = (S + 63) / 64;
    const int cw = w_raw >= 4 ? 4 : (w_raw >= 2 ? 2 : 1);
    const int32_t W = (w_raw + cw - 1) / cw * cw;
    GBX_CHECK(w.ms_cap_words >= (int64_t)G->n * W && w.n_cap >= G->n && w.ms_t_cap > G->n, GBX_ERR_INVALID_VALUE,
              "batch scratch not reserved");
    MsArgs a;
    a.n = G->n;
    a.S = S;
    a.W = W;
    a.nwords = G->nwords;
    a.nnz = G->nnz;
    a.out_ptr = G->out_ptr;
    a.out_col = G->out_col;
    a.in_ptr = G->in_ptr;
    a.in_col = G->in_col;
    a.nz_in = G->nz_in;
    a.V = w.msV;
    for (int k = 0; k < 3; ++k) a.Fb[k] = w.msF[k];
    for (int k = 0; k < kMsPlanes; ++k) a.P[k] = w.msP + (size_t)k * (size_t)G->n * (size_t)W;
    a.D = w.bm[2];
    a.Tb[0] = w.bm[3];
    a.Tb[1] = w.bm[0];
    a.Tb[2] = w.bm[1];
    a.tlist = w.msT;
    a.depth = depth;
    a.rows = rows;
    a.depth16 = depth16;
    a.src = src_dev;
    a.ids[0] = w.q[0];
    a.ids[1] = w.q[1];
    a.ids[2] = w.list;
    for (int i = 0; i < 2; ++i) {
        a.qp[i] = w.qp[i];
        a.qd[i] = w.qd[i];
    }
    a.ctr = w.ctr;
    a.bar = w.bar;
    a.bar_parity = w.bar_parity;
    a.trace = w.trace;
    a.status = w.status;
    a.alpha = d.alpha;
    a.mode = d.direction;
    a.symmetric = G->symmetric;
    a.trace_cap = kTraceCap;
    a.probe = d.pull_probe > 0 ? d.pull_probe : kMsProbe;
    a.timeout_ns = wait_timeout_ns();
    // the lean build only when this batch has the GPU to itself: concurrent cooperative
    // grids of one register budget tile the SMs exactly, mixed budgets need not
    const bool lean = blocks <= 1 && d.blocks_per_sm >= kMsOccLean && cw <= 2;
    const int cap = lean ? 0 : d.blocks_per_sm;
    gbx_status st;
    if (cw == 4)
        st = ms_launch<4, kMsOcc>(G, a, blocks, cap, s);
    else if (cw == 2)
        st = lean ? ms_launch<2, kMsOccLean>(G, a, blocks, cap, s) : ms_launch<2, kMsOcc>(G, a, blocks, cap, s);
    else
        st = lean ? ms_launch<1, kMsOccLean>(G, a, blocks, cap, s) : ms_launch<1, kMsOcc>(G, a, blocks, cap, s);
    if (st != GBX_OK) return st;
    w.bar_parity ^= 1u;
    w.last_stream = s;
    w.last_traced = 2;  // batched trace
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_bfs_batch(gbx_graph* g, const int32_t* sources, int32_t S, void* depth, int32_t depth_type,
                                    const gbx_desc* desc, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    GBX_CHECK(S >= 1, GBX_ERR_INVALID_VALUE, "S must be >= 1");
    GBX_CHECK(sources != nullptr && depth != nullptr, GBX_ERR_NULL_POINTER, "sources or depth is NULL");
    GBX_CHECK(depth_type == GBX_DEPTH_I32 || depth_type == GBX_DEPTH_I16, GBX_ERR_INVALID_VALUE, "depth_type");
    for (int32_t k = 0; k < S; ++k)
        GBX_CHECK(sources[k] >= 0 && sources[k] < G->n, GBX_ERR_INVALID_INDEX, "source outside [0, n)");
    gbx_desc d;
    if (desc)
        d = *desc;
    else
        gbx_desc_init(&d);
    GBX_CHECK(d.direction >= GBX_DIR_AUTO && d.direction <= GBX_DIR_PULL, GBX_ERR_INVALID_VALUE, "desc.direction");
    GBX_CHECK(d.alpha >= 0.0f && d.alpha == d.alpha, GBX_ERR_INVALID_VALUE, "desc.alpha must be >= 0");
    GBX_CHECK(d.pull_probe == 0 || (d.pull_probe >= 4 && d.pull_probe <= 1024), GBX_ERR_INVALID_VALUE,
              "desc.pull_probe must be 0 or in [4, 1024]");
    GBX_CHECK(d.push_sort == 0, GBX_ERR_NOT_SUPPORTED, "desc.push_sort applies to gbx_mxv only");
    GBX_CHECK(d.blocks_per_sm >= 0, GBX_ERR_INVALID_VALUE, "desc.blocks_per_sm must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    GBX_TRY(ms_reserve(G->ws, G->n, S, s));
    if (G->ws.ms_src_cap < S) {
        if (G->ws.ms_src) {
            GBX_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(G->ws.ms_src);
            cudaFreeHost(G->ws.ms_src_pinned);
            G->ws.ms_src = nullptr;
            G->ws.ms_src_pinned = nullptr;
        }
        GBX_CUDA_TRY(cudaMalloc((void**)&G->ws.ms_src, sizeof(int32_t) * (size_t)S));
        GBX_CUDA_TRY(cudaMallocHost((void**)&G->ws.ms_src_pinned, sizeof(int32_t) * (size_t)S));
        G->ws.ms_src_cap = S;
    }
    if (!G->ws.ms_src_ready) GBX_CUDA_TRY(cudaEventCreateWithFlags(&G->ws.ms_src_ready, cudaEventDisableTiming));
    // sources: pinned staging, then one async copy (the staging buffer is reused only
    // after the previous copy has completed)
    GBX_CUDA_TRY(cudaEventSynchronize(G->ws.ms_src_ready));
    for (int32_t k = 0; k < S; ++k) G->ws.ms_src_pinned[k] = sources[k];
    GBX_CUDA_TRY(cudaMemcpyAsync(G->ws.ms_src, G->ws.ms_src_pinned, sizeof(int32_t) * (size_t)S, cudaMemcpyHostToDevice, s));
    GBX_CUDA_TRY(cudaEventRecord(G->ws.ms_src_ready, s));
    return ms_run(G, G->ws, S, G->ws.ms_src, depth, nullptr, depth_type == GBX_DEPTH_I16 ? 1 : 0, d, 0, s);
}

extern "C" gbx_status gbx_bfs_batch_trace(gbx_graph* g, gbx_level* levels, int32_t cap, int32_t* nlevels) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    GBX_CHECK(nlevels != nullptr, GBX_ERR_NULL_POINTER, "nlevels is NULL");
    GBX_CHECK(cap == 0 || levels != nullptr, GBX_ERR_NULL_POINTER, "levels is NULL");
    GBX_CHECK(G->ws.last_traced == 2, GBX_ERR_INVALID_VALUE, "the last run on this graph was not a batched BFS");
    if (G->ws.last_stream) GBX_CUDA_TRY(cudaStreamSynchronize(G->ws.last_stream));
    int32_t st[ST_WORDS];
    GBX_CUDA_TRY(cudaMemcpy(st, G->ws.status, sizeof(st), cudaMemcpyDeviceToHost));
    GBX_CHECK(st[ST_ERROR] == 0, (gbx_status)st[ST_ERROR], "the last batched BFS recorded a device-side error");
    *nlevels = st[ST_LEVELS];
    const int32_t L = st[ST_LEVELS] < kTraceCap ? st[ST_LEVELS] : kTraceCap;
    const int32_t ncopy = L < cap ? L : cap;
    if (ncopy <= 0) return GBX_OK;
    LevelRec* recs = new LevelRec[ncopy];
    const cudaError_t e = cudaMemcpy(recs, G->ws.trace, sizeof(LevelRec) * ncopy, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] recs;
        GBX_CUDA_TRY(e);
    }
    for (int32_t l = 0; l < ncopy; ++l) {
        const LevelRec& r = recs[l];
        gbx_level o = {};
        o.direction = r.direction;
        o.level = r.level;
        o.nf = r.nf;          // active vertices (any lane)
        o.mf = r.mf;          // their out-edges
        o.nu = -1;
        o.nu_nz = -1;
        o.mu = r.mu;          // (vertex, lane) pairs found at the previous level
        o.e_exam = r.e_exam;  // pull: edges examined (per 256-lane chunk)
        o.n_new = r.n_new;    // (vertex, lane) pairs found at this level
        o.mf_new = r.mf_new;  // out-edges of the next active list
        o.time_ns = r.t_ns;
        levels[l] = o;
    }
    delete[] recs;
    return GBX_OK;
}
