// Direction-optimized BFS (Algorithm 1) as one persistent cooperative kernel.
//
// Every level computes f' = A^T f .* !v (the GrB_mxv of Algorithm 1, line 8)
// either as
//   push: column-based masked matvec (Eq 5, Section 4.1) -- the edges of the
//         frontier queue are split evenly over all warps (an exclusive prefix
//         of out-degrees is stored with every queue entry, so a warp finds its
//         first vertex by binary search and the rest by a 32-entry window), and
//         each child is claimed with atomicOr on the visited bitmap.  The
//         bitmap claim replaces the radix sort + segmented reduction of
//         Algorithm 3 (Section 6.2): it deduplicates exactly, in one pass.
//   pull: row-based masked matvec (Eq 4, Algorithm 2) over the rows the mask
//         !v lets through (Section 5.2), each row stopping at its first parent
//         (early exit, Section 5.3), testing "visited before this level"
//         instead of "in the frontier" (operand reuse, Section 5.4).  A warp
//         owns 32 consecutive vertices (one bitmap word); a lane probes its own
//         row first and long rows are then scanned by the whole warp with
//         __ballot_sync, so power-law rows do not serialise a lane.
// and picks the next level's direction on the device (Section 6.3).  The
// GrB_assign of line 7 (depth stamp) and the GrB_reduce of line 9 (frontier
// count) are fused into the level; levels are separated by a bounded grid
// barrier instead of kernel launches.
#include <atomic>

#include "frontier.cuh"
#include "gbx_internal.cuh"

namespace gbx {

#ifndef GBX_BFS_THREADS
#define GBX_BFS_THREADS 512
#endif
#ifndef GBX_BFS_MIN_BLOCKS
#define GBX_BFS_MIN_BLOCKS 2
#endif
#ifndef GBX_PULL_PROBE
#define GBX_PULL_PROBE 16
#endif
constexpr int kBfsThreads = GBX_BFS_THREADS;
constexpr int kBfsMinBlocks = GBX_BFS_MIN_BLOCKS;
constexpr int kProbe = GBX_PULL_PROBE;  // default in-neighbours a lane examines before the warp takes the row
enum { DIR_PUSH = GBX_DIR_PUSH, DIR_PULL = GBX_DIR_PULL };

struct BfsArgs {
    int32_t n, nwords, source;
    long long nnz;
    const int32_t* out_ptr;
    const int32_t* out_col;
    const int32_t* in_ptr;
    const int32_t* in_col;
    const uint32_t* nz_in;
    const uint32_t* multi_in;
    const int32_t* first_in;
    const int4* next_in;
    int32_t* depth;
    int32_t* parent;
    uint32_t* vis[2];
    uint32_t* fbm;
    int32_t* q[2];
    int32_t* qp[2];
    int32_t* qd[2];
    int32_t* hfirst;  // per deferred long row: first in-edge index found in the frontier
    LevelCtr* ctr;
    GridBar* bar;
    LevelRec* trace;
    int32_t* status;
    float alpha, beta;
    int32_t heuristic, mode, early_exit, masking, operand_reuse, symmetric, need_indeg, need_deg, trace_cap, probe,
        tile_words;
    unsigned long long timeout_ns;
    unsigned int bar_parity;
};

// Adds the block's counts of this level to cout (every thread of the block calls it).
__device__ __forceinline__ void flush_acc(const Acc& acc, LevelCtr* cout, bool with_exam,
                                          unsigned long long (*sm)[4]) {
    block_add_counts<kBfsThreads / 32>(sm, acc.n_new, acc.mf, acc.indeg, with_exam ? acc.exam : 0ull, &cout->n_new,
                                       &cout->mf_new, &cout->indeg_new, &cout->e_exam);
}

// ---------------------------------------------------------------- push (Eq 5)


// The warp's edge range is walked as a software pipeline of four stages, each on
// a different step of kBfsStep edges: (1) map the edges to queue entries and load
// their frontier vertex and row offset, (2) load the child, (3) load the child's
// visited word, (4) claim unvisited children with atomicOr.  One iteration issues
// the memory operations of all four stages (on steps s, s-1, s-2, s-3) before it
// waits for any of them, so a step costs about one memory round trip instead of
// four dependent ones.
#ifndef GBX_BFS_PUSH_ILP
#define GBX_BFS_PUSH_ILP 2
#endif
constexpr int kBfsIlp = GBX_BFS_PUSH_ILP;  // edges per lane and step
constexpr int kBfsStep = 32 * kBfsIlp;
// stamp: write depth and parent of the claimed children (level 0 leaves them to the
// start of level 1, when the concurrently initialised outputs are complete).
__device__ __forceinline__ void push_level(const BfsArgs& a, int32_t L, int cur, int vcur, uint32_t qcount,
                                           uint32_t qedges, Stage& stg, unsigned long long* bsm, Acc& acc,
                                           bool stamp) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    const int32_t* q = a.q[cur];
    const int32_t* qp = a.qp[cur];
    const int32_t* qd = a.qd[cur];
    uint32_t* vis = a.vis[vcur];
    const int32_t E = (int32_t)qedges;
    int32_t chunk = (int32_t)(((long long)E + nwarps - 1) / nwarps);
    // a level with at most 32 edges per warp gives each warp 32 (one slot of a step filled):
    // twice the warps of full steps, each with a single step's round trips
    chunk = chunk <= 32 ? 32 : ((chunk + kBfsStep - 1) / kBfsStep) * kBfsStep;
    for (long long e0l = (long long)gwarp * chunk; e0l < E; e0l += (long long)nwarps * chunk) {
        const int32_t e0 = (int32_t)e0l;
        const int32_t e1 = E - e0 > chunk ? e0 + chunk : E;
        const int32_t nsteps = (e1 - e0 + kBfsStep - 1) / kBfsStep;
        PushCursorT<kBfsIlp> cur_;
        cur_.k = warp_find_entry(qp, (int32_t)qcount, e0);
        cur_.wlast = -1;
        if (nsteps == 1) {
            // a single step (a small frontier): no pipeline fill and drain
            for (int32_t base = e0; base < e1; base += kBfsStep) {
                const PushStepT<kBfsIlp> now = cur_.gather(a.out_col, q, qp, qd, qcount, base, e1);
                // every slot's probe, then every slot's claim: the slots' round trips overlap
                uint32_t w[kBfsIlp], old[kBfsIlp];
#pragma unroll
                for (int t = 0; t < kBfsIlp; ++t) w[t] = now.u[t] >= 0 ? __ldca(vis + (now.v[t] >> 5)) : 0xffffffffu;
#pragma unroll
                for (int t = 0; t < kBfsIlp; ++t) {
                    const uint32_t bit = 1u << (now.v[t] & 31);
                    old[t] = (now.u[t] >= 0 && !(w[t] & bit)) ? atomicOr(vis + (now.v[t] >> 5), bit) : 0xffffffffu;
                }
#pragma unroll
                for (int t = 0; t < kBfsIlp; ++t) {
                    const uint32_t bit = 1u << (now.v[t] & 31);
                    const bool claimed = now.u[t] >= 0 && !(old[t] & bit);
                    if (claimed) {
                        if (stamp) {
                            a.depth[now.v[t]] = L + 1;
                            if (a.parent) a.parent[now.v[t]] = now.u[t];
                        }
                        acc.n_new += 1;
                    }
                    stg.put(claimed, now.v[t]);
                }
            }
            continue;
        }
        // stage registers: u < 0 marks an empty slot (past e1, or pipeline fill and drain)
        int32_t u1[kBfsIlp], d1[kBfsIlp];                 // after stage 1: vertex, row start - prefix
        int32_t u2[kBfsIlp], v2[kBfsIlp];                 // after stage 2: vertex, child
        int32_t u3[kBfsIlp], v3[kBfsIlp];                 // after stage 3: vertex, child, visited word
        uint32_t w3[kBfsIlp];
#pragma unroll
        for (int t = 0; t < kBfsIlp; ++t) {
            u1[t] = u2[t] = u3[t] = -1;
            d1[t] = v2[t] = v3[t] = 0;
            w3[t] = 0xffffffffu;
        }
        for (int32_t it = 0; it < nsteps + 3; ++it) {
            // stage 4 (step it - 3): claim the children whose visited bit was clear
            uint32_t old[kBfsIlp];
#pragma unroll
            for (int t = 0; t < kBfsIlp; ++t) {
                const uint32_t bit = 1u << (v3[t] & 31);
                // L1-cached probe of stage 3: a stale word only costs an extra atomic, the atomic decides
                old[t] = (u3[t] >= 0 && !(w3[t] & bit)) ? atomicOr(vis + (v3[t] >> 5), bit) : 0xffffffffu;
            }
            // stage 3 (step it - 2): visited words of the children
            uint32_t w2[kBfsIlp];
#pragma unroll
            for (int t = 0; t < kBfsIlp; ++t) w2[t] = u2[t] >= 0 ? __ldca(vis + (v2[t] >> 5)) : 0xffffffffu;
            // stage 2 (step it - 1): children
            int32_t c1[kBfsIlp];
            const int32_t b1 = e0 + (it - 1) * kBfsStep;
#pragma unroll
            for (int t = 0; t < kBfsIlp; ++t) c1[t] = u1[t] >= 0 ? __ldg(a.out_col + b1 + 32 * t + lane + d1[t]) : 0;
            // stage 1 (step it): queue entries
            int32_t u0[kBfsIlp], d0[kBfsIlp];
            if (it == 0) {
                cur_.map(q, qp, qd, qcount, e0, e1, u0, d0);
            } else if (it < nsteps) {
                const int32_t ul = __shfl_sync(0xffffffffu, u1[kBfsIlp - 1], 31);
                const int32_t dl = __shfl_sync(0xffffffffu, d1[kBfsIlp - 1], 31);
                cur_.map_after(q, qp, qd, qcount, e0 + it * kBfsStep, e1, ul, dl, u0, d0);
            } else {
#pragma unroll
                for (int t = 0; t < kBfsIlp; ++t) {
                    u0[t] = -1;
                    d0[t] = 0;
                }
            }
            // stage 4, continued: stamp the claimed children (the fused GrB_assign) and stage them
#pragma unroll
            for (int t = 0; t < kBfsIlp; ++t) {
                const bool claimed = u3[t] >= 0 && !(old[t] & (1u << (v3[t] & 31)));
                if (claimed) {
                    if (stamp) {
                        a.depth[v3[t]] = L + 1;
                        if (a.parent) a.parent[v3[t]] = u3[t];
                    }
                    acc.n_new += 1;
                }
                stg.put(claimed, v3[t]);
            }
            // advance the pipeline
#pragma unroll
            for (int t = 0; t < kBfsIlp; ++t) {
                u3[t] = u2[t];
                v3[t] = v2[t];
                w3[t] = w2[t];
                u2[t] = u1[t];
                v2[t] = c1[t];
                u1[t] = u0[t];
                d1[t] = d0[t];
            }
        }
    }
    stg.flush_block<kBfsThreads / 32>(bsm);
}

// ---------------------------------------------------------------- pull (Eq 4, Algorithm 2)

#ifndef GBX_PULL_ILP
#define GBX_PULL_ILP 2
#endif
constexpr int kPullIlp = GBX_PULL_ILP;  // candidate rows per lane per round (independent probe chains)
#ifndef GBX_PULL_STEP
#define GBX_PULL_STEP 2
#endif
constexpr int kPullStep = GBX_PULL_STEP;  // in-neighbours a lane loads per probe step (loads in flight)
// Bitmap words one warp takes at a time in a pull level, a.tile_words: 32, 16 or
// 8 (lane l holds word l of the tile).  The host picks the width whose round-robin
// critical path, ceil(tiles / warps) * width, is shortest (ties: the wider), so a
// graph with fewer 32-word tiles than warps still keeps every warp busy.
int32_t pull_tile_words(int32_t nwords, long long nwarps) {
    int32_t best = 32;
    long long best_cost = -1;
    for (int32_t tw = 32; tw >= 8; tw >>= 1) {
        const long long tiles = ((long long)nwords + tw - 1) / tw;
        const long long cost = (tiles + nwarps - 1) / nwarps * tw;
        if (best_cost < 0 || cost < best_cost) {
            best = tw;
            best_cost = cost;
        }
    }
    return best;
}
// A row with more than kPullHugeRow in-edges left after the lane probe is not
// scanned by the warp that met it: it is listed and, once every tile is done,
// the whole grid scans its edges in chunks of kPullChunk (a hub row of 10^5+
// edges would otherwise hold one warp for milliseconds while the rest idle).
#ifndef GBX_PULL_HUGE_ROW
#define GBX_PULL_HUGE_ROW 512
#endif
#ifndef GBX_PULL_CHUNK
#define GBX_PULL_CHUNK 1024
#endif
constexpr int32_t kPullHugeRow = GBX_PULL_HUGE_ROW;
constexpr int32_t kPullChunk = GBX_PULL_CHUNK;

// Deferred long rows of one pull level, kept in the arrays of the queue that the
// level does not use: row (bitwise NOT of it when the tile phase already found a
// parent, so the chunks only count examined edges), first edge left, and the
// ascending prefix of their chunk counts.
struct HugeRows {
    int32_t* row;
    int32_t* k;
    int32_t* base;
    int32_t* first;  // smallest edge index with a hit found so far (INT32_MAX: none)
};

// One warp-wide scan of in_col[kk, kk + 32 * kT) against tbm (kT loads in
// flight per lane).  Returns the position of the first edge whose source is in
// tbm (32 * kT if none in range) and that source in *jf.
template <int kT>
__device__ __forceinline__ int warp_scan(const int32_t* __restrict__ in_col, const uint32_t* tbm, int32_t kk,
                                         int32_t ee, int32_t* jf) {
    const int lane = threadIdx.x & 31;
    int32_t j[kT];
#pragma unroll
    for (int t = 0; t < kT; ++t) {
        const int32_t idx = kk + 32 * t + lane;
        j[t] = idx < ee ? __ldg(in_col + idx) : -1;
    }
    uint32_t b[kT];
#pragma unroll
    for (int t = 0; t < kT; ++t) b[t] = __ballot_sync(0xffffffffu, j[t] >= 0 && bit_test(tbm, j[t]));
    int pos = 32 * kT;
    int32_t jsel = j[kT - 1];
#pragma unroll
    for (int t = kT - 1; t >= 0; --t) {
        if (b[t]) {
            pos = 32 * t + __ffs(b[t]) - 1;
            jsel = j[t];
        }
    }
    if (pos < 32 * kT) *jf = __shfl_sync(0xffffffffu, jsel, pos & 31);
    return pos;
}

// A warp takes a tile of a.tile_words bitmap words and finds the rows the mask
// lets through (unvisited, with in-edges), listed in shared memory in row order
// (put_tile_list).  Pass 1 tests every such row's first in-neighbour (the dense
// first_in array) against the frontier, kP1 rows per lane in flight; most rows
// of a power-law graph settle here.  Pass 2 takes the rows pass 1 left open that
// have more in-neighbours, 32 * kPullIlp per round, kPullIlp rows per lane probing
// in lockstep: in-neighbours 1..4 from the dense next_in array, then the lane
// probe; rows longer than the probe depth are finished by the whole warp, or by
// the whole grid when they are very long.
#ifndef GBX_PULL_P1
#define GBX_PULL_P1 4
#endif
constexpr int kP1 = GBX_PULL_P1;  // pass-1 rows per lane per round

// The rows of a tile whose bits are set in the lane words `m` (lane l holds word l
// of the tile), in row order, as offsets in the tile: the lane writes its word's
// rows at its exclusive prefix `excl` of the words' bit counts.  One pass over the
// set bits, where a per-round search of the packed list costs a warp-wide binary
// search of shuffles and an n-th-set-bit per entry.  The warp syncs before (earlier
// readers of the list) and after.
__device__ __forceinline__ void put_tile_list(uint16_t* clist, uint32_t m, uint32_t excl) {
    __syncwarp();
    const uint32_t rowbase = (threadIdx.x & 31) << 5;
    while (m) {
        const uint32_t b = __ffs(m) - 1;
        m &= m - 1;
        clist[excl++] = (uint16_t)(rowbase + b);
    }
    __syncwarp();
}

template <bool kHuge>
__device__ __forceinline__ void pull_level(const BfsArgs& a, int32_t L, int vcur, bool use_fbm, bool append,
                                           const HugeRows& hr, Stage& st, unsigned long long* bsm, uint32_t* snew,
                                           uint16_t* clist, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    const uint32_t* vprev = a.vis[vcur];
    uint32_t* vnext = a.vis[vcur ^ 1];
    const uint32_t* tbm = use_fbm ? a.fbm : vprev;
    const int32_t tw = a.tile_words;
    const int32_t ntiles = (a.nwords + tw - 1) / tw;
    const bool want_deg = a.need_deg != 0;
    for (int32_t tile = gwarp; tile < ntiles; tile += nwarps) {
        const int32_t w = tile * tw + lane;
        const bool wok = lane < tw && w < a.nwords;
        const uint32_t cw = wok ? vprev[w] : 0xffffffffu;
        const uint32_t nz = wok ? a.nz_in[w] : 0u;
        const uint32_t cand = a.masking ? (~cw & nz) : nz;
        snew[lane] = 0u;
        __syncwarp();
        const uint32_t cntc = __popc(cand);
        const uint32_t inclc = warp_inclusive_sum(cntc);
        const uint32_t totalc = __shfl_sync(0xffffffffu, inclc, 31);
        // a tile with no more candidates than one pass-2 round takes them all there (one pass, whose
        // row offsets load with the first in-neighbour); fuller tiles run pass 1 first
        const bool two_pass = totalc > 32u * kPullIlp;
        // ---- pass 1: the first in-neighbour of every candidate row
        if (two_pass) {
            const uint32_t total = totalc;
            put_tile_list(clist, cand, inclc - cntc);
            acc.exam += cntc;  // every candidate examines its first in-neighbour
            for (uint32_t base = 0; base < total; base += 32 * kP1) {
                int32_t i[kP1], f0[kP1];
#pragma unroll
                for (int r = 0; r < kP1; ++r) {
                    const uint32_t c = base + 32 * r + lane;
                    i[r] = c < total ? ((tile * tw) << 5) + (int)clist[c] : -1;
                }
#pragma unroll
                for (int r = 0; r < kP1; ++r) f0[r] = i[r] >= 0 ? __ldg(a.first_in + i[r]) : -1;
                // every probe of the round is loaded before the round's first store: a store to
                // depth or parent may alias the bitmap as far as the compiler knows, and a load
                // after it would wait for the one before
                bool hitr[kP1];
#pragma unroll
                for (int r = 0; r < kP1; ++r) hitr[r] = f0[r] >= 0 && bit_test(tbm, f0[r]);
#pragma unroll
                for (int r = 0; r < kP1; ++r) {
                    const int j = (i[r] >> 5) - tile * tw;  // word of the tile (any lane when i < 0)
                    const int bp = i[r] & 31;
                    const uint32_t cwj = __shfl_sync(0xffffffffu, cw, j & 31);
                    const bool hit = hitr[r];
                    if (hit) atomicOr(snew + j, 1u << bp);
                    // without masking a visited row may find a parent too; only unvisited rows are new
                    const bool isnew = hit && !((cwj >> bp) & 1u);
                    if (isnew) {
                        a.depth[i[r]] = L + 1;
                        if (a.parent) a.parent[i[r]] = f0[r];
                        acc.n_new += 1;
                        if (want_deg) {  // m_f and m_u of the level (trace, Beamer's rule)
                            const int32_t rs = __ldg(a.in_ptr + i[r]), re = __ldg(a.in_ptr + i[r] + 1);
                            const int32_t od = a.symmetric ? re - rs
                                                           : __ldg(a.out_ptr + i[r] + 1) - __ldg(a.out_ptr + i[r]);
                            acc.mf += (uint32_t)od;
                            acc.indeg += (uint32_t)(re - rs);
                        }
                    }
                    if (append) st.put(isnew, i[r]);
                }
            }
        }
        __syncwarp();
        const uint32_t f1 = snew[lane];  // rows of my word that pass 1 found
        // ---- pass 2: rows with more in-neighbours that pass 1 did not settle
        const uint32_t multi = wok ? a.multi_in[w] : 0u;
        const uint32_t sv = two_pass ? cand & multi & (a.early_exit ? ~f1 : 0xffffffffu) : cand;
        const uint32_t cntw = __popc(sv);
        const uint32_t incl = warp_inclusive_sum(cntw);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) put_tile_list(clist, sv, incl - cntw);
        for (uint32_t base = 0; base < total; base += 32 * kPullIlp) {
            bool mine[kPullIlp], found[kPullIlp], found1[kPullIlp], done[kPullIlp];
            int jw[kPullIlp], bitpos[kPullIlp];
            uint32_t cwj[kPullIlp];
            int32_t i[kPullIlp], beg[kPullIlp], end[kPullIlp], k[kPullIlp], par[kPullIlp];
            unsigned long long exam[kPullIlp];
#pragma unroll
            for (int r = 0; r < kPullIlp; ++r) {
                const uint32_t c = base + 32 * r + lane;
                mine[r] = c < total;
                const int off = mine[r] ? (int)clist[c] : 0;
                const int j = off >> 5;
                jw[r] = j;
                const uint32_t f1j = __shfl_sync(0xffffffffu, f1, j);
                cwj[r] = __shfl_sync(0xffffffffu, cw, j);
                bitpos[r] = off & 31;
                i[r] = ((tile * tw + j) << 5) + bitpos[r];
                // only without early exit does pass 2 see rows pass 1 already found
                found1[r] = mine[r] && ((f1j >> bitpos[r]) & 1u);
                found[r] = found1[r];
                done[r] = false;
                exam[r] = 0;
            }
            int4 nx[kPullIlp];
#pragma unroll
            for (int r = 0; r < kPullIlp; ++r) {
                beg[r] = mine[r] ? __ldg(a.in_ptr + i[r]) : 0;
                end[r] = mine[r] ? __ldg(a.in_ptr + i[r] + 1) : 0;
                par[r] = (mine[r] && (!two_pass || found1[r])) ? __ldg(a.first_in + i[r]) : -1;
                nx[r] = mine[r] ? __ldg(a.next_in + i[r]) : make_int4(-1, -1, -1, -1);
            }
#pragma unroll
            for (int r = 0; r < kPullIlp; ++r) {
                k[r] = beg[r] + 1;  // the first in-neighbour is examined (by pass 1, or right here)
                if (!two_pass && mine[r]) {
                    exam[r] = 1;
                    if (bit_test(tbm, par[r])) {  // a candidate has in-edges: par holds its first
                        found[r] = true;
                        done[r] = a.early_exit != 0;
                    } else {
                        par[r] = -1;
                    }
                }
            }
            // in-neighbours 1..4 from the dense next-entries array (one 16-byte load, four probes
            // in flight); the first hit in row order is the parent
#pragma unroll
            for (int r = 0; r < kPullIlp; ++r) {
                if (!mine[r] || done[r]) continue;
                const bool h0 = nx[r].x >= 0 && bit_test(tbm, nx[r].x);
                const bool h1 = nx[r].y >= 0 && bit_test(tbm, nx[r].y);
                const bool h2 = nx[r].z >= 0 && bit_test(tbm, nx[r].z);
                const bool h3 = nx[r].w >= 0 && bit_test(tbm, nx[r].w);
                const int nv = (nx[r].x >= 0) + (nx[r].y >= 0) + (nx[r].z >= 0) + (nx[r].w >= 0);
                const int hit = h0 ? 0 : (h1 ? 1 : (h2 ? 2 : (h3 ? 3 : -1)));
                if (hit >= 0 && !found[r]) {
                    found[r] = true;
                    par[r] = hit == 0 ? nx[r].x : (hit == 1 ? nx[r].y : (hit == 2 ? nx[r].z : nx[r].w));
                }
                const bool stop = hit >= 0 && a.early_exit;
                const int used = stop ? hit + 1 : nv;
                exam[r] += (unsigned long long)used;
                k[r] += used;
                done[r] = stop;
            }
            // lane probes: up to a.probe in-neighbours per row, kPullStep at a time, both rows in lockstep
            for (int it = 0; it < (a.probe + kPullStep - 1) / kPullStep; ++it) {
                int32_t jj[kPullIlp][kPullStep];
                int32_t cnt[kPullIlp];
                bool act[kPullIlp];
#pragma unroll
                for (int r = 0; r < kPullIlp; ++r) {
                    const int32_t lim = end[r] < beg[r] + a.probe ? end[r] : beg[r] + a.probe;
                    act[r] = mine[r] && !done[r] && k[r] < lim;
                    cnt[r] = act[r] ? (lim - k[r] < kPullStep ? lim - k[r] : kPullStep) : 0;
#pragma unroll
                    for (int t = 0; t < kPullStep; ++t) jj[r][t] = t < cnt[r] ? __ldg(a.in_col + k[r] + t) : 0;
                }
                bool any = false;
#pragma unroll
                for (int r = 0; r < kPullIlp; ++r) any |= act[r];
                if (!any) break;
#pragma unroll
                for (int r = 0; r < kPullIlp; ++r) {
                    if (!act[r]) continue;
                    int hit = -1;
#pragma unroll
                    for (int t = kPullStep - 1; t >= 0; --t)
                        if (t < cnt[r] && bit_test(tbm, jj[r][t])) hit = t;
                    if (hit >= 0 && !found[r]) {
                        found[r] = true;
                        par[r] = jj[r][0];
#pragma unroll
                        for (int t = 1; t < kPullStep; ++t)
                            if (hit == t) par[r] = jj[r][t];
                        if (a.early_exit) {
                            exam[r] += (unsigned long long)(hit + 1);
                            k[r] += hit + 1;
                            done[r] = true;
                            continue;
                        }
                    }
                    exam[r] += (unsigned long long)cnt[r];
                    k[r] += cnt[r];
                }
            }
            // rows longer than the lane probe: the whole warp scans them (32, then 128 edges a step),
            // or lists them for the grid-wide phase when more than kPullHugeRow are left
#pragma unroll
            for (int r = 0; r < kPullIlp; ++r) {
                uint32_t pend = __ballot_sync(0xffffffffu, mine[r] && !done[r] && k[r] < end[r]);
                while (pend) {
                    const int t = __ffs(pend) - 1;
                    pend &= pend - 1;
                    int32_t kk = __shfl_sync(0xffffffffu, k[r], t);
                    const int32_t ee = __shfl_sync(0xffffffffu, end[r], t);
                    bool tf = __shfl_sync(0xffffffffu, found[r], t);
                    int32_t tp = __shfl_sync(0xffffffffu, par[r], t);
                    unsigned long long tx = 0;
                    if (kHuge && ee - kk > kPullHugeRow) {
                        const int32_t row = __shfl_sync(0xffffffffu, i[r], t);
                        if (lane == 0) {
                            const unsigned long long nch = (unsigned long long)((ee - kk + kPullChunk - 1) / kPullChunk);
                            const unsigned long long old = atomicAdd(&st.cout->huge, (nch << 32) | 1ull);
                            const uint32_t slot = (uint32_t)old;
                            hr.row[slot] = tf ? ~row : row;
                            hr.k[slot] = kk;
                            hr.base[slot] = (int32_t)(old >> 32);
                            hr.first[slot] = INT32_MAX;
                        }
                        kk = ee;
                    }
                    // 32 edges first (an early hit then costs no wider read), then 128 at a time
                    for (int step = 32; kk < ee; kk += step, step = 128) {
                        int32_t jf = 0;
                        const int pos = step == 32 ? warp_scan<1>(a.in_col, tbm, kk, ee, &jf)
                                                   : warp_scan<4>(a.in_col, tbm, kk, ee, &jf);
                        if (pos < step) {
                            if (!tf) {
                                tf = true;
                                tp = jf;
                            }
                            if (a.early_exit) {
                                tx += (unsigned long long)(pos + 1);
                                break;
                            }
                        }
                        tx += (unsigned long long)(ee - kk < step ? ee - kk : step);
                    }
                    if (lane == t) {
                        found[r] = tf;
                        par[r] = tp;
                        exam[r] += tx;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kPullIlp; ++r) {
                // new: found here, not by pass 1, and not visited before (rows without masking may be)
                const bool isnew = found[r] && !found1[r] && !((cwj[r] >> bitpos[r]) & 1u);
                if (isnew) {
                    atomicOr(snew + jw[r], 1u << bitpos[r]);
                    a.depth[i[r]] = L + 1;
                    if (a.parent) a.parent[i[r]] = par[r];
                    const int32_t od = a.symmetric ? end[r] - beg[r]
                                                   : __ldg(a.out_ptr + i[r] + 1) - __ldg(a.out_ptr + i[r]);
                    acc.n_new += 1;
                    acc.mf += (uint32_t)od;
                    acc.indeg += (uint32_t)(end[r] - beg[r]);
                }
                acc.exam += exam[r];
                if (append) st.put(isnew, i[r]);
            }
        }
        __syncwarp();
        if (wok) vnext[w] = cw | snew[lane];
        __syncwarp();
    }
    if (append) st.flush_block<kBfsThreads / 32>(bsm);
}

// The grid-wide phase of a pull level: warps take the listed long rows' edge
// chunks round-robin.  A row is claimed in the next visited bitmap by the first
// chunk that finds a parent (atomicOr), which writes its depth and parent.  With
// early exit a chunk records its first hit in hr.first (atomicMin) and chunks
// that start past a known hit are skipped; with exact_exam (traced runs) only
// those are, so that pull_huge_exam can count the edges a row-ordered scan
// examines, otherwise every chunk of a row with a known hit is.
#ifndef GBX_PULL_HUGE_INLINE
#define GBX_PULL_HUGE_INLINE __forceinline__
#endif
__device__ GBX_PULL_HUGE_INLINE void pull_huge(const BfsArgs& a, int32_t L, int cur, int vcur, int32_t entries,
                                               int32_t chunks, bool exact_exam, StageBuf* sb, LevelCtr* cout,
                                               unsigned long long* bsm, Acc& acc) {
    const int lane = threadIdx.x & 31;
    // everything below is rebuilt from the arguments so that little stays live across the level
    const bool use_fbm = !a.operand_reuse;
    const bool append = use_fbm;
    const HugeRows hr{a.q[cur], a.qp[cur], a.qd[cur], a.hfirst};
    Stage st{sb, 0, cout, a.q[cur ^ 1], a.qp[cur ^ 1], a.qd[cur ^ 1], a.out_ptr, a.in_ptr, 0, a.need_indeg, &acc};
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    const uint32_t* vprev = a.vis[vcur];
    uint32_t* vnext = a.vis[vcur ^ 1];
    const uint32_t* tbm = use_fbm ? a.fbm : vprev;
    for (int32_t c = gwarp; c < chunks; c += nwarps) {
        const int32_t e = warp_find_entry(hr.base, entries, c);
        const int32_t code = hr.row[e];
        const bool known = code < 0;
        const int32_t i = known ? ~code : code;
        const int32_t rend = __ldg(a.in_ptr + i + 1);
        const int32_t beg = hr.k[e] + (c - hr.base[e]) * kPullChunk;
        const int32_t end = rend - beg < kPullChunk ? rend : beg + kPullChunk;
        if (a.early_exit) {
            const int32_t fk = ld_volatile_i32(hr.first + e);
            if (exact_exam ? fk < beg : fk != INT32_MAX) continue;
        }
        // rows visited before this level (scanned only without masking) are never new
        const bool cand = !known && !bit_test(vprev, i);
        bool hit = false;
        int32_t par = -1, hit_at = 0;
        unsigned long long ex = 0;
        for (int32_t kk = beg; kk < end; kk += 128) {
            int32_t jf = 0;
            const int pos = warp_scan<4>(a.in_col, tbm, kk, end, &jf);
            if (pos < 128) {
                if (!hit) {
                    hit = true;
                    par = jf;
                    hit_at = kk + pos;
                }
                if (a.early_exit) break;
            }
            ex += (unsigned long long)(end - kk < 128 ? end - kk : 128);
        }
        bool isnew = false;
        int32_t od = 0;
        if (lane == 0) {
            if (a.early_exit) {
                if (hit) atomicMin(hr.first + e, hit_at);
            } else {
                acc.exam += ex;
            }
            if (hit && cand) {
                const uint32_t bit = 1u << (i & 31);
                isnew = !(atomicOr(vnext + (i >> 5), bit) & bit);
            }
            if (isnew) {
                const int32_t rbeg = __ldg(a.in_ptr + i);
                a.depth[i] = L + 1;
                if (a.parent) a.parent[i] = par;
                od = a.symmetric ? rend - rbeg : __ldg(a.out_ptr + i + 1) - __ldg(a.out_ptr + i);
                acc.n_new += 1;
                acc.mf += (uint32_t)od;
                acc.indeg += (uint32_t)(rend - rbeg);
            }
        }
        if (append) st.put(isnew && od > 0, i);
    }
    if (append) st.flush_block<kBfsThreads / 32>(bsm);
}

// Edges a row-ordered scan with early exit examines in the listed rows: up to
// and including the first hit, or all that were left after the tile phase.
__device__ __forceinline__ void pull_huge_exam(const BfsArgs& a, const HugeRows& hr, int32_t entries, Acc& acc) {
    const long long gtid = (long long)blockIdx.x * kBfsThreads + threadIdx.x;
    for (long long e = gtid; e < entries; e += (long long)gridDim.x * kBfsThreads) {
        const int32_t code = hr.row[e];
        const int32_t i = code < 0 ? ~code : code;
        const int32_t fk = hr.first[e];
        const int32_t stop = fk != INT32_MAX ? fk + 1 : __ldg(a.in_ptr + i + 1);
        acc.exam += (uint32_t)(stop - hr.k[e]);
    }
}

// DENSE2SPARSE at a pull -> push switch: F_{L+1} = visited now AND NOT visited before.
__device__ __forceinline__ void bitmap_to_queue(const BfsArgs& a, int vcur, Stage& st, unsigned long long* bsm) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    const int32_t ntiles = (a.nwords + 31) >> 5;
    for (int32_t tile = gwarp; tile < ntiles; tile += nwarps) {
        // lane l loads word tile*32 + l (coalesced), then the warp walks the nonempty words
        const int32_t wl = (tile << 5) + lane;
        const uint32_t mine = wl < a.nwords ? (a.vis[vcur][wl] & ~a.vis[vcur ^ 1][wl]) : 0u;
        uint32_t todo = __ballot_sync(0xffffffffu, mine != 0u);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t nw = __shfl_sync(0xffffffffu, mine, j);
            st.put((nw >> lane) & 1u, (((tile << 5) + j) << 5) + lane);
        }
    }
    st.flush_block<kBfsThreads / 32>(bsm);
}

// out[i] = fill for all i < n except out[special] = special_value; 16-byte stores when aligned.
__device__ __forceinline__ void fill_outputs(int32_t* out, int32_t n, int32_t fill, int32_t special,
                                             int32_t special_value, long long gtid, long long gstride) {
    if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
        const long long n4 = n >> 2;
        int4* o4 = reinterpret_cast<int4*>(out);
        for (long long q = gtid; q < n4; q += gstride) {
            int4 v = make_int4(fill, fill, fill, fill);
            const long long b = q << 2;
            if (special >= b && special < b + 4) {
                const int r = (int)(special - b);
                if (r == 0) v.x = special_value;
                if (r == 1) v.y = special_value;
                if (r == 2) v.z = special_value;
                if (r == 3) v.w = special_value;
            }
            o4[q] = v;
        }
        for (long long i = (n4 << 2) + gtid; i < n; i += gstride) out[i] = i == special ? special_value : fill;
    } else {
        for (long long i = gtid; i < n; i += gstride) out[i] = i == special ? special_value : fill;
    }
}

struct LoopState {
    unsigned long long qv;  // queue of the next level: entries (low 32 bits), out-degree sum (high 32)
    long long nf, mf, mu;   // |F_L|, out-edges of F_L, in-edges of the rows unvisited before level L
    unsigned long long t_mark;
    int next, stop;
};

// End of level L, by thread 0 of every block (all blocks read the same counters and
// decide alike): the trace record and the status words (block 0 only), the stop
// test, and the direction of level L + 1 (Section 6.3).
template <bool kTrace>
__device__ __forceinline__ void level_end(const BfsArgs& a, int32_t L, int dir, const unsigned long long* lvl,
                                          LoopState& ls) {
    const long long n_new = (long long)lvl[0];
    const long long mf_new = (long long)lvl[1];
    const long long in_new = (long long)lvl[2];
    const bool lead = blockIdx.x == 0;
    if (kTrace && lead && L < a.trace_cap) {
        LevelRec r;
        r.direction = dir;
        r.level = L;
        r.nf = ls.nf;
        r.mf = ls.mf;
        r.mu = ls.mu;
        r.e_exam = dir == DIR_PULL ? (long long)lvl[3] : -1;
        r.n_new = n_new;
        r.mf_new = mf_new;
        const unsigned long long now = global_timer_ns();
        r.t_ns = (long long)(now - ls.t_mark);
        ls.t_mark = now;
        a.trace[L] = r;
    }
    if (n_new == 0) {
        if (lead) a.status[ST_LEVELS] = L + 1;
        ls.stop = 1;
        return;
    }
    if (L + 1 >= a.n) {  // a BFS has at most n levels; more means corrupted state
        if (lead) atomicCAS(a.status + ST_ERROR, 0, (int)GBX_ERR_OVERFLOW);
        ls.stop = 1;
        return;
    }
    int next = dir;
    if (a.mode == GBX_DIR_AUTO) {
        const double r_new = (double)n_new / (double)a.n;
        if (dir == DIR_PUSH) {
            if (a.heuristic == GBX_HEUR_RATIO) {
                if (r_new > (double)a.alpha && n_new > ls.nf) next = DIR_PULL;
            } else {
                const long long mu_next = ls.mu - in_new;
                if (mu_next > 0 && (double)mf_new / (double)mu_next > (double)a.alpha) next = DIR_PULL;
            }
        } else if (r_new < (double)a.beta && (a.heuristic != GBX_HEUR_RATIO || n_new < ls.nf)) {
            // the ratio rule also wants r decreasing; Beamer's way back is r < beta alone
            next = DIR_PUSH;
        }
    }
    ls.next = next;
    ls.qv = lvl[4];
    ls.mu -= in_new;
    ls.nf = n_new;
    ls.mf = mf_new;
}

// kHuge: long pull rows go to the grid-wide phase.  Launched for runs that
// expect full row scans (no early exit, or pull on every level); with the
// direction rule and early exit a pull level rarely meets a long row without a
// parent, and those runs keep the kernel without that phase (fewer registers).
template <bool kTrace, bool kHuge>
__global__ void __launch_bounds__(kBfsThreads, kBfsMinBlocks) bfs_kernel(BfsArgs a) {
    const long long gtid = (long long)blockIdx.x * kBfsThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kBfsThreads;
    const int32_t s = a.source;
    // an error of an earlier launch not yet read by the host: this launch does nothing
    const int pending = threadIdx.x == 0 ? ld_volatile_i32(a.status + ST_ERROR) : 0;
    unsigned long long t_mark = kTrace && gtid == 0 ? global_timer_ns() : 0ull;
    // Algorithm 1, lines 2-5: f = e_s, v = {s}; outputs initialised.  When level 0 pushes,
    // its claims (the source's out-neighbours, all new) write no outputs, so the outputs
    // are initialised during level 0 instead, hidden behind its latency, and level 1
    // starts by stamping the source's out-neighbours (depth 1, parent s).
    const bool fill_in_level0 = a.mode != GBX_DIR_PULL;
    if (!fill_in_level0) {
        fill_outputs(a.depth, a.n, -1, s, 0, gtid, gstride);
        if (a.parent) fill_outputs(a.parent, a.n, -1, s, s, gtid, gstride);
    }
    for (long long w = gtid; w < a.nwords; w += gstride) a.vis[0][w] = w == (s >> 5) ? 1u << (s & 31) : 0u;
    const int32_t s_rs = __ldg(a.out_ptr + s);
    const int32_t s_od = __ldg(a.out_ptr + s + 1) - s_rs;
    const int32_t s_id = __ldg(a.in_ptr + s + 1) - __ldg(a.in_ptr + s);
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
        z.n_new = 1;
        z.mf_new = (unsigned long long)s_od;
        a.ctr[0] = z;
        a.status[ST_LEVELS] = 0;
        a.bar->count[a.bar_parity ^ 1u] = 0u;  // the next launch's counter
    }
    unsigned int* barc = a.bar->count + a.bar_parity;
    unsigned int bar_round = 0;
    if (__syncthreads_or(pending)) return;
    if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;

    __shared__ StageBuf stage_mem[kBfsThreads / 32];
    __shared__ uint32_t tile_new[kBfsThreads / 32][32];
    __shared__ uint16_t tile_list[kBfsThreads / 32][1024];  // a pull tile's candidate rows (offsets in the tile)
    __shared__ unsigned long long lvl[6];  // counters of the level just finished, read once per block
    __shared__ unsigned long long acc_mem[kBfsThreads / 32][4];  // per-warp counts before the block's atomics
    __shared__ unsigned long long stage_sum[kBfsThreads / 32];   // per-warp queue ranges of a block flush
    // block-uniform loop state, kept by thread 0 in shared memory rather than in every
    // thread's registers (which the level code needs)
    __shared__ LoopState ls;
    const int wib = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        ls.qv = s_od > 0 ? (((unsigned long long)s_od << 32) | 1ull) : 0ull;
        ls.nf = 1;
        ls.mf = s_od;
        ls.mu = a.nnz - s_id;
        ls.t_mark = t_mark;
        ls.next = 0;
        ls.stop = 0;
    }
    __syncthreads();
    int dir = a.mode == GBX_DIR_PULL ? DIR_PULL : DIR_PUSH;
    int cur = 0, vcur = 0;
    for (int32_t L = 0;; ++L) {
        LevelCtr* cout = a.ctr + ((L + 1) % 3);
        if (gtid == 0) {
            LevelCtr z = {};
            a.ctr[(L + 2) % 3] = z;
        }
        const unsigned long long qv = ls.qv;
        const uint32_t qcount = (uint32_t)qv, qedges = (uint32_t)(qv >> 32);
        Acc acc;
        bool appended;
        Stage st{stage_mem + wib, 0, cout, a.q[cur ^ 1], a.qp[cur ^ 1], a.qd[cur ^ 1],
                 a.out_ptr, a.in_ptr, dir == DIR_PUSH, a.need_indeg, &acc};
        if (dir == DIR_PUSH) {
            const bool first = L == 0 && fill_in_level0;
            push_level(a, L, cur, vcur, qcount, qedges, st, stage_sum, acc, !first);
            if (first) {
                fill_outputs(a.depth, a.n, -1, s, 0, gtid, gstride);
                if (a.parent) fill_outputs(a.parent, a.n, -1, s, s, gtid, gstride);
            }
            appended = true;
        } else {
            const bool use_fbm = !a.operand_reuse;
            if (use_fbm) {
                // frontier bitmap of F_L from its queue (vertices without out-edges cannot be parents)
                for (long long w = gtid; w < a.nwords; w += gstride) a.fbm[w] = 0u;
                if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
                for (long long k = gtid; k < qcount; k += gstride) {
                    const int32_t v = a.q[cur][k];
                    atomicOr(a.fbm + (v >> 5), 1u << (v & 31));
                }
                if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
            }
            appended = use_fbm;
            pull_level<kHuge>(a, L, vcur, use_fbm, appended, HugeRows{a.q[cur], a.qp[cur], a.qd[cur], a.hfirst}, st,
                              stage_sum, tile_new[wib], tile_list[wib], acc);
        }
        flush_acc(acc, cout, kTrace, acc_mem);
        if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
        if (threadIdx.x == 0) {
            lvl[0] = ld_volatile_u64(&cout->n_new);
            lvl[1] = ld_volatile_u64(&cout->mf_new);
            lvl[2] = ld_volatile_u64(&cout->indeg_new);
            lvl[3] = ld_volatile_u64(&cout->e_exam);
            lvl[4] = ld_volatile_u64(&cout->q);
            lvl[5] = kHuge ? ld_volatile_u64(&cout->huge) : 0ull;
        }
        __syncthreads();
        if (kHuge && lvl[5] != 0ull) {  // the pull level listed long rows: the grid scans them now
            const int32_t entries = (int32_t)(uint32_t)lvl[5];
            Acc acc2;
            pull_huge(a, L, cur, vcur, entries, (int32_t)(lvl[5] >> 32), kTrace, stage_mem + wib, cout, stage_sum,
                      acc2);
            flush_acc(acc2, cout, kTrace, acc_mem);
            if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
            if (kTrace && a.early_exit) {
                Acc acc3;
                pull_huge_exam(a, HugeRows{a.q[cur], a.qp[cur], a.qd[cur], a.hfirst}, entries, acc3);
                flush_acc(acc3, cout, true, acc_mem);
                if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
            }
            if (threadIdx.x == 0) {
                lvl[0] = ld_volatile_u64(&cout->n_new);
                lvl[1] = ld_volatile_u64(&cout->mf_new);
                lvl[2] = ld_volatile_u64(&cout->indeg_new);
                lvl[3] = ld_volatile_u64(&cout->e_exam);
                lvl[4] = ld_volatile_u64(&cout->q);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) level_end<kTrace>(a, L, dir, lvl, ls);
        __syncthreads();
        if (ls.stop) return;
        if (L == 0 && fill_in_level0) {  // the outputs are initialised everywhere now
            for (long long k = gtid; k < s_od; k += gstride) {
                const int32_t v = __ldg(a.out_col + s_rs + k);
                if (v != s) {
                    a.depth[v] = 1;
                    if (a.parent) a.parent[v] = s;
                }
            }
        }
        const int next = ls.next;
        if (dir == DIR_PULL) vcur ^= 1;
        if (dir == DIR_PULL && next == DIR_PUSH && !appended) {
            bitmap_to_queue(a, vcur, st, stage_sum);
            if (!grid_barrier(barc, gridDim.x, bar_round, a.status, a.timeout_ns)) return;
            if (threadIdx.x == 0) ls.qv = ld_volatile_u64(&cout->q);
            __syncthreads();
        }
        cur ^= 1;
        dir = next;
    }
}

// ---------------------------------------------------------------- host side

static std::atomic<unsigned long long> g_timeout_ns{5000000000ull};

uint64_t wait_timeout_ns() { return g_timeout_ns.load(); }

static gbx_status check_desc(const gbx_desc* d) {
    GBX_CHECK(d->direction >= GBX_DIR_AUTO && d->direction <= GBX_DIR_PULL, GBX_ERR_INVALID_VALUE, "desc.direction");
    GBX_CHECK(d->heuristic == GBX_HEUR_RATIO || d->heuristic == GBX_HEUR_BEAMER, GBX_ERR_INVALID_VALUE,
              "desc.heuristic");
    GBX_CHECK(d->alpha >= 0.0f && d->beta >= 0.0f && d->alpha == d->alpha && d->beta == d->beta,
              GBX_ERR_INVALID_VALUE, "desc.alpha / desc.beta must be >= 0");
    GBX_CHECK(d->pull_probe == 0 || (d->pull_probe >= 4 && d->pull_probe <= 1024), GBX_ERR_INVALID_VALUE,
              "desc.pull_probe must be 0 or in [4, 1024]");
    GBX_CHECK(d->blocks_per_sm >= 0, GBX_ERR_INVALID_VALUE, "desc.blocks_per_sm must be >= 0");
    GBX_CHECK(d->push_sort == 0, GBX_ERR_NOT_SUPPORTED, "desc.push_sort applies to gbx_mxv only");
    for (int k = 0; k < 2; ++k) GBX_CHECK(d->reserved[k] == 0, GBX_ERR_INVALID_VALUE, "desc.reserved must be 0");
    return GBX_OK;
}

static gbx_status bfs_geometry(Graph* G) {
    if (G->bfs_blocks > 0) return GBX_OK;  // blocks per SM that fit (cached per graph)
    const void* fns[] = {(const void*)bfs_kernel<false, false>, (const void*)bfs_kernel<true, false>,
                         (const void*)bfs_kernel<false, true>, (const void*)bfs_kernel<true, true>};
    int per_sm = 1 << 30;
    for (const void* fn : fns) {
        int b = 0;
        GBX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kBfsThreads, 0));
        per_sm = b < per_sm ? b : per_sm;
    }
    GBX_CHECK(per_sm >= 1, GBX_ERR_CUDA, "BFS kernel cannot be resident");
    G->bfs_blocks = per_sm;
    return GBX_OK;
}

static gbx_status launch_bfs(Graph* G, int32_t source, int32_t* depth, int32_t* parent, const gbx_desc& d,
                             cudaStream_t s) {
    GBX_TRY(bfs_geometry(G));
    BfsArgs a;
    a.n = G->n;
    a.nwords = G->nwords;
    a.source = source;
    a.nnz = G->nnz;
    a.out_ptr = G->out_ptr;
    a.out_col = G->out_col;
    a.in_ptr = G->in_ptr;
    a.in_col = G->in_col;
    a.nz_in = G->nz_in;
    a.multi_in = G->multi_in;
    a.first_in = G->first_in;
    a.next_in = G->next_in;
    a.depth = depth;
    a.parent = parent;
    a.vis[0] = G->ws.bm[0];
    a.vis[1] = G->ws.bm[1];
    a.fbm = G->ws.bm[2];
    a.hfirst = G->ws.list;
    for (int i = 0; i < 2; ++i) {
        a.q[i] = G->ws.q[i];
        a.qp[i] = G->ws.qp[i];
        a.qd[i] = G->ws.qd[i];
    }
    a.ctr = G->ws.ctr;
    a.bar = G->ws.bar;
    a.trace = G->ws.trace;
    a.status = G->ws.status;
    a.alpha = d.alpha;
    a.beta = d.beta;
    a.heuristic = d.heuristic;
    a.mode = d.direction;
    a.early_exit = d.early_exit ? 1 : 0;
    a.masking = d.masking ? 1 : 0;
    a.operand_reuse = d.operand_reuse ? 1 : 0;
    a.symmetric = G->symmetric;
    a.need_indeg = (!G->symmetric && (d.trace || d.heuristic == GBX_HEUR_BEAMER)) ? 1 : 0;
    a.need_deg = (d.trace || d.heuristic == GBX_HEUR_BEAMER) ? 1 : 0;  // m_f and m_u of the found rows
    a.trace_cap = kTraceCap;
    a.probe = d.pull_probe > 0 ? (d.pull_probe + 3) / 4 * 4 : kProbe;
    a.timeout_ns = wait_timeout_ns();
    a.bar_parity = G->ws.bar_parity;
    void* args[] = {&a};
    const bool huge = !d.early_exit || d.direction == GBX_DIR_PULL;
    const void* fn = d.trace ? (huge ? (const void*)bfs_kernel<true, true> : (const void*)bfs_kernel<true, false>)
                             : (huge ? (const void*)bfs_kernel<false, true> : (const void*)bfs_kernel<false, false>);
    const int per_sm = d.blocks_per_sm > 0 && d.blocks_per_sm < G->bfs_blocks ? d.blocks_per_sm : G->bfs_blocks;
    a.tile_words = pull_tile_words(G->nwords, (long long)per_sm * G->num_sms * (kBfsThreads / 32));
    GBX_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(per_sm * G->num_sms), dim3(kBfsThreads), args, 0, s));
    G->ws.bar_parity ^= 1u;
    G->ws.last_stream = s;
    G->ws.last_traced = d.trace ? 1 : 0;
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

namespace gbx {
// One participant short: nobody ever completes the barrier, every block times out.
__global__ void selftest_barrier_kernel(GridBar* bar, unsigned int parity, int32_t* status,
                                        unsigned long long timeout_ns) {
    if (blockIdx.x == 0 && threadIdx.x == 0) bar->count[parity ^ 1u] = 0u;
    unsigned int round = 0;
    grid_barrier(bar->count + parity, gridDim.x + 1, round, status, timeout_ns);
}
}  // namespace gbx

extern "C" gbx_status gbx_selftest_barrier_timeout(gbx_graph* g, uint64_t timeout_ns, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    selftest_barrier_kernel<<<4, 32, 0, (cudaStream_t)stream>>>(G->ws.bar, G->ws.bar_parity, G->ws.status,
                                                                 (unsigned long long)timeout_ns);
    G->ws.bar_parity ^= 1u;
    GBX_CUDA_TRY(cudaGetLastError());
    G->ws.last_stream = (cudaStream_t)stream;
    return GBX_OK;
}

extern "C" gbx_status gbx_set_wait_timeout_ns(uint64_t ns) {
    clear_error();
    g_timeout_ns.store(ns);
    return GBX_OK;
}

extern "C" gbx_status gbx_bfs(gbx_graph* g, int32_t source, int32_t* depth, int32_t* parent, const gbx_desc* desc,
                              void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    GBX_CHECK(depth != nullptr, GBX_ERR_NULL_POINTER, "depth is NULL");
    GBX_CHECK(source >= 0 && source < G->n, GBX_ERR_INVALID_INDEX, "source outside [0, n)");
    gbx_desc d;
    if (desc)
        d = *desc;
    else
        gbx_desc_init(&d);
    GBX_TRY(check_desc(&d));
    return launch_bfs(G, source, depth, parent, d, (cudaStream_t)stream);
}

extern "C" gbx_status gbx_bfs_host(gbx_graph* g, const int32_t* sources, int32_t count, int32_t* depth_host,
                                   int32_t* parent_host, const gbx_desc* desc, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    GBX_CHECK(count >= 0, GBX_ERR_INVALID_VALUE, "count < 0");
    GBX_CHECK(count == 0 || (sources && depth_host), GBX_ERR_NULL_POINTER, "sources or depth_host is NULL");
    for (int32_t k = 0; k < count; ++k)
        GBX_CHECK(sources[k] >= 0 && sources[k] < G->n, GBX_ERR_INVALID_INDEX, "source outside [0, n)");
    gbx_desc d;
    if (desc)
        d = *desc;
    else
        gbx_desc_init(&d);
    GBX_TRY(check_desc(&d));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(int32_t) * (size_t)G->n;
    if (!G->copy_stream) {
        // all or nothing: a partial setup would leave null buffers behind a live copy stream
        cudaStream_t cs = nullptr;
        int32_t* buf[4] = {nullptr, nullptr, nullptr, nullptr};  // depth 0, 1, parent 0, 1
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // done 0, 1, copied 0, 1
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc((void**)&buf[i], bytes);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        for (int i = 2; i < 4 && e == cudaSuccess; ++i) e = cudaEventRecord(ev[i], cs);
        if (e != cudaSuccess) {
            for (int i = 0; i < 4; ++i) {
                if (buf[i]) cudaFree(buf[i]);
                if (ev[i]) cudaEventDestroy(ev[i]);
            }
            if (cs) cudaStreamDestroy(cs);
            GBX_CUDA_TRY(e);
        }
        for (int i = 0; i < 2; ++i) {
            G->hdepth[i] = buf[i];
            G->hparent[i] = buf[2 + i];
            G->ev_done[i] = ev[i];
            G->ev_copied[i] = ev[2 + i];
        }
        G->copy_stream = cs;
    }
    for (int32_t k = 0; k < count; ++k) {
        const int b = k & 1;
        // the device buffer set b is free once its previous copy has finished
        GBX_CUDA_TRY(cudaStreamWaitEvent(s, G->ev_copied[b], 0));
        GBX_TRY(launch_bfs(G, sources[k], G->hdepth[b], parent_host ? G->hparent[b] : nullptr, d, s));
        GBX_CUDA_TRY(cudaEventRecord(G->ev_done[b], s));
        GBX_CUDA_TRY(cudaStreamWaitEvent(G->copy_stream, G->ev_done[b], 0));
        GBX_CUDA_TRY(cudaMemcpyAsync(depth_host + (size_t)k * G->n, G->hdepth[b], bytes, cudaMemcpyDeviceToHost,
                                     G->copy_stream));
        if (parent_host)
            GBX_CUDA_TRY(cudaMemcpyAsync(parent_host + (size_t)k * G->n, G->hparent[b], bytes,
                                         cudaMemcpyDeviceToHost, G->copy_stream));
        GBX_CUDA_TRY(cudaEventRecord(G->ev_copied[b], G->copy_stream));
    }
    GBX_CUDA_TRY(cudaStreamSynchronize(G->copy_stream));
    return gbx_graph_sync(g, stream);
}

extern "C" gbx_status gbx_bfs_trace(gbx_graph* g, gbx_level* levels, int32_t cap, int32_t* nlevels) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    GBX_CHECK(nlevels != nullptr, GBX_ERR_NULL_POINTER, "nlevels is NULL");
    GBX_CHECK(cap == 0 || levels != nullptr, GBX_ERR_NULL_POINTER, "levels is NULL");
    GBX_CHECK(G->ws.last_traced, GBX_ERR_INVALID_VALUE, "the last BFS on this graph was not traced");
    if (G->ws.last_stream) GBX_CUDA_TRY(cudaStreamSynchronize(G->ws.last_stream));
    GBX_CUDA_TRY(cudaDeviceSynchronize());
    int32_t st[ST_WORDS];
    GBX_CUDA_TRY(cudaMemcpy(st, G->ws.status, sizeof(st), cudaMemcpyDeviceToHost));
    GBX_CHECK(st[ST_ERROR] == 0, (gbx_status)st[ST_ERROR], "the last BFS recorded a device-side error");
    const int32_t L = st[ST_LEVELS] < kTraceCap ? st[ST_LEVELS] : kTraceCap;
    *nlevels = st[ST_LEVELS];
    const int32_t ncopy = L < cap ? L : cap;
    if (ncopy <= 0) return GBX_OK;
    LevelRec* recs = new LevelRec[ncopy];
    const cudaError_t e = cudaMemcpy(recs, G->ws.trace, sizeof(LevelRec) * ncopy, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] recs;
        GBX_CUDA_TRY(e);
    }
    // unvisited counts follow from the frontier sizes: U_L = n - |F_0 u ... u F_L|;
    // every vertex found after level 0 was reached over an in-edge
    int64_t visited = 0;
    int64_t nz_total = 0;
    {
        int32_t* words = new int32_t[G->nwords];
        const cudaError_t e2 = cudaMemcpy(words, G->nz_in, sizeof(uint32_t) * G->nwords, cudaMemcpyDeviceToHost);
        if (e2 != cudaSuccess) {
            delete[] words;
            delete[] recs;
            GBX_CUDA_TRY(e2);
        }
        for (int32_t w = 0; w < G->nwords; ++w) nz_total += __builtin_popcount((uint32_t)words[w]);
        delete[] words;
    }
    const int64_t src_nz = (recs[0].mu != G->nnz) ? 1 : 0;  // mu_0 = nnz - indeg(source)
    int64_t found_after_0 = 0;
    for (int32_t l = 0; l < ncopy; ++l) {
        const LevelRec& r = recs[l];
        visited += r.nf;
        if (l > 0) found_after_0 += r.nf;
        gbx_level o;
        o.direction = r.direction;
        o.level = r.level;
        o.nf = r.nf;
        o.mf = r.mf;
        o.nu = (int64_t)G->n - visited;
        o.nu_nz = nz_total - src_nz - found_after_0;
        o.mu = r.mu;
        o.e_exam = r.e_exam;
        o.n_new = r.n_new;
        o.mf_new = r.mf_new;
        o.time_ns = r.t_ns;
        levels[l] = o;
    }
    delete[] recs;
    return GBX_OK;
}
