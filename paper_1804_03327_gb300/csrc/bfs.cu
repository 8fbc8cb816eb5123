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

#include "gbx_internal.cuh"

namespace gbx {

constexpr int kBfsThreads = 256;
constexpr int kBfsMinBlocks = 4;
constexpr int kProbe = 16;  // in-neighbours one lane examines before the warp takes over the row
enum { DIR_PUSH = GBX_DIR_PUSH, DIR_PULL = GBX_DIR_PULL };

struct BfsArgs {
    int32_t n, nwords, source;
    long long nnz;
    const int32_t* out_ptr;
    const int32_t* out_col;
    const int32_t* in_ptr;
    const int32_t* in_col;
    const uint32_t* nz_in;
    int32_t* depth;
    int32_t* parent;
    uint32_t* vis[2];
    uint32_t* fbm;
    int32_t* q[2];
    int32_t* qp[2];
    int32_t* qd[2];
    LevelCtr* ctr;
    GridBar* bar;
    LevelRec* trace;
    int32_t* status;
    float alpha, beta;
    int32_t heuristic, mode, early_exit, masking, operand_reuse, symmetric, need_indeg, trace_cap;
    unsigned long long timeout_ns;
};

struct Acc {
    unsigned long long n_new = 0, mf = 0, indeg = 0, exam = 0;
};

// Append the lanes with `take` to the next frontier queue.  One packed 64-bit
// atomic per warp reserves both the queue slots and the out-degree prefix.
__device__ __forceinline__ void warp_append(bool take, int32_t v, int32_t rs, int32_t od, LevelCtr* cout, int32_t* nq,
                                            int32_t* nqp, int32_t* nqd) {
    const uint32_t app = __ballot_sync(0xffffffffu, take);
    if (!app) return;
    const uint32_t inc = warp_inclusive_sum(take ? (uint32_t)od : 0u);
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
    unsigned long long old = 0;
    if ((threadIdx.x & 31) == 0) old = atomicAdd(&cout->q, ((unsigned long long)tot << 32) | (unsigned long long)__popc(app));
    old = __shfl_sync(0xffffffffu, old, 0);
    if (take) {
        const int32_t pos = (int32_t)(uint32_t)old + __popc(app & lanemask_lt());
        const int32_t pre = (int32_t)(old >> 32) + (int32_t)(inc - (uint32_t)od);
        nq[pos] = v;
        nqp[pos] = pre;
        nqd[pos] = rs - pre;
    }
}

// Largest k in [0, count) with qp[k] <= e (qp ascending, qp[0] = 0).
__device__ __forceinline__ int32_t find_entry(const int32_t* qp, int32_t count, long long e) {
    int32_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((long long)qp[mid] <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void flush_acc(const Acc& acc, LevelCtr* cout, bool with_exam) {
    const unsigned long long a = warp_sum_u64(acc.n_new);
    const unsigned long long b = warp_sum_u64(acc.mf);
    const unsigned long long c = warp_sum_u64(acc.indeg);
    const unsigned long long d = with_exam ? warp_sum_u64(acc.exam) : 0ull;
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&cout->n_new, a);
        if (b) atomicAdd(&cout->mf_new, b);
        if (c) atomicAdd(&cout->indeg_new, c);
        if (d) atomicAdd(&cout->e_exam, d);
    }
}

// ---------------------------------------------------------------- push (Eq 5)

__device__ __forceinline__ void push_level(const BfsArgs& a, int32_t L, int cur, int vcur, uint32_t qcount,
                                           uint32_t qedges, LevelCtr* cout, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    const int32_t* q = a.q[cur];
    const int32_t* qp = a.qp[cur];
    const int32_t* qd = a.qd[cur];
    int32_t* nq = a.q[cur ^ 1];
    int32_t* nqp = a.qp[cur ^ 1];
    int32_t* nqd = a.qd[cur ^ 1];
    uint32_t* vis = a.vis[vcur];
    const long long E = qedges;
    long long chunk = (E + nwarps - 1) / nwarps;
    chunk = chunk < 64 ? 64 : ((chunk + 31) & ~31ll);
    for (long long e0 = (long long)gwarp * chunk; e0 < E; e0 += (long long)nwarps * chunk) {
        const long long e1 = e0 + chunk < E ? e0 + chunk : E;
        int32_t k = 0;
        if (lane == 0) k = find_entry(qp, (int32_t)qcount, e0);
        k = __shfl_sync(0xffffffffu, k, 0);
        for (long long base = e0; base < e1; base += 32) {
            // queue entries whose edge ranges start inside [base, base + 32)
            const int32_t wi = k + 1 + lane;
            const long long bnd = wi < (int32_t)qcount ? (long long)qp[wi] : (long long)INT64_MAX;
            const long long rel = bnd - base;
            const uint32_t bits = __reduce_or_sync(0xffffffffu, (rel >= 0 && rel < 32) ? (1u << (int)rel) : 0u);
            const long long e = base + lane;
            bool claimed = false;
            int32_t u = 0, v = 0;
            if (e < e1) {
                const int32_t kk = k + __popc(bits & (0xffffffffu >> (31 - lane)));
                u = q[kk];
                v = __ldg(a.out_col + (e + qd[kk]));
                const uint32_t bit = 1u << (v & 31);
                uint32_t* wp = vis + (v >> 5);
                if (!(__ldcg(wp) & bit)) claimed = !(atomicOr(wp, bit) & bit);
            }
            int32_t rs = 0, od = 0;
            if (claimed) {
                a.depth[v] = L + 1;
                if (a.parent) a.parent[v] = u;
                rs = __ldg(a.out_ptr + v);
                od = __ldg(a.out_ptr + v + 1) - rs;
                acc.n_new += 1;
                acc.mf += (unsigned long long)od;
                if (a.need_indeg)
                    acc.indeg += (unsigned long long)(__ldg(a.in_ptr + v + 1) - __ldg(a.in_ptr + v));
                else
                    acc.indeg += (unsigned long long)od;
            }
            warp_append(claimed && od > 0, v, rs, od, cout, nq, nqp, nqd);
            k += __popc(bits);
        }
    }
}

// ---------------------------------------------------------------- pull (Eq 4, Algorithm 2)

__device__ __forceinline__ void pull_level(const BfsArgs& a, int32_t L, int cur, int vcur, bool use_fbm, bool append,
                                           LevelCtr* cout, Acc& acc) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    const uint32_t* vprev = a.vis[vcur];
    uint32_t* vnext = a.vis[vcur ^ 1];
    const uint32_t* tbm = use_fbm ? a.fbm : vprev;
    int32_t* nq = a.q[cur ^ 1];
    int32_t* nqp = a.qp[cur ^ 1];
    int32_t* nqd = a.qd[cur ^ 1];
    for (int32_t w = gwarp; w < a.nwords; w += nwarps) {
        const uint32_t cw = vprev[w];
        const uint32_t nz = a.nz_in[w];
        const uint32_t cand = a.masking ? (~cw & nz) : nz;
        if (cand == 0) {
            if (lane == 0) vnext[w] = cw;
            continue;
        }
        const int32_t i = (w << 5) + lane;
        const bool mine = (cand >> lane) & 1u;
        int32_t beg = 0, end = 0, k = 0, par = -1;
        bool found = false, done = false;
        unsigned long long exam = 0;
        if (mine) {
            beg = __ldg(a.in_ptr + i);
            end = __ldg(a.in_ptr + i + 1);
            k = beg;
            const int32_t lim = end < beg + kProbe ? end : beg + kProbe;
            while (k < lim) {
                const int32_t cnt = lim - k < 4 ? lim - k : 4;
                const int32_t j0 = __ldg(a.in_col + k);
                const int32_t j1 = cnt > 1 ? __ldg(a.in_col + k + 1) : j0;
                const int32_t j2 = cnt > 2 ? __ldg(a.in_col + k + 2) : j0;
                const int32_t j3 = cnt > 3 ? __ldg(a.in_col + k + 3) : j0;
                const bool h0 = bit_test(tbm, j0);
                const bool h1 = cnt > 1 && bit_test(tbm, j1);
                const bool h2 = cnt > 2 && bit_test(tbm, j2);
                const bool h3 = cnt > 3 && bit_test(tbm, j3);
                if (!found && (h0 | h1 | h2 | h3)) {
                    const int hit = h0 ? 0 : (h1 ? 1 : (h2 ? 2 : 3));
                    found = true;
                    par = hit == 0 ? j0 : (hit == 1 ? j1 : (hit == 2 ? j2 : j3));
                    if (a.early_exit) {
                        exam += (unsigned long long)(hit + 1);
                        k += hit + 1;
                        done = true;
                        break;
                    }
                }
                exam += (unsigned long long)cnt;
                k += cnt;
            }
        }
        // rows longer than the lane probe: the whole warp scans them 32 at a time
        uint32_t pend = __ballot_sync(0xffffffffu, mine && !done && k < end);
        while (pend) {
            const int t = __ffs(pend) - 1;
            pend &= pend - 1;
            int32_t kk = __shfl_sync(0xffffffffu, k, t);
            const int32_t ee = __shfl_sync(0xffffffffu, end, t);
            bool tf = __shfl_sync(0xffffffffu, found, t);
            int32_t tp = __shfl_sync(0xffffffffu, par, t);
            unsigned long long tx = 0;
            for (; kk < ee; kk += 32) {
                const int32_t idx = kk + lane;
                const int32_t j = idx < ee ? __ldg(a.in_col + idx) : 0;
                const uint32_t hb = __ballot_sync(0xffffffffu, idx < ee && bit_test(tbm, j));
                if (hb) {
                    const int f = __ffs(hb) - 1;
                    const int32_t jf = __shfl_sync(0xffffffffu, j, f);
                    if (!tf) {
                        tf = true;
                        tp = jf;
                    }
                    if (a.early_exit) {
                        tx += (unsigned long long)(f + 1);
                        break;
                    }
                }
                tx += (unsigned long long)(ee - kk < 32 ? ee - kk : 32);
            }
            if (lane == t) {
                found = tf;
                par = tp;
                exam += tx;
            }
        }
        const uint32_t fmask = __ballot_sync(0xffffffffu, found);
        const uint32_t newm = fmask & ~cw;
        if (lane == 0) vnext[w] = cw | newm;
        const bool isnew = (newm >> lane) & 1u;
        int32_t rs = 0, od = 0;
        if (isnew) {
            a.depth[i] = L + 1;
            if (a.parent) a.parent[i] = par;
            if (a.symmetric) {
                rs = beg;
                od = end - beg;
            } else {
                rs = __ldg(a.out_ptr + i);
                od = __ldg(a.out_ptr + i + 1) - rs;
            }
            acc.n_new += 1;
            acc.mf += (unsigned long long)od;
            acc.indeg += (unsigned long long)(end - beg);
        }
        acc.exam += exam;
        if (append) warp_append(isnew && od > 0, i, rs, od, cout, nq, nqp, nqd);
    }
}

// DENSE2SPARSE at a pull -> push switch: F_{L+1} = visited now AND NOT visited before.
__device__ __forceinline__ void bitmap_to_queue(const BfsArgs& a, int cur, int vcur, LevelCtr* cout) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * kBfsThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * kBfsThreads) >> 5);
    for (int32_t w = gwarp; w < a.nwords; w += nwarps) {
        const uint32_t nw = a.vis[vcur][w] & ~a.vis[vcur ^ 1][w];
        if (!nw) continue;
        const int32_t i = (w << 5) + lane;
        const bool isnew = (nw >> lane) & 1u;
        int32_t rs = 0, od = 0;
        if (isnew) {
            rs = __ldg(a.out_ptr + i);
            od = __ldg(a.out_ptr + i + 1) - rs;
        }
        warp_append(isnew && od > 0, i, rs, od, cout, a.q[cur ^ 1], a.qp[cur ^ 1], a.qd[cur ^ 1]);
    }
}

template <bool kTrace>
__global__ void __launch_bounds__(kBfsThreads, kBfsMinBlocks) bfs_kernel(BfsArgs a) {
    const long long gtid = (long long)blockIdx.x * kBfsThreads + threadIdx.x;
    const long long gstride = (long long)gridDim.x * kBfsThreads;
    const int32_t s = a.source;
    // Algorithm 1, lines 2-5: f = e_s, v = {s}; outputs initialised
    for (long long i = gtid; i < a.n; i += gstride) {
        a.depth[i] = i == s ? 0 : -1;
        if (a.parent) a.parent[i] = i == s ? s : -1;
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
    }
    if (!grid_barrier(a.bar, gridDim.x, a.status, a.timeout_ns)) return;

    int dir = a.mode == GBX_DIR_PULL ? DIR_PULL : DIR_PUSH;
    int cur = 0, vcur = 0;
    long long nf = 1, mf = s_od, mu = a.nnz - s_id;
    for (int32_t L = 0;; ++L) {
        LevelCtr* cin = a.ctr + (L % 3);
        LevelCtr* cout = a.ctr + ((L + 1) % 3);
        if (gtid == 0) {
            LevelCtr z = {};
            a.ctr[(L + 2) % 3] = z;
        }
        const unsigned long long qv = ld_volatile_u64(&cin->q);
        const uint32_t qcount = (uint32_t)qv, qedges = (uint32_t)(qv >> 32);
        Acc acc;
        bool appended;
        if (dir == DIR_PUSH) {
            push_level(a, L, cur, vcur, qcount, qedges, cout, acc);
            appended = true;
        } else {
            const bool use_fbm = !a.operand_reuse;
            if (use_fbm) {
                // frontier bitmap of F_L from its queue (vertices without out-edges cannot be parents)
                for (long long w = gtid; w < a.nwords; w += gstride) a.fbm[w] = 0u;
                if (!grid_barrier(a.bar, gridDim.x, a.status, a.timeout_ns)) return;
                for (long long k = gtid; k < qcount; k += gstride) {
                    const int32_t v = a.q[cur][k];
                    atomicOr(a.fbm + (v >> 5), 1u << (v & 31));
                }
                if (!grid_barrier(a.bar, gridDim.x, a.status, a.timeout_ns)) return;
            }
            appended = use_fbm;
            pull_level(a, L, cur, vcur, use_fbm, appended, cout, acc);
        }
        flush_acc(acc, cout, kTrace);
        if (!grid_barrier(a.bar, gridDim.x, a.status, a.timeout_ns)) return;
        const long long n_new = (long long)ld_volatile_u64(&cout->n_new);
        const long long mf_new = (long long)ld_volatile_u64(&cout->mf_new);
        const long long in_new = (long long)ld_volatile_u64(&cout->indeg_new);
        if (kTrace && gtid == 0 && L < a.trace_cap) {
            LevelRec r;
            r.direction = dir;
            r.level = L;
            r.nf = nf;
            r.mf = mf;
            r.mu = mu;
            r.e_exam = dir == DIR_PULL ? (long long)ld_volatile_u64(&cout->e_exam) : -1;
            r.n_new = n_new;
            r.mf_new = mf_new;
            a.trace[L] = r;
        }
        if (n_new == 0) {
            if (gtid == 0) a.status[ST_LEVELS] = L + 1;
            return;
        }
        if (L + 1 >= a.n) {  // a BFS has at most n levels; more means corrupted state
            if (gtid == 0) atomicCAS(a.status + ST_ERROR, 0, (int)GBX_ERR_OVERFLOW);
            return;
        }
        // Section 6.3: choose the direction of level L + 1
        int next = dir;
        if (a.mode == GBX_DIR_AUTO) {
            const double r_new = (double)n_new / (double)a.n;
            if (dir == DIR_PUSH) {
                if (a.heuristic == GBX_HEUR_RATIO) {
                    if (r_new > (double)a.alpha && n_new > nf) next = DIR_PULL;
                } else {
                    const long long mu_next = mu - in_new;
                    if (mu_next > 0 && (double)mf_new / (double)mu_next > (double)a.alpha) next = DIR_PULL;
                }
            } else {
                if (r_new < (double)a.beta && n_new < nf) next = DIR_PUSH;
            }
        }
        if (dir == DIR_PULL) vcur ^= 1;
        if (dir == DIR_PULL && next == DIR_PUSH && !appended) {
            bitmap_to_queue(a, cur, vcur, cout);
            if (!grid_barrier(a.bar, gridDim.x, a.status, a.timeout_ns)) return;
        }
        mu -= in_new;
        nf = n_new;
        mf = mf_new;
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
    for (int k = 0; k < 5; ++k) GBX_CHECK(d->reserved[k] == 0, GBX_ERR_INVALID_VALUE, "desc.reserved must be 0");
    return GBX_OK;
}

static gbx_status bfs_geometry(Graph* G) {
    if (G->bfs_blocks > 0) return GBX_OK;
    int b0 = 0, b1 = 0;
    GBX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, bfs_kernel<false>, kBfsThreads, 0));
    GBX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, bfs_kernel<true>, kBfsThreads, 0));
    const int per_sm = b0 < b1 ? b0 : b1;
    GBX_CHECK(per_sm >= 1, GBX_ERR_CUDA, "BFS kernel cannot be resident");
    G->bfs_blocks = per_sm * G->num_sms;
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
    a.depth = depth;
    a.parent = parent;
    a.vis[0] = G->bm[0];
    a.vis[1] = G->bm[1];
    a.fbm = G->bm[2];
    for (int i = 0; i < 2; ++i) {
        a.q[i] = G->q[i];
        a.qp[i] = G->qp[i];
        a.qd[i] = G->qd[i];
    }
    a.ctr = G->ctr;
    a.bar = G->bar;
    a.trace = G->trace;
    a.status = G->status;
    a.alpha = d.alpha;
    a.beta = d.beta;
    a.heuristic = d.heuristic;
    a.mode = d.direction;
    a.early_exit = d.early_exit ? 1 : 0;
    a.masking = d.masking ? 1 : 0;
    a.operand_reuse = d.operand_reuse ? 1 : 0;
    a.symmetric = G->symmetric;
    a.need_indeg = (!G->symmetric && (d.trace || d.heuristic == GBX_HEUR_BEAMER)) ? 1 : 0;
    a.trace_cap = kTraceCap;
    a.timeout_ns = wait_timeout_ns();
    void* args[] = {&a};
    const void* fn = d.trace ? (const void*)bfs_kernel<true> : (const void*)bfs_kernel<false>;
    GBX_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(G->bfs_blocks), dim3(kBfsThreads), args, 0, s));
    G->last_stream = s;
    G->last_traced = d.trace ? 1 : 0;
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

namespace gbx {
// One participant short: nobody ever completes the barrier, every block times out.
__global__ void selftest_barrier_kernel(GridBar* bar, int32_t* status, unsigned long long timeout_ns) {
    grid_barrier(bar, gridDim.x + 1, status, timeout_ns);
}
}  // namespace gbx

extern "C" gbx_status gbx_selftest_barrier_timeout(gbx_graph* g, uint64_t timeout_ns, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    Graph* G = as_impl(g);
    selftest_barrier_kernel<<<4, 32, 0, (cudaStream_t)stream>>>(G->bar, G->status, (unsigned long long)timeout_ns);
    GBX_CUDA_TRY(cudaGetLastError());
    G->last_stream = (cudaStream_t)stream;
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
        GBX_CUDA_TRY(cudaStreamCreateWithFlags(&G->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            GBX_CUDA_TRY(cudaMalloc((void**)&G->hdepth[i], bytes));
            GBX_CUDA_TRY(cudaMalloc((void**)&G->hparent[i], bytes));
            GBX_CUDA_TRY(cudaEventCreateWithFlags(&G->ev_done[i], cudaEventDisableTiming));
            GBX_CUDA_TRY(cudaEventCreateWithFlags(&G->ev_copied[i], cudaEventDisableTiming));
            GBX_CUDA_TRY(cudaEventRecord(G->ev_copied[i], G->copy_stream));
        }
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
    GBX_CHECK(G->last_traced, GBX_ERR_INVALID_VALUE, "the last BFS on this graph was not traced");
    if (G->last_stream) GBX_CUDA_TRY(cudaStreamSynchronize(G->last_stream));
    GBX_CUDA_TRY(cudaDeviceSynchronize());
    int32_t st[ST_WORDS];
    GBX_CUDA_TRY(cudaMemcpy(st, G->status, sizeof(st), cudaMemcpyDeviceToHost));
    GBX_CHECK(st[ST_ERROR] == 0, (gbx_status)st[ST_ERROR], "the last BFS recorded a device-side error");
    const int32_t L = st[ST_LEVELS] < kTraceCap ? st[ST_LEVELS] : kTraceCap;
    *nlevels = st[ST_LEVELS];
    const int32_t ncopy = L < cap ? L : cap;
    if (ncopy <= 0) return GBX_OK;
    LevelRec* recs = new LevelRec[ncopy];
    const cudaError_t e = cudaMemcpy(recs, G->trace, sizeof(LevelRec) * ncopy, cudaMemcpyDeviceToHost);
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
        levels[l] = o;
    }
    delete[] recs;
    return GBX_OK;
}
