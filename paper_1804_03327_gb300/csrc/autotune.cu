// Autotuner for the BFS descriptors: times candidate settings on the caller's
// graph and sources and keeps the fastest.  Section 6.3 picks its switch point
// by comparing against running both directions on every level and choosing the
// faster; here the candidates are whole descriptors (direction rule, thresholds,
// lane probe depth, persistent blocks per SM) timed end to end with CUDA events.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gbx_internal.cuh"

namespace gbx {

struct TuneKey {
    int32_t kind, n, sym, S;
    long long nnz;
};

static bool cache_lookup(const char* path, const TuneKey& k, gbx_desc* d, double* ms) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        int kind, n, sym, S, heur, probe, bps, dir;
        long long nnz;
        float alpha, beta;
        double t;
        if (std::sscanf(line, "%d %d %lld %d %d %d %d %f %f %d %d %lf", &kind, &n, &nnz, &sym, &S, &dir, &heur, &alpha,
                        &beta, &probe, &bps, &t) != 12)
            continue;
        if (kind == k.kind && n == k.n && nnz == k.nnz && sym == k.sym && S == k.S) {
            gbx_desc_init(d);
            d->direction = dir;
            d->heuristic = heur;
            d->alpha = alpha;
            d->beta = beta;
            d->pull_probe = probe;
            d->blocks_per_sm = bps;
            *ms = t;
            found = true;  // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

static void cache_store(const char* path, const TuneKey& k, const gbx_desc& d, double ms) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %lld %d %d %d %d %.9g %.9g %d %d %.6f\n", k.kind, k.n, k.nnz, k.sym, k.S, d.direction,
                 d.heuristic, d.alpha, d.beta, d.pull_probe, d.blocks_per_sm, ms);
    std::fclose(f);
}

// Section 6.3's rule (ratio form) decides level L + 1 at the end of level L from
// r = |F_{L+1}| / n: push -> pull when r > alpha and the frontier grew, pull ->
// push when r < beta and it shrank.  Returns the thresholds that switch where the
// per-level best schedule `best` (level 0 pushes) switches, as far as the rule can.
static void thresholds_for_schedule(const gbx_level* tr, const std::vector<int32_t>& best, int32_t n, float* alpha,
                                    float* beta) {
    const int32_t nl = (int32_t)best.size();
    auto r = [&](int32_t L) { return (double)tr[L].n_new / (double)n; };
    auto grew = [&](int32_t L) { return tr[L].n_new > tr[L].nf; };
    auto shrank = [&](int32_t L) { return tr[L].n_new < tr[L].nf; };
    int32_t lp = -1;
    for (int32_t L = 1; L < nl && lp < 0; ++L)
        if (best[L] == GBX_DIR_PULL) lp = L;
    if (lp < 0) {  // push throughout: never switch
        *alpha = 1e30f;
        *beta = 0.0f;
        return;
    }
    // switch at the end of level lp - 1, not at an earlier level whose frontier grew
    const double hi = r(lp - 1);
    double lo = 0.0;
    for (int32_t L = 0; L < lp - 1; ++L)
        if (grew(L) && r(L) > lo) lo = r(L);
    double a = hi * 0.5;
    if (lo > 0.0 && lo < hi) a = std::sqrt(lo * hi);
    *alpha = (float)a;
    int32_t lq = -1;
    for (int32_t L = lp + 1; L < nl && lq < 0; ++L)
        if (best[L] == GBX_DIR_PUSH) lq = L;
    if (lq < 0) {  // pull to the end
        *beta = 0.0f;
        return;
    }
    // back to push at the end of level lq - 1, not at an earlier pull level that shrank
    const double blo = r(lq - 1);
    double bhi = 1e300;
    for (int32_t L = lp; L < lq - 1; ++L)
        if (shrank(L) && r(L) < bhi) bhi = r(L);
    double b = blo * 2.0 + 1.0 / (double)n;
    if (bhi < 1e300 && blo < bhi) b = std::sqrt((blo > 0.0 ? blo : 1.0 / (double)n) * bhi);
    *beta = (float)b;
}

}  // namespace gbx

using namespace gbx;

extern "C" gbx_status gbx_tune_thresholds(const gbx_level* push, const gbx_level* pull, int32_t nlevels, int32_t n,
                                          float* alpha, float* beta, int32_t* schedule) {
    clear_error();
    GBX_CHECK(push != nullptr && pull != nullptr && alpha != nullptr && beta != nullptr, GBX_ERR_NULL_POINTER,
              "push, pull, alpha and beta are required");
    GBX_CHECK(nlevels >= 1 && n >= 1, GBX_ERR_INVALID_VALUE, "nlevels and n must be >= 1");
    std::vector<int32_t> best((size_t)nlevels);
    for (int32_t L = 0; L < nlevels; ++L) {
        GBX_CHECK(push[L].nf == pull[L].nf && push[L].n_new == pull[L].n_new && push[L].level == L &&
                      pull[L].level == L,
                  GBX_ERR_INVALID_VALUE, "the two traces are not the levels of one BFS");
        best[L] = L > 0 && pull[L].time_ns < push[L].time_ns ? GBX_DIR_PULL : GBX_DIR_PUSH;
        if (schedule) schedule[L] = best[L];
    }
    thresholds_for_schedule(push, best, n, alpha, beta);
    return GBX_OK;
}

extern "C" gbx_status gbx_autotune(gbx_graph* g, int32_t kind, const int32_t* sources, int32_t count, gbx_desc* best,
                                   double* best_ms, const char* cache_path, void* stream) {
    clear_error();
    GBX_TRY(check_graph(g));
    GBX_CHECK(kind == GBX_TUNE_BFS || kind == GBX_TUNE_BATCH || kind == GBX_TUNE_SSSP, GBX_ERR_INVALID_VALUE,
              "unknown tuning kind");
    GBX_CHECK(count >= 1 && sources != nullptr && best != nullptr, GBX_ERR_NULL_POINTER,
              "sources and best are required, count >= 1");
    Graph* G = as_impl(g);
    for (int32_t k = 0; k < count; ++k)
        GBX_CHECK(sources[k] >= 0 && sources[k] < G->n, GBX_ERR_INVALID_INDEX, "source outside [0, n)");
    const TuneKey key{kind, G->n, G->symmetric, kind == GBX_TUNE_BATCH ? count : 0, (long long)G->nnz};
    double cached = 0.0;
    if (cache_lookup(cache_path, key, best, &cached)) {
        if (best_ms) *best_ms = cached;
        return GBX_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // candidate descriptors
    std::vector<gbx_desc> cand;
    gbx_desc base;
    gbx_desc_init(&base);
    if (kind == GBX_TUNE_BFS) {
        const float ratio_a[] = {0.0005f, 0.001f, 0.002f, 0.005f, 0.01f, 0.02f, 0.05f, 0.1f};
        const float beamer_a[] = {1.0f / 256, 1.0f / 128, 1.0f / 64, 1.0f / 32, 1.0f / 16, 1.0f / 14, 1.0f / 8, 1.0f / 4};
        // beta = 0: once pulling, never back to push (the tail levels stay row-based)
        const float betas[] = {0.0f, 0.001f, 0.01f, 0.05f};
        for (float b : betas) {
            for (float a : ratio_a) {
                gbx_desc d = base;
                d.heuristic = GBX_HEUR_RATIO;
                d.alpha = a;
                d.beta = b;
                cand.push_back(d);
            }
            for (float a : beamer_a) {
                gbx_desc d = base;
                d.heuristic = GBX_HEUR_BEAMER;
                d.alpha = a;
                d.beta = b;
                cand.push_back(d);
            }
        }
    } else if (kind == GBX_TUNE_BATCH) {
        const float alphas[] = {0.002f, 0.005f, 0.01f, 0.02f, 0.05f, 0.1f, 0.2f, 0.5f, 1e30f};
        for (float a : alphas) {
            gbx_desc d = base;
            d.alpha = a;
            cand.push_back(d);
        }
    } else {
        // SSSP: the switch rule on the improved-set size (beta = 0 keeps the two
        // phases of Section 5.6; a large beta returns to push as soon as the
        // improved set shrinks), push only and pull only
        const float alphas[] = {0.002f, 0.01f, 0.05f, 0.2f};
        const float betas[] = {0.0f, 0.01f, 0.1f, 0.3f};
        for (float b : betas)
            for (float a : alphas) {
                gbx_desc d = base;
                d.alpha = a;
                d.beta = b;
                cand.push_back(d);
            }
        gbx_desc d = base;
        d.direction = GBX_DIR_PUSH;
        cand.push_back(d);
        d.direction = GBX_DIR_PULL;
        cand.push_back(d);
    }
    // buffers
    if (kind == GBX_TUNE_SSSP)
        GBX_CHECK(G->out_val != nullptr, GBX_ERR_INVALID_VALUE, "GBX_TUNE_SSSP needs edge weights");
    void* depth = nullptr;
    const size_t bytes = kind == GBX_TUNE_BATCH ? sizeof(int16_t) * (size_t)G->n * (size_t)count
                                                : sizeof(int32_t) * (size_t)G->n;  // int32 depths or float distances
    GBX_CUDA_TRY(cudaMallocAsync(&depth, bytes, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gbx_status st = GBX_OK;
    auto run_once = [&](const gbx_desc& d) -> gbx_status {
        if (kind == GBX_TUNE_BFS) {
            for (int32_t k = 0; k < count; ++k)
                GBX_TRY(gbx_bfs(g, sources[k], static_cast<int32_t*>(depth), nullptr, &d, stream));
            return GBX_OK;
        }
        if (kind == GBX_TUNE_SSSP) {
            for (int32_t k = 0; k < count; ++k) GBX_TRY(gbx_sssp(g, sources[k], static_cast<float*>(depth), &d, stream));
            return GBX_OK;
        }
        return gbx_bfs_batch(g, sources, count, depth, GBX_DEPTH_I16, &d, stream);
    };
    // a warm-up run, then the better of two timed runs (a single run of a few milliseconds
    // occasionally lands on a slow moment and would misrank close candidates)
    auto time_desc = [&](const gbx_desc& d, double* ms) -> gbx_status {
        GBX_TRY(run_once(d));
        double best = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            GBX_CUDA_TRY(cudaEventRecord(e0, s));
            GBX_TRY(run_once(d));
            GBX_CUDA_TRY(cudaEventRecord(e1, s));
            GBX_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.0f;
            GBX_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            best = t < best ? t : best;
        }
        GBX_TRY(gbx_graph_sync(g, stream));
        *ms = best;
        return GBX_OK;
    };
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        st = GBX_ERR_CUDA;
        set_error(std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
    }
    // Section 6.3 set its thresholds by comparison with running both directions on
    // every level.  A BFS visits the same levels whichever direction each takes, so
    // traced push-only and pull-only runs of (up to 8 of) the tuning sources give each
    // level's cost both ways; the ratio-rule thresholds that reproduce each source's
    // per-level best schedule join the timed candidates.
    if (kind == GBX_TUNE_BFS && st == GBX_OK) {
        std::vector<gbx_level> tp(kTraceCap), tq(kTraceCap);
        for (int32_t k = 0; k < count && k < 8 && st == GBX_OK; ++k) {
            int32_t np = 0, nq = 0;
            gbx_desc dp = base, dq = base;
            dp.direction = GBX_DIR_PUSH;
            dq.direction = GBX_DIR_PULL;
            dp.trace = dq.trace = 1;
            st = gbx_bfs(g, sources[k], static_cast<int32_t*>(depth), nullptr, &dp, stream);
            if (st == GBX_OK) st = gbx_bfs_trace(g, tp.data(), kTraceCap, &np);
            if (st == GBX_OK) st = gbx_bfs(g, sources[k], static_cast<int32_t*>(depth), nullptr, &dq, stream);
            if (st == GBX_OK) st = gbx_bfs_trace(g, tq.data(), kTraceCap, &nq);
            if (st != GBX_OK || np != nq || np < 1 || np >= kTraceCap) continue;
            gbx_desc d = base;
            d.heuristic = GBX_HEUR_RATIO;
            if (gbx_tune_thresholds(tp.data(), tq.data(), np, G->n, &d.alpha, &d.beta, nullptr) != GBX_OK) continue;
            bool seen = false;
            for (const gbx_desc& c : cand)
                if (c.heuristic == d.heuristic && std::fabs(c.alpha - d.alpha) <= 0.05f * d.alpha &&
                    std::fabs(c.beta - d.beta) <= 0.05f * d.beta)
                    seen = true;
            if (!seen) cand.push_back(d);
        }
        if (st == GBX_OK) clear_error();
    }
    gbx_desc winner = base;
    double win_ms = 1e300;
    std::vector<double> cand_ms(cand.size(), 1e300);
    for (size_t c = 0; c < cand.size() && st == GBX_OK; ++c) {
        double ms = 0.0;
        st = time_desc(cand[c], &ms);
        cand_ms[c] = ms;
        if (st == GBX_OK && ms < win_ms) {
            win_ms = ms;
            winner = cand[c];
        }
    }
    // Batches: the time is a step function of alpha (a level either pushes or pulls),
    // and other sources put the step elsewhere; among thresholds within 3 % of the
    // best, the largest (pulling latest) is the safest choice.
    if (kind == GBX_TUNE_BATCH && st == GBX_OK) {
        const double best = win_ms;
        for (size_t c = 0; c < cand.size(); ++c)
            if (cand_ms[c] <= best * 1.03 && cand[c].alpha > winner.alpha) {
                winner = cand[c];
                win_ms = cand_ms[c];
            }
    }
    // second stage: lane probe depth and persistent blocks per SM on the winning rule
    const int32_t probes_bfs[] = {8, 32};
    const int32_t probes_batch[] = {4, 16};
    const int32_t* probes = kind == GBX_TUNE_BFS ? probes_bfs : probes_batch;
    for (int i = 0; i < 2 && st == GBX_OK && kind != GBX_TUNE_SSSP; ++i) {
        gbx_desc d = winner;
        d.pull_probe = probes[i];
        double ms = 0.0;
        st = time_desc(d, &ms);
        if (st == GBX_OK && ms < win_ms) {
            win_ms = ms;
            winner = d;
        }
    }
    // batches of at most 128 sources and SSSP: the register-lean build at three blocks per SM
    if (((kind == GBX_TUNE_BATCH && count <= 128) || kind == GBX_TUNE_SSSP) && st == GBX_OK) {
        gbx_desc d = winner;
        d.blocks_per_sm = 3;
        double ms = 0.0;
        st = time_desc(d, &ms);
        if (st == GBX_OK && ms < win_ms) {
            win_ms = ms;
            winner = d;
        }
    }
    if (kind == GBX_TUNE_BFS && st == GBX_OK && G->bfs_blocks > 1) {
        gbx_desc d = winner;
        d.blocks_per_sm = G->bfs_blocks - 1;
        double ms = 0.0;
        st = time_desc(d, &ms);
        if (st == GBX_OK && ms < win_ms) {
            win_ms = ms;
            winner = d;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(depth, s);
    if (st != GBX_OK) return st;
    GBX_CUDA_TRY(cudaStreamSynchronize(s));
    *best = winner;
    if (best_ms) *best_ms = win_ms;
    cache_store(cache_path, key, winner, win_ms);
    return GBX_OK;
}
