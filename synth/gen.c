/*
 * Seeded synthetic inputs for the push-pull BFS workloads.
 *
 * This module only draws raw inputs: directed edge samples (with the
 * self-loops and duplicates a generator naturally produces), vertex subsets
 * and BFS sources.  It holds none of the method's arithmetic: no CSR build,
 * no symmetrisation, no deduplication, no traversal.  Both the CPU oracle and
 * the CUDA path receive the arrays produced here and build their own graphs.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: draw(seed, i) is the i-th output of the SplitMix64 stream whose
 * state starts at `seed`.  Every draw depends only on (seed, i), so results do
 * not depend on the number of threads.
 *
 * Workload recipes (the paper gives no generator parameters, only the graph
 * classes of its Table 3):
 *   RMAT: 2^scale vertices, edge_factor * 2^scale samples; each of the `scale`
 *         bit levels picks a quadrant with probabilities a, b, c, d = 1-a-b-c,
 *         most significant bit first; no noise; then a seeded random vertex
 *         relabelling.
 *   Grid: W x H 4-neighbour mesh, vertex id y*W + x, each undirected edge
 *         deleted independently with probability p_delete.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (0-based) of the SplitMix64 stream started at state `seed`. */
uint64_t synth_draw(uint64_t seed, uint64_t i) { return sm_mix(seed + (i + 1) * GOLDEN); }

/* Sub-seed for an independent stream `id` derived from a user seed. */
uint64_t synth_subseed(uint64_t seed, uint64_t id) { return synth_draw(seed ^ 0x5EEDBA5Eull, id); }

static inline double unit_double(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Stream ids used by the recipes. */
enum { STREAM_RMAT = 1, STREAM_PERM = 2, STREAM_SRC = 3, STREAM_GRID_DEL = 4, STREAM_SET = 5 };

typedef struct { uint64_t key; int32_t v; } keyed_t;

static int cmp_keyed(const void* x, const void* y) {
    const keyed_t* p = (const keyed_t*)x;
    const keyed_t* q = (const keyed_t*)y;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->v < q->v ? -1 : (p->v > q->v);
}

/* perm[v] = new label of vertex v: vertices ranked by a seeded 64-bit key. */
int synth_permutation(int32_t n, uint64_t seed, int32_t* perm) {
    keyed_t* t = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
    if (!t) return -1;
    uint64_t s = synth_subseed(seed, STREAM_PERM);
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; ++v) { t[v].key = synth_draw(s, (uint64_t)v); t[v].v = v; }
    qsort(t, (size_t)n, sizeof(keyed_t), cmp_keyed);
    for (int32_t r = 0; r < n; ++r) perm[t[r].v] = r;
    free(t);
    return 0;
}

/* RMAT samples: m = edge_factor << scale directed pairs (src[e], dst[e]). */
int synth_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, uint64_t seed,
               int32_t relabel, int32_t* src, int32_t* dst) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    const int64_t n = (int64_t)1 << scale;
    const int64_t m = (int64_t)edge_factor * n;
    const double ab = a + b, abc = a + b + c;
    const uint64_t s = synth_subseed(seed, STREAM_RMAT);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int64_t r = 0, q = 0;
        for (int32_t l = 0; l < scale; ++l) {
            const double u = unit_double(synth_draw(s, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
            const int64_t bit = (int64_t)1 << (scale - 1 - l);
            if (u < a) {
            } else if (u < ab) {
                q |= bit;
            } else if (u < abc) {
                r |= bit;
            } else {
                r |= bit;
                q |= bit;
            }
        }
        src[e] = (int32_t)r;
        dst[e] = (int32_t)q;
    }
    if (relabel) {
        int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) return -2;
        if (synth_permutation((int32_t)n, seed, perm) != 0) { free(perm); return -2; }
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < m; ++e) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
        free(perm);
    }
    return 0;
}

/* Number of undirected mesh edges before deletion. */
int64_t synth_grid_edge_slots(int32_t w, int32_t h) {
    return (int64_t)h * (w - 1) + (int64_t)(h - 1) * w;
}

/* W x H 4-neighbour grid; each undirected edge kept with probability 1 - p_delete.
 * Writes the kept edges once each (src < dst) and returns their count. */
int64_t synth_grid(int32_t w, int32_t h, double p_delete, uint64_t seed, int32_t* src, int32_t* dst) {
    if (w < 1 || h < 1) return -1;
    const uint64_t s = synth_subseed(seed, STREAM_GRID_DEL);
    const int64_t nh = (int64_t)h * (w - 1);
    const int64_t slots = synth_grid_edge_slots(w, h);
    int64_t k = 0;
    for (int64_t id = 0; id < slots; ++id) {
        if (p_delete > 0.0 && unit_double(synth_draw(s, (uint64_t)id)) < p_delete) continue;
        int64_t u, v;
        if (id < nh) {
            const int64_t y = id / (w - 1), x = id % (w - 1);
            u = y * w + x;
            v = u + 1;
        } else {
            const int64_t j = id - nh;
            const int64_t y = j / w, x = j % w;
            u = y * w + x;
            v = u + w;
        }
        src[k] = (int32_t)u;
        dst[k] = (int32_t)v;
        ++k;
    }
    return k;
}

/* Up to k distinct sources drawn uniformly (seeded) among vertices that touch at
 * least one edge whose endpoints differ.  Returns the number written. */
int32_t synth_sources(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t k,
                      uint64_t seed, int32_t* out) {
    uint8_t* touched = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!touched) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] != dst[e]) { touched[src[e]] = 1; touched[dst[e]] = 1; }
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!cand) { free(touched); return -1; }
    int32_t nc = 0;
    for (int32_t v = 0; v < n; ++v)
        if (touched[v]) cand[nc++] = v;
    uint8_t* taken = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    const uint64_t s = synth_subseed(seed, STREAM_SRC);
    int32_t got = 0;
    for (uint64_t t = 0; got < k && got < nc && t < (uint64_t)64 * (uint64_t)(k + nc); ++t) {
        const int32_t v = cand[synth_draw(s, t) % (uint64_t)nc];
        if (taken[v]) continue;
        taken[v] = 1;
        out[got++] = v;
    }
    free(taken);
    free(cand);
    free(touched);
    return got;
}

/* Bernoulli(density) membership per vertex, seeded: writes a 0/1 byte per vertex. */
int synth_vertex_set(int32_t n, double density, uint64_t seed, uint64_t stream, uint8_t* out) {
    const uint64_t s = synth_subseed(seed, (uint64_t)STREAM_SET + 16u * stream);
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; ++v) out[v] = unit_double(synth_draw(s, (uint64_t)v)) < density ? 1 : 0;
    return 0;
}
