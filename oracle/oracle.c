/*
 * CPU ORACLE for the push-pull BFS hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code.  The product (the CUDA library and its binding) never calls
 * it, and it shares no code, header, table or helper with the CUDA path.
 *
 * Everything here is the plain, slow, obviously correct definition:
 *   - oracle_csr_build / oracle_transpose: the graph of Section 7.1 ("converted
 *     to undirected graphs; self-loops and duplicated edges are removed") as a
 *     CSR with ascending neighbour lists (Section 3: sparse vectors and lists
 *     are sorted).
 *   - oracle_bfs: textbook FIFO-queue BFS; depth = number of hops from the
 *     source (Section 2.1); children visited in ascending order.
 *   - oracle_bfs_trace: per-level statistics of Algorithm 1's loop, computed
 *     from the final depths: frontier size and out-edges, unvisited count and
 *     in-edges (Eq 1), and the number of in-edges a pull step with early exit
 *     (Section 5.3, Algorithm 2) examines in ascending neighbour order.
 *   - oracle_mxv: masked matvec by its definition, Eq 2-5 over the Boolean
 *     semiring ({0,1}, OR, AND, 0) of Algorithm 1, with the structural
 *     complement (Section 3.2) and accumulate flag of Algorithm 2.
 *   - oracle_csr_weights / oracle_mxv_minplus / oracle_sssp_bf: the generalised
 *     semiring of Section 4 (D, x, +, I) instantiated as (R u {+inf}, +, min,
 *     +inf), the tropical semiring Section 5.6 names for SSSP: edge weights on
 *     the CSR (duplicates keep the smallest weight), the masked matvec over it
 *     in double precision, and Bellman-Ford as the repeated matvec
 *     d <- min(d, A^T d) until nothing changes, with every addition rounded to
 *     binary32 (the precision the device computes in).
 * Pins: tests/test_oracle_pins.py checks each function against brute force,
 * closed forms and invariants that do not come from this file.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_i32(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Build the CSR of A from directed pairs (src[e] -> dst[e]).  With `symmetrize`
 * every pair is also stored reversed; with `drop_self_loops` pairs with
 * src == dst are skipped; duplicates are always removed and each row is sorted
 * ascending (Section 7.1).  `col` must hold m (or 2m when symmetrising)
 * entries.  Returns nnz, or -1 on an out-of-range vertex, -2 on allocation
 * failure, -3 if nnz does not fit int32 offsets.
 */
int64_t oracle_csr_build(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t symmetrize,
                         int32_t drop_self_loops, int32_t* row_ptr, int32_t* col) {
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!start) return -2;
    /* count entries per row */
    for (int64_t e = 0; e < m; ++e) {
        if (drop_self_loops && src[e] == dst[e]) continue;
        start[src[e] + 1] += 1;
        if (symmetrize) start[dst[e] + 1] += 1;
    }
    for (int32_t i = 0; i < n; ++i) start[i + 1] += start[i];
    int64_t* cursor = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!cursor) { free(start); return -2; }
    memcpy(cursor, start, ((size_t)n + 1) * sizeof(int64_t));
    /* scatter every entry into its row */
    for (int64_t e = 0; e < m; ++e) {
        if (drop_self_loops && src[e] == dst[e]) continue;
        col[cursor[src[e]]++] = dst[e];
        if (symmetrize) col[cursor[dst[e]]++] = src[e];
    }
    free(cursor);
    /* sort each row, drop repeats, and pack rows to the front */
    int64_t out = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int64_t b = start[i], e = start[i + 1];
        qsort(col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        for (int64_t k = b; k < e; ++k) {
            if (k > b && col[k] == col[k - 1]) continue;
            col[out++] = col[k];
        }
        if (out > INT32_MAX) { free(start); return -3; }
        row_ptr[i + 1] = (int32_t)out;
    }
    free(start);
    return out;
}

/* CSR of A^T from the CSR of A (rows of A^T come out ascending because rows of A
 * are visited in ascending order). */
int oracle_transpose(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* t_row_ptr, int32_t* t_col) {
    int32_t* cursor = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    if (!cursor) return -2;
    memset(t_row_ptr, 0, ((size_t)n + 1) * sizeof(int32_t));
    for (int64_t k = 0; k < row_ptr[n]; ++k) t_row_ptr[col[k] + 1] += 1;
    for (int32_t i = 0; i < n; ++i) t_row_ptr[i + 1] += t_row_ptr[i];
    memcpy(cursor, t_row_ptr, ((size_t)n + 1) * sizeof(int32_t));
    for (int32_t r = 0; r < n; ++r)
        for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) t_col[cursor[col[k]]++] = r;
    free(cursor);
    return 0;
}

/*
 * Queue BFS over out-neighbours (row u of A lists the children of u; Section
 * 2.1).  depth[s] = 0, unreached = -1; parent[s] = s, parent of a reached
 * vertex = the vertex that first discovered it in queue order, unreached = -1.
 * Returns the number of levels (max depth + 1), or -1 for a bad source.
 */
int32_t oracle_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t s, int32_t* depth,
                   int32_t* parent) {
    if (s < 0 || s >= n) return -1;
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!queue) return -2;
    for (int32_t i = 0; i < n; ++i) { depth[i] = -1; if (parent) parent[i] = -1; }
    int64_t head = 0, tail = 0;
    depth[s] = 0;
    if (parent) parent[s] = s;
    queue[tail++] = s;
    int32_t maxd = 0;
    while (head < tail) {
        const int32_t u = queue[head++];
        for (int32_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            const int32_t w = col[k];
            if (depth[w] == -1) {
                depth[w] = depth[u] + 1;
                if (parent) parent[w] = u;
                if (depth[w] > maxd) maxd = depth[w];
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    return maxd + 1;
}

/* One record per BFS step L (the step that turns frontier F_L, the vertices of
 * depth L, into F_{L+1}). */
typedef struct {
    int64_t nf;      /* |F_L| = nnz(f) */
    int64_t mf;      /* sum of out-degrees over F_L = nnz(m_f^+) */
    int64_t nu;      /* |U_L|: vertices not visited before step L (depth > L or unreached) */
    int64_t nu_nz;   /* members of U_L with nonzero in-degree */
    int64_t mu;      /* sum of in-degrees over U_L = nnz(m_u^-), Eq 1 */
    int64_t e_exam;  /* in-edges a masked pull with early exit examines, ascending order */
    int64_t n_new;   /* |F_{L+1}| */
    int64_t mf_new;  /* sum of out-degrees over F_{L+1} */
} oracle_level;

/*
 * Level statistics of Algorithm 1 for the given final depths (from oracle_bfs on
 * the same graph and source).  out_* is the CSR of A, in_* the CSR of A^T.
 * For each L in 0..levels-1 (the last step finds nothing) fills trace[L].
 * e_exam follows Algorithm 2 with the break of its early-exit option: for each
 * unvisited row i, in-neighbours are examined in ascending order up to and
 * including the first j in the frontier (depth[j] == L); rows with no such j
 * examine all of their in-neighbours.
 * Returns the number of records written.
 */
int32_t oracle_bfs_trace(int32_t n, const int32_t* out_ptr, const int32_t* in_ptr, const int32_t* in_col,
                         const int32_t* depth, int32_t levels, oracle_level* trace, int32_t cap) {
    int32_t nrec = 0;
    for (int32_t L = 0; L < levels && nrec < cap; ++L) {
        oracle_level r;
        memset(&r, 0, sizeof(r));
        for (int32_t v = 0; v < n; ++v) {
            const int64_t outdeg = out_ptr[v + 1] - out_ptr[v];
            const int64_t indeg = in_ptr[v + 1] - in_ptr[v];
            if (depth[v] == L) { r.nf += 1; r.mf += outdeg; }
            if (depth[v] == L + 1) { r.n_new += 1; r.mf_new += outdeg; }
            if (depth[v] == -1 || depth[v] > L) {
                r.nu += 1;
                r.mu += indeg;
                if (indeg > 0) r.nu_nz += 1;
                int64_t examined = 0;
                for (int32_t k = in_ptr[v]; k < in_ptr[v + 1]; ++k) {
                    examined += 1;
                    if (depth[in_col[k]] == L) break;
                }
                r.e_exam += examined;
            }
        }
        trace[nrec++] = r;
    }
    return nrec;
}

/*
 * Masked matvec over the Boolean semiring, by definition (Eq 2-5):
 *   t(i) = OR over stored entries A'(i, j) of (u(j) != 0), with A' = A, or A^T
 *          when `transpose` (Algorithm 1 multiplies by A^T);
 *   pass(i) = (mask(i) != 0, or 1 when there is no mask) XOR complement
 *          (structural complement, Section 3.2; the test of Algorithm 2);
 *   w(i) = pass(i) ? (accum ? w_old(i) OR t(i) : t(i))
 *                  : (accum ? w_old(i)          : 0)     (Eq 4 writes 0).
 * A is nrows x ncols in CSR; u has length ncols (nrows when transposed), w and
 * mask have length nrows (ncols when transposed).  Vectors are 0/1 bytes.
 */
int oracle_mxv(int32_t nrows, int32_t ncols, const int32_t* row_ptr, const int32_t* col, int32_t transpose,
               const uint8_t* u, const uint8_t* mask, int32_t complement, int32_t accum, uint8_t* w) {
    const int32_t nout = transpose ? ncols : nrows;
    uint8_t* t = (uint8_t*)calloc((size_t)(nout > 0 ? nout : 1), 1);
    if (!t) return -2;
    for (int32_t r = 0; r < nrows; ++r) {
        for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            const int32_t c = col[k];
            if (transpose) {
                if (u[r]) t[c] = 1; /* (A^T u)(c) ORs A(r, c) AND u(r) */
            } else {
                if (u[c]) t[r] = 1; /* (A u)(r) ORs A(r, c) AND u(c) */
            }
        }
    }
    for (int32_t i = 0; i < nout; ++i) {
        const int m = mask ? (mask[i] != 0) : 1;
        const int pass = m ^ (complement != 0);
        const uint8_t old = accum ? (w[i] != 0) : 0;
        w[i] = pass ? (uint8_t)(old | t[i]) : old;
    }
    free(t);
    return 0;
}

/*
 * Weights of the CSR (row_ptr, col) built by oracle_csr_build from the same edge
 * list: val[k] = the smallest w[e] over input pairs e that map to entry k (the
 * pair itself, and its reverse when symmetrising).  Entries are located by
 * binary search in the row (rows are sorted ascending).
 * Returns 0, or -1 if a pair has no entry (the CSR was not built from this list).
 */
int oracle_csr_weights(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const float* w,
                       int32_t symmetrize, int32_t drop_self_loops, const int32_t* row_ptr, const int32_t* col,
                       double* val) {
    const int64_t nnz = row_ptr[n];
    for (int64_t k = 0; k < nnz; ++k) val[k] = 1.0 / 0.0;
    for (int64_t e = 0; e < m; ++e) {
        if (drop_self_loops && src[e] == dst[e]) continue;
        for (int dir = 0; dir < (symmetrize ? 2 : 1); ++dir) {
            const int32_t r = dir ? dst[e] : src[e];
            const int32_t c = dir ? src[e] : dst[e];
            int64_t lo = row_ptr[r], hi = row_ptr[r + 1], at = -1;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] == c) {
                    at = mid;
                    break;
                }
                if (col[mid] < c)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            if (at < 0) return -1;
            if ((double)w[e] < val[at]) val[at] = (double)w[e];
        }
    }
    return 0;
}

/* Transpose of a weighted CSR: entry (r, c, v) becomes (c, r, v), rows ascending. */
int oracle_transpose_weighted(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                              int32_t* t_row_ptr, int32_t* t_col, double* t_val) {
    const int64_t nnz = row_ptr[n];
    for (int32_t i = 0; i <= n; ++i) t_row_ptr[i] = 0;
    for (int64_t k = 0; k < nnz; ++k) t_row_ptr[col[k] + 1] += 1;
    for (int32_t i = 0; i < n; ++i) t_row_ptr[i + 1] += t_row_ptr[i];
    int32_t* cur = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!cur) return -2;
    memcpy(cur, t_row_ptr, ((size_t)n + 1) * sizeof(int32_t));
    /* rows r visited in ascending order, so each transposed row comes out sorted */
    for (int32_t r = 0; r < n; ++r)
        for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            const int32_t p = cur[col[k]]++;
            t_col[p] = r;
            t_val[p] = val[k];
        }
    free(cur);
    return 0;
}

/*
 * Masked matvec over (R u {+inf}, +, min, +inf), in double:
 *   t(i) = min over j with A'(i, j) of ( A'(i, j) + u(j) ),  +inf if there is none,
 *   A' = A^T when `transpose` (then t(c) takes the entries (r, c) of A), else A;
 *   pass(i) = (mask(i) != 0, or 1 without a mask) XOR complement;
 *   w(i) = pass(i) ? (accum ? min(w_old(i), t(i)) : t(i)) : (accum ? w_old(i) : +inf).
 * An absent entry of u, w or the result is +inf (the semiring's identity).
 */
int oracle_mxv_minplus(int32_t nrows, int32_t ncols, const int32_t* row_ptr, const int32_t* col, const double* val,
                       int32_t transpose, const double* u, const uint8_t* mask, int32_t complement, int32_t accum,
                       double* w) {
    const int32_t nout = transpose ? ncols : nrows;
    const double inf = 1.0 / 0.0;
    double* t = (double*)malloc((size_t)(nout > 0 ? nout : 1) * sizeof(double));
    if (!t) return -2;
    for (int32_t i = 0; i < nout; ++i) t[i] = inf;
    for (int32_t r = 0; r < nrows; ++r) {
        for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            const int32_t c = col[k];
            if (transpose) {
                const double x = val[k] + u[r];
                if (x < t[c]) t[c] = x;
            } else {
                const double x = val[k] + u[c];
                if (x < t[r]) t[r] = x;
            }
        }
    }
    for (int32_t i = 0; i < nout; ++i) {
        const int m = mask ? (mask[i] != 0) : 1;
        const int pass = m ^ (complement != 0);
        const double old = accum ? w[i] : inf;
        if (pass)
            w[i] = (accum && old < t[i]) ? old : t[i];
        else
            w[i] = old;
    }
    free(t);
    return 0;
}

/*
 * Single-source shortest paths as Bellman-Ford in the (min, +) semiring:
 * d_0 = e_s (0 at s, +inf elsewhere); d_{k+1}(i) = min(d_k(i), min over edges
 * (j -> i) of fl32(d_k(j) + a(j, i))), i.e. d_{k+1} = min(d_k, A^T d_k), until
 * d_{k+1} = d_k.  Every sum is rounded to binary32 as it is formed.  For
 * non-negative weights the fixpoint is, for every i, the smallest binary32
 * left-to-right rounded sum over the paths from s to i, whatever order the
 * relaxations run in.  Returns the number of iterations that changed d, or
 * -2 on allocation failure.
 */
int32_t oracle_sssp_bf(int32_t n, const int32_t* row_ptr, const int32_t* col, const float* val, int32_t s,
                       float* d) {
    const float inf = 1.0f / 0.0f;
    float* nd = (float*)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    if (!nd) return -2;
    for (int32_t i = 0; i < n; ++i) d[i] = inf;
    d[s] = 0.0f;
    int32_t iters = 0;
    for (;;) {
        int changed = 0;
        memcpy(nd, d, (size_t)n * sizeof(float));
        for (int32_t j = 0; j < n; ++j) {
            if (d[j] == inf) continue;
            for (int64_t k = row_ptr[j]; k < row_ptr[j + 1]; ++k) {
                volatile float x = d[j] + val[k]; /* one binary32 rounding */
                if (x < nd[col[k]]) nd[col[k]] = x;
            }
        }
        for (int32_t i = 0; i < n; ++i)
            if (nd[i] != d[i]) changed = 1;
        if (!changed) break;
        memcpy(d, nd, (size_t)n * sizeof(float));
        ++iters;
    }
    free(nd);
    return iters;
}
