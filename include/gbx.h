/*
 * gbx.h -- C ABI of the GB300-native push-pull BFS library (libgbx.so).
 *
 * The library implements the hot path of "Implementing Push-Pull Efficiently
 * in GraphBLAS" (Yang, Buluc, Owens, arXiv 1804.03327): the Boolean-semiring
 * masked matvec f' = A^T f .* !v that every level of direction-optimized BFS
 * runs (Algorithm 1), in its column-based "push" form (Eq 5, Algorithm 3),
 * its row-based "pull" form restricted by the mask with early exit (Eq 4,
 * Algorithm 2, Sections 5.2-5.3), and the per-level direction switch between
 * them (Section 6.3).
 *
 * Conventions shared by every entry point:
 *  - Errors: every call returns a gbx_status and never throws or aborts.  A
 *    human-readable message for the last failing call on the calling thread is
 *    returned by gbx_last_error().  No partial output is promised on error.
 *  - Ownership: the library owns gbx_graph handles (and all memory reachable
 *    from them) and frees them in gbx_graph_free.  The caller owns every
 *    buffer it passes in (vectors, depth/parent arrays, edge lists) and keeps
 *    it alive until the work that uses it has completed on the stream.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Device work is enqueued on it and the call returns
 *    without synchronising unless its comment says otherwise.  Work on one
 *    graph handle uses that handle's scratch memory (and the launch sequences
 *    gbx_mxv keeps for it), so calls on the same graph must be ordered (one
 *    stream, or explicit events) and issued by one host thread at a time.
 *  - Device pointers are plain CUDA device addresses (for example the
 *    data_ptr() of a CUDA tensor); host pointers are ordinary addresses.
 *  - Indices are int32; a graph holds fewer than 2^31 stored edges.
 */
#ifndef GBX_H
#define GBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes, modelled on GrB_Info of the GraphBLAS C API the paper targets. */
typedef enum {
    GBX_OK = 0,
    GBX_ERR_INVALID_VALUE = 1,      /* a size, flag or descriptor field out of range */
    GBX_ERR_INVALID_INDEX = 2,      /* a vertex id outside [0, n) */
    GBX_ERR_DIMENSION_MISMATCH = 3, /* vector length differs from the graph's n */
    GBX_ERR_OUT_OF_MEMORY = 4,      /* a device or host allocation failed */
    GBX_ERR_NOT_SUPPORTED = 5,      /* e.g. a semiring other than GBX_LOR_LAND */
    GBX_ERR_TIMEOUT = 6,            /* a bounded device-side wait ran out */
    GBX_ERR_CUDA = 7,               /* a CUDA runtime call failed (message has details) */
    GBX_ERR_OVERFLOW = 8,           /* a count exceeded its type (e.g. >= 2^31 edges) */
    GBX_ERR_BUSY = 9,               /* a resource is in use */
    GBX_ERR_NULL_POINTER = 10       /* a required pointer argument is NULL */
} gbx_status;

/* Message for the last failing call on this thread ("" if none).  The string is
 * owned by the library and valid until the next call on this thread. */
const char* gbx_last_error(void);
/* Static name of a status code. */
const char* gbx_status_string(gbx_status s);
/* Library version, major * 10000 + minor * 100 + patch. */
int32_t gbx_version(void);

/* ------------------------------------------------------------------ graphs */

typedef struct gbx_graph gbx_graph;

/* Build flags for gbx_graph_build. */
#define GBX_SYMMETRIZE 0x1u      /* store every edge in both directions (undirected graph) */
#define GBX_DROP_SELF_LOOPS 0x2u /* drop edges u -> u */
#define GBX_DEVICE_EDGES 0x4u    /* src and dst are device pointers (else host) */

/*
 * Build a graph from m directed edges src[e] -> dst[e] on vertices [0, n).
 * Section 7.1: datasets are made undirected with self-loops and duplicate
 * edges removed; duplicates are always removed here, the other two steps are
 * selected by `flags`.  The library stores the adjacency matrix A (A(u,v) = 1
 * for an edge u -> v) twice, as CSR of A (out-edges, the columns push reads)
 * and CSR of A^T (in-edges, the rows pull reads, Algorithm 2 takes A^T); for
 * a symmetrised graph the two are one array.  Neighbour lists are sorted
 * ascending.  The build runs on the device (radix sort of packed (row, col)
 * keys); it synchronises `stream` before returning.
 * Errors: NULL_POINTER (out, or src/dst with m > 0), INVALID_VALUE (n < 1 or
 * m < 0 or unknown flag bits), INVALID_INDEX (an endpoint outside [0, n)),
 * OVERFLOW (2^31 or more stored edges), OUT_OF_MEMORY, CUDA.
 * On success *out receives a handle to be released with gbx_graph_free.
 */
gbx_status gbx_graph_build(gbx_graph** out, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                           uint32_t flags, void* stream);

/* Release a graph and all device memory it owns.  NULL is accepted. */
gbx_status gbx_graph_free(gbx_graph* g);

/* Vertex count, stored-edge count (nnz of A) and whether A is symmetric. Any
 * output pointer may be NULL. */
gbx_status gbx_graph_info(const gbx_graph* g, int32_t* n, int64_t* nnz, int32_t* symmetric);

/* Device pointers to the CSR arrays of A (transpose = 0) or A^T (transpose =
 * 1): row_ptr int32[n + 1] and col int32[nnz].  Owned by the graph; valid
 * until gbx_graph_free. */
gbx_status gbx_graph_csr(const gbx_graph* g, int32_t transpose, const int32_t** row_ptr, const int32_t** col);

/*
 * Attach binary32 edge weights for the (min, +) semiring (Section 5.6; the
 * Boolean path of Section 5.5 needs none).  (src[e], dst[e], w[e]) for e < m
 * must be the edge list the graph was built from: w[e] goes to the stored
 * entry of that pair, and to its reverse when the graph was symmetrised;
 * parallel pairs keep the smallest weight; self-loops are skipped when the
 * build dropped them.  Host arrays, or device arrays with GBX_DEVICE_EDGES in
 * flags.  Weights must be finite.  Calling again replaces all weights (entries
 * no pair reaches get +inf).  Synchronous.  Errors: NULL_POINTER,
 * INVALID_INDEX (vertex outside [0, n) or a weight that is not finite),
 * INVALID_VALUE (a pair the graph does not store, unknown flags; the weights
 * are then unspecified), OUT_OF_MEMORY, CUDA.
 */
gbx_status gbx_graph_set_weights(gbx_graph* g, int64_t m, const int32_t* src, const int32_t* dst, const float* w,
                                 uint32_t flags, void* stream);

/* Copy the edge weights of A (transpose = 0: aligned with the CSR of A) or A^T
 * (transpose = 1: aligned with the CSR of A^T) into dst (float[nnz], host or
 * device).  Synchronous.  Errors: NULL_POINTER, INVALID_VALUE (no weights). */
gbx_status gbx_graph_copy_weights(const gbx_graph* g, int32_t transpose, float* dst);

/* Copy the CSR arrays of A (transpose = 0) or A^T (transpose = 1) into
 * caller buffers row_ptr_dst (int32[n + 1]) and col_dst (int32[nnz]), each
 * host or device memory.  Synchronous. */
gbx_status gbx_graph_copy_csr(const gbx_graph* g, int32_t transpose, int32_t* row_ptr_dst, int32_t* col_dst);

/* Wait for the work enqueued on `stream` and report device-side errors that
 * kernels of this graph recorded since the last check (e.g. GBX_ERR_TIMEOUT
 * from a bounded wait).  Clears the recorded error. */
gbx_status gbx_graph_sync(gbx_graph* g, void* stream);

/* ------------------------------------------------------------------ vectors */

/* Vector formats (Section 6.3 stores the frontier as a DenseVector for
 * row-based and a SparseVector for column-based matvec). */
#define GBX_DENSE 0  /* data: uint8_t[size], entry i is true iff data[i] != 0 */
#define GBX_SPARSE 1 /* data: int32_t[capacity] indices, ascending and unique (Section 3);
                        *nnz (a device int32) holds how many are stored */
#define GBX_DENSE_F32 2 /* data: float[size], the values of the (min, +) semiring; +inf marks
                           an absent entry (the semiring's identity) */

/* A non-owning view of a vector in device memory. */
typedef struct {
    int32_t format;   /* GBX_DENSE, GBX_SPARSE or GBX_DENSE_F32 */
    int32_t size;     /* logical length; must equal the graph's n */
    void* data;       /* device pointer, layout per format */
    int32_t* nnz;     /* GBX_SPARSE: device pointer to the stored count (read for inputs,
                         written for outputs); ignored for GBX_DENSE */
    int32_t capacity; /* GBX_SPARSE: entries `data` can hold; an output needs capacity >= size */
} gbx_vector;

/* ------------------------------------------------------------------ descriptor */

#define GBX_DIR_AUTO 0 /* push or pull chosen on the device (Section 6.3) */
#define GBX_DIR_PUSH 1 /* column-based matvec (Eq 3/5, Algorithm 3) */
#define GBX_DIR_PULL 2 /* row-based matvec (Eq 2/4, Algorithm 2) */

#define GBX_HEUR_RATIO 0  /* Section 6.3: r = nnz(f)/M against alpha (up) and beta (down) */
/* Beamer's test that Section 6.3 starts from: nnz(m_f)/nnz(m_u) > alpha up, nnz(f)/M < beta down */
#define GBX_HEUR_BEAMER 1

/*
 * Operation modifiers.  Section 6.3 carries the sparse/dense switch point
 * as a float in the descriptor; Section 3.2 adds the structural complement;
 * Algorithm 2 adds accumulation and the optional early-exit break; Sections
 * 5.2-5.4 are the BFS-level switches.  Initialise with gbx_desc_init and
 * change fields.
 */
typedef struct {
    int32_t transpose;       /* mxv: 1 computes A^T u (what BFS multiplies by), 0 computes A u */
    int32_t mask_complement; /* use !mask instead of mask (Section 3.2) */
    int32_t early_exit;      /* pull: stop a row at its first hit (Section 5.3; OR semiring only) */
    int32_t accum;           /* w(i) = w_old(i) OR t(i) on passing rows, w_old(i) elsewhere */
    int32_t direction;       /* GBX_DIR_AUTO / PUSH / PULL */
    int32_t heuristic;       /* GBX_HEUR_RATIO or GBX_HEUR_BEAMER (BFS, AUTO only) */
    float alpha;             /* push -> pull threshold (default 0.01) */
    float beta;              /* pull -> push threshold (default 0.01) */
    int32_t masking;         /* BFS pull visits only unvisited rows (Section 5.2; default 1) */
    int32_t operand_reuse;   /* BFS pull tests "visited" instead of "in frontier" (Section 5.4; default 1) */
    int32_t trace;           /* BFS: record per-level statistics (see gbx_bfs_trace) */
    int32_t pull_probe;      /* BFS pull: in-neighbours one lane scans before its warp takes the row over
                                (0 = default: 16 single-source, 8 batched; otherwise 4..1024) */
    int32_t blocks_per_sm;   /* BFS and SSSP kernels: persistent blocks per SM (0 = as many as fit).
                                gbx_bfs_batch and gbx_sssp: 1 or 2 caps the default build (two per
                                SM); 3 or more selects a register-lean build at three per SM (batches:
                                at most 128 sources run alone; server batches keep the default build) */
    int32_t push_sort;       /* gbx_mxv push: 1 = Algorithm 3 / Section 6.2 (gather the selected columns,
                                key-only radix sort, segmented reduction, mask) instead of the one-pass
                                bitmap claim; same result.  Takes the AUTO decision on the host (one
                                stream synchronisation) and allocates its sort buffers per call.
                                gbx_bfs and gbx_bfs_batch reject 1 (GBX_ERR_NOT_SUPPORTED). */
    int32_t reserved[2];     /* must be 0 */
} gbx_desc;

/* Defaults: transpose 1, mask_complement 0, early_exit 1, accum 0,
 * direction AUTO, heuristic RATIO, alpha = beta = 0.01 (Section 6.3),
 * masking 1, operand_reuse 1, trace 0, pull_probe 0, blocks_per_sm 0, push_sort 0. */
void gbx_desc_init(gbx_desc* d);

/* ------------------------------------------------------------------ matvec */

#define GBX_LOR_LAND 0 /* Boolean semiring ({0,1}, OR, AND, 0) of Algorithm 1 */
#define GBX_MIN_PLUS_F32 1 /* tropical semiring (R u {+inf}, +, min, +inf) over binary32, the one
                              Section 5.6 names for SSSP; needs edge weights (gbx_graph_set_weights)
                              and GBX_DENSE_F32 u and w */

/*
 * w = (A u) .* mask  (or A^T u with desc->transpose), over `semiring`.
 * Definition (Eq 2-5): t(i) = OR_j A'(i,j) AND u(j); pass(i) = (mask(i) != 0,
 * 1 if mask is NULL) XOR desc->mask_complement; w(i) = pass(i) ? (accum ?
 * w_old(i) OR t(i) : t(i)) : (accum ? w_old(i) : 0).  The result does not
 * depend on the direction or on early exit (Section 4).
 * Direction: PUSH expands the columns selected by u's nonzeros and dedups
 * them with a bitmap (Eq 5); PULL computes only passing rows, each stopping at
 * its first hit when early_exit is set (Eq 4, Algorithm 2); AUTO picks push
 * when nnz(u)/n <= desc->alpha, else pull, on the device without a host round
 * trip.  u, mask and w may be DENSE or SPARSE; a SPARSE w receives sorted
 * indices and its count in *w->nnz.  All vectors live in device memory and
 * must have size == n.  w must not alias u or mask.  Asynchronous on `stream`.
 * A call's launch sequence depends only on the graph, the vectors' buffers and
 * count addresses, the semiring and the descriptor; it is captured once into a
 * CUDA graph and replayed for later calls with the same ones (the 32 most
 * recent per graph are kept; push_sort calls are issued directly).
 * Errors: NULL_POINTER, NOT_SUPPORTED (semiring), DIMENSION_MISMATCH,
 * INVALID_VALUE (format, capacity < size for a SPARSE output, desc fields).
 *
 * With semiring GBX_MIN_PLUS_F32 (Section 4's generalised semiring, Section
 * 5.6): t(i) = min over entries (i, j) of A' of (A'(i, j) + u(j)), +inf if none;
 * w(i) = pass(i) ? (accum ? min(w_old(i), t(i)) : t(i)) : (accum ? w_old(i) :
 * +inf).  u and w are GBX_DENSE_F32, the mask stays Boolean (DENSE or SPARSE);
 * every sum is one binary32 addition, so w equals the exact result rounded
 * to binary32.  early_exit is ignored (it exists for Boolean semirings only,
 * Section 5.6) and push_sort must be 0 (NOT_SUPPORTED).  PUSH folds u's finite
 * entries' columns into w with atomic minima; PULL computes each passing row.
 * The graph must have weights (INVALID_VALUE otherwise).
 */
gbx_status gbx_mxv(gbx_vector* w, const gbx_vector* mask, int32_t semiring, const gbx_graph* A,
                   const gbx_vector* u, const gbx_desc* desc, void* stream);

/* Work counters of the last gbx_mxv on A that ran with desc->trace = 1 (Table 1's
 * cost terms): rows the pull computed, entries it examined (up to each row's
 * first hit with early exit), nonzeros of u the push expanded, and the edges
 * it expanded (nnz(m_f^+)).  Synchronises the stream of that call.  Any
 * output pointer may be NULL. */
gbx_status gbx_mxv_stats(const gbx_graph* A, int64_t* rows, int64_t* examined, int64_t* u_nnz, int64_t* edges);

/*
 * Allocation-free variant of the pull (row-based) matvec, for callers that
 * cannot allocate device memory when they call in: a serving process whose
 * device memory is all preallocated by its own pool, a latency-bound loop that
 * must not pay for the device-wide synchronisation cudaMalloc/cudaFree can
 * cause, or an embedding that forbids allocation after start-up.  The paper
 * has no counterpart to this entry point.
 * Computes, like gbx_mxv with direction PULL, transpose 0 and accum 0:
 *   w(i) = pass(i) ? OR over j in row i of (u(j) != 0) : 0,
 *   pass(i) = (mask(i) != 0, or 1 when mask is NULL) XOR mask_complement,
 * stopping each row at its first hit when early_exit is set (same result).
 * The matrix is given as caller-owned device CSR arrays row_ptr (int32[n+1]) and
 * col (int32[row_ptr[n]], values in [0, n)); pass the CSR of A^T (for example
 * from gbx_graph_csr with transpose = 1) to compute A^T u as BFS does.
 * u, mask (may be NULL) and w are device uint8_t[n]; w must not alias u or mask.
 * Scratch: four n-bit bitmaps in one fixed device array inside the library, so
 * n is limited to 16777216 (larger n returns GBX_ERR_INVALID_VALUE); the array
 * (8 MiB) stays allocated on every GPU that loads the library until exit.  No
 * cudaMalloc, cudaFree or allocating library routine is called.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress with
 * that device current).  With CUDA's default lazy module loading that first
 * call is also when the library's module, and the 8 MiB array with it, is
 * placed on the device: it can allocate device memory, synchronise, and fail
 * with GBX_ERR_OUT_OF_MEMORY.  So make one warm-up call per device at start-up,
 * before any stream capture; later calls allocate nothing.  The address is kept
 * for the life of the process: do not call this entry point again after
 * cudaDeviceReset on a device it has used.  All
 * calls share the array: calls whose work overlaps on the GPU (different
 * streams, or concurrent host threads) race and must be ordered by the caller.
 * Each call rewrites every scratch word it reads.  Asynchronous on `stream`.
 * Errors: INVALID_VALUE, NULL_POINTER, NOT_SUPPORTED (device index >= 64),
 * OUT_OF_MEMORY (first call: the array could not be placed), CUDA.
 */
gbx_status gbx_mxv_pull_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col, const uint8_t* u,
                                const uint8_t* mask, int32_t mask_complement, int32_t early_exit, uint8_t* w,
                                void* stream);

/* ------------------------------------------------------------------ BFS */

/*
 * Breadth-first search from `source` (Algorithm 1): every level runs the
 * masked matvec f <- A^T f .* !v in the direction the descriptor selects
 * (AUTO: start in push, switch per desc->heuristic after every level, decided
 * on the device).  The whole level loop runs in one persistent cooperative
 * kernel, so no level costs a host round trip.
 * Outputs (device, int32[n], caller-owned): depth[v] = hops from the source
 * (depth[source] = 0, unreached = -1); parent (may be NULL): parent[source] =
 * source, parent[v] = some in-neighbour u of v with depth[u] = depth[v] - 1,
 * unreached = -1.  Asynchronous on `stream`; device-side errors (bounded
 * waits that ran out) are reported by gbx_graph_sync.
 * Errors: NULL_POINTER, INVALID_INDEX (source), INVALID_VALUE (desc), CUDA.
 */
gbx_status gbx_bfs(gbx_graph* g, int32_t source, int32_t* depth, int32_t* parent, const gbx_desc* desc,
                   void* stream);

/*
 * As gbx_bfs for `count` sources, writing into HOST buffers depth_host and
 * parent_host (int32[count][n] each; parent_host may be NULL; pinned memory
 * gives the fastest copies).  Results are computed on the device and copied
 * back while the next source runs (two device buffer sets, a copy stream).
 * Synchronous: returns when every result is in host memory.
 */
gbx_status gbx_bfs_host(gbx_graph* g, const int32_t* sources, int32_t count, int32_t* depth_host,
                        int32_t* parent_host, const gbx_desc* desc, void* stream);

/* Per-level statistics of the last gbx_bfs run with desc->trace = 1. */
typedef struct {
    int32_t direction; /* GBX_DIR_PUSH or GBX_DIR_PULL used for this level */
    int32_t level;     /* L: the level that turns frontier F_L into F_{L+1} */
    int64_t nf;        /* |F_L| */
    int64_t mf;        /* out-edges of F_L, nnz(m_f^+) */
    int64_t nu;        /* vertices not visited before this level */
    int64_t nu_nz;     /* ... of which with nonzero in-degree */
    int64_t mu;        /* in-edges of the unvisited vertices, nnz(m_u^-) (Eq 1) */
    int64_t e_exam;    /* pull levels: in-edges examined, in ascending order, up to each row's
                          first hit (all of them without early exit); -1 on push levels */
    int64_t n_new;     /* |F_{L+1}| */
    int64_t mf_new;    /* out-edges of F_{L+1} */
    int64_t time_ns;   /* device time of this level, barrier to barrier (%globaltimer); level 0
                          includes the initialisation of depth, parent and the visited bitmap */
} gbx_level;

/* Copy the trace of the last traced BFS on g into levels[0..cap) and its
 * length into *nlevels.  Synchronises the graph's last BFS stream. */
gbx_status gbx_bfs_trace(gbx_graph* g, gbx_level* levels, int32_t cap, int32_t* nlevels);

/*
 * Single-source shortest paths over the edge weights (gbx_graph_set_weights),
 * the direction-optimised Bellman-Ford that Section 5.6 sketches for the
 * (min, +) semiring: d <- min(d, A^T d) restricted, while it is small, to the
 * columns of the vertices whose distance improved in the last iteration (push,
 * Eq 5 with atomic minima), and over every row once that set is large (pull,
 * Eq 2 without mask or early exit).  The switch uses Section 6.3's rule on the
 * improved-set size (desc->alpha up, desc->beta down; beta = 0 keeps the two
 * phases of Section 5.6); desc->direction PUSH or PULL forces one.  dist is a
 * device float[n]: dist[source] = 0, +inf where unreachable.  Every relaxation
 * is one binary32 addition; for non-negative weights the result is, per vertex,
 * the smallest left-to-right rounded path sum, independent of the schedule.
 * A negative cycle ends in GBX_ERR_OVERFLOW after n iterations (reported by
 * gbx_graph_sync).  One persistent cooperative launch, asynchronous on
 * `stream`; desc->blocks_per_sm >= 3 selects a register-lean build at three
 * blocks per SM (faster on long push iterations over skewed graphs, slower with
 * pull iterations; GBX_TUNE_SSSP times both).  Errors: NULL_POINTER, INVALID_INDEX, INVALID_VALUE (no weights,
 * desc fields), NOT_SUPPORTED (push_sort), CUDA.
 */
gbx_status gbx_sssp(gbx_graph* g, int32_t source, float* dist, const gbx_desc* desc, void* stream);

/* Per-iteration records of the last traced gbx_sssp on g (synchronises): direction,
 * iteration, nf = vertices improved by the previous iteration (1 for the first),
 * mf = their out-edges (push iterations; -1 on pull), e_exam = edges relaxed,
 * n_new = vertices improved, mf_new, time_ns; nu, nu_nz and mu are -1. */
gbx_status gbx_sssp_trace(gbx_graph* g, gbx_level* levels, int32_t cap, int32_t* nlevels);

/* Depth element types of gbx_bfs_batch. */
#define GBX_DEPTH_I32 0
#define GBX_DEPTH_I16 1 /* a depth of 32767 or more fails with GBX_ERR_OVERFLOW */

/*
 * Batched multi-source BFS: S independent BFS runs (Algorithm 1 for each source)
 * carried together as bit lanes -- lane b of vertex v is one bit of a uint64
 * word, and the Boolean semiring acts lane-wise (OR = bitwise OR over words).
 * Every level runs push (Eq 5 lane-wise, 64-bit atomicOr into the next words) or
 * pull (Eq 4 lane-wise: masking by the unvisited lanes, early exit once every
 * unvisited lane of a vertex has a parent, operand reuse) for the whole batch;
 * with desc->direction = AUTO the device picks pull when the active vertices'
 * out-edges exceed desc->alpha * nnz, else push.  Sources may repeat.
 * sources: host int32[S] in [0, n).  depth: device buffer [S][n] of int32
 * (GBX_DEPTH_I32) or int16 (GBX_DEPTH_I16): depth[b][v] = hops from sources[b],
 * -1 if unreached -- each row equals gbx_bfs from that source.  Scratch (4 x n x W
 * uint64, W = ceil(S/64) rounded up to a multiple of the word chunk 1, 2 or 4, plus
 * int32[n+1]) is allocated on the first call and kept by the graph, grown when a
 * wider batch comes.  desc->blocks_per_sm >= 3 with S <= 128 selects a register-lean
 * build of the kernel at three blocks per SM (faster on skewed graphs with few wide
 * levels, slower on long chains of small ones; GBX_TUNE_BATCH times both).
 * Asynchronous on `stream`; device-side errors are reported by gbx_graph_sync.
 * Errors: NULL_POINTER, INVALID_VALUE (S < 1, depth_type, desc), INVALID_INDEX,
 * NOT_SUPPORTED (push_sort), OUT_OF_MEMORY, CUDA.
 */
gbx_status gbx_bfs_batch(gbx_graph* g, const int32_t* sources, int32_t S, void* depth, int32_t depth_type,
                         const gbx_desc* desc, void* stream);

/* Per-level records of the last gbx_bfs_batch on g (synchronises): direction,
 * nf = active vertices, mf = their out-edges, mu = (vertex, lane) pairs found at
 * the previous level, e_exam = edges examined by pull levels (once per 256-lane
 * chunk), n_new = pairs found at this level, mf_new, time_ns; nu and nu_nz are -1. */
gbx_status gbx_bfs_batch_trace(gbx_graph* g, gbx_level* levels, int32_t cap, int32_t* nlevels);

/* ------------------------------------------------------------------ autotuner */

#define GBX_TUNE_BFS 0   /* single-source gbx_bfs, timed over `count` separate runs */
#define GBX_TUNE_BATCH 1 /* gbx_bfs_batch with the `count` sources as one batch */
#define GBX_TUNE_SSSP 2  /* gbx_sssp, timed over `count` separate runs (the graph needs weights) */

/*
 * Time candidate descriptors on g with the given host sources and return the
 * fastest in *best (and its time in ms in *best_ms, may be NULL).  Section 6.3
 * chose its switch point by comparison with running both directions on every
 * level; here whole descriptors are compared: for GBX_TUNE_BFS the direction
 * rule (ratio / Beamer) x alpha x beta plus the ratio-rule thresholds that
 * gbx_tune_thresholds derives from traced push-only and pull-only runs of up
 * to 8 of the sources, then the pull probe depth and the
 * persistent blocks per SM; for GBX_TUNE_BATCH the batch alpha, then the probe
 * depth; for GBX_TUNE_SSSP alpha x beta (beta 0: two phases), push only and pull
 * only.  Results never change (every candidate computes the same output).  If
 * cache_path is not NULL, a previous result for the same graph shape (n, nnz,
 * symmetric, kind, batch size) is returned from that text file without timing,
 * and new results are appended to it.  Synchronises `stream`.  Allocates a
 * temporary depth buffer.  Errors: NULL_POINTER, INVALID_VALUE, INVALID_INDEX, CUDA.
 */
gbx_status gbx_autotune(gbx_graph* g, int32_t kind, const int32_t* sources, int32_t count, gbx_desc* best,
                        double* best_ms, const char* cache_path, void* stream);

/*
 * Section 6.3 set its switch thresholds by comparison with running both
 * directions on every level.  push and pull are the traces (gbx_bfs_trace, host
 * arrays of nlevels records) of one source's BFS run with direction GBX_DIR_PUSH
 * and GBX_DIR_PULL: the same levels, each timed both ways.  The per-level faster
 * direction is the best schedule (level 0 pushes, as the rule starts), written to
 * schedule[0 .. nlevels) if schedule is not NULL.  *alpha and *beta receive the
 * thresholds of the ratio rule (GBX_HEUR_RATIO) that switch where that schedule
 * switches: to pull at its first pull level, back to push at its first push level
 * after that, as far as the rule's conditions (frontier grew / shrank) allow.
 * alpha = 1e30 when the schedule never pulls, beta = 0 when it never returns to
 * push.  gbx_autotune(GBX_TUNE_BFS) adds these thresholds, from up to 8 of its
 * sources, to its timed candidates.  Host only, no device work.  Errors:
 * NULL_POINTER, INVALID_VALUE (nlevels or n < 1, or traces whose level sizes
 * differ: not one BFS).
 */
gbx_status gbx_tune_thresholds(const gbx_level* push, const gbx_level* pull, int32_t nlevels, int32_t n,
                               float* alpha, float* beta, int32_t* schedule);

/* ------------------------------------------------------------------ server */

/*
 * Continuous-batching BFS server over several resident graphs (the batched
 * form of Algorithm 1 applied to queries as they arrive; the paper runs one
 * source at a time, this is the serving pattern built on gbx_bfs_batch).
 * Queries queue per graph; whenever one of `slots` streams is free, the graph
 * whose oldest query has waited longest sends up to its lane width of queued
 * queries as one batched BFS, each lane writing its depths straight into the
 * query's output row; each slot has its own scratch and its batch's persistent
 * kernel gets 1/slots of the GPU, so batches -- of different graphs or of the
 * same graph -- run side by side.  The graphs are only read by the server.
 */
typedef struct gbx_server gbx_server;

typedef struct {
    int32_t max_batch;     /* sources per batch, <= 4096 (default 64) */
    int32_t slots;         /* batches in flight at once, 1..16 (default 2) */
    int32_t depth_type;    /* GBX_DEPTH_I32 (default) or GBX_DEPTH_I16 output rows */
    float alpha;           /* batch push -> pull threshold, as desc.alpha of gbx_bfs_batch (default 0.05) */
    int64_t max_pending;   /* queued queries beyond which submit fails with GBX_ERR_BUSY (default 65536) */
    int64_t memory_budget; /* device bytes of batch scratch the slots may hold (each slot keeps scratch for
                              the widest batch of any graph); 0 = unlimited.  A graph's lane width is the
                              largest that fits (admission by memory). */
    int32_t reserved[4];   /* must be 0 */
} gbx_server_config;

/* One finished query.  Times are host seconds since the server was created:
 * submitted, its batch launched, its completion observed by submit/poll. */
typedef struct {
    uint64_t tag;
    int32_t graph_id;
    int32_t source;
    int32_t status;     /* GBX_OK, or the error of its batch: recorded on the device, or of its
                           launch (a batch that cannot be launched completes at once) */
    int32_t levels;     /* levels of its batch (max over the batch's lanes) */
    int32_t batch_size; /* queries in its batch */
    int32_t reserved;
    double t_submit;
    double t_launch;
    double t_done;
} gbx_completion;

void gbx_server_config_init(gbx_server_config* c);
/* Create a server (allocates per-slot streams and staging).  Errors: NULL_POINTER,
 * INVALID_VALUE (config), OUT_OF_MEMORY, CUDA. */
gbx_status gbx_server_create(gbx_server** out, const gbx_server_config* cfg);
/* Register a graph (not owned: free it after gbx_server_destroy); reserves its
 * batch scratch within the memory budget.  Errors: OUT_OF_MEMORY when not even one
 * lane fits, INVALID_VALUE if already added. */
gbx_status gbx_server_add_graph(gbx_server* s, gbx_graph* g, int32_t* graph_id);
/* Lane width (sources per batch) the server chose for a graph. */
gbx_status gbx_server_graph_lanes(gbx_server* s, int32_t graph_id, int32_t* lanes);
/* Descriptor of the batches of one graph (direction, alpha, pull_probe as in
 * gbx_bfs_batch; e.g. from gbx_autotune with GBX_TUNE_BATCH on sources of that
 * graph).  Default: gbx_desc_init with alpha = the config's alpha.  Applies to
 * batches launched after the call.  Errors: NULL_POINTER, INVALID_INDEX (graph
 * id), INVALID_VALUE (desc fields), NOT_SUPPORTED (push_sort). */
gbx_status gbx_server_set_graph_desc(gbx_server* s, int32_t graph_id, const gbx_desc* desc);
/* Queue a BFS from `source` on graph `graph_id`; its depths (n entries of the
 * server's depth type, device memory, caller-owned, untouched until the query
 * completes) go to depth_out.  The server's streams do not wait on the caller's:
 * work of other streams on depth_out must have finished before the call.  May
 * start batches.  Errors: BUSY (queue full), INVALID_INDEX, NULL_POINTER. */
gbx_status gbx_server_submit(gbx_server* s, int32_t graph_id, int32_t source, void* depth_out, uint64_t tag);
/* Collect finished batches, start new ones on free slots, and return up to max
 * completions (oldest first) in out; *nout receives how many. */
gbx_status gbx_server_poll(gbx_server* s, gbx_completion* out, int32_t max, int32_t* nout);
/* Queued queries, queries in flight, submissions refused, scratch bytes held. */
gbx_status gbx_server_stats(gbx_server* s, int64_t* queued, int32_t* in_flight, int64_t* rejected,
                            int64_t* scratch_bytes);
/* Wait for batches in flight and release the server (not the graphs). */
gbx_status gbx_server_destroy(gbx_server* s);

/* Upper bound, in nanoseconds, of every device-side wait in this library (the
 * persistent kernels' grid barriers).  When it runs out the kernel records
 * GBX_ERR_TIMEOUT and returns.  Default 5e9.  Process-wide. */
gbx_status gbx_set_wait_timeout_ns(uint64_t ns);

/* Failure-detection self-test: runs the persistent kernels' bounded grid
 * barrier on g's own barrier and status words with one participant that never
 * arrives, so every waiting block runs out of its timeout_ns limit, records
 * GBX_ERR_TIMEOUT and returns.  Until gbx_graph_sync reports (and clears) that
 * error, BFS kernels on g see it at their first barrier and return at once.
 * Asynchronous on `stream`.  Causes no GPU fault. */
gbx_status gbx_selftest_barrier_timeout(gbx_graph* g, uint64_t timeout_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBX_H */
