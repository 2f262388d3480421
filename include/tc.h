/*
 * tc.h -- C ABI of the GB300 exact triangle counter (libtc.so).
 *
 * The library computes the exact number of triangles of an undirected simple
 * graph with the cover-edge method of D. A. Bader, "Fast Triangle Counting"
 * (arXiv 2309.09064), Algorithm 4 with the degree ordering of its Sec. II
 * ("BaderD"):
 *   1. BFS levels L over every component (Algorithm 4, BFS loop; each
 *      component's root is its first vertex in the working order);
 *   2. partition of E into horizontal edges E0 (L(u) == L(v)) and
 *      level-spanning edges E1 (Algorithm 4, partition loop);
 *   3. triangles inside G0 by the forward method on G0 oriented by the
 *      working order (Algorithm 2, called from Algorithm 4);
 *   4. triangles with one horizontal edge by intersecting the G1 lists of the
 *      two endpoints of every horizontal edge (Algorithm 4, hashed loop);
 *   5. T = (3) + (4), an exact 64-bit integer.
 * Every step runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions
 *   - Vertex ids are uint32_t in [0, n), n < 2^32 - 1.  Row offsets are
 *     uint64_t.  A CSR is (row_ptr[n+1], col[row_ptr[n]]): symmetric, no
 *     self-loops, no repeated entries, each row ascending.
 *   - Pointers marked "host" are ordinary (ideally pinned) host memory;
 *     "device" pointers are CUDA global memory of the context's device.
 *   - Inputs are never written (the paper's read-only input convention,
 *     Sec. III).  The library allocates its scratch memory itself (a
 *     context-owned arena reused across calls and released by tc_destroy)
 *     and never leaks it.
 *   - Every function returns a tc_status.  The library never aborts, prints
 *     or traps; on failure tc_last_error(ctx) gives a one-line message.
 *   - A context is not thread-safe: one host thread at a time per context,
 *     except tc_submit / tc_poll which are safe from any thread.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tc_status {
    TC_OK = 0,
    TC_ERR_INVALID = 1,   /* bad argument or malformed graph */
    TC_ERR_OOM = 2,       /* device or host allocation failed */
    TC_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    TC_ERR_TIMEOUT = 4,   /* a bounded device wait gave up */
    TC_ERR_BUSY = 5,      /* request queue full */
    TC_NOT_READY = 6,     /* tc_poll: result not ready yet */
    TC_ERR_CAPACITY = 7   /* tc_list_triangles: more triangles than the output holds */
} tc_status;

typedef struct tc_ctx tc_ctx;
typedef struct tc_graph tc_graph;

/* where a pointer lives */
enum { TC_HOST = 0, TC_DEVICE = 1 };

/* tc_graph_from_csr flags */
enum {
    TC_COPY = 0,       /* copy the arrays into library-owned device memory */
    TC_BORROW = 1,     /* keep the caller's DEVICE pointers (must outlive the graph) */
    TC_VALIDATE = 2    /* check symmetry, order, loops, repeats and bounds first */
};

/* vertex working order (Sec. II): which vertex is "smaller" in u < v */
enum {
    TC_ORDER_DEGREE = 0,  /* BaderD: decreasing degree, ties by ascending id (default) */
    TC_ORDER_ID = 1       /* Bader: ascending vertex id */
};

typedef struct tc_options {
    uint32_t order;        /* TC_ORDER_DEGREE or TC_ORDER_ID */
    uint32_t flags;        /* reserved, 0 */
    void *stream;          /* cudaStream_t to run on; NULL: the context creates its own */
    uint32_t max_queue;    /* tc_submit queue capacity (0: 65536) */
    uint32_t reserved[7];
} tc_options;

/* Per-call statistics (tc_count).  Counts are exact. */
typedef struct tc_stats {
    uint64_t n;                 /* vertices */
    uint64_t m;                 /* undirected edges (row_ptr[n] / 2) */
    uint64_t triangles;         /* T */
    uint64_t t_same;            /* triangles wholly inside G0 (step 3) */
    uint64_t t_cross;           /* triangles with one horizontal edge (step 4) */
    uint64_t horizontal_edges;  /* |E0| */
    uint64_t levels;            /* number of BFS levels (max L + 1) */
    uint64_t components;        /* BFS roots (components, isolated vertices included) */
    uint64_t probes;            /* elements probed in steps 3-4 */
    uint64_t row2_slots;        /* total length of the compacted [G0 out | G1] rows */
    uint64_t alg_bytes;         /* algorithmic bytes of the whole count (traffic model) */
    uint64_t isect_bytes;       /* algorithmic bytes of the intersection stage alone */
    float ms_total;             /* device time of the whole count */
    float ms_levels;            /* degrees + BFS levels */
    float ms_mark;              /* partition, orientation, compaction, planning */
    float ms_isect;             /* intersections + reduction */
    /* intersection classes: [0] warp (shared table per warp), [1] block (shared table), [2] hub (L2
       bitmaps + shared prefilter), [3] tiny (thread-per-row sorted merges) */
    uint64_t class_rows[4];     /* tasks (warp, block, hub) or rows (tiny) */
    uint64_t class_probes[4];   /* probed elements */
    uint64_t class_bytes[4];    /* algorithmic bytes: hashed rows once + probed rows */
    float ms_class[4];          /* device time of each class's kernel (0 if not launched) */
    uint64_t class_inserts[4];  /* table / prefilter inserts done, rebuilds on other blocks included */
    uint32_t launches;          /* kernels this call launched */
    uint32_t reserved;
} tc_stats;

/*
 * Launch-shape knobs of the intersection stage (Algorithm 4's hashed loop):
 * rows are classed by the size s(u) of the hashed row of the first endpoint.
 */
typedef struct tc_tuning {
    uint32_t warp_cap;         /* s(u) <= warp_cap: one warp per task, per-warp shared table (1..4096) */
    uint32_t block_cap;        /* s(u) <= block_cap: one block per task, shared table (warp_cap..16384, see
                                  table_kind);
                                  larger rows are hub rows (L2 bitmaps + shared prefilter) */
    uint32_t task_work;        /* target probes per block task (large rows are split) */
    uint32_t warps_per_block;  /* warp-class kernel block size in warps (1..8) */
    uint32_t block_threads;    /* block-class kernel threads (64..1024, multiple of 32) */
    uint32_t warp_task_work;   /* target probes per warp task */
    uint32_t hub_task_work;    /* target probes per hub task */
    uint32_t max_v;            /* out-neighbour rows per block / hub task (64..4096) */
    uint32_t hub_group;        /* hub rows probed per launch, one n-bit bitmap each (1..64); plain counts
                                  run two groups at a time on two streams and keep 2 x hub_group bitmaps */
    uint32_t hub_filter_log2;  /* hub prefilter size: 2^k bits of shared memory (10..20) */
    uint32_t hub_threads;      /* hub kernel threads (64..1024, multiple of 32) */
    uint32_t tiny_cap;         /* s(u) <= tiny_cap (and degree <= 4 tiny_cap, |G1(u)| <= 8): one thread per
                                  row, sorted merges instead of a table; takes precedence over the classes
                                  above (0..64; 0 turns it off) */
    uint32_t table_kind;        /* shared-memory sets of the warp and block classes: 0 two-choice cuckoo
                                   tables (two 32-bit loads per lookup; block_cap up to 13107), 1 bucketed
                                   tables (block_cap up to 16384) */
    uint32_t flat_cap;          /* warp class: probe ranges shorter than this are concatenated so that every
                                   lane of a warp has work; longer ones are walked range by range (0..4096) */
    uint32_t block_bits_log2;   /* plain counts, block class with cuckoo tables: the set's ranks below 2^k
                                   live in a direct bitmap in shared memory (one bit per rank, 2^k / 8 bytes),
                                   only the others in the cuckoo table, which shrinks to fit beside it (rows
                                   whose other ranks do not fit go to the hub class); the rows stage puts
                                   every level-spanning part's ranks below 2^k first, and probe pieces below
                                   and above 2^k take one kind of lookup each.  0 turns it off; else 10..20 */
    uint32_t batch_small_slots; /* tc_count_batch / serving: graphs of at most 65536 vertices and at most this
                                   many CSR slots are counted one thread block each, all in one launch; the
                                   others as one disjoint union through the pipeline (0: all of them) */
    uint32_t reserved[2];
} tc_tuning;

/* ------------------------------------------------------------------ context */

/*
 * Create a context on CUDA device `device`; opt (host, nullable: defaults) is
 * copied.  No counterpart in the paper, whose counters are single serial
 * functions: the context holds what Sec. III charges to every count -- the
 * scratch memory (one grow-only device arena, reused by later counts on the
 * context and freed by tc_destroy), the stream and the tuning.  *out gets the
 * context; TC_ERR_CUDA if the device cannot be used, TC_ERR_OOM if host
 * memory runs out.
 */
tc_status tc_create(tc_ctx **out, int device, const tc_options *opt);
/* Destroy a context: waits for its work, frees its arena and request slots
 * (Sec. III: all auxiliary memory is freed; nothing leaks).  Graphs made on
 * the context must be freed first. */
tc_status tc_destroy(tc_ctx *ctx);
/* One-line description of the last error on this context ("" if none; the
 * string is owned by the context).  No counterpart in the paper. */
const char *tc_last_error(const tc_ctx *ctx);
/* Run subsequent work on `stream` (a cudaStream_t owned by the caller, which
 * must outlive its use; NULL: the context's own).  No counterpart in the
 * paper. */
tc_status tc_set_stream(tc_ctx *ctx, void *stream);
/* Copy the context's tuning (the launch-shape knobs of Algorithm 4's hashed
 * loops, above) to *out (host). */
tc_status tc_get_tuning(const tc_ctx *ctx, tc_tuning *out);
/* Replace the context's tuning with a copy of *t (host), used from the next
 * count on; TC_ERR_INVALID (tuning unchanged) if a field is out of its range
 * or the kernels' shared memory would not fit.  Any valid tuning gives the
 * same exact counts (it only reshapes the hashed loops of Algorithm 4). */
tc_status tc_set_tuning(tc_ctx *ctx, const tc_tuning *t);
/* Bytes of device memory currently held by the context's arena (*bytes,
 * host): the auxiliary memory that Sec. III charges to the count. */
tc_status tc_arena_bytes(const tc_ctx *ctx, uint64_t *bytes);

/*
 * No counterpart in the paper (failure handling of this library).
 * Self-test of the bounded device-wide wait used by the persistent BFS: one
 * launch waits at a grid barrier that can never complete (one arrival is
 * missing), gives up after timeout_ms (1..10000) and reports it.  Returns
 * TC_ERR_TIMEOUT when the wait ended as designed; the context stays usable.
 * Fault injection: if the environment variable TC_FAIL_ALLOC_AT=k is set when
 * a context is created, the context's k-th device allocation fails (once)
 * and the call that made it returns TC_ERR_OOM with nothing leaked.
 */
tc_status tc_selftest_barrier(tc_ctx *ctx, uint32_t timeout_ms);

/* ------------------------------------------------------------------- graphs */

/*
 * Build the CSR of the simple undirected graph spanned by n_tuples tuples
 * (src[i], dst[i]): the input form of the method (Sec. I: an undirected
 * graph G = (V, E) stored in CSR; the paper takes that CSR as given, so the
 * build itself has no counterpart there).  Both directions are added,
 * self-loops dropped, repeats removed and rows sorted (device radix sort).
 * src/dst are host or device arrays (`where`), uint32_t[n_tuples] each,
 * read only.  Ids >= n give TC_ERR_INVALID; TC_ERR_OOM if device memory runs
 * out.  *out gets a graph that owns its device arrays (tc_graph_free).
 */
tc_status tc_build_csr(tc_ctx *ctx, uint32_t n, uint64_t n_tuples, const uint32_t *src,
                       const uint32_t *dst, int where, tc_graph **out);

/*
 * Wrap an existing CSR (row_ptr[n+1], col[row_ptr[n]]), host or device
 * (`where`): the paper's input, one undirected graph in CSR (Sec. I), treated
 * as read only (Sec. III).  TC_COPY copies into library memory (host input
 * is always copied); TC_BORROW keeps device pointers (caller keeps them
 * alive and unchanged).  TC_VALIDATE runs the well-formedness check
 * (symmetric, rows ascending, no loops, no repeats, ids < n) and returns
 * TC_ERR_INVALID on the first violation; without it a malformed CSR gives
 * unspecified counts.  *out gets the graph (tc_graph_free).
 */
tc_status tc_graph_from_csr(tc_ctx *ctx, uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                            int where, int flags, tc_graph **out);

/* Device pointers and sizes of a graph (valid until tc_graph_free); any
 * output pointer may be NULL.  No counterpart in the paper. */
tc_status tc_graph_info(const tc_graph *g, uint32_t *n, uint64_t *slots, const uint64_t **d_row_ptr,
                        const uint32_t **d_col);

/*
 * Copy a graph's CSR out: row_ptr gets n+1 offsets, col gets row_ptr[n] ids,
 * into host or device buffers (`where`) the caller owns.  Blocks until the
 * copy is done.  No counterpart in the paper.
 */
tc_status tc_graph_copy_out(tc_ctx *ctx, const tc_graph *g, uint64_t *row_ptr, uint32_t *col, int where);

/* Check a graph's CSR against the input the method assumes (Sec. I: a simple
 * undirected graph -- symmetric, ascending rows, no loops, no repeats);
 * *ok (host) = 1 if well formed, 0 otherwise. */
tc_status tc_validate(tc_ctx *ctx, const tc_graph *g, int *ok);

/* Release a graph (and its device arrays unless borrowed): the library
 * frees what it allocated (Sec. III).  NULL is accepted. */
tc_status tc_graph_free(tc_graph *g);

/* ----------------------------------------------------------------- counting */

/*
 * Exact triangle count of g (Algorithm 4, steps 1-5 above).  *triangles gets
 * T; stats (nullable) gets the breakdown.  Blocks until the result is on the
 * host.
 */
tc_status tc_count(tc_ctx *ctx, const tc_graph *g, uint64_t *triangles, tc_stats *stats);

/*
 * Same as tc_count, and additionally writes the BFS level of every vertex to
 * d_levels (device uint32_t[n], nullable) -- the L of Algorithm 4 under the
 * context's working order.
 */
tc_status tc_count_levels(tc_ctx *ctx, const tc_graph *g, uint32_t *d_levels, uint64_t *triangles,
                          tc_stats *stats);

/*
 * Triangles through every vertex (Sec. I names clustering coefficients as a
 * use of triangle counts): d_counts (device uint64_t[n], written by
 * the library) gets t(x), the number of triangles containing x, and
 * *triangles gets T (sum of t(x) = 3T).  The local clustering coefficient of
 * x is 2 t(x) / (d(x) (d(x) - 1)).  Same method as tc_count; each triangle
 * found adds one to its three vertices (one atomic per triangle for the
 * third vertex, so this mode is slower than tc_count).
 */
tc_status tc_count_vertices(tc_ctx *ctx, const tc_graph *g, uint64_t *d_counts, uint64_t *triangles,
                            tc_stats *stats);

/*
 * Count with levels the caller already has (Sec. III: the method pays most
 * where a BFS has been run anyway): d_levels is a device
 * uint32_t[n], read only, e.g. the hop distances of any BFS forest.  The BFS
 * of Algorithm 4 is skipped; everything else is as in tc_count.  The count is
 * exact for any labelling in which the two ends of every edge differ by at
 * most one level (then every triangle has one or three horizontal edges);
 * the library checks that on the device and returns TC_ERR_INVALID if some
 * edge breaks it.  t_same / t_cross and |E0| follow the given levels.
 */
tc_status tc_count_with_levels(tc_ctx *ctx, const tc_graph *g, const uint32_t *d_levels, uint64_t *triangles,
                               tc_stats *stats);

/*
 * Algorithm 3 (cover-edge triangle counting, Sec. III) as a comparison
 * kernel: the same BFS levels and working order as tc_count, then for every
 * horizontal edge u -> v (u earlier) the full intersection of N(u) and N(v)
 * on the CSR as given, a common neighbour w counting when it lies on another
 * level or on the same level after v.  Same T and t_same / t_cross as
 * tc_count with more work per edge (stats->probes = elements of both rows
 * over all horizontal edges); ms_isect is this kernel's time.
 */
tc_status tc_count_alg3(tc_ctx *ctx, const tc_graph *g, uint64_t *triangles, tc_stats *stats);

/*
 * List every triangle of g exactly once.  Algorithm 4 finds each triangle
 * once (one or three horizontal edges; Sec. III), so its hits are the list:
 * d_triples (device uint32_t[3 * capacity], nullable when capacity is 0)
 * gets T rows {u, v, w} of vertex ids -- u the vertex whose set was hashed,
 * v the probed one (u -> v a horizontal edge, u earlier in the working
 * order), w the third vertex -- in no particular order; *triangles gets T.
 * One pass of the intersections: every warp writes the triangles it finds
 * into chunks of output rows it takes from a global cursor; a compaction
 * then moves the rows written past T into the gaps the last, partly filled
 * chunks left (rows past T are scratch: their contents are unspecified).
 * The tiny rows (one thread each) are counted first and written at exact
 * offsets after the others.  If T > capacity the call returns
 * TC_ERR_CAPACITY with *triangles = T (the output rows are unspecified), so
 * that the caller can size the output and call again.  stats as in tc_count
 * (the class times are those of the listing kernels).
 */
tc_status tc_list_triangles(tc_ctx *ctx, const tc_graph *g, uint32_t *d_triples, uint64_t capacity,
                            uint64_t *triangles, tc_stats *stats);

/*
 * One shard of a count split across nshards processes or devices (the
 * multi-GPU form of the method, Sec. V: BFS levels and rows are computed in full on
 * every shard, the intersection tasks -- contiguous slices of the oriented
 * horizontal edges, of about equal probe work -- are divided, and the exact
 * total is the sum of the nshards partial counts, one 8-byte exchange).
 * *partial gets this shard's share; shard < nshards.
 */
tc_status tc_count_shard(tc_ctx *ctx, const tc_graph *g, uint32_t shard, uint32_t nshards, uint64_t *partial,
                         tc_stats *stats);

/*
 * Count G independent graphs in one batched launch sequence.  No counterpart
 * in the paper (it counts one graph per call): each graph's count is
 * Algorithm 4 exactly as in tc_count, the G graphs run as one disjoint union
 * (Sec. V names parallelising the BFS, the partition and the intersections;
 * here they run over all graphs at once).  graphs: host array of G graph
 * handles (read only, any mix of sizes); counts: host uint64_t[G], written
 * on success.  Every count equals tc_count on the same graph.  TC_ERR_OOM if
 * the union does not fit in device memory.
 */
tc_status tc_count_batch(tc_ctx *ctx, uint32_t G, const tc_graph *const *graphs, uint64_t *counts);

/*
 * Exact count of one small graph that allocates nothing (no counterpart in
 * the paper; an interface for callers that cannot allocate device memory when
 * they count, e.g. code running inside another allocator or a process whose
 * memory pool already owns the whole device).  Same method and same results
 * as tc_count, run by one thread block with all scratch in a fixed array of
 * device memory declared in the library (about 5.8 MB).
 *   d_row_ptr, d_col: device CSR (well formed, as for TC_BORROW), n <= 65536
 *     vertices, slots = row_ptr[n] <= 1048576 (TC_ERR_INVALID beyond that);
 *   order: TC_ORDER_DEGREE or TC_ORDER_ID;
 *   d_out: device uint64_t[4], written when the stream reaches the kernel:
 *     [0] = T, [1] = triangles inside G0, [2] = cross-level triangles,
 *     [3] = 0 on success, 1 if the device saw row_ptr[n] beyond the limit
 *     (then [0..2] = 0);
 *   stream: cudaStream_t (NULL: the legacy default stream).
 * Asynchronous: returns after the launch; TC_ERR_CUDA if the launch itself
 * failed (an earlier, unrelated CUDA error of the process is neither reported
 * nor cleared).  Every call shares the one array, so calls that overlap on
 * the GPU (other streams or threads) race; serialise them.
 * Set-up: the CUDA driver loads a library's device code lazily by default,
 * so the array is allocated on a device by the first call on that device
 * (which looks up its address); only later calls allocate nothing.  Make a
 * first call on every device at start-up, before memory is handed out (n = 0
 * with a one-element row_ptr holding 0 is enough), and outside any stream
 * capture.  The array then stays until the process exits.  Cost: O(n + m)
 * for the levels (all components at once) plus the hashed intersections.
 */
tc_status tc_count_noalloc(const uint64_t *d_row_ptr, const uint32_t *d_col, uint32_t n, uint64_t slots,
                           uint32_t order, uint64_t *d_out, void *stream);

/* ------------------------------------------------------------------ serving */

/*
 * Queue a count of g (which must stay alive until its ticket completes) and
 * return at once with a ticket (*ticket, host).  No counterpart in the paper
 * (the served form of the counter); every result is Algorithm 4's exact T,
 * as tc_count gives it.  Server threads owned by the context admit queued
 * requests while free device memory allows, batch them, and overlap their
 * work on the device; large graphs go to a lane of their own so that they
 * do not hold up small ones.  TC_ERR_BUSY if the queue is full.
 */
tc_status tc_submit(tc_ctx *ctx, const tc_graph *g, uint64_t *ticket);

/*
 * Non-blocking: TC_OK with *triangles (host) set to T when the ticket is done
 * (the ticket is then released), TC_NOT_READY while it is queued or running,
 * another status if it failed or the ticket is unknown.  No counterpart in
 * the paper (served form).
 */
tc_status tc_poll(tc_ctx *ctx, uint64_t ticket, uint64_t *triangles);

/*
 * tc_poll that also returns the request's latency in nanoseconds
 * (*latency_ns, host, nullable), from its tc_submit to the moment the server
 * published its result (the library's steady clock), so a client that polls
 * late does not inflate it.  No counterpart in the paper (served form).
 */
tc_status tc_poll_ex(tc_ctx *ctx, uint64_t ticket, uint64_t *triangles, uint64_t *latency_ns);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
