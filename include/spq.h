/*
 * spq.h — shortest-path distance queries on a partitioned undirected graph, on one GPU.
 *
 * The data structure is the one of Chapuis & Djidjev, "Shortest-Path Queries in Planar
 * Graphs on GPU-Accelerated Architectures" (arXiv 1503.07192):
 *   - Algorithm 1, per-component step: for every component C of a given k-partition, the table
 *     APSP(C) of distances dist_C inside the subgraph induced by C (Sec. 2 defines
 *     dist_H for a subgraph H);
 *   - Algorithm 1, clique edges and BG: the boundary graph BG on all boundary vertices (Sec. 2:
 *     vertices with a neighbour in another component), with G's edges between boundary
 *     vertices plus one edge per pair of boundary vertices of a component, weighted
 *     dist_C;
 *   - Algorithm 1, APSP of BG: all-pairs distances in BG (Lemma 1: they equal the
 *     distances in G), held as one |BG| x |BG| matrix, rows and columns grouped by
 *     component (Sec. 4, Fig. 1);
 *   - Algorithm 2 (correct by Lemma 3): dist(v1, v2) = min over b1 in B(C1), b2 in B(C2)
 *     of dist_C1(v1, b1) + dist_BG(b1, b2) + dist_C2(b2, v2), and, if C1 = C2, also
 *     dist_C1(v1, v2).
 * Every step runs in CUDA kernels on the device of the stream passed in.
 *
 * Conventions for every call:
 *   - Pointer arguments may point to host memory or to device memory of the current
 *     device; the library tells them apart with cudaPointerGetAttributes.  Inputs are
 *     borrowed for the duration of the call only; outputs are owned by the caller.
 *   - A handle lives on the device that was current when it was built; every call that
 *     takes a handle must be made with that device current (SPQ_EINVAL otherwise, before
 *     any work is queued).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is queued on
 *     it.  spq_build returns after its work has completed.  spq_query with host output
 *     returns after the results are in host memory; with device output it returns once
 *     the work is queued (read the result after synchronising the stream, and call
 *     spq_query_status for range errors).
 *   - Nothing aborts or prints: every failure is a returned spq_status.
 */
#ifndef SPQ_H
#define SPQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spq_handle spq_handle; /* opaque; owns all device tables of one graph */

typedef enum {
    SPQ_OK = 0,
    SPQ_EINVAL = 1,       /* malformed input: see spq_build / spq_query */
    SPQ_ENOMEM = 2,       /* the tables do not fit in free device memory, or host malloc failed */
    SPQ_ECUDA = 3,        /* a CUDA runtime call failed (the CUDA error is kept: spq_last_cuda_error) */
    SPQ_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    SPQ_EUNSUPPORTED = 5, /* a valid request this build does not handle (e.g. dtype) */
} spq_status;

typedef enum {
    SPQ_I32 = 0, /* int32 edge weights and distances; results are exact */
    SPQ_F32 = 1, /* float32 edge weights and distances (IEEE single-precision sums) */
} spq_dtype;

/* Distance reported for an unreachable pair in SPQ_I32 mode (2^29).  Every finite
 * distance must be below it; the sum of three table entries then stays below 2^31.
 * In SPQ_F32 mode an unreachable pair reports +infinity. */
#define SPQ_INF_I32 0x20000000

/* How the min-plus arithmetic of the Floyd-Warshall steps is carried out for SPQ_I32
 * graphs.  Both give bit-identical results; see spq_build. */
typedef enum {
    SPQ_ARITH_AUTO = 0, /* float32 when exact (see below), else int32 */
    SPQ_ARITH_I32 = 1,  /* int32 add and min */
    SPQ_ARITH_F32 = 2,  /* float32 add and min over exact integers, falling back to int32 */
} spq_arith;

/* Order of the boundary vertices along the boundary-graph matrix.  Floyd-Warshall gives
 * the same distances for any order of its intermediate vertices; the order decides how
 * many tile updates are provably no-ops (an all-infinite pivot panel) and skipped. */
typedef enum {
    SPQ_ORDER_AUTO = 0,       /* the cheapest of the orders below, by a symbolic cost model */
    SPQ_ORDER_ID = 1,         /* grouped by component, components in id order (the
                                 paper's Fig. 1 layout) */
    SPQ_ORDER_DISSECTION = 2, /* grouped by component, components in nested-dissection
                                 order of the component adjacency graph */
    SPQ_ORDER_VERTEX_DISSECTION = 3 /* the same bisections refined to vertex level: only
                                 the boundary vertices on a cut become separator vertices */
} spq_order;

/* How the boundary graph's all-pairs distances D are computed (Algorithm 1's APSP of
 * BG; both give the same D).
 *   SPQ_BG_FW: three-phase blocked Floyd-Warshall, every round over the whole matrix.
 *   SPQ_BG_ELIM: the same rounds restricted to the tiles right of and below the pivot
 *     (block elimination in the (min, +) semiring), then back-substitution from the last
 *     row block to the first: for row block R, d(R, J) = min over the columns k right of
 *     R with a finite eliminated entry F(R, k) of F(R, k) + d(k, J).  Exact for any
 *     order; far fewer updates than Floyd-Warshall when the order is a dissection order
 *     (few such k per row block).
 *   SPQ_BG_AUTO (default): SPQ_BG_ELIM when the chosen order is a dissection order,
 *     else SPQ_BG_FW. */
typedef enum {
    SPQ_BG_AUTO = 0,
    SPQ_BG_FW = 1,
    SPQ_BG_ELIM = 2
} spq_bg_method;

typedef struct spq_opts {
    int32_t struct_size; /* sizeof(spq_opts); lets later versions grow the struct */
    int32_t arith;       /* spq_arith */
    int32_t order;       /* spq_order */
    int32_t skip_inf_tiles; /* 1 (default when opts is NULL): the boundary-graph
                               Floyd-Warshall skips tile updates whose pivot row or
                               column panel is entirely infinite (they cannot change
                               anything); 0: update every tile every round */
    int32_t profile_kernels; /* 1: time every launch of the boundary-graph
                               Floyd-Warshall's phase-3 kernel with CUDA events (see
                               spq_build_profile); 0 (default): no per-launch events */
    int32_t query_grouped;  /* 1 (default): spq_query batches of >= 4096 pairs are sorted
                               by component pair (stream-ordered scratch of 16 bytes per
                               pair) so that each boundary-graph block is read once per
                               group; 0: one warp per pair in input order, no scratch */
    int32_t bg_method;      /* spq_bg_method.  A struct_size that ends before this field
                               (an earlier version of the struct) means SPQ_BG_AUTO */
    int32_t bg_panel_mib;   /* SPQ_BG_ELIM: most MiB of device scratch for the gathered
                               back-substitution panels at a time (the row blocks are
                               then done in several launches); 0 (default): 1024 */
    int32_t comp_method;    /* spq_bg_method for the component tables APSP(C): SPQ_BG_FW
                               blocked Floyd-Warshall; SPQ_BG_ELIM elimination +
                               back-substitution in a nested-dissection order of each
                               component (components of up to 4096 vertices; larger ones
                               take Floyd-Warshall); SPQ_BG_AUTO (default, and what a
                               struct_size ending before this field means): elimination */
    int32_t query_kernel;   /* kernel of the grouped queries.  0 (default, and what a
                               struct_size ending before this field means): a persistent
                               kernel stages each boundary-graph block in shared memory with
                               asynchronous copies, pipelined across blocks (blocks with up
                               to 512 rows and columns; larger ones as with 1); 1: every block
                               gathered by the earlier kernel (autotuned between two
                               configurations, see spq_query_tuning) */
} spq_opts;

/* Fill *opts with the defaults (also what opts == NULL means). */
void spq_opts_default(spq_opts* opts);

/*
 * Build the query structure for the undirected graph G and the k-partition `part`.
 *
 *   n        number of vertices, >= 1
 *   row_ptr  int64[n + 1], CSR row offsets; row_ptr[0] = 0, nondecreasing; m = row_ptr[n]
 *   col      int32[m], neighbour ids in [0, n)
 *   w        int32[m] (SPQ_I32) or float[m] (SPQ_F32): weight of the CSR slot
 *   wt       element type of w
 *   part     int32[n], part[v] in [0, k): the component of v (Sec. 2's k-partition;
 *            components may be disconnected or have no boundary vertex)
 *   k        number of components, >= 1 (empty components are allowed)
 *   opts     NULL for the defaults
 *   stream   cudaStream_t to queue the work on
 *   out      receives the handle (NULL on failure)
 *
 * G must be symmetric: for every slot u -> v (u != v) there is a slot v -> u, and the
 * smallest weight over the parallel slots u -> v equals that over v -> u.  Parallel
 * slots are allowed (the smallest weight is the edge's weight, as a path takes the
 * lightest) and self-loops are ignored.  Weights must be >= 0 (and finite for SPQ_F32);
 * SPQ_I32 weights must be below SPQ_INF_I32, and every finite distance must be too.
 *
 * Arithmetic: with SPQ_ARITH_AUTO or _F32 the Floyd-Warshall updates of an SPQ_I32
 * graph run in float32 and the library then checks that every finite table entry is
 * below 2^24; below that bound each stored value is an exact integer (a float32 sum of
 * two exact integers whose result is below 2^24 is exact, and a sum at or above 2^24
 * never rounds below 2^24), so the tables equal the int32 ones.  If the check fails the
 * build is redone with int32 arithmetic.
 *
 * Errors: SPQ_EINVAL for n < 1, k < 1, a bad row_ptr, col or part entry, a negative or
 * non-finite weight, an SPQ_I32 weight >= SPQ_INF_I32, or an asymmetric graph; SPQ_ENOMEM if the tables (about
 * 4 * (sum over C of |C|^2 + |BG|^2) bytes, rows padded to 4 entries) exceed free device
 * memory; SPQ_ECUDA on a CUDA failure.  On error nothing is leaked and *out is NULL.
 */
spq_status spq_build(int32_t n, const int64_t* row_ptr, const int32_t* col, const void* w, spq_dtype wt,
                     const int32_t* part, int32_t k, const spq_opts* opts, void* stream, spq_handle** out);

/*
 * Answer q distance queries (Algorithm 2 for each pair).
 *
 *   pairs     int32[q][2]: (v1, v2) vertex ids of the original numbering
 *   q         number of pairs, >= 0 (0 is a no-op)
 *   dist_out  int32[q] (SPQ_I32 graphs) or float[q] (SPQ_F32) : dist(v1, v2);
 *             SPQ_INF_I32 / +inf if v2 is unreachable from v1; 0 if v1 == v2
 *   pairs and dist_out must both be host memory or both device memory.
 *
 * A pair with an id outside [0, n) yields -1 (SPQ_I32) or NaN (SPQ_F32) in its slot and
 * marks the handle: with host buffers the call then returns SPQ_EINVAL; with device
 * buffers, spq_query_status reports it.
 *
 * Kernel choice: with the default query_kernel (0), batches of at least 4,096 pairs are
 * answered by the staged kernel (blocks of up to 512 boundary vertices; wider ones by the
 * gathering kernel).  For the gathering kernel (query_kernel = 1, and those wider
 * blocks), the first launch of a size class (see spq_query_tuning) in the process runs
 * both of its configurations on its inputs, timed with CUDA events (the answers are the
 * same), so that call costs about twice that kernel's device time; the host does not wait
 * for the timing, which a later launch of the class reads once it is complete.
 */
spq_status spq_query(spq_handle* h, const int32_t* pairs, int64_t q, void* dist_out, void* stream);

/*
 * spq_query without memory allocation (the paper has no counterpart: it is for callers
 * of this library that cannot let it allocate device memory on their request path, such
 * as a serving process that has given all free device memory to its own pool or runs
 * under a fixed budget where an allocation could fail or stall).
 *
 * Same results and rules as spq_query, except:
 *   - q <= SPQ_NOALLOC_MAX_PAIRS (a larger q returns SPQ_EINVAL and queues nothing);
 *   - pairs and dist_out must be device memory (else SPQ_EINVAL); the call returns once
 *     the work is queued, and spq_query_status reports out-of-range pairs;
 *   - its scratch is one fixed array of about 23.1 MB in the library's device memory,
 *     present on every GPU that loads the library until the process exits.  The first
 *     call on a device looks up that array's address (cudaGetSymbolAddress, once per
 *     device); make that first call before any stream capture.  All calls share the
 *     array, so calls whose work overlaps on the GPU race: order them (one stream, or
 *     events).
 * It calls no allocation routine (no cudaMalloc, cudaMallocAsync or cudaFree).
 */
#define SPQ_NOALLOC_MAX_PAIRS 262144
spq_status spq_query_noalloc(spq_handle* h, const int32_t* pairs, int64_t q, void* dist_out, void* stream);

/*
 * Many independent graphs at once (the batching pattern: many small planar instances of
 * uneven size).  graphs[i] describes instance i exactly as spq_build's arguments do (all
 * with the same weight type); outs[i] receives its handle.  The instances share one
 * device allocation (released with the last of their handles) and, where the work
 * allows, the same kernel launches: validation with one readback for all, one stable
 * sort of every instance's vertices, the component Floyd-Warshall of all components of
 * all instances, and the boundary-graph Floyd-Warshall of all instances round by round.
 * Results are identical to building each instance with spq_build.  On error no handle is
 * returned (every outs[i] is NULL).  spq_stats of such a handle reports the whole batch's
 * boundary-graph update count.
 */
typedef struct spq_graph {
    int32_t n;
    const int64_t* row_ptr;
    const int32_t* col;
    const void* w;
    spq_dtype wt;
    const int32_t* part;
    int32_t k;
} spq_graph;
spq_status spq_build_many(int32_t count, const spq_graph* graphs, const spq_opts* opts, void* stream,
                          spq_handle** outs);

/*
 * Build plan (CUDA graph) for re-weighting: Algorithm 1 on the same `count` graphs and
 * partitions, again and again, with new edge weights.  spq_build_plan_create takes the
 * arguments of spq_build_many (host or device arrays; the plan copies them, so they may be
 * freed on return), builds once, and captures the weight-dependent launches (component
 * tables, boundary-graph assembly and all-pairs distances, exactness check) into one CUDA
 * graph; the steps that depend on the structure alone (numbering, boundary-slot order,
 * elimination forms and their frontier bookkeeping) are not repeated.
 *   handles[count] receives the instances' handles.  They belong to the plan: query them as
 *   any handle, but do not pass them to spq_free (it ignores them); spq_build_plan_free
 *   releases them with the plan.
 * spq_build_plan_run(plan, weights, stream): weights[i] holds instance i's m_i weights in
 * its CSR slot order and the plan's dtype (host or device memory).  They are copied and
 * checked as spq_build checks them (SPQ_EINVAL before any table changes), then the graph
 * replays on `stream` and the call returns when the tables are final (it synchronises the
 * stream).  The handles' tables then hold the new distances, bit-identical to a fresh
 * spq_build_many of the same graphs.  If the float32 tables of an SPQ_I32 plan fail the
 * exactness check, that run is redone in int32 (spq_stats reports the arithmetic of the
 * last run; a spq_query_plan made on these handles keeps the arithmetic it was made with,
 * so remake it when that changes).  Queries on the handles must not overlap a run.
 * SPQ_ETIMEOUT as spq_build; SPQ_ECUDA if the capture or a replay fails.  A plan is used by
 * one thread at a time; spq_build_plan_free synchronises the device.
 */
typedef struct spq_build_plan spq_build_plan;
spq_status spq_build_plan_create(int32_t count, const spq_graph* graphs, const spq_opts* opts, void* stream,
                                 spq_build_plan** out, spq_handle** handles);
spq_status spq_build_plan_run(spq_build_plan* plan, const void* const* weights, void* stream);
void spq_build_plan_free(spq_build_plan* plan);

/*
 * spq_query for `count` handles at once: pairs[i] (int32[q[i]][2]) against hs[i], answers
 * in dist_out[i].  All buffers host memory (synchronous; SPQ_EINVAL if any pair was out of
 * range) or all device memory (queued; spq_query_status per handle).  One scratch
 * allocation serves every instance, reused in stream order.
 */
spq_status spq_query_many(int32_t count, spq_handle* const* hs, const int32_t* const* pairs, const int64_t* q,
                          void* const* dist_out, void* stream);

/*
 * Batched query plan (CUDA graph): the launches of spq_query_many for these handles,
 * DEVICE pair/output buffers and sizes, run once eagerly on `stream` (so the call also
 * answers the batch) and captured into a CUDA graph; spq_query_plan_run replays the whole
 * batch with one graph launch on any stream, answering the pairs the buffers hold at that
 * time (write new pairs in place between replays).  The handles and buffers must outlive
 * the plan; the plan owns its sort scratch.  Out-of-range pairs are reported as by
 * spq_query on device buffers (spq_query_status per handle).  SPQ_EINVAL for host buffers
 * or misaligned ones (pairs 8-byte, outputs 4-byte aligned); SPQ_ECUDA if the capture or
 * the instantiation fails.  spq_query_plan_free synchronises the device.  A plan is used
 * by one thread at a time.
 */
typedef struct spq_query_plan spq_query_plan;
spq_status spq_query_plan_create(int32_t count, spq_handle* const* hs, const int32_t* const* pairs, const int64_t* q,
                                 void* const* dist_out, void* stream, spq_query_plan** out);
spq_status spq_query_plan_run(spq_query_plan* plan, void* stream);
void spq_query_plan_free(spq_query_plan* plan);

/*
 * Many-to-many distances: dist_out[i * nt + j] = dist(sources[i], targets[j]) (int32 for
 * SPQ_I32 graphs, SPQ_INF_I32 if unreachable; float for SPQ_F32).  Algorithm 2 split in
 * its two stages: for a source v1 in C1 and a target component C2, t(b2) = min over b1 of
 * dist_C1(v1, b1) + dist_BG(b1, b2) is computed once and reused for every target in C2
 * (|B1||B2| updates per source and target component, plus |B2| per pair).
 *   sources int32[ns], targets int32[nt]: vertex ids; duplicates allowed.
 *   dist_out: ns x nt, row-major, caller-owned; all three buffers on the device
 *     (asynchronous; out-of-range ids give -1 / NaN and a mark reported by
 *     spq_query_status) or all on the host (synchronous; ns x nt <= 2^31; SPQ_EINVAL if an
 *     id is out of range).
 * Errors: SPQ_EINVAL for NULL buffers, mixed host/device buffers, ns or nt < 0 or above
 * 2^31 - 1; SPQ_EUNSUPPORTED for handles of spq_build_many or a component with more than
 * about 3,000 boundary vertices (the reuse buffer of a CTA).
 */
spq_status spq_query_matrix(spq_handle* h, const int32_t* sources, int64_t ns, const int32_t* targets, int64_t nt,
                            void* dist_out, void* stream);

/*
 * Distances with the path witness, and their gradients (the differentiation pattern;
 * meant for SPQ_F32 graphs, also defined for SPQ_I32).  Device buffers only.
 *
 * spq_query_saved: like spq_query, and saved[i] (int32[2]) receives the local boundary
 * indices (b1, b2) of the minimising pair of Algorithm 2 (ties: the smallest (b1, b2)),
 * or (-1, -1) when the same-component distance dist_C1(v1, v2) is the answer, (-2, -2)
 * when v1 = v2, (-3, -3) when v2 is unreachable or the pair is out of range.
 *
 * spq_query_backward: adds grad_dist[i] to grad_w[e] (float[m], accumulated, not
 * cleared) for every CSR slot e on the shortest path of pair i, in the direction of
 * travel from v1 to v2.  The path is not stored: it is walked again from the tables (next
 * hop = the neighbour minimising edge weight + table distance to the target).  Where the
 * path is unique this is the derivative of sum_i grad_dist[i] * dist_i with respect to the
 * slot weights (an undirected edge's derivative is the sum over its two slots).
 * pairs and saved must be those of the forward call on the same handle.  A walk that
 * cannot reach its target (zero-length cycles) sets a mark reported by spq_query_status.
 * Handles from spq_build_many return SPQ_EUNSUPPORTED.
 */
spq_status spq_query_saved(spq_handle* h, const int32_t* pairs, int64_t q, void* dist_out, int32_t* saved,
                           void* stream);
spq_status spq_query_backward(spq_handle* h, const int32_t* pairs, int64_t q, const int32_t* saved,
                              const float* grad_dist, float* grad_w, void* stream);

/*
 * Path retrieval: the vertex sequence of each pair's shortest path, found by the same
 * walk as spq_query_backward (Section 3's decomposition of a path into an in-component
 * piece, a boundary-graph piece and an in-component piece, each recovered hop by hop from
 * the stored distance tables; nothing but the tables is kept per graph).
 *
 * pairs, saved: int32[q][2] device, those of a spq_query_saved call on the same handle.
 * verts: int32[q][max_len] device (row-major; may be NULL when max_len = 0).  Row i gets
 *   v1, ..., v2, the vertices in order of travel (v1 alone when v1 = v2).
 * lens: int32[q] device.  lens[i] = number of vertices of the path, or -1 when v2 is
 *   unreachable or the pair out of range.  A path longer than max_len is counted in full
 *   but only its first max_len vertices are stored (lens[i] > max_len tells).
 * Errors: SPQ_EINVAL for NULL or host buffers, misaligned pairs/saved (8 bytes), q or
 *   max_len < 0; SPQ_EUNSUPPORTED for handles of spq_build_many.  A walk that cannot reach
 *   its target sets the mark reported by spq_query_status (SPQ_ETIMEOUT).
 */
spq_status spq_query_paths(spq_handle* h, const int32_t* pairs, int64_t q, const int32_t* saved, int32_t max_len,
                           int32_t* verts, int32_t* lens, void* stream);

/*
 * Native continuous-batching server (the serving pattern): a scheduler thread inside the
 * library keeps up to `slots` query launches in flight, each on its own CUDA stream with
 * pinned staging and preallocated device buffers (no allocation per request).  A free
 * slot takes the oldest waiting request and every other waiting request for the same
 * graph, up to max_pairs pairs in all, and answers them with one launch; requests that
 * arrive meanwhile join the next free slot.
 *
 * spq_server_create: device, slots in [1, 64], max_pairs in [1, 2^28] (the largest
 *   fused launch; also the largest request), memory_budget in bytes for the tables of the
 *   admitted graphs (0: 90% of the free device memory).
 * spq_server_add_graph: admits a built handle under the id gid if its footprint fits the
 *   budget (SPQ_ENOMEM otherwise, SPQ_EINVAL for a used id).  The caller keeps owning h
 *   and frees it only after spq_server_remove_graph or spq_server_destroy.
 * spq_server_remove_graph: waits until no queued or running request uses gid.
 * spq_server_submit: copies the q pairs (host int32[q][2], ids checked: SPQ_EINVAL) and
 *   queues them; the distances go to out (host, q x 4 bytes: int32, or float for SPQ_F32
 *   graphs), which must stay valid until the request completes; *ticket identifies it.
 *   Thread-safe.  SPQ_ENOMEM if q > max_pairs.
 * spq_server_poll: 1 done (the ticket is then released), 0 pending, -1 unknown ticket or
 *   a failed launch.  spq_server_wait: blocks until done (SPQ_OK, releasing the ticket),
 *   SPQ_ETIMEOUT after timeout_s seconds, SPQ_ECUDA for a failed launch.
 * spq_server_stats: p50 / p99 latency (ms, submission to completion on the host) of the
 *   requests completed so far, their number and pairs; reset != 0 starts a new window.
 * spq_server_destroy: answers what is queued, stops the scheduler, frees the server's
 *   buffers (not the graphs' handles).
 */
typedef struct spq_server spq_server;
spq_status spq_server_create(int device, int32_t slots, int64_t max_pairs, size_t memory_budget, spq_server** out);
spq_status spq_server_add_graph(spq_server* s, int32_t gid, spq_handle* h);
spq_status spq_server_remove_graph(spq_server* s, int32_t gid);
spq_status spq_server_submit(spq_server* s, int32_t gid, const int32_t* pairs, int64_t q, void* out, int64_t* ticket);
int32_t spq_server_poll(spq_server* s, int64_t ticket);
spq_status spq_server_wait(spq_server* s, int64_t ticket, double timeout_s);
spq_status spq_server_stats(spq_server* s, double* p50_ms, double* p99_ms, int64_t* requests, int64_t* pairs,
                            int32_t reset);
void spq_server_destroy(spq_server* s);

/* Synchronise `stream`, return SPQ_EINVAL if any spq_query on h since the last call
 * met an out-of-range pair, or SPQ_ETIMEOUT if a gradient walk did not reach its target
 * (and clear the marks), else SPQ_OK (or SPQ_ECUDA). */
spq_status spq_query_status(spq_handle* h, void* stream);

/* Release every device table of h.  NULL-safe.  Synchronises the device.  The memory of
 * the tables returns to a library-owned memory pool per device and is kept there for the
 * next spq_build (mapping and unmapping tens of gigabytes takes tens of milliseconds);
 * spq_build counts the kept memory as free. */
void spq_free(spq_handle* h);

/* Give the memory kept by that pool back to the device (like emptying a caching
 * allocator): the freed tables and the stream-ordered scratch of every entry point
 * (build temporaries, query sort buffers), which the pool also serves and keeps.
 * Synchronises the device.  Live handles are not affected. */
void spq_release_cached_memory(void);

/* Static English text for a status code. */
const char* spq_strerror(spq_status s);

/* The CUDA error code (cudaError_t) behind the most recent SPQ_ECUDA of this thread. */
int spq_last_cuda_error(void);

/* Device bytes owned by h (tables and per-vertex/per-component arrays). */
size_t spq_footprint_bytes(const spq_handle* h);

/* Build statistics of h, for reporting.  Any pointer may be NULL.
 *   n_bg          |BG|, the number of boundary vertices
 *   comp_updates  min-plus updates issued by the component Floyd-Warshall (sum of
 *                 padded |C|^3)
 *   bg_updates    min-plus updates issued by the boundary-graph Floyd-Warshall
 *                 (|BG|^3 minus the skipped tiles' share)
 *   arith         the spq_arith actually used (SPQ_ARITH_I32 or SPQ_ARITH_F32) */
void spq_stats(const spq_handle* h, int64_t* n_bg, double* comp_updates, double* bg_updates, int32_t* arith);

/* Device time (ms, CUDA events on the build stream) of the build's stages, in order:
 *   [0] validation and boundary detection, [1] table sizing and vertex reordering,
 *   [2] component tables (init + batched Floyd-Warshall), [3] boundary-graph assembly,
 *   [4] boundary-graph Floyd-Warshall, [5] exactness check and float32 -> int32
 *   conversion (float32 arithmetic only);
 * and, when the build ran with opts.profile_kernels = 1:
 *   [6] summed device ms of the phase-3 kernel launches of the boundary-graph
 *   Floyd-Warshall, [7] their number, [8] the min-plus updates they issued (128^3 per
 *   updated tile);
 * and [9] the order used along the boundary-graph matrix: 0 components in id order,
 *   1 / 2 components in level-structure / id-range nested-dissection order, 3 / 4 the
 *   vertex-level refinements of 1 / 2;
 * [10] the spq_bg_method used (SPQ_BG_FW or SPQ_BG_ELIM); for SPQ_BG_ELIM, with
 *   opts.profile_kernels = 1: [11] summed device ms of the back-substitution kernel's
 *   launches, [12] its min-plus updates (|K(R)| x 128^2 per tile of row block R), [13]
 *   its tiles, [14] its launches.  Stage [4] covers elimination and back-substitution,
 *   and [6]-[8] then describe the elimination's phase-3 launches.
 * Writes min(count, 15) values; returns how many it wrote (0 if h is NULL).  With the
 * float32 arithmetic falling back to int32, stages 2-5 hold the int32 run's times. */
int32_t spq_build_profile(const spq_handle* h, double* ms, int32_t count);

/* Copy out the tables (device or host destination, same rules as spq_query), for
 * inspection and tests.  Layouts:
 *   comp[n], local[n]     component of each vertex and its index inside the component
 *                         (boundary vertices first, each class in ascending vertex id)
 *   csize[k], nb[k]       |C| and |B(C)|
 *   bg_off[k]             BG index of the first boundary vertex of C (its boundary
 *                         vertex with local index i has BG index bg_off[c] + i)
 * spq_get_meta copies these (any pointer may be NULL).  spq_get_apsp copies APSP(C) of
 * component c as a dense |C| x |C| int32/float matrix in local-index order.
 * spq_get_bg copies the |BG| x |BG| distance matrix of BG in BG-index order
 * (|BG|^2 elements: large graphs need a large buffer). */
spq_status spq_get_meta(const spq_handle* h, int32_t* comp, int32_t* local, int32_t* csize, int32_t* nb,
                        int32_t* bg_off, void* stream);
spq_status spq_get_apsp(const spq_handle* h, int32_t c, void* out, void* stream);
spq_status spq_get_bg(const spq_handle* h, void* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPQ_H */
