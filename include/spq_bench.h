/*
 * spq_bench.h — measurement helper of the distance-query library (not part of the
 * query API).  The paper has no counterpart: it only reports wall times.
 */
#ifndef SPQ_BENCH_H
#define SPQ_BENCH_H

#include <stdint.h>

#include "spq.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Issue-rate micro-benchmark of the min-plus update c = min(c, a + b) with all operands
 * in registers, on the current device, over SMs * blocks_per_sm CTAs of 256 threads.
 *   mode 0: float32 add + two-input min          (one update per add)
 *   mode 1: float32 add + three-input min         (two updates per min)
 *   mode 2: packed float32x2 add + three-input min
 *   mode 3: int32 add + min
 *   mode 4: int32 fused add-min (__viaddmin_s32)
 *   mode 5: int32 add, add, min, min               (two updates)
 * Writes the achieved updates per second and the timed launch's milliseconds (the
 * second of two identical launches).  Returns 0 or a cudaError_t code. */
int spq_peak_minplus(int mode, int iters, int blocks_per_sm, double* updates_per_s, double* ms);

/* Host-only: the component order the build uses along the boundary-graph matrix, for
 * a component adjacency graph given as CSR (adj_ptr[k+1], adj) with weights (boundary
 * sizes).  method 0 = id order, 1 = level-structure nested dissection, 2 = id-range
 * nested dissection, 3 = the least costly of the three.  Writes the order (k ids) and
 * the three symbolic costs (Floyd-Warshall work with infinite-panel skipping, in
 * weight^3 units) when cost_out != NULL.  Returns the method used, or -1 on bad input.
 * Needs no GPU. */
int spq_component_order_host(int k, const long long* adj_ptr, const int* adj, const int* weight, int method,
                             int* order_out, double* cost_out);

/* Host-only: the vertex-level nested-dissection order of the boundary slots for one of
 * the component bisection rules (1 level structure, 2 id ranges).  Slots are numbered
 * component by component (slot_off[k+1]); snb_ptr[nslots+1] / snb list, per slot, the
 * other components its vertex has an edge into.  Writes the slots in elimination order.
 * Returns 0, or a negative value on bad input.  Needs no GPU. */
int spq_boundary_order_host(int k, const long long* adj_ptr, const int* adj, const long long* slot_off,
                            const long long* snb_ptr, const int* snb, int rule, int* slot_order_out);

/* Host-only: the same order laid out for the elimination form with `depth` levels of
 * concurrent runs (0..5), as a build does: bgpos_out[slot] = the slot's row of the
 * boundary-graph matrix, *npad_out = the matrix order before rounding (slots plus the
 * alignment padding that starts every piece and separator on a 128-row boundary), and per
 * run of rounds 5 ints in tasks_out: first and last-plus-one block row, the block row from
 * which its tiles may be shared with concurrent runs, and the indices of the (up to two)
 * runs it waits for (-1: none).  Returns the number of runs (0: no split, one run over
 * every block row; at most cap_tasks are written), or a negative value on bad input.
 * Needs no GPU. */
int spq_boundary_layout_host(int k, const long long* adj_ptr, const int* adj, const long long* slot_off,
                             const long long* snb_ptr, const int* snb, int rule, int depth, int* bgpos_out,
                             long long* npad_out, int* tasks_out, int cap_tasks);

/* The grouped query's autotuner: its choices so far, per (device, size class), as
 * keys[i] = device * 256 + class and choices[i] = configuration (0: 4 pairs per warp,
 * two CTAs per SM; 1: 2 pairs per warp, three CTAs per SM; -1: measured, not read yet).  The class is
 * 16 * (clamp(floor(log2(pairs per component pair)), -6, 9) + 6)
 *    + min(floor(log2(boundary slots per component)), 15).
 * Writes at most cap entries; returns how many there are. */
int32_t spq_query_tuning(int32_t* keys, int32_t* choices, int32_t cap);

/* The build's autotuner: how many bisection levels of the boundary graph's dissection
 * (elimination form) run as concurrent chains of rounds, per (device, size class):
 * keys[i] = device * 256 + class (class = bit length of |BG|), depths[i] = the chosen
 * depth (3, 4 or 5; -1 while the candidates are still being tried, one per build), and
 * ms[3 * i + j] = the boundary-graph stage time measured with candidate j (depth 3 + j;
 * -1 if not tried yet).  Graphs with fewer than 4,096 boundary vertices are not tuned.
 * Writes at most cap entries; returns how many there are. */
int32_t spq_build_tuning(int32_t* keys, int32_t* depths, double* ms, int32_t cap);

/* Test hook of the back-substitution's bounded dependency waits (a CTA waits on a flag that
 * another CTA of the same launch sets when it finishes a tile the first one reads; each
 * wait gives up after a bound, the launch stops and the build returns SPQ_ETIMEOUT).
 *   limit_ns  the bound of one wait in nanoseconds; 0 restores the default (2 s)
 *   withhold  nonzero: the launches compute every tile but set none of those flags, so the
 *             first tile that depends on another waits until the bound runs out
 * Applies to the launches queued after the call, process-wide.  No wait is unbounded
 * either way, and nothing faults: the launch returns and the device stays usable. */
void spq_test_backsub_wait(unsigned long long limit_ns, int32_t withhold);

/* The last launch of the staged grouped query kernel on h (h built with
 * opts.profile_kernels = 1): its device time (CUDA events on the query's stream), its
 * min-plus updates (sum over pairs of |B1| x |B2|) and the bytes it must move: each item's
 * block once (|B1| x |B2| x 4), per pair its two table rows (4 x (|B1| + |B2|), each rounded
 * up to 4) plus 16 bytes (the pair, its position, its answer).  Waits for that launch.
 * SPQ_EUNSUPPORTED if h was not built for profiling or has run no such launch. */
spq_status spq_query_profile(const spq_handle* h, double* kernel_ms, double* updates, double* bytes);

/* Bytes of the library's device memory pool on `device` (the tables and the
 * stream-ordered scratch of every entry point come from it): in use by live allocations,
 * and reserved from the device.  Returns 0, or a cudaError_t code. */
int spq_pool_usage(int device, unsigned long long* used, unsigned long long* reserved);

/* Number of kernels this library has launched in this process so far (all entry
 * points, all devices; the micro-benchmark above excluded). */
unsigned long long spq_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SPQ_BENCH_H */
