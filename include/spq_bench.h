/*
 * spq_bench.h — measurement helper of the distance-query library (not part of the
 * query API).  The paper has no counterpart: it only reports wall times.
 */
#ifndef SPQ_BENCH_H
#define SPQ_BENCH_H

#include <stdint.h>

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

/* The grouped query's autotuner: its choices so far, per (device, size class), as
 * keys[i] = device * 256 + class and choices[i] = configuration (0: 4 pairs per warp,
 * two CTAs per SM; 1: 2 pairs per warp, three CTAs per SM).  The class is
 * 16 * (clamp(floor(log2(pairs per component pair)), -6, 9) + 6)
 *    + min(floor(log2(boundary slots per component)), 15).
 * Writes at most cap entries; returns how many there are. */
int32_t spq_query_tuning(int32_t* keys, int32_t* choices, int32_t cap);

/* Number of kernels this library has launched in this process so far (all entry
 * points, all devices; the micro-benchmark above excluded). */
unsigned long long spq_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SPQ_BENCH_H */
