// Order of the components along the boundary-graph matrix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spq.h"

namespace spq {

// A bisection of the vertex-level nested dissection (positions in its slot order).
struct NdNode {
    int64_t begin = 0, sep_begin = 0, end = 0;
    int depth = 0, parent = -1;
    int child[2] = {-1, -1};
};

// A run of elimination rounds (block rows [lo, hi)) done in order, possibly beside other
// runs: two runs without a dependency between them touch disjoint tiles except those
// with both indices >= shared_from (the separators of common ancestors).
struct ElimTask {
    int32_t lo = 0, hi = 0;
    int32_t shared_from = 0;
    std::vector<int32_t> deps;  // runs that must finish first (earlier in the list)
};

// Layout of the boundary-graph matrix for the elimination form: the matrix order
// (slots plus alignment padding) and the runs of elimination rounds.  With npad == 0 the
// slots are packed (npad = number of slots) and there is a single run.
// Most bisection levels whose pieces become concurrent runs (up to 2^depth leaf runs,
// 2^(depth + 1) - 1 runs and as many aligned piece starts in all).
constexpr int kMaxRunDepth = 5;
struct BgLayout {
    int32_t depth = kMaxRunDepth;  // in: bisection levels to align and run side by side
    int64_t npad = 0;
    std::vector<ElimTask> tasks;
};

// Position of every boundary slot along the boundary-graph matrix.  Slots are numbered
// component by component (slot_off[c] + local index, boundary vertices first in each
// component); bgpos[slot] is the matrix row/column of that slot.  Floyd-Warshall is
// correct for any order of the intermediate vertices; the order decides how many tile
// updates are provably no-ops and skipped.  The component order is the cheapest, by a
// symbolic cost model, of: id order, level-structure nested dissection and id-range
// nested dissection of the component adjacency graph.  SPQ_ORDER_DISSECTION keeps each
// component's slots contiguous in that order; SPQ_ORDER_AUTO and
// SPQ_ORDER_VERTEX_DISSECTION refine the chosen bisections to vertex level (only the
// boundary vertices on a cut become separator vertices).  *method: 0 id order, 1 / 2
// component-level level-structure / id-range dissection, 3 / 4 their vertex-level forms.
// The positions, in two steps so that the host part can overlap other GPU work: the
// device gathers of the component adjacency and the slots' neighbouring components
// (boundary_pairs, waits for the stream), then the ordering on the host
// (boundary_order_from).  With layout != NULL and a vertex-level order, the pieces of the
// top bisections start at multiples of 128 (the tile edge; isolated padding positions
// between them) so that their elimination rounds can run side by side (layout->tasks);
// otherwise the positions are packed.
struct BoundaryPairs {
    bool want = false;  // false: the packed component order (no dissection)
    std::vector<uint32_t> hk;
    std::vector<int32_t> hs, hcmp;
};
spq_status boundary_pairs(int32_t n, int64_t m, const int64_t* d_rp, const int32_t* d_col, const int32_t* d_part,
                          const int32_t* d_local, const int32_t* d_slot_off, int32_t k, const std::vector<int32_t>& nb,
                          spq_order ord, cudaStream_t st, BoundaryPairs* out);
spq_status boundary_order_from(int32_t k, const std::vector<int32_t>& nb, BoundaryPairs& bp, spq_order ord,
                               std::vector<int32_t>* bgpos, int32_t* method, BgLayout* layout);

// The ordering itself (host): hk = component pair keys cu * k + cv (any order,
// duplicates allowed), (hs[i], hcmp[i]) = (slot, neighbouring component) pairs.
spq_status boundary_order_host(int32_t k, const std::vector<int32_t>& nb, std::vector<uint32_t> hk,
                               const std::vector<int32_t>& hs, const std::vector<int32_t>& hcmp, spq_order ord,
                               std::vector<int32_t>* bgpos, int32_t* method, BgLayout* layout = nullptr);

// One key cu * k + cv per CSR slot joining components cu != cv (appended at *count).
cudaError_t launch_emit_comp_pairs(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* part, int32_t k,
                                   uint32_t* keys, uint32_t* count, cudaStream_t st);
// One (slot of u, component of v) pair per CSR slot u -> v joining two components.
cudaError_t launch_emit_slot_pairs(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* part,
                                   const int32_t* local, const int32_t* slot_off, int32_t* slots, int32_t* comps,
                                   uint32_t* count, cudaStream_t st);

// Host-only nested dissection of a graph given as adjacency lists (exposed for tests).
void nested_dissection(int32_t k, const std::vector<int64_t>& adj_ptr, const std::vector<int32_t>& adj,
                       const std::vector<int32_t>& weight, std::vector<int32_t>* order);

// Copy a rows x cols block (row stride ld, elements of 4 bytes) to dense `out` (host or
// device), converting float32 exact integers to int32 (+inf -> SPQ_INF_I32) if to_i32.
// With pos != NULL (device, rows == cols entries) element (i, j) is taken from
// src[pos[i]][pos[j]] instead.
cudaError_t copy_table_out(bool to_i32, const void* src, int64_t rows, int64_t cols, int64_t ld, const int32_t* pos,
                           void* out, cudaStream_t st);

}  // namespace spq
