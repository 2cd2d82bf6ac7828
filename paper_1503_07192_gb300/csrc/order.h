// Order of the components along the boundary-graph matrix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spq.h"

namespace spq {

// Fills *order with a permutation of the k components.  SPQ_ORDER_DISSECTION (and
// AUTO, when it applies) orders them by nested dissection of the component adjacency
// graph (two components are adjacent when an edge of G joins them), each component
// weighted by its boundary size nb[c]: the two sides of a separator come first, each
// ordered recursively, and the separator last.  Floyd-Warshall is correct for any
// order of the intermediate vertices; in this order the pivot panels of the early
// rounds stay infinite outside the current sub-region, so those tile updates are
// provably no-ops and are skipped.
spq_status component_order(int32_t n, int64_t m, const int64_t* d_rp, const int32_t* d_col, const int32_t* d_part,
                           int32_t k, const std::vector<int32_t>& nb, spq_order ord, cudaStream_t st,
                           std::vector<int32_t>* order);

// Host-only nested dissection of a graph given as adjacency lists (exposed for tests).
void nested_dissection(int32_t k, const std::vector<int64_t>& adj_ptr, const std::vector<int32_t>& adj,
                       const std::vector<int32_t>& weight, std::vector<int32_t>* order);

// Copy a rows x cols block (row stride ld, elements of 4 bytes) to dense `out` (host or
// device), converting float32 exact integers to int32 (+inf -> SPQ_INF_I32) if to_i32.
cudaError_t copy_table_out(bool to_i32, const void* src, int64_t rows, int64_t cols, int64_t ld, void* out,
                           cudaStream_t st);

}  // namespace spq
