// The query structure of one graph (definition shared by the library's host files).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "common.cuh"

namespace spq {

// One device allocation shared by the handles of a batch (spq_build_many); freed with
// the last of them.
struct Arena {
    void* base = nullptr;
    std::atomic<int> refs{0};
};

}  // namespace spq

struct spq_handle {
    int device = 0;
    int32_t n = 0, k = 0;
    spq_dtype wt = SPQ_I32;
    bool f32store = false;  // tables hold float32 values
    int32_t arith = SPQ_ARITH_I32;
    int32_t* comp = nullptr;
    int32_t* local = nullptr;
    spq::MatDesc* descs = nullptr;
    int32_t* nb = nullptr;
    int32_t* bg_off = nullptr;  // first slot of each component (component-grouped numbering)
    int32_t* bgpos = nullptr;   // matrix position of each slot
    int32_t order_method = 0;
    int32_t bg_method = SPQ_BG_FW;  // how D was computed (spq_bg_method)
    int32_t query_grouped = 1;
    int32_t* csize = nullptr;
    void* apsp = nullptr;
    void* D = nullptr;
    int32_t query_kernel = 0;  // opts.query_kernel
    int32_t max_nb = 0;        // the largest |B(C)|
    // profiling of the grouped query kernel (opts.profile_kernels)
    cudaEvent_t qev[2] = {nullptr, nullptr};
    unsigned long long* qstats = nullptr;  // device: updates, bytes of the last profiled launch
    bool qprof_ran = false;
    uint32_t* err = nullptr;
    int64_t N = 0, nbg = 0;
    int64_t apsp_elems = 0;
    size_t bytes = 0;
    double comp_updates = 0.0, bg_updates = 0.0;
    double prof_ms[7] = {0, 0, 0, 0, 0, 0, 0};
    spq::FwProfile fwprof;
    std::vector<int32_t> h_csize, h_nb, h_bgoff;
    std::vector<spq::MatDesc> h_descs;
    spq::Arena* arena = nullptr;  // set: every device pointer above lies in the arena
    bool plan_owned = false;      // belongs to a build plan (spq_free leaves it alone)
    // kept for path walks (gradients): the graph's CSR and, per component, the vertices
    // in local order (vorder[vstart[c] + i] = vertex with local index i in component c)
    int64_t m = 0;
    int64_t* csr_rp = nullptr;
    int32_t* csr_col = nullptr;
    void* csr_w = nullptr;
    int32_t* vorder = nullptr;
    int32_t* vstart = nullptr;
};
