// Component tables APSP(C) (Algorithm 1's per-component all-pairs distances) by the
// elimination form: the same block elimination + back-substitution as the boundary
// graph's (elim.cu), in a nested-dissection order of each component's induced subgraph.
//
// Floyd-Warshall is correct in any order of its intermediate vertices, and so is the
// elimination; the order only decides which tiles hold a finite entry.  In a dissection
// order, a block's frontier (the later vertices its vertices reach through earlier ones)
// is the separators around its piece, so the forward rounds skip most tiles and each
// back-substitution tile costs |frontier| instead of 128 steps per pivot block: on the
// 1,024-vertex components of a planar graph about a quarter of Floyd-Warshall's updates.
//
// The order: three levels of level-structure bisection inside each component, one CTA
// per component (components of up to kNdMax vertices).  Each piece runs a breadth-first
// search from a pseudo-peripheral vertex (the vertex farthest from its lowest-index
// vertex) and is cut at the level L where half of its vertices have been reached; its
// separator is the set of level-L vertices with a neighbour at level L + 1.  Every edge
// of the piece joins equal or adjacent levels, so the separator cuts levels <= L from
// levels > L (and from the vertices the search did not reach).  The pieces and
// separators are laid out in post-order (a separator after both of its halves), local
// order inside each.  The tables are built in that order into a second buffer, then
// permuted back to the component's local order (boundary vertices first, Sec. 4).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace spq {

namespace {

constexpr int kNdThreads = 1024;
constexpr uint16_t kUnset = 0xffffu;
constexpr int kNdMinSplit = 64;  // pieces smaller than this stay whole

// Post-order rank of the nodes of the depth-3 bisection tree, heap numbering (1 = the
// root, children 2x and 2x + 1): node 8 first, the root's separator last.
__constant__ int8_t c_post[16] = {-1, 14, 6, 13, 2, 5, 9, 12, 0, 1, 3, 4, 7, 8, 10, 11};

// One breadth-first search per splitting node (node[v] in [lo, hi), size >= kNdMinSplit)
// from src[node], inside the node: lev[v] = distance, kUnset if not reached.  With
// half != nullptr, also records per node the first level at which half of its vertices
// have been reached, or (fewer reached: a disconnected piece) its last level.
__device__ void nd_bfs(int32_t c, int32_t nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const int32_t* __restrict__ part, const int32_t* __restrict__ local,
                       const int32_t* __restrict__ verts, int32_t voff, const uint8_t* node, uint16_t* lev,
                       const int32_t* src,
                       const int32_t* size, int lo, int hi, int32_t* fcnt, int32_t* cum, int32_t* last,
                       int32_t* half) {
    const int tid = threadIdx.x;
    for (int32_t v = tid; v < nc; v += kNdThreads) {
        const int x = node[v];
        lev[v] = (x >= lo && x < hi && size[x] >= kNdMinSplit && src[x] == v) ? 0 : kUnset;
    }
    if (tid < 16) {
        fcnt[tid] = 0;
        cum[tid] = 0;
        last[tid] = -1;
        if (half) half[tid] = -1;
    }
    __syncthreads();
    for (int32_t cur = 0; cur < nc; ++cur) {
        int any = 0;
        for (int32_t v = tid; v < nc; v += kNdThreads) {
            if (lev[v] != (uint16_t)cur) continue;
            const int x = node[v];
            atomicAdd(&fcnt[x], 1);
            const int32_t g = verts[v] - voff;
            for (int64_t e = rp[g]; e < rp[g + 1]; ++e) {
                const int32_t u = col[e];
                if (part[u] != c) continue;
                const int32_t lu = local[u];
                if (node[lu] == x && lev[lu] == kUnset) {
                    lev[lu] = (uint16_t)(cur + 1);  // (every writer stores the same value)
                    any = 1;
                }
            }
        }
        any = __syncthreads_or(any);
        if (tid < 16) {
            cum[tid] += fcnt[tid];
            if (half && half[tid] < 0 && fcnt[tid] > 0 && 2 * cum[tid] >= size[tid]) half[tid] = cur;
            if (fcnt[tid] > 0) last[tid] = cur;
            fcnt[tid] = 0;
        }
        __syncthreads();
        if (!any) break;
    }
    if (half && tid < 16 && half[tid] < 0 && last[tid] >= 0) half[tid] = last[tid];
    __syncthreads();
}

// Dissection order of component blockIdx.x (grid-strided): ndpos[vstart[c] + v] = the
// position of local vertex v.  Components outside [min_n, max_n] keep the local order.
// The components may belong to several graphs (a batch): component c is component
// c - kbase of graphs[cgraph[c]] (cgraph null: one graph), whose vertices are numbered
// from vbase in vorder and local; vorder[vstart[c] + v] - vbase = the vertex (an index
// into that graph's rp) of local index v.
__global__ void __launch_bounds__(kNdThreads) k_comp_nd(const NdGraph* __restrict__ graphs,
                                                        const int32_t* __restrict__ cgraph,
                                                        const int32_t* __restrict__ local,
                                                        const int32_t* __restrict__ vorder,
                                                        const int32_t* __restrict__ vstart,
                                                        const int32_t* __restrict__ csize, int32_t k, int32_t min_n,
                                                        int32_t max_n, int32_t* __restrict__ ndpos) {
    __shared__ uint8_t node[kNdMax];
    __shared__ uint8_t node2[kNdMax];
    __shared__ uint16_t lev[kNdMax];
    __shared__ int32_t size[16], src[16], fcnt[16], cum[16], last[16], half[16], off[16];
    __shared__ unsigned long long far[16];
    const int tid = threadIdx.x;
    for (int32_t cg = blockIdx.x; cg < k; cg += gridDim.x) {
        const NdGraph gr = graphs[cgraph ? cgraph[cg] : 0];
        const int64_t* __restrict__ rp = gr.rp;
        const int32_t* __restrict__ col = gr.col;
        const int32_t* __restrict__ part = gr.part;
        const int32_t voff = gr.vbase;
        const int32_t c = cg - gr.kbase;  // the component's id in its graph
        const int32_t* glocal = local + gr.vbase;
        const int32_t nc = csize[cg];
        const int32_t* verts = vorder + vstart[cg];
        int32_t* out = ndpos + vstart[cg];
        if (nc < min_n || nc > max_n) {
            for (int32_t v = tid; v < nc; v += kNdThreads) out[v] = v;
            continue;
        }
        for (int32_t v = tid; v < nc; v += kNdThreads) node[v] = 1;
        for (int d = 0; d < 3; ++d) {
            const int lo = 1 << d, hi = 2 << d;
            if (tid < 16) {
                size[tid] = 0;
                src[tid] = 0x7fffffff;
                far[tid] = 0ull;
            }
            __syncthreads();
            for (int32_t v = tid; v < nc; v += kNdThreads) {
                const int x = node[v];
                if (x >= lo && x < hi) {
                    atomicAdd(&size[x], 1);
                    atomicMin(&src[x], v);
                }
            }
            __syncthreads();
            // pseudo-peripheral start: the farthest vertex from the lowest-index one
            nd_bfs(c, nc, rp, col, part, glocal, verts, voff, node, lev, src, size, lo, hi, fcnt, cum, last, nullptr);
            for (int32_t v = tid; v < nc; v += kNdThreads) {
                const int x = node[v];
                if (x >= lo && x < hi && lev[v] != kUnset)
                    atomicMax(&far[x], ((unsigned long long)lev[v] << 32) | (unsigned long long)(0xffffffffu - (uint32_t)v));
            }
            __syncthreads();
            if (tid >= lo && tid < hi && size[tid] >= kNdMinSplit) src[tid] = (int32_t)(0xffffffffu - (uint32_t)(far[tid] & 0xffffffffull));
            __syncthreads();
            nd_bfs(c, nc, rp, col, part, glocal, verts, voff, node, lev, src, size, lo, hi, fcnt, cum, last, half);
            // split: separator (level L with a neighbour at L + 1) stays in x, the rest
            // moves to 2x (levels <= L) or 2x + 1 (levels > L, or not reached)
            for (int32_t v = tid; v < nc; v += kNdThreads) {
                const int x = node[v];
                uint8_t y = (uint8_t)x;
                if (x >= lo && x < hi && size[x] >= kNdMinSplit && half[x] >= 0) {
                    const int L = half[x];
                    const int lv = lev[v] == kUnset ? 0x7fffffff : (int)lev[v];
                    if (lv > L) {
                        y = (uint8_t)(2 * x + 1);
                    } else {
                        bool sep = false;
                        if (lv == L) {
                            const int32_t g = verts[v] - voff;
                            for (int64_t e = rp[g]; e < rp[g + 1] && !sep; ++e) {
                                const int32_t u = col[e];
                                if (part[u] != c) continue;
                                const int32_t lu = glocal[u];
                                sep = node[lu] == x && lev[lu] == (uint16_t)(L + 1);
                            }
                        }
                        y = sep ? (uint8_t)x : (uint8_t)(2 * x);
                    }
                }
                node2[v] = y;
            }
            __syncthreads();
            for (int32_t v = tid; v < nc; v += kNdThreads) node[v] = node2[v];
            __syncthreads();
        }
        // positions: nodes in post-order, local order inside a node
        if (tid < 16) size[tid] = 0;
        __syncthreads();
        for (int32_t v = tid; v < nc; v += kNdThreads) atomicAdd(&size[node[v]], 1);
        __syncthreads();
        if (tid == 0) {
            int32_t byrank[15];
            for (int x = 1; x < 16; ++x) byrank[c_post[x]] = x;
            int32_t p = 0;
            for (int r = 0; r < 15; ++r) {
                off[byrank[r]] = p;
                p += size[byrank[r]];
            }
            for (int32_t v = 0; v < nc; ++v) out[v] = off[node[v]]++;
        }
        __syncthreads();
    }
}

// Every vertex's dissection position inside its component (for the edge scatter).
__global__ void k_vertex_ndpos(int32_t n, const int32_t* __restrict__ part, const int32_t* __restrict__ local,
                               const int32_t* __restrict__ vstart, const int32_t* __restrict__ ndpos,
                               int32_t* __restrict__ vpos) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) vpos[v] = ndpos[vstart[part[v]] + local[v]];
}

// A[a][b] = P[pos(a)][pos(b)] for the components taking the elimination form (sel),
// pos = the dissection position of a local vertex (padding positions map to themselves).
template <typename T>
__global__ void __launch_bounds__(256) k_unpermute(T* __restrict__ A, const T* __restrict__ P,
                                                   const MatDesc* __restrict__ descs, const int32_t* __restrict__ sel,
                                                   int32_t nsel, const int32_t* __restrict__ csize,
                                                   const int32_t* __restrict__ vstart,
                                                   const int32_t* __restrict__ ndpos) {
    // row pos[a] of P staged in shared memory with 16-byte loads, then gathered into row
    // a of A and written with 16-byte stores (rows are multiples of 4 cells and start on
    // 16-byte boundaries: every table's order and offset are multiples of 4)
    __shared__ __align__(16) T row[kNdMax];
    for (int32_t s = blockIdx.y; s < nsel; s += gridDim.y) {
        const int32_t c = sel[s];
        const MatDesc d = descs[c];
        const int32_t a = blockIdx.x;
        if (a >= d.n) continue;  // (the same for the whole block)
        const int32_t nc = csize[c];
        const int32_t* pos = ndpos + vstart[c];
        const int32_t pa = a < nc ? pos[a] : a;
        const int4* prow = reinterpret_cast<const int4*>(P + d.off + (int64_t)pa * d.n);
        for (int32_t b4 = threadIdx.x; b4 < d.n / 4; b4 += blockDim.x) reinterpret_cast<int4*>(row)[b4] = prow[b4];
        __syncthreads();
        int4* arow = reinterpret_cast<int4*>(A + d.off + (int64_t)a * d.n);
        for (int32_t b4 = threadIdx.x; b4 < d.n / 4; b4 += blockDim.x) {
            T v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int32_t bb = 4 * b4 + e;
                v[e] = row[bb < nc ? pos[bb] : bb];
            }
            arow[b4] = *reinterpret_cast<const int4*>(v);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t comp_nd_order(const NdGraph* d_graphs, const int32_t* d_cgraph, const int32_t* local,
                          const int32_t* vorder, const int32_t* d_vstart, const int32_t* d_csize, int32_t k,
                          int32_t* ndpos, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    k_comp_nd<<<std::min<int32_t>(k, 65535), kNdThreads, 0, st>>>(d_graphs, d_cgraph, local, vorder, d_vstart, d_csize,
                                                                  k, kTile + 1, kNdMax, ndpos);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t comp_nd_scatter(T* P, const MatDesc* d_descs, int32_t n, const int64_t* rp, const int32_t* col,
                            const void* w, bool f32w, const int32_t* part, const int32_t* local,
                            const int32_t* d_vstart, const int32_t* d_csize, const int32_t* ndpos, int32_t* vpos,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_vertex_ndpos<<<(n + 255) / 256, 256, 0, st>>>(n, part, local, d_vstart, ndpos, vpos);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_scatter_intra_sel<T>(f32w, n, rp, col, w, part, vpos, d_descs, d_csize, kNdMax, kTile, P, st);
}

template <typename T>
cudaError_t comp_elim_finish(T* apsp, T* P, const MatDesc* d_descs, const std::vector<MatDesc>& ed,
                             const int32_t* d_sel, const MatDesc* d_ed, const int32_t* d_csize,
                             const int32_t* d_vstart, const int32_t* ndpos, double* updates, cudaStream_t st,
                             CompElimPlan<T>* keep) {
    if (updates) *updates = 0.0;
    if (ed.empty()) {
        if (keep) keep->ready = true;
        return cudaSuccess;
    }
    const bool replay = keep && keep->ready;
    int32_t max_el = 0;
    for (const MatDesc& d : ed) max_el = std::max(max_el, d.n);
    uint32_t *scratch = replay ? keep->scratch : nullptr, *err = replay ? keep->err : nullptr;
    cudaError_t e = cudaSuccess;
    if (!replay) {
        e = scratch_alloc((void**)&scratch, (size_t)fw_many_scratch_words((int32_t)ed.size(), max_el) * 4, st);
        if (e == cudaSuccess) e = scratch_alloc((void**)&err, 4, st);
    }
    auto done = [&](cudaError_t r) {
        if (keep && !replay && r == cudaSuccess) {
            keep->scratch = scratch;
            keep->err = err;
            keep->max_el = max_el;
            keep->ready = true;
            return r;
        }
        if (replay) return r;
        if (keep) keep->bs.release(st);
        if (scratch) cudaFreeAsync(scratch, st);
        if (err) cudaFreeAsync(err, st);
        return r;
    };
    if (e != cudaSuccess) return done(e);
    if ((e = cudaMemsetAsync(err, 0, 4, st)) != cudaSuccess) return done(e);
    // forward rounds of all the tables in shared launches, then one back-substitution
    double fwd = 0.0, bs = 0.0;
    if ((e = fw_many_skip<T>(P, d_ed, (int32_t)ed.size(), max_el, scratch, &fwd, st, true, !replay)) != cudaSuccess)
        return done(e);
    std::vector<BsInput<T>> bin;
    for (const MatDesc& d : ed) bin.push_back(BsInput<T>{P + d.off, (int64_t)d.n, nullptr});
    if ((e = bg_backsub_many<T>(bin, err, nullptr, (size_t)2 << 30, &bs, nullptr, st, keep ? &keep->bs : nullptr)) !=
        cudaSuccess)
        return done(e);
    // back to the local order
    const dim3 g((unsigned)max_el, (unsigned)std::min<size_t>(ed.size(), 65535));
    k_unpermute<T><<<g, 256, 0, st>>>(apsp, P, d_descs, d_sel, (int32_t)ed.size(), d_csize, d_vstart, ndpos);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
    if (replay) {
        // (the caller reads keep->err after the replay)
        if (updates) *updates = keep->updates;
        return done(cudaSuccess);
    }
    uint32_t f = 0;
    if ((e = cudaMemcpyAsync(&f, err, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return done(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(e);
    if (f & kErrWait) return done(kWaitGaveUp);
    if (updates) *updates = fwd + bs;
    if (keep) keep->updates = fwd + bs;
    return done(cudaSuccess);
}

template <typename T>
cudaError_t comp_tables_elim(T* apsp, const MatDesc* d_descs, const std::vector<MatDesc>& h_descs,
                             const std::vector<int32_t>& h_csize, int32_t k, int32_t n, const int64_t* rp,
                             const int32_t* col, const void* w, bool f32w, const int32_t* part, const int32_t* local,
                             const int32_t* vorder, const int32_t* d_vstart, const int32_t* d_csize, double* updates,
                             cudaStream_t st) {
    if (updates) *updates = 0.0;
    // the components of at most kNdMax vertices (with more than one tile row) take the
    // elimination form; the others Floyd-Warshall (after this call, by the caller)
    std::vector<int32_t> sel;
    std::vector<MatDesc> ed;
    int64_t pelems = 0;  // the tables in dissection order share the offsets of apsp
    for (int32_t c = 0; c < k; ++c)
        if (comp_takes_elim(h_csize[c], h_descs[c].n)) {
            sel.push_back(c);
            ed.push_back(h_descs[c]);
            pelems = std::max(pelems, h_descs[c].off + (int64_t)h_descs[c].n * h_descs[c].n);
        }
    if (sel.empty()) return cudaSuccess;
    T* P = nullptr;
    int32_t *ndpos = nullptr, *vpos = nullptr, *d_sel = nullptr;
    MatDesc* d_ed = nullptr;
    NdGraph* d_graph = nullptr;
    const NdGraph hg{rp, col, part, 0, 0};
    cudaError_t e = scratch_alloc((void**)&P, (size_t)pelems * sizeof(T), st);
    if (e == cudaSuccess) e = scratch_alloc((void**)&d_graph, sizeof(NdGraph), st);
    if (e == cudaSuccess) e = scratch_alloc((void**)&ndpos, (size_t)n * 4, st);
    if (e == cudaSuccess) e = scratch_alloc((void**)&vpos, (size_t)n * 4, st);
    if (e == cudaSuccess) e = scratch_alloc((void**)&d_sel, sel.size() * 4, st);
    if (e == cudaSuccess) e = scratch_alloc((void**)&d_ed, ed.size() * sizeof(MatDesc), st);
    auto done = [&](cudaError_t r) {
        for (void* p : {(void*)P, (void*)ndpos, (void*)vpos, (void*)d_sel, (void*)d_ed, (void*)d_graph})
            if (p) cudaFreeAsync(p, st);
        return r;
    };
    if (e != cudaSuccess) return done(e);
    if ((e = cudaMemcpyAsync(d_sel, sel.data(), sel.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return done(e);
    if ((e = cudaMemcpyAsync(d_ed, ed.data(), ed.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return done(e);
    if ((e = cudaMemcpyAsync(d_graph, &hg, sizeof(NdGraph), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return done(e);
    if ((e = launch_fill_blocks<T>(P, d_ed, (int32_t)ed.size(), st)) != cudaSuccess) return done(e);
    if ((e = comp_nd_order(d_graph, nullptr, local, vorder, d_vstart, d_csize, k, ndpos, st)) != cudaSuccess)
        return done(e);
    e = comp_nd_scatter<T>(P, d_descs, n, rp, col, w, f32w, part, local, d_vstart, d_csize, ndpos, vpos, st);
    if (e != cudaSuccess) return done(e);
    return done(comp_elim_finish<T>(apsp, P, d_descs, ed, d_sel, d_ed, d_csize, d_vstart, ndpos, updates, st));
}

template cudaError_t comp_tables_elim<float>(float*, const MatDesc*, const std::vector<MatDesc>&,
                                             const std::vector<int32_t>&, int32_t, int32_t, const int64_t*,
                                             const int32_t*, const void*, bool, const int32_t*, const int32_t*,
                                             const int32_t*, const int32_t*, const int32_t*, double*, cudaStream_t);
#define SPQ_COMP_ND_INST(T)                                                                                      \
    template cudaError_t comp_nd_scatter<T>(T*, const MatDesc*, int32_t, const int64_t*, const int32_t*, const void*, \
                                            bool, const int32_t*, const int32_t*, const int32_t*, const int32_t*,      \
                                            const int32_t*, int32_t*, cudaStream_t);                                    \
    template cudaError_t comp_elim_finish<T>(T*, T*, const MatDesc*, const std::vector<MatDesc>&, const int32_t*,      \
                                             const MatDesc*, const int32_t*, const int32_t*, const int32_t*, double*,  \
                                             cudaStream_t, CompElimPlan<T>*);
SPQ_COMP_ND_INST(float)
SPQ_COMP_ND_INST(int32_t)

template cudaError_t comp_tables_elim<int32_t>(int32_t*, const MatDesc*, const std::vector<MatDesc>&,
                                               const std::vector<int32_t>&, int32_t, int32_t, const int64_t*,
                                               const int32_t*, const void*, bool, const int32_t*, const int32_t*,
                                               const int32_t*, const int32_t*, const int32_t*, double*, cudaStream_t);

}  // namespace spq
