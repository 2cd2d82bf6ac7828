// Gradients of query distances with respect to edge weights (float32 graphs).
//
// Forward (spq_query_saved): Algorithm 2 as in query.cu, one warp per pair, keeping the
// minimising boundary pair (b1*, b2*) (local boundary indices; ties broken towards the
// smallest (b1, b2) so the choice does not depend on the launch), or a marker: -1 the
// same-component distance dist_C1(v1, v2) won, -2 v1 = v2, -3 no path.
//
// Backward (spq_query_backward): the distance is the length of a shortest path, so its
// derivative with respect to the weight of a CSR slot is the number of times the path
// uses that slot (where the path is unique).  Each pair's path is walked again without
// having been stored: inside a component, from x towards target t, the next slot is the
// one minimising w(x, u) + dist_C(u, t) over the slots x -> u staying in the component
// (the APSP(C) tables hold dist_C); across the boundary graph, from boundary vertex b
// towards b2*, the next move minimises either dist_C(b, y) + dist_BG(y, b2*) over the
// other boundary vertices y of b's component (a clique edge, expanded into its path
// inside the component) or w(b, u) + dist_BG(u, b2*) over the slots b -> u into other
// components.  Each slot on the path receives the pair's upstream gradient (atomicAdd).
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "handle.h"

namespace spq {
namespace {

constexpr int GTH = 256;
constexpr int kNoPath = -3, kSame = -2, kDirect = -1;

template <typename T>
__device__ __forceinline__ bool less_lex(T a, int64_t ai, T b, int64_t bi) {
    return a < b || (a == b && ai < bi);
}

// Warp-wide lexicographic argmin of (value, index).
template <typename T>
__device__ __forceinline__ void warp_argmin(T& v, int64_t& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (less_lex(v2, i2, v, i)) {
            v = v2;
            i = i2;
        }
    }
}

template <typename T>
struct View {
    int32_t n;
    const int32_t* comp;
    const int32_t* local;
    const MatDesc* descs;
    const int32_t* nb;
    const int32_t* bg_off;
    const int32_t* bgpos;
    const T* apsp;
    const T* D;
    int64_t N;
    const int64_t* rp;
    const int32_t* col;
    const T* w;
    const int32_t* vorder;
    const int32_t* vstart;
};

// Forward with the minimising boundary pair.  dist_out: T[q]; saved: int2[q].
template <typename T>
__global__ void __launch_bounds__(GTH) k_query_saved(const View<T> V, const int2* __restrict__ pairs, int64_t q,
                                                     T* __restrict__ dist_out, int2* __restrict__ saved,
                                                     uint32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * GTH) >> 5;
    const T inf = Inf<T>::value();
    for (int64_t qi = ((int64_t)blockIdx.x * GTH + threadIdx.x) >> 5; qi < q; qi += nw) {
        const int2 pr = pairs[qi];
        const int32_t v = pr.x, w = pr.y;
        if (v < 0 || v >= V.n || w < 0 || w >= V.n) {
            if (lane == 0) {
                dist_out[qi] = (T)-1;
                saved[qi] = make_int2(kNoPath, kNoPath);
                atomicOr(err, kErrPair);
            }
            continue;
        }
        if (v == w) {
            if (lane == 0) {
                dist_out[qi] = T(0);
                saved[qi] = make_int2(kSame, kSame);
            }
            continue;
        }
        const int32_t c1 = V.comp[v], c2 = V.comp[w];
        const MatDesc d1 = V.descs[c1], d2 = V.descs[c2];
        const T* A1 = V.apsp + d1.off + (int64_t)V.local[v] * d1.n;
        const T* A2 = V.apsp + d2.off + (int64_t)V.local[w] * d2.n;
        const int32_t nb1 = V.nb[c1], nb2 = V.nb[c2];
        const int32_t* pos1 = V.bgpos + V.bg_off[c1];
        const int32_t* pos2 = V.bgpos + V.bg_off[c2];
        // lane-owned columns j; per column the best row i (smallest on ties)
        T best = inf;
        int64_t bidx = INT64_MAX;  // (i << 32) + j
        for (int32_t j = lane; j < nb2; j += 32) {
            const T cj = A2[j];
            const int64_t colp = pos2[j];
            T t = inf;
            int32_t ti = 0;
            for (int32_t i = 0; i < nb1; ++i) {
                const T cand = A1[i] + V.D[(int64_t)pos1[i] * V.N + colp];
                if (cand < t) {
                    t = cand;
                    ti = i;
                }
            }
            const T tot = t + cj;
            const int64_t idx = ((int64_t)ti << 32) + j;
            if (less_lex(tot, idx, best, bidx)) {
                best = tot;
                bidx = idx;
            }
        }
        warp_argmin(best, bidx);
        if (lane == 0) {
            int2 sv = best < inf ? make_int2((int32_t)(bidx >> 32), (int32_t)(bidx & 0xffffffff))
                                 : make_int2(kNoPath, kNoPath);
            if (c1 == c2) {
                const T direct = A1[V.local[w]];
                if (direct <= best && direct < inf) {
                    best = direct;
                    sv = make_int2(kDirect, kDirect);
                }
            }
            dist_out[qi] = best;
            saved[qi] = sv;
        }
    }
}

// Walk inside component c from vertex x to the vertex of local index tl, adding g to
// every slot taken.  All lanes of the warp take part; returns false if the walk did not
// reach its target within `limit` steps.
// Visitors of the slots a walk takes (called by lane 0 only).
struct AddGrad {
    float g;
    float* grad;
    __device__ void operator()(int64_t e, int32_t /*to*/) const { atomicAdd(&grad[e], g); }
};
struct RecordPath {
    int32_t* verts;  // this pair's row of max_len vertices
    int32_t max_len;
    int32_t* len;    // vertices written so far (may exceed max_len: the path did not fit)
    __device__ void operator()(int64_t /*e*/, int32_t to) const {
        const int32_t i = (*len)++;
        if (i < max_len) verts[i] = to;
    }
};

template <typename T, typename Visit>
__device__ bool walk_in_component(const View<T>& V, int32_t c, int32_t x, int32_t tl, const Visit& visit,
                                  int64_t limit, int lane) {
    const MatDesc d = V.descs[c];
    const T* A = V.apsp + d.off;
    const T inf = Inf<T>::value();
    for (int64_t step = 0; V.local[x] != tl; ++step) {
        if (step >= limit) return false;
        T best = inf;
        int64_t be = INT64_MAX;
        for (int64_t e = V.rp[x] + lane; e < V.rp[x + 1]; e += 32) {
            const int32_t u = V.col[e];
            if (u == x || V.comp[u] != c) continue;
            const T cand = V.w[e] + A[(int64_t)V.local[u] * d.n + tl];
            if (less_lex(cand, e, best, be)) {
                best = cand;
                be = e;
            }
        }
        warp_argmin(best, be);
        if (be == INT64_MAX) return false;
        x = V.col[be];
        if (lane == 0) visit(be, x);
    }
    return true;
}

// Walk through the boundary graph from boundary vertex b to boundary vertex b2.
template <typename T, typename Visit>
__device__ bool walk_boundary_graph(const View<T>& V, int32_t b, int32_t b2, const Visit& visit, int64_t limit,
                                    int lane) {
    const T inf = Inf<T>::value();
    const int64_t pb2 = V.bgpos[V.bg_off[V.comp[b2]] + V.local[b2]];
    const int64_t kInter = (int64_t)1 << 40;
    for (int64_t step = 0; b != b2; ++step) {
        if (step >= limit) return false;
        const int32_t cb = V.comp[b], lb = V.local[b];
        const MatDesc d = V.descs[cb];
        const T* Ab = V.apsp + d.off + (int64_t)lb * d.n;
        const int32_t* posb = V.bgpos + V.bg_off[cb];
        T best = inf;
        int64_t bi = INT64_MAX;
        for (int32_t y = lane; y < V.nb[cb]; y += 32) {  // clique edges of b's component
            if (y == lb) continue;
            const T cand = Ab[y] + V.D[(int64_t)posb[y] * V.N + pb2];
            if (less_lex(cand, (int64_t)y, best, bi)) {
                best = cand;
                bi = y;
            }
        }
        for (int64_t e = V.rp[b] + lane; e < V.rp[b + 1]; e += 32) {  // edges into other components
            const int32_t u = V.col[e];
            const int32_t cu = V.comp[u];
            if (cu == cb) continue;
            const T cand = V.w[e] + V.D[(int64_t)V.bgpos[V.bg_off[cu] + V.local[u]] * V.N + pb2];
            if (less_lex(cand, kInter + e, best, bi)) {
                best = cand;
                bi = kInter + e;
            }
        }
        warp_argmin(best, bi);
        if (bi == INT64_MAX) return false;
        if (bi < kInter) {
            const int32_t y = (int32_t)bi;
            if (!walk_in_component(V, cb, b, y, visit, limit, lane)) return false;
            b = V.vorder[V.vstart[cb] + y];
        } else {
            const int64_t e = bi - kInter;
            b = V.col[e];
            if (lane == 0) visit(e, b);
        }
    }
    return true;
}

// The whole path of one pair: v1 -> b1* inside C1, b1* -> b2* through the boundary
// graph, b2* -> v2 inside C2 (or v1 -> v2 inside C1 when the direct distance won).
template <typename T, typename Visit>
__device__ bool walk_pair(const View<T>& V, int32_t v, int32_t w, int2 sv, const Visit& visit, int64_t limit,
                          int lane) {
    const int32_t c1 = V.comp[v], c2 = V.comp[w];
    // a witness that is not one this handle's forward call can produce fails the walk
    if (sv.x == kDirect) return c1 == c2 && walk_in_component(V, c1, v, V.local[w], visit, limit, lane);
    if (sv.x < 0 || sv.x >= V.nb[c1] || sv.y < 0 || sv.y >= V.nb[c2]) return false;
    const int32_t b1 = V.vorder[V.vstart[c1] + sv.x];
    const int32_t b2 = V.vorder[V.vstart[c2] + sv.y];
    return walk_in_component(V, c1, v, sv.x, visit, limit, lane) &&
           walk_boundary_graph(V, b1, b2, visit, limit, lane) &&
           walk_in_component(V, c2, b2, V.local[w], visit, limit, lane);
}

template <typename T>
__global__ void __launch_bounds__(GTH) k_query_backward(const View<T> V, const int2* __restrict__ pairs,
                                                        const int2* __restrict__ saved, int64_t q,
                                                        const float* __restrict__ gdist, float* __restrict__ grad,
                                                        uint32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * GTH) >> 5;
    const int64_t limit = (int64_t)V.n + 1;
    for (int64_t qi = ((int64_t)blockIdx.x * GTH + threadIdx.x) >> 5; qi < q; qi += nw) {
        const int2 pr = pairs[qi];
        const int2 sv = saved[qi];
        const float g = gdist[qi];
        if (sv.x == kSame || sv.x == kNoPath || g == 0.0f) continue;
        if (pr.x < 0 || pr.x >= V.n || pr.y < 0 || pr.y >= V.n) continue;
        const AddGrad visit{g, grad};
        if (!walk_pair(V, pr.x, pr.y, sv, visit, limit, lane) && lane == 0) atomicOr(err, kErrWalk);
    }
}

// Vertex sequence of each pair's shortest path: verts[i][0] = v1, ..., up to v2;
// lens[i] = number of vertices (-1: no path; > max_len: did not fit, truncated).
template <typename T>
__global__ void __launch_bounds__(GTH) k_query_paths(const View<T> V, const int2* __restrict__ pairs,
                                                     const int2* __restrict__ saved, int64_t q, int32_t max_len,
                                                     int32_t* __restrict__ verts, int32_t* __restrict__ lens,
                                                     uint32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * GTH) >> 5;
    const int64_t limit = (int64_t)V.n + 1;
    for (int64_t qi = ((int64_t)blockIdx.x * GTH + threadIdx.x) >> 5; qi < q; qi += nw) {
        const int2 pr = pairs[qi];
        const int2 sv = saved[qi];
        int32_t* row = verts + qi * (int64_t)max_len;
        if (sv.x == kNoPath || pr.x < 0 || pr.x >= V.n || pr.y < 0 || pr.y >= V.n) {
            if (lane == 0) lens[qi] = -1;
            continue;
        }
        int32_t len = 1;
        if (lane == 0 && max_len > 0) row[0] = pr.x;
        if (sv.x != kSame) {
            const RecordPath visit{row, max_len, &len};
            if (!walk_pair(V, pr.x, pr.y, sv, visit, limit, lane) && lane == 0) atomicOr(err, kErrWalk);
        }
        if (lane == 0) lens[qi] = len;
    }
}

int grad_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename T>
View<T> view_of(const spq_handle* h) {
    return View<T>{h->n,       h->comp,         h->local, h->descs, h->nb,    h->bg_off, h->bgpos, (const T*)h->apsp,
                   (const T*)h->D, h->N, h->csr_rp, h->csr_col, (const T*)h->csr_w, h->vorder, h->vstart};
}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace spq

extern "C" {

spq_status spq_query_saved(spq_handle* h, const int32_t* pairs, int64_t q, void* dist_out, int32_t* saved,
                           void* stream) {
    using namespace spq;
    if (!h || q < 0 || !on_handle_device(h)) return SPQ_EINVAL;
    if (q == 0) return SPQ_OK;
    if (!h->vorder || !h->csr_rp) return SPQ_EUNSUPPORTED;
    if (!on_device(pairs) || !on_device(dist_out) || !on_device(saved)) return SPQ_EINVAL;
    if (((uintptr_t)pairs & 7u) || ((uintptr_t)saved & 7u) || ((uintptr_t)dist_out & 3u)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t blocks = (q + 7) / 8;
    const int64_t cap = (int64_t)grad_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (h->f32store)
        k_query_saved<float><<<(unsigned)blocks, GTH, 0, st>>>(view_of<float>(h), (const int2*)pairs, q,
                                                                (float*)dist_out, (int2*)saved, h->err);
    else
        k_query_saved<int32_t><<<(unsigned)blocks, GTH, 0, st>>>(view_of<int32_t>(h), (const int2*)pairs, q,
                                                                  (int32_t*)dist_out, (int2*)saved, h->err);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SPQ_OK : SPQ_ECUDA;
}

spq_status spq_query_backward(spq_handle* h, const int32_t* pairs, int64_t q, const int32_t* saved,
                              const float* grad_dist, float* grad_w, void* stream) {
    using namespace spq;
    if (!h || q < 0 || !on_handle_device(h)) return SPQ_EINVAL;
    if (q == 0) return SPQ_OK;
    if (!h->vorder || !h->csr_rp) return SPQ_EUNSUPPORTED;
    if (!on_device(pairs) || !on_device(saved) || !on_device(grad_dist) || !on_device(grad_w)) return SPQ_EINVAL;
    if (((uintptr_t)pairs & 7u) || ((uintptr_t)saved & 7u)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t blocks = (q + 7) / 8;
    const int64_t cap = (int64_t)grad_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (h->f32store)
        k_query_backward<float><<<(unsigned)blocks, GTH, 0, st>>>(view_of<float>(h), (const int2*)pairs,
                                                                   (const int2*)saved, q, grad_dist, grad_w, h->err);
    else
        k_query_backward<int32_t><<<(unsigned)blocks, GTH, 0, st>>>(view_of<int32_t>(h), (const int2*)pairs,
                                                                     (const int2*)saved, q, grad_dist, grad_w,
                                                                     h->err);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SPQ_OK : SPQ_ECUDA;
}

spq_status spq_query_paths(spq_handle* h, const int32_t* pairs, int64_t q, const int32_t* saved, int32_t max_len,
                           int32_t* verts, int32_t* lens, void* stream) {
    using namespace spq;
    if (!h || q < 0 || max_len < 0 || !on_handle_device(h)) return SPQ_EINVAL;
    if (q == 0) return SPQ_OK;
    if (!h->vorder || !h->csr_rp) return SPQ_EUNSUPPORTED;
    if (!on_device(pairs) || !on_device(saved) || !on_device(lens) || (max_len > 0 && !on_device(verts)))
        return SPQ_EINVAL;
    if (((uintptr_t)pairs & 7u) || ((uintptr_t)saved & 7u)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t blocks = (q + 7) / 8;
    const int64_t cap = (int64_t)grad_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (h->f32store)
        k_query_paths<float><<<(unsigned)blocks, GTH, 0, st>>>(view_of<float>(h), (const int2*)pairs,
                                                                (const int2*)saved, q, max_len, verts, lens, h->err);
    else
        k_query_paths<int32_t><<<(unsigned)blocks, GTH, 0, st>>>(view_of<int32_t>(h), (const int2*)pairs,
                                                                  (const int2*)saved, q, max_len, verts, lens,
                                                                  h->err);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? SPQ_OK : SPQ_ECUDA;
}

}  // extern "C"
