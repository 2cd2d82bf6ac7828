// Preparation of the query structure (the paper's Phase 1 after partitioning, Sec. 4):
//  - validation of the CSR graph and the partition;
//  - boundary detection (Sec. 2: a vertex with a neighbour in another component);
//  - the vertex reordering of Sec. 4 / Fig. 1: vertices grouped by component, boundary
//    vertices first inside each component (each class in ascending vertex id), done
//    with a stable LSD radix sort on the key 2 * part + (interior ? 1 : 0).
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace spq {

namespace {

// int32 weights: below SPQ_INF_I32, the sentinel of an unreachable pair (a weight at or
// above it would read as infinity, and sums of such weights could overflow)
__device__ __forceinline__ bool weight_ok(int32_t w) { return w >= 0 && w < SPQ_INF_I32; }
__device__ __forceinline__ bool weight_ok(float w) { return isfinite(w) && w >= 0.0f; }

// One thread per vertex v: range checks of its CSR row, its weights and its part, the
// boundary flag, per-component counts, and the symmetry check of each distinct
// neighbour u (smallest weight of the slots v->u equals that of u->v).  Cost is
// O(sum over v of deg(v)^2).
template <typename W>
__device__ __forceinline__ void validate_vertex(int32_t v, int32_t n, int64_t m, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const W* __restrict__ w,
                                                const int32_t* __restrict__ part, int32_t k,
                                                uint8_t* __restrict__ bflag, int32_t* __restrict__ cnt_c,
                                                int32_t* __restrict__ cnt_b, uint32_t* __restrict__ err) {
    uint32_t bits = 0;
    int64_t a = rp[v], b = rp[v + 1];
    int32_t p = part[v];
    if (p < 0 || p >= k) {
        bits |= kErrPart;
        p = -1;
    }
    bool bnd = false;
    if (a < 0 || b < a || b > m) {
        atomicOr(err, bits | kErrCsr);
        bflag[v] = 0;
        return;
    }
    for (int64_t e = a; e < b; ++e) {
        int32_t u = col[e];
        if (u < 0 || u >= n) {
            bits |= kErrCsr;
            continue;
        }
        W we = w[e];
        if (!weight_ok(we)) bits |= kErrWeight;
        if (u == v) continue;  // self-loops never shorten a path
        if (part[u] != p) bnd = true;
        // symmetry: handle each distinct neighbour once, at its first slot
        bool first = true;
        for (int64_t e2 = a; e2 < e; ++e2)
            if (col[e2] == u) {
                first = false;
                break;
            }
        if (!first) continue;
        W mvu = we;
        for (int64_t e2 = e + 1; e2 < b; ++e2)
            if (col[e2] == u && w[e2] < mvu) mvu = w[e2];
        int64_t a2 = rp[u], b2 = rp[u + 1];
        if (a2 < 0 || b2 < a2 || b2 > m) continue;  // reported by u's own thread
        bool found = false;
        W muv = mvu;
        for (int64_t e3 = a2; e3 < b2; ++e3) {
            if (col[e3] == v) {
                if (!found || w[e3] < muv) muv = w[e3];
                found = true;
            }
        }
        if (!found || !(muv == mvu)) bits |= kErrAsym;
    }
    if (bits) atomicOr(err, bits);
    bflag[v] = bnd ? 1 : 0;
    if (p >= 0) {
        atomicAdd(&cnt_c[p], 1);
        if (bnd) atomicAdd(&cnt_b[p], 1);
    }
}

template <typename W>
__global__ void k_validate(int32_t n, int64_t m, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const W* __restrict__ w, const int32_t* __restrict__ part, int32_t k,
                           uint8_t* __restrict__ bflag, int32_t* __restrict__ cnt_c, int32_t* __restrict__ cnt_b,
                           uint32_t* __restrict__ err) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) validate_vertex<W>(v, n, m, rp, col, w, part, k, bflag, cnt_c, cnt_b, err);
}

// Every vertex of several graphs in one launch: global vertex gv belongs to the graph g
// with vbase[g] <= gv < vbase[g + 1] (found by binary search), whose flags and counts
// start at its vbase and kbase and whose status word is err[g].
template <typename W>
__global__ void k_validate_many(const ValGraph* __restrict__ gs, const int64_t* __restrict__ vbase, int32_t G,
                                uint8_t* __restrict__ bflag, int32_t* __restrict__ cnt_c, int32_t* __restrict__ cnt_b,
                                uint32_t* __restrict__ err) {
    const int64_t gv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gv >= vbase[G]) return;
    int32_t lo = 0, hi = G;  // the last graph starting at or before gv
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (vbase[mid] <= gv) lo = mid; else hi = mid;
    }
    while (lo + 1 < G && vbase[lo + 1] <= gv) ++lo;  // (empty graphs share a start)
    const ValGraph g = gs[lo];
    const int32_t v = (int32_t)(gv - vbase[lo]);
    validate_vertex<W>(v, g.n, g.m, g.rp, g.col, reinterpret_cast<const W*>(g.w), g.part, g.k, bflag + vbase[lo],
                       cnt_c + g.kbase, cnt_b + g.kbase, err + lo);
}

__global__ void k_make_keys(int32_t n, const int32_t* __restrict__ part, const uint8_t* __restrict__ bflag,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    keys[v] = 2u * (uint32_t)part[v] + (bflag[v] ? 0u : 1u);
    vals[v] = (uint32_t)v;
}

__global__ void k_assign_local(int32_t n, const uint32_t* __restrict__ sorted_vals, const int32_t* __restrict__ part,
                               const int32_t* __restrict__ vstart, int32_t* __restrict__ local,
                               int32_t* __restrict__ comp) {
    int32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    int32_t v = (int32_t)sorted_vals[pos];
    int32_t c = part[v];
    local[v] = pos - vstart[c];
    comp[v] = c;
}

// ---------------- stable LSD radix sort, 8-bit digits ----------------
constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

// hist[d * ntiles + t] = number of keys of tile t whose digit is d.
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                        uint32_t* __restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = base + it * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of len words by one block of 1024 threads (contiguous chunk
// per thread, block scan of the chunk sums, then the chunks rewritten).
__global__ void __launch_bounds__(1024) k_scan_excl(uint32_t* __restrict__ a, int64_t len) {
    __shared__ uint32_t s[1024];
    int64_t chunk = (len + 1023) / 1024;
    int64_t lo = threadIdx.x * chunk;
    int64_t hi = lo + chunk < len ? lo + chunk : len;
    uint32_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += a[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - sum;  // exclusive prefix of this chunk
    for (int64_t i = lo; i < hi; ++i) {
        uint32_t x = a[i];
        a[i] = run;
        run += x;
    }
}

// The radix sort's histogram: block d turns the counts of digit d over the tiles,
// hist[d * ntiles ..), into their exclusive prefix sums in place (1,024 coalesced counts at
// a time, the carry kept in a register) and writes the digit's total to tot[d].
__global__ void __launch_bounds__(1024) k_scan_digits(uint32_t* __restrict__ hist, int64_t ntiles,
                                                      uint32_t* __restrict__ tot) {
    __shared__ uint32_t ws[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* h = hist + (int64_t)blockIdx.x * ntiles;
    uint32_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += 1024) {
        const int64_t i = base + tid;
        const uint32_t x = i < ntiles ? h[i] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            ws[lane] = w;  // inclusive over the warps
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? ws[warp - 1] : 0u) + incl - x;
        if (i < ntiles) h[i] = carry + before;
        carry += ws[31];
        __syncthreads();
    }
    if (tid == 0) tot[blockIdx.x] = carry;
}

// Stable scatter of one tile: element it*256 + tid of the tile goes after every earlier
// element of the tile with the same digit (earlier rounds, then lower warps, then lower
// lanes of the same warp).
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           int64_t n, int shift, const uint32_t* __restrict__ hist,
                                                           int64_t ntiles) {
    __shared__ uint32_t gofs[256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kRsWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the digit's start: the totals of the smaller digits (hist + 256 * ntiles, exclusive
    // scan over the 256 digits here), plus the earlier tiles' counts of the digit
    {
        const uint32_t t = hist[256 * ntiles + tid];
        uint32_t incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) run[warp] = incl;
        __syncthreads();
        uint32_t before = incl - t;
        for (int w = 0; w < warp; ++w) before += run[w];
        gofs[tid] = before + hist[(int64_t)tid * ntiles + blockIdx.x];
        __syncthreads();
    }
    run[tid] = 0;
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = base + it * kRsThreads + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = run[d];
            for (int w = 0; w < warp; ++w) off += wcnt[w][d];
            uint32_t pos = gofs[d] + off + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < kRsWarps; ++w) {
            tot += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += tot;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_validate(bool f32, int32_t n, int64_t m, const int64_t* rp, const int32_t* col, const void* w,
                            const int32_t* part, int32_t k, uint8_t* bflag, int32_t* cnt_c, int32_t* cnt_b,
                            uint32_t* err, cudaStream_t st) {
    int blocks = (n + 255) / 256;
    if (f32)
        k_validate<float><<<blocks, 256, 0, st>>>(n, m, rp, col, (const float*)w, part, k, bflag, cnt_c, cnt_b, err);
    else
        k_validate<int32_t>
            <<<blocks, 256, 0, st>>>(n, m, rp, col, (const int32_t*)w, part, k, bflag, cnt_c, cnt_b, err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_validate_many(bool f32, const ValGraph* gs, const int64_t* vbase, int32_t G, int64_t ntot,
                                 uint8_t* bflag, int32_t* cnt_c, int32_t* cnt_b, uint32_t* err, cudaStream_t st) {
    if (ntot <= 0 || G <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((ntot + 255) / 256);
    if (f32)
        k_validate_many<float><<<blocks, 256, 0, st>>>(gs, vbase, G, bflag, cnt_c, cnt_b, err);
    else
        k_validate_many<int32_t><<<blocks, 256, 0, st>>>(gs, vbase, G, bflag, cnt_c, cnt_b, err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_make_keys(int32_t n, const int32_t* part, const uint8_t* bflag, uint32_t* keys, uint32_t* vals,
                             cudaStream_t st) {
    k_make_keys<<<(n + 255) / 256, 256, 0, st>>>(n, part, bflag, keys, vals);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_assign_local(int32_t n, const uint32_t* sorted_vals, const int32_t* part, const int32_t* vstart,
                                int32_t* local, int32_t* comp, cudaStream_t st) {
    k_assign_local<<<(n + 255) / 256, 256, 0, st>>>(n, sorted_vals, part, vstart, local, comp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scan_excl(uint32_t* a, int64_t len, cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    k_scan_excl<<<1, 1024, 0, st>>>(a, len);
    return cudaGetLastError();
}

int64_t radix_hist_words(int64_t n) {
    int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    return 256 * (ntiles > 0 ? ntiles : 1) + 256;  // per digit and tile, then per digit
}

cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist, int64_t n,
                             int key_bits, bool* in_k1, cudaStream_t st) {
    *in_k1 = false;
    if (n <= 0) return cudaSuccess;
    int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    bool flip = false;
    for (int shift = 0; shift < key_bits; shift += 8) {
        const uint32_t* ki = flip ? k1 : k0;
        const uint32_t* vi = flip ? v1 : v0;
        uint32_t* ko = flip ? k0 : k1;
        uint32_t* vo = flip ? v0 : v1;
        k_rs_hist<<<(unsigned)ntiles, kRsThreads, 0, st>>>(ki, n, shift, hist, ntiles);
        k_scan_digits<<<256, 1024, 0, st>>>(hist, ntiles, hist + 256 * ntiles);
        k_rs_scatter<<<(unsigned)ntiles, kRsThreads, 0, st>>>(ki, vi, ko, vo, n, shift, hist, ntiles);
        count_launches(3);
        flip = !flip;
    }
    *in_k1 = flip;
    return cudaGetLastError();
}

}  // namespace spq
