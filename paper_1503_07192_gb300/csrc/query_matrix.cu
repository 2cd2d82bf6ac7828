// Many-to-many distances: dist(s, w) for every source s and target w (row-major ns x nt).
//
// Algorithm 2 in two stages (its first loop depends on the source and the target's
// component only): for a source v1 in C1 and a target component C2,
//   t(b2) = min over b1 in B(C1) of dist_C1(v1, b1) + dist_BG(b1, b2)          (once)
// and then for every target v2 in C2
//   dist = min over b2 of t(b2) + dist_C2(b2, v2), and dist_C1(v1, v2) if C1 = C2,
// so a (source, target component) pair costs |B1||B2| updates once plus |B2| per target
// instead of |B1||B2| per pair.  Sources and targets are sorted by component; one CTA
// takes a target component and a group of eight sources: each warp computes t for its
// source from the rows of dist_BG(B(C1), B(C2)) (read in place: the block of a source
// component is shared by its sources through L2), the eight t rows stay in shared
// memory, and every target of C2 is reduced against all of them, one target per lane, so
// a target's row of APSP(C2) is read once per eight sources.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace spq {

namespace {

constexpr int MTH = 256;           // 8 warps
constexpr int MSRC = MTH / 32;     // sources per batch: one per warp
constexpr int MCOLS = 256;         // block columns per pass (8 per lane)

template <typename T>
__device__ __forceinline__ T tmin2(T a, T b) {
    return a < b ? a : b;
}
__device__ __forceinline__ int32_t add_min(int32_t a, int32_t b, int32_t t) { return __viaddmin_s32(a, b, t); }
__device__ __forceinline__ float add_min(float a, float b, float t) { return fminf(t, a + b); }
template <typename T>
__device__ __forceinline__ T warp_min2(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = tmin2(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// key = component of the vertex (k for an id out of range: sorted last), val = position
__global__ void k_comp_keys(const int32_t* __restrict__ ids, int64_t n, int32_t nv, const int32_t* __restrict__ comp,
                            uint32_t k, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t v = ids[i];
    keys[i] = (v >= 0 && v < nv) ? (uint32_t)comp[v] : k;
    vals[i] = (uint32_t)i;
}

// flags[i] = 1 where a run of equal sorted keys starts (flags[n] = 0)
__global__ void k_run_heads(const uint32_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    flags[i] = (i < n && (i == 0 || keys[i] != keys[i - 1])) ? 1u : 0u;
}

// after the exclusive scan of flags: run r starts at start[r], has key rkey[r]; start[nrun] = n
__global__ void k_run_starts(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ scanned, int64_t n,
                             uint32_t* __restrict__ start, uint32_t* __restrict__ rkey) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i == n) {
        start[scanned[n]] = (uint32_t)n;
    } else if (i == 0 || keys[i] != keys[i - 1]) {
        start[scanned[i]] = (uint32_t)i;
        rkey[scanned[i]] = keys[i];
    }
}

template <typename T, bool OUT_F32>
__device__ __forceinline__ void put(void* out, int64_t at, T v) {
    if (OUT_F32)
        ((float*)out)[at] = (float)v;
    else
        ((int32_t*)out)[at] = (int32_t)tmin2<int32_t>((int32_t)v, SPQ_INF_I32);
}

// Item (target run jr, group of MSRC consecutive sources in component order).
template <typename T, bool OUT_F32>
__global__ void __launch_bounds__(MTH)
    k_query_matrix(const QueryCtx<T> ctx, uint32_t k, const int32_t* __restrict__ sid,
                   const uint32_t* __restrict__ sval, int64_t ns, const int32_t* __restrict__ tid_,
                   const uint32_t* __restrict__ tval, const uint32_t* __restrict__ tstart,
                   const uint32_t* __restrict__ tkey, uint32_t ntrun, int64_t nt, int32_t ldt,
                   void* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tb = reinterpret_cast<T*>(smem_raw);  // t of the group's sources: [MSRC][ldt]
    __shared__ int32_t srcv[MSRC];           // the group's source vertices (-1: out of range)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T inf = Inf<T>::value();
    const int64_t ngroups = (ns + MSRC - 1) / MSRC;
    for (int64_t item = blockIdx.x; item < ngroups * ntrun; item += gridDim.x) {
        const uint32_t jr = (uint32_t)(item % ntrun);
        const int64_t sb = (item / ntrun) * MSRC;
        const int nsrc = (int)((ns - sb) < MSRC ? (ns - sb) : MSRC);
        const uint32_t c2 = tkey[jr];
        const uint32_t w0 = tstart[jr], w1 = tstart[jr + 1];
        // ---- stage 1: warp w computes t for source sb + w, reading its block rows of D
        // (lanes over the columns B(C2), through the slot positions) ----
        int32_t v1 = -1;
        if (warp < nsrc) {
            const int32_t v = sid[sval[sb + warp]];
            v1 = (v >= 0 && v < ctx.n) ? v : -1;
        }
        if (lane == 0) srcv[warp] = v1;
        if (c2 < k && v1 >= 0) {
            const uint32_t c1 = (uint32_t)ctx.comp[v1];
            const MatDesc d1 = ctx.descs[c1];
            const int32_t nb1 = ctx.nb[c1], nb2 = ctx.nb[c2];
            const int32_t* pos1 = ctx.bgpos + ctx.bg_off[c1];
            const int32_t* pos2 = ctx.bgpos + ctx.bg_off[c2];
            const T* a1 = ctx.apsp + d1.off + (int64_t)ctx.local[v1] * d1.n;
            for (int32_t jb = 0; jb < nb2; jb += MCOLS) {
                const int cols = (nb2 - jb) < MCOLS ? (nb2 - jb) : MCOLS;
                const int jmax = (cols + 31) >> 5;
                int32_t colpos[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = jj * 32 + lane;
                    colpos[jj] = j < cols ? pos2[jb + j] : 0;
                }
                T t[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) t[jj] = inf;
                for (int32_t ib = 0; ib < nb1; ib += 32) {
                    const T areg = ib + lane < nb1 ? a1[ib + lane] : inf;
                    const int32_t preg = ib + lane < nb1 ? pos1[ib + lane] : 0;
                    const int iend = (nb1 - ib) < 32 ? (nb1 - ib) : 32;
#pragma unroll 2
                    for (int ii = 0; ii < iend; ++ii) {
                        const T a = __shfl_sync(0xffffffffu, areg, ii);
                        const T* drow = ctx.D + (int64_t)__shfl_sync(0xffffffffu, preg, ii) * ctx.N;
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj)
                            if (jj < jmax && jj * 32 + lane < cols) t[jj] = add_min(a, drow[colpos[jj]], t[jj]);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = jj * 32 + lane;
                    if (jj < jmax && j < cols) tb[warp * ldt + jb + j] = t[jj];
                }
            }
        }
        __syncthreads();
        // ---- stage 2: one target per lane against the group's t (broadcast from shared
        // memory), walking the target's row of APSP(C2) ----
        if (c2 >= k) {  // targets out of range
            for (uint32_t b = w0 + tid; b < w1; b += MTH)
                for (int s = 0; s < nsrc; ++s) {
                    const int64_t at = (int64_t)sval[sb + s] * nt + tval[b];
                    if (OUT_F32)
                        ((float*)out)[at] = __int_as_float(0x7fc00000);
                    else
                        ((int32_t*)out)[at] = -1;
                }
            if (tid == 0) atomicOr(ctx.err, kErrPair);
        } else {
            const MatDesc d2 = ctx.descs[c2];
            const int32_t nb2 = ctx.nb[c2];
            for (uint32_t b0 = w0 + (uint32_t)warp * 32; b0 < w1; b0 += MSRC * 32) {
                const uint32_t b = b0 + lane;
                const bool tv = b < w1;
                const int32_t v2 = tv ? tid_[tval[b]] : 0;
                const int32_t l2 = tv ? ctx.local[v2] : 0;
                const T* a2 = ctx.apsp + d2.off + (int64_t)l2 * d2.n;
                T acc[MSRC];
#pragma unroll
                for (int s = 0; s < MSRC; ++s) acc[s] = inf;
#pragma unroll 4
                for (int32_t c = 0; c < nb2; ++c) {
                    const T x = tv ? a2[c] : inf;
#pragma unroll
                    for (int s = 0; s < MSRC; ++s)
                        if (s < nsrc) acc[s] = add_min(x, tb[s * ldt + c], acc[s]);
                }
                if (tv) {
#pragma unroll
                    for (int s = 0; s < MSRC; ++s) {
                        if (s >= nsrc) break;
                        const int64_t at = (int64_t)sval[sb + s] * nt + tval[b];
                        const int32_t v1s = srcv[s];
                        if (v1s < 0) {
                            if (OUT_F32)
                                ((float*)out)[at] = __int_as_float(0x7fc00000);
                            else
                                ((int32_t*)out)[at] = -1;
                            continue;
                        }
                        T y = acc[s];
                        const uint32_t c1s = (uint32_t)ctx.comp[v1s];
                        if (c1s == c2) {
                            const MatDesc d1s = ctx.descs[c1s];
                            y = tmin2(y, ctx.apsp[d1s.off + (int64_t)ctx.local[v1s] * d1s.n + l2]);
                        }
                        if (v1s == v2) y = T(0);
                        put<T, OUT_F32>(out, at, y);
                    }
                }
            }
            if (tid == 0)
                for (int s = 0; s < nsrc; ++s)
                    if (srcv[s] < 0) atomicOr(ctx.err, kErrPair);
        }
        __syncthreads();  // tb and srcv are rewritten by the next item
    }
}

int g_msms = 0;
int msms() {
    if (g_msms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_msms, cudaDevAttrMultiProcessorCount, dev);
        if (g_msms <= 0) g_msms = 1;
    }
    return g_msms;
}

// Sort ids by component and find the runs; returns the run count (host).
cudaError_t runs_by_component(const int32_t* ids, int64_t n, int32_t nv, const int32_t* comp, uint32_t k,
                              uint32_t* buf, uint32_t** vals, uint32_t** start, uint32_t** rkey, uint32_t* nrun,
                              cudaStream_t st) {
    uint32_t* k0 = buf;
    uint32_t* v0 = k0 + n;
    uint32_t* k1 = v0 + n;
    uint32_t* v1 = k1 + n;
    uint32_t* fl = v1 + n;  // n + 1
    uint32_t* sta = fl + n + 1;
    uint32_t* rk = sta + n + 1;
    uint32_t* hist = rk + n + 1;
    const unsigned g = (unsigned)((n + 256) / 256);
    k_comp_keys<<<g, 256, 0, st>>>(ids, n, nv, comp, k, k0, v0);
    count_launches(1);
    int bits = 0;
    while (bits < 32 && ((uint64_t)k >> bits)) ++bits;
    bool in_k1 = false;
    cudaError_t e = radix_sort_pairs(k0, v0, k1, v1, hist, n, bits, &in_k1, st);
    if (e != cudaSuccess) return e;
    const uint32_t* ks = in_k1 ? k1 : k0;
    *vals = in_k1 ? v1 : v0;
    k_run_heads<<<g, 256, 0, st>>>(ks, n, fl);
    if ((e = launch_scan_excl(fl, n + 1, st)) != cudaSuccess) return e;
    k_run_starts<<<g, 256, 0, st>>>(ks, fl, n, sta, rk);
    count_launches(3);
    *start = sta;
    *rkey = rk;
    if ((e = cudaMemcpyAsync(nrun, fl + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

int64_t runs_words(int64_t n) { return 4 * n + 3 * (n + 1) + radix_hist_words(n); }

}  // namespace
}  // namespace spq

extern "C" spq_status spq_query_matrix(spq_handle* h, const int32_t* sources, int64_t ns, const int32_t* targets,
                                       int64_t nt, void* dist_out, void* stream) {
    using namespace spq;
    if (!h || ns < 0 || nt < 0 || !on_handle_device(h)) return SPQ_EINVAL;
    if (ns == 0 || nt == 0) return SPQ_OK;
    if (!sources || !targets || !dist_out) return SPQ_EINVAL;
    if (ns > INT32_MAX || nt > INT32_MAX) return SPQ_EINVAL;
    if (h->arena) return SPQ_EUNSUPPORTED;
    cudaPointerAttributes a;
    auto on_dev = [&](const void* p) {
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    };
    const bool ds = on_dev(sources), dt = on_dev(targets), dd = on_dev(dist_out);
    if (ds != dt || ds != dd) return SPQ_EINVAL;
    if (!ds && (ns * nt > ((int64_t)1 << 31))) return SPQ_EINVAL;  // host output: bounded
    cudaStream_t st = (cudaStream_t)stream;
    QueryCtx<int32_t> ci;
    QueryCtx<float> cf;
    bool f32store = false, out_f32 = false;
    int32_t k = 0;
    handle_query_view(h, &ci, &cf, &f32store, &out_f32, &k);
    int32_t nbmax = 0;
    for (int32_t c = 0; c < k; ++c) nbmax = std::max(nbmax, h->h_nb[c]);
    const int32_t ldt = ((nbmax > 0 ? nbmax : 1) + 31) & ~31;
    const size_t smem = (size_t)(MSRC * ldt) * 4;
    if (smem > 200 * 1024) return SPQ_EUNSUPPORTED;  // a component with more than ~6,000 boundary vertices
    std::vector<void*> tmp;
    auto alloc = [&](void** p, size_t bytes) {
        cudaError_t e = scratch_alloc(p, bytes ? bytes : 4, st);
        if (e == cudaSuccess) tmp.push_back(*p);
        return e;
    };
    auto finish = [&](spq_status s) {
        for (void* p : tmp) cudaFreeAsync(p, st);
        return s;
    };
    auto fail = [&](cudaError_t err) {
        note_cuda_error(err);
        return finish(SPQ_ECUDA);
    };
    const int32_t *d_s = sources, *d_t = targets;
    void* d_out = dist_out;
    cudaError_t e = cudaSuccess;
    if (!ds) {
        void *p1, *p2, *p3;
        if ((e = alloc(&p1, (size_t)ns * 4)) != cudaSuccess || (e = alloc(&p2, (size_t)nt * 4)) != cudaSuccess ||
            (e = alloc(&p3, (size_t)(ns * nt) * 4)) != cudaSuccess)
            return fail(e);
        cudaMemcpyAsync(p1, sources, (size_t)ns * 4, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(p2, targets, (size_t)nt * 4, cudaMemcpyHostToDevice, st);
        d_s = (const int32_t*)p1;
        d_t = (const int32_t*)p2;
        d_out = p3;
    }
    void *bs, *bt;
    if ((e = alloc(&bs, (size_t)runs_words(ns) * 4)) != cudaSuccess ||
        (e = alloc(&bt, (size_t)runs_words(nt) * 4)) != cudaSuccess)
        return fail(e);
    uint32_t *sval, *sstart, *skey, *tval, *tstart, *tkey, nsrun = 0, ntrun = 0;
    if ((e = runs_by_component(d_s, ns, h->n, h->comp, (uint32_t)k, (uint32_t*)bs, &sval, &sstart, &skey, &nsrun, st)) !=
            cudaSuccess ||
        (e = runs_by_component(d_t, nt, h->n, h->comp, (uint32_t)k, (uint32_t*)bt, &tval, &tstart, &tkey, &ntrun, st)) !=
            cudaSuccess)
        return fail(e);
    const int64_t items = ((ns + MSRC - 1) / MSRC) * (int64_t)ntrun;
    const unsigned grid = (unsigned)std::min<int64_t>(items, (int64_t)msms() * 16);
    (void)nsrun;
    (void)sstart;
    (void)skey;
    if (f32store) {
        auto kern = out_f32 ? k_query_matrix<float, true> : k_query_matrix<float, false>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return fail(e);
        kern<<<grid, MTH, smem, st>>>(cf, (uint32_t)k, d_s, sval, ns, d_t, tval, tstart, tkey, ntrun, nt, ldt, d_out);
    } else {
        auto kern = out_f32 ? k_query_matrix<int32_t, true> : k_query_matrix<int32_t, false>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return fail(e);
        kern<<<grid, MTH, smem, st>>>(ci, (uint32_t)k, d_s, sval, ns, d_t, tval, tstart, tkey, ntrun, nt, ldt, d_out);
    }
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    if (!ds) {
        if ((e = cudaMemcpyAsync(dist_out, d_out, (size_t)(ns * nt) * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return fail(e);
        uint32_t f = 0;
        cudaMemcpyAsync(&f, h->err, sizeof(f), cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        if (f & kErrPair) {
            cudaMemsetAsync(h->err, 0, sizeof(uint32_t), st);
            cudaStreamSynchronize(st);
            return finish(SPQ_EINVAL);
        }
    }
    return finish(SPQ_OK);
}
