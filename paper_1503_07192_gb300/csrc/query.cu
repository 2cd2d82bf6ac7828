// Distance queries: Algorithm 2 of the paper, one warp per query pair.
//
// For (v1, v2) with components C1, C2:
//   t(b2)  = min over b1 in B(C1) of dist_C1(v1, b1) + dist_BG(b1, b2)   (first loop)
//   dist   = min over b2 in B(C2) of t(b2) + dist_C2(b2, v2)              (second loop)
//   if C1 = C2: dist = min(dist, dist_C1(v1, v2))                         (same component)
// dist_C1(v1, b1) is row v1 of APSP(C1) restricted to its first |B(C1)| columns (the
// boundary vertices come first in the local order); dist_C2(b2, v2) is row v2 of
// APSP(C2) (the tables are symmetric); dist_BG(b1, b2) is the |B(C1)| x |B(C2)| block of
// the boundary-graph matrix at (bg_off[C1], bg_off[C2]) (the paper's Fig. 2: two
// diagonal submatrices and one off-diagonal one).  Lanes own columns b2 (coalesced
// reads of each block row), rows b1 are walked in order with dist_C1(v1, b1) broadcast
// by shuffle, and a butterfly min-reduction over the warp finishes the second loop.
#include <cuda_runtime.h>
#include <math.h>

#include <atomic>
#include <map>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace spq {

namespace {

constexpr int QTH = 256;
constexpr int JPL = 8;  // columns per lane per pass: 256 columns of the block per pass

// Output modes.
enum { kOutI32 = 0, kOutF32 = 2 };

template <typename T>
__device__ __forceinline__ T tmin(T a, T b) {
    return a < b ? a : b;
}

template <typename T>
__device__ __forceinline__ T warp_min(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = tmin(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(QTH) k_query(const QueryCtx<T> ctx, const int2* __restrict__ pairs, int64_t q,
                                               void* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * QTH + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * QTH) >> 5;
    const T inf = Inf<T>::value();
    for (int64_t qi = wg; qi < q; qi += nw) {
        const int2 pr = pairs[qi];
        int32_t v = pr.x, w = pr.y;
        if (v < 0 || v >= ctx.n || w < 0 || w >= ctx.n) {
            if (lane == 0) {
                if (MODE == kOutF32)
                    ((float*)out)[qi] = __int_as_float(0x7fc00000);
                else
                    ((int32_t*)out)[qi] = -1;
                atomicOr(ctx.err, kErrPair);
            }
            continue;
        }
        if (v == w) {
            if (lane == 0) {
                if (MODE == kOutF32)
                    ((float*)out)[qi] = 0.0f;
                else
                    ((int32_t*)out)[qi] = 0;
            }
            continue;
        }
        int32_t c1 = ctx.comp[v], c2 = ctx.comp[w];
        if (c1 > c2) {  // answered from the lower-numbered component's side, as the grouped form does,
            const int32_t tv = v, tc = c1;  // so that float sums round the same in both forms
            v = w;
            w = tv;
            c1 = c2;
            c2 = tc;
        }
        const int32_t l1 = ctx.local[v], l2 = ctx.local[w];
        const MatDesc d1 = ctx.descs[c1], d2 = ctx.descs[c2];
        const int32_t nb1 = ctx.nb[c1], nb2 = ctx.nb[c2];
        const int64_t bo1 = ctx.bg_off[c1], bo2 = ctx.bg_off[c2];
        const T* A1 = ctx.apsp + d1.off + (int64_t)l1 * d1.n;
        const T* A2 = ctx.apsp + d2.off + (int64_t)l2 * d2.n;
        // matrix positions of the boundary slots: rows of C1's, columns of C2's
        const int32_t* pos1 = ctx.bgpos + bo1;
        const int32_t* pos2 = ctx.bgpos + bo2;
        T r = inf;
        for (int32_t jb = 0; jb < nb2; jb += 32 * JPL) {
            T t[JPL], cj[JPL];
            int32_t colj[JPL];
#pragma unroll
            for (int jj = 0; jj < JPL; ++jj) {
                const int32_t j = jb + jj * 32 + lane;
                t[jj] = inf;
                cj[jj] = j < nb2 ? A2[j] : inf;
                colj[jj] = j < nb2 ? pos2[j] : 0;
            }
            for (int32_t ib = 0; ib < nb1; ib += 32) {
                const T areg = (ib + lane < nb1) ? A1[ib + lane] : inf;
                const int32_t rreg = (ib + lane < nb1) ? pos1[ib + lane] : 0;
                const int32_t iend = (nb1 - ib) < 32 ? (nb1 - ib) : 32;
#pragma unroll 2
                for (int32_t ii = 0; ii < iend; ++ii) {
                    const T ai = __shfl_sync(0xffffffffu, areg, ii);
                    const T* rowp = ctx.D + (int64_t)__shfl_sync(0xffffffffu, rreg, ii) * ctx.N;
#pragma unroll
                    for (int jj = 0; jj < JPL; ++jj) {
                        if (jb + jj * 32 + lane < nb2) t[jj] = tmin(t[jj], ai + rowp[colj[jj]]);
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < JPL; ++jj) r = tmin(r, t[jj] + cj[jj]);
        }
        r = warp_min(r);
        if (c1 == c2) r = tmin(r, A1[l2]);
        if (MODE == kOutI32) {
            if (lane == 0) ((int32_t*)out)[qi] = (int32_t)tmin<int32_t>((int32_t)r, SPQ_INF_I32);
        } else {
            if (lane == 0) ((float*)out)[qi] = (float)r;
        }
    }
}

int query_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

// ---------------- grouped form ----------------
// Queries sorted by their unordered component pair {C1, C2}: every segment of equal keys
// shares one block dist_BG(B(C1), B(C2)), which is staged into shared memory in chunks of
// rows (gathered through the slot positions) and reused by all of the segment's queries.
// A segment starts where the key changes or at a multiple of GSEGCAP positions (so no CTA
// gets an unbounded run), and it is answered by the CTA whose 64-position tile holds its
// first position, however far it extends past the tile.  dist is symmetric, so a pair is
// answered as (v, w) with comp(v) = C1 <= C2 = comp(w).
//
// Per batch the 8 warps hold QPW queries each; lanes own block columns b2 and walk the rows
// b1 with dist_C1(v1, b1) broadcast by shuffle (one fused add-min per update for int32).
constexpr int GTH = 256;  // 8 warps
constexpr int GTILE = 64;
constexpr int GSEGCAP = 1024;         // longest segment (a power of two)
// Two configurations of the grouped kernel, chosen per size class by measurement (see
// launch_query): 4 queries per warp, 96 KB of staged block per CTA, two CTAs per SM; or
// 2 queries per warp, 64 KB, three CTAs per SM (more CTAs to overlap one another's block
// gathers, fewer queries sharing each staged chunk).  Every answer is computed with the
// same operations in both.
constexpr int GCOLS = 256;            // block columns per pass (two groups of 128)

__global__ void k_query_keys(const int2* __restrict__ pairs, int64_t q, int32_t n, const int32_t* __restrict__ comp,
                             uint32_t k, uint32_t* __restrict__ keys, uint32_t* __restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    int2 p = pairs[i];
    uint32_t key = k * k;  // sentinel: invalid pair, sorted last
    if (p.x >= 0 && p.x < n && p.y >= 0 && p.y < n) {
        uint32_t a = (uint32_t)comp[p.x], b = (uint32_t)comp[p.y];
        key = a <= b ? a * k + b : b * k + a;
    }
    keys[i] = key;
    idx[i] = (uint32_t)i;
}

// t = min(t, a + b): one fused add-min for int32, add then min for float
__device__ __forceinline__ int32_t addmin(int32_t a, int32_t b, int32_t t) { return __viaddmin_s32(a, b, t); }
__device__ __forceinline__ float addmin(float a, float b, float t) { return fminf(t, a + b); }

__device__ __forceinline__ int32_t round_up4(int32_t x) { return (x + 3) & ~3; }

__device__ __forceinline__ bool seg_head(const uint32_t* __restrict__ keys, int64_t p) {
    return p == 0 || keys[p] != keys[p - 1] || (p & (GSEGCAP - 1)) == 0;
}

// One pass over up to NG x 128 block columns [jb, jb + cols) for a warp's QPW queries:
// r[u] = min(r[u], min over b1, b2 of dist_C1(v1, b1) + D(b1, b2) + dist_C2(b2, v2)).
// The block rows are staged in chunks into S (row length NG x 128); each lane owns four
// consecutive columns per 128-column group (one 16-byte shared load per row and group)
// and dist_C1(v1, b1) is broadcast by shuffle.
template <typename T, int NG, int QPW, int SMEM>
__device__ __forceinline__ void seg_pass(const QueryCtx<T>& ctx, T* __restrict__ S, const int32_t* __restrict__ pos1,
                                         const int32_t* __restrict__ pos2, int32_t nb1, int32_t jb, int cols,
                                         const int64_t (&a1off)[QPW], const int64_t (&a2off)[QPW],
                                         const bool (&val)[QPW], bool active, T (&r)[QPW], int tid, int lane,
                                         int warp) {
    constexpr int ld = NG * 128;
    constexpr int rows_per_chunk = SMEM / ld;
    const T inf = Inf<T>::value();
    int32_t colpos[NG * 4];
#pragma unroll
    for (int jj = 0; jj < NG * 4; ++jj) {
        const int j = jj * 32 + lane;
        colpos[jj] = j < cols ? pos2[jb + j] : -1;
    }
    T t[QPW][NG][4];
#pragma unroll
    for (int u = 0; u < QPW; ++u)
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int e = 0; e < 4; ++e) t[u][g][e] = inf;
    for (int32_t rc = 0; rc < nb1; rc += rows_per_chunk) {
        const int rows = (nb1 - rc) < rows_per_chunk ? (nb1 - rc) : rows_per_chunk;
        __syncthreads();
        // stage the chunk: SR rows x (NG x 4) column groups of independent loads per lane
        constexpr int SR = 8 / NG;
        for (int i0 = warp; i0 < rows; i0 += 8 * SR) {
            int64_t rb[SR];
#pragma unroll
            for (int rr = 0; rr < SR; ++rr) {
                const int ii = i0 + 8 * rr;
                rb[rr] = ii < rows ? (int64_t)pos1[rc + ii] * ctx.N : -1;
            }
            T v[SR][NG * 4];
#pragma unroll
            for (int rr = 0; rr < SR; ++rr)
#pragma unroll
                for (int jj = 0; jj < NG * 4; ++jj)
                    v[rr][jj] = (rb[rr] >= 0 && colpos[jj] >= 0) ? ctx.D[rb[rr] + colpos[jj]] : inf;
#pragma unroll
            for (int rr = 0; rr < SR; ++rr) {
                const int ii = i0 + 8 * rr;
                if (ii < rows)
#pragma unroll
                    for (int jj = 0; jj < NG * 4; ++jj) S[ii * ld + jj * 32 + lane] = v[rr][jj];
            }
        }
        __syncthreads();
        if (!active) continue;
        for (int ib = 0; ib < rows; ib += 32) {
            T areg[QPW];
#pragma unroll
            for (int u = 0; u < QPW; ++u)
                areg[u] = (val[u] && ib + lane < rows) ? ctx.apsp[a1off[u] + rc + ib + lane] : inf;
            const int iend = (rows - ib) < 32 ? (rows - ib) : 32;
#pragma unroll 2
            for (int ii = 0; ii < iend; ++ii) {
                T ai[QPW];
#pragma unroll
                for (int u = 0; u < QPW; ++u) ai[u] = __shfl_sync(0xffffffffu, areg[u], ii);
                const T* srow = S + (ib + ii) * ld + lane * 4;
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const int4 sv = *reinterpret_cast<const int4*>(srow + g * 128);
                    const T s4[4] = {*reinterpret_cast<const T*>(&sv.x), *reinterpret_cast<const T*>(&sv.y),
                                     *reinterpret_cast<const T*>(&sv.z), *reinterpret_cast<const T*>(&sv.w)};
#pragma unroll
                    for (int u = 0; u < QPW; ++u)
#pragma unroll
                        for (int e = 0; e < 4; ++e) t[u][g][e] = addmin(ai[u], s4[e], t[u][g][e]);
                }
            }
        }
    }
    if (!active) return;
    // dist_C2(b2, v2) for this pass's columns (a lane's four consecutive columns)
#pragma unroll
    for (int u = 0; u < QPW; ++u)
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const int j0 = g * 128 + lane * 4;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = j0 + e;
                const T c = (val[u] && j < cols) ? ctx.apsp[a2off[u] + jb + j] : inf;
                r[u] = tmin(r[u], t[u][g][e] + c);
            }
        }
}

template <typename T, int MODE, int QPW, int SMEM, int MINB>
__global__ void __launch_bounds__(GTH, MINB) k_query_grouped(const QueryCtx<T> ctx, const int2* __restrict__ pairs,
                                                       const uint32_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ idx, int64_t q, uint32_t k,
                                                       int32_t min_ld, void* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);  // SMEM elements, rows of `ld` = cols rounded up to 32
    __shared__ int32_t heads[GTILE + 1];
    __shared__ uint32_t hb[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * GTILE;
    const int tn = (int)((q - t0) < GTILE ? (q - t0) : GTILE);
    const T inf = Inf<T>::value();
    bool h = false;
    if (tid < GTILE) {
        h = tid < tn && seg_head(keys, t0 + tid);
        unsigned b = __ballot_sync(0xffffffffu, h);
        if (lane == 0) hb[warp] = b;
    }
    __syncthreads();
    if (tid < GTILE && h) {
        int pos = __popc(hb[warp] & ((1u << lane) - 1u)) + (warp == 1 ? __popc(hb[0]) : 0);
        heads[pos] = tid;
    }
    const int nh = __popc(hb[0]) + __popc(hb[1]);
    if (warp == 0 && nh > 0) {
        // the last segment runs to the next head at or after the tile's end
        int64_t e = t0 + tn;
        for (;;) {
            const int64_t p = e + lane;
            const unsigned b = __ballot_sync(0xffffffffu, p >= q || seg_head(keys, p));
            if (b) {
                e += __ffs(b) - 1;
                break;
            }
            e += 32;
        }
        if (lane == 0) heads[nh] = (int32_t)(e - t0);
    }
    __syncthreads();
    for (int sg = 0; sg < nh; ++sg) {
        const int s0 = heads[sg], s1 = heads[sg + 1];
        const uint32_t key = keys[t0 + s0];
        // (with min_ld >= 0 only the blocks with a side longer than min_ld come here: the
        //  others, the empty blocks and the out-of-range pairs are answered by the staged
        //  kernel of query_blocks.cu)
        if (min_ld >= 0 &&
            (key >= k * k || ctx.nb[key / k] == 0 || ctx.nb[key % k] == 0 ||
             (ctx.nb[key / k] <= min_ld && ctx.nb[key % k] <= min_ld)))
            continue;
        if (key >= k * k) {  // out-of-range pairs
            for (int u = tid; u < s1 - s0; u += GTH) {
                const uint32_t qi = idx[t0 + s0 + u];
                if (MODE == kOutF32)
                    ((float*)out)[qi] = __int_as_float(0x7fc00000);
                else
                    ((int32_t*)out)[qi] = -1;
                atomicOr(ctx.err, kErrPair);
            }
            continue;
        }
        const int32_t c1 = (int32_t)(key / k), c2 = (int32_t)(key % k);
        const MatDesc d1 = ctx.descs[c1], d2 = ctx.descs[c2];
        const int32_t nb1 = ctx.nb[c1], nb2 = ctx.nb[c2];
        const int32_t* pos1 = ctx.bgpos + ctx.bg_off[c1];
        const int32_t* pos2 = ctx.bgpos + ctx.bg_off[c2];
        for (int bq = s0; bq < s1; bq += 8 * QPW) {
            // this warp's queries: bq + warp * QPW + u (warps past the segment's end idle
            // through the compute and only help staging)
            int64_t a1off[QPW], a2off[QPW];
            int32_t l2s[QPW];
            uint32_t qis[QPW];
            bool val[QPW], same_v[QPW];
            T r[QPW];
#pragma unroll
            for (int u = 0; u < QPW; ++u) {
                const int sp = bq + warp * QPW + u;
                val[u] = sp < s1;
                qis[u] = 0;
                a1off[u] = a2off[u] = 0;
                l2s[u] = 0;
                same_v[u] = false;
                r[u] = inf;
                if (val[u]) {
                    qis[u] = idx[t0 + sp];
                    int2 p = pairs[qis[u]];
                    if (ctx.comp[p.x] != c1) {
                        const int32_t tmp = p.x;
                        p.x = p.y;
                        p.y = tmp;
                    }
                    same_v[u] = p.x == p.y;
                    l2s[u] = ctx.local[p.y];
                    a1off[u] = d1.off + (int64_t)ctx.local[p.x] * d1.n;
                    a2off[u] = d2.off + (int64_t)l2s[u] * d2.n;
                }
            }
            const bool active = val[0];
            for (int32_t jb = 0; jb < nb2; jb += GCOLS) {
                const int cols = (nb2 - jb) < GCOLS ? (nb2 - jb) : GCOLS;
                if (cols > 128)
                    seg_pass<T, 2, QPW, SMEM>(ctx, S, pos1, pos2, nb1, jb, cols, a1off, a2off, val, active, r, tid, lane, warp);
                else
                    seg_pass<T, 1, QPW, SMEM>(ctx, S, pos1, pos2, nb1, jb, cols, a1off, a2off, val, active, r, tid, lane, warp);
            }
#pragma unroll
            for (int u = 0; u < QPW; ++u) {
                T y = warp_min(r[u]);
                if (val[u]) {
                    if (c1 == c2) y = tmin(y, ctx.apsp[a1off[u] + l2s[u]]);
                    if (same_v[u]) y = T(0);
                    if (lane == 0) {
                        if (MODE == kOutF32)
                            ((float*)out)[qis[u]] = (float)y;
                        else
                            ((int32_t*)out)[qis[u]] = (int32_t)tmin<int32_t>((int32_t)y, SPQ_INF_I32);
                    }
                }
            }
        }
    }
}

namespace {

// One configuration of the grouped kernel (QPW queries per warp, SMEMK x 1024 staged
// elements per CTA, MINB CTAs per SM).
template <typename T, int MODE, int QPW, int SMEMK, int MINB>
cudaError_t launch_grouped_one(unsigned blocks, const QueryCtx<T>& ctx, const int2* p2, const uint32_t* sk,
                               const uint32_t* sv, int64_t q, uint32_t k, int32_t min_ld, void* out, cudaStream_t st) {
    constexpr size_t smem = sizeof(T) * SMEMK * 1024;
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        const cudaError_t e = cudaFuncSetAttribute(k_query_grouped<T, MODE, QPW, SMEMK * 1024, MINB>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr.store(true);
    }
    k_query_grouped<T, MODE, QPW, SMEMK * 1024, MINB><<<blocks, GTH, smem, st>>>(ctx, p2, sk, sv, q, k, min_ld, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grouped(int cfg, bool mode_f32, unsigned blocks, const QueryCtx<T>& ctx, const int2* p2,
                           const uint32_t* sk, const uint32_t* sv, int64_t q, uint32_t k, int32_t min_ld, void* out,
                           cudaStream_t st) {
    if (cfg == 0)
        return mode_f32 ? launch_grouped_one<T, kOutF32, 4, 24, 2>(blocks, ctx, p2, sk, sv, q, k, min_ld, out, st)
                        : launch_grouped_one<T, kOutI32, 4, 24, 2>(blocks, ctx, p2, sk, sv, q, k, min_ld, out, st);
    return mode_f32 ? launch_grouped_one<T, kOutF32, 2, 16, 3>(blocks, ctx, p2, sk, sv, q, k, min_ld, out, st)
                    : launch_grouped_one<T, kOutI32, 2, 16, 3>(blocks, ctx, p2, sk, sv, q, k, min_ld, out, st);
}

// Size class of a grouped launch: log2 of the pairs per component pair (which decides how
// many queries share a staged block) and log2 of the mean boundary slots per component
// (the block's size).
int grouped_size_class(int64_t q, uint32_t k, int64_t N) {
    const double cp = (double)k * ((double)k + 1.0) / 2.0;
    const double ppp = (double)q / (cp > 0.0 ? cp : 1.0);
    const double nb = (double)N / (k > 0 ? (double)k : 1.0);
    int a = (int)floor(log2(ppp > 1e-9 ? ppp : 1e-9));
    a = (a < -6 ? -6 : (a > 9 ? 9 : a)) + 6;
    int b = (int)floor(log2(nb > 1.0 ? nb : 1.0));
    b = b > 15 ? 15 : b;
    return a * 16 + b;
}

// The autotuner's choices per (device, size class), measured on the first grouped launch
// of each class in the process.  The measurement is never waited for: the events of the
// two timed launches are kept as pending, and a later launch of the class reads them once
// they have completed (cudaEventQuery); until then the class takes the first configuration.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tune;
struct PendingTune {
    cudaEvent_t ev[3];
};
std::map<std::pair<int, int>, PendingTune> g_pending;

// -1: never measured (the caller measures now); -2: measured, result not ready yet;
// else the chosen configuration.
int tuned_config(int cls) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({dev, cls});
    if (it != g_tune.end()) return it->second;
    auto pt = g_pending.find({dev, cls});
    if (pt == g_pending.end()) return -1;
    const cudaError_t q = cudaEventQuery(pt->second.ev[2]);
    if (q == cudaErrorNotReady) return -2;
    int cfg = 0;
    float ms0 = 0.f, ms1 = 0.f;
    if (q == cudaSuccess && cudaEventElapsedTime(&ms0, pt->second.ev[0], pt->second.ev[1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms1, pt->second.ev[1], pt->second.ev[2]) == cudaSuccess)
        cfg = ms1 < ms0 ? 1 : 0;
    cudaGetLastError();
    for (cudaEvent_t x : pt->second.ev) cudaEventDestroy(x);
    g_pending.erase(pt);
    g_tune[{dev, cls}] = cfg;
    return cfg;
}

// The stored choice of a class without reading pending measurements (-1 if none).
int tuned_choice(int cls) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({dev, cls});
    return it == g_tune.end() ? -1 : it->second;
}

// Keeps the events of a measurement; false if the class is already pending or tuned
// (another thread measured it meanwhile: the caller destroys its events).
bool store_pending(int cls, const cudaEvent_t (&ev)[3]) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.count({dev, cls}) || g_pending.count({dev, cls})) return false;
    g_pending[{dev, cls}] = PendingTune{{ev[0], ev[1], ev[2]}};
    return true;
}

}  // namespace

int64_t query_scratch_words(int64_t q) { return 4 * q + radix_hist_words(q) + 4 + query_blocks_scratch_words(q); }

template <typename T>
cudaError_t launch_query(const QueryCtx<T>& ctx, const int32_t* pairs, int64_t q, void* out, bool out_f32,
                         uint32_t k, uint32_t* scratch, cudaStream_t st) {
    if (q <= 0) return cudaSuccess;
    const int2* p2 = reinterpret_cast<const int2*>(pairs);
    const bool mode_f32 = !std::is_same<T, int32_t>::value;
    if (scratch && k <= 65535u && q <= (int64_t)UINT32_MAX) {
        uint32_t* keys = scratch;
        uint32_t* vals = scratch + q;
        uint32_t* k1 = scratch + 2 * q;
        uint32_t* v1 = scratch + 3 * q;
        uint32_t* hist = scratch + 4 * q;
        k_query_keys<<<(unsigned)((q + 255) / 256), 256, 0, st>>>(p2, q, ctx.n, ctx.comp, k, keys, vals);
        count_launches(1);
        int bits = 0;
        const uint64_t mx = (uint64_t)k * k;
        while (bits < 32 && (mx >> bits)) ++bits;
        bool in_k1 = false;
        cudaError_t e = radix_sort_pairs(keys, vals, k1, v1, hist, q, bits, &in_k1, st);
        if (e != cudaSuccess) return e;
        const uint32_t* sk = in_k1 ? k1 : keys;
        const uint32_t* sv = in_k1 ? v1 : vals;
        const unsigned blocks = (unsigned)((q + GTILE - 1) / GTILE);
        int32_t min_ld = -1;  // -1: every block by the gathering kernel below
        if (ctx.staged) {
            // blocks with at most query_blocks_max_nb() rows and columns by the staged kernel;
            // larger ones (if a component has that many boundary vertices) gathered below
            if ((e = launch_query_blocks<T>(ctx, pairs, q, out, out_f32, k, sk, sv, hist + radix_hist_words(q) + 4,
                                            st)) != cudaSuccess)
                return e;
            if (ctx.max_nb <= query_blocks_max_nb()) return cudaSuccess;
            min_ld = query_blocks_max_nb();
        }
        const int cls = grouped_size_class(q, k, ctx.N);
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        // inside a graph capture: the stored choice or the first configuration, no timing
        // and no event query (the capture would be invalidated)
        int cfg = cap != cudaStreamCaptureStatusNone ? tuned_choice(cls) : tuned_config(cls);
        if (cfg == -2 || (cfg == -1 && cap != cudaStreamCaptureStatusNone)) cfg = 0;  // not read yet / no timing
        if (cfg >= 0) return launch_grouped<T>(cfg, mode_f32, blocks, ctx, p2, sk, sv, q, k, min_ld, out, st);
        // first grouped launch of this size class on this device: time both configurations
        // on these inputs (the second writes the same answers again) with events that a
        // later launch reads; nothing here waits for the device
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        for (auto& x : ev)
            if (e == cudaSuccess) e = cudaEventCreate(&x);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
        if (e == cudaSuccess) e = launch_grouped<T>(0, mode_f32, blocks, ctx, p2, sk, sv, q, k, min_ld, out, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = launch_grouped<T>(1, mode_f32, blocks, ctx, p2, sk, sv, q, k, min_ld, out, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
        if (e != cudaSuccess || !store_pending(cls, ev))
            for (auto& x : ev)
                if (x) cudaEventDestroy(x);
        return e;
    }
    int64_t blocks = (q + (QTH / 32) - 1) / (QTH / 32);
    int64_t cap = (int64_t)query_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (!mode_f32 && !out_f32)
        k_query<T, kOutI32><<<(unsigned)blocks, QTH, 0, st>>>(ctx, p2, q, out);
    else
        k_query<T, kOutF32><<<(unsigned)blocks, QTH, 0, st>>>(ctx, p2, q, out);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_query<int32_t>(const QueryCtx<int32_t>&, const int32_t*, int64_t, void*, bool, uint32_t,
                                           uint32_t*, cudaStream_t);
template cudaError_t launch_query<float>(const QueryCtx<float>&, const int32_t*, int64_t, void*, bool, uint32_t,
                                         uint32_t*, cudaStream_t);

}  // namespace spq

extern "C" int32_t spq_query_tuning(int32_t* keys, int32_t* choices, int32_t cap) {
    std::lock_guard<std::mutex> lk(spq::g_tune_mu);
    int32_t n = 0;
    for (const auto& kv : spq::g_tune) {
        if (n < cap && keys && choices) {
            keys[n] = kv.first.first * 256 + kv.first.second;
            choices[n] = kv.second;
        }
        ++n;
    }
    for (const auto& kv : spq::g_pending) {  // measured, not read yet
        if (n < cap && keys && choices) {
            keys[n] = kv.first.first * 256 + kv.first.second;
            choices[n] = -1;
        }
        ++n;
    }
    return n;
}
