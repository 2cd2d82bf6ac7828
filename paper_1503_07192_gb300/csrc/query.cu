// Distance queries: Algorithm 2 of the paper, one warp per query pair.
//
// For (v1, v2) with components C1, C2 (Algorithm 2, line 1):
//   t(b2)  = min over b1 in B(C1) of dist_C1(v1, b1) + dist_BG(b1, b2)   (lines 2-7)
//   dist   = min over b2 in B(C2) of t(b2) + dist_C2(b2, v2)              (lines 9-12)
//   if C1 = C2: dist = min(dist, dist_C1(v1, v2))                         (line 13)
// dist_C1(v1, b1) is row v1 of APSP(C1) restricted to its first |B(C1)| columns (the
// boundary vertices come first in the local order); dist_C2(b2, v2) is row v2 of
// APSP(C2) (the tables are symmetric); dist_BG(b1, b2) is the |B(C1)| x |B(C2)| block of
// the boundary-graph matrix at (bg_off[C1], bg_off[C2]) (the paper's Fig. 2: two
// diagonal submatrices and one off-diagonal one).  Lanes own columns b2 (coalesced
// reads of each block row), rows b1 are walked in order with dist_C1(v1, b1) broadcast
// by shuffle, and a butterfly min-reduction over the warp finishes line 10-12.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "common.cuh"

namespace spq {

namespace {

constexpr int QTH = 256;
constexpr int JPL = 8;  // columns per lane per pass: 256 columns of the block per pass

// Output modes.
enum { kOutI32 = 0, kOutI32FromF32 = 1, kOutF32 = 2 };

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

// Exact int64 recomputation for float tables whose float answer reached 2^24 (float
// sums at or above 2^24 may have rounded).  Every table entry is an exact integer.
template <typename T>
__device__ int64_t exact_query(const T* __restrict__ A1, const T* __restrict__ A2, const T* __restrict__ D, int64_t N,
                               const int32_t* pos1, const int32_t* pos2, int32_t nb1, int32_t nb2, bool same,
                               int32_t l2, int lane) {
    const int64_t big = (int64_t)1 << 40;
    int64_t best = big;
    for (int32_t j = lane; j < nb2; j += 32) {
        float cj = (float)A2[j];
        if (isinf(cj)) continue;
        for (int32_t i = 0; i < nb1; ++i) {
            float ai = (float)A1[i], dij = (float)D[(int64_t)pos1[i] * N + pos2[j]];
            if (isinf(ai) || isinf(dij)) continue;
            int64_t s = (int64_t)ai + (int64_t)dij + (int64_t)cj;
            best = s < best ? s : best;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y < best ? y : best;
    }
    if (same) {
        float s = (float)A1[l2];
        if (!isinf(s) && (int64_t)s < best) best = (int64_t)s;
    }
    return best;
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
        const int32_t v = pr.x, w = pr.y;
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
        const int32_t c1 = ctx.comp[v], c2 = ctx.comp[w];
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
        } else if (MODE == kOutF32) {
            if (lane == 0) ((float*)out)[qi] = (float)r;
        } else {
            const float rf = (float)r;
            int32_t res;
            if (isinf(rf)) {
                res = SPQ_INF_I32;
            } else if (rf < 16777216.0f) {
                res = (int32_t)rf;
            } else {
                int64_t ex = exact_query<T>(A1, A2, ctx.D, ctx.N, pos1, pos2, nb1, nb2, c1 == c2, l2, lane);
                res = ex >= SPQ_INF_I32 ? SPQ_INF_I32 : (int32_t)ex;
            }
            if (lane == 0) ((int32_t*)out)[qi] = res;
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

template <typename T>
cudaError_t launch_query(const QueryCtx<T>& ctx, const int32_t* pairs, int64_t q, void* out, bool out_f32,
                         cudaStream_t st) {
    if (q <= 0) return cudaSuccess;
    int64_t blocks = (q + (QTH / 32) - 1) / (QTH / 32);
    int64_t cap = (int64_t)query_sms() * 16;
    if (blocks > cap) blocks = cap;
    const int2* p2 = reinterpret_cast<const int2*>(pairs);
    if (sizeof(T) == 4 && !out_f32) {
        if (std::is_same<T, int32_t>::value)
            k_query<T, kOutI32><<<(unsigned)blocks, QTH, 0, st>>>(ctx, p2, q, out);
        else
            k_query<T, kOutI32FromF32><<<(unsigned)blocks, QTH, 0, st>>>(ctx, p2, q, out);
    } else {
        k_query<T, kOutF32><<<(unsigned)blocks, QTH, 0, st>>>(ctx, p2, q, out);
    }
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_query<int32_t>(const QueryCtx<int32_t>&, const int32_t*, int64_t, void*, bool,
                                           cudaStream_t);
template cudaError_t launch_query<float>(const QueryCtx<float>&, const int32_t*, int64_t, void*, bool, cudaStream_t);

}  // namespace spq
