// Blocked Floyd-Warshall in the (min, +) semiring, for the component tables APSP(C)
// (Algorithm 1, per-component APSP) and for the boundary graph (Algorithm 1, APSP of BG).
//
// The paper computes APSP(C) with the GPU algorithm of its reference [ipdps-apsp] and
// the boundary-graph rows with Dijkstra's algorithm; both are exact all-pairs distance
// computations, and here both are the three-phase blocked Floyd-Warshall of
// Venkataraman, Sahni and Mukhopadhyaya (J. Exp. Algorithmics 8, 2003).  For pivot block r:
//   phase 1: close the diagonal tile (r, r) with plain Floyd-Warshall, in shared memory;
//   phase 2: row tiles (r, J) <- D*(r, r) (x) D(r, J)   [(x) = min-plus product]
//   phase 3: tiles (I, J), I, J != r <- min(D(I, J), D(I, r) (x) D(r, J)).
// Every matrix here is symmetric (undirected graphs; a + b = b + a and min is
// order-free, so float sums keep the symmetry exactly), so phase 2 writes each row tile
// also transposed into the column tile (J, r), and phase 3 reads the column panel
// D(I, r) as the transpose of the row tile D(r, I).  Both panels of phase 3 are then
// row-major rows of the pivot block, staged into shared memory with cp.async.
//
// Arithmetic: int32 (add, min) or float32 (add, three-input min over two k steps).
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>

#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fw_tile.cuh"
#include "order.h"

namespace spq {

namespace {

// ---------------- phase 1: closure of the diagonal tile ----------------
template <typename T>
__global__ void __launch_bounds__(NTH) k_phase1(T* __restrict__ base, const MatDesc* __restrict__ descs,
                                                int32_t nmat, int32_t r, const int32_t* __restrict__ sel) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*S)[T_] = reinterpret_cast<T(*)[T_]>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int32_t mi = blockIdx.y; mi < nmat; mi += gridDim.y) {
        const MatDesc d = descs[sel ? sel[mi] : mi];
        const int64_t n = d.n;
        const int32_t R = (int32_t)((n + T_ - 1) / T_);
        if (r >= R) continue;
        T* M = base + d.off;
        const int64_t o = (int64_t)r * T_;
        for (int idx = tid; idx < T_ * T_ / 4; idx += NTH) {
            int i = idx >> 5, c4 = idx & 31;
            int64_t gr = o + i, gc = o + c4 * 4;
            int4 v = (gr < n && gc < n) ? *reinterpret_cast<const int4*>(M + gr * n + gc) : inf4<T>();
            *reinterpret_cast<int4*>(&S[i][c4 * 4]) = v;
        }
        __syncthreads();
        T acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = S[own(ty, i)][own(tx, j)];
        const int K = (int)((n - o) < T_ ? (n - o) : T_);
        int k = 0;
        if constexpr (std::is_same<T, float>::value) {
            // two pivot steps per barrier: row k + 1 after step k is formed on the fly,
            // min(D(k+1, x), D(k+1, k) + D(k, x)), and both steps fold into one
            // three-input min; the owners then publish rows k + 2 and k + 3
            for (; k + 1 < K; k += 2) {
                float a0[8], b0[8], a1[8], b1[8];
                const float4 p0 = *reinterpret_cast<const float4*>(&S[k][ty * 4]);
                const float4 p1 = *reinterpret_cast<const float4*>(&S[k][64 + ty * 4]);
                const float4 q0 = *reinterpret_cast<const float4*>(&S[k][tx * 4]);
                const float4 q1 = *reinterpret_cast<const float4*>(&S[k][64 + tx * 4]);
                const float4 u0 = *reinterpret_cast<const float4*>(&S[k + 1][ty * 4]);
                const float4 u1 = *reinterpret_cast<const float4*>(&S[k + 1][64 + ty * 4]);
                const float4 v0 = *reinterpret_cast<const float4*>(&S[k + 1][tx * 4]);
                const float4 v1 = *reinterpret_cast<const float4*>(&S[k + 1][64 + tx * 4]);
                const float skk = S[k][k + 1];
                const float pa[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
                const float qa[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                const float ua[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                const float va[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    a0[i] = pa[i];
                    b0[i] = qa[i];
                    a1[i] = fminf(ua[i], skk + pa[i]);
                    b1[i] = fminf(va[i], skk + qa[i]);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmin3(acc[i][j], a0[i] + b0[j], a1[i] + b1[j]);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int row = own(ty, i);
                    if (row == k + 2 || row == k + 3) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) S[row][own(tx, j)] = acc[i][j];
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll 1
        for (; k < K; ++k) {
            // row k of S is current: by symmetry it is also column k
            T a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                a[i] = S[k][own(ty, i)];
                b[i] = S[k][own(tx, i)];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = MP<T>::upd1(acc[i][j], a[i], b[j]);
            const int kn = k + 1;
            if (kn < K) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (own(ty, i) == kn) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) S[kn][own(tx, j)] = acc[i][j];
                    }
            }
            __syncthreads();
        }
        store_c<T>(acc, M, n, o, o, tx, ty);
        __syncthreads();
    }
}

// Phase 1 of round r of one matrix with 1,024 threads, each owning a 4 x 4 block (rows
// 4ty.., columns 4tx..): the same two pivot steps per barrier as k_phase1, with four
// times the warps to hide each step's latency, and the sums formed two at a time by
// packed f32x2 adds.  For the elimination rounds of one boundary graph, where the closure
// of the diagonal tile lies on the critical path of every round.  Every step is the
// same rounded float operation as in k_phase1, so the results are identical.
__global__ void __launch_bounds__(1024, 1) k_phase1_wide(float* __restrict__ M, int64_t n, int32_t r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float(*S)[T_] = reinterpret_cast<float(*)[T_]>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int64_t o = (int64_t)r * T_;
    for (int idx = tid; idx < T_ * T_ / 4; idx += 1024) {
        const int i = idx >> 5, c4 = idx & 31;
        const int64_t gr = o + i, gc = o + c4 * 4;
        int4 v = (gr < n && gc < n) ? *reinterpret_cast<const int4*>(M + gr * n + gc) : inf4<float>();
        *reinterpret_cast<int4*>(&S[i][c4 * 4]) = v;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(&S[4 * ty + i][4 * tx]);
        acc[i][0] = v.x;
        acc[i][1] = v.y;
        acc[i][2] = v.z;
        acc[i][3] = v.w;
    }
    const int K = (int)((n - o) < T_ ? (n - o) : T_);
    int k = 0;
    // rows k and k + 1 are current (by symmetry also columns k and k + 1); row k + 1
    // after step k is min(D(k+1, x), D(k+1, k) + D(k, x)), formed on the fly
    for (; k + 1 < K; k += 2) {
        const float4 p = *reinterpret_cast<const float4*>(&S[k][4 * ty]);
        const float4 q = *reinterpret_cast<const float4*>(&S[k][4 * tx]);
        const float4 u = *reinterpret_cast<const float4*>(&S[k + 1][4 * ty]);
        const float4 v = *reinterpret_cast<const float4*>(&S[k + 1][4 * tx]);
        const float skk = S[k][k + 1];
        const float a0[4] = {p.x, p.y, p.z, p.w};
        const float a1[4] = {fminf(u.x, skk + p.x), fminf(u.y, skk + p.y), fminf(u.z, skk + p.z),
                             fminf(u.w, skk + p.w)};
        const float2 b0l = make_float2(q.x, q.y), b0h = make_float2(q.z, q.w);
        const float2 b1l = make_float2(fminf(v.x, skk + q.x), fminf(v.y, skk + q.y));
        const float2 b1h = make_float2(fminf(v.z, skk + q.z), fminf(v.w, skk + q.w));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 x0 = make_float2(a0[i], a0[i]), x1 = make_float2(a1[i], a1[i]);
            const float2 s0l = __fadd2_rn(x0, b0l), s0h = __fadd2_rn(x0, b0h);
            const float2 s1l = __fadd2_rn(x1, b1l), s1h = __fadd2_rn(x1, b1h);
            acc[i][0] = fmin3(acc[i][0], s0l.x, s1l.x);
            acc[i][1] = fmin3(acc[i][1], s0l.y, s1l.y);
            acc[i][2] = fmin3(acc[i][2], s0h.x, s1h.x);
            acc[i][3] = fmin3(acc[i][3], s0h.y, s1h.y);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = 4 * ty + i;
            if (row == k + 2 || row == k + 3)
                *reinterpret_cast<float4*>(&S[row][4 * tx]) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
        __syncthreads();
    }
    for (; k < K; ++k) {
        const float4 p = *reinterpret_cast<const float4*>(&S[k][4 * ty]);
        const float4 q = *reinterpret_cast<const float4*>(&S[k][4 * tx]);
        const float a[4] = {p.x, p.y, p.z, p.w}, b[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fminf(acc[i][j], a[i] + b[j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * ty + i == k + 1)
                *reinterpret_cast<float4*>(&S[k + 1][4 * tx]) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = o + 4 * ty + i, gc = o + 4 * tx;
        if (gr < n && gc < n)
            *reinterpret_cast<float4*>(M + gr * n + gc) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
}

// ---------------- phase 2: pivot row tiles (and their transposes) ----------------
template <typename T>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS) k_phase2(T* __restrict__ base, const MatDesc* __restrict__ descs,
                                                   int32_t nmat, int32_t r, uint32_t* __restrict__ row_finite,
                                                   int32_t flag_stride, const int32_t* __restrict__ sel,
                                                   int32_t trail = 0, uint32_t* __restrict__ kmask = nullptr,
                                                   int32_t kstride = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int32_t mi = blockIdx.y; mi < nmat; mi += gridDim.y) {
        const MatDesc d = descs[sel ? sel[mi] : mi];
        const int64_t n = d.n;
        const int32_t R = (int32_t)((n + T_ - 1) / T_);
        // (elimination form: the row tiles right of the pivot only)
        const int32_t J = trail ? r + 1 + (int32_t)blockIdx.x : (int32_t)blockIdx.x + ((int32_t)blockIdx.x >= r ? 1 : 0);
        if (r >= R || J >= R) continue;
        T* M = base + d.off;
        const int64_t o = (int64_t)r * T_, cj = (int64_t)J * T_;
        T acc[8][8];
        load_c<T>(acc, M, n, o, cj, tx, ty);
        // An all-infinite row tile stays all-infinite (D*(r,r) (x) inf = inf), and so
        // does its transpose: nothing to compute or store.
        bool fin = false;
        const T inf = Inf<T>::value();
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) fin |= acc[i][j] < inf;
        if (!__syncthreads_or(fin)) continue;
        if (kmask) {  // (as in k_phase2_cand: chunk skipping, then the row mask for phase 3)
            __shared__ uint32_t rm[4];
            tile_row_mask<T>(acc, rm, tid, tx, ty);
            uint32_t cm = 0u;
#pragma unroll
            for (int c = 0; c < NCHUNK; ++c) cm |= rm[c] ? (1u << c) : 0u;
            minplus_panels_masked<T>(acc, M, n, o, o, cj, sm, tid, tx, ty, cm);
            tile_row_mask<T>(acc, rm, tid, tx, ty);
            if (tid < 4) kmask[(int64_t)mi * kstride + (int64_t)J * 4 + tid] = rm[tid];
        } else {
            minplus_panels<T>(acc, M, n, o, o, cj, sm, tid, tx, ty);
        }
        store_c<T>(acc, M, n, o, cj, tx, ty);
        store_c_transposed<T>(acc, M, n, o, cj, tx, ty);
        if (row_finite && tid == 0) row_finite[(int64_t)mi * flag_stride + J] = 1u;
    }
}

// Ordered list of the marked tiles J in [lo, hi) of one flag row: out[0] = count,
// out[1..] = J ascending.  Whole block; ends with a barrier.
__device__ void compact_row(const uint32_t* __restrict__ f, int32_t lo, int32_t hi, uint32_t* __restrict__ out) {
    __shared__ uint32_t cnt;
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int32_t base = lo; base < hi; base += blockDim.x) {
        const int32_t J = base + threadIdx.x;
        const bool take = J < hi && __ldcg(f + J) != 0u;
        const unsigned ballot = __ballot_sync(0xffffffffu, take);
        if (lane == 0) wsum[warp] = __popc(ballot);
        __syncthreads();
        uint32_t off = cnt;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (take) out[1 + off + __popc(ballot & ((1u << lane) - 1u))] = (uint32_t)J;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
            cnt += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = cnt;
    __syncthreads();
}

// Elimination form, after phase 2 of round r (r = -1: before round 0):
//   list = the finite row tiles J > r of round r (phase 3 updates list x list);
//   marks every pair of the list as a tile that may hold a finite entry from now on
//   (2 where it was unmarked: only the marked tiles were initialised);
//   cand = the marked tiles J > r + 1 of row r + 1 (phase 2 of the next round).
__device__ void compact_trail(uint32_t* __restrict__ rowflags, int32_t R, int32_t r, uint32_t* __restrict__ list,
                              uint32_t* __restrict__ cand, unsigned long long* __restrict__ tiles, int32_t do_list) {
    if (r >= 0 && do_list) {
        compact_row(rowflags + (int64_t)r * R, r + 1, R, list);
        const uint32_t c = list[0];
        for (uint32_t t = threadIdx.x; t < c * c; t += blockDim.x) {
            const uint32_t x = t / c, y = t % c;
            if (y > x) {
                // 2: newly marked, its cells are not initialised yet (phase 3 starts it
                // from infinity and then marks it 1)
                uint32_t* f = rowflags + (int64_t)list[1 + x] * R + list[1 + y];
                if (__ldcg(f) == 0u) *f = 2u;
            }
        }
        if (threadIdx.x == 0) {
            tiles[0] += (unsigned long long)c * (c + 1) / 2;  // phase-3 tiles of this round
            tiles[1] += (unsigned long long)c;                // phase-2 tiles computed (finite)
        }
        __syncthreads();
    }
    if (r + 1 < R) compact_row(rowflags + (int64_t)(r + 1) * R, r + 2, R, cand);
}

__global__ void k_compact_trail(uint32_t* __restrict__ rowflags, int32_t R, int32_t r, uint32_t* __restrict__ list,
                                uint32_t* __restrict__ cand, unsigned long long* __restrict__ tiles, int32_t do_list) {
    compact_trail(rowflags, R, r, list, cand, tiles, do_list);
}

// ---------------- phase 2, elimination form: candidate row tiles only ----------------
// cand[0] = count, cand[1..] = the tiles J > r of row r that may hold a finite entry (the
// assembly's and earlier rounds' marks).  A candidate that is all-infinite is unmarked
// (it stays infinite); the others are updated, with their transposes.
// With counter != NULL the last CTA to finish (counted there; the counter is left at 0)
// also does the round's compaction (compact_trail; with mark_all, after marking every
// tile J > r of row r): no separate launch on the round's critical path.
template <typename T>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS) k_phase2_cand(T* __restrict__ M, int64_t n, int32_t r,
                                                                      int32_t R, uint32_t* __restrict__ cand,
                                                                      uint32_t* __restrict__ rowflags,
                                                                      uint32_t* __restrict__ list,
                                                                      unsigned long long* __restrict__ tiles,
                                                                      uint32_t* __restrict__ counter,
                                                                      int32_t mark_all,
                                                                      uint32_t* __restrict__ kmask) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t o = (int64_t)r * T_;
    const uint32_t c = cand[0];
    const T inf = Inf<T>::value();
    for (uint32_t ci = blockIdx.x; ci < c; ci += gridDim.x) {
        const int32_t J = (int32_t)cand[1 + ci];
        const int64_t cj = (int64_t)J * T_;
        T acc[8][8];
        load_c<T>(acc, M, n, o, cj, tx, ty);
        bool fin = false;
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) fin |= acc[i][j] < inf;
        if (!__syncthreads_or(fin)) {
            if (tid == 0) rowflags[(int64_t)r * R + J] = 0u;
            continue;
        }
        if (kmask) {
            // the B panel is this tile's own rows: skip the chunks of rows that are all
            // infinite; then record the updated tile's finite rows for phase 3
            __shared__ uint32_t rm[4];
            tile_row_mask<T>(acc, rm, tid, tx, ty);
            uint32_t cm = 0u;
#pragma unroll
            for (int c = 0; c < NCHUNK; ++c) cm |= rm[c] ? (1u << c) : 0u;
            minplus_panels_masked<T>(acc, M, n, o, o, cj, sm, tid, tx, ty, cm);
            tile_row_mask<T>(acc, rm, tid, tx, ty);
            if (tid < 4) kmask[(int64_t)J * 4 + tid] = rm[tid];
        } else {
            minplus_panels<T>(acc, M, n, o, o, cj, sm, tid, tx, ty);
        }
        store_c<T>(acc, M, n, o, cj, tx, ty);
        store_c_transposed<T>(acc, M, n, o, cj, tx, ty);
    }
    if (counter == nullptr) return;
    __shared__ uint32_t last;
    __threadfence();  // (this CTA's tiles and flags, before its ticket)
    __syncthreads();
    if (tid == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1u ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();  // (every other CTA's writes, after their tickets)
    if (mark_all)
        for (int32_t J = r + 1 + tid; J < R; J += blockDim.x) rowflags[(int64_t)r * R + J] = 0xffffffffu;
    __syncthreads();
    compact_trail(rowflags, R, r, list, cand, tiles, 1);
    if (tid == 0) *counter = 0u;
}

__global__ void k_add_u64(unsigned long long* __restrict__ dst, const unsigned long long* __restrict__ src, int n) {
    if ((int)threadIdx.x < n) dst[threadIdx.x] += src[threadIdx.x];
}

// Upper-triangle task t (0 <= t < c(c+1)/2) -> pair (x, y), 0 <= x <= y < c, row-major.
// (float estimate of the row, then exact integer correction; c < 2^16 tiles.)
__device__ __forceinline__ void tri_pair(int64_t t, int64_t c, int64_t& x, int64_t& y) {
    const int32_t ti = (int32_t)t, ci = (int32_t)c;
    const float b = 2.0f * (float)ci + 1.0f;
    int32_t xx = (int32_t)((b - sqrtf(fmaxf(b * b - 8.0f * (float)ti, 0.0f))) * 0.5f);
    xx = xx < 0 ? 0 : (xx > ci - 1 ? ci - 1 : xx);
    while (xx > 0 && xx * ci - xx * (xx - 1) / 2 > ti) --xx;
    while (xx + 1 < ci && (xx + 1) * ci - (xx + 1) * xx / 2 <= ti) ++xx;
    x = xx;
    y = xx + (ti - (xx * ci - xx * (xx - 1) / 2));
}

// Phase-3 update of tile (I, J), I <= J, and, by symmetry, of (J, I) = (I, J)^T.
template <typename T>
__device__ __forceinline__ void phase3_tile(T* __restrict__ M, int64_t n, int64_t o, int64_t I, int64_t J,
                                            PanelSmem<T>& sm, int tid, int tx, int ty) {
    const int64_t ci = I * T_, cj = J * T_;
    T acc[8][8];
    load_c<T>(acc, M, n, ci, cj, tx, ty);
    minplus_panels<T>(acc, M, n, o, ci, cj, sm, tid, tx, ty);
    store_c<T>(acc, M, n, ci, cj, tx, ty);
    if (I != J) store_c_transposed<T>(acc, M, n, ci, cj, tx, ty);
}

// ---------------- phase 3, batched form: tiles (I, J), I <= J, I, J != r ----------------
template <typename T>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS) k_phase3_batched(T* __restrict__ base, const MatDesc* __restrict__ descs,
                                                           int32_t nmat, int32_t r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int32_t mi = blockIdx.y; mi < nmat; mi += gridDim.y) {
        const MatDesc d = descs[mi];
        const int64_t n = d.n;
        const int32_t R = (int32_t)((n + T_ - 1) / T_);
        const int64_t Rm = R - 1;
        if (r >= R || (int64_t)blockIdx.x >= Rm * (Rm + 1) / 2) continue;
        int64_t I, J;
        tri_pair((int64_t)blockIdx.x, Rm, I, J);
        I += (I >= r);
        J += (J >= r);
        phase3_tile<T>(base + d.off, n, (int64_t)r * T_, I, J, sm, tid, tx, ty);
    }
}

// ---------------- phase 3 over the matrices active in round r ----------------
// sel[0..nsel) = matrices with more than r + 1 tile rows; p3off[0..nsel] = exclusive
// prefix of their task counts Rm(Rm + 1)/2 (Rm = tiles per side minus the pivot).
template <typename T>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS) k_phase3_sel(T* __restrict__ base,
                                                                     const MatDesc* __restrict__ descs,
                                                                     const int32_t* __restrict__ sel, int32_t nsel,
                                                                     const int64_t* __restrict__ p3off, int32_t r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t total = p3off[nsel];
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        int32_t lo = 0, hi = nsel;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (p3off[mid] <= t) lo = mid; else hi = mid;
        }
        const MatDesc d = descs[sel[lo]];
        const int64_t Rm = (d.n + T_ - 1) / T_ - 1;
        int64_t I, J;
        tri_pair(t - p3off[lo], Rm, I, J);
        I += (I >= r);
        J += (J >= r);
        phase3_tile<T>(base + d.off, d.n, (int64_t)r * T_, I, J, sm, tid, tx, ty);
    }
}

// ---------------- phase 3, single large matrix: persistent over a tile list ----------------
// list[0] = count c, list[1..c] = ascending tile indices J != r whose row tile (r, J)
// holds a finite entry; every (I, J) in list x list is updated, the pairs I < J once
// for both triangles.  Tiles outside list x list keep their values: their pivot panel
// is entirely infinite, so min(D, inf + x) = D.
// With rowflags (elimination form), a target marked 2 was never initialised: it starts
// from infinity instead of being loaded, and is marked 1 afterwards.  Targets (I, J) with
// I >= shared_from may be updated by concurrent runs of rounds: stored with atomicMin.
template <typename T>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS) k_phase3_list(T* __restrict__ M, int64_t n, int32_t r,
                                                        const uint32_t* __restrict__ list,
                                                        uint32_t* __restrict__ rowflags, int32_t R,
                                                        int32_t shared_from,
                                                        const uint32_t* __restrict__ kmask = nullptr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t c = list[0];
    const int64_t o = (int64_t)r * T_;
    for (int64_t t = blockIdx.x; t < c * (c + 1) / 2; t += gridDim.x) {
        int64_t x, y;
        tri_pair(t, c, x, y);
        const int64_t I = list[1 + x], J = list[1 + y];
        uint32_t* f = (rowflags && I < J) ? rowflags + I * R + J : nullptr;
        if (!kmask) {
            if (f && *f == 2u) {
                const int64_t ci = I * T_, cj = J * T_;
                T acc[8][8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = Inf<T>::value();
                minplus_panels<T>(acc, M, n, o, ci, cj, sm, tid, tx, ty);
                store_c<T>(acc, M, n, ci, cj, tx, ty);
                store_c_transposed<T>(acc, M, n, ci, cj, tx, ty);
                if (tid == 0) *f = 1u;  // (every thread read the flag before the panel barriers)
            } else if (I >= shared_from) {
                const int64_t ci = I * T_, cj = J * T_;
                T acc[8][8];
                load_c<T>(acc, M, n, ci, cj, tx, ty);
                minplus_panels<T>(acc, M, n, o, ci, cj, sm, tid, tx, ty);
                store_c_min<T>(acc, M, n, ci, cj, tx, ty);
                if (I != J) store_c_transposed_min<T>(acc, M, n, ci, cj, tx, ty);
            } else {
                phase3_tile<T>(M, n, o, I, J, sm, tid, tx, ty);
            }
            continue;
        }
        // with the row masks of this round's row tiles (kmask: 4 words per tile, set by
        // phase 2): only the chunks of pivot rows finite in both panels
        uint32_t cm = 0u;
#pragma unroll
        for (int q = 0; q < NCHUNK; ++q) cm |= (kmask[I * 4 + q] & kmask[J * 4 + q]) ? (1u << q) : 0u;
        const bool fresh = f && *f == 2u;
        __syncthreads();  // (every thread has read the mark before thread 0 may change it)
        const int64_t ci = I * T_, cj = J * T_;
        T acc[8][8];
        if (fresh) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = Inf<T>::value();
        } else {
            load_c<T>(acc, M, n, ci, cj, tx, ty);
        }
        minplus_panels_masked<T>(acc, M, n, o, ci, cj, sm, tid, tx, ty, cm);
        if (!fresh && I >= shared_from) {
            store_c_min<T>(acc, M, n, ci, cj, tx, ty);
            if (I != J) store_c_transposed_min<T>(acc, M, n, ci, cj, tx, ty);
        } else {
            store_c<T>(acc, M, n, ci, cj, tx, ty);
            if (I != J) store_c_transposed<T>(acc, M, n, ci, cj, tx, ty);
        }
        if (fresh && tid == 0) *f = 1u;
    }
}

// Build the tile list of round r from the flags phase 2 set (and clear the flags).
// Also accumulates the number of phase-3 tiles into tiles[0] and of phase-2 tiles with a
// finite entry (the ones phase 2 computed) into tiles[1].
__global__ void k_compact(uint32_t* __restrict__ flags, int32_t R, int32_t r, uint32_t* __restrict__ list,
                          unsigned long long* __restrict__ tiles) {
    __shared__ uint32_t cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int32_t base = 0; base < R; base += blockDim.x) {
        int32_t J = base + threadIdx.x;
        bool take = J < R && J != r && flags[J] != 0u;
        unsigned ballot = __ballot_sync(0xffffffffu, take);
        // ordered compaction: warp prefix, then warps in order
        __shared__ uint32_t wsum[32];
        int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) wsum[warp] = __popc(ballot);
        __syncthreads();
        uint32_t off = cnt;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (take) list[1 + off + __popc(ballot & ((1u << lane) - 1u))] = (uint32_t)J;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
            cnt += tot;
        }
        __syncthreads();
    }
    for (int32_t J = threadIdx.x; J < R; J += blockDim.x) flags[J] = 0u;
    if (threadIdx.x == 0) {
        list[0] = cnt;
        tiles[0] += (unsigned long long)cnt * (cnt + 1) / 2;  // phase-3 tiles of this round
        tiles[1] += (unsigned long long)cnt;                  // phase-2 tiles computed (finite)
    }
}

// ---------------- many matrices with infinite-panel skipping ----------------
// Per matrix mi (one CTA each): compact the flags of round r into the list at
// lists[mi * lstride] (count, then tile indices) and write the matrix's phase-3 task
// count c(c+1)/2 into offs[mi] (offs is scanned to task offsets afterwards).
__global__ void k_compact_many(uint32_t* __restrict__ flags, int32_t fstride, const MatDesc* __restrict__ descs,
                               int32_t nmat, int32_t r, uint32_t* __restrict__ lists, int32_t lstride,
                               uint32_t* __restrict__ offs, unsigned long long* __restrict__ tiles) {
    __shared__ uint32_t cnt;
    __shared__ uint32_t wsum[32];
    const int32_t mi = blockIdx.x;
    if (mi >= nmat) return;
    const int32_t R = (descs[mi].n + T_ - 1) / T_;
    uint32_t* f = flags + (int64_t)mi * fstride;
    uint32_t* list = lists + (int64_t)mi * lstride;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int32_t base = 0; base < R && r < R; base += blockDim.x) {
        const int32_t J = base + threadIdx.x;
        const bool take = J < R && J != r && f[J] != 0u;
        const unsigned ballot = __ballot_sync(0xffffffffu, take);
        if (lane == 0) wsum[warp] = __popc(ballot);
        __syncthreads();
        uint32_t off = cnt;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (take) list[1 + off + __popc(ballot & ((1u << lane) - 1u))] = (uint32_t)J;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
            cnt += tot;
        }
        __syncthreads();
    }
    for (int32_t J = threadIdx.x; J < R; J += blockDim.x) f[J] = 0u;
    if (threadIdx.x == 0) {
        const uint32_t c = r < R ? cnt : 0u;
        list[0] = c;
        offs[mi] = c * (c + 1) / 2;
        atomicAdd(&tiles[0], (unsigned long long)c * (c + 1) / 2);
        atomicAdd(&tiles[1], (unsigned long long)c);
    }
}

// Phase 3 over the task lists of every matrix: offs[0..nmat] holds the exclusive task
// offsets (offs[nmat] = total); task t belongs to the matrix whose range holds it.
template <typename T>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS) k_phase3_many(T* __restrict__ base,
                                                                      const MatDesc* __restrict__ descs, int32_t nmat,
                                                                      int32_t r, const uint32_t* __restrict__ lists,
                                                                      int32_t lstride,
                                                                      const uint32_t* __restrict__ offs,
                                                                      const uint32_t* __restrict__ kmask = nullptr,
                                                                      int32_t kstride = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t total = offs[nmat];
    const int64_t o = (int64_t)r * T_;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        int32_t lo = 0, hi = nmat;  // largest mi with offs[mi] <= t
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if ((int64_t)offs[mid] <= t) lo = mid; else hi = mid;
        }
        const MatDesc d = descs[lo];
        const uint32_t* list = lists + (int64_t)lo * lstride;
        int64_t x, y;
        tri_pair(t - (int64_t)offs[lo], (int64_t)list[0], x, y);
        const int64_t I = list[1 + x], J = list[1 + y];
        if (!kmask) {
            phase3_tile<T>(base + d.off, d.n, o, I, J, sm, tid, tx, ty);
            continue;
        }
        // only the chunks of pivot rows finite in both row tiles (masks set by k_phase2)
        const uint32_t* km = kmask + (int64_t)lo * kstride;
        uint32_t cm = 0u;
#pragma unroll
        for (int q = 0; q < NCHUNK; ++q) cm |= (km[I * 4 + q] & km[J * 4 + q]) ? (1u << q) : 0u;
        T* M = base + d.off;
        const int64_t ci = I * T_, cj = J * T_;
        T acc[8][8];
        load_c<T>(acc, M, d.n, ci, cj, tx, ty);
        minplus_panels_masked<T>(acc, M, d.n, o, ci, cj, sm, tid, tx, ty, cm);
        store_c<T>(acc, M, d.n, ci, cj, tx, ty);
        if (I != J) store_c_transposed<T>(acc, M, d.n, ci, cj, tx, ty);
    }
}

int g_sms = 0;
int sms() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

template <typename T>
cudaError_t set_smem_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e;
    e = cudaFuncSetAttribute(k_phase1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, T_ * T_ * (int)sizeof(T));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase1_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, T_ * T_ * (int)sizeof(float));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PanelSmem<T>));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase3_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PanelSmem<T>));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase3_list<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PanelSmem<T>));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase2_cand<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PanelSmem<T>));

    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase3_many<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PanelSmem<T>));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_phase3_sel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PanelSmem<T>));
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

}  // namespace

// One round r of the elimination form: phase 1, phase 2 over the candidates of row r,
// the compaction (phase-3 list, marks, next candidates), phase 3 over the list.
template <typename T>
cudaError_t elim_round(T* M, const MatDesc* dd, int64_t N, int32_t r, int32_t R, uint32_t* rowflags, uint32_t* cand,
                       uint32_t* list, bool skip_inf, unsigned long long* tiles, uint32_t* counter,
                       uint32_t* kmask, int32_t shared_from, cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t st) {
    const size_t psm = sizeof(PanelSmem<T>);
    const int grid = sms() * 2;
    if constexpr (std::is_same<T, float>::value)
        k_phase1_wide<<<1, 1024, T_ * T_ * sizeof(float), st>>>(M, N, r);
    else
        k_phase1<T><<<dim3(1, 1), NTH, T_ * T_ * sizeof(T), st>>>(M, dd, 1, r, nullptr);
    count_launches(1);
    const int32_t np2 = R - 1 - r;
    if (np2 > 0) {
        // phase 2, and the compaction in its last CTA (without skipping: every tile J > r
        // marked, so the compaction lists them all)
        // (with skipping, phase 2 records the row masks of the row tiles it computed and
        //  phase 3 skips the pivot-row chunks that are infinite in either panel)
        uint32_t* km = skip_inf ? kmask : nullptr;
        k_phase2_cand<T><<<np2 < grid ? np2 : grid, NTH, psm, st>>>(M, N, r, R, cand, rowflags, list, tiles,
                                                                     counter, skip_inf ? 0 : 1, km);
        if (ev0) cudaEventRecord(ev0, st);
        k_phase3_list<T><<<grid, NTH, psm, st>>>(M, N, r, list, rowflags, R, shared_from, km);
        if (ev1) cudaEventRecord(ev1, st);
        count_launches(2);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t fw_batched(T* base, const MatDesc* d_descs, const MatDesc* h_descs, int32_t nmat, int32_t max_n,
                       cudaStream_t st, int32_t** keep_buf) {
    if (nmat <= 0 || max_n <= 0) return cudaSuccess;
    cudaError_t e = set_smem_attrs<T>();
    if (e != cudaSuccess) return e;
    const int32_t R = (max_n + T_ - 1) / T_;
    // per round: the matrices still active (more than r tile rows), in one host buffer
    //   [sel_0 | p3off_0 (as two int32 words each) | sel_1 | ...]
    std::vector<int64_t> start(R + 1, 0);
    std::vector<int32_t> nsel(R, 0);
    std::vector<int32_t> buf;
    for (int32_t r = 0; r < R; ++r) {
        start[r] = (int64_t)buf.size();
        std::vector<int32_t> sel;
        for (int32_t m = 0; m < nmat; ++m)
            if ((h_descs[m].n + T_ - 1) / T_ > r) sel.push_back(m);
        nsel[r] = (int32_t)sel.size();
        buf.insert(buf.end(), sel.begin(), sel.end());
        if (buf.size() & 1) buf.push_back(0);  // 8-byte alignment of the offsets
        int64_t acc = 0;
        for (size_t i = 0; i <= sel.size(); ++i) {
            int32_t w2[2];
            memcpy(w2, &acc, 8);
            buf.push_back(w2[0]);
            buf.push_back(w2[1]);
            if (i < sel.size()) {
                const int64_t Rm = (h_descs[sel[i]].n + T_ - 1) / T_ - 1;
                acc += Rm * (Rm + 1) / 2;
            }
        }
    }
    int32_t* d_buf = keep_buf ? *keep_buf : nullptr;
    if (!d_buf) {
        e = scratch_alloc((void**)&d_buf, buf.size() * sizeof(int32_t), st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(d_buf, buf.data(), buf.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (keep_buf) *keep_buf = d_buf;
    }
    const size_t psm = sizeof(PanelSmem<T>);
    const int p3_grid = sms() * 2;
    for (int32_t r = 0; r < R && e == cudaSuccess; ++r) {
        const int32_t ns = nsel[r];
        if (ns == 0) break;
        const int32_t* sel = d_buf + start[r];
        const int64_t* p3off = reinterpret_cast<const int64_t*>(d_buf + start[r] + ns + (ns & 1));
        const unsigned gy = (unsigned)(ns < 65535 ? ns : 65535);
        k_phase1<T><<<dim3(1, gy), NTH, T_ * T_ * sizeof(T), st>>>(base, d_descs, ns, r, sel);
        count_launches(1);
        if (R > 1) {
            k_phase2<T><<<dim3(R - 1, gy), NTH, psm, st>>>(base, d_descs, ns, r, nullptr, 0, sel);
            k_phase3_sel<T><<<p3_grid, NTH, psm, st>>>(base, d_descs, sel, ns, p3off, r);
            count_launches(2);
        }
        e = cudaGetLastError();
    }
    if (!keep_buf) cudaFreeAsync(d_buf, st);  // (the pageable upload above completed before it returned)
    return e;
}

int64_t fw_single_scratch_words(int64_t N) {
    int64_t R = (N + T_ - 1) / T_;
    return 3 * R + 8;  // flags[R], list[1 + R] (+1 pad), two tile counters (u64), cand[1 + R] (+1)
}

template <typename T>
cudaError_t fw_single(T* M, int64_t N, bool skip_inf, uint32_t* scratch, uint32_t* rowflags, double* updates,
                      FwProfile* prof, cudaStream_t st, const std::vector<ElimTask>* tasks) {
    if (updates) *updates = 0.0;
    if (N <= 0) return cudaSuccess;
    cudaError_t e = set_smem_attrs<T>();
    if (e != cudaSuccess) return e;
    const int32_t R = (int32_t)((N + T_ - 1) / T_);
    uint32_t* flags = scratch;
    uint32_t* list = scratch + R;
    unsigned long long* tiles = reinterpret_cast<unsigned long long*>(scratch + 2 * R + 2);
    e = cudaMemsetAsync(scratch, 0, fw_single_scratch_words(N) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    MatDesc h{0, (int32_t)N, 0};
    MatDesc* dd = nullptr;
    e = scratch_alloc((void**)&dd, sizeof(MatDesc), st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dd, &h, sizeof(MatDesc), cudaMemcpyHostToDevice, st);
    const size_t psm = sizeof(PanelSmem<T>);
    const int p3_grid = sms() * 2;
    // optional per-launch timing of phase 3 (one event pair per round)
    std::vector<cudaEvent_t> evs;
    if (prof && R > 1) {
        evs.resize(2 * (size_t)R, nullptr);
        for (auto& ev : evs)
            if (e == cudaSuccess) e = cudaEventCreate(&ev);
    }
    // runs of elimination rounds: one run over every block row, or the caller's runs (side
    // by side on their own streams where they do not depend on each other)
    std::vector<ElimTask> one(1);
    one[0].lo = 0;
    one[0].hi = R;
    one[0].shared_from = R;
    const std::vector<ElimTask>& runs = (rowflags && tasks && !tasks->empty()) ? *tasks : one;
    const size_t nrun = rowflags ? runs.size() : 0;
    // per run: list[R + 2], cand[R + 2], tiles (2 x u64), the phase-2 CTA counter (+ pad),
    // the row masks of the round's row tiles (4 words per tile)
    const int64_t rw = 6 * (int64_t)R + 10;
    uint32_t* run_scratch = nullptr;
    std::vector<cudaStream_t> rs(nrun, nullptr);
    std::vector<cudaEvent_t> done(nrun, nullptr);
    cudaEvent_t start_ev = nullptr;
    if (nrun > 0) {
        if (e == cudaSuccess) e = scratch_alloc((void**)&run_scratch, nrun * rw * sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(run_scratch, 0, nrun * rw * sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(start_ev, st);
        for (size_t i = 0; i < nrun && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&rs[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(rs[i], start_ev, 0);
        }
        // issue the rounds of every startable run in turn, one round at a time
        std::vector<int32_t> next(nrun, 0), state(nrun, 0);  // 0 waiting, 1 issuing, 2 issued
        size_t finished = 0;
        while (finished < nrun && e == cudaSuccess) {
            for (size_t i = 0; i < nrun && e == cudaSuccess; ++i) {
                const ElimTask& tk = runs[i];
                uint32_t* rl = run_scratch + i * rw;
                uint32_t* rc = rl + R + 2;
                unsigned long long* rt = reinterpret_cast<unsigned long long*>(rl + 2 * R + 4);
                if (state[i] == 0) {
                    bool ready = true;
                    for (int32_t d : tk.deps) ready = ready && state[d] == 2;
                    if (!ready) continue;
                    for (int32_t d : tk.deps) cudaStreamWaitEvent(rs[i], done[d], 0);
                    if (tk.lo < tk.hi) {  // candidates of the run's first round
                        k_compact_trail<<<1, 1024, 0, rs[i]>>>(rowflags, R, tk.lo - 1, rl, rc, rt, 0);
                        count_launches(1);
                    }
                    next[i] = tk.lo;
                    state[i] = 1;
                }
                if (state[i] == 1) {
                    if (next[i] < tk.hi) {
                        const int32_t r = next[i]++;
                        e = elim_round<T>(M, dd, N, r, R, rowflags, rc, rl, skip_inf, rt, rl + 2 * R + 8,
                                          rl + 2 * R + 10, tk.shared_from,
                                          evs.empty() ? nullptr : evs[2 * r], evs.empty() ? nullptr : evs[2 * r + 1],
                                          rs[i]);
                    } else {
                        e = cudaEventRecord(done[i], rs[i]);
                        state[i] = 2;
                        ++finished;
                    }
                }
            }
        }
        for (size_t i = 0; i < nrun && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, done[i], 0);
        // tile counters of every run, summed
        for (size_t i = 0; i < nrun && e == cudaSuccess; ++i) {
            k_add_u64<<<1, 32, 0, st>>>(tiles, reinterpret_cast<unsigned long long*>(run_scratch + i * rw + 2 * R + 4),
                                        2);
            count_launches(1);
        }
    }
    for (int32_t r = 0; r < R && e == cudaSuccess && !rowflags; ++r) {
        k_phase1<T><<<dim3(1, 1), NTH, T_ * T_ * sizeof(T), st>>>(M, dd, 1, r, nullptr);
        count_launches(1);
        if (R > 1) {
            k_phase2<T><<<dim3(R - 1, 1), NTH, psm, st>>>(M, dd, 1, r, flags, 0, nullptr);
            if (!skip_inf) {
                // mark every tile: the compaction then lists all J != r
                cudaMemsetAsync(flags, 0xff, R * sizeof(uint32_t), st);
            }
            k_compact<<<1, 1024, 0, st>>>(flags, R, r, list, tiles);
            if (!evs.empty()) cudaEventRecord(evs[2 * r], st);
            k_phase3_list<T><<<p3_grid, NTH, psm, st>>>(M, N, r, list, nullptr, 0, (int32_t)R);
            if (!evs.empty()) cudaEventRecord(evs[2 * r + 1], st);
            count_launches(3);
        }
        e = cudaGetLastError();
    }
    unsigned long long htv[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(htv, tiles, sizeof(htv), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(dd, st);
    if (run_scratch) cudaFreeAsync(run_scratch, st);
    for (auto& x : rs)
        if (x) cudaStreamDestroy(x);
    for (auto& x : done)
        if (x) cudaEventDestroy(x);
    if (start_ev) cudaEventDestroy(start_ev);
    if (prof) {
        prof->p3_ms = 0.0;
        prof->p3_launches = 0;
        for (size_t r = 0; e == cudaSuccess && 2 * r + 1 < evs.size(); ++r) {
            if (rowflags && (int32_t)r + 1 >= R) break;  // no phase 3 in the last round
            float t = 0.f;
            if (cudaEventElapsedTime(&t, evs[2 * r], evs[2 * r + 1]) == cudaSuccess) {
                prof->p3_ms += t;
                prof->p3_launches += 1;
            }
        }
        prof->p3_updates = (double)htv[0] * (double)T_ * T_ * T_;
    }
    for (auto& ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (updates) {
        double t3 = (double)T_ * T_ * T_;
        *updates = ((double)htv[0] + (double)htv[1] + (double)R) * t3;  // phase 3, phase 2, phase 1 tiles
    }
    return e;
}

int64_t fw_many_scratch_words(int32_t nmat, int32_t max_n) {
    const int64_t R = (max_n + T_ - 1) / T_;
    // flags, lists, offsets, (alignment), two u64 counters, row masks (4 words per tile)
    return (int64_t)nmat * R + (int64_t)nmat * (R + 1) + nmat + 1 + 1 + 4 + (int64_t)nmat * R * 4;
}

template <typename T>
cudaError_t fw_many_skip(T* base, const MatDesc* d_descs, int32_t nmat, int32_t max_n, uint32_t* scratch,
                         double* updates, cudaStream_t st, bool trail, bool stats) {
    if (updates && stats) *updates = 0.0;
    if (nmat <= 0 || max_n <= 0) return cudaSuccess;
    cudaError_t e = set_smem_attrs<T>();
    if (e != cudaSuccess) return e;
    const int32_t R = (max_n + T_ - 1) / T_;
    uint32_t* flags = scratch;
    uint32_t* lists = flags + (int64_t)nmat * R;
    uint32_t* offs = lists + (int64_t)nmat * (R + 1);
    int64_t toff = (int64_t)nmat * R + (int64_t)nmat * (R + 1) + nmat + 1;
    toff += toff & 1;  // 8-byte alignment of the counters
    unsigned long long* tiles = reinterpret_cast<unsigned long long*>(scratch + toff);
    uint32_t* kmask = scratch + toff + 4;  // per matrix R x 4 words
    const int32_t kstride = 4 * R;
    e = cudaMemsetAsync(scratch, 0, (size_t)(toff + 4) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned gy = (unsigned)(nmat < 65535 ? nmat : 65535);
    const size_t psm = sizeof(PanelSmem<T>);
    const int p3_grid = sms() * 2;
    for (int32_t r = 0; r < R && e == cudaSuccess; ++r) {
        k_phase1<T><<<dim3(1, gy), NTH, T_ * T_ * sizeof(T), st>>>(base, d_descs, nmat, r, nullptr);
        count_launches(1);
        if (R > 1 && (!trail || r + 1 < R)) {
            // (elimination form: the flags of the tiles left of r stay clear, so the lists
            //  and phase 3 hold only tiles right of / below the pivot block)
            // (row masks: phase 3 skips the pivot-row chunks infinite in either row tile)
            if (trail)
                k_phase2<T><<<dim3(R - 1 - r, gy), NTH, psm, st>>>(base, d_descs, nmat, r, flags, R, nullptr, 1,
                                                                    kmask, kstride);
            else
                k_phase2<T><<<dim3(R - 1, gy), NTH, psm, st>>>(base, d_descs, nmat, r, flags, R, nullptr, 0, kmask,
                                                                kstride);
            k_compact_many<<<nmat, 1024, 0, st>>>(flags, R, d_descs, nmat, r, lists, R + 1, offs, tiles);
            launch_scan_excl(offs, nmat + 1, st);
            k_phase3_many<T><<<p3_grid, NTH, psm, st>>>(base, d_descs, nmat, r, lists, R + 1, offs, kmask, kstride);
            count_launches(4);
        }
        e = cudaGetLastError();
    }
    if (!stats) return e;
    unsigned long long htv[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(htv, tiles, sizeof(htv), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // phase-3 and phase-2 tiles; the caller adds the phase-1 (diagonal) tiles
    if (updates) *updates = ((double)htv[0] + (double)htv[1]) * (double)T_ * T_ * T_;
    return e;
}

template cudaError_t fw_many_skip<int32_t>(int32_t*, const MatDesc*, int32_t, int32_t, uint32_t*, double*,
                                           cudaStream_t, bool, bool);
template cudaError_t fw_many_skip<float>(float*, const MatDesc*, int32_t, int32_t, uint32_t*, double*, cudaStream_t,
                                         bool, bool);

template cudaError_t fw_batched<int32_t>(int32_t*, const MatDesc*, const MatDesc*, int32_t, int32_t, cudaStream_t,
                                         int32_t**);
template cudaError_t fw_batched<float>(float*, const MatDesc*, const MatDesc*, int32_t, int32_t, cudaStream_t,
                                       int32_t**);
template cudaError_t fw_single<int32_t>(int32_t*, int64_t, bool, uint32_t*, uint32_t*, double*, FwProfile*,
                                        cudaStream_t, const std::vector<ElimTask>*);
template cudaError_t fw_single<float>(float*, int64_t, bool, uint32_t*, uint32_t*, double*, FwProfile*, cudaStream_t,
                                      const std::vector<ElimTask>*);

}  // namespace spq
