// Tile machinery shared by the Floyd-Warshall kernels (fw.cu) and the elimination /
// back-substitution kernels of the boundary graph (elim.cu): a 128 x 128 tile per CTA of
// 256 threads, each thread owning an 8 x 8 block; min-plus panels staged in 32-row chunks
// through shared memory with cp.async (double-buffered).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace spq {
namespace {

// Compile-time tuning of the phase-2/3 kernels: resident CTAs per SM requested from the
// register allocator, and unrolling of the float32 inner loop (two k steps per trip).
#ifndef SPQ_FW_MIN_CTAS
#define SPQ_FW_MIN_CTAS 2
#endif
#ifndef SPQ_FW_UNROLL
#define SPQ_FW_UNROLL 1
#endif

constexpr int kInnerUnroll = SPQ_FW_UNROLL;
constexpr int T_ = kTile;  // 128
constexpr int KC = 32;     // k rows per staged panel chunk
constexpr int NTH = 256;   // threads per CTA; each owns an 8 x 8 block of the tile
constexpr int NCHUNK = T_ / KC;

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

template <typename T>
struct MP;
template <>
struct MP<float> {
    // min(c, a0 + b0, a1 + b1)
    static __device__ __forceinline__ float upd2(float c, float a0, float b0, float a1, float b1) {
        return fmin3(c, a0 + b0, a1 + b1);
    }
    static __device__ __forceinline__ float upd1(float c, float a, float b) { return fminf(c, a + b); }
};
template <>
struct MP<int32_t> {
    static __device__ __forceinline__ int32_t upd2(int32_t c, int32_t a0, int32_t b0, int32_t a1, int32_t b1) {
        return __viaddmin_s32(a0, b0, __viaddmin_s32(a1, b1, c));
    }
    static __device__ __forceinline__ int32_t upd1(int32_t c, int32_t a, int32_t b) { return __viaddmin_s32(a, b, c); }
};

template <typename T>
__device__ __forceinline__ int4 inf4() {
    T v = Inf<T>::value();
    int x = *reinterpret_cast<int*>(&v);
    return make_int4(x, x, x, x);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename T>
struct alignas(16) PanelSmem {
    T a[2][KC][T_];
    T b[2][KC][T_];
};

// Thread-owned rows / columns inside a tile: {q*4 .. q*4+3} and {64 + q*4 .. 64+q*4+3}.
__device__ __forceinline__ int own(int q, int i) { return (i < 4) ? q * 4 + i : 64 + q * 4 + (i - 4); }

// Stage rows [row0, row0+KC) x cols [col0, col0+128) of M (n x n) into P; cells outside
// the matrix read as infinity.
template <typename T>
__device__ __forceinline__ void stage_chunk(T (*P)[T_], const T* __restrict__ M, int64_t n, int64_t row0,
                                            int64_t col0, int tid) {
#pragma unroll
    for (int it = 0; it < (KC * T_ / 4) / NTH; ++it) {
        int idx = it * NTH + tid;
        int kk = idx >> 5, c4 = idx & 31;
        int64_t r = row0 + kk, c = col0 + c4 * 4;
        T* dst = &P[kk][c4 * 4];
        if (r < n && c < n)
            cp_async16(dst, M + r * n + c);
        else
            *reinterpret_cast<int4*>(dst) = inf4<T>();
    }
}

template <typename T>
__device__ __forceinline__ void load_c(T (&acc)[8][8], const T* __restrict__ M, int64_t n, int64_t r0, int64_t c0,
                                       int tx, int ty) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int64_t r = r0 + own(ty, i);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int64_t c = c0 + own(tx, h * 4);
            int4 v = (r < n && c < n) ? *reinterpret_cast<const int4*>(M + r * n + c) : inf4<T>();
            acc[i][h * 4 + 0] = *reinterpret_cast<T*>(&v.x);
            acc[i][h * 4 + 1] = *reinterpret_cast<T*>(&v.y);
            acc[i][h * 4 + 2] = *reinterpret_cast<T*>(&v.z);
            acc[i][h * 4 + 3] = *reinterpret_cast<T*>(&v.w);
        }
    }
}

template <typename T>
__device__ __forceinline__ void store_c(const T (&acc)[8][8], T* __restrict__ M, int64_t n, int64_t r0, int64_t c0,
                                        int tx, int ty) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int64_t r = r0 + own(ty, i);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int64_t c = c0 + own(tx, h * 4);
            if (r < n && c < n) {
                int4 v;
                v.x = *reinterpret_cast<const int*>(&acc[i][h * 4 + 0]);
                v.y = *reinterpret_cast<const int*>(&acc[i][h * 4 + 1]);
                v.z = *reinterpret_cast<const int*>(&acc[i][h * 4 + 2]);
                v.w = *reinterpret_cast<const int*>(&acc[i][h * 4 + 3]);
                *reinterpret_cast<int4*>(M + r * n + c) = v;
            }
        }
    }
}

// Transposed store: acc[i][j] -> M[c0 + col(j)][r0 + row(i)].  Each thread writes
// 4 consecutive transposed columns (its rows q*4..q*4+3) as one 16-byte vector.
template <typename T>
__device__ __forceinline__ void store_c_transposed(const T (&acc)[8][8], T* __restrict__ M, int64_t n, int64_t r0,
                                                   int64_t c0, int tx, int ty) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int64_t tr = c0 + own(tx, j);  // transposed row
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int64_t tc = r0 + own(ty, h * 4);  // transposed column (multiple of 4)
            if (tr < n && tc < n) {
                int4 v;
                v.x = *reinterpret_cast<const int*>(&acc[h * 4 + 0][j]);
                v.y = *reinterpret_cast<const int*>(&acc[h * 4 + 1][j]);
                v.z = *reinterpret_cast<const int*>(&acc[h * 4 + 2][j]);
                v.w = *reinterpret_cast<const int*>(&acc[h * 4 + 3][j]);
                *reinterpret_cast<int4*>(M + tr * n + tc) = v;
            }
        }
    }
}

// Stores of tiles that concurrent writers may update (the min of every contribution
// wins): atomicMin on the 32-bit patterns, which order like the values for int32 and for
// non-negative float32 (distances are never negative).
template <typename T>
__device__ __forceinline__ void store_c_min(const T (&acc)[8][8], T* __restrict__ M, int64_t n, int64_t r0,
                                            int64_t c0, int tx, int ty) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + own(ty, i);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t c = c0 + own(tx, j);
            if (r < n && c < n) atomicMin(reinterpret_cast<int*>(M + r * n + c), *reinterpret_cast<const int*>(&acc[i][j]));
        }
    }
}
template <typename T>
__device__ __forceinline__ void store_c_transposed_min(const T (&acc)[8][8], T* __restrict__ M, int64_t n, int64_t r0,
                                                       int64_t c0, int tx, int ty) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t tr = c0 + own(tx, j);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t tc = r0 + own(ty, i);
            if (tr < n && tc < n)
                atomicMin(reinterpret_cast<int*>(M + tr * n + tc), *reinterpret_cast<const int*>(&acc[i][j]));
        }
    }
}

// acc = min(acc, A (x) B) over the KC-row chunk held in stage s:
// A[i][k] = a[s][k][i] (the panel is stored k-major), B[k][j] = b[s][k][j].
// (kend: the chunk's rows actually used, even, <= KC)
template <typename T>
__device__ __forceinline__ void compute_chunk(T (&acc)[8][8], const PanelSmem<T>& sm, int s, int tx, int ty,
                                              int kend = KC) {
#pragma unroll 1
    for (int kk = 0; kk < kend; kk += 2) {
        T a0[8], a1[8], b0[8], b1[8];
        {
            const int4 x0 = *reinterpret_cast<const int4*>(&sm.a[s][kk][ty * 4]);
            const int4 x1 = *reinterpret_cast<const int4*>(&sm.a[s][kk][64 + ty * 4]);
            const int4 y0 = *reinterpret_cast<const int4*>(&sm.a[s][kk + 1][ty * 4]);
            const int4 y1 = *reinterpret_cast<const int4*>(&sm.a[s][kk + 1][64 + ty * 4]);
            const int4 z0 = *reinterpret_cast<const int4*>(&sm.b[s][kk][tx * 4]);
            const int4 z1 = *reinterpret_cast<const int4*>(&sm.b[s][kk][64 + tx * 4]);
            const int4 w0 = *reinterpret_cast<const int4*>(&sm.b[s][kk + 1][tx * 4]);
            const int4 w1 = *reinterpret_cast<const int4*>(&sm.b[s][kk + 1][64 + tx * 4]);
            const int xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            const int ya[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
            const int zb[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
            const int wb[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                a0[i] = *reinterpret_cast<const T*>(&xa[i]);
                a1[i] = *reinterpret_cast<const T*>(&ya[i]);
                b0[i] = *reinterpret_cast<const T*>(&zb[i]);
                b1[i] = *reinterpret_cast<const T*>(&wb[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = MP<T>::upd2(acc[i][j], a0[i], b0[j], a1[i], b1[j]);
    }
}

// float32 form: the sums of two neighbouring columns come from one packed f32x2 add
// (sm_100 family), and a three-input min folds two k steps into each accumulator.
template <>
__device__ __forceinline__ void compute_chunk<float>(float (&acc)[8][8], const PanelSmem<float>& sm, int s, int tx,
                                                     int ty, int kend) {
#pragma unroll kInnerUnroll
    for (int kk = 0; kk < kend; kk += 2) {
        const float4 x0 = *reinterpret_cast<const float4*>(&sm.a[s][kk][ty * 4]);
        const float4 x1 = *reinterpret_cast<const float4*>(&sm.a[s][kk][64 + ty * 4]);
        const float4 y0 = *reinterpret_cast<const float4*>(&sm.a[s][kk + 1][ty * 4]);
        const float4 y1 = *reinterpret_cast<const float4*>(&sm.a[s][kk + 1][64 + ty * 4]);
        const float4 z0 = *reinterpret_cast<const float4*>(&sm.b[s][kk][tx * 4]);
        const float4 z1 = *reinterpret_cast<const float4*>(&sm.b[s][kk][64 + tx * 4]);
        const float4 w0 = *reinterpret_cast<const float4*>(&sm.b[s][kk + 1][tx * 4]);
        const float4 w1 = *reinterpret_cast<const float4*>(&sm.b[s][kk + 1][64 + tx * 4]);
        const float a0[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const float a1[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
        const float2 b0[4] = {make_float2(z0.x, z0.y), make_float2(z0.z, z0.w), make_float2(z1.x, z1.y),
                              make_float2(z1.z, z1.w)};
        const float2 b1[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                              make_float2(w1.z, w1.w)};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 p0 = make_float2(a0[i], a0[i]);
            const float2 p1 = make_float2(a1[i], a1[i]);
#pragma unroll
            for (int jp = 0; jp < 4; ++jp) {
                const float2 s0 = __fadd2_rn(p0, b0[jp]);
                const float2 s1 = __fadd2_rn(p1, b1[jp]);
                acc[i][2 * jp] = fmin3(acc[i][2 * jp], s0.x, s1.x);
                acc[i][2 * jp + 1] = fmin3(acc[i][2 * jp + 1], s0.y, s1.y);
            }
        }
    }
}

// acc = min(acc, A (x) B) with A[i][k] = M[arow0 + k][acol0 + i] and
// B[k][j] = M[arow0 + k][bcol0 + j], k over the pivot block [arow0, arow0 + 128).
template <typename T>
__device__ __forceinline__ void minplus_panels(T (&acc)[8][8], const T* __restrict__ M, int64_t n, int64_t prow0,
                                               int64_t acol0, int64_t bcol0, PanelSmem<T>& sm, int tid, int tx,
                                               int ty) {
    stage_chunk<T>(sm.a[0], M, n, prow0, acol0, tid);
    stage_chunk<T>(sm.b[0], M, n, prow0, bcol0, tid);
    cp_async_commit();
#pragma unroll 1
    for (int ch = 0; ch < NCHUNK; ++ch) {
        if (ch + 1 < NCHUNK) {
            const int s = (ch + 1) & 1;
            stage_chunk<T>(sm.a[s], M, n, prow0 + (ch + 1) * KC, acol0, tid);
            stage_chunk<T>(sm.b[s], M, n, prow0 + (ch + 1) * KC, bcol0, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        compute_chunk<T>(acc, sm, ch & 1, tx, ty);
        __syncthreads();
    }
}

// minplus_panels restricted to the 32-row chunks of the pivot block whose bit is set in
// cmask (bit c: rows [32c, 32c + 32)).  A chunk whose rows are all infinite in the A panel
// or in the B panel (row by row) changes nothing: each of its terms is infinite.  cmask
// must be the same for the whole CTA.
template <typename T>
__device__ __forceinline__ void minplus_panels_masked(T (&acc)[8][8], const T* __restrict__ M, int64_t n,
                                                      int64_t prow0, int64_t acol0, int64_t bcol0, PanelSmem<T>& sm,
                                                      int tid, int tx, int ty, uint32_t cmask) {
    int chs[NCHUNK];
    int nch = 0;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c)
        if ((cmask >> c) & 1u) chs[nch++] = c;
    if (nch == 0) return;
    stage_chunk<T>(sm.a[0], M, n, prow0 + chs[0] * KC, acol0, tid);
    stage_chunk<T>(sm.b[0], M, n, prow0 + chs[0] * KC, bcol0, tid);
    cp_async_commit();
#pragma unroll 1
    for (int t = 0; t < nch; ++t) {
        if (t + 1 < nch) {
            const int s = (t + 1) & 1;
            stage_chunk<T>(sm.a[s], M, n, prow0 + chs[t + 1] * KC, acol0, tid);
            stage_chunk<T>(sm.b[s], M, n, prow0 + chs[t + 1] * KC, bcol0, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        compute_chunk<T>(acc, sm, t & 1, tx, ty);
        __syncthreads();
    }
}

// Rows of the CTA's 128 x 128 tile (held in acc, 8 x 8 per thread) with a finite cell, as
// a 128-bit mask in words[0 .. 4) (shared memory, cleared here).  Whole CTA; starts and
// ends with a barrier.
template <typename T>
__device__ __forceinline__ void tile_row_mask(const T (&acc)[8][8], uint32_t* words, int tid, int tx, int ty) {
    __syncthreads();  // (earlier readers of words are done)
    if (tid < 4) words[tid] = 0u;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        bool f = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) f |= acc[i][j] < Inf<T>::value();
        if (f) {
            const int row = own(ty, i);
            atomicOr(&words[row >> 5], 1u << (row & 31));
        }
    }
    (void)tx;
    __syncthreads();
}

}  // namespace
}  // namespace spq
