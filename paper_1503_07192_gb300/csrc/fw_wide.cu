// Latency form of the elimination rounds (the forward pass before bg_backsub): the same
// three phases as fw.cu, but each 128 x 128 tile is handled by a CTA of 1024 threads with
// a 4 x 4 block per thread.  A round of the elimination updates only a few tiles (the
// pivot's frontier), one after the other over about a thousand rounds, so the time per
// tile, not the throughput over many tiles, is what counts here: four times the threads
// per tile cut each thread's share of a tile product by four.
#include <cuda_runtime.h>

#include <type_traits>

#include "common.cuh"
#include "fw_tile.cuh"

namespace spq {

namespace {

constexpr int NTW = 1024;  // threads per CTA: tx = lane (columns 4 tx ..), ty = warp (rows 4 ty ..)

template <typename T>
__device__ __forceinline__ void load_c_w(T (&acc)[4][4], const T* __restrict__ M, int64_t n, int64_t r0, int64_t c0,
                                         int tx, int ty) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + ty * 4 + i, c = c0 + tx * 4;
        const int4 v = (r < n && c < n) ? *reinterpret_cast<const int4*>(M + r * n + c) : inf4<T>();
        acc[i][0] = *reinterpret_cast<const T*>(&v.x);
        acc[i][1] = *reinterpret_cast<const T*>(&v.y);
        acc[i][2] = *reinterpret_cast<const T*>(&v.z);
        acc[i][3] = *reinterpret_cast<const T*>(&v.w);
    }
}

template <typename T>
__device__ __forceinline__ void store_c_w(const T (&acc)[4][4], T* __restrict__ M, int64_t n, int64_t r0, int64_t c0,
                                          int tx, int ty) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + ty * 4 + i, c = c0 + tx * 4;
        if (r < n && c < n) {
            int4 v;
            v.x = *reinterpret_cast<const int*>(&acc[i][0]);
            v.y = *reinterpret_cast<const int*>(&acc[i][1]);
            v.z = *reinterpret_cast<const int*>(&acc[i][2]);
            v.w = *reinterpret_cast<const int*>(&acc[i][3]);
            *reinterpret_cast<int4*>(M + r * n + c) = v;
        }
    }
}

// acc[i][j] -> M[c0 + 4 tx + j][r0 + 4 ty + i]
template <typename T>
__device__ __forceinline__ void store_c_transposed_w(const T (&acc)[4][4], T* __restrict__ M, int64_t n, int64_t r0,
                                                     int64_t c0, int tx, int ty) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t tr = c0 + tx * 4 + j, tc = r0 + ty * 4;
        if (tr < n && tc < n) {
            int4 v;
            v.x = *reinterpret_cast<const int*>(&acc[0][j]);
            v.y = *reinterpret_cast<const int*>(&acc[1][j]);
            v.z = *reinterpret_cast<const int*>(&acc[2][j]);
            v.w = *reinterpret_cast<const int*>(&acc[3][j]);
            *reinterpret_cast<int4*>(M + tr * n + tc) = v;
        }
    }
}

// One KC x 128 chunk: one 16-byte piece per thread.
template <typename T>
__device__ __forceinline__ void stage_chunk_w(T (*P)[T_], const T* __restrict__ M, int64_t n, int64_t row0,
                                              int64_t col0, int tid) {
    const int kk = tid >> 5, c4 = tid & 31;
    const int64_t r = row0 + kk, c = col0 + c4 * 4;
    T* dst = &P[kk][c4 * 4];
    if (r < n && c < n)
        cp_async16(dst, M + r * n + c);
    else
        *reinterpret_cast<int4*>(dst) = inf4<T>();
}

__device__ __forceinline__ void as4(const float4 v, float (&x)[4]) {
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
}

// acc = min(acc, A (x) B) over one staged chunk: A[i][k] = a[s][k][i], B[k][j] = b[s][k][j]
template <typename T>
__device__ __forceinline__ void compute_chunk_w(T (&acc)[4][4], const PanelSmem<T>& sm, int s, int tx, int ty) {
#pragma unroll 4
    for (int kk = 0; kk < KC; kk += 2) {
        const int4 xa = *reinterpret_cast<const int4*>(&sm.a[s][kk][ty * 4]);
        const int4 ya = *reinterpret_cast<const int4*>(&sm.a[s][kk + 1][ty * 4]);
        const int4 xb = *reinterpret_cast<const int4*>(&sm.b[s][kk][tx * 4]);
        const int4 yb = *reinterpret_cast<const int4*>(&sm.b[s][kk + 1][tx * 4]);
        const int a0[4] = {xa.x, xa.y, xa.z, xa.w}, a1[4] = {ya.x, ya.y, ya.z, ya.w};
        const int b0[4] = {xb.x, xb.y, xb.z, xb.w}, b1[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                acc[i][j] = MP<T>::upd2(acc[i][j], *reinterpret_cast<const T*>(&a0[i]),
                                        *reinterpret_cast<const T*>(&b0[j]), *reinterpret_cast<const T*>(&a1[i]),
                                        *reinterpret_cast<const T*>(&b1[j]));
    }
}

template <>
__device__ __forceinline__ void compute_chunk_w<float>(float (&acc)[4][4], const PanelSmem<float>& sm, int s, int tx,
                                                       int ty) {
#pragma unroll 1
    for (int kk = 0; kk < KC; kk += 2) {
        float a0[4], a1[4], b0[4], b1[4];
        as4(*reinterpret_cast<const float4*>(&sm.a[s][kk][ty * 4]), a0);
        as4(*reinterpret_cast<const float4*>(&sm.a[s][kk + 1][ty * 4]), a1);
        as4(*reinterpret_cast<const float4*>(&sm.b[s][kk][tx * 4]), b0);
        as4(*reinterpret_cast<const float4*>(&sm.b[s][kk + 1][tx * 4]), b1);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 p0 = make_float2(a0[i], a0[i]), p1 = make_float2(a1[i], a1[i]);
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const float2 s0 = __fadd2_rn(p0, make_float2(b0[2 * jp], b0[2 * jp + 1]));
                const float2 s1 = __fadd2_rn(p1, make_float2(b1[2 * jp], b1[2 * jp + 1]));
                acc[i][2 * jp] = fmin3(acc[i][2 * jp], s0.x, s1.x);
                acc[i][2 * jp + 1] = fmin3(acc[i][2 * jp + 1], s0.y, s1.y);
            }
        }
    }
}

// acc = min(acc, A (x) B), A[i][k] = M[prow0 + k][acol0 + i], B[k][j] = M[prow0 + k][bcol0 + j]
template <typename T>
__device__ __forceinline__ void minplus_panels_w(T (&acc)[4][4], const T* __restrict__ M, int64_t n, int64_t prow0,
                                                 int64_t acol0, int64_t bcol0, PanelSmem<T>& sm, int tid, int tx,
                                                 int ty) {
    stage_chunk_w<T>(sm.a[0], M, n, prow0, acol0, tid);
    stage_chunk_w<T>(sm.b[0], M, n, prow0, bcol0, tid);
    cp_async_commit();
#pragma unroll 1
    for (int ch = 0; ch < NCHUNK; ++ch) {
        if (ch + 1 < NCHUNK) {
            const int s = (ch + 1) & 1;
            stage_chunk_w<T>(sm.a[s], M, n, prow0 + (ch + 1) * KC, acol0, tid);
            stage_chunk_w<T>(sm.b[s], M, n, prow0 + (ch + 1) * KC, bcol0, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        compute_chunk_w<T>(acc, sm, ch & 1, tx, ty);
        __syncthreads();
    }
}

// Four consecutive shared-memory elements (16-byte aligned) as one vector load.
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&x)[4]) {
    const int4 v = *reinterpret_cast<const int4*>(p);
    x[0] = *reinterpret_cast<const T*>(&v.x);
    x[1] = *reinterpret_cast<const T*>(&v.y);
    x[2] = *reinterpret_cast<const T*>(&v.z);
    x[3] = *reinterpret_cast<const T*>(&v.w);
}

// Phase 1: closure of the diagonal tile (r, r) in shared memory.
template <typename T>
__global__ void __launch_bounds__(NTW, 1) k_phase1_w(T* __restrict__ M, int64_t n, int32_t r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*S)[T_] = reinterpret_cast<T(*)[T_]>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int64_t o = (int64_t)r * T_;
    {
        const int i = tid >> 3, c16 = (tid & 7) * 16;  // 8 threads per row, 16 elements each
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t gr = o + i, gc = o + c16 + q * 4;
            const int4 v = (gr < n && gc < n) ? *reinterpret_cast<const int4*>(M + gr * n + gc) : inf4<T>();
            *reinterpret_cast<int4*>(&S[i][c16 + q * 4]) = v;
        }
    }
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = S[ty * 4 + i][tx * 4 + j];
    const int K = (int)((n - o) < T_ ? (n - o) : T_);
    int k = 0;
    // two pivot steps per barrier (see fw.cu's k_phase1): row k + 1 after step k is formed
    // on the fly; the owners then publish rows k + 2 and k + 3
#pragma unroll 1
    for (; k + 1 < K; k += 2) {
        T a0[4], b0[4], a1[4], b1[4], ar[4], br[4];
        const T skk = S[k][k + 1];
        ld4<T>(&S[k][ty * 4], a0);
        ld4<T>(&S[k][tx * 4], b0);
        ld4<T>(&S[k + 1][ty * 4], ar);
        ld4<T>(&S[k + 1][tx * 4], br);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a1[i] = MP<T>::upd1(ar[i], skk, a0[i]);
            b1[i] = MP<T>::upd1(br[i], skk, b0[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = MP<T>::upd2(acc[i][j], a0[i], b0[j], a1[i], b1[j]);
        const int w = (k + 2) >> 2;  // the warp owning rows k + 2 and k + 3 (k even)
        if (ty == w) {
            const int i0 = (k + 2) & 3;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i == i0 || i == i0 + 1)
#pragma unroll
                    for (int j = 0; j < 4; ++j) S[ty * 4 + i][tx * 4 + j] = acc[i][j];
        }
        __syncthreads();
    }
    if (k < K) {  // an odd last step
        T a[4], b[4];
        ld4<T>(&S[k][ty * 4], a);
        ld4<T>(&S[k][tx * 4], b);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = MP<T>::upd1(acc[i][j], a[i], b[j]);
    }
    store_c_w<T>(acc, M, n, o, o, tx, ty);
}

// Phase 2 over the candidate row tiles (see fw.cu's k_phase2_cand).
template <typename T>
__global__ void __launch_bounds__(NTW, 1) k_phase2_cand_w(T* __restrict__ M, int64_t n, int32_t r, int32_t R,
                                                          const uint32_t* __restrict__ cand,
                                                          uint32_t* __restrict__ rowflags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int64_t o = (int64_t)r * T_;
    const uint32_t c = cand[0];
    const T inf = Inf<T>::value();
    for (uint32_t ci = blockIdx.x; ci < c; ci += gridDim.x) {
        const int32_t J = (int32_t)cand[1 + ci];
        const int64_t cj = (int64_t)J * T_;
        T acc[4][4];
        load_c_w<T>(acc, M, n, o, cj, tx, ty);
        bool fin = false;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) fin |= acc[i][j] < inf;
        if (!__syncthreads_or(fin)) {
            if (tid == 0) rowflags[(int64_t)r * R + J] = 0u;
            continue;
        }
        minplus_panels_w<T>(acc, M, n, o, o, cj, sm, tid, tx, ty);
        store_c_w<T>(acc, M, n, o, cj, tx, ty);
        store_c_transposed_w<T>(acc, M, n, o, cj, tx, ty);
    }
}

// Phase 3 over list x list (see fw.cu's k_phase3_list).
// A target tile marked 2 was never initialised (it held no finite entry so far): it
// starts from infinity instead of being loaded, and is marked 1 afterwards.
template <typename T>
__global__ void __launch_bounds__(NTW, 1) k_phase3_list_w(T* __restrict__ M, int64_t n, int32_t r,
                                                          const uint32_t* __restrict__ list,
                                                          uint32_t* __restrict__ rowflags, int32_t R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int64_t c = list[0];
    const int64_t o = (int64_t)r * T_;
    for (int64_t t = blockIdx.x; t < c * (c + 1) / 2; t += gridDim.x) {
        // t -> (x, y), x <= y, row-major over the upper triangle of list x list
        int64_t x = 0, rem = t;
        while (rem >= c - x) {
            rem -= c - x;
            ++x;
        }
        const int64_t I = list[1 + x], J = list[1 + x + rem];
        const int64_t ci = I * T_, cj = J * T_;
        uint32_t* f = I < J ? rowflags + I * R + J : nullptr;
        const bool fresh = f && *f == 2u;
        T acc[4][4];
        if (fresh) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = Inf<T>::value();
        } else {
            load_c_w<T>(acc, M, n, ci, cj, tx, ty);
        }
        minplus_panels_w<T>(acc, M, n, o, ci, cj, sm, tid, tx, ty);
        store_c_w<T>(acc, M, n, ci, cj, tx, ty);
        if (I != J) store_c_transposed_w<T>(acc, M, n, ci, cj, tx, ty);
        if (fresh && tid == 0) *f = 1u;  // (no other CTA of this launch reads the flag)
    }
}

}  // namespace

template <typename T>
cudaError_t wide_round(T* M, int64_t N, int32_t r, int32_t R, uint32_t* rowflags, const uint32_t* cand,
                       uint32_t* list, bool skip_inf, int grid, unsigned long long* tiles, cudaEvent_t ev0,
                       cudaEvent_t ev1, cudaStream_t st) {
    static bool attrs = false;
    if (!attrs) {
        cudaError_t e = cudaFuncSetAttribute(k_phase1_w<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             T_ * T_ * (int)sizeof(T));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_phase2_cand_w<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(PanelSmem<T>));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_phase3_list_w<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(PanelSmem<T>));
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    const size_t psm = sizeof(PanelSmem<T>);
    k_phase1_w<T><<<1, NTW, T_ * T_ * sizeof(T), st>>>(M, N, r);
    count_launches(1);
    const int32_t np2 = R - 1 - r;
    if (np2 > 0) {
        k_phase2_cand_w<T><<<np2 < grid ? np2 : grid, NTW, psm, st>>>(M, N, r, R, cand, rowflags);
        if (!skip_inf)  // mark every tile: the compaction then lists all J > r
            cudaMemsetAsync(rowflags + (int64_t)r * R + r + 1, 0xff, (size_t)np2 * sizeof(uint32_t), st);
        launch_compact_trail(rowflags, R, r, list, const_cast<uint32_t*>(cand), tiles, st);
        if (ev0) cudaEventRecord(ev0, st);
        k_phase3_list_w<T><<<grid, NTW, psm, st>>>(M, N, r, list, rowflags, R);
        if (ev1) cudaEventRecord(ev1, st);
        count_launches(2);
    }
    return cudaGetLastError();
}

template cudaError_t wide_round<float>(float*, int64_t, int32_t, int32_t, uint32_t*, const uint32_t*, uint32_t*, bool,
                                       int, unsigned long long*, cudaEvent_t, cudaEvent_t, cudaStream_t);
template cudaError_t wide_round<int32_t>(int32_t*, int64_t, int32_t, int32_t, uint32_t*, const uint32_t*, uint32_t*,
                                         bool, int, unsigned long long*, cudaEvent_t, cudaEvent_t, cudaStream_t);

}  // namespace spq
