// Table initialisation (Sec. 4: cell (i, j) holds wt(i, j) if the edge exists, else
// infinity, and 0 on the diagonal) and boundary-graph assembly (Algorithm 1: clique edges, BG).
#include <cuda_runtime.h>

#include "common.cuh"

namespace spq {

namespace {

template <typename T>
__device__ __forceinline__ void atomic_min_cell(T* p, T val);
template <>
__device__ __forceinline__ void atomic_min_cell<int32_t>(int32_t* p, int32_t val) {
    atomicMin(p, val);
}
template <>
__device__ __forceinline__ void atomic_min_cell<float>(float* p, float val) {
    // nonnegative floats (and +inf) order like their bit patterns as signed ints
    atomicMin(reinterpret_cast<int32_t*>(p), __float_as_int(val + 0.0f));
}

template <typename T>
__device__ __forceinline__ T weight_as(const void* w, int64_t e, bool f32w);
template <>
__device__ __forceinline__ int32_t weight_as<int32_t>(const void* w, int64_t e, bool f32w) {
    return f32w ? (int32_t)((const float*)w)[e] : ((const int32_t*)w)[e];
}
template <>
__device__ __forceinline__ float weight_as<float>(const void* w, int64_t e, bool f32w) {
    return f32w ? ((const float*)w)[e] : (float)((const int32_t*)w)[e];
}

// Fill each n x n block with infinity and a zero diagonal; one CTA per matrix at a time.
template <typename T>
__global__ void k_fill_blocks(T* __restrict__ base, const MatDesc* __restrict__ descs, int32_t nmat) {
    const T inf = Inf<T>::value();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int32_t mi = blockIdx.x; mi < nmat; mi += gridDim.x) {
        MatDesc d = descs[mi];
        T* M = base + d.off;
        const int32_t n4 = d.n / 4;
        for (int32_t i = warp; i < d.n; i += nwarps) {
            int4* row = reinterpret_cast<int4*>(M + (int64_t)i * d.n);
            for (int32_t j4 = lane; j4 < n4; j4 += 32) {
                T v[4] = {inf, inf, inf, inf};
                if ((i >> 2) == j4) v[i & 3] = T(0);
                row[j4] = make_int4(*(int*)&v[0], *(int*)&v[1], *(int*)&v[2], *(int*)&v[3]);
            }
        }
    }
}

// Intra-component edges: APSP(C)[local u][local v] = min(., w(u, v)).  With csize !=
// NULL only the components of at most max_n vertices and more than min_ld rows, at the
// positions `local` gives (a dissection order).
template <typename T>
__global__ void k_scatter_intra(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const void* __restrict__ w, bool f32w, const int32_t* __restrict__ part,
                                const int32_t* __restrict__ local, const MatDesc* __restrict__ descs,
                                T* __restrict__ apsp, const int32_t* __restrict__ csize = nullptr, int32_t max_n = 0,
                                int32_t min_ld = 0) {
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int32_t c = part[u];
    MatDesc d = descs[c];
    if (csize && (csize[c] > max_n || d.n <= min_ld)) return;
    T* row = apsp + d.off + (int64_t)local[u] * d.n;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        int32_t v = col[e];
        if (v == u || part[v] != c) continue;
        atomic_min_cell<T>(row + local[v], weight_as<T>(w, e, f32w));
    }
}

// D = infinity everywhere, 0 on the diagonal; rows strided over the grid.
template <typename T>
__global__ void k_bg_fill(T* __restrict__ D, int64_t N) {
    const T inf = Inf<T>::value();
    int4 pinf;
    {
        T v = inf;
        int x = *(int*)&v;
        pinf = make_int4(x, x, x, x);
    }
    for (int64_t i = blockIdx.x; i < N; i += gridDim.x) {
        int4* row = reinterpret_cast<int4*>(D + i * N);
        for (int64_t j4 = threadIdx.x; j4 < N / 4; j4 += blockDim.x) {
            int4 pk = pinf;
            if (i / 4 == j4) {
                T z = T(0);
                int zi = *(int*)&z;
                switch (i & 3) {
                    case 0: pk.x = zi; break;
                    case 1: pk.y = zi; break;
                    case 2: pk.z = zi; break;
                    default: pk.w = zi; break;
                }
            }
            row[j4] = pk;
        }
    }
}

// Clique edges of Algorithm 1: D[B(C), B(C)] = APSP(C)[0:|B|, 0:|B|] (the
// boundary vertices have the lowest local indices), at the slots' matrix positions.
// One CTA per component at a time.
template <typename T>
__global__ void k_bg_clique(const T* __restrict__ apsp, const MatDesc* __restrict__ descs,
                            const int32_t* __restrict__ nb, const int32_t* __restrict__ bg_off,
                            const int32_t* __restrict__ bgpos, int32_t k, T* __restrict__ D, int64_t N) {
    for (int32_t c = blockIdx.x; c < k; c += gridDim.x) {
        int32_t b = nb[c];
        if (b == 0) continue;
        MatDesc d = descs[c];
        const T* A = apsp + d.off;
        const int32_t* pos = bgpos + bg_off[c];
        for (int32_t i = threadIdx.y; i < b; i += blockDim.y) {
            T* row = D + (int64_t)pos[i] * N;
            for (int32_t j = threadIdx.x; j < b; j += blockDim.x) row[pos[j]] = A[(int64_t)i * d.n + j];
        }
    }
}

// G's edges between boundary vertices of different components (every such edge joins
// two boundary vertices by definition): D[bg(u)][bg(v)] = min(., w(u, v)).
template <typename T>
__global__ void k_bg_inter(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const void* __restrict__ w, bool f32w, const int32_t* __restrict__ part,
                           const int32_t* __restrict__ local, const int32_t* __restrict__ bg_off,
                           const int32_t* __restrict__ bgpos, T* __restrict__ D, int64_t N) {
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int32_t cu = part[u];
    int64_t bu = -1;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        int32_t v = col[e];
        int32_t cv = part[v];
        if (cv == cu) continue;
        if (bu < 0) bu = bgpos[bg_off[cu] + local[u]];
        int64_t bv = bgpos[bg_off[cv] + local[v]];
        atomic_min_cell<T>(D + bu * N + bv, weight_as<T>(w, e, f32w));
    }
}

// Float32 -> int32 in place, flagging any finite entry >= 2^24 (float32 values below
// 2^24 reached by the Floyd-Warshall updates are provably exact integers).
__device__ __forceinline__ int32_t to_i32(float x, bool& bad) {
    bad |= (x >= 16777216.0f) && !isinf(x);
    return isinf(x) ? SPQ_INF_I32 : (int32_t)x;
}
__global__ void k_check_convert(float4* __restrict__ a, int64_t count4, uint32_t* __restrict__ err) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 x = a[i];
        int4 y = make_int4(to_i32(x.x, bad), to_i32(x.y, bad), to_i32(x.z, bad), to_i32(x.w, bad));
        reinterpret_cast<int4*>(a)[i] = y;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrExact);
}

int sm_count() {
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
cudaError_t launch_fill_blocks(T* apsp, const MatDesc* descs, int32_t nmat, cudaStream_t st) {
    if (nmat <= 0) return cudaSuccess;
    int blocks = nmat < 65535 ? nmat : 65535;
    k_fill_blocks<T><<<blocks, 256, 0, st>>>(apsp, descs, nmat);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_intra(bool f32w, int32_t n, const int64_t* rp, const int32_t* col, const void* w,
                                 const int32_t* part, const int32_t* local, const MatDesc* descs, T* apsp,
                                 cudaStream_t st) {
    k_scatter_intra<T><<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, w, f32w, part, local, descs, apsp);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_intra_sel(bool f32w, int32_t n, const int64_t* rp, const int32_t* col, const void* w,
                                     const int32_t* part, const int32_t* pos, const MatDesc* descs,
                                     const int32_t* csize, int32_t max_n, int32_t min_ld, T* apsp, cudaStream_t st) {
    k_scatter_intra<T><<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, w, f32w, part, pos, descs, apsp, csize, max_n,
                                                          min_ld);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bg_fill(T* D, int64_t N, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    int64_t blocks = N < (int64_t)sm_count() * 16 ? N : (int64_t)sm_count() * 16;
    k_bg_fill<T><<<(unsigned)blocks, 256, 0, st>>>(D, N);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bg_clique(const T* apsp, const MatDesc* descs, const int32_t* nb, const int32_t* bg_off,
                             const int32_t* bgpos, int32_t k, T* D, int64_t N, cudaStream_t st) {
    if (k <= 0 || N <= 0) return cudaSuccess;
    int blocks = k < 65535 ? k : 65535;
    k_bg_clique<T><<<blocks, dim3(32, 8), 0, st>>>(apsp, descs, nb, bg_off, bgpos, k, D, N);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bg_inter(bool f32w, int32_t n, const int64_t* rp, const int32_t* col, const void* w,
                            const int32_t* part, const int32_t* local, const int32_t* bg_off, const int32_t* bgpos, T* D,
                            int64_t N, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_bg_inter<T><<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, w, f32w, part, local, bg_off, bgpos, D, N);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_convert(float* a, int64_t count, uint32_t* err, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int64_t c4 = count / 4;  // every table's element count is a multiple of 4
    int64_t blocks = (c4 + 255) / 256;
    int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_check_convert<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<float4*>(a), c4, err);
    count_launches(1);
    return cudaGetLastError();
}

#define SPQ_INST(T)                                                                                                \
    template cudaError_t launch_fill_blocks<T>(T*, const MatDesc*, int32_t, cudaStream_t);                         \
    template cudaError_t launch_scatter_intra<T>(bool, int32_t, const int64_t*, const int32_t*, const void*,       \
                                                 const int32_t*, const int32_t*, const MatDesc*, T*, cudaStream_t); \
    template cudaError_t launch_scatter_intra_sel<T>(bool, int32_t, const int64_t*, const int32_t*, const void*,   \
                                                     const int32_t*, const int32_t*, const MatDesc*, const int32_t*, \
                                                     int32_t, int32_t, T*, cudaStream_t);                          \
    template cudaError_t launch_bg_fill<T>(T*, int64_t, cudaStream_t);                                             \
    template cudaError_t launch_bg_clique<T>(const T*, const MatDesc*, const int32_t*, const int32_t*,           \
                                             const int32_t*, int32_t, T*, int64_t, cudaStream_t);                 \
    template cudaError_t launch_bg_inter<T>(bool, int32_t, const int64_t*, const int32_t*, const void*,            \
                                            const int32_t*, const int32_t*, const int32_t*, const int32_t*, T*,   \
                                            int64_t, cudaStream_t);
SPQ_INST(int32_t)
SPQ_INST(float)

}  // namespace spq
