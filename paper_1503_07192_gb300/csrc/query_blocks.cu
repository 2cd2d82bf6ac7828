// Grouped distance queries over the component-blocked copy of the boundary-graph matrix
// (Algorithm 2 for batches of pairs sorted by component pair).
//
// The block copy.  For components C1 <= C2 the |B(C1)| x |B(C2)| block dist_BG(B(C1),
// B(C2)) of the paper's Fig. 2 is stored contiguously, row-major, its rows padded to
// ld(C2) = |B(C2)| rounded up to 4 (padding columns infinite); the blocks are laid out row
// of blocks by row of blocks (C1 ascending, then C2 >= C1 ascending):
//   P[c]  = sum over c' < c of ld(c')                 (padded column start of c)
//   S[c1] = sum over c < c1 of |B(c)| * (P[k] - P[c]) (start of c1's row of blocks)
//   block (c1, c2) starts at S[c1] + |B(c1)| * (P[c2] - P[c1]).
// Every block start and row is a multiple of 16 bytes, so a block's rows are staged with
// 16-byte asynchronous copies.  This is the upper block-triangle of the matrix in the
// component order of the paper's Fig. 1: half the matrix.
//
// The queries.  Pairs are sorted by their unordered component pair (query.cu) and cut
// into items of at most 64 pairs sharing one block.  A persistent kernel (two CTAs of 256
// threads per SM) walks its items in a fixed stride; each item's block is staged in row
// chunks together with the chunk's piece of dist_C1(v1, .) for every pair, double
// buffered across chunk and item boundaries, so the copy of the next chunk (or of the
// next item's first chunk) overlaps the current one's arithmetic.  For an item of s pairs
// and a block of ld columns a thread owns 4 pairs x 4 columns of t(b2) = min over b1 of
// dist_C1(v1, b1) + D(b1, b2) in registers, for a share of the chunk's rows (the rows are
// split so that the (pairs/4) x (ld/4) tiles times the splits fill the 256 threads); at
// the item's end, min over its columns of t(b2) + dist_C2(b2, v2) is folded into a
// per-pair minimum in shared memory.  The minimum over row splits commutes with adding
// dist_C2(b2, v2) (x -> x + c is monotone, also in float arithmetic), so each answer is
// the same value the one-warp-per-pair form computes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "fw_tile.cuh"

namespace spq {

namespace {

constexpr int QB_TH = 256;
constexpr int QB_S = 8192;     // staged block elements per buffer (32 KB)
constexpr int QB_A = 4096;     // staged dist_C1 elements per buffer (pairs x chunk rows)
constexpr int QB_MAXP = 64;    // pairs per item
constexpr int QB_UMAX = 3;     // 4 x 4 tiles per thread

struct QItem {
    uint32_t start;  // first position in the sorted pairs
    int32_t count;   // pairs
    int32_t c1, c2;  // component pair, c1 <= c2
};

template <typename T>
struct QbSmem {
    T s[2][QB_S];                // block rows of the chunk, row-major, ld columns
    T a[2][QB_A];                // dist_C1(v1, rows of the chunk), one row of `chr` per pair
    int64_t a2off[2][QB_MAXP];   // per item parity: row of dist_C2(., v2) in the tables
    uint32_t qidx[2][QB_MAXP];   // the pair's position in the caller's arrays
    T init[2][QB_MAXP];          // the answer's starting value (same component, v == w)
    int32_t res[2][QB_MAXP];     // running minimum over the item's tiles (bit pattern)
};

// Largest pair count of an item on a block of ld columns: (pairs / 4) x (ld / 4) tiles
// must fit the CTA's threads with at most QB_UMAX tiles each.
__host__ __device__ __forceinline__ int32_t qb_pair_cap(int32_t ld) {
    const int32_t H = ld / 4 > 0 ? ld / 4 : 1;
    const int32_t g = (QB_TH * QB_UMAX) / H;
    const int32_t cap = 4 * (g < 1 ? 1 : g);
    return cap < QB_MAXP ? cap : QB_MAXP;
}

struct QbParams {
    int64_t off;             // block start in the copy
    int32_t nb1, ld2;        // block rows, padded columns
    int32_t chr, nch;        // rows per chunk (a multiple of 4), chunks
    int32_t G, H, Rs;        // pair groups, column groups, row splits
};

__device__ __forceinline__ QbParams qb_params(const QItem& it, const int32_t* __restrict__ nb,
                                              const int64_t* __restrict__ S, const int64_t* __restrict__ P) {
    QbParams p;
    p.nb1 = nb[it.c1];
    const int64_t P1 = P[it.c1], P2 = P[it.c2];
    p.ld2 = (int32_t)(P[it.c2 + 1] - P2);
    p.off = S[it.c1] + (int64_t)p.nb1 * (P2 - P1);
    const int32_t spad = (it.count + 3) & ~3;
    int32_t chr = QB_S / p.ld2;
    chr = min(chr, QB_A / spad);
    chr = min(chr, 64) & ~3;
    p.nch = (p.nb1 + chr - 1) / chr;
    p.chr = (((p.nb1 + p.nch - 1) / p.nch) + 3) & ~3;  // balanced chunks, at most chr rows
    p.nch = (p.nb1 + p.chr - 1) / p.chr;                // (no empty last chunk)
    p.G = spad / 4;
    p.H = p.ld2 / 4;
    const int32_t U = p.G * p.H;
    // row splits: the most threads busy, at most QB_UMAX tiles each
    int32_t best = 1, bneed = U, bnu = (U + QB_TH - 1) / QB_TH;
    for (int32_t r = 2; r <= 8 && 4 * r <= p.chr; ++r) {
        const int32_t need = U * r, nu = (need + QB_TH - 1) / QB_TH;
        if (nu > QB_UMAX) break;
        if ((int64_t)need * bnu > (int64_t)bneed * nu) {
            best = r;
            bneed = need;
            bnu = nu;
        }
    }
    p.Rs = best;
    return p;
}

template <typename T>
struct QbCtx {
    const T* apsp;
    const T* Dc;
    const int32_t* nb;
    const int64_t* S;
    const int64_t* P;
};

template <typename T>
__device__ __forceinline__ int32_t enc_min(T v);
template <>
__device__ __forceinline__ int32_t enc_min<int32_t>(int32_t v) {
    return v;
}
template <>
__device__ __forceinline__ int32_t enc_min<float>(float v) {
    return __float_as_int(v + 0.0f);  // non-negative floats order as their bit patterns (-0 -> +0)
}
template <typename T>
__device__ __forceinline__ T dec_min(int32_t b);
template <>
__device__ __forceinline__ int32_t dec_min<int32_t>(int32_t b) {
    return b;
}
template <>
__device__ __forceinline__ float dec_min<float>(int32_t b) {
    return __int_as_float(b);
}
template <typename T>
__device__ __forceinline__ int32_t res_reset() {
    return std::is_same<T, float>::value ? 0x7f800000 : 0x7fffffff;
}

__device__ __forceinline__ int32_t qb_addmin(int32_t a, int32_t b, int32_t t) { return __viaddmin_s32(a, b, t); }
__device__ __forceinline__ float qb_addmin(float a, float b, float t) { return fminf(t, a + b); }

// Queue the asynchronous copies of chunk ch of item it into buffer b: the block rows (all
// threads) and dist_C1(v1, rows) of pair tid (thread tid < count).  Rows of the last
// chunk past the block's end are set to infinity.
template <typename T>
__device__ __forceinline__ void qb_issue(QbSmem<T>& sm, int b, const QbCtx<T>& c, const QItem& it,
                                         const QbParams& p, int ch, int64_t a1off, int tid) {
    const int32_t r0 = ch * p.chr;
    const int32_t nrows = min(p.chr, p.nb1 - r0);
    const int32_t nr4 = (nrows + 3) & ~3;
    const T* src = c.Dc + p.off + (int64_t)r0 * p.ld2;
    const int32_t n16 = nrows * p.ld2 / 4;
    T* dst = sm.s[b];
    for (int32_t x = tid; x < n16; x += QB_TH) cp_async16(dst + 4 * x, src + 4 * x);
    const int32_t nfill = (nr4 - nrows) * p.ld2;
    const T inf = Inf<T>::value();
    for (int32_t x = tid; x < nfill; x += QB_TH) dst[nrows * p.ld2 + x] = inf;
    if (tid < it.count) {
        const T* a = c.apsp + a1off + r0;
        T* d = sm.a[b] + tid * p.chr;
        for (int32_t x = 0; x < nr4; x += 4) cp_async16(d + x, a + x);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(QB_TH, 2)
    k_qb_blocks(const QbCtx<T> c, const QItem* __restrict__ items, const uint32_t* __restrict__ nitems_p,
                const longlong2* __restrict__ rows, const T* __restrict__ init, const uint32_t* __restrict__ idx,
                void* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char qb_raw[];
    QbSmem<T>& sm = *reinterpret_cast<QbSmem<T>*>(qb_raw);
    const int tid = threadIdx.x;
    const uint32_t nitems = *nitems_p;
    const uint32_t G = gridDim.x;
    uint32_t it = blockIdx.x;
    if (it >= nitems) return;
    if (tid < 2 * QB_MAXP) sm.res[tid / QB_MAXP][tid % QB_MAXP] = res_reset<T>();
    const T inf = Inf<T>::value();
    // the current item, the next one (with its per-pair records) and the one after that
    // (its record only): loads are issued an item ahead of their use
    QItem cur = items[it];
    longlong2 crow = tid < cur.count ? rows[cur.start + tid] : make_longlong2(0, 0);
    if (tid < cur.count) {
        sm.a2off[0][tid] = crow.y;
        sm.init[0][tid] = init[cur.start + tid];
        sm.qidx[0][tid] = idx[cur.start + tid];
    }
    uint32_t itn = it + G;
    QItem nxt = itn < nitems ? items[itn] : QItem{0, 0, 0, 0};
    longlong2 nrow = tid < nxt.count ? rows[nxt.start + tid] : make_longlong2(0, 0);
    T ninit = tid < nxt.count ? init[nxt.start + tid] : T(0);
    uint32_t nidx = tid < nxt.count ? idx[nxt.start + tid] : 0u;
    QItem nn = itn + G < nitems ? items[itn + G] : QItem{0, 0, 0, 0};

    QbParams p = qb_params(cur, c.nb, c.S, c.P);
    int ch = 0, b = 0, par = 0;
    qb_issue<T>(sm, 0, c, cur, p, 0, crow.x, tid);
    cp_async_commit();
    T acc[QB_UMAX][4][4];
    for (;;) {
        const bool next_same = ch + 1 < p.nch;
        const bool has_next = next_same || itn < nitems;
        if (next_same) {
            qb_issue<T>(sm, b ^ 1, c, cur, p, ch + 1, crow.x, tid);
        } else if (has_next) {
            // the next item's first chunk; its epilogue records go to the other parity
            // (last read by the item before this one, behind a barrier since)
            if (tid < nxt.count) {
                sm.a2off[par ^ 1][tid] = nrow.y;
                sm.init[par ^ 1][tid] = ninit;
                sm.qidx[par ^ 1][tid] = nidx;
            }
            qb_issue<T>(sm, b ^ 1, c, nxt, qb_params(nxt, c.nb, c.S, c.P), 0, nrow.x, tid);
        }
        if (has_next) {
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // ---- the chunk's arithmetic ----
        const int32_t r0 = ch * p.chr;
        const int32_t nq = (min(p.chr, p.nb1 - r0) + 3) >> 2;
        const int32_t U = p.G * p.H, need = U * p.Rs;
        if (ch == 0) {
#pragma unroll
            for (int k = 0; k < QB_UMAX; ++k)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[k][i][e] = inf;
        }
#pragma unroll
        for (int k = 0; k < QB_UMAX; ++k) {
            const int32_t x = tid + k * QB_TH;
            if (x < need) {
                const int32_t r = x / U, rest = x - r * U;
                const int32_t g = rest / p.H, h = rest - g * p.H;
                const int32_t q0 = r * nq / p.Rs, q1 = (r + 1) * nq / p.Rs;
                const T* ap = sm.a[b] + 4 * g * p.chr;
                const T* sp = sm.s[b] + 4 * h;
#pragma unroll 1
                for (int32_t qq = q0; qq < q1; ++qq) {
                    T av[4][4], sv[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int4 v = *reinterpret_cast<const int4*>(ap + i * p.chr + 4 * qq);
                        av[i][0] = *reinterpret_cast<const T*>(&v.x);
                        av[i][1] = *reinterpret_cast<const T*>(&v.y);
                        av[i][2] = *reinterpret_cast<const T*>(&v.z);
                        av[i][3] = *reinterpret_cast<const T*>(&v.w);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int4 v = *reinterpret_cast<const int4*>(sp + (4 * qq + j) * p.ld2);
                        sv[j][0] = *reinterpret_cast<const T*>(&v.x);
                        sv[j][1] = *reinterpret_cast<const T*>(&v.y);
                        sv[j][2] = *reinterpret_cast<const T*>(&v.z);
                        sv[j][3] = *reinterpret_cast<const T*>(&v.w);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[k][i][e] = qb_addmin(av[i][j], sv[j][e], acc[k][i][e]);
                }
            }
        }
        if (!next_same) {
            // ---- the item's end: + dist_C2(b2, v2), min over the columns, per pair ----
#pragma unroll
            for (int k = 0; k < QB_UMAX; ++k) {
                const int32_t x = tid + k * QB_TH;
                if (x < need) {
                    const int32_t rest = x % U;
                    const int32_t g = rest / p.H, h = rest - g * p.H;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int32_t u = 4 * g + i;
                        if (u < cur.count) {
                            const int4 cv = __ldg(reinterpret_cast<const int4*>(c.apsp + sm.a2off[par][u] + 4 * h));
                            const T c4[4] = {*reinterpret_cast<const T*>(&cv.x), *reinterpret_cast<const T*>(&cv.y),
                                             *reinterpret_cast<const T*>(&cv.z), *reinterpret_cast<const T*>(&cv.w)};
                            T v = acc[k][i][0] + c4[0];
#pragma unroll
                            for (int e = 1; e < 4; ++e) {
                                const T y = acc[k][i][e] + c4[e];
                                v = y < v ? y : v;
                            }
                            atomicMin(&sm.res[par][u], enc_min<T>(v));
                        }
                    }
                }
            }
            __syncthreads();
            if (tid < cur.count) {
                T y = dec_min<T>(sm.res[par][tid]);
                const T z = sm.init[par][tid];
                y = z < y ? z : y;
                sm.res[par][tid] = res_reset<T>();
                const uint32_t qi = sm.qidx[par][tid];
                if (MODE == 2)
                    ((float*)out)[qi] = (float)y;
                else
                    ((int32_t*)out)[qi] = (int32_t)min((int32_t)y, (int32_t)SPQ_INF_I32);
            }
        }
        __syncthreads();  // buffer b is free for the next issue
        if (!has_next) break;
        if (next_same) {
            ++ch;
        } else {
            it = itn;
            itn = it + G;
            cur = nxt;
            crow = nrow;
            p = qb_params(cur, c.nb, c.S, c.P);
            ch = 0;
            par ^= 1;
            nxt = nn;
            nrow = tid < nxt.count ? rows[nxt.start + tid] : make_longlong2(0, 0);
            ninit = tid < nxt.count ? init[nxt.start + tid] : T(0);
            nidx = tid < nxt.count ? idx[nxt.start + tid] : 0u;
            nn = itn + G < nitems ? items[itn + G] : QItem{0, 0, 0, 0};
        }
        b ^= 1;
    }
}

// Per sorted position: the pair oriented so that v1 lies in the lower component, the
// table rows of dist_C1(v1, .) and dist_C2(., v2), and the starting value of its answer:
// 0 if v1 = v2, dist_C1(v1, v2) if both lie in one component, else infinity.  Pairs with
// an id out of range (sorted last) are answered here (-1 / NaN) and mark the handle; so
// are pairs whose block is empty (a component without boundary vertices): their answer is
// the starting value.
template <typename T, int MODE>
__global__ void k_qb_prep(const QueryCtx<T> ctx, const int2* __restrict__ pairs, const uint32_t* __restrict__ keys,
                          const uint32_t* __restrict__ idx, int64_t q, uint32_t k, longlong2* __restrict__ rows,
                          T* __restrict__ init, void* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= q) return;
    const uint32_t key = keys[p], qi = idx[p];
    if (key >= k * k) {
        if (MODE == 2)
            ((float*)out)[qi] = __int_as_float(0x7fc00000);
        else
            ((int32_t*)out)[qi] = -1;
        atomicOr(ctx.err, kErrPair);
        return;
    }
    const int32_t c1 = (int32_t)(key / k), c2 = (int32_t)(key % k);
    int2 pr = pairs[qi];
    if (ctx.comp[pr.x] != c1) pr = make_int2(pr.y, pr.x);
    const MatDesc d1 = ctx.descs[c1], d2 = ctx.descs[c2];
    const int64_t a1 = d1.off + (int64_t)ctx.local[pr.x] * d1.n;
    const int64_t a2 = d2.off + (int64_t)ctx.local[pr.y] * d2.n;
    rows[p] = make_longlong2(a1, a2);
    T z = Inf<T>::value();
    if (pr.x == pr.y)
        z = T(0);
    else if (c1 == c2)
        z = ctx.apsp[a1 + ctx.local[pr.y]];
    init[p] = z;
    if (ctx.nb[c1] == 0 || ctx.nb[c2] == 0) {
        if (MODE == 2)
            ((float*)out)[qi] = (float)z;
        else
            ((int32_t*)out)[qi] = (int32_t)z;
    }
}

// Items: every run of one component pair (a nonempty block no wider than the copy's
// limit) cut into nearly equal pieces of at most qb_pair_cap(ld) pairs; the order of the
// item list is arbitrary.
__global__ void k_qb_items(const uint32_t* __restrict__ keys, int64_t q, uint32_t k, const int32_t* __restrict__ nb,
                           const int64_t* __restrict__ P, int32_t max_ld, QItem* __restrict__ items,
                           uint32_t* __restrict__ nitems, unsigned long long* __restrict__ stats) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= q) return;
    const uint32_t key = keys[p];
    if (key >= k * k || (p > 0 && keys[p - 1] == key)) return;
    const int32_t c1 = (int32_t)(key / k), c2 = (int32_t)(key % k);
    const int32_t ld2 = (int32_t)(P[c2 + 1] - P[c2]);
    if (nb[c1] == 0 || nb[c2] == 0 || ld2 > max_ld) return;
    int64_t lo = p + 1, hi = q;  // the run's end: first position with a larger key
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] == key)
            lo = mid + 1;
        else
            hi = mid;
    }
    const int64_t n = lo - p;
    const int64_t cap = qb_pair_cap(ld2);
    const int64_t pieces = (n + cap - 1) / cap;
    const uint32_t base = atomicAdd(nitems, (uint32_t)pieces);
    if (stats) {
        // algorithmic work of the run: |B1| x |B2| updates per pair; bytes: each item's
        // block once, per pair its two table rows, the pair, its position and its answer
        const int64_t nb1 = nb[c1], nb2 = nb[c2];
        atomicAdd(&stats[0], (unsigned long long)(n * nb1 * nb2));
        atomicAdd(&stats[1], (unsigned long long)(4 * pieces * nb1 * ld2 + n * (4 * (((nb1 + 3) & ~3) + ld2) + 16)));
    }
    for (int64_t i = 0; i < pieces; ++i) {
        const int64_t s0 = p + i * n / pieces, s1 = p + (i + 1) * n / pieces;
        items[base + i] = QItem{(uint32_t)s0, (int32_t)(s1 - s0), c1, c2};
    }
}

// The block copy from the boundary-graph matrix (any order of its rows, reached through
// bgpos): one CTA per boundary slot s of component c1, writing row s - bg_off[c1] of every
// block (c1, c2 >= c1); pcomp[u] is the component of padded column u.
template <typename T>
__global__ void __launch_bounds__(256) k_build_dc(const T* __restrict__ D, int64_t N, const int32_t* __restrict__ bgpos,
                                                  const int32_t* __restrict__ bg_off, const int32_t* __restrict__ nb,
                                                  const int64_t* __restrict__ S, const int64_t* __restrict__ P,
                                                  const int32_t* __restrict__ pcomp, int32_t k, int64_t nbg,
                                                  T* __restrict__ Dc) {
    const T inf = Inf<T>::value();
    const int64_t Pk = P[k];
    for (int64_t s = blockIdx.x; s < nbg; s += gridDim.x) {
        int32_t lo = 0, hi = k;  // the last component whose first slot is <= s
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (bg_off[mid] <= s) lo = mid; else hi = mid;
        }
        const int32_t c1 = lo;
        const int64_t b1 = s - bg_off[c1];
        const int64_t nb1 = nb[c1], P1 = P[c1];
        const T* drow = D + (int64_t)bgpos[s] * N;
        const int64_t base = S[c1];
        for (int64_t u = P1 + threadIdx.x; u < Pk; u += blockDim.x) {
            const int32_t c2 = pcomp[u];
            const int64_t P2 = P[c2];
            const int64_t j = u - P2, ld2 = P[c2 + 1] - P2;
            const T v = j < nb[c2] ? drow[bgpos[bg_off[c2] + j]] : inf;
            Dc[base + nb1 * (P2 - P1) + b1 * ld2 + j] = v;
        }
    }
}

__global__ void k_pcomp(const int64_t* __restrict__ P, int32_t k, int32_t* __restrict__ pcomp) {
    const int32_t c = blockIdx.x * blockDim.y + threadIdx.y;
    if (c >= k) return;
    for (int64_t u = P[c] + threadIdx.x; u < P[c + 1]; u += blockDim.x) pcomp[u] = c;
}

int qb_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename T, int MODE>
cudaError_t launch_blocks_kernel(const QbCtx<T>& c, const QItem* items, const uint32_t* nitems, const longlong2* rows,
                                 const T* init, const uint32_t* idx, void* out, int64_t q, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    const size_t smem = sizeof(QbSmem<T>);
    if (!attr.load()) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_qb_blocks<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr.store(true);
    }
    int64_t grid = (int64_t)qb_sms() * 2;
    if (grid > q) grid = q;  // at most q items
    k_qb_blocks<T, MODE><<<(unsigned)grid, QB_TH, smem, st>>>(c, items, nitems, rows, init, idx, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int32_t query_blocks_max_ld() { return 2048; }

int64_t query_blocks_scratch_words(int64_t q) {
    // rows (4 words per pair), starting values (1), items (4), the item counter (+ 4 for
    // 16-byte alignment of what follows a word count that is not a multiple of 4)
    return 9 * q + 8;
}

void dc_layout(const std::vector<int32_t>& nb, std::vector<int64_t>* S, std::vector<int64_t>* P, int64_t* elems,
               int32_t* max_ld) {
    const int32_t k = (int32_t)nb.size();
    P->assign((size_t)k + 1, 0);
    S->assign((size_t)k, 0);
    int32_t mx = 0;
    for (int32_t c = 0; c < k; ++c) {
        const int32_t ld = (int32_t)round_up(nb[c], 4);
        (*P)[c + 1] = (*P)[c] + ld;
        mx = std::max(mx, ld);
    }
    int64_t acc = 0;
    for (int32_t c = 0; c < k; ++c) {
        (*S)[c] = acc;
        acc += (int64_t)nb[c] * ((*P)[k] - (*P)[c]);
    }
    *elems = acc;
    *max_ld = mx;
}

template <typename T>
cudaError_t launch_build_dc(const T* D, int64_t N, const int32_t* bgpos, const int32_t* bg_off, const int32_t* nb,
                            const int64_t* S, const int64_t* P, int32_t k, int64_t nbg, int64_t Pk, T* Dc,
                            cudaStream_t st) {
    if (nbg <= 0) return cudaSuccess;
    int32_t* pcomp = nullptr;
    cudaError_t e = scratch_alloc((void**)&pcomp, (size_t)(Pk > 0 ? Pk : 1) * 4, st);
    if (e != cudaSuccess) return e;
    k_pcomp<<<(unsigned)((k + 7) / 8), dim3(32, 8), 0, st>>>(P, k, pcomp);
    const int64_t grid = std::min<int64_t>(nbg, (int64_t)qb_sms() * 16);
    k_build_dc<T><<<(unsigned)grid, 256, 0, st>>>(D, N, bgpos, bg_off, nb, S, P, pcomp, k, nbg, Dc);
    count_launches(2);
    e = cudaGetLastError();
    cudaFreeAsync(pcomp, st);
    return e;
}

template <typename T>
cudaError_t launch_query_blocks(const QueryCtx<T>& ctx, const int32_t* pairs, int64_t q, void* out, bool out_f32,
                                uint32_t k, const uint32_t* keys, const uint32_t* idx, uint32_t* scratch,
                                cudaStream_t st) {
    // scratch: rows (16-byte aligned) | starting values | items | counter
    uint32_t* base = (uint32_t*)(((uintptr_t)scratch + 15) & ~(uintptr_t)15);
    longlong2* rows = reinterpret_cast<longlong2*>(base);
    T* init = reinterpret_cast<T*>(base + 4 * q);
    QItem* items = reinterpret_cast<QItem*>(base + ((5 * q + 3) & ~(int64_t)3));
    uint32_t* nitems = base + ((5 * q + 3) & ~(int64_t)3) + 4 * q;
    const int2* p2 = reinterpret_cast<const int2*>(pairs);
    const bool mode_f32 = out_f32 || !std::is_same<T, int32_t>::value;
    cudaError_t e = cudaMemsetAsync(nitems, 0, 4, st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((q + 255) / 256);
    if (mode_f32)
        k_qb_prep<T, 2><<<g, 256, 0, st>>>(ctx, p2, keys, idx, q, k, rows, init, out);
    else
        k_qb_prep<T, 0><<<g, 256, 0, st>>>(ctx, p2, keys, idx, q, k, rows, init, out);
    // profiling (not inside a graph capture): the kernel's events and algorithmic counts
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool prof = ctx.qev && ctx.qstats && cap == cudaStreamCaptureStatusNone;
    if (prof && (e = cudaMemsetAsync(ctx.qstats, 0, 16, st)) != cudaSuccess) return e;
    k_qb_items<<<g, 256, 0, st>>>(keys, q, k, ctx.nb, ctx.dcP, query_blocks_max_ld(), items, nitems,
                                  prof ? ctx.qstats : nullptr);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const QbCtx<T> c{ctx.apsp, ctx.Dc, ctx.nb, ctx.dcS, ctx.dcP};
    if (prof && (e = cudaEventRecord(ctx.qev[0], st)) != cudaSuccess) return e;
    e = mode_f32 ? launch_blocks_kernel<T, 2>(c, items, nitems, rows, init, idx, out, q, st)
                 : launch_blocks_kernel<T, 0>(c, items, nitems, rows, init, idx, out, q, st);
    if (e == cudaSuccess && prof) e = cudaEventRecord(ctx.qev[1], st);
    return e;
}

template cudaError_t launch_build_dc<int32_t>(const int32_t*, int64_t, const int32_t*, const int32_t*, const int32_t*,
                                              const int64_t*, const int64_t*, int32_t, int64_t, int64_t, int32_t*,
                                              cudaStream_t);
template cudaError_t launch_build_dc<float>(const float*, int64_t, const int32_t*, const int32_t*, const int32_t*,
                                            const int64_t*, const int64_t*, int32_t, int64_t, int64_t, float*,
                                            cudaStream_t);
template cudaError_t launch_query_blocks<int32_t>(const QueryCtx<int32_t>&, const int32_t*, int64_t, void*, bool,
                                                  uint32_t, const uint32_t*, const uint32_t*, uint32_t*, cudaStream_t);
template cudaError_t launch_query_blocks<float>(const QueryCtx<float>&, const int32_t*, int64_t, void*, bool, uint32_t,
                                                const uint32_t*, const uint32_t*, uint32_t*, cudaStream_t);

}  // namespace spq
