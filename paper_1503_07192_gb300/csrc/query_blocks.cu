// Grouped distance queries (Algorithm 2 for batches of pairs sorted by component pair),
// staging each boundary-graph block in shared memory with asynchronous copies.
//
// Pairs are sorted by their unordered component pair (query.cu) and cut into items of at
// most 64 pairs sharing one block dist_BG(B(C1), B(C2)) (the paper's Fig. 2: the block of
// the boundary matrix whose rows are C1's boundary slots and columns C2's).  A persistent
// kernel (three CTAs of 256 threads per SM) walks its items in a fixed stride; each item's
// block is staged in row chunks, gathered from the matrix through the slots' positions with
// 4-byte asynchronous copies (a component's slots form a few long runs in the matrix
// order, so a warp's consecutive columns mostly read consecutive addresses), together with
// the chunk's piece of dist_C1(v1, .) for every pair (16-byte copies), double buffered
// across chunk and item boundaries: the copy of the next chunk (or of the next item's first
// chunk) overlaps the current one's arithmetic.  For an item of s pairs and a block of ld
// columns (|B2| rounded up to 4) a thread owns 4 pairs x 4 columns of
// t(b2) = min over b1 of dist_C1(v1, b1) + D(b1, b2) in registers, for a share of the
// chunk's rows (the rows are split so that the (pairs/4) x (ld/4) tiles times the splits
// fill the 256 threads); at the item's end, min over its columns of t(b2) + dist_C2(b2, v2)
// is folded into a per-pair minimum in shared memory.  The minimum over row splits
// commutes with adding dist_C2(b2, v2) (x -> x + c is monotone, also in float arithmetic),
// so each answer is the same value the one-warp-per-pair form computes.  Blocks with more
// than 512 rows or columns are left to the gathering kernel of query.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "fw_tile.cuh"

namespace spq {

namespace {

constexpr int QB_TH = 256;
constexpr int QB_S = 4096;     // staged block elements per buffer (16 KB)
constexpr int QB_A = 2048;     // staged dist_C1 elements per buffer (pairs x chunk rows)
constexpr int QB_MAXP = 64;    // pairs per item
constexpr int QB_UMAX = 2;     // 4 x 4 tiles per thread
constexpr int QB_CTAS = 3;     // CTAs per SM
constexpr int QB_PMAX = 512;   // widest block side (rows or columns) staged here
constexpr int QB_PREG = (2 * QB_PMAX) / (2 * QB_TH);  // prefetched positions per thread and side

// One item: its pairs (a run of sorted positions) and the shape of its staged work, set
// once by the item builder.
struct QItem {
    uint32_t start;          // first position in the sorted pairs
    int32_t count;           // pairs (at most QB_MAXP)
    int32_t c1, c2;          // component pair, c1 <= c2
    int32_t nb1, ld2, nb2;   // block rows, padded columns, columns
    int32_t chr, nch;        // rows per chunk (a multiple of 4), chunks
    int32_t G, H, Rs;        // pair groups (of 4), column groups (of 4), row splits
};
static_assert(sizeof(QItem) == 48, "item records are 12 words");

template <typename T>
struct QbSmem {
    T s[2][QB_S];                // block rows of the chunk, row-major, ld columns
    T a[2][QB_A];                // dist_C1(v1, rows of the chunk), one row of `chr` per pair
    int32_t pos1[2][QB_PMAX];    // per item parity: matrix rows of C1's slots
    int32_t pos2[2][QB_PMAX];    //                  matrix columns of C2's slots
    int64_t a1off[2][QB_MAXP];   //                  row of dist_C1(v1, .) in the tables
    int64_t a2off[2][QB_MAXP];   //                  row of dist_C2(., v2)
    uint32_t qidx[2][QB_MAXP];   //                  the pair's position in the caller's arrays
    T init[2][QB_MAXP];          //                  the answer's starting value
    int32_t res[2][QB_MAXP];     //                  running minimum (bit pattern)
    QItem item[4];               // the records of items m .. m + 3 (item m in slot m & 3)
};

// Largest pair count of an item on a block of ld columns: (pairs / 4) x (ld / 4) tiles
// must fit the CTA's threads with at most QB_UMAX tiles each.
__host__ __device__ __forceinline__ int32_t qb_pair_cap(int32_t ld) {
    const int32_t H = ld / 4 > 0 ? ld / 4 : 1;
    const int32_t g = (QB_TH * QB_UMAX) / H;
    const int32_t cap = 4 * (g < 1 ? 1 : g);
    return cap < QB_MAXP ? cap : QB_MAXP;
}

// The item of `count` pairs from `start` on block (c1, c2): rows staged in balanced chunks
// of at most 64 rows (a multiple of 4) that fit the buffers, and the row splits that keep
// the most threads busy with at most QB_UMAX tiles of 4 pairs x 4 columns each.
__device__ __forceinline__ QItem qb_make_item(uint32_t start, int32_t count, int32_t c1, int32_t c2,
                                              const int32_t* __restrict__ nb) {
    QItem p;
    p.start = start;
    p.count = count;
    p.c1 = c1;
    p.c2 = c2;
    p.nb1 = nb[c1];
    p.nb2 = nb[c2];
    p.ld2 = (p.nb2 + 3) & ~3;
    const int32_t spad = (count + 3) & ~3;
    int32_t chr = QB_S / p.ld2;
    chr = min(chr, QB_A / spad);
    chr = min(chr, 64) & ~3;
    p.nch = (p.nb1 + chr - 1) / chr;
    p.chr = (((p.nb1 + p.nch - 1) / p.nch) + 3) & ~3;  // balanced chunks, at most chr rows
    p.nch = (p.nb1 + p.chr - 1) / p.chr;                // (no empty last chunk)
    p.G = spad / 4;
    p.H = p.ld2 / 4;
    const int32_t U = p.G * p.H;
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

// A thread's tiles of an item: tile k is x = tid + k * QB_TH of the (row split, pair group,
// column group) space, packed as r << 28 | g << 20 | h (h < 2^20), or -1 past its end.
__device__ __forceinline__ void qb_units(const QItem& p, int tid, int32_t (&u)[QB_UMAX]) {
    const int32_t U = p.G * p.H, need = U * p.Rs;
#pragma unroll
    for (int k = 0; k < QB_UMAX; ++k) {
        const int32_t x = tid + k * QB_TH;
        if (x < need) {
            const int32_t r = x / U, rest = x - r * U, g = rest / p.H, h = rest - g * p.H;
            u[k] = (r << 28) | (g << 20) | h;
        } else {
            u[k] = -1;
        }
    }
}

template <typename T>
struct QbCtx {
    const T* apsp;
    const T* D;
    int64_t N;
    const int32_t* bgpos;
    const int32_t* bg_off;
};

// An item's slot positions (matrix rows of C1's slots, columns of C2's) into parity pp.
template <typename T>
__device__ __forceinline__ void qb_load_pos(QbSmem<T>& sm, int pp, const QbCtx<T>& c, const QItem& p, int tid) {
    if (p.count == 0) return;
    for (int32_t i = tid; i < p.nb1; i += QB_TH) sm.pos1[pp][i] = c.bgpos[c.bg_off[p.c1] + i];
    for (int32_t i = tid; i < p.nb2; i += QB_TH) sm.pos2[pp][i] = c.bgpos[c.bg_off[p.c2] + i];
}
// The same in two steps: loads into registers (issued an item ahead of their use) ...
template <typename T>
__device__ __forceinline__ void qb_fetch_pos(const QbCtx<T>& c, const QItem& p, int tid, int32_t (&r1)[QB_PREG],
                                             int32_t (&r2)[QB_PREG]) {
#pragma unroll
    for (int u = 0; u < QB_PREG; ++u) {
        const int32_t i = tid + u * QB_TH;
        r1[u] = (p.count > 0 && i < p.nb1) ? c.bgpos[c.bg_off[p.c1] + i] : 0;
        r2[u] = (p.count > 0 && i < p.nb2) ? c.bgpos[c.bg_off[p.c2] + i] : 0;
    }
}
// ... and the stores into parity pp.
template <typename T>
__device__ __forceinline__ void qb_store_pos(QbSmem<T>& sm, int pp, const QItem& p, int tid,
                                             const int32_t (&r1)[QB_PREG], const int32_t (&r2)[QB_PREG]) {
#pragma unroll
    for (int u = 0; u < QB_PREG; ++u) {
        const int32_t i = tid + u * QB_TH;
        if (p.count > 0 && i < p.nb1) sm.pos1[pp][i] = r1[u];
        if (p.count > 0 && i < p.nb2) sm.pos2[pp][i] = r2[u];
    }
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}

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

// Queue the asynchronous copies of chunk ch of item p (per-item records in parity pp)
// into buffer b: the block rows gathered from the matrix (warps over rows, lanes over
// columns) and the pieces dist_C1(v1, rows) of every pair, spread over all threads.
// Padding columns past |B2| and rows of the last chunk past the block's end are set to
// infinity.
template <typename T>
__device__ __forceinline__ void qb_issue(QbSmem<T>& sm, int b, int pp, const QbCtx<T>& c, const QItem& p, int ch,
                                         int tid) {
    const int32_t r0 = ch * p.chr;
    const int32_t nrows = min(p.chr, p.nb1 - r0);
    const int32_t nr4 = (nrows + 3) & ~3;
    const int warp = tid >> 5, lane = tid & 31;
    T* dst = sm.s[b];
    const T inf = Inf<T>::value();
    if (p.nb2 <= 128) {  // (the usual case: a lane's columns in registers)
        int32_t col[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) col[k] = lane + 32 * k < p.nb2 ? sm.pos2[pp][lane + 32 * k] : 0;
        for (int32_t ii = warp; ii < nr4; ii += QB_TH / 32) {
            T* d = dst + ii * p.ld2;
            if (ii < nrows) {
                const T* row = c.D + (int64_t)sm.pos1[pp][r0 + ii] * c.N;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (lane + 32 * k < p.nb2) cp_async4(d + lane + 32 * k, row + col[k]);
                if (p.nb2 + lane < p.ld2) d[p.nb2 + lane] = inf;
            } else {
                for (int32_t jj = lane; jj < p.ld2; jj += 32) d[jj] = inf;
            }
        }
    } else {
        for (int32_t ii = warp; ii < nr4; ii += QB_TH / 32) {
            T* d = dst + ii * p.ld2;
            if (ii < nrows) {
                const T* row = c.D + (int64_t)sm.pos1[pp][r0 + ii] * c.N;
                for (int32_t jj = lane; jj < p.nb2; jj += 32) cp_async4(d + jj, row + sm.pos2[pp][jj]);
                if (p.nb2 + lane < p.ld2) d[p.nb2 + lane] = inf;
            } else {
                for (int32_t jj = lane; jj < p.ld2; jj += 32) d[jj] = inf;
            }
        }
    }
    const int32_t nq4 = nr4 >> 2;
    for (int32_t x = tid; x < p.count * nq4; x += QB_TH) {
        const int32_t u = x / nq4, q4 = x - u * nq4;
        cp_async16(sm.a[b] + u * p.chr + 4 * q4, c.apsp + sm.a1off[pp][u] + r0 + 4 * q4);
    }
}

// ENC (int32 tables whose finite entries are all below 2^24): the int32 values are read
// as the bit patterns of floats (m -> m x 2^-149, subnormal or in the lowest normal
// binade): float addition of two of them is exact integer addition of the patterns while
// the sum stays below 2^24, float order is integer order, and a sum at or above 2^24 never
// rounds below it; SPQ_INF_I32 (2^29) reads as 2^-63, far above.  Packed f32x2 adds and
// three-input mins then do the updates.  An answer below 2^24 is exact (its minimising
// sum has no term at or above 2^24); an answer at or above it (a long or an unreachable
// pair) is listed in fb and recomputed exactly in int32 by k_qb_fallback.  No subnormal
// is flushed: the kernel is built without fast math or .ftz.
template <typename T, int MODE, bool ENC>
__global__ void __launch_bounds__(QB_TH, QB_CTAS)
    k_qb_blocks(const QbCtx<T> c, const QItem* __restrict__ items, const uint32_t* __restrict__ nitems_p,
                const longlong2* __restrict__ rows, const T* __restrict__ init, const uint32_t* __restrict__ idx,
                void* __restrict__ out, uint32_t* __restrict__ fb, uint32_t* __restrict__ nfb) {
    using CT = typename std::conditional<ENC, float, T>::type;  // the arithmetic's type
    extern __shared__ __align__(16) unsigned char qb_raw[];
    QbSmem<T>& sm = *reinterpret_cast<QbSmem<T>*>(qb_raw);
    const int tid = threadIdx.x;
    const uint32_t nitems = *nitems_p;
    const uint32_t G = gridDim.x;
    if (blockIdx.x >= nitems) return;
    // the CTA's items are m = 0, 1, ...: item id blockIdx.x + m * G, record in slot m & 3,
    // per-pair records and slot positions in parity m & 1.  After the switch to item m,
    // shared memory holds the records of items m .. m + 3 and the per-pair records and
    // positions of m and m + 1; registers hold those of m + 2 (loaded an item ahead).
    auto item_at = [&](uint32_t m) { const uint32_t i = blockIdx.x + m * G; return i < nitems ? items[i] : QItem{}; };
    if (tid < 4) sm.item[tid] = item_at(tid);
    if (tid < 2 * QB_MAXP) sm.res[tid / QB_MAXP][tid % QB_MAXP] = res_reset<CT>();
    __syncthreads();
    for (int pp = 0; pp < 2; ++pp) {
        const QItem& p = sm.item[pp];
        if (tid < p.count) {
            const longlong2 r = rows[p.start + tid];
            sm.a1off[pp][tid] = r.x;
            sm.a2off[pp][tid] = r.y;
            sm.init[pp][tid] = init[p.start + tid];
            sm.qidx[pp][tid] = idx[p.start + tid];
        }
        qb_load_pos(sm, pp, c, p, tid);
    }
    longlong2 nrow;
    T ninit;
    uint32_t nidx;
    int32_t pr1[QB_PREG], pr2[QB_PREG];
    {
        const QItem& p = sm.item[2];
        nrow = tid < p.count ? rows[p.start + tid] : make_longlong2(0, 0);
        ninit = tid < p.count ? init[p.start + tid] : T(0);
        nidx = tid < p.count ? idx[p.start + tid] : 0u;
        qb_fetch_pos(c, p, tid, pr1, pr2);
    }
    __syncthreads();
    const CT inf = ENC ? __int_as_float(SPQ_INF_I32) : (CT)Inf<T>::value();

    uint32_t m = 0;
    int32_t unit[QB_UMAX];
    qb_units(sm.item[0], tid, unit);
    int ch = 0, b = 0;
    qb_issue<T>(sm, 0, 0, c, sm.item[0], 0, tid);
    cp_async_commit();
    CT acc[QB_UMAX][4][4];
    for (;;) {
        const QItem& cur = sm.item[m & 3];
        const int par = m & 1;
        const int32_t nch = cur.nch, chr = cur.chr, ld2 = cur.ld2, Rs = cur.Rs;
        const bool next_same = ch + 1 < nch;
        const bool has_next = next_same || sm.item[(m + 1) & 3].count > 0;
        if (next_same)
            qb_issue<T>(sm, b ^ 1, par, c, cur, ch + 1, tid);
        else if (has_next)
            qb_issue<T>(sm, b ^ 1, par ^ 1, c, sm.item[(m + 1) & 3], 0, tid);
        if (has_next) {
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // ---- the chunk's arithmetic: row split r takes the quads r, r + Rs, ... ----
        const int32_t nq = (min(chr, cur.nb1 - ch * chr) + 3) >> 2;
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
            if (unit[k] >= 0) {
                const int32_t r = unit[k] >> 28, g = (unit[k] >> 20) & 0xff, h = unit[k] & 0xfffff;
                const T* ap = sm.a[b] + 4 * g * chr;
                const T* sp = sm.s[b] + 4 * h;
#pragma unroll 1
                for (int32_t qq = r; qq < nq; qq += Rs) {
                    if constexpr (ENC) {
                        float4 av[4], sv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4*>(ap + i * chr + 4 * qq);
#pragma unroll
                        for (int j = 0; j < 4; ++j) sv[j] = *reinterpret_cast<const float4*>(sp + (4 * qq + j) * ld2);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float a[4] = {av[i].x, av[i].y, av[i].z, av[i].w};  // rows 4qq..4qq+3
#pragma unroll
                            for (int jp = 0; jp < 2; ++jp) {
                                const float2 p0 = make_float2(a[2 * jp], a[2 * jp]);
                                const float2 p1 = make_float2(a[2 * jp + 1], a[2 * jp + 1]);
                                const float4 s0 = sv[2 * jp], s1 = sv[2 * jp + 1];
                                const float2 t0 = __fadd2_rn(p0, make_float2(s0.x, s0.y));
                                const float2 u0 = __fadd2_rn(p1, make_float2(s1.x, s1.y));
                                const float2 t1 = __fadd2_rn(p0, make_float2(s0.z, s0.w));
                                const float2 u1 = __fadd2_rn(p1, make_float2(s1.z, s1.w));
                                acc[k][i][0] = fmin3(acc[k][i][0], t0.x, u0.x);
                                acc[k][i][1] = fmin3(acc[k][i][1], t0.y, u0.y);
                                acc[k][i][2] = fmin3(acc[k][i][2], t1.x, u1.x);
                                acc[k][i][3] = fmin3(acc[k][i][3], t1.y, u1.y);
                            }
                        }
                    } else {
                        T av[4][4], sv[4][4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int4 v = *reinterpret_cast<const int4*>(ap + i * chr + 4 * qq);
                            av[i][0] = *reinterpret_cast<const T*>(&v.x);
                            av[i][1] = *reinterpret_cast<const T*>(&v.y);
                            av[i][2] = *reinterpret_cast<const T*>(&v.z);
                            av[i][3] = *reinterpret_cast<const T*>(&v.w);
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int4 v = *reinterpret_cast<const int4*>(sp + (4 * qq + j) * ld2);
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
                                for (int e = 0; e < 4; ++e)
                                    acc[k][i][e] = qb_addmin(av[i][j], sv[j][e], acc[k][i][e]);
                    }
                }
            }
        }
        if (!next_same) {
            // ---- the item's end: + dist_C2(b2, v2), min over the columns, per pair ----
            const int32_t count = cur.count, nb2 = cur.nb2;
#pragma unroll
            for (int k = 0; k < QB_UMAX; ++k) {
                if (unit[k] >= 0) {
                    const int32_t g = (unit[k] >> 20) & 0xff, h = unit[k] & 0xfffff;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int32_t u = 4 * g + i;
                        if (u < count) {
                            const int4 cv = __ldg(reinterpret_cast<const int4*>(c.apsp + sm.a2off[par][u] + 4 * h));
                            const CT c4[4] = {*reinterpret_cast<const CT*>(&cv.x), *reinterpret_cast<const CT*>(&cv.y),
                                              *reinterpret_cast<const CT*>(&cv.z), *reinterpret_cast<const CT*>(&cv.w)};
                            // (padding columns past |B2| hold no distance: skipped)
                            CT v = acc[k][i][0] + c4[0];
#pragma unroll
                            for (int e = 1; e < 4; ++e) {
                                const CT y = acc[k][i][e] + c4[e];
                                v = (y < v && 4 * h + e < nb2) ? y : v;
                            }
                            atomicMin(&sm.res[par][u], enc_min<CT>(v));
                        }
                    }
                }
            }
            __syncthreads();
            if (tid < count) {
                const uint32_t qi = sm.qidx[par][tid];
                const T z = sm.init[par][tid];
                if constexpr (ENC) {
                    // the bit pattern is the exact integer below 2^24
                    const int32_t y = sm.res[par][tid];
                    const int32_t zi = *reinterpret_cast<const int32_t*>(&z);
                    if (y < (1 << 24) || zi < (1 << 24))
                        ((int32_t*)out)[qi] = zi < y ? zi : y;
                    else
                        fb[atomicAdd(nfb, 1u)] = qi;  // recomputed exactly in int32
                } else {
                    T y = dec_min<T>(sm.res[par][tid]);
                    y = z < y ? z : y;
                    if (MODE == 2)
                        ((float*)out)[qi] = (float)y;
                    else
                        ((int32_t*)out)[qi] = (int32_t)min((int32_t)y, (int32_t)SPQ_INF_I32);
                }
                sm.res[par][tid] = res_reset<CT>();
            }
        }
        __syncthreads();  // buffer b is free for the next issue
        if (!has_next) break;
        if (next_same) {
            ++ch;
        } else {
            // the switch to item m + 1: item m's records make room for m + 2 (from the
            // registers) and m + 4 (its record, by one thread)
            ++m;
            ch = 0;
            {
                const QItem& p2 = sm.item[(m + 1) & 3];
                const int pp = (m + 1) & 1;
                if (tid < p2.count) {
                    sm.a1off[pp][tid] = nrow.x;
                    sm.a2off[pp][tid] = nrow.y;
                    sm.init[pp][tid] = ninit;
                    sm.qidx[pp][tid] = nidx;
                }
                qb_store_pos(sm, pp, p2, tid, pr1, pr2);
            }
            if (tid == 0) sm.item[(m + 3) & 3] = item_at(m + 3);
            qb_units(sm.item[m & 3], tid, unit);
            __syncthreads();
            const QItem& p3 = sm.item[(m + 2) & 3];
            nrow = tid < p3.count ? rows[p3.start + tid] : make_longlong2(0, 0);
            ninit = tid < p3.count ? init[p3.start + tid] : T(0);
            nidx = tid < p3.count ? idx[p3.start + tid] : 0u;
            qb_fetch_pos(c, p3, tid, pr1, pr2);
        }
        b ^= 1;
    }
}

// The listed pairs (positions in the caller's arrays) in exact int32 arithmetic, one warp
// per pair, reading the block through the slot positions: the answers of the encoded form
// at or above 2^24.
__global__ void __launch_bounds__(256) k_qb_fallback(const QueryCtx<int32_t> ctx, const int2* __restrict__ pairs,
                                                     const uint32_t* __restrict__ fb, const uint32_t* __restrict__ nfb,
                                                     int32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint32_t n = *nfb;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t qi = fb[w];
        int2 pr = pairs[qi];
        int32_t c1 = ctx.comp[pr.x], c2 = ctx.comp[pr.y];
        if (c1 > c2) {
            pr = make_int2(pr.y, pr.x);
            const int32_t t = c1;
            c1 = c2;
            c2 = t;
        }
        const MatDesc d1 = ctx.descs[c1], d2 = ctx.descs[c2];
        const int32_t* A1 = ctx.apsp + d1.off + (int64_t)ctx.local[pr.x] * d1.n;
        const int32_t* A2 = ctx.apsp + d2.off + (int64_t)ctx.local[pr.y] * d2.n;
        const int32_t nb1 = ctx.nb[c1], nb2 = ctx.nb[c2];
        const int32_t* pos1 = ctx.bgpos + ctx.bg_off[c1];
        const int32_t* pos2 = ctx.bgpos + ctx.bg_off[c2];
        int32_t r = SPQ_INF_I32;
        for (int32_t jb = 0; jb < nb2; jb += 32) {
            const int32_t j = jb + lane;
            const int32_t col = j < nb2 ? pos2[j] : 0;
            int32_t t = SPQ_INF_I32;
            for (int32_t b1 = 0; b1 < nb1; ++b1)
                if (j < nb2) t = __viaddmin_s32(A1[b1], ctx.D[(int64_t)pos1[b1] * ctx.N + col], t);
            if (j < nb2) r = min(r, t + A2[j]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = min(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (c1 == c2) r = min(r, A1[ctx.local[pr.y]]);
        if (pr.x == pr.y) r = 0;
        if (lane == 0) out[qi] = min(r, (int32_t)SPQ_INF_I32);
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

// Items: every run of one component pair (a nonempty block with at most QB_PMAX rows and
// columns) cut into nearly equal pieces of at most qb_pair_cap(ld) pairs; the order of the
// item list is arbitrary.  A run's first position finds the run's end by a galloping
// search (runs are short), and a warp takes the slots of all its runs' items with one
// atomic (as it adds its runs' profiling counts).
__global__ void k_qb_items(const uint32_t* __restrict__ keys, int64_t q, uint32_t k, const int32_t* __restrict__ nb,
                           QItem* __restrict__ items, uint32_t* __restrict__ nitems,
                           unsigned long long* __restrict__ stats) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t key = 0, pieces = 0;
    int32_t c1 = 0, c2 = 0, nb1 = 0, nb2 = 0;
    int64_t n = 0;
    if (p < q) {
        key = keys[p];
        if (key < k * k && (p == 0 || keys[p - 1] != key)) {
            c1 = (int32_t)(key / k);
            c2 = (int32_t)(key % k);
            nb1 = nb[c1];
            nb2 = nb[c2];
            if (nb1 > 0 && nb2 > 0 && nb1 <= QB_PMAX && nb2 <= QB_PMAX) {
                // keys[lo] == key; hi = q or keys[hi] != key (a larger key)
                int64_t lo = p, hi = q, step = 1;
                for (;;) {
                    const int64_t nx = lo + step;
                    if (nx >= q || keys[nx] != key) {
                        hi = nx < q ? nx : q;
                        break;
                    }
                    lo = nx;
                    step <<= 1;
                }
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (keys[mid] == key)
                        lo = mid;
                    else
                        hi = mid;
                }
                n = hi - p;
                const int64_t cap = qb_pair_cap((nb2 + 3) & ~3);
                pieces = (uint32_t)((n + cap - 1) / cap);
            }
        }
    }
    // the warp's item slots: an inclusive scan of the piece counts, one atomic
    uint32_t incl = pieces;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t wbase = 0;
    if (lane == 31 && incl > 0) wbase = atomicAdd(nitems, incl);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    if (stats) {
        // algorithmic work of the run: |B1| x |B2| updates per pair; bytes: each item's
        // block once, per pair its two table rows, the pair, its position and its answer
        unsigned long long w = pieces ? (unsigned long long)(n * nb1 * nb2) : 0ull;
        unsigned long long by = pieces ? (unsigned long long)(4 * (int64_t)pieces * nb1 * nb2 +
                                                              n * (4 * (((nb1 + 3) & ~3) + ((nb2 + 3) & ~3)) + 16))
                                       : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w += __shfl_down_sync(0xffffffffu, w, o);
            by += __shfl_down_sync(0xffffffffu, by, o);
        }
        if (lane == 0 && w > 0) {
            atomicAdd(&stats[0], w);
            atomicAdd(&stats[1], by);
        }
    }
    const uint32_t base = wbase + incl - pieces;
    for (int64_t i = 0; i < (int64_t)pieces; ++i) {
        const int64_t s0 = p + i * n / pieces, s1 = p + (i + 1) * n / pieces;
        items[base + i] = qb_make_item((uint32_t)s0, (int32_t)(s1 - s0), c1, c2, nb);
    }
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

template <typename T, int MODE, bool ENC>
cudaError_t launch_blocks_kernel(const QbCtx<T>& c, const QItem* items, const uint32_t* nitems, const longlong2* rows,
                                 const T* init, const uint32_t* idx, void* out, uint32_t* fb, uint32_t* nfb, int64_t q,
                                 cudaStream_t st) {
    static std::atomic<bool> attr{false};
    const size_t smem = sizeof(QbSmem<T>);
    if (!attr.load()) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_qb_blocks<T, MODE, ENC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr.store(true);
    }
    int64_t grid = (int64_t)qb_sms() * QB_CTAS;
    if (grid > q) grid = q;  // at most q items
    k_qb_blocks<T, MODE, ENC><<<(unsigned)grid, QB_TH, smem, st>>>(c, items, nitems, rows, init, idx, out, fb, nfb);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int32_t query_blocks_max_nb() { return QB_PMAX; }

int64_t query_blocks_scratch_words(int64_t q) {
    // rows (4 words per pair), starting values (1), items (12), the fallback list (1), two
    // counters, and up to 6 words of 16-byte alignment
    return 18 * q + 8;
}

template <typename T>
cudaError_t launch_query_blocks(const QueryCtx<T>& ctx, const int32_t* pairs, int64_t q, void* out, bool out_f32,
                                uint32_t k, const uint32_t* keys, const uint32_t* idx, uint32_t* scratch,
                                cudaStream_t st) {
    // scratch: rows (16-byte aligned) | starting values | items | fallback list | counters
    uint32_t* base = (uint32_t*)(((uintptr_t)scratch + 15) & ~(uintptr_t)15);
    longlong2* rows = reinterpret_cast<longlong2*>(base);
    T* init = reinterpret_cast<T*>(base + 4 * q);
    const int64_t o_items = (5 * q + 3) & ~(int64_t)3;
    QItem* items = reinterpret_cast<QItem*>(base + o_items);
    uint32_t* fb = base + o_items + 12 * q;
    uint32_t* nitems = fb + q;
    uint32_t* nfb = nitems + 1;
    const int2* p2 = reinterpret_cast<const int2*>(pairs);
    const bool mode_f32 = out_f32 || !std::is_same<T, int32_t>::value;
    // int32 tables with every finite entry below 2^24: the float-encoded arithmetic
    const bool enc = std::is_same<T, int32_t>::value && !mode_f32 && ctx.exact24;
    cudaError_t e = cudaMemsetAsync(nitems, 0, 8, st);
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
    k_qb_items<<<g, 256, 0, st>>>(keys, q, k, ctx.nb, items, nitems, prof ? ctx.qstats : nullptr);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const QbCtx<T> c{ctx.apsp, ctx.D, ctx.N, ctx.bgpos, ctx.bg_off};
    if (prof && (e = cudaEventRecord(ctx.qev[0], st)) != cudaSuccess) return e;
    if (mode_f32)
        e = launch_blocks_kernel<T, 2, false>(c, items, nitems, rows, init, idx, out, fb, nfb, q, st);
    else if (enc)
        e = launch_blocks_kernel<T, 0, true>(c, items, nitems, rows, init, idx, out, fb, nfb, q, st);
    else
        e = launch_blocks_kernel<T, 0, false>(c, items, nitems, rows, init, idx, out, fb, nfb, q, st);
    if (e == cudaSuccess && prof) e = cudaEventRecord(ctx.qev[1], st);
    if constexpr (std::is_same<T, int32_t>::value) {
        if (e == cudaSuccess && enc) {
            k_qb_fallback<<<(unsigned)(qb_sms() * 4), 256, 0, st>>>(ctx, p2, fb, nfb, (int32_t*)out);
            count_launches(1);
            e = cudaGetLastError();
        }
    }
    return e;
}

template cudaError_t launch_query_blocks<int32_t>(const QueryCtx<int32_t>&, const int32_t*, int64_t, void*, bool,
                                                  uint32_t, const uint32_t*, const uint32_t*, uint32_t*, cudaStream_t);
template cudaError_t launch_query_blocks<float>(const QueryCtx<float>&, const int32_t*, int64_t, void*, bool, uint32_t,
                                                const uint32_t*, const uint32_t*, uint32_t*, cudaStream_t);

}  // namespace spq
