// All-pairs distances of the boundary graph by tropical elimination and
// back-substitution (the boundary-graph APSP of Algorithm 1, computed exactly, with fewer
// min-plus updates than Floyd-Warshall in a nested-dissection order).
//
// Forward (fw_single with rowflags): block elimination in the matrix order.  After it,
// for row block R and any column j right of R, F(r, j) (r in R) is the length of a
// shortest r-j path whose inner vertices all lie in blocks <= R, and the diagonal tile
// (R, R) holds the shortest paths inside blocks <= R.
//
// Back-substitution (here), row blocks from the last to the first.  Take a shortest path
// from r in R to any vertex j, and on it the first vertex k after r that lies right of
// block R.  The part r..k has its inner vertices in blocks <= R, so it is F(r, k); the
// rest is d(k, j).  Hence, with K(R) = the columns k right of R with a finite F(r, k) for
// some r in R (the "frontier" of R, small in a dissection order):
//   d(R, J) = min over k in K(R) of F(R, k) + d(k, J)       for J right of R,
//   d(R, R) = min(F(R, R), min over k in K(R) of F(R, k) + d(k, R)),
// where d(k, J) and d(k, R) = d(R, k) are already final.  Each is a min-plus product of
// a 128 x |K(R)| panel (gathered once, before the back-substitution overwrites row R)
// with |K(R)| gathered rows of the matrix.
//
// One persistent launch walks the tiles in that order through an atomic work counter:
// row blocks from the last to the first, inside a row the tiles right of the diagonal,
// then the diagonal tile.  Tile (R, J) needs the final tiles (min(k, J), max(k, J)) for
// the blocks k of K(R); the diagonal needs (R, k).  All of them come earlier in the
// order, so every tile a CTA waits for is held by a CTA that is already running and
// waits only for tiles earlier still: the waits always end.  Each wait is bounded
// anyway (2 s of %globaltimer); past that the launch records kErrWait and stops.
#include <cuda_runtime.h>

#include <math.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fw_tile.cuh"
#include "sync.cuh"

namespace spq {

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of one dependency wait

// Test hook (spq_test_backsub_wait): a shorter bound, and launches that release none of
// their tiles, so that a dependency wait runs out without any fault or hang.
std::atomic<unsigned long long> g_wait_ns{kWaitNs};
std::atomic<int> g_withhold{0};


// Integer encoding of the converted (CONV) back-substitution.  An int32 table value m
// with 0 <= m < 2^24, read as the bits of a float, is the float m * 2^-149 (a subnormal
// below 2^23, the smallest binade of normals from 2^23 to 2^24): float addition of two
// such values is exact integer addition of the bit patterns while the sum stays below
// 2^24, and float order is integer order.  So the tiles stored as int32 are read back as
// floats without any conversion; only the forward values (true floats) are converted
// once, and SPQ_INF_I32 (2^29, read as 2^-63) is infinity (every finite distance of an
// int32 graph is below it).  Subnormals are kept: no flush-to-zero in these kernels.
__device__ __forceinline__ float enc(float x) { return __int_as_float(x < 536870912.0f ? (int)x : SPQ_INF_I32); }

// Encoded results -> stored int32: sums of infinities clamp to SPQ_INF_I32; true if a
// finite value is >= 2^24 (then not provably exact).
__device__ __forceinline__ bool clamp_enc(float (&acc)[8][8]) {
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int b = __float_as_int(acc[i][j]);
            bad |= b >= (1 << 24) && b < SPQ_INF_I32;
            acc[i][j] = __int_as_float(b < SPQ_INF_I32 ? b : SPQ_INF_I32);
        }
    return bad;
}

// Marks of the tiles (I < J) the assembled boundary-graph matrix may hold a finite entry
// in (flags[I * nR + J] = 1): every pair of tiles a component's slots fall into (its
// clique), and the tiles of the edges between components.
__global__ void __launch_bounds__(256) k_mark_clique(const int32_t* __restrict__ nb, const int32_t* __restrict__ bg_off,
                                                     const int32_t* __restrict__ bgpos, int32_t k, int32_t nR,
                                                     uint32_t* __restrict__ flags) {
    __shared__ int32_t blk[256];
    __shared__ int32_t nblk;
    for (int32_t c = blockIdx.x; c < k; c += gridDim.x) {
        const int32_t b = nb[c];
        const int32_t* pos = bgpos + bg_off[c];
        if (threadIdx.x == 0) nblk = 0;
        __syncthreads();
        // distinct tiles of the component's slots (a slot's tile differs from the previous
        // slot's only a few times; duplicates beyond that are harmless)
        for (int32_t i = threadIdx.x; i < b; i += blockDim.x) {
            const int32_t t = pos[i] / T_;
            if (i == 0 || pos[i - 1] / T_ != t) {
                const int32_t at = atomicAdd(&nblk, 1);
                if (at < 256) blk[at] = t;
            }
        }
        __syncthreads();
        const int32_t m = nblk;
        if (m <= 256) {
            for (int32_t x = threadIdx.x; x < m * m; x += blockDim.x) {
                const int32_t I = blk[x / m], J = blk[x % m];
                if (I < J) flags[(int64_t)I * nR + J] = 1u;
            }
        } else {  // many runs: mark from every slot pair
            for (int32_t x = threadIdx.x; x < b * b; x += blockDim.x) {
                const int32_t I = pos[x / b] / T_, J = pos[x % b] / T_;
                if (I < J) flags[(int64_t)I * nR + J] = 1u;
            }
        }
        __syncthreads();
    }
}

// Every pair of the listed tiles (the separators shared by concurrent runs of rounds).
__global__ void k_mark_pairs(const int32_t* __restrict__ blocks, int32_t nb, int32_t nR, uint32_t* __restrict__ flags) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * nb; t += gridDim.x * blockDim.x) {
        const int32_t I = blocks[t / nb], J = blocks[t % nb];
        if (I < J) flags[(int64_t)I * nR + J] = 1u;
    }
}

__global__ void k_mark_inter(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ part, const int32_t* __restrict__ local,
                             const int32_t* __restrict__ bg_off, const int32_t* __restrict__ bgpos, int32_t nR,
                             uint32_t* __restrict__ flags) {
    const int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int32_t cu = part[u];
    int32_t tu = -1;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        const int32_t v = col[e];
        const int32_t cv = part[v];
        if (cv == cu) continue;
        if (tu < 0) tu = bgpos[bg_off[cu] + local[u]] / T_;
        const int32_t tv = bgpos[bg_off[cv] + local[v]] / T_;
        if (tu < tv) flags[(int64_t)tu * nR + tv] = 1u;
        else if (tv < tu) flags[(int64_t)tv * nR + tu] = 1u;
    }
}

// Infinity in the marked tiles (and their mirrors) and the diagonal tiles, 0 on the
// diagonal: the only tiles the elimination reads before the back-substitution writes
// every tile.
template <typename T>
__global__ void __launch_bounds__(256) k_fill_marked(T* __restrict__ M, int64_t N, int32_t nR,
                                                     const uint32_t* __restrict__ flags) {
    const int32_t R = blockIdx.x;
    const T inf = Inf<T>::value();
    for (int32_t J = R; J < nR; ++J) {
        if (J != R && flags[(int64_t)R * nR + J] == 0u) continue;
        for (int32_t x = threadIdx.x; x < T_ * T_ / 4; x += blockDim.x) {
            const int64_t i = (int64_t)R * T_ + (x >> 5), c = (int64_t)J * T_ + (x & 31) * 4;
            if (i < N && c < N) {
                T v[4] = {inf, inf, inf, inf};
                if (J == R && i >= c && i < c + 4) v[i - c] = T(0);
                *reinterpret_cast<int4*>(M + i * N + c) = *reinterpret_cast<const int4*>(v);
            }
            // the mirror tile (J, R), all infinite
            const int64_t mi = (int64_t)J * T_ + (x >> 5), mc = (int64_t)R * T_ + (x & 31) * 4;
            if (J != R && mi < N && mc < N) *reinterpret_cast<int4*>(M + mi * N + mc) = inf4<T>();
        }
    }
}

// One matrix of a back-substitution launch: its table, order and row blocks, and where
// its per-tile-pair (masks, fblk, tflags) and per-row-block (fcnt, kcnt, koff) records
// sit in the launch's arrays.
template <typename T>
struct BsMat {
    T* M;
    int64_t N;
    int32_t nR;
    const uint32_t* rowflags;  // nR x nR marks of the forward pass, or null (every tile)
    int64_t pair0;             // offset of its nR x nR records
    int64_t row0;              // offset of its nR records
};

// A run of the work order: row block R of matrix mat, its tiles right of the diagonal and
// then the diagonal tile, as the items [start, start + nR - R).
struct BsRun {
    int64_t start;
    int32_t mat, R;
};

// Per row block R of matrix blockIdx.y: the column tiles J > R holding a finite entry of
// F (the forward pass's marks narrow the search), the 128-bit mask of their finite
// columns (fblk / masks at pair0 + R * nR + i), their number and the number of finite
// columns |K(R)|.
template <typename T>
__global__ void __launch_bounds__(256) k_colmask(const BsMat<T>* __restrict__ mats, uint4* __restrict__ masks,
                                                 int32_t* __restrict__ fblk, int32_t* __restrict__ fcnt,
                                                 int32_t* __restrict__ kcnt, const int32_t* __restrict__ kplan,
                                                 uint32_t* __restrict__ err) {
    __shared__ uint32_t colf[2][T_];
    __shared__ uint32_t wm[4];
    const BsMat<T> m = mats[blockIdx.y];
    const int32_t R = blockIdx.x, nR = m.nR;
    if (R >= nR) return;
    const int64_t N = m.N;
    const int tid = threadIdx.x, c = tid & (T_ - 1), h = tid >> 7;
    const T inf = Inf<T>::value();
    const int64_t r0 = (int64_t)R * T_;
    const int64_t nrows = (N - r0) < T_ ? (N - r0) : T_;
    int32_t cnt = 0, kc = 0;
    for (int32_t J = R + 1; J < nR; ++J) {
        if (m.rowflags && m.rowflags[(int64_t)R * nR + J] == 0u) continue;
        const int64_t col = (int64_t)J * T_ + c;
        uint32_t f = 0;
        if (col < N)
            for (int64_t i = h; i < nrows; i += 2) f |= (m.M[(r0 + i) * N + col] < inf) ? 1u : 0u;
        colf[h][c] = f;
        __syncthreads();
        if (tid < T_) {
            const unsigned b = __ballot_sync(0xffffffffu, (colf[0][tid] | colf[1][tid]) != 0u);
            if ((tid & 31) == 0) wm[tid >> 5] = b;
        }
        __syncthreads();
        const uint4 mk = make_uint4(wm[0], wm[1], wm[2], wm[3]);
        const int pc = __popc(mk.x) + __popc(mk.y) + __popc(mk.z) + __popc(mk.w);
        if (pc) {
            if (tid == 0) {
                fblk[m.pair0 + (int64_t)R * nR + cnt] = J;
                masks[m.pair0 + (int64_t)R * nR + cnt] = mk;
            }
            ++cnt;
            kc += pc;
        }
        __syncthreads();
    }
    if (tid == 0) {
        // (a replay: more finite columns than recorded would overrun the recorded lists;
        //  the row block is left out and the caller told to rebuild)
        if (kplan && kc > kplan[m.row0 + R]) {
            cnt = 0;
            kc = 0;
            atomicOr(err, kErrPlan);
        }
        fcnt[m.row0 + R] = cnt;
        kcnt[m.row0 + R] = kc;
    }
}

// K(R) of row block blockIdx.x of matrix blockIdx.y as ascending column indices at
// klist[koff ..), padded to a multiple of KC with copies of its first entry (their panel
// rows are infinite, so they change nothing).
template <typename T>
__global__ void __launch_bounds__(T_) k_klist(const BsMat<T>* __restrict__ mats, const uint4* __restrict__ masks,
                                              const int32_t* __restrict__ fblk, const int32_t* __restrict__ fcnt,
                                              const int32_t* __restrict__ kcnt, const int64_t* __restrict__ koff,
                                              int32_t* __restrict__ klist) {
    const BsMat<T> m = mats[blockIdx.y];
    const int32_t R = blockIdx.x, nR = m.nR;
    if (R >= nR) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t base = koff[m.row0 + R];
    const int32_t nf = fcnt[m.row0 + R];
    int32_t pos = 0;
    for (int32_t i = 0; i < nf; ++i) {
        const uint4 mk = masks[m.pair0 + (int64_t)R * nR + i];
        const uint32_t words[4] = {mk.x, mk.y, mk.z, mk.w};
        const uint32_t word = words[w];
        int32_t woff = 0;
        for (int x = 0; x < w; ++x) woff += __popc(words[x]);
        if ((word >> lane) & 1u)
            klist[base + pos + woff + __popc(word & ((1u << lane) - 1u))] =
                fblk[m.pair0 + (int64_t)R * nR + i] * T_ + w * 32 + lane;
        pos += __popc(mk.x) + __popc(mk.y) + __popc(mk.z) + __popc(mk.w);
    }
    __syncthreads();
    const int32_t kc = kcnt[m.row0 + R];
    const int32_t kp = (kc + KC - 1) / KC * KC;
    if (kc > 0)
        for (int32_t j = kc + tid; j < kp; j += T_) klist[base + j] = klist[base];
}

// A panels of the row blocks [R0, R1) of the matrices mat0 + blockIdx.y:
// A[(koff - aoff0 + k) * 128 + i] = F(R*128 + i, klist[k]), read as its mirror
// F(klist[k], R*128 + i) (one contiguous row piece); padding rows infinite.
template <typename T, bool CONV>
__global__ void __launch_bounds__(256) k_gather_a(const BsMat<T>* __restrict__ mats, int32_t mat0, int32_t R0,
                                                  int32_t R1, const int64_t* __restrict__ koff,
                                                  const int32_t* __restrict__ kcnt, const int32_t* __restrict__ klist,
                                                  int64_t aoff0, T* __restrict__ A) {
    const BsMat<T> m = mats[mat0 + blockIdx.y];
    const int32_t R = R0 + blockIdx.x;
    if (R >= R1 || R >= m.nR) return;
    const int64_t N = m.N;
    const int64_t base = koff[m.row0 + R];
    const int32_t kc = kcnt[m.row0 + R];
    const int32_t kp = (kc + KC - 1) / KC * KC;
    const int64_t col0 = (int64_t)R * T_;
    for (int64_t idx = threadIdx.x; idx < (int64_t)kp * (T_ / 4); idx += blockDim.x) {
        const int32_t k = (int32_t)(idx >> 5), c4 = (int32_t)(idx & 31);
        int4 v = inf4<T>();
        if (k < kc && col0 + c4 * 4 < N)
            v = *reinterpret_cast<const int4*>(m.M + (int64_t)klist[base + k] * N + col0 + c4 * 4);
        if constexpr (CONV) {
            const float4 f = *reinterpret_cast<const float4*>(&v);
            const float4 g = make_float4(enc(f.x), enc(f.y), enc(f.z), enc(f.w));
            v = *reinterpret_cast<const int4*>(&g);
        }
        *reinterpret_cast<int4*>(A + (base - aoff0 + k) * T_ + c4 * 4) = v;
    }
}

// Stage KC gathered rows klist[kbase ..) of M, columns [col0, col0 + 128), into P.
template <typename T>
__device__ __forceinline__ void stage_rows(T (*P)[T_], const T* __restrict__ M, int64_t N,
                                           const int32_t* __restrict__ rows, int64_t col0, int tid, int4 fill) {
#pragma unroll
    for (int it = 0; it < (KC * T_ / 4) / NTH; ++it) {
        const int idx = it * NTH + tid;
        const int kk = idx >> 5, c4 = idx & 31;
        const int64_t c = col0 + c4 * 4;
        T* dst = &P[kk][c4 * 4];
        if (c < N)
            cp_async16(dst, M + (int64_t)rows[kk] * N + c);
        else
            *reinterpret_cast<int4*>(dst) = fill;
    }
}

// Stage KC contiguous panel rows (128 wide) into P.
template <typename T>
__device__ __forceinline__ void stage_panel(T (*P)[T_], const T* __restrict__ A, int tid) {
#pragma unroll
    for (int it = 0; it < (KC * T_ / 4) / NTH; ++it) {
        const int idx = it * NTH + tid;
        cp_async16(&P[idx >> 5][(idx & 31) * 4], A + (int64_t)(idx >> 5) * T_ + (idx & 31) * 4);
    }
}

// CONV (float tables of an int32 graph): every tile is stored as int32 (the final table
// type) as soon as it is final, and the arithmetic runs on the integer encoding above
// (tiles read as rows of d need no conversion); a finite value >= 2^24 sets kErrExact.
// Items [0, nitems) follow the runs (ascending starts); one launch may hold the rows of
// several independent matrices, interleaved.
template <typename T, bool CONV>
__global__ void __launch_bounds__(NTH, SPQ_FW_MIN_CTAS)
    k_backsub(const BsMat<T>* __restrict__ mats, const BsRun* __restrict__ runs, int32_t nruns, int64_t nitems,
              const int64_t* __restrict__ koff, const int32_t* __restrict__ kcnt, const int32_t* __restrict__ klist,
              const T* __restrict__ A, int64_t aoff0, const int32_t* __restrict__ fblk,
              const int32_t* __restrict__ fcnt, uint32_t* __restrict__ tflags,
              unsigned long long* __restrict__ counter, uint32_t* __restrict__ err, uint32_t* __restrict__ exact,
              unsigned long long wait_ns, int withhold) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PanelSmem<T>& sm = *reinterpret_cast<PanelSmem<T>*>(smem_raw);
    __shared__ int64_t s_item;
    __shared__ int32_t s_mat, s_R, s_J;
    __shared__ int s_fail;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (;;) {
        if (tid == 0) {
            int64_t t = (int64_t)atomicAdd(counter, 1ull);
            if (*reinterpret_cast<volatile uint32_t*>(err) & kErrWait) t = nitems;
            s_item = t;
            s_fail = 0;
            if (t < nitems) {
                int32_t lo = 0, hi = nruns;  // the last run starting at or before t
                while (hi - lo > 1) {
                    const int32_t mid = (lo + hi) >> 1;
                    if (runs[mid].start <= t) lo = mid; else hi = mid;
                }
                const BsRun ru = runs[lo];
                const int64_t p = t - ru.start;
                const int32_t last = mats[ru.mat].nR - 1 - ru.R;  // tiles right of the diagonal
                s_mat = ru.mat;
                s_R = ru.R;
                s_J = p < last ? ru.R + 1 + (int32_t)p : ru.R;
            }
        }
        __syncthreads();
        const int64_t t = s_item;
        if (t >= nitems) break;
        const BsMat<T> m = mats[s_mat];
        const int32_t R = s_R, J = s_J, nR = m.nR;
        T* __restrict__ M = m.M;
        const int64_t N = m.N;
        const int32_t kc = kcnt[m.row0 + R];
        const int64_t r0 = (int64_t)R * T_, c0 = (int64_t)J * T_;
        const int4 fill = CONV ? make_int4(SPQ_INF_I32, SPQ_INF_I32, SPQ_INF_I32, SPQ_INF_I32) : inf4<T>();
        const T vinf = CONV ? __int_as_float(SPQ_INF_I32) : Inf<T>::value();
        if (kc > 0) {
            // dependencies: the final tiles this one reads
            if (tid < 32) {
                const int32_t nf = fcnt[m.row0 + R];
                for (int32_t i = tid; i < nf; i += 32) {
                    const int32_t K = fblk[m.pair0 + (int64_t)R * nR + i];
                    const int32_t a = (J == R) ? R : (K < J ? K : J);
                    const int32_t b = (J == R) ? K : (K < J ? J : K);
                    const uint32_t* f = tflags + m.pair0 + (int64_t)a * nR + b;
                    if (ld_acquire(f) == 0u) {
                        const unsigned long long t0 = global_ns();
                        while (ld_acquire(f) == 0u) {
                            __nanosleep(256);
                            // another CTA gave up (the launch is abandoned), or the bound ran out
                            if (*reinterpret_cast<volatile uint32_t*>(err) & kErrWait) {
                                s_fail = 1;
                                break;
                            }
                            if (global_ns() - t0 > wait_ns) {
                                atomicOr(err, kErrWait);
                                s_fail = 1;
                                break;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (s_fail) break;
            T acc[8][8];
            if (J == R) {
                load_c<T>(acc, M, N, r0, r0, tx, ty);
                if constexpr (CONV)
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = enc(acc[i][j]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = vinf;
            }
            const int64_t kb = koff[m.row0 + R];
            const int32_t nch = (kc + KC - 1) / KC;
            const T* Ap = A + (kb - aoff0) * T_;
            const int32_t* rows = klist + kb;
            stage_panel<T>(sm.a[0], Ap, tid);
            stage_rows<T>(sm.b[0], M, N, rows, c0, tid, fill);
            cp_async_commit();
#pragma unroll 1
            for (int32_t ch = 0; ch < nch; ++ch) {
                if (ch + 1 < nch) {
                    const int s = (ch + 1) & 1;
                    stage_panel<T>(sm.a[s], Ap + (int64_t)(ch + 1) * KC * T_, tid);
                    stage_rows<T>(sm.b[s], M, N, rows + (ch + 1) * KC, c0, tid, fill);
                    cp_async_commit();
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                // the last chunk's rows past |K(R)| are infinite padding: skipped
                const int kend = ch + 1 < nch ? KC : ((kc - ch * KC) + 1) & ~1;
                compute_chunk<T>(acc, sm, ch & 1, tx, ty, kend);
                __syncthreads();
            }
            if constexpr (CONV)
                if (clamp_enc(acc)) atomicOr(exact, kErrExact);
            store_c<T>(acc, M, N, r0, c0, tx, ty);
            if (J != R) store_c_transposed<T>(acc, M, N, r0, c0, tx, ty);
        } else if (CONV || J != R) {
            // no finite entry right of R: d(R, J) = F(R, J) = inf, stored here (an unmarked
            // tile was never initialised), and d(R, R) = F(R, R), already in place (with
            // conversion: final but still float, stored as int32)
            T acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = vinf;
            if constexpr (CONV) {
                if (J == R) {
                    load_c<T>(acc, M, N, r0, r0, tx, ty);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = enc(acc[i][j]);
                }
                if (clamp_enc(acc)) atomicOr(exact, kErrExact);
            }
            store_c<T>(acc, M, N, r0, c0, tx, ty);
            if (J != R) store_c_transposed<T>(acc, M, N, r0, c0, tx, ty);
        }
        __syncthreads();
        if (tid == 0 && !withhold) {
            __threadfence();
            st_release(tflags + m.pair0 + (int64_t)R * nR + J, 1u);
        }
    }
}

int g_sms_e = 0;
int sms_e() {
    if (g_sms_e == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms_e, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms_e <= 0) g_sms_e = 1;
    }
    return g_sms_e;
}

}  // namespace

cudaError_t launch_mark_bg_tiles(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* part,
                                 const int32_t* local, const int32_t* nb, const int32_t* bg_off, const int32_t* bgpos,
                                 int32_t k, int64_t N, uint32_t* flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int32_t nR = (int32_t)((N + T_ - 1) / T_);
    k_mark_clique<<<k < 65535 ? k : 65535, 256, 0, st>>>(nb, bg_off, bgpos, k, nR, flags);
    k_mark_inter<<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, part, local, bg_off, bgpos, nR, flags);
    count_launches(2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill_marked(T* M, int64_t N, const uint32_t* flags, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const int32_t nR = (int32_t)((N + T_ - 1) / T_);
    k_fill_marked<T><<<nR, 256, 0, st>>>(M, N, nR, flags);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mark_pairs(const std::vector<int32_t>& blocks, int64_t N, uint32_t* flags, cudaStream_t st) {
    if (blocks.empty() || N <= 0) return cudaSuccess;
    const int32_t nR = (int32_t)((N + T_ - 1) / T_);
    int32_t* d = nullptr;
    cudaError_t e = scratch_alloc((void**)&d, blocks.size() * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d, blocks.data(), blocks.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int32_t nb = (int32_t)blocks.size();
        k_mark_pairs<<<(nb * nb + 255) / 256 < 1024 ? (nb * nb + 255) / 256 : 1024, 256, 0, st>>>(d, nb, nR, flags);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // (the host list may go away)
    cudaFreeAsync(d, st);
    return e;
}

size_t bg_backsub_scratch_bytes(int64_t N) {
    const int64_t nR = (N + T_ - 1) / T_;
    // masks (16 B), fblk and tile flags (4 B each) per tile pair; per row block: fcnt,
    // kcnt, koff and a run of the work order; the work counter and the matrix record
    return (size_t)(nR * nR) * 24 + (size_t)nR * 32 + 256;
}

// The launches of a back-substitution after its bookkeeping (klist, A panels, work
// order): the k lists, then per launch its A panels and the persistent kernel.
template <typename T>
cudaError_t bs_enqueue(const BsPlan<T>& p, uint32_t* err, uint32_t* exact, std::vector<cudaEvent_t>* ev,
                       cudaStream_t st) {
    const bool conv = std::is_same<T, float>::value && exact != nullptr;
    auto kern = conv ? k_backsub<T, std::is_same<T, float>::value> : k_backsub<T, false>;
    const BsMat<T>* mats = static_cast<const BsMat<T>*>(p.mats);
    const uint4* masks = static_cast<const uint4*>(p.masks);
    const BsRun* runs = static_cast<const BsRun*>(p.runs);
    k_klist<T><<<dim3(p.nRmax, p.nmat), T_, 0, st>>>(mats, masks, p.fblk, p.fcnt, p.kcnt, p.koff, p.klist);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    const size_t psm = sizeof(PanelSmem<T>);
    const int grid = sms_e() * SPQ_FW_MIN_CTAS;
    for (size_t l = 0; l < p.launches.size() && e == cudaSuccess; ++l) {
        const typename BsPlan<T>::Launch& L = p.launches[l];
        const dim3 gg((unsigned)(std::min(L.R1, p.nRmax) - L.R0), (unsigned)L.nm);
        // A panels of the launch's rows: read before the launch overwrites those rows
        if (conv)
            k_gather_a<T, std::is_same<T, float>::value><<<gg, 256, 0, st>>>(mats, L.mat0, L.R0, L.R1, p.koff, p.kcnt,
                                                                              p.klist, L.aoff0, p.A);
        else
            k_gather_a<T, false><<<gg, 256, 0, st>>>(mats, L.mat0, L.R0, L.R1, p.koff, p.kcnt, p.klist, L.aoff0, p.A);
        cudaMemsetAsync(p.counter, 0, 8, st);
        if (ev) cudaEventRecord((*ev)[2 * l], st);
        kern<<<grid, NTH, psm, st>>>(mats, runs + L.run0, (int32_t)(L.run1 - L.run0), L.nit, p.koff, p.kcnt, p.klist,
                                     p.A, L.aoff0, p.fblk, p.fcnt, p.tflags, p.counter, err, exact, g_wait_ns.load(),
                                     g_withhold.load());
        if (ev) cudaEventRecord((*ev)[2 * l + 1], st);
        count_launches(2);
        e = cudaGetLastError();
    }
    return e;
}

// A recorded back-substitution again (the matrices' contents may differ, their structure
// not): frontier marks afresh, checked against the recorded |K(R)|, then the same
// launches; no host step, no allocation.
template <typename T>
cudaError_t bs_replay(const BsPlan<T>& p, uint32_t* err, uint32_t* exact, cudaStream_t st) {
    if (p.nmat == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.tflags, 0, (size_t)p.P2 * 4, st);
    if (e != cudaSuccess) return e;
    k_colmask<T><<<dim3(p.nRmax, p.nmat), 256, 0, st>>>(static_cast<const BsMat<T>*>(p.mats),
                                                        static_cast<uint4*>(p.masks), p.fblk, p.fcnt, p.kcnt, p.kplan,
                                                        err);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return bs_enqueue<T>(p, err, exact, nullptr, st);
}

template <typename T>
cudaError_t bg_backsub_many(const std::vector<BsInput<T>>& in, uint32_t* err, uint32_t* exact, size_t apanel_budget,
                            double* updates, FwProfile* prof, cudaStream_t st, BsPlan<T>* keep) {
    if (keep && keep->ready) {
        if (updates) *updates = keep->updates;
        return bs_replay<T>(*keep, err, exact, st);
    }
    if (updates) *updates = 0.0;
    BsPlan<T> p;
    std::vector<BsMat<T>> hm;
    for (const BsInput<T>& x : in) {
        if (x.N <= 0) continue;
        const int32_t nR = (int32_t)((x.N + T_ - 1) / T_);
        hm.push_back(BsMat<T>{x.M, x.N, nR, x.rowflags, p.P2, p.RR});
        p.P2 += (int64_t)nR * nR;
        p.RR += nR;
        p.nRmax = std::max(p.nRmax, nR);
    }
    p.nmat = (int32_t)hm.size();
    if (p.nmat == 0) {
        if (keep) keep->ready = true;  // nothing to replay
        return cudaSuccess;
    }
    if (p.nmat > 65535) return cudaErrorInvalidValue;
    const int64_t P2 = p.P2, RR = p.RR;
    const int32_t nmat = p.nmat, nRmax = p.nRmax;
    // exact != NULL (float tables only): store int32 tables, checking exactness
    const bool conv = std::is_same<T, float>::value && exact != nullptr;
    auto kern = conv ? k_backsub<T, std::is_same<T, float>::value> : k_backsub<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PanelSmem<T>));
    if (e != cudaSuccess) return e;
    // one scratch block: masks | fblk | tflags | koff | fcnt | kcnt | kplan | runs | counter | mats
    const size_t o_fblk = (size_t)P2 * 16, o_tfl = o_fblk + (size_t)P2 * 4, o_koff = o_tfl + (size_t)P2 * 4;
    const size_t o_fcnt = o_koff + (size_t)RR * 8, o_kcnt = o_fcnt + (size_t)RR * 4, o_kpl = o_kcnt + (size_t)RR * 4;
    const size_t o_runs = (o_kpl + (size_t)RR * 4 + 15) & ~(size_t)15;
    const size_t o_ctr = o_runs + (size_t)RR * sizeof(BsRun);
    const size_t o_mats = (o_ctr + 8 + 15) & ~(size_t)15;
    const size_t bytes = o_mats + (size_t)nmat * sizeof(BsMat<T>);
    if ((e = scratch_alloc((void**)&p.scratch, bytes, st)) != cudaSuccess) return e;
    unsigned char* scratch = p.scratch;
    p.masks = scratch;
    p.fblk = reinterpret_cast<int32_t*>(scratch + o_fblk);
    p.tflags = reinterpret_cast<uint32_t*>(scratch + o_tfl);
    p.koff = reinterpret_cast<int64_t*>(scratch + o_koff);
    p.fcnt = reinterpret_cast<int32_t*>(scratch + o_fcnt);
    p.kcnt = reinterpret_cast<int32_t*>(scratch + o_kcnt);
    p.kplan = reinterpret_cast<int32_t*>(scratch + o_kpl);
    p.runs = scratch + o_runs;
    p.counter = reinterpret_cast<unsigned long long*>(scratch + o_ctr);
    p.mats = scratch + o_mats;
    std::vector<cudaEvent_t> ev;  // per launch of k_backsub: start, end (profiling only)
    std::vector<int32_t> hk(RR);
    std::vector<int64_t> hoff(RR + 1, 0);
    std::vector<BsRun> hruns;
    auto done = [&](cudaError_t r) {
        for (auto& x : ev)
            if (x) cudaEventDestroy(x);
        if (keep && r == cudaSuccess) {
            p.ready = true;
            *keep = std::move(p);
        } else {
            p.release(st);
        }
        return r;
    };
    if ((e = cudaMemcpyAsync(p.mats, hm.data(), hm.size() * sizeof(BsMat<T>), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return done(e);
    if ((e = cudaMemsetAsync(p.tflags, 0, (size_t)P2 * 4, st)) != cudaSuccess) return done(e);
    k_colmask<T><<<dim3(nRmax, nmat), 256, 0, st>>>(static_cast<const BsMat<T>*>(p.mats), static_cast<uint4*>(p.masks),
                                                    p.fblk, p.fcnt, p.kcnt, nullptr, nullptr);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
    if ((e = cudaMemcpyAsync(hk.data(), p.kcnt, (size_t)RR * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return done(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(e);
    double upd = 0.0, items = 0.0;
    for (const BsMat<T>& m : hm)
        for (int32_t R = 0; R < m.nR; ++R) {
            const int64_t i = m.row0 + R;
            hoff[i + 1] = hoff[i] + round_up(hk[i], KC);
            upd += (double)hk[i] * T_ * T_ * (double)(m.nR - R);
            items += (double)(m.nR - R);
        }
    p.updates = upd;
    if (updates) *updates = upd;
    if (prof) {
        prof->bs_updates = upd;
        prof->bs_items = items;
    }
    const int64_t ktot = hoff[RR];
    if ((e = cudaMemcpyAsync(p.koff, hoff.data(), (size_t)RR * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return done(e);
    if ((e = cudaMemcpyAsync(p.kplan, hk.data(), (size_t)RR * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return done(e);
    if ((e = scratch_alloc((void**)&p.klist, (size_t)(ktot > 0 ? ktot : 1) * 4, st)) != cudaSuccess) return done(e);
    // Launches whose A panels fit the budget: whole matrices side by side, or (a matrix
    // whose panels alone exceed it) ranges of its row blocks from the last rows down.
    // Each launch's panels are contiguous in the koff order.
    using Launch = typename BsPlan<T>::Launch;
    std::vector<Launch>& launches = p.launches;
    const int64_t row_bytes = (int64_t)T_ * sizeof(T);
    auto whole = [&](int32_t g0, int32_t g1) { launches.push_back(Launch{g0, g1 - g0, 0, nRmax, 0, 0, 0, 0}); };
    {
        int32_t g0 = 0;
        int64_t gk = 0;
        for (int32_t i = 0; i < nmat; ++i) {
            const BsMat<T>& m = hm[i];
            const int64_t mk = hoff[m.row0 + m.nR] - hoff[m.row0];
            if (mk * row_bytes <= (int64_t)apanel_budget) {
                if (i > g0 && (gk + mk) * row_bytes > (int64_t)apanel_budget) {
                    whole(g0, i);
                    g0 = i;
                    gk = 0;
                }
                gk += mk;
                continue;
            }
            if (i > g0) whole(g0, i);
            std::vector<int32_t> cuts{m.nR};
            for (int32_t R = m.nR - 1; R >= 0; --R) {
                const int64_t lo_k = hoff[m.row0 + R], hi_k = hoff[m.row0 + cuts.back()];
                if (R < cuts.back() - 1 && (hi_k - lo_k) * row_bytes > (int64_t)apanel_budget) cuts.push_back(R + 1);
            }
            cuts.push_back(0);
            for (size_t c = 0; c + 1 < cuts.size(); ++c)
                launches.push_back(Launch{i, 1, cuts[c + 1], cuts[c], 0, 0, 0, 0});
            g0 = i + 1;
            gk = 0;
        }
        if (g0 < nmat) whole(g0, nmat);
    }
    // the runs of every launch: row blocks from the last down, the matrices of a launch
    // interleaved (their q-th rows from the end side by side)
    int64_t maxk = 0;
    for (Launch& L : launches) {
        L.run0 = hruns.size();
        int64_t start = 0;
        int32_t depth = 0;
        for (int32_t i = L.mat0; i < L.mat0 + L.nm; ++i) depth = std::max(depth, std::min(hm[i].nR, L.R1) - L.R0);
        for (int32_t q = 0; q < depth; ++q)
            for (int32_t i = L.mat0; i < L.mat0 + L.nm; ++i) {
                const int32_t R = std::min(hm[i].nR, L.R1) - 1 - q;
                if (R < L.R0) continue;
                hruns.push_back(BsRun{start, i, R});
                start += hm[i].nR - R;
            }
        L.run1 = hruns.size();
        L.nit = start;
        L.aoff0 = hoff[hm[L.mat0].row0 + L.R0];
        const BsMat<T>& z = hm[L.mat0 + L.nm - 1];
        maxk = std::max(maxk, hoff[z.row0 + std::min(z.nR, L.R1)] - L.aoff0);
    }
    if ((e = cudaMemcpyAsync(p.runs, hruns.data(), hruns.size() * sizeof(BsRun), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return done(e);
    if ((e = scratch_alloc((void**)&p.A, (size_t)(maxk > 0 ? maxk : 1) * row_bytes, st)) != cudaSuccess)
        return done(e);
    if (prof) {
        ev.assign(2 * launches.size(), nullptr);
        for (auto& x : ev)
            if ((e = cudaEventCreate(&x)) != cudaSuccess) return done(e);
    }
    e = bs_enqueue<T>(p, err, exact, prof ? &ev : nullptr, st);
    if (prof && e == cudaSuccess && !ev.empty() && (e = cudaEventSynchronize(ev.back())) == cudaSuccess) {
        prof->bs_ms = 0.0;
        prof->bs_launches = 0;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) {
                prof->bs_ms += ms;
                prof->bs_launches += 1;
            }
        }
    }
    // (the host lists above are uploaded from pageable memory: staged before return)
    return done(e);
}

template <typename T>
cudaError_t bg_backsub(T* M, int64_t N, const uint32_t* rowflags, uint32_t* err, uint32_t* exact, size_t apanel_budget,
                       double* updates, FwProfile* prof, cudaStream_t st) {
    return bg_backsub_many<T>(std::vector<BsInput<T>>{BsInput<T>{M, N, rowflags}}, err, exact, apanel_budget, updates,
                              prof, st, nullptr);
}

template cudaError_t bg_backsub<float>(float*, int64_t, const uint32_t*, uint32_t*, uint32_t*, size_t, double*,
                                       FwProfile*, cudaStream_t);
template cudaError_t bg_backsub<int32_t>(int32_t*, int64_t, const uint32_t*, uint32_t*, uint32_t*, size_t, double*,
                                         FwProfile*, cudaStream_t);
template cudaError_t bg_backsub_many<float>(const std::vector<BsInput<float>>&, uint32_t*, uint32_t*, size_t, double*,
                                            FwProfile*, cudaStream_t, BsPlan<float>*);
template cudaError_t bg_backsub_many<int32_t>(const std::vector<BsInput<int32_t>>&, uint32_t*, uint32_t*, size_t,
                                              double*, FwProfile*, cudaStream_t, BsPlan<int32_t>*);

template cudaError_t launch_fill_marked<float>(float*, int64_t, const uint32_t*, cudaStream_t);
template cudaError_t launch_fill_marked<int32_t>(int32_t*, int64_t, const uint32_t*, cudaStream_t);

}  // namespace spq

namespace spq {
unsigned long long wait_bound_ns() { return g_wait_ns.load(); }
int wait_withhold() { return g_withhold.load(); }
}  // namespace spq

extern "C" void spq_test_backsub_wait(unsigned long long limit_ns, int32_t withhold) {
    spq::g_wait_ns.store(limit_ns > 0 ? limit_ns : spq::kWaitNs);
    spq::g_withhold.store(withhold != 0 ? 1 : 0);
}
