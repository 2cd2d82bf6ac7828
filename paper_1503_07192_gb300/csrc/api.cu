// C-ABI entry points and host orchestration of the build (Algorithm 1) and of queries
// (Algorithm 2).  The host only sizes and allocates the tables, orders the components
// and launches kernels; every per-vertex, per-edge and per-cell step runs on the GPU.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "order.h"

using namespace spq;

namespace spq {
extern std::atomic<unsigned long long> g_kernel_launches;
std::atomic<unsigned long long> g_kernel_launches{0};
void count_launches(int n) { g_kernel_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace spq

namespace spq {
spq_status read_opts(const spq_opts* in, spq_opts* o) {
    spq_opts_default(o);
    if (!in) return SPQ_OK;
    // earlier, shorter versions of the struct end before bg_method
    const int32_t v1 = (int32_t)offsetof(spq_opts, bg_method);
    if (in->struct_size < v1) return SPQ_EINVAL;
    memcpy(o, in, (size_t)std::min<int32_t>(in->struct_size, (int32_t)sizeof(spq_opts)));
    o->struct_size = (int32_t)sizeof(spq_opts);
    if (o->arith < SPQ_ARITH_AUTO || o->arith > SPQ_ARITH_F32) return SPQ_EINVAL;
    if (o->order < SPQ_ORDER_AUTO || o->order > SPQ_ORDER_VERTEX_DISSECTION) return SPQ_EINVAL;
    if (o->bg_method < SPQ_BG_AUTO || o->bg_method > SPQ_BG_ELIM || o->bg_panel_mib < 0) return SPQ_EINVAL;
    if (o->comp_method < SPQ_BG_AUTO || o->comp_method > SPQ_BG_ELIM) return SPQ_EINVAL;
    if (o->query_kernel != 0 && o->query_kernel != 1) return SPQ_EINVAL;
    return SPQ_OK;
}
}  // namespace spq

namespace {
thread_local int g_last_cuda = 0;
}  // namespace

namespace spq {
void note_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }
}  // namespace spq

namespace {


// Below this many pairs a query batch is answered in input order (no sort).
constexpr int64_t kGroupedMinQueries = 4096;

spq_status cuda_fail(cudaError_t e) {
    if (e == kWaitGaveUp) return SPQ_ETIMEOUT;
    g_last_cuda = (int)e;
    return SPQ_ECUDA;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stream-ordered temporaries released together (on scope exit).
struct Temps {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Temps(cudaStream_t s) : st(s) {}
    ~Temps() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = scratch_alloc((void**)p, count * sizeof(T), st);
        if (e == cudaSuccess) ptrs.push_back((void*)*p);
        return e;
    }
};

// The tables of a single build come from a library-owned stream-ordered memory pool per
// device that keeps freed memory for the next build (a 71 GB table costs tens of
// milliseconds to map and unmap); spq_release_cached_memory gives it back.
constexpr int kMaxDevices = 64;
cudaMemPool_t g_pools[kMaxDevices] = {};
std::mutex g_pool_mu;

cudaError_t table_pool(int dev, cudaMemPool_t* out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;  // never trimmed implicitly
        e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// Bytes the pool holds but no live table uses (free for the next build).
size_t pool_cached_bytes(int dev) {
    cudaMemPool_t pool;
    if (table_pool(dev, &pool) != cudaSuccess) return 0;
    uint64_t reserved = 0, used = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    return reserved > used ? (size_t)(reserved - used) : 0;
}

void free_handle_memory(spq_handle* h) {
    if (h->arena) {
        if (h->arena->refs.fetch_sub(1) == 1) {
            cudaFreeAsync(h->arena->base, 0);  // back to the pool
            cudaStreamSynchronize(0);
            delete h->arena;
        }
        h->arena = nullptr;
        return;
    }
    void* ps[] = {h->comp,   h->local,   h->descs,   h->nb,  h->bg_off, h->bgpos,  h->csize, h->apsp,
                  h->D,      h->err,     h->csr_rp,  h->csr_col, h->csr_w, h->vorder, h->vstart,
                  h->qstats};
    for (void* p : ps)
        if (p) cudaFreeAsync(p, 0);  // back to the pool
    cudaStreamSynchronize(0);
    for (cudaEvent_t& e : h->qev)
        if (e) cudaEventDestroy(e);
}

}  // namespace

size_t spq::pool_cached_bytes_current() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return pool_cached_bytes(dev);
}

// Temporaries of every entry point come from the same pool as the tables, so that the
// memory of one build or query batch is reused by the next instead of being unmapped at
// each synchronisation and mapped again.
cudaError_t spq::scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (e == cudaSuccess) e = table_pool(dev, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 4, pool, st);
}

namespace {

template <typename T>
cudaError_t dev_alloc(T** p, size_t count, size_t* total, cudaStream_t st) {
    if (count == 0) count = 1;
    *total += count * sizeof(T);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (e == cudaSuccess) e = table_pool(dev, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync((void**)p, count * sizeof(T), pool, st);
}

int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

// CUDA events bracketing the build stages (see spq_build_profile).
// ---- the build's autotuned knob ----
// How many bisection levels of the boundary graph's dissection become concurrent runs of
// elimination rounds (up to 2^depth leaf runs, each on its own stream).  Deeper levels
// give more and shorter runs, but more alignment padding, another frontier structure for
// the back-substitution, and more streams than the context may have hardware queues for;
// the best depth depends on the graph and the device.  Per device and size class of the
// boundary graph (bit length of |BG|), the first builds try the candidate depths in turn,
// each timed by the build's own stage events (the boundary graph's all-pairs stage), and
// later builds take the fastest.  Every depth gives the same distances (only the matrix
// order changes, and everything reaches the matrix through bgpos).
constexpr int kDepthCand[3] = {3, 4, 5};
struct DepthClass {
    double ms[3] = {-1.0, -1.0, -1.0};
    int next = 0;     // the next candidate to try
    int chosen = -1;  // the fastest, once all are measured
};
std::mutex g_depth_mu;
std::map<std::pair<int, int>, DepthClass> g_depth;

int depth_pick(int dev, int cls) {
    std::lock_guard<std::mutex> lk(g_depth_mu);
    const DepthClass& c = g_depth[{dev, cls}];
    return c.chosen >= 0 ? c.chosen : c.next;
}

void depth_report(int dev, int cls, int idx, double ms) {
    std::lock_guard<std::mutex> lk(g_depth_mu);
    DepthClass& c = g_depth[{dev, cls}];
    if (c.chosen >= 0 || idx != c.next || !(ms > 0.0)) return;  // (a concurrent build measured it)
    c.ms[idx] = ms;
    c.next = idx + 1;
    if (c.next == 3) {
        int b = 0;
        for (int i = 1; i < 3; ++i)
            if (c.ms[i] < c.ms[b]) b = i;
        c.chosen = b;
    }
}

struct StageEvents {
    cudaEvent_t ev[8] = {};
    bool ok = true;
    StageEvents() {
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) ok = false;
    }
    ~StageEvents() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
    void mark(int i, cudaStream_t st) {
        if (ok) cudaEventRecord(ev[i], st);
    }
    void collect(double* ms) {
        for (int i = 0; i < 7; ++i) {
            float t = 0.f;
            ms[i] = (ok && cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) ? (double)t : 0.0;
        }
        cudaGetLastError();
    }
};

struct BuildInputs {
    int32_t n;
    int64_t m;
    const int64_t* rp;
    const int32_t* col;
    const void* w;
    const int32_t* part;
    bool f32w;
};

// How the boundary graph's all-pairs distances are computed: Floyd-Warshall, or the
// elimination form of its rounds followed by back-substitution (elim.cu).
struct BgPlan {
    bool elim = false;
    uint32_t* rowflags = nullptr;  // R x R words (elimination only)
    size_t apanel_budget = 0;
    bool wait_failed = false;      // a bounded wait of the back-substitution gave up
    BgLayout layout;               // aligned pieces and their runs of rounds (elimination)
};

// Tables of Algorithm 1 in element type T: component blocks, their Floyd-Warshall,
// boundary-graph assembly and its all-pairs distances.  Sets *inexact if a float32 table
// holds a finite entry >= 2^24.
// Component tables APSP(C) in element type T (queued on st; no host wait).
// With elim, the components that comp_takes_elim selects by elimination in a dissection
// order (waits on the host), the others by Floyd-Warshall.  Sets h->comp_updates.
template <typename T>
cudaError_t build_comp_tables(spq_handle* h, const BuildInputs& in, int32_t max_n, bool elim, StageEvents& evs,
                              cudaStream_t st) {
    evs.mark(2, st);
    T* apsp = (T*)h->apsp;
    cudaError_t e;
    // (when every component takes the elimination form, its permutation back writes every
    //  cell of the tables: no initialisation in the local order)
    bool all_elim = elim;
    for (int32_t c = 0; c < h->k && all_elim; ++c)
        all_elim = h->h_descs[c].n == 0 || comp_takes_elim(h->h_csize[c], h->h_descs[c].n);
    if (!all_elim) {
        if ((e = launch_fill_blocks<T>(apsp, h->descs, h->k, st)) != cudaSuccess) return e;
        if ((e = launch_scatter_intra<T>(in.f32w, in.n, in.rp, in.col, in.w, in.part, h->local, h->descs, apsp,
                                         st)) != cudaSuccess)
            return e;
    }
    std::vector<MatDesc> fwd = h->h_descs;  // the Floyd-Warshall set (others: n = 0, skipped)
    double eu = 0.0;
    if (elim) {
        e = comp_tables_elim<T>(apsp, h->descs, h->h_descs, h->h_csize, h->k, in.n, in.rp, in.col, in.w, in.f32w,
                                in.part, h->local, h->vorder, h->vstart, h->csize, &eu, st);
        if (e != cudaSuccess) return e;
        for (int32_t c = 0; c < h->k; ++c)
            if (comp_takes_elim(h->h_csize[c], fwd[c].n)) fwd[c].n = 0;
    }
    int32_t max_fw = 0;
    double cu = 0.0;
    for (const MatDesc& d : fwd) {
        max_fw = std::max(max_fw, d.n);
        // per round: the diagonal tile, R - 1 row tiles, R(R - 1)/2 upper-triangle tiles
        const double R = (double)((d.n + kTile - 1) / kTile);
        cu += R * (1.0 + (R - 1.0) + R * (R - 1.0) / 2.0) * (double)kTile * kTile * kTile;
    }
    if (max_fw > 0 && (e = fw_batched<T>(apsp, h->descs, fwd.data(), h->k, max_fw, st)) != cudaSuccess) return e;
    h->comp_updates = cu + eu;
    evs.mark(3, st);
    return cudaSuccess;
}

// The boundary graph's table in element type T (after build_comp_tables<T>): assembly,
// all-pairs distances, and (check_exact) the exactness check of every float32 table.
template <typename T>
cudaError_t build_bg_tables(spq_handle* h, const BuildInputs& in, bool check_exact, bool skip_inf, bool profile,
                            uint32_t* d_flag, uint32_t* fw_scratch, BgPlan& plan, bool* inexact, StageEvents& evs,
                            cudaStream_t st) {
    *inexact = false;
    T* apsp = (T*)h->apsp;
    T* D = (T*)h->D;
    cudaError_t e;
    const int64_t R = (h->N + kTile - 1) / kTile;
    // elimination form with skipping: only the marked tiles and the diagonal are read
    // before the back-substitution writes every tile, so only those are initialised
    const bool fill_marked = plan.elim && skip_inf;
    if (h->N > 0) {
        if (plan.elim) {
            if ((e = cudaMemsetAsync(plan.rowflags, 0, (size_t)(R * R) * 4, st)) != cudaSuccess) return e;
            if ((e = launch_mark_bg_tiles(in.n, in.rp, in.col, in.part, h->local, h->nb, h->bg_off, h->bgpos, h->k,
                                          h->N, plan.rowflags, st)) != cudaSuccess)
                return e;
            // the separators' tiles, which concurrent runs of rounds update together, are
            // marked (and so initialised) from the start
            std::vector<int32_t> shared;
            for (const ElimTask& tk : plan.layout.tasks)
                if (!tk.deps.empty())
                    for (int32_t b = tk.lo; b < tk.hi; ++b) shared.push_back(b);
            if ((e = launch_mark_pairs(shared, h->N, plan.rowflags, st)) != cudaSuccess) return e;
        }
        if ((e = fill_marked ? launch_fill_marked<T>(D, h->N, plan.rowflags, st) : launch_bg_fill<T>(D, h->N, st)) !=
            cudaSuccess)
            return e;
        if ((e = launch_bg_clique<T>(apsp, h->descs, h->nb, h->bg_off, h->bgpos, h->k, D, h->N, st)) != cudaSuccess)
            return e;
        if ((e = launch_bg_inter<T>(in.f32w, in.n, in.rp, in.col, in.w, in.part, h->local, h->bg_off, h->bgpos, D,
                                    h->N, st)) != cudaSuccess)
            return e;
    }
    evs.mark(4, st);
    if (check_exact && (e = cudaMemsetAsync(d_flag, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    // the elimination stores the float32 boundary-graph table as int32 itself (checked)
    const bool d_converted = plan.elim && check_exact && h->N > 0;
    if (h->N > 0 && !plan.elim) {
        if ((e = fw_single<T>(D, h->N, skip_inf, fw_scratch, nullptr, &h->bg_updates, profile ? &h->fwprof : nullptr,
                              st)) != cudaSuccess)
            return e;
    } else if (h->N > 0) {
        double fwd = 0.0, bs = 0.0;
        if ((e = fw_single<T>(D, h->N, skip_inf, fw_scratch, plan.rowflags, &fwd, profile ? &h->fwprof : nullptr,
                              st, plan.layout.tasks.empty() ? nullptr : &plan.layout.tasks)) != cudaSuccess)
            return e;
        if ((e = bg_backsub<T>(D, h->N, plan.rowflags, h->err, d_converted ? d_flag : nullptr, plan.apanel_budget, &bs,
                               profile ? &h->fwprof : nullptr, st)) != cudaSuccess)
            return e;
        h->bg_updates = fwd + bs;
        uint32_t bits = 0;
        if ((e = cudaMemcpyAsync(&bits, h->err, sizeof(bits), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (bits & kErrWait) {
            plan.wait_failed = true;
            return cudaSuccess;
        }
    }
    evs.mark(5, st);
    if (check_exact) {
        // the float32 tables become int32 ones (every entry below 2^24 is an exact integer)
        if ((e = launch_check_convert((float*)h->apsp, h->apsp_elems, d_flag, st)) != cudaSuccess) return e;
        if (h->N > 0 && !d_converted && (e = launch_check_convert((float*)h->D, h->N * h->N, d_flag, st)) != cudaSuccess)
            return e;
        uint32_t f = 0;
        if ((e = cudaMemcpyAsync(&f, d_flag, sizeof(f), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        *inexact = (f & kErrExact) != 0;
    }
    evs.mark(6, st);
    return cudaSuccess;
}

spq_status build_impl(int32_t n, const int64_t* row_ptr, const int32_t* col, const void* w, spq_dtype wt,
                      const int32_t* part, int32_t k, const spq_opts& opts, cudaStream_t st, spq_handle* h) {
    Temps tmp(st);
    StageEvents evs;
    // ---- inputs on the device ----
    const bool rp_dev = is_device_ptr(row_ptr);
    int64_t rp_ends[2] = {0, 0};
    if (rp_dev) {
        CK(cudaMemcpyAsync(&rp_ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&rp_ends[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        rp_ends[0] = row_ptr[0];
        rp_ends[1] = row_ptr[n];
    }
    const int64_t m = rp_ends[1];
    if (rp_ends[0] != 0 || m < 0 || m > INT32_MAX) return SPQ_EINVAL;
    if (m > 0 && (!col || !w)) return SPQ_EINVAL;
    const size_t wsz = 4;
    const int64_t* d_rp = row_ptr;
    const int32_t* d_col = col;
    const void* d_w = w;
    const int32_t* d_part = part;
    if (!rp_dev) {
        int64_t* p;
        CK(tmp.alloc(&p, (size_t)n + 1));
        CK(cudaMemcpyAsync(p, row_ptr, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        d_rp = p;
    }
    if (m > 0 && !is_device_ptr(col)) {
        int32_t* p;
        CK(tmp.alloc(&p, (size_t)m));
        CK(cudaMemcpyAsync(p, col, (size_t)m * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        d_col = p;
    }
    if (m > 0 && !is_device_ptr(w)) {
        uint32_t* p;
        CK(tmp.alloc(&p, (size_t)m));
        CK(cudaMemcpyAsync(p, w, (size_t)m * wsz, cudaMemcpyHostToDevice, st));
        d_w = p;
    }
    if (!is_device_ptr(part)) {
        int32_t* p;
        CK(tmp.alloc(&p, (size_t)n));
        CK(cudaMemcpyAsync(p, part, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        d_part = p;
    }
    const bool f32w = wt == SPQ_F32;
    evs.mark(0, st);

    // ---- validation, boundary flags, per-component counts (GPU) ----
    uint8_t* d_bflag;
    int32_t* d_cnt;
    uint32_t* d_flag;
    CK(tmp.alloc(&d_bflag, (size_t)n));
    CK(tmp.alloc(&d_cnt, 2 * (size_t)k));
    CK(tmp.alloc(&d_flag, 1));
    CK(cudaMemsetAsync(d_cnt, 0, 2 * (size_t)k * sizeof(int32_t), st));
    CK(cudaMemsetAsync(d_flag, 0, sizeof(uint32_t), st));
    CK(launch_validate(f32w, n, m, d_rp, d_col, d_w, d_part, k, d_bflag, d_cnt, d_cnt + k, d_flag, st));
    evs.mark(1, st);
    std::vector<int32_t> cnt(2 * (size_t)k);
    uint32_t flag = 0;
    CK(cudaMemcpyAsync(cnt.data(), d_cnt, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&flag, d_flag, sizeof(flag), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag != 0) return SPQ_EINVAL;

    // ---- sizes and offsets of the tables (host, O(k)) ----
    h->h_csize.assign(cnt.begin(), cnt.begin() + k);
    h->h_nb.assign(cnt.begin() + k, cnt.end());
    std::vector<int32_t> vstart(k);
    h->h_descs.resize(k);
    int64_t acc = 0, vs = 0;
    int32_t max_n = 0;
    for (int32_t c = 0; c < k; ++c) {
        vstart[c] = (int32_t)vs;
        vs += h->h_csize[c];
        int32_t ld = (int32_t)round_up(h->h_csize[c], 4);
        h->h_descs[c] = MatDesc{acc, ld, 0};
        acc += (int64_t)ld * ld;
        max_n = std::max(max_n, ld);
    }
    h->apsp_elems = acc;
    // boundary slots, numbered component by component (their matrix positions, bgpos,
    // are chosen after the reordering below)
    h->h_bgoff.assign(k, 0);
    int64_t bo = 0;
    for (int32_t c = 0; c < k; ++c) {
        h->h_bgoff[c] = (int32_t)bo;
        bo += h->h_nb[c];
    }
    h->nbg = bo;
    h->max_nb = k > 0 ? *std::max_element(h->h_nb.begin(), h->h_nb.end()) : 0;
    // matrix order: the slots, plus (elimination form) one alignment gap of < 128 per
    // aligned piece start
    const bool may_elim = opts.bg_method != SPQ_BG_FW && bo > 0;
    const int64_t max_runs = ((int64_t)2 << kMaxRunDepth) - 1;
    const int64_t n_max = round_up(bo + (may_elim ? max_runs * (kTile - 1) : 0), 4);
    if (n_max > 0 && n_max * n_max > (int64_t)1 << 40) return SPQ_ENOMEM;

    // ---- memory check (with the largest matrix order), then allocation ----
    const int64_t hist_words = radix_hist_words(n);
    const size_t panel_cap = opts.bg_panel_mib > 0 ? ((size_t)opts.bg_panel_mib << 20) : ((size_t)1 << 30);
    int64_t nR = (n_max + kTile - 1) / kTile;
    const int64_t fw_words_max = n_max > 0 ? fw_single_scratch_words(n_max) : 1;
    size_t apanel_budget = std::min<size_t>(panel_cap, 4 * (size_t)n_max * (size_t)n_max + (1u << 20));
    // elimination scratch: per-round row flags, back-substitution bookkeeping, A panels,
    // and per-run compaction lists
    const size_t elim_bytes = may_elim ? 4 * (size_t)(nR * nR) + bg_backsub_scratch_bytes(n_max) + apanel_budget +
                                             (size_t)max_runs * 4 * (size_t)(6 * nR + 10)
                                       : 0;
    // (+ the component tables in dissection order, a second copy, for their elimination)
    const size_t comp_elim_bytes = opts.comp_method != SPQ_BG_FW ? 4 * (size_t)h->apsp_elems + 8 * (size_t)n : 0;
    size_t need = 4 * (size_t)h->apsp_elems + comp_elim_bytes + 4 * (size_t)n_max * (size_t)n_max + 8 * (size_t)n +
                  (size_t)k * (sizeof(MatDesc) + 16) + 16 * (size_t)n + 4 * (size_t)(fw_words_max + hist_words) +
                  8 * ((size_t)n + 1) + 8 * (size_t)m + 4 * (size_t)n + elim_bytes + (64u << 20);
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    free_b += pool_cached_bytes(h->device);
    if (need > free_b) return SPQ_ENOMEM;
    size_t bytes = 0;
    CK(dev_alloc(&h->comp, (size_t)n, &bytes, st));
    CK(dev_alloc(&h->local, (size_t)n, &bytes, st));
    CK(dev_alloc(&h->descs, (size_t)k, &bytes, st));
    CK(dev_alloc(&h->nb, (size_t)k, &bytes, st));
    CK(dev_alloc(&h->bg_off, (size_t)k, &bytes, st));
    CK(dev_alloc(&h->bgpos, (size_t)h->nbg, &bytes, st));
    CK(dev_alloc(&h->csize, (size_t)k, &bytes, st));
    CK(dev_alloc(&h->err, 4, &bytes, st));
    CK(dev_alloc(&h->csr_rp, (size_t)n + 1, &bytes, st));
    CK(dev_alloc(&h->csr_col, (size_t)m, &bytes, st));
    CK(dev_alloc((uint32_t**)&h->csr_w, (size_t)m, &bytes, st));
    CK(dev_alloc(&h->vorder, (size_t)n, &bytes, st));
    CK(dev_alloc(&h->vstart, (size_t)k, &bytes, st));
    h->m = m;
    CK(dev_alloc((uint32_t**)&h->apsp, (size_t)h->apsp_elems, &bytes, st));
    CK(cudaMemsetAsync(h->err, 0, 4 * sizeof(uint32_t), st));
    CK(cudaMemcpyAsync(h->descs, h->h_descs.data(), (size_t)k * sizeof(MatDesc), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->nb, h->h_nb.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->bg_off, h->h_bgoff.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->csize, h->h_csize.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    int32_t* d_vstart;
    CK(tmp.alloc(&d_vstart, (size_t)k));
    CK(cudaMemcpyAsync(d_vstart, vstart.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st));

    // ---- vertex reordering (Sec. 4, Fig. 1): stable sort by (component, interior) ----
    {
        uint32_t *k0, *v0, *k1, *v1, *hist;
        CK(tmp.alloc(&k0, (size_t)n));
        CK(tmp.alloc(&v0, (size_t)n));
        CK(tmp.alloc(&k1, (size_t)n));
        CK(tmp.alloc(&v1, (size_t)n));
        CK(tmp.alloc(&hist, (size_t)hist_words));
        CK(launch_make_keys(n, d_part, d_bflag, k0, v0, st));
        bool in_k1 = false;
        int key_bits = bits_for(2 * (uint64_t)k - 1);
        CK(radix_sort_pairs(k0, v0, k1, v1, hist, n, key_bits, &in_k1, st));
        CK(launch_assign_local(n, in_k1 ? v1 : v0, d_part, d_vstart, h->local, h->comp, st));
        // kept for path walks: vertices in (component, local) order, component starts, CSR
        CK(cudaMemcpyAsync(h->vorder, in_k1 ? v1 : v0, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(h->vstart, d_vstart, (size_t)k * 4, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(h->csr_rp, d_rp, ((size_t)n + 1) * 8, cudaMemcpyDeviceToDevice, st));
        if (m > 0) {
            CK(cudaMemcpyAsync(h->csr_col, d_col, (size_t)m * 4, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(h->csr_w, d_w, (size_t)m * 4, cudaMemcpyDeviceToDevice, st));
        }
    }

    // ---- the component tables go to the GPU while the host orders the boundary slots ----
    BgPlan plan;
    BoundaryPairs bpairs;
    if (h->nbg > 0) {
        spq_status s = boundary_pairs(n, m, d_rp, d_col, d_part, h->local, h->bg_off, k, h->h_nb,
                                      (spq_order)opts.order, st, &bpairs);
        if (s != SPQ_OK) return s;
    }
    BuildInputs in{n, m, d_rp, d_col, d_w, d_part, f32w};
    const bool skip = opts.skip_inf_tiles != 0;
    const bool prof = opts.profile_kernels != 0;
    // float32 arithmetic first (exact below 2^24, checked), int32 if asked or if the check fails
    const bool first_f32 = f32w || opts.arith != SPQ_ARITH_I32;
    const bool comp_elim = opts.comp_method != SPQ_BG_FW;
    // the boundary slots' order on a host thread meanwhile (the component elimination
    // waits on the host for its own bookkeeping)
    std::vector<int32_t> bgpos;
    spq_status order_status = SPQ_OK;
    std::thread order_thread;
    // the autotuned depth of concurrent runs (the root split needs two pieces of 16 tiles)
    const int tune_cls = bits_for((uint64_t)h->nbg);
    const int depth_idx = (may_elim && h->nbg >= 2 * 16 * kTile) ? depth_pick(h->device, tune_cls) : -1;
    if (depth_idx >= 0) plan.layout.depth = kDepthCand[depth_idx];
    if (h->nbg > 0)
        order_thread = std::thread([&]() {
            order_status = boundary_order_from(k, h->h_nb, bpairs, (spq_order)opts.order, &bgpos, &h->order_method,
                                               may_elim ? &plan.layout : nullptr);
        });
    struct Join {
        std::thread& t;
        ~Join() {
            if (t.joinable()) t.join();
        }
    } join_order{order_thread};
    if (first_f32)
        CK(build_comp_tables<float>(h, in, max_n, comp_elim, evs, st));
    else
        CK(build_comp_tables<int32_t>(h, in, max_n, comp_elim, evs, st));
    if (order_thread.joinable()) order_thread.join();
    if (h->nbg > 0) {
        if (order_status != SPQ_OK) return order_status;
        CK(cudaMemcpyAsync(h->bgpos, bgpos.data(), bgpos.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // bgpos (host) goes out of scope
    }
    h->N = round_up(plan.layout.npad > 0 ? plan.layout.npad : h->nbg, 4);
    if (h->N > 0) CK(dev_alloc((uint32_t**)&h->D, (size_t)(h->N * h->N), &bytes, st));
    h->bytes = bytes;
    nR = (h->N + kTile - 1) / kTile;
    const int64_t fw_words = h->N > 0 ? fw_single_scratch_words(h->N) : 1;
    apanel_budget = std::min<size_t>(panel_cap, 4 * (size_t)h->N * (size_t)h->N + (1u << 20));

    // ---- boundary graph, its all-pairs distances ----
    uint32_t* fw_scratch;
    CK(tmp.alloc(&fw_scratch, (size_t)fw_words));
    // elimination + back-substitution pays off in a dissection order (small frontiers);
    // in the id order every row's frontier is most of the matrix
    plan.elim = may_elim && (opts.bg_method == SPQ_BG_ELIM || h->order_method != 0);
    h->bg_method = plan.elim ? SPQ_BG_ELIM : SPQ_BG_FW;
    if (plan.elim) {
        CK(tmp.alloc(&plan.rowflags, (size_t)(nR * nR)));
        plan.apanel_budget = apanel_budget;
    }
    if (f32w) {
        h->f32store = true;
        h->arith = SPQ_ARITH_F32;
        bool inexact = false;
        CK(build_bg_tables<float>(h, in, false, skip, prof, d_flag, fw_scratch, plan, &inexact, evs, st));
        if (plan.wait_failed) return SPQ_ETIMEOUT;
    } else {
        bool inexact = false;
        if (first_f32) {
            h->f32store = true;
            h->arith = SPQ_ARITH_F32;
            CK(build_bg_tables<float>(h, in, true, skip, prof, d_flag, fw_scratch, plan, &inexact, evs, st));
            if (plan.wait_failed) return SPQ_ETIMEOUT;
        }
        h->f32store = false;  // converted to int32 by the exactness check
        if (!first_f32 || inexact) {
            h->arith = SPQ_ARITH_I32;
            if (inexact) CK(build_comp_tables<int32_t>(h, in, max_n, comp_elim, evs, st));
            CK(build_bg_tables<int32_t>(h, in, false, skip, prof, d_flag, fw_scratch, plan, &inexact, evs, st));
            if (plan.wait_failed) return SPQ_ETIMEOUT;
        }
    }
    if (opts.profile_kernels && h->nbg > 0) {  // timing of the staged grouped query kernel
        CK(dev_alloc(&h->qstats, 2, &bytes, st));
        CK(cudaEventCreate(&h->qev[0]));
        CK(cudaEventCreate(&h->qev[1]));
        h->bytes = bytes;
    }
    evs.mark(7, st);
    CK(cudaStreamSynchronize(st));
    evs.collect(h->prof_ms);
    if (depth_idx >= 0 && plan.elim && plan.layout.tasks.size() > 1)
        depth_report(h->device, tune_cls, depth_idx, h->prof_ms[4]);
    return SPQ_OK;
}

}  // namespace

extern "C" {

void spq_opts_default(spq_opts* o) {
    if (!o) return;
    o->struct_size = (int32_t)sizeof(spq_opts);
    o->arith = SPQ_ARITH_AUTO;
    o->order = SPQ_ORDER_AUTO;
    o->skip_inf_tiles = 1;
    o->profile_kernels = 0;
    o->query_grouped = 1;
    o->bg_method = SPQ_BG_AUTO;
    o->bg_panel_mib = 0;
    o->comp_method = SPQ_BG_AUTO;
    o->query_kernel = 0;
}

spq_status spq_build(int32_t n, const int64_t* row_ptr, const int32_t* col, const void* w, spq_dtype wt,
                     const int32_t* part, int32_t k, const spq_opts* opts, void* stream, spq_handle** out) {
    if (!out) return SPQ_EINVAL;
    *out = nullptr;
    if (n < 1 || k < 1 || !row_ptr || !part) return SPQ_EINVAL;
    if (wt != SPQ_I32 && wt != SPQ_F32) return SPQ_EINVAL;
    spq_opts o;
    if (spq_status so = read_opts(opts, &o)) return so;
    spq_handle* h = new (std::nothrow) spq_handle();
    if (!h) return SPQ_ENOMEM;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e);
    }
    h->n = n;
    h->k = k;
    h->wt = wt;
    h->query_grouped = o.query_grouped;
    h->query_kernel = o.query_kernel;
    spq_status s = build_impl(n, row_ptr, col, w, wt, part, k, o, (cudaStream_t)stream, h);
    if (s != SPQ_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        free_handle_memory(h);
        delete h;
        return s;
    }
    *out = h;
    return SPQ_OK;
}

spq_status spq_query(spq_handle* h, const int32_t* pairs, int64_t q, void* dist_out, void* stream) {
    if (!h || q < 0) return SPQ_EINVAL;
    if (q == 0) return SPQ_OK;
    if (!pairs || !dist_out || !on_handle_device(h)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool pd = is_device_ptr(pairs), od = is_device_ptr(dist_out);
    if (pd != od) return SPQ_EINVAL;
    const bool out_f32 = h->wt == SPQ_F32;
    Temps tmp(st);
    // the grouped form sorts the pairs by component pair in stream-ordered scratch
    uint32_t* scratch = nullptr;
    if (h->query_grouped && q >= kGroupedMinQueries && h->k <= 65535)
        CK(tmp.alloc(&scratch, (size_t)query_scratch_words(q)));
    auto launch = [&](const int32_t* p, void* o) -> cudaError_t {
        QueryCtx<int32_t> ci;
        QueryCtx<float> cf;
        bool f32store = false, of32 = false;
        int32_t k = 0;
        handle_query_view(h, &ci, &cf, &f32store, &of32, &k);
        return f32store ? launch_query<float>(cf, p, q, o, out_f32, (uint32_t)k, scratch, st)
                        : launch_query<int32_t>(ci, p, q, o, out_f32, (uint32_t)k, scratch, st);
    };
    if (pd) {
        if (((uintptr_t)pairs & 7u) || ((uintptr_t)dist_out & 3u)) return SPQ_EINVAL;
        CK(launch(pairs, dist_out));
        return SPQ_OK;
    }
    int32_t* dp;
    int32_t* dout;
    CK(tmp.alloc(&dp, 2 * (size_t)q));
    CK(tmp.alloc(&dout, (size_t)q));
    CK(cudaMemcpyAsync(dp, pairs, 2 * (size_t)q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(launch(dp, dout));
    CK(cudaMemcpyAsync(dist_out, dout, (size_t)q * 4, cudaMemcpyDeviceToHost, st));
    uint32_t f = 0;
    CK(cudaMemcpyAsync(&f, h->err, sizeof(f), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (f & kErrPair) {
        CK(cudaMemsetAsync(h->err, 0, sizeof(uint32_t), st));
        CK(cudaStreamSynchronize(st));
        return SPQ_EINVAL;
    }
    return SPQ_OK;
}

spq_status spq_query_status(spq_handle* h, void* stream) {
    if (!h || !on_handle_device(h)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t f = 0;
    CK(cudaMemcpyAsync(&f, h->err, sizeof(f), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (f & (kErrPair | kErrWalk)) {
        CK(cudaMemsetAsync(h->err, 0, sizeof(uint32_t), st));
        CK(cudaStreamSynchronize(st));
        return (f & kErrPair) ? SPQ_EINVAL : SPQ_ETIMEOUT;
    }
    return SPQ_OK;
}

void spq_free(spq_handle* h) {
    if (!h || h->plan_owned) return;
    cudaDeviceSynchronize();
    free_handle_memory(h);
    delete h;
}

void spq_release_cached_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    cudaDeviceSynchronize();
    for (int d = 0; d < kMaxDevices; ++d)
        if (g_pools[d]) cudaMemPoolTrimTo(g_pools[d], 0);
}

const char* spq_strerror(spq_status s) {
    switch (s) {
        case SPQ_OK: return "success";
        case SPQ_EINVAL: return "invalid argument or malformed graph, partition or query pair";
        case SPQ_ENOMEM: return "not enough device (or host) memory for the tables";
        case SPQ_ECUDA: return "CUDA runtime error";
        case SPQ_ETIMEOUT: return "bounded device-side wait ran out";
        case SPQ_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

int spq_last_cuda_error(void) { return g_last_cuda; }

size_t spq_footprint_bytes(const spq_handle* h) { return h ? h->bytes : 0; }

void spq_stats(const spq_handle* h, int64_t* n_bg, double* comp_updates, double* bg_updates, int32_t* arith) {
    if (!h) return;
    if (n_bg) *n_bg = h->nbg;
    if (comp_updates) *comp_updates = h->comp_updates;
    if (bg_updates) *bg_updates = h->bg_updates;
    if (arith) *arith = h->arith;
}

int32_t spq_build_profile(const spq_handle* h, double* ms, int32_t count) {
    if (!h || !ms || count <= 0) return 0;
    double v[15];
    for (int i = 0; i < 6; ++i) v[i] = h->prof_ms[i];
    v[6] = h->fwprof.p3_ms;
    v[7] = (double)h->fwprof.p3_launches;
    v[8] = h->fwprof.p3_updates;
    v[9] = (double)h->order_method;
    v[10] = (double)h->bg_method;
    v[11] = h->fwprof.bs_ms;
    v[12] = h->fwprof.bs_updates;
    v[13] = h->fwprof.bs_items;
    v[14] = (double)h->fwprof.bs_launches;
    int32_t c = count < 15 ? count : 15;
    for (int32_t i = 0; i < c; ++i) ms[i] = v[i];
    return c;
}

unsigned long long spq_kernel_launches(void) { return spq::g_kernel_launches.load(); }

int32_t spq_build_tuning(int32_t* keys, int32_t* depths, double* ms, int32_t cap) {
    std::lock_guard<std::mutex> lk(g_depth_mu);
    int32_t n = 0;
    for (const auto& kv : g_depth) {
        if (n < cap) {
            if (keys) keys[n] = kv.first.first * 256 + kv.first.second;
            if (depths) depths[n] = kv.second.chosen >= 0 ? kDepthCand[kv.second.chosen] : -1;
            if (ms)
                for (int i = 0; i < 3; ++i) ms[3 * n + i] = kv.second.ms[i];
        }
        ++n;
    }
    return n;
}

spq_status spq_query_profile(const spq_handle* h, double* kernel_ms, double* updates, double* bytes) {
    if (!h || !h->qstats || !h->qprof_ran) return SPQ_EUNSUPPORTED;
    unsigned long long st[2] = {0, 0};
    float ms = 0.f;
    CK(cudaEventSynchronize(h->qev[1]));
    CK(cudaEventElapsedTime(&ms, h->qev[0], h->qev[1]));
    CK(cudaMemcpy(st, h->qstats, sizeof(st), cudaMemcpyDeviceToHost));
    if (kernel_ms) *kernel_ms = ms;
    if (updates) *updates = (double)st[0];
    if (bytes) *bytes = (double)st[1];
    return SPQ_OK;
}

int spq_pool_usage(int device, unsigned long long* used, unsigned long long* reserved) {
    cudaMemPool_t pool;
    cudaError_t e = table_pool(device, &pool);
    uint64_t u = 0, r = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
    if (used) *used = u;
    if (reserved) *reserved = r;
    return (int)e;
}

spq_status spq_get_meta(const spq_handle* h, int32_t* comp, int32_t* local, int32_t* csize, int32_t* nb,
                        int32_t* bg_off, void* stream) {
    if (!h || !on_handle_device(h)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    struct Item {
        int32_t* dst;
        const void* src;
        size_t bytes;
        bool src_dev;
    } items[] = {{comp, h->comp, (size_t)h->n * 4, true},
                 {local, h->local, (size_t)h->n * 4, true},
                 {csize, h->h_csize.data(), (size_t)h->k * 4, false},
                 {nb, h->h_nb.data(), (size_t)h->k * 4, false},
                 {bg_off, h->h_bgoff.data(), (size_t)h->k * 4, false}};
    for (auto& it : items) {
        if (!it.dst) continue;
        CK(cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDefault, st));
    }
    CK(cudaStreamSynchronize(st));
    return SPQ_OK;
}

spq_status spq_get_apsp(const spq_handle* h, int32_t c, void* out, void* stream) {
    if (!h || c < 0 || c >= h->k || !out || !on_handle_device(h)) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t sz = h->h_csize[c];
    if (sz == 0) return SPQ_OK;
    const MatDesc d = h->h_descs[c];
    const void* src = (const char*)h->apsp + d.off * 4;
    return copy_table_out(h->f32store && h->wt == SPQ_I32, src, sz, sz, d.n, nullptr, out, st) == cudaSuccess
               ? SPQ_OK
               : cuda_fail(cudaGetLastError());
}

spq_status spq_get_bg(const spq_handle* h, void* out, void* stream) {
    if (!h || !out || !on_handle_device(h)) return SPQ_EINVAL;
    if (h->nbg == 0) return SPQ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return copy_table_out(h->f32store && h->wt == SPQ_I32, h->D, h->nbg, h->nbg, h->N, h->bgpos, out, st) == cudaSuccess
               ? SPQ_OK
               : cuda_fail(cudaGetLastError());
}

}  // extern "C"

namespace spq {

bool on_handle_device(const spq_handle* h) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return dev == h->device;
}

// Read-only view of a handle's device tables for entry points defined in other files.
void handle_query_view(const spq_handle* h, QueryCtx<int32_t>* ci, QueryCtx<float>* cf, bool* f32store, bool* out_f32,
                       int32_t* k) {
    *ci = QueryCtx<int32_t>{h->n,      h->comp,   h->local, h->descs, h->nb, h->bg_off, h->bgpos, (const int32_t*)h->apsp,
                            (const int32_t*)h->D, h->N, h->err, h->query_kernel == 0 ? 1 : 0, h->max_nb};
    *cf = QueryCtx<float>{h->n,    h->comp, h->local, h->descs, h->nb, h->bg_off, h->bgpos, (const float*)h->apsp,
                          (const float*)h->D, h->N, h->err, h->query_kernel == 0 ? 1 : 0, h->max_nb};
    // float32 arithmetic of an int32 graph passed the exactness check: every finite entry
    // of the (converted) int32 tables is below 2^24
    ci->exact24 = (h->wt == SPQ_I32 && !h->f32store && h->arith == SPQ_ARITH_F32) ? 1 : 0;
    if (h->qstats) {
        spq_handle* m = const_cast<spq_handle*>(h);
        m->qprof_ran = true;
        ci->qev = cf->qev = m->qev;
        ci->qstats = cf->qstats = m->qstats;
    }
    *f32store = h->f32store;
    *out_f32 = h->wt == SPQ_F32;
    *k = h->k;
}

}  // namespace spq
