// Many graphs at once: spq_build_many (Algorithm 1 for a batch of independent
// instances) and spq_query_many (Algorithm 2 for a query stream per instance).
//
// The instances share every launch where the work allows: one validation readback, one
// device arena for all tables, one stable sort over every instance's vertices, one
// readback of every instance's component adjacency (the host orders the instances'
// boundary vertices in parallel threads), the component Floyd-Warshall of all
// components of all instances in the same launches, and the boundary-graph
// Floyd-Warshall of all instances round by round in the same launches (each instance
// with its own list of tiles with a finite pivot panel).  The per-instance work left is
// a handful of O(n + m) kernels (edge scatter, boundary-graph assembly).
//
// Instances with a large boundary graph take the elimination form instead, which needs
// a fraction of the Floyd-Warshall updates there, batched the same way: the forward
// rounds (restricted to the trailing tiles, in a vertex nested-dissection order) of all
// of them in the same launches, then one persistent back-substitution over all their
// tiles, their rows interleaved so that their dependency chains overlap.  Both sets of
// instances are computed side by side on two streams.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "spq_bench.h"
#include "order.h"

using namespace spq;

namespace {

thread_local int g_batch_cuda_error = 0;

// Boundary-graph order from which an instance of a batch takes the elimination form by
// default: below it the batched Floyd-Warshall rounds cost less than the latency of the
// elimination's own rounds and back-substitution.
constexpr int64_t kBatchElimMin = 4096;

spq_status batch_cuda_fail(cudaError_t e) {
    if (e == kWaitGaveUp) return SPQ_ETIMEOUT;
    g_batch_cuda_error = (int)e;
    note_cuda_error(e);  // (spq_last_cuda_error)
    return SPQ_ECUDA;
}

#define BCK(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return batch_cuda_fail(e_); \
    } while (0)

bool dev_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct TempList {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit TempList(cudaStream_t s) : st(s) {}
    ~TempList() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t count) {
        *p = nullptr;
        cudaError_t e = scratch_alloc((void**)p, (count ? count : 1) * sizeof(T), st);
        if (e == cudaSuccess) ptrs.push_back((void*)*p);
        return e;
    }
};

// keys[vbase + v] = 2 * (kbase + part[v]) + (interior ? 1 : 0), vals = vbase + v.
__global__ void k_make_keys_many(int32_t n, const int32_t* __restrict__ part, const uint8_t* __restrict__ bflag,
                                 uint32_t kbase, uint32_t vbase, uint32_t* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
    const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    keys[vbase + v] = 2u * (kbase + (uint32_t)part[v]) + (bflag[v] ? 0u : 1u);
    vals[vbase + v] = vbase + (uint32_t)v;
}

// After the stable sort by (global component, interior): the vertex at sorted position
// pos gets its index inside its component and its instance-local component id.
__global__ void k_assign_local_many(int64_t ntot, const uint32_t* __restrict__ skeys,
                                    const uint32_t* __restrict__ svals, const int64_t* __restrict__ cstart,
                                    const int32_t* __restrict__ ckbase, int32_t* __restrict__ local,
                                    int32_t* __restrict__ comp) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= ntot) return;
    const uint32_t gv = svals[pos];
    const uint32_t gc = skeys[pos] >> 1;
    local[gv] = (int32_t)(pos - cstart[gc]);
    comp[gv] = (int32_t)gc - ckbase[gc];
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace {

// One instance of the batch: its device inputs and the place of its tables.
struct Inst {
    int32_t n = 0, k = 0;
    int64_t m = 0;
    const int64_t* rp = nullptr;
    const int32_t* col = nullptr;
    const void* w = nullptr;
    const int32_t* part = nullptr;
    int64_t vbase = 0, kbase = 0, mbase = 0, slotbase = 0;  // offsets in the batch-wide arrays
    int64_t apsp_off = 0, apsp_elems = 0, d_off = 0, N = 0, nbg = 0;
    int32_t max_ld = 0;
    bool elim = false;  // boundary graph by elimination + back-substitution
    std::vector<int32_t> csize, nb, bgoff;
    std::vector<MatDesc> descs;  // relative to the instance's own APSP base
};

// Batch-wide device arrays (all inside the arena).
struct BatchPtrs {
    int32_t* comp = nullptr;
    int32_t* local = nullptr;
    MatDesc* descs = nullptr;
    int32_t* nb = nullptr;
    int32_t* bgoff = nullptr;
    int32_t* csize = nullptr;
    int32_t* bgpos = nullptr;
    uint32_t* err = nullptr;
    uint32_t* tables = nullptr;  // every APSP(C), then every boundary-graph matrix
    int64_t table_elems = 0;
};

// The instances whose boundary graph takes the elimination form: their matrices'
// descriptors (device), the forward rounds' scratch, the A-panel budget of the
// back-substitution and its status word.
struct BatchElim {
    int dev = 0;
    int32_t n = 0, max_N = 0;
    MatDesc* descs = nullptr;
    uint32_t* scratch = nullptr;
    uint32_t* err = nullptr;
    size_t panel_cap = 0;
};

// The components whose tables take the elimination form (comp_takes_elim) across the
// batch: their global indices and descriptors, per-component vertex starts (within the
// instance and in the batch), the sorted vertex array, and the scratch of the dissection
// order and of the tables in that order.
struct CompElim {
    int32_t nsel = 0;
    std::vector<MatDesc> ed;           // global descriptors of the selected components
    int32_t* d_sel = nullptr;
    MatDesc* d_ed = nullptr;
    int32_t* vstart_local = nullptr;   // [ktot]: start of component c in its instance
    int32_t* vstart_global = nullptr;  // [ktot]: the same in the batch's sorted order
    const int32_t* sorted_v = nullptr; // [ntot]: batch vertex ids by (component, local)
    int32_t* ndpos = nullptr;          // [ntot]
    int32_t* vpos = nullptr;           // [ntot]
    void* P = nullptr;                 // the component tables in dissection order
    NdGraph* d_graphs = nullptr;       // [G]: the instances' CSR and numbering offsets
    int32_t* d_cgraph = nullptr;       // [ktot]: instance of each component
    int64_t ktot = 0;
};

// The weight-dependent launches of a batched build in element type T, kept for replay
// (build plans): the components' elimination, the Floyd-Warshall round lists, the
// boundary graphs' back-substitution, and the second stream of the boundary graphs'
// Floyd-Warshall with its fork / join events.  Recorded by the first build (ready = false
// on entry), replayed by a stream capture (ready = true: no host step, no allocation).
template <typename T>
struct StageKeep {
    bool ready = false;
    CompElimPlan<T> ce;
    int32_t* fwb = nullptr;
    BsPlan<T> bg;
    cudaStream_t s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    void release(cudaStream_t st) {
        ce.release(st);
        bg.release(st);
        if (fwb) cudaFreeAsync(fwb, st);
        fwb = nullptr;
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s2) {
            cudaStreamSynchronize(s2);
            cudaStreamDestroy(s2);
        }
        fork = join = nullptr;
        s2 = nullptr;
        ready = false;
    }
};

// Component tables of every instance in element type T (Algorithm 1 after the
// reordering; independent of the boundary slots' order).  ev: stage events (may be null);
// keep: record / replay (may be null).
template <typename T>
cudaError_t batch_comp_tables(std::vector<Inst>& I, const BatchPtrs& P, const MatDesc* d_cdescs,
                              const MatDesc* h_cdescs, int64_t ktot, int32_t max_ld, bool f32w, const CompElim& ce,
                              double* comp_elim_updates, cudaEvent_t* ev, cudaStream_t st,
                              StageKeep<T>* keep = nullptr) {
    T* base = reinterpret_cast<T*>(P.tables);
    cudaError_t e;
    if (ev) cudaEventRecord(ev[2], st);
    if ((e = launch_fill_blocks<T>(base, d_cdescs, (int32_t)ktot, st)) != cudaSuccess) return e;
    for (auto& x : I) {
        if (x.n == 0) continue;
        e = launch_scatter_intra<T>(f32w, x.n, x.rp, x.col, x.w, x.part, P.local + x.vbase, P.descs + x.kbase,
                                    base + x.apsp_off, st);
        if (e != cudaSuccess) return e;
    }
    // component tables: the elimination form for those selected (dissection order per
    // instance, then the elimination of all of them at once), Floyd-Warshall for the rest
    // (h_cdescs holds n = 0 for the selected ones)
    *comp_elim_updates = 0.0;
    if (ce.nsel > 0) {
        T* Pc = reinterpret_cast<T*>(ce.P);
        if ((e = launch_fill_blocks<T>(Pc, ce.d_ed, ce.nsel, st)) != cudaSuccess) return e;
        e = comp_nd_order(ce.d_graphs, ce.d_cgraph, P.local, ce.sorted_v, ce.vstart_global, P.csize,
                          (int32_t)ce.ktot, ce.ndpos, st);
        if (e != cudaSuccess) return e;
        for (auto& x : I) {
            if (x.n == 0) continue;
            e = comp_nd_scatter<T>(Pc + x.apsp_off, P.descs + x.kbase, x.n, x.rp, x.col, x.w, f32w, x.part,
                                   P.local + x.vbase, ce.vstart_local + x.kbase, P.csize + x.kbase,
                                   ce.ndpos + x.vbase, ce.vpos + x.vbase, st);
            if (e != cudaSuccess) return e;
        }
        e = comp_elim_finish<T>(base, Pc, d_cdescs, ce.ed, ce.d_sel, ce.d_ed, P.csize, ce.vstart_global, ce.ndpos,
                                comp_elim_updates, st, keep ? &keep->ce : nullptr);
        if (e != cudaSuccess) return e;
    }
    if (max_ld > 0 &&
        (e = fw_batched<T>(base, d_cdescs, h_cdescs, (int32_t)ktot, max_ld, st, keep ? &keep->fwb : nullptr)) !=
            cudaSuccess)
        return e;
    if (ev) cudaEventRecord(ev[3], st);
    return cudaSuccess;
}

// Boundary graphs of every instance in element type T (after batch_comp_tables<T>):
// assembly, all-pairs distances, and (check) the exactness check of every float32 table.
// ev: stage events (may be null).  keep: record / replay (may be null); a replay leaves
// the check's flag in d_flag and the status in be.err for the caller to read.
template <typename T>
cudaError_t batch_bg_tables(std::vector<Inst>& I, const BatchPtrs& P, const MatDesc* d_bdescs, int32_t nbmat,
                            int32_t max_N, bool f32w, uint32_t* fw_scratch, uint32_t* d_flag, bool check,
                            bool* inexact, double* bg_updates, const BatchElim& be, cudaEvent_t* ev, cudaStream_t st,
                            StageKeep<T>* keep = nullptr) {
    *inexact = false;
    const bool replay = keep && keep->ready;
    T* base = reinterpret_cast<T*>(P.tables);
    cudaError_t e;
    for (auto& x : I) {
        if (x.N == 0) continue;
        T* D = base + x.d_off;
        if ((e = launch_bg_fill<T>(D, x.N, st)) != cudaSuccess) return e;
        e = launch_bg_clique<T>(base + x.apsp_off, P.descs + x.kbase, P.nb + x.kbase, P.bgoff + x.kbase,
                                P.bgpos + x.slotbase, x.k, D, x.N, st);
        if (e != cudaSuccess) return e;
        e = launch_bg_inter<T>(f32w, x.n, x.rp, x.col, x.w, x.part, P.local + x.vbase, P.bgoff + x.kbase,
                               P.bgpos + x.slotbase, D, x.N, st);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[4], st);
    // The Floyd-Warshall instances' rounds on a second stream, the elimination instances'
    // forward rounds and back-substitution here: both sets of launches side by side.  A
    // build waits on the host for the first set on a helper thread; a replay forks and
    // joins the second stream with events (branches of the captured graph).
    double fw_upd = 0.0;
    cudaError_t fw_err = cudaSuccess;
    cudaStream_t s2 = nullptr;
    cudaEvent_t fw_done = nullptr;
    std::thread fw_thread;
    if (nbmat > 0 && replay) {
        if ((e = cudaEventRecord(keep->fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(keep->s2, keep->fork, 0)) != cudaSuccess) return e;
        if ((e = fw_many_skip<T>(base, d_bdescs, nbmat, max_N, fw_scratch, nullptr, keep->s2, false, false)) !=
            cudaSuccess)
            return e;
        if ((e = cudaEventRecord(keep->join, keep->s2)) != cudaSuccess) return e;
    } else if (nbmat > 0) {
        if ((e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&fw_done, cudaEventDisableTiming)) != cudaSuccess) {
            cudaStreamDestroy(s2);
            return e;
        }
        if (ev) {
            cudaStreamWaitEvent(s2, ev[4], 0);
        } else {
            // (no stage events: order s2 after the assembly with fw_done itself)
            cudaEventRecord(fw_done, st);
            cudaStreamWaitEvent(s2, fw_done, 0);
        }
        fw_thread = std::thread([&, dev = be.dev]() {
            fw_err = cudaSetDevice(dev);
            if (fw_err == cudaSuccess) fw_err = fw_many_skip<T>(base, d_bdescs, nbmat, max_N, fw_scratch, &fw_upd, s2);
            if (fw_err == cudaSuccess) fw_err = cudaEventRecord(fw_done, s2);
        });
    }
    double el_upd = 0.0;
    if (be.n > 0) {
        double fwd = 0.0, bs = 0.0;
        e = fw_many_skip<T>(base, be.descs, be.n, be.max_N, be.scratch, &fwd, st, true, !replay);
        if (e == cudaSuccess) {
            std::vector<BsInput<T>> bin;
            for (auto& x : I)
                if (x.elim) bin.push_back(BsInput<T>{base + x.d_off, x.N, nullptr});
            e = bg_backsub_many<T>(bin, be.err, nullptr, be.panel_cap, &bs, nullptr, st, keep ? &keep->bg : nullptr);
        }
        el_upd = fwd + bs;
    }
    if (replay) {
        if (nbmat > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(st, keep->join, 0);
        if (e != cudaSuccess) return e;
    } else {
        if (fw_thread.joinable()) fw_thread.join();
        if (fw_done) {
            if (fw_err == cudaSuccess) cudaStreamWaitEvent(st, fw_done, 0);
            cudaEventDestroy(fw_done);
        }
        if (s2) {
            if (fw_err != cudaSuccess) cudaStreamSynchronize(s2);
            cudaStreamDestroy(s2);
        }
        if (e != cudaSuccess) return e;
        if (fw_err != cudaSuccess) return fw_err;
        *bg_updates = fw_upd + el_upd;
    }
    if (ev) cudaEventRecord(ev[5], st);
    if (check) {
        if ((e = cudaMemsetAsync(d_flag, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
        if ((e = launch_check_convert(reinterpret_cast<float*>(P.tables), P.table_elems, d_flag, st)) != cudaSuccess)
            return e;
        if (!replay) {
            uint32_t f = 0;
            if ((e = cudaMemcpyAsync(&f, d_flag, sizeof(f), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            *inexact = (f & kErrExact) != 0;
        }
    }
    if (ev) cudaEventRecord(ev[6], st);
    return cudaSuccess;
}

int bits_of(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

}  // namespace

namespace {

// What a build plan keeps of its first build: the batch's layout and device temporaries,
// and the recorded weight-dependent launches of both element types.
struct BuildKeep {
    std::vector<void*> temps;  // device temporaries of the first build
    std::vector<Inst> I;
    BatchPtrs P;
    MatDesc* d_cd = nullptr;
    std::vector<MatDesc> cd_fw;
    int64_t ktot = 0, mtot = 0;
    int32_t max_ld_fw = 0;
    bool f32w = false;
    CompElim ce;
    MatDesc* d_bd = nullptr;
    int32_t nbmat = 0, max_N_fw = 0;
    uint32_t* fw_scratch = nullptr;
    uint32_t* d_flag = nullptr;
    BatchElim be;
    int32_t arith = SPQ_ARITH_I32;
    // the validation launch of every instance (its records and outputs)
    ValGraph* d_vg = nullptr;
    int64_t* d_vb = nullptr;
    uint8_t* bflag = nullptr;
    int32_t* cnt = nullptr;
    uint32_t* errs = nullptr;
    int64_t ntot = 0;
    StageKeep<float> kf;
    StageKeep<int32_t> ki;
    void release(cudaStream_t st) {
        kf.release(st);
        ki.release(st);
        for (void* p : temps) cudaFreeAsync(p, st);
        temps.clear();
    }
};

spq_status build_many_impl(int32_t G, const spq_graph* gs, const spq_opts& o, cudaStream_t st,
                           std::vector<spq_handle*>* out, BuildKeep* keep = nullptr) {
    TempList tmp(st);
    const spq_dtype wt = gs[0].wt;
    const bool f32w = wt == SPQ_F32;
    std::vector<Inst> I(G);
    int64_t ntot = 0, ktot = 0, mtot = 0;
    // ---- inputs on the device ----
    for (int32_t g = 0; g < G; ++g) {
        const spq_graph& a = gs[g];
        if (a.n < 1 || a.k < 1 || !a.row_ptr || !a.part || a.wt != wt) return SPQ_EINVAL;
        Inst& x = I[g];
        x.n = a.n;
        x.k = a.k;
        int64_t ends[2] = {0, 0};
        const bool rp_dev = dev_pointer(a.row_ptr);
        if (rp_dev) {
            BCK(cudaMemcpyAsync(&ends[0], a.row_ptr, 8, cudaMemcpyDeviceToHost, st));
            BCK(cudaMemcpyAsync(&ends[1], a.row_ptr + a.n, 8, cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
        } else {
            ends[0] = a.row_ptr[0];
            ends[1] = a.row_ptr[a.n];
        }
        x.m = ends[1];
        if (ends[0] != 0 || x.m < 0 || x.m > INT32_MAX || (x.m > 0 && (!a.col || !a.w))) return SPQ_EINVAL;
        x.rp = a.row_ptr;
        x.col = a.col;
        x.w = a.w;
        x.part = a.part;
        if (!rp_dev) {
            int64_t* p;
            BCK(tmp.alloc(&p, (size_t)a.n + 1));
            BCK(cudaMemcpyAsync(p, a.row_ptr, ((size_t)a.n + 1) * 8, cudaMemcpyHostToDevice, st));
            x.rp = p;
        }
        if (x.m > 0 && !dev_pointer(a.col)) {
            int32_t* p;
            BCK(tmp.alloc(&p, (size_t)x.m));
            BCK(cudaMemcpyAsync(p, a.col, (size_t)x.m * 4, cudaMemcpyHostToDevice, st));
            x.col = p;
        }
        if (x.m > 0 && !dev_pointer(a.w)) {
            uint32_t* p;
            BCK(tmp.alloc(&p, (size_t)x.m));
            BCK(cudaMemcpyAsync(p, a.w, (size_t)x.m * 4, cudaMemcpyHostToDevice, st));
            x.w = p;
        }
        if (!dev_pointer(a.part)) {
            int32_t* p;
            BCK(tmp.alloc(&p, (size_t)a.n));
            BCK(cudaMemcpyAsync(p, a.part, (size_t)a.n * 4, cudaMemcpyHostToDevice, st));
            x.part = p;
        }
        x.vbase = ntot;
        x.kbase = ktot;
        x.mbase = mtot;
        ntot += a.n;
        ktot += a.k;
        mtot += x.m;
    }
    if (ntot >= ((int64_t)1 << 31) || 2 * ktot >= ((int64_t)1 << 32)) return SPQ_EUNSUPPORTED;
    cudaEvent_t ev[7] = {};
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard() {
            for (int i = 0; i < 7; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } evguard{ev};
    for (auto& e : ev) BCK(cudaEventCreate(&e));
    cudaEventRecord(ev[0], st);

    // ---- validation, boundary flags and counts of every instance; one readback ----
    uint8_t* bflag;
    int32_t* cnt;
    uint32_t* errs;
    BCK(tmp.alloc(&bflag, (size_t)ntot));
    BCK(tmp.alloc(&cnt, 2 * (size_t)ktot));
    BCK(tmp.alloc(&errs, (size_t)G + 1));
    BCK(cudaMemsetAsync(cnt, 0, 2 * (size_t)ktot * 4, st));
    BCK(cudaMemsetAsync(errs, 0, ((size_t)G + 1) * 4, st));
    // every instance in one launch
    std::vector<ValGraph> vg;
    std::vector<int64_t> vb;
    for (auto& x : I) {
        vg.push_back(ValGraph{x.n, x.k, x.m, x.rp, x.col, x.w, x.part, x.kbase});
        vb.push_back(x.vbase);
    }
    vb.push_back(ntot);
    ValGraph* d_vg;
    int64_t* d_vb;
    BCK(tmp.alloc(&d_vg, vg.size()));
    BCK(tmp.alloc(&d_vb, vb.size()));
    BCK(cudaMemcpyAsync(d_vg, vg.data(), vg.size() * sizeof(ValGraph), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(d_vb, vb.data(), vb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    BCK(launch_validate_many(f32w, d_vg, d_vb, G, ntot, bflag, cnt, cnt + ktot, errs, st));
    std::vector<int32_t> hcnt(2 * (size_t)ktot);
    std::vector<uint32_t> herr(G);
    BCK(cudaMemcpyAsync(hcnt.data(), cnt, hcnt.size() * 4, cudaMemcpyDeviceToHost, st));
    BCK(cudaMemcpyAsync(herr.data(), errs, (size_t)G * 4, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    for (uint32_t f : herr)
        if (f) return SPQ_EINVAL;
    cudaEventRecord(ev[1], st);

    // ---- plan: sizes and offsets of every table ----
    int64_t apsp_tot = 0, slot_tot = 0;
    int32_t max_ld = 0;
    for (auto& x : I) {
        x.csize.assign(hcnt.begin() + x.kbase, hcnt.begin() + x.kbase + x.k);
        x.nb.assign(hcnt.begin() + ktot + x.kbase, hcnt.begin() + ktot + x.kbase + x.k);
        x.descs.resize(x.k);
        x.bgoff.resize(x.k);
        int64_t acc = 0, bo = 0;
        for (int32_t c = 0; c < x.k; ++c) {
            const int32_t ld = (int32_t)round_up(x.csize[c], 4);
            x.descs[c] = MatDesc{acc, ld, 0};
            acc += (int64_t)ld * ld;
            x.max_ld = std::max(x.max_ld, ld);
            x.bgoff[c] = (int32_t)bo;
            bo += x.nb[c];
        }
        x.apsp_elems = acc;
        x.apsp_off = apsp_tot;
        apsp_tot += acc;
        x.nbg = bo;
        x.N = round_up(bo, 4);
        x.slotbase = slot_tot;
        slot_tot += bo;
        max_ld = std::max(max_ld, x.max_ld);
    }
    int64_t d_tot = 0;
    int32_t max_N = 0, nbmat = 0;
    for (auto& x : I) {
        x.d_off = apsp_tot + d_tot;
        d_tot += x.N * x.N;
        if (x.N > 0) {
            ++nbmat;
            max_N = std::max(max_N, (int32_t)x.N);
        }
    }
    // arena: metadata arrays, then the tables (16-byte aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off = align256(off + bytes);
        return o2;
    };
    const size_t o_comp = take(4 * (size_t)ntot), o_local = take(4 * (size_t)ntot);
    const size_t o_descs = take(sizeof(MatDesc) * (size_t)ktot), o_nb = take(4 * (size_t)ktot);
    const size_t o_bgoff = take(4 * (size_t)ktot), o_csize = take(4 * (size_t)ktot);
    const size_t o_bgpos = take(4 * (size_t)slot_tot), o_err = take(16 * (size_t)G);
    const int64_t table_elems = apsp_tot + d_tot;
    const size_t o_tables = take(4 * (size_t)table_elems);
    const size_t arena_bytes = off;
    const int64_t fw_words = nbmat > 0 ? fw_many_scratch_words(nbmat, max_N) : 1;
    const bool comp_elim = o.comp_method != SPQ_BG_FW;
    const size_t temp_bytes = 16 * (size_t)ntot + 4 * (size_t)radix_hist_words(ntot) + 12 * (size_t)mtot +
                              4 * (size_t)fw_words + (64u << 20) +
                              (comp_elim ? 4 * (size_t)apsp_tot + 16 * (size_t)ntot : 0);
    size_t free_b = 0, total_b = 0;
    BCK(cudaMemGetInfo(&free_b, &total_b));
    free_b += pool_cached_bytes_current();
    if (arena_bytes + temp_bytes > free_b) return SPQ_ENOMEM;
    void* arena_base = nullptr;
    {
        // (from the library's pool: a batch's tens of gigabytes are kept mapped for the next)
        cudaError_t e = scratch_alloc(&arena_base, arena_bytes, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SPQ_ENOMEM : batch_cuda_fail(e);
    }
    struct ArenaGuard {
        void* p;
        ~ArenaGuard() {
            if (p) {
                cudaFreeAsync(p, 0);
                cudaStreamSynchronize(0);
            }
        }
    } aguard{arena_base};
    char* ab = static_cast<char*>(arena_base);
    BatchPtrs P;
    P.comp = reinterpret_cast<int32_t*>(ab + o_comp);
    P.local = reinterpret_cast<int32_t*>(ab + o_local);
    P.descs = reinterpret_cast<MatDesc*>(ab + o_descs);
    P.nb = reinterpret_cast<int32_t*>(ab + o_nb);
    P.bgoff = reinterpret_cast<int32_t*>(ab + o_bgoff);
    P.csize = reinterpret_cast<int32_t*>(ab + o_csize);
    P.bgpos = reinterpret_cast<int32_t*>(ab + o_bgpos);
    P.err = reinterpret_cast<uint32_t*>(ab + o_err);
    P.tables = reinterpret_cast<uint32_t*>(ab + o_tables);
    P.table_elems = table_elems;
    {
        std::vector<MatDesc> hd;
        std::vector<int32_t> hnb, hbo, hcs;
        hd.reserve(ktot);
        for (auto& x : I) {
            hd.insert(hd.end(), x.descs.begin(), x.descs.end());
            hnb.insert(hnb.end(), x.nb.begin(), x.nb.end());
            hbo.insert(hbo.end(), x.bgoff.begin(), x.bgoff.end());
            hcs.insert(hcs.end(), x.csize.begin(), x.csize.end());
        }
        BCK(cudaMemcpyAsync(P.descs, hd.data(), hd.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(P.nb, hnb.data(), hnb.size() * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(P.bgoff, hbo.data(), hbo.size() * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(P.csize, hcs.data(), hcs.size() * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemsetAsync(P.err, 0, 16 * (size_t)G, st));
        BCK(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }

    // ---- one stable sort of every instance's vertices by (global component, interior) ----
    const uint32_t* sorted_v = nullptr;  // (kept for the components' dissection order)
    {
        uint32_t *k0, *v0, *k1, *v1, *hist;
        BCK(tmp.alloc(&k0, (size_t)ntot));
        BCK(tmp.alloc(&v0, (size_t)ntot));
        BCK(tmp.alloc(&k1, (size_t)ntot));
        BCK(tmp.alloc(&v1, (size_t)ntot));
        BCK(tmp.alloc(&hist, (size_t)radix_hist_words(ntot)));
        for (auto& x : I) {
            k_make_keys_many<<<(x.n + 255) / 256, 256, 0, st>>>(x.n, x.part, bflag + x.vbase, (uint32_t)x.kbase,
                                                                (uint32_t)x.vbase, k0, v0);
            count_launches(1);
        }
        BCK(cudaGetLastError());
        bool in_k1 = false;
        BCK(radix_sort_pairs(k0, v0, k1, v1, hist, ntot, bits_of(2 * (uint64_t)ktot - 1), &in_k1, st));
        std::vector<int64_t> cstart(ktot);
        std::vector<int32_t> ckbase(ktot);
        int64_t pos = 0;
        for (auto& x : I)
            for (int32_t c = 0; c < x.k; ++c) {
                cstart[x.kbase + c] = pos;
                ckbase[x.kbase + c] = (int32_t)x.kbase;
                pos += x.csize[c];
            }
        int64_t* d_cstart;
        int32_t* d_ckbase;
        BCK(tmp.alloc(&d_cstart, (size_t)ktot));
        BCK(tmp.alloc(&d_ckbase, (size_t)ktot));
        BCK(cudaMemcpyAsync(d_cstart, cstart.data(), (size_t)ktot * 8, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(d_ckbase, ckbase.data(), (size_t)ktot * 4, cudaMemcpyHostToDevice, st));
        sorted_v = in_k1 ? v1 : v0;
        k_assign_local_many<<<(unsigned)((ntot + 255) / 256), 256, 0, st>>>(
            ntot, in_k1 ? k1 : k0, in_k1 ? v1 : v0, d_cstart, d_ckbase, P.local, P.comp);
        count_launches(1);
        BCK(cudaGetLastError());
        BCK(cudaStreamSynchronize(st));  // cstart / ckbase go out of scope
    }

    // ---- boundary-slot order of every instance: one gather, host ordering in threads (on
    // a background thread, while the GPU computes the component tables) ----
    std::vector<int32_t> bgpos(slot_tot);
    std::vector<int32_t> methods(G, 0);
    std::vector<std::vector<uint32_t>> hk(G);
    std::vector<std::vector<int32_t>> hs(G), hcm(G);
    std::atomic<int32_t> next{0};
    std::atomic<int> bad{0};
    std::thread order_thread;
    bool order_pending = false;
    struct Join {
        std::thread& t;
        ~Join() {
            if (t.joinable()) t.join();
        }
    } join_order{order_thread};
    for (auto& x : I)
        for (int64_t i = 0; i < x.nbg; ++i) bgpos[x.slotbase + i] = (int32_t)i;
    if ((spq_order)o.order != SPQ_ORDER_ID && mtot > 0) {
        uint32_t *keys, *counters;
        int32_t *slots, *comps;
        BCK(tmp.alloc(&keys, (size_t)mtot));
        BCK(tmp.alloc(&slots, (size_t)mtot));
        BCK(tmp.alloc(&comps, (size_t)mtot));
        BCK(tmp.alloc(&counters, 2 * (size_t)G));
        BCK(cudaMemsetAsync(counters, 0, 2 * (size_t)G * 4, st));
        for (int32_t g = 0; g < G; ++g) {
            const Inst& x = I[g];
            if (x.m == 0 || x.k < 4 || x.k > 65536 || x.nbg == 0) continue;
            BCK(launch_emit_comp_pairs(x.n, x.rp, x.col, x.part, x.k, keys + x.mbase, counters + 2 * g, st));
            BCK(launch_emit_slot_pairs(x.n, x.rp, x.col, x.part, P.local + x.vbase, P.bgoff + x.kbase,
                                       slots + x.mbase, comps + x.mbase, counters + 2 * g + 1, st));
        }
        std::vector<uint32_t> hc(2 * (size_t)G);
        BCK(cudaMemcpyAsync(hc.data(), counters, hc.size() * 4, cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        for (int32_t g = 0; g < G; ++g) {
            const Inst& x = I[g];
            hk[g].resize(hc[2 * g]);
            hs[g].resize(hc[2 * g + 1]);
            hcm[g].resize(hc[2 * g + 1]);
            if (hc[2 * g])
                BCK(cudaMemcpyAsync(hk[g].data(), keys + x.mbase, hc[2 * g] * 4, cudaMemcpyDeviceToHost, st));
            if (hc[2 * g + 1]) {
                BCK(cudaMemcpyAsync(hs[g].data(), slots + x.mbase, hc[2 * g + 1] * 4, cudaMemcpyDeviceToHost, st));
                BCK(cudaMemcpyAsync(hcm[g].data(), comps + x.mbase, hc[2 * g + 1] * 4, cudaMemcpyDeviceToHost, st));
            }
        }
        BCK(cudaStreamSynchronize(st));
        order_pending = true;
        order_thread = std::thread([&, order = (spq_order)o.order]() {
        auto worker = [&]() {
            for (;;) {
                const int32_t g = next.fetch_add(1);
                if (g >= G) return;
                Inst& x = I[g];
                if (hk[g].empty()) continue;
                std::vector<int32_t> bp;
                int32_t meth = 0;
                if (boundary_order_host(x.k, x.nb, std::move(hk[g]), hs[g], hcm[g], order, &bp, &meth) != SPQ_OK ||
                    (int64_t)bp.size() != x.nbg) {
                    bad = 1;
                    continue;
                }
                std::copy(bp.begin(), bp.end(), bgpos.begin() + x.slotbase);
                methods[g] = meth;
            }
        };
        const int nth = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 16));
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(worker);
        worker();
        for (auto& t : pool) t.join();
        });
    }

    // ---- component tables of every instance (while the host orders the slots) ----
    std::vector<MatDesc> cd, bd, ed;
    cd.reserve(ktot);
    // components by elimination (selected), the others by Floyd-Warshall (cd_fw: n = 0
    // for the selected ones)
    CompElim ce;
    std::vector<MatDesc> cd_fw;
    int32_t max_ld_fw = 0;
    double comp_fw_updates = 0.0;
    {
        std::vector<int32_t> vsl(ktot), vsg(ktot), sel, cgraph(ktot);
        std::vector<NdGraph> graphs;
        for (auto& x : I) {
            graphs.push_back(NdGraph{x.rp, x.col, x.part, (int32_t)x.vbase, (int32_t)x.kbase});
            for (int32_t c = 0; c < x.k; ++c) cgraph[x.kbase + c] = (int32_t)(&x - I.data());
            int32_t acc = 0;
            for (int32_t c = 0; c < x.k; ++c) {
                const MatDesc d = x.descs[c];
                vsl[x.kbase + c] = acc;
                vsg[x.kbase + c] = (int32_t)x.vbase + acc;
                acc += x.csize[c];
                const MatDesc g{x.apsp_off + d.off, d.n, 0};
                if (comp_elim && comp_takes_elim(x.csize[c], d.n)) {
                    sel.push_back((int32_t)(x.kbase + c));
                    ce.ed.push_back(g);
                    cd_fw.push_back(MatDesc{g.off, 0, 0});
                } else {
                    cd_fw.push_back(g);
                    max_ld_fw = std::max(max_ld_fw, d.n);
                    const double R = (double)((d.n + kTile - 1) / kTile);
                    comp_fw_updates += R * (1.0 + (R - 1.0) + R * (R - 1.0) / 2.0) * (double)kTile * kTile * kTile;
                }
            }
        }
        ce.nsel = (int32_t)sel.size();
        if (ce.nsel > 0) {
            BCK(tmp.alloc(&ce.d_sel, sel.size()));
            BCK(tmp.alloc(&ce.d_ed, ce.ed.size()));
            BCK(tmp.alloc(&ce.vstart_local, (size_t)ktot));
            BCK(tmp.alloc(&ce.vstart_global, (size_t)ktot));
            BCK(tmp.alloc(&ce.ndpos, (size_t)ntot));
            BCK(tmp.alloc(&ce.vpos, (size_t)ntot));
            uint32_t* pc = nullptr;
            BCK(tmp.alloc(&pc, (size_t)apsp_tot));
            ce.P = pc;
            ce.sorted_v = reinterpret_cast<const int32_t*>(sorted_v);
            BCK(cudaMemcpyAsync(ce.d_sel, sel.data(), sel.size() * 4, cudaMemcpyHostToDevice, st));
            BCK(cudaMemcpyAsync(ce.d_ed, ce.ed.data(), ce.ed.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, st));
            BCK(cudaMemcpyAsync(ce.vstart_local, vsl.data(), (size_t)ktot * 4, cudaMemcpyHostToDevice, st));
            BCK(cudaMemcpyAsync(ce.vstart_global, vsg.data(), (size_t)ktot * 4, cudaMemcpyHostToDevice, st));
            BCK(tmp.alloc(&ce.d_graphs, graphs.size()));
            BCK(tmp.alloc(&ce.d_cgraph, (size_t)ktot));
            BCK(cudaMemcpyAsync(ce.d_graphs, graphs.data(), graphs.size() * sizeof(NdGraph), cudaMemcpyHostToDevice,
                                st));
            BCK(cudaMemcpyAsync(ce.d_cgraph, cgraph.data(), (size_t)ktot * 4, cudaMemcpyHostToDevice, st));
            ce.ktot = ktot;
            BCK(cudaStreamSynchronize(st));  // the host vectors go out of scope
        }
    }
    for (auto& x : I)
        for (const MatDesc& d : x.descs) cd.push_back(MatDesc{x.apsp_off + d.off, d.n, 0});
    MatDesc *d_cd, *d_bd;
    uint32_t *fw_scratch, *d_flag;
    BCK(tmp.alloc(&d_cd, cd.size()));
    BCK(tmp.alloc(&d_flag, 1));
    BCK(cudaMemcpyAsync(d_cd, cd.data(), cd.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, st));
    double bg_updates = 0.0, comp_elim_updates = 0.0;
    bool f32store = false;
    int32_t arith = SPQ_ARITH_I32;
    bool inexact = false;
    // float32 first (exact below 2^24, checked), int32 if asked or if the check fails
    const bool first_f32 = f32w || o.arith != SPQ_ARITH_I32;
    StageKeep<float>* kf = keep ? &keep->kf : nullptr;
    StageKeep<int32_t>* ki = keep ? &keep->ki : nullptr;
    if (first_f32)
        BCK(batch_comp_tables<float>(I, P, d_cd, cd_fw.data(), ktot, max_ld_fw, f32w, ce, &comp_elim_updates, ev, st,
                                     kf));
    else
        BCK(batch_comp_tables<int32_t>(I, P, d_cd, cd_fw.data(), ktot, max_ld_fw, f32w, ce, &comp_elim_updates, ev,
                                       st, ki));

    // ---- the slots' order, and the form of each boundary graph: elimination +
    // back-substitution when asked for, or by default from kBatchElimMin slots on in a
    // dissection order ----
    if (order_thread.joinable()) order_thread.join();
    if (order_pending && bad) return SPQ_EINVAL;
    if (slot_tot > 0) BCK(cudaMemcpyAsync(P.bgpos, bgpos.data(), (size_t)slot_tot * 4, cudaMemcpyHostToDevice, st));
    for (int32_t g = 0; g < G; ++g) {
        Inst& x = I[g];
        x.elim = x.nbg > 0 && (o.bg_method == SPQ_BG_ELIM ||
                               (o.bg_method == SPQ_BG_AUTO && x.nbg >= kBatchElimMin && methods[g] != 0));
    }
    for (auto& x : I)
        if (x.N > 0) (x.elim ? ed : bd).push_back(MatDesc{x.d_off, (int32_t)x.N, 0});
    int32_t max_N_fw = 0, max_N_el = 0;
    for (const MatDesc& d : bd) max_N_fw = std::max(max_N_fw, d.n);
    for (const MatDesc& d : ed) max_N_el = std::max(max_N_el, d.n);
    BatchElim be;
    BCK(cudaGetDevice(&be.dev));
    be.n = (int32_t)ed.size();
    be.max_N = max_N_el;
    be.panel_cap = o.bg_panel_mib > 0 ? ((size_t)o.bg_panel_mib << 20) : ((size_t)2 << 30);
    if (be.n > 0) {
        BCK(tmp.alloc(&be.descs, ed.size()));
        BCK(tmp.alloc(&be.scratch, (size_t)fw_many_scratch_words(be.n, be.max_N)));
        BCK(tmp.alloc(&be.err, 1));
        BCK(cudaMemcpyAsync(be.descs, ed.data(), ed.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, st));
        BCK(cudaMemsetAsync(be.err, 0, 4, st));
    }
    BCK(tmp.alloc(&d_bd, bd.size()));
    BCK(tmp.alloc(&fw_scratch, (size_t)fw_words));
    if (!bd.empty()) BCK(cudaMemcpyAsync(d_bd, bd.data(), bd.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, st));
    if (f32w) {
        f32store = true;
        arith = SPQ_ARITH_F32;
        BCK(batch_bg_tables<float>(I, P, d_bd, (int32_t)bd.size(), max_N_fw, true, fw_scratch, d_flag, false, &inexact,
                                   &bg_updates, be, ev, st, kf));
    } else {
        if (first_f32) {
            arith = SPQ_ARITH_F32;
            BCK(batch_bg_tables<float>(I, P, d_bd, (int32_t)bd.size(), max_N_fw, false, fw_scratch, d_flag, true,
                                       &inexact, &bg_updates, be, ev, st, kf));
        }
        if (!first_f32 || inexact) {
            arith = SPQ_ARITH_I32;
            if (inexact)
                BCK(batch_comp_tables<int32_t>(I, P, d_cd, cd_fw.data(), ktot, max_ld_fw, false, ce,
                                               &comp_elim_updates, ev, st, ki));
            BCK(batch_bg_tables<int32_t>(I, P, d_bd, (int32_t)bd.size(), max_N_fw, false, fw_scratch, d_flag, false,
                                         &inexact, &bg_updates, be, ev, st, ki));
        }
    }
    BCK(cudaStreamSynchronize(st));
    if (be.n > 0) {
        // a bounded wait of the back-substitution that gave up leaves its matrices incomplete
        uint32_t f = 0;
        BCK(cudaMemcpy(&f, be.err, 4, cudaMemcpyDeviceToHost));
        if (f & kErrWait) return SPQ_ETIMEOUT;
    }
    if (keep) {
        keep->I = I;
        keep->P = P;
        keep->d_cd = d_cd;
        keep->cd_fw = cd_fw;
        keep->ktot = ktot;
        keep->mtot = mtot;
        keep->max_ld_fw = max_ld_fw;
        keep->f32w = f32w;
        keep->ce = ce;
        keep->d_bd = d_bd;
        keep->nbmat = (int32_t)bd.size();
        keep->max_N_fw = max_N_fw;
        keep->fw_scratch = fw_scratch;
        keep->d_flag = d_flag;
        keep->be = be;
        keep->arith = arith;
        keep->d_vg = d_vg;
        keep->d_vb = d_vb;
        keep->bflag = bflag;
        keep->cnt = cnt;
        keep->errs = errs;
        keep->ntot = ntot;
        keep->temps = std::move(tmp.ptrs);
        tmp.ptrs.clear();
    }
    double prof[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 6; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) prof[i] = t;
    }
    cudaGetLastError();

    // ---- one handle per instance, all pointing into the arena ----
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    Arena* ar = new (std::nothrow) Arena();
    if (!ar) return SPQ_ENOMEM;
    ar->base = arena_base;
    ar->refs = G;
    aguard.p = nullptr;  // owned by the handles from here on
    out->resize(G, nullptr);
    for (int32_t g = 0; g < G; ++g) {
        const Inst& x = I[g];
        spq_handle* h = new (std::nothrow) spq_handle();
        if (!h) {  // nothing was handed out yet: release everything
            for (int32_t j = 0; j < g; ++j) delete (*out)[j];
            cudaFreeAsync(ar->base, 0);
            cudaStreamSynchronize(0);
            delete ar;
            out->clear();
            return SPQ_ENOMEM;
        }
        h->device = dev;
        h->n = x.n;
        h->k = x.k;
        h->wt = wt;
        h->f32store = f32store;
        h->arith = arith;
        h->query_grouped = o.query_grouped;
        h->query_kernel = o.query_kernel;
        h->max_nb = x.k > 0 ? *std::max_element(x.nb.begin(), x.nb.end()) : 0;
        h->order_method = methods[g];
        h->bg_method = x.elim ? SPQ_BG_ELIM : SPQ_BG_FW;
        h->comp = P.comp + x.vbase;
        h->local = P.local + x.vbase;
        h->descs = P.descs + x.kbase;
        h->nb = P.nb + x.kbase;
        h->bg_off = P.bgoff + x.kbase;
        h->csize = P.csize + x.kbase;
        h->bgpos = P.bgpos + x.slotbase;
        h->err = P.err + 4 * (int64_t)g;
        h->apsp = P.tables + x.apsp_off;
        h->D = x.N > 0 ? (void*)(P.tables + x.d_off) : nullptr;
        h->N = x.N;
        h->nbg = x.nbg;
        h->apsp_elems = x.apsp_elems;
        h->bytes = 4 * (size_t)(x.apsp_elems + x.N * x.N) + 8 * (size_t)x.n + 16 * (size_t)x.k + 4 * (size_t)x.nbg;
        h->comp_updates = comp_fw_updates + comp_elim_updates;  // the whole batch's component updates
        h->bg_updates = bg_updates;  // the whole batch's boundary-graph updates
        for (int i = 0; i < 6; ++i) h->prof_ms[i] = prof[i];
        h->h_csize = x.csize;
        h->h_nb = x.nb;
        h->h_bgoff = x.bgoff;
        h->h_descs = x.descs;
        h->arena = ar;
        (*out)[g] = h;
    }
    return SPQ_OK;
}

}  // namespace

extern "C" {

spq_status spq_build_many(int32_t count, const spq_graph* graphs, const spq_opts* opts, void* stream,
                          spq_handle** outs) {
    if (count < 1 || !graphs || !outs) return SPQ_EINVAL;
    for (int32_t g = 0; g < count; ++g) outs[g] = nullptr;
    spq_opts o;
    if (spq_status so = read_opts(opts, &o)) return so;
    std::vector<spq_handle*> hs;
    const spq_status s = build_many_impl(count, graphs, o, (cudaStream_t)stream, &hs);
    if (s != SPQ_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        return s;
    }
    for (int32_t g = 0; g < count; ++g) outs[g] = hs[g];
    return SPQ_OK;
}

spq_status spq_query_many(int32_t count, spq_handle* const* hs, const int32_t* const* pairs, const int64_t* q,
                          void* const* dist_out, void* stream) {
    if (count < 0 || (count > 0 && (!hs || !pairs || !q || !dist_out))) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t qmax = 0, qtot = 0;
    bool any_dev = false, any_host = false;
    for (int32_t i = 0; i < count; ++i) {
        if (!hs[i] || q[i] < 0 || (q[i] > 0 && (!pairs[i] || !dist_out[i]))) return SPQ_EINVAL;
        if (!on_handle_device(hs[i])) return SPQ_EINVAL;
        if (q[i] == 0) continue;
        const bool pd = dev_pointer(pairs[i]), od = dev_pointer(dist_out[i]);
        if (pd != od) return SPQ_EINVAL;
        if (pd && (((uintptr_t)pairs[i] & 7u) || ((uintptr_t)dist_out[i] & 3u))) return SPQ_EINVAL;
        (pd ? any_dev : any_host) = true;
        qmax = std::max(qmax, q[i]);
        qtot += q[i];
    }
    if (qtot == 0) return SPQ_OK;
    if (any_dev && any_host) return SPQ_EINVAL;
    TempList tmp(st);
    // one scratch for every instance's grouped form, reused in stream order
    uint32_t* scratch;
    BCK(tmp.alloc(&scratch, (size_t)query_scratch_words(qmax)));
    int32_t* dpairs = nullptr;
    int32_t* dout = nullptr;
    if (any_host) {
        BCK(tmp.alloc(&dpairs, 2 * (size_t)qtot));
        BCK(tmp.alloc(&dout, (size_t)qtot));
    }
    int64_t base = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (q[i] == 0) continue;
        const int32_t* p = pairs[i];
        void* o = dist_out[i];
        if (any_host) {
            BCK(cudaMemcpyAsync(dpairs + 2 * base, pairs[i], 2 * (size_t)q[i] * 4, cudaMemcpyHostToDevice, st));
            p = dpairs + 2 * base;
            o = dout + base;
        }
        QueryCtx<int32_t> ci;
        QueryCtx<float> cf;
        bool f32store = false, out_f32 = false;
        int32_t k = 0;
        handle_query_view(hs[i], &ci, &cf, &f32store, &out_f32, &k);
        uint32_t* sc = hs[i]->query_grouped ? scratch : nullptr;
        BCK(f32store ? launch_query<float>(cf, p, q[i], o, out_f32, (uint32_t)k, sc, st)
                     : launch_query<int32_t>(ci, p, q[i], o, out_f32, (uint32_t)k, sc, st));
        if (any_host)
            BCK(cudaMemcpyAsync(dist_out[i], dout + base, (size_t)q[i] * 4, cudaMemcpyDeviceToHost, st));
        base += q[i];
    }
    if (any_host) {
        BCK(cudaStreamSynchronize(st));
        bool bad = false;
        for (int32_t i = 0; i < count; ++i) {
            if (q[i] == 0) continue;
            uint32_t f = 0;
            BCK(cudaMemcpy(&f, hs[i]->err, sizeof(f), cudaMemcpyDeviceToHost));
            if (f & kErrPair) {
                bad = true;
                BCK(cudaMemset(hs[i]->err, 0, sizeof(uint32_t)));
            }
        }
        if (bad) return SPQ_EINVAL;
    }
    return SPQ_OK;
}

// A batched query plan: the launches of spq_query_many for fixed handles, device buffers
// and sizes, captured once into a CUDA graph and replayed by one graph launch.
struct spq_query_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t* scratch = nullptr;
};

namespace {

void plan_destroy(spq_query_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->scratch) {
        cudaDeviceSynchronize();  // (replays queued on any stream are done)
        cudaFreeAsync(p->scratch, 0);
        cudaStreamSynchronize(0);
    }
    delete p;
}

// The launches of one batch on stream st (device buffers; the grouped form's scratch is
// shared in stream order).
cudaError_t issue_queries(int32_t count, spq_handle* const* hs, const int32_t* const* pairs, const int64_t* q,
                          void* const* dist_out, uint32_t* scratch, cudaStream_t st) {
    for (int32_t i = 0; i < count; ++i) {
        if (q[i] == 0) continue;
        QueryCtx<int32_t> ci;
        QueryCtx<float> cf;
        bool f32store = false, out_f32 = false;
        int32_t k = 0;
        handle_query_view(hs[i], &ci, &cf, &f32store, &out_f32, &k);
        uint32_t* sc = hs[i]->query_grouped ? scratch : nullptr;
        const cudaError_t e = f32store ? launch_query<float>(cf, pairs[i], q[i], dist_out[i], out_f32, (uint32_t)k, sc, st)
                                       : launch_query<int32_t>(ci, pairs[i], q[i], dist_out[i], out_f32, (uint32_t)k,
                                                               sc, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

spq_status spq_query_plan_create(int32_t count, spq_handle* const* hs, const int32_t* const* pairs, const int64_t* q,
                                 void* const* dist_out, void* stream, spq_query_plan** out) {
    if (!out) return SPQ_EINVAL;
    *out = nullptr;
    if (count < 0 || (count > 0 && (!hs || !pairs || !q || !dist_out))) return SPQ_EINVAL;
    int64_t qmax = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (!hs[i] || q[i] < 0 || (q[i] > 0 && (!pairs[i] || !dist_out[i]))) return SPQ_EINVAL;
        if (!on_handle_device(hs[i])) return SPQ_EINVAL;
        if (q[i] == 0) continue;
        if (!dev_pointer(pairs[i]) || !dev_pointer(dist_out[i])) return SPQ_EINVAL;
        if (((uintptr_t)pairs[i] & 7u) || ((uintptr_t)dist_out[i] & 3u)) return SPQ_EINVAL;
        qmax = std::max(qmax, q[i]);
    }
    spq_query_plan* p = new (std::nothrow) spq_query_plan();
    if (!p) return SPQ_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStream_t cs = nullptr;
    cudaError_t e = scratch_alloc((void**)&p->scratch, (size_t)query_scratch_words(std::max<int64_t>(qmax, 1)) * 4, st);
    // one eager pass first (every kernel attribute set, the batch checked), then the capture
    if (e == cudaSuccess) e = issue_queries(count, hs, pairs, q, dist_out, p->scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e1 = issue_queries(count, hs, pairs, q, dist_out, p->scratch, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
        e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        plan_destroy(p);
        cudaGetLastError();  // a failed capture leaves no error behind for later calls
        return batch_cuda_fail(e);
    }
    *out = p;
    return SPQ_OK;
}

spq_status spq_query_plan_run(spq_query_plan* p, void* stream) {
    if (!p || !p->exec) return SPQ_EINVAL;
    const cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? SPQ_OK : batch_cuda_fail(e);
}

void spq_query_plan_free(spq_query_plan* p) { plan_destroy(p); }

}  // extern "C"

// ---- build plans: fixed topologies, changing weights ----

namespace {

// The weight-dependent launches of a plan in element type T, with the recorded plans of
// sk: replayed (sk.ready: the stream capture) or run afresh (sk = null).  ev-less.
template <typename T>
cudaError_t plan_stage(BuildKeep& K, StageKeep<T>* sk, bool check, bool* inexact, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (K.be.n > 0) e = cudaMemsetAsync(K.be.err, 0, 4, st);
    double cu = 0.0, bu = 0.0;
    *inexact = false;
    if (e == cudaSuccess)
        e = batch_comp_tables<T>(K.I, K.P, K.d_cd, K.cd_fw.data(), K.ktot, K.max_ld_fw, K.f32w, K.ce, &cu, nullptr,
                                 st, sk);
    if (e == cudaSuccess)
        e = batch_bg_tables<T>(K.I, K.P, K.d_bd, K.nbmat, K.max_N_fw, K.f32w, K.fw_scratch, K.d_flag, check, inexact,
                               &bu, K.be, nullptr, st, sk);
    return e;
}

// An uncaptured pass (fresh bookkeeping): float32 first when asked, int32 after it if
// the float32 tables fail the exactness check (check: int32 weights in float32).
cudaError_t plan_rebuild(BuildKeep& K, bool f32, bool check, int32_t* arith, cudaStream_t st) {
    bool inexact = false;
    cudaError_t e = cudaSuccess;
    if (f32) {
        e = plan_stage<float>(K, nullptr, check, &inexact, st);
        *arith = SPQ_ARITH_F32;
    }
    if (e == cudaSuccess && (!f32 || inexact)) {
        e = plan_stage<int32_t>(K, nullptr, false, &inexact, st);
        *arith = SPQ_ARITH_I32;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && K.be.n > 0) {
        uint32_t f = 0;
        e = cudaMemcpy(&f, K.be.err, 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && (f & kErrWait)) e = kWaitGaveUp;
    }
    return e;
}

}  // namespace

// A batched build kept for re-weighting (Algorithm 1 again on the same graphs and
// partitions with new edge weights).  The steps that depend on the structure only
// (numbering, boundary-slot order, elimination forms, the back-substitution's frontier
// bookkeeping) are done once; the weight-dependent launches are captured once into a
// CUDA graph, replayed by every run.
struct spq_build_plan {
    int dev = 0;
    int32_t G = 0;
    spq_dtype wt = SPQ_I32;
    BuildKeep keep;
    std::vector<spq_handle*> hs;
    std::vector<int64_t> m, woff;  // per instance: edges, offset of its weights in wbuf
    uint32_t* wbuf = nullptr;      // every instance's weights (the graph reads them here)
    std::vector<void*> own;        // the plan's copies of the CSR arrays and partitions
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool f32_path = false;  // the captured launches compute in float32
    bool check = false;     // ... and end with the exactness check (int32 weights)
    unsigned long long launches = 0;  // kernels per replay
};

namespace {

void build_plan_destroy(spq_build_plan* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->keep.release(0);
    for (void* x : p->own) cudaFreeAsync(x, 0);
    if (p->wbuf) cudaFreeAsync(p->wbuf, 0);
    cudaStreamSynchronize(0);
    for (spq_handle* h : p->hs)
        if (h) {
            h->plan_owned = false;
            spq_free(h);
        }
    delete p;
}

}  // namespace

extern "C" {

spq_status spq_build_plan_create(int32_t count, const spq_graph* graphs, const spq_opts* opts, void* stream,
                                 spq_build_plan** out, spq_handle** handles) {
    if (!out) return SPQ_EINVAL;
    *out = nullptr;
    if (count < 1 || !graphs || !handles) return SPQ_EINVAL;
    for (int32_t g = 0; g < count; ++g) handles[g] = nullptr;
    spq_opts o;
    if (spq_status so = read_opts(opts, &o)) return so;
    const spq_dtype wt = graphs[0].wt;
    for (int32_t g = 0; g < count; ++g) {
        const spq_graph& a = graphs[g];
        if (a.n < 1 || a.k < 1 || !a.row_ptr || !a.part || a.wt != wt) return SPQ_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    spq_build_plan* p = new (std::nothrow) spq_build_plan();
    if (!p) return SPQ_ENOMEM;
    struct Guard {
        spq_build_plan*& p;
        ~Guard() { build_plan_destroy(p); }
    } guard{p};
    p->G = count;
    p->wt = wt;
    BCK(cudaGetDevice(&p->dev));
    // the plan's own copies of every instance's arrays (the caller's may go away), the
    // weights of all instances in one buffer
    int64_t mtot = 0;
    std::vector<spq_graph> gs(count);
    for (int32_t g = 0; g < count; ++g) {
        const spq_graph& a = graphs[g];
        int64_t m = 0;
        if (dev_pointer(a.row_ptr)) {
            BCK(cudaMemcpy(&m, a.row_ptr + a.n, 8, cudaMemcpyDeviceToHost));
        } else {
            m = a.row_ptr[a.n];
        }
        if (m < 0 || m > INT32_MAX || (m > 0 && (!a.col || !a.w))) return SPQ_EINVAL;
        p->m.push_back(m);
        p->woff.push_back(mtot);
        mtot += m;
        int64_t* rp;
        int32_t *col = nullptr, *part;
        BCK(scratch_alloc((void**)&rp, ((size_t)a.n + 1) * 8, st));
        p->own.push_back(rp);
        BCK(scratch_alloc((void**)&part, (size_t)a.n * 4, st));
        p->own.push_back(part);
        BCK(cudaMemcpyAsync(rp, a.row_ptr, ((size_t)a.n + 1) * 8, cudaMemcpyDefault, st));
        BCK(cudaMemcpyAsync(part, a.part, (size_t)a.n * 4, cudaMemcpyDefault, st));
        if (m > 0) {
            BCK(scratch_alloc((void**)&col, (size_t)m * 4, st));
            p->own.push_back(col);
            BCK(cudaMemcpyAsync(col, a.col, (size_t)m * 4, cudaMemcpyDefault, st));
        }
        gs[g] = spq_graph{a.n, rp, col, nullptr, wt, part, a.k};
    }
    BCK(scratch_alloc((void**)&p->wbuf, (size_t)(mtot > 0 ? mtot : 1) * 4, st));
    for (int32_t g = 0; g < count; ++g) {
        if (p->m[g] > 0)
            BCK(cudaMemcpyAsync(p->wbuf + p->woff[g], graphs[g].w, (size_t)p->m[g] * 4, cudaMemcpyDefault, st));
        gs[g].w = p->wbuf + p->woff[g];
    }
    BCK(cudaStreamSynchronize(st));
    // the first build, recording the launches' bookkeeping
    if (spq_status s = build_many_impl(count, gs.data(), o, st, &p->hs, &p->keep)) {
        cudaStreamSynchronize(st);
        return s;
    }
    for (spq_handle* h : p->hs) h->plan_owned = true;
    BuildKeep& K = p->keep;
    p->f32_path = K.arith == SPQ_ARITH_F32;
    p->check = p->f32_path && !K.f32w;
    // the capture: the recorded launches of the arithmetic the first build ended in
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    auto prep = [&](auto& sk) {
        cudaError_t r = cudaStreamCreateWithFlags(&sk.s2, cudaStreamNonBlocking);
        if (r == cudaSuccess) r = cudaEventCreateWithFlags(&sk.fork, cudaEventDisableTiming);
        if (r == cudaSuccess) r = cudaEventCreateWithFlags(&sk.join, cudaEventDisableTiming);
        sk.ready = true;
        return r;
    };
    if (e == cudaSuccess) e = p->f32_path ? prep(K.kf) : prep(K.ki);
    // (the bookkeeping of the other element type is not needed)
    if (p->f32_path)
        K.ki.release(st);
    else
        K.kf.release(st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const unsigned long long n0 = spq_kernel_launches();
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        bool inexact = false;
        const cudaError_t e1 = p->f32_path ? plan_stage<float>(K, &K.kf, p->check, &inexact, cs)
                                           : plan_stage<int32_t>(K, &K.ki, false, &inexact, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
        e = e1 != cudaSuccess ? e1 : e2;
    }
    p->launches = spq_kernel_launches() - n0;
    count_launches(-(int)p->launches);  // (captured, not launched)
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();  // a failed capture leaves no error behind for later calls
        return batch_cuda_fail(e);
    }
    for (int32_t g = 0; g < count; ++g) handles[g] = p->hs[g];
    *out = p;
    p = nullptr;  // (kept)
    return SPQ_OK;
}

spq_status spq_build_plan_run(spq_build_plan* p, const void* const* weights, void* stream) {
    if (!p || !p->exec || !weights) return SPQ_EINVAL;
    for (int32_t g = 0; g < p->G; ++g)
        if (p->m[g] > 0 && !weights[g]) return SPQ_EINVAL;
    int dev = 0;
    BCK(cudaGetDevice(&dev));
    if (dev != p->dev) return SPQ_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    BuildKeep& K = p->keep;
    for (int32_t g = 0; g < p->G; ++g)
        if (p->m[g] > 0)
            BCK(cudaMemcpyAsync(p->wbuf + p->woff[g], weights[g], (size_t)p->m[g] * 4, cudaMemcpyDefault, st));
    // the new weights checked as a build checks them, before any table is touched
    BCK(cudaMemsetAsync(K.cnt, 0, 2 * (size_t)K.ktot * 4, st));
    BCK(cudaMemsetAsync(K.errs, 0, ((size_t)p->G + 1) * 4, st));
    BCK(launch_validate_many(K.f32w, K.d_vg, K.d_vb, p->G, K.ntot, K.bflag, K.cnt, K.cnt + K.ktot, K.errs, st));
    std::vector<uint32_t> herr(p->G);
    BCK(cudaMemcpyAsync(herr.data(), K.errs, (size_t)p->G * 4, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    for (uint32_t f : herr)
        if (f) return SPQ_EINVAL;
    // the recorded launches; then their status words
    BCK(cudaGraphLaunch(p->exec, st));
    count_launches((int)p->launches);
    uint32_t flag = 0, cerr = 0, berr = 0;
    const uint32_t* ce_err = p->f32_path ? K.kf.ce.err : K.ki.ce.err;
    if (p->check) BCK(cudaMemcpyAsync(&flag, K.d_flag, 4, cudaMemcpyDeviceToHost, st));
    if (ce_err) BCK(cudaMemcpyAsync(&cerr, ce_err, 4, cudaMemcpyDeviceToHost, st));
    if (K.be.n > 0) BCK(cudaMemcpyAsync(&berr, K.be.err, 4, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    if ((cerr | berr) & kErrWait) return SPQ_ETIMEOUT;
    int32_t arith = p->f32_path ? SPQ_ARITH_F32 : SPQ_ARITH_I32;
    if ((cerr | berr) & kErrPlan) {
        // another finite-tile structure than recorded (distances at the int32 limit): the
        // launches again with fresh bookkeeping
        BCK(plan_rebuild(K, p->f32_path, p->check, &arith, st));
    } else if (p->check && (flag & kErrExact)) {
        BCK(plan_rebuild(K, false, false, &arith, st));
    }
    for (spq_handle* h : p->hs) h->arith = arith;
    return SPQ_OK;
}

void spq_build_plan_free(spq_build_plan* p) { build_plan_destroy(p); }

}  // extern "C"
