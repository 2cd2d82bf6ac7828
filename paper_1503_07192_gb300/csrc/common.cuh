// Shared definitions of the distance-query library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "spq.h"

namespace spq {

// Bits of the device-side status word.
enum : uint32_t {
    kErrCsr = 1u,     // row_ptr / col out of range
    kErrPart = 2u,    // part[v] outside [0, k)
    kErrWeight = 4u,  // negative or non-finite weight
    kErrAsym = 8u,    // slot u->v without a matching v->u of the same smallest weight
    kErrPair = 16u,   // query pair id outside [0, n)
    kErrExact = 32u,  // float32 tables hold a finite entry >= 2^24 (not provably exact)
    kErrWalk = 64u,   // a gradient path walk did not reach its target (ties of zero length)
    kErrWait = 128u,  // a bounded device-side wait gave up (back-substitution dependencies)
    kErrPlan = 256u,  // a replayed build met a finite-tile structure other than the recorded one
};

// Internal return code of the host helpers when a bounded device-side wait gave up (the
// back-substitution's kErrWait); the entry points turn it into SPQ_ETIMEOUT.
constexpr cudaError_t kWaitGaveUp = cudaErrorLaunchTimeout;

constexpr int kTile = 128;  // Floyd-Warshall tile edge (rows = columns = pivot block)

// +infinity / the int32 sentinel, per table element type.
template <typename T>
struct Inf;
template <>
struct Inf<int32_t> {
    __host__ __device__ static constexpr int32_t value() { return SPQ_INF_I32; }
};
template <>
struct Inf<float> {
    __host__ __device__ static float value() { return __builtin_inff(); }
};

// One square matrix of a batched Floyd-Warshall: element offset from the batch base,
// and its size n (= its row stride; a multiple of 4 so rows stay 16-byte aligned).
struct MatDesc {
    int64_t off;
    int32_t n;
    int32_t pad_;
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Process-wide count of this library's kernel launches (read by spq_kernel_launches).
void count_launches(int n);
// Stream-ordered device scratch from the library's memory pool of the current device
// (kept for reuse across calls; spq_release_cached_memory returns it).  Free with
// cudaFreeAsync.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);

// Bytes the library's pool on the current device holds but no allocation uses (free for
// the next build; api.cu).
size_t pool_cached_bytes_current();

// Record a CUDA error for spq_last_cuda_error (entry points outside api.cu).
void note_cuda_error(cudaError_t e);

// Validated copy of the caller's options (NULL: the defaults); accepts the shorter
// earlier versions of the struct (struct_size).
spq_status read_opts(const spq_opts* in, spq_opts* out);

// Per-launch timing of the boundary-graph Floyd-Warshall's phase-3 kernel (filled only
// when requested: CUDA events around each launch).
struct FwProfile {
    double p3_ms = 0.0;
    int64_t p3_launches = 0;
    double p3_updates = 0.0;
    double bs_ms = 0.0;       // back-substitution kernel time (elimination form)
    int64_t bs_launches = 0;  // its launches (one per panel budget piece)
    double bs_updates = 0.0;  // its min-plus updates (unpadded)
    double bs_items = 0.0;    // its tiles
};

// ---- prep.cu: input validation, boundary detection, stable radix sort ----
cudaError_t launch_validate(bool f32, int32_t n, int64_t m, const int64_t* rp, const int32_t* col, const void* w,
                            const int32_t* part, int32_t k, uint8_t* bflag, int32_t* cnt_c, int32_t* cnt_b,
                            uint32_t* err, cudaStream_t st);
// The same for G graphs at once (one launch): graph g's vertices are the global indices
// [vbase[g], vbase[g + 1]); its flags at bflag + vbase[g], its counts at kbase, its status
// word err[g].
struct ValGraph {
    int32_t n, k;
    int64_t m;
    const int64_t* rp;
    const int32_t* col;
    const void* w;
    const int32_t* part;
    int64_t kbase;
};
cudaError_t launch_validate_many(bool f32, const ValGraph* gs, const int64_t* vbase, int32_t G, int64_t ntot,
                                 uint8_t* bflag, int32_t* cnt_c, int32_t* cnt_b, uint32_t* err, cudaStream_t st);
// Stable LSD radix sort of (key, val) by the low key_bits bits.  Buffers: k0/v0 hold
// the input, k1/v1 are scratch of the same size; hist needs radix_hist_words(n) words.
// Returns (via *in_k1) whether the sorted result ended in k1/v1.
int64_t radix_hist_words(int64_t n);
// In-place exclusive prefix sum of len words (one CTA; for short arrays).
cudaError_t launch_scan_excl(uint32_t* a, int64_t len, cudaStream_t st);
cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist, int64_t n,
                             int key_bits, bool* in_k1, cudaStream_t st);
cudaError_t launch_make_keys(int32_t n, const int32_t* part, const uint8_t* bflag, uint32_t* keys, uint32_t* vals,
                             cudaStream_t st);
cudaError_t launch_assign_local(int32_t n, const uint32_t* sorted_vals, const int32_t* part, const int32_t* vstart,
                                int32_t* local, int32_t* comp, cudaStream_t st);

// ---- assemble.cu: table initialisation and boundary-graph assembly ----
template <typename T>
cudaError_t launch_fill_blocks(T* apsp, const MatDesc* descs, int32_t nmat, cudaStream_t st);
template <typename T>
cudaError_t launch_scatter_intra(bool f32w, int32_t n, const int64_t* rp, const int32_t* col, const void* w,
                                 const int32_t* part, const int32_t* local, const MatDesc* descs, T* apsp,
                                 cudaStream_t st);
// The same for the components of at most max_n vertices and more than min_ld rows only,
// at the per-vertex positions pos.
template <typename T>
cudaError_t launch_scatter_intra_sel(bool f32w, int32_t n, const int64_t* rp, const int32_t* col, const void* w,
                                     const int32_t* part, const int32_t* pos, const MatDesc* descs,
                                     const int32_t* csize, int32_t max_n, int32_t min_ld, T* apsp, cudaStream_t st);
template <typename T>
cudaError_t launch_bg_fill(T* D, int64_t N, cudaStream_t st);
template <typename T>
cudaError_t launch_bg_clique(const T* apsp, const MatDesc* descs, const int32_t* nb, const int32_t* bg_off,
                             const int32_t* bgpos, int32_t k, T* D, int64_t N, cudaStream_t st);
template <typename T>
cudaError_t launch_bg_inter(bool f32w, int32_t n, const int64_t* rp, const int32_t* col, const void* w,
                            const int32_t* part, const int32_t* local, const int32_t* bg_off, const int32_t* bgpos, T* D,
                            int64_t N, cudaStream_t st);
// In place: float32 table -> int32 (+inf -> SPQ_INF_I32), flagging kErrExact if a
// finite entry is >= 2^24 (then the converted values are not used).
cudaError_t launch_check_convert(float* a, int64_t count, uint32_t* err, cudaStream_t st);

// ---- fw.cu: blocked Floyd-Warshall (Venkataraman, Sahni & Mukhopadhyaya 2003) ----
// Many matrices (descs on the device and on the host); each round touches only the
// matrices that still have tiles left.
// keep_buf (build plans): if *keep_buf is null, the per-round lists are uploaded into a
// buffer left in *keep_buf; if not, that buffer is used again (no upload).
template <typename T>
cudaError_t fw_batched(T* base, const MatDesc* d_descs, const MatDesc* h_descs, int32_t nmat, int32_t max_n,
                       cudaStream_t st, int32_t** keep_buf = nullptr);
// One matrix of size N, optionally skipping tiles whose pivot panel is all infinite.
// *updates receives the number of min-plus updates issued (host-side count).
// rowflags == NULL: the full Floyd-Warshall.  rowflags = R x R words (R = ceil(N/128)),
// zeroed: the elimination (forward) form: round r updates only tiles right of and below
// the pivot (I, J > r), and rowflags[r][J] marks the row tiles (r, J > r) that hold a
// finite entry; bg_backsub then completes the matrix.
// tasks (elimination form only, may be NULL): runs of rounds to do side by side where
// they do not depend on each other (see ElimTask in order.h); NULL: one run in order.
struct ElimTask;
template <typename T>
cudaError_t fw_single(T* M, int64_t N, bool skip_inf, uint32_t* scratch_flags, uint32_t* rowflags, double* updates,
                      FwProfile* prof, cudaStream_t st, const std::vector<ElimTask>* tasks = nullptr);
int64_t fw_single_scratch_words(int64_t N);
// ---- elim.cu: back-substitution after the forward form of fw_single ----
// Completes M (N x N, symmetric storage) to all-pairs distances.  err: device status
// word (kErrWait if a bounded wait gave up).  *updates: min-plus updates issued.
// Needs bg_backsub_scratch_bytes(N) bytes of device scratch plus its A panels, which it
// allocates stream-ordered in pieces of at most apanel_budget bytes.
// With exact != NULL (float tables of an int32 graph) the tables are stored as int32 as
// they become final, and a finite value >= 2^24 sets kErrExact in *exact.
template <typename T>
cudaError_t bg_backsub(T* M, int64_t N, const uint32_t* rowflags, uint32_t* err, uint32_t* exact, size_t apanel_budget,
                       double* updates, FwProfile* prof, cudaStream_t st);
// The same for several independent matrices in the fewest launches (rowflags may be
// null: every tile right of the diagonal is examined); err and exact are shared.
template <typename T>
struct BsInput {
    T* M;
    int64_t N;
    const uint32_t* rowflags;
};
// A back-substitution kept for replay (build plans): its bookkeeping, which depends on
// the matrices' finite-tile structure only, and its device buffers.  bg_backsub_many with
// keep != NULL records into *keep (if not ready) or replays it (if ready): the same
// launches with no host step and no allocation, the frontier marks taken afresh and
// checked against the recorded ones (a row block with more finite columns than recorded
// is left out and kErrPlan set in err).
template <typename T>
struct BsPlan {
    struct Launch {
        int32_t mat0, nm, R0, R1;  // matrices [mat0, mat0 + nm), row blocks [R0, R1)
        int64_t aoff0, nit;        // first A-panel row; work items
        size_t run0, run1;         // its runs of the work order
    };
    bool ready = false;
    int32_t nmat = 0, nRmax = 0;
    int64_t P2 = 0, RR = 0;
    unsigned char* scratch = nullptr;  // the records below, one allocation
    void *masks = nullptr, *runs = nullptr, *mats = nullptr;
    int32_t *fblk = nullptr, *fcnt = nullptr, *kcnt = nullptr, *kplan = nullptr;
    uint32_t* tflags = nullptr;
    int64_t* koff = nullptr;
    unsigned long long* counter = nullptr;
    int32_t* klist = nullptr;
    T* A = nullptr;
    std::vector<Launch> launches;
    double updates = 0.0;
    void release(cudaStream_t st) {
        if (klist) cudaFreeAsync(klist, st);
        if (A) cudaFreeAsync(A, st);
        if (scratch) cudaFreeAsync(scratch, st);
        klist = nullptr;
        A = nullptr;
        scratch = nullptr;
        ready = false;
        launches.clear();
    }
};
template <typename T>
cudaError_t bg_backsub_many(const std::vector<BsInput<T>>& in, uint32_t* err, uint32_t* exact, size_t apanel_budget,
                            double* updates, FwProfile* prof, cudaStream_t st, BsPlan<T>* keep = nullptr);
// Marks of every pair of the given tiles (host list).
cudaError_t launch_mark_pairs(const std::vector<int32_t>& blocks, int64_t N, uint32_t* flags, cudaStream_t st);
// Infinity (0 on the diagonal) in the marked tiles, their mirrors and the diagonal tiles.
template <typename T>
cudaError_t launch_fill_marked(T* M, int64_t N, const uint32_t* flags, cudaStream_t st);
size_t bg_backsub_scratch_bytes(int64_t N);
// Marks (flags[I * R + J] = 1, I < J, R = ceil(N/128)) of the tiles the assembled
// boundary-graph matrix may hold a finite entry in: the elimination form's candidates.
cudaError_t launch_mark_bg_tiles(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* part,
                                 const int32_t* local, const int32_t* nb, const int32_t* bg_off, const int32_t* bgpos,
                                 int32_t k, int64_t N, uint32_t* flags, cudaStream_t st);
// Many matrices (sizes up to max_n) at once, with infinite-panel skipping per matrix;
// *updates receives the phase-2 and phase-3 min-plus updates issued.  trail: the
// elimination form's forward pass instead (each round's phases 2 and 3 restricted to the
// tiles right of / below the pivot block), for bg_backsub_many to complete.  stats = false:
// no host read of the update count (*updates untouched; for stream capture).
template <typename T>
cudaError_t fw_many_skip(T* base, const MatDesc* d_descs, int32_t nmat, int32_t max_n, uint32_t* scratch,
                         double* updates, cudaStream_t st, bool trail = false, bool stats = true);
int64_t fw_many_scratch_words(int32_t nmat, int32_t max_n);

// ---- comp_nd.cu: component tables by elimination in a dissection order ----
constexpr int32_t kNdMax = 4096;  // largest component ordered (one CTA each)
// APSP(C) of the components of at most kNdMax vertices and more than one tile row, into
// apsp (local order), after launch_fill_blocks / launch_scatter_intra of the same tables
// (their contents there are replaced).  The other components are left to the caller.
// Waits on the host for the back-substitution's bookkeeping and status.
template <typename T>
cudaError_t comp_tables_elim(T* apsp, const MatDesc* d_descs, const std::vector<MatDesc>& h_descs,
                             const std::vector<int32_t>& h_csize, int32_t k, int32_t n, const int64_t* rp,
                             const int32_t* col, const void* w, bool f32w, const int32_t* part, const int32_t* local,
                             const int32_t* vorder, const int32_t* d_vstart, const int32_t* d_csize, double* updates,
                             cudaStream_t st);
// The parts of comp_tables_elim for several graphs sharing one elimination: the
// dissection order of every component of every graph (one launch; ndpos at vstart[c] + v
// in the batch-wide numbering); per graph, each vertex's position and the scatter of its
// edges into P (the tables in that order, offsets as in d_descs); then, once for all of
// them, the elimination of the selected tables ed (global descriptors; d_sel their
// component indices) and their permutation back into apsp.
struct NdGraph {
    const int64_t* rp;
    const int32_t* col;
    const int32_t* part;
    int32_t vbase, kbase;  // its first vertex / component in the batch-wide numbering
};
cudaError_t comp_nd_order(const NdGraph* d_graphs, const int32_t* d_cgraph, const int32_t* local,
                          const int32_t* vorder, const int32_t* d_vstart, const int32_t* d_csize, int32_t k,
                          int32_t* ndpos, cudaStream_t st);
template <typename T>
cudaError_t comp_nd_scatter(T* P, const MatDesc* d_descs, int32_t n, const int64_t* rp, const int32_t* col,
                            const void* w, bool f32w, const int32_t* part, const int32_t* local,
                            const int32_t* d_vstart, const int32_t* d_csize, const int32_t* ndpos, int32_t* vpos,
                            cudaStream_t st);
// keep (build plans): as for bg_backsub_many.  Recording keeps the scratch, the status
// word and the back-substitution; a replay enqueues the same launches and leaves the
// status word (kErrWait, kErrPlan) in keep->err for the caller to read.
template <typename T>
struct CompElimPlan {
    bool ready = false;
    uint32_t* scratch = nullptr;
    uint32_t* err = nullptr;
    int32_t max_el = 0;
    double updates = 0.0;
    BsPlan<T> bs;
    void release(cudaStream_t st) {
        bs.release(st);
        if (scratch) cudaFreeAsync(scratch, st);
        if (err) cudaFreeAsync(err, st);
        scratch = nullptr;
        err = nullptr;
        ready = false;
    }
};
template <typename T>
cudaError_t comp_elim_finish(T* apsp, T* P, const MatDesc* d_descs, const std::vector<MatDesc>& ed,
                             const int32_t* d_sel, const MatDesc* d_ed, const int32_t* d_csize,
                             const int32_t* d_vstart, const int32_t* ndpos, double* updates, cudaStream_t st,
                             CompElimPlan<T>* keep = nullptr);
// Whether component c takes the elimination form in comp_tables_elim.
inline bool comp_takes_elim(int32_t csize, int32_t ld) { return csize <= kNdMax && ld > kTile; }

// ---- query.cu ----
template <typename T>
struct QueryCtx {
    int32_t n;
    const int32_t* comp;
    const int32_t* local;
    const MatDesc* descs;
    const int32_t* nb;
    const int32_t* bg_off;
    const int32_t* bgpos;
    const T* apsp;
    const T* D;
    int64_t N;
    uint32_t* err;
    // grouped queries: 1 by the staged kernel of query_blocks.cu (blocks of up to
    // query_blocks_max_nb() rows and columns; the rest gathered), 0 all gathered; max_nb:
    // the largest |B(C)|
    int32_t staged = 0;
    int32_t max_nb = 0;
    // profiling (built with opts.profile_kernels): events around the block-copy kernel
    // and its algorithmic counts (min-plus updates, bytes), or null
    cudaEvent_t* qev = nullptr;
    unsigned long long* qstats = nullptr;
    // 1: int32 tables whose finite entries are all below 2^24 (the build's exactness
    // check passed), so the queries may use the float encoding of query_blocks.cu
    int32_t exact24 = 0;
};
// Queries; with scratch (query_scratch_words(q) words) and k <= 65535 the grouped form
// (sorted by component pair), else one warp per query in input order.
int64_t query_scratch_words(int64_t q);
template <typename T>
cudaError_t launch_query(const QueryCtx<T>& ctx, const int32_t* pairs, int64_t q, void* out, bool out_f32,
                         uint32_t k, uint32_t* scratch, cudaStream_t st);

// ---- query_blocks.cu ----
// Largest block side (|B1| or |B2|) the staged grouped kernel handles; larger blocks take
// the gathering kernel of query.cu.
int32_t query_blocks_max_nb();
// Scratch words of launch_query_blocks beyond the sort's.
int64_t query_blocks_scratch_words(int64_t q);
// The staged grouped queries, given the pairs' sorted keys and positions.
template <typename T>
cudaError_t launch_query_blocks(const QueryCtx<T>& ctx, const int32_t* pairs, int64_t q, void* out, bool out_f32,
                                uint32_t k, const uint32_t* keys, const uint32_t* idx, uint32_t* scratch,
                                cudaStream_t st);

// True if the current device is the one h was built on (api.cu).  Every entry point that
// queues work on a handle's tables checks this first: the tables and the library's scratch
// pool are per device, so work queued with another device current would read another
// GPU's memory.
bool on_handle_device(const spq_handle* h);

// Read-only view of a handle's device tables (api.cu), for other entry points.
void handle_query_view(const spq_handle* h, QueryCtx<int32_t>* ci, QueryCtx<float>* cf, bool* f32store, bool* out_f32,
                       int32_t* k);

}  // namespace spq
