// Component order for the boundary-graph matrix (nested dissection of the component
// adjacency graph), and table read-back for inspection.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "order.h"
#include "spq_bench.h"

namespace spq {

namespace {

// One key cu * k + cv per slot u -> v joining two components.
__global__ void k_emit_comp_pairs(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ part, uint32_t k, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals, uint32_t* __restrict__ count) {
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    uint32_t cu = (uint32_t)part[u];
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        uint32_t cv = (uint32_t)part[col[e]];
        if (cv == cu) continue;
        uint32_t i = atomicAdd(count, 1u);
        keys[i] = cu * k + cv;
        if (vals) vals[i] = 0u;
    }
}

// One pair (slot of u, component of v) per slot u -> v joining two components; the slot
// of boundary vertex u is slot_off[part[u]] + local[u] (component-grouped numbering).
__global__ void k_emit_slot_pairs(int32_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ part, const int32_t* __restrict__ local,
                                  const int32_t* __restrict__ slot_off, int32_t* __restrict__ slots,
                                  int32_t* __restrict__ comps, uint32_t* __restrict__ count) {
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int32_t cu = part[u];
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        const int32_t cv = part[col[e]];
        if (cv == cu) continue;
        uint32_t i = atomicAdd(count, 1u);
        slots[i] = slot_off[cu] + local[u];
        comps[i] = cv;
    }
}

// out[i][j] = src[pos[i]][pos[j]] (i, j < rows): the boundary-graph matrix in slot order.
template <bool CONV>
__global__ void k_gather_out(const uint32_t* __restrict__ src, int64_t rows, int64_t ld,
                             const int32_t* __restrict__ pos, uint32_t* __restrict__ dst) {
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        const int64_t ri = pos[i];
        for (int64_t j = threadIdx.x; j < rows; j += blockDim.x) {
            uint32_t x = src[ri * ld + pos[j]];
            if (CONV) {
                float f = __uint_as_float(x);
                x = isinf(f) ? (uint32_t)SPQ_INF_I32 : (uint32_t)(int32_t)f;
            }
            dst[i * rows + j] = x;
        }
    }
}

template <bool CONV>
__global__ void k_copy_out(const uint32_t* __restrict__ src, int64_t rows, int64_t cols, int64_t ld,
                           uint32_t* __restrict__ dst) {
    for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
            uint32_t x = src[i * ld + j];
            if (CONV) {
                float f = __uint_as_float(x);
                x = isinf(f) ? (uint32_t)SPQ_INF_I32 : (uint32_t)(int32_t)f;
            }
            dst[i * cols + j] = x;
        }
    }
}

bool dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Nested dissection on the subgraph induced by `nodes` (George's level-structure
// bisection).  Appends the nodes to `out`: side A, side B, then the separator.
struct ND {
    const std::vector<int64_t>& ptr;
    const std::vector<int32_t>& adj;
    const std::vector<int32_t>& wt;
    std::vector<int32_t> mark;   // subset id of each node (current recursion)
    std::vector<int32_t> level;  // BFS level scratch
    int32_t next_id = 1;
    std::vector<int32_t>* out;

    ND(const std::vector<int64_t>& p, const std::vector<int32_t>& a, const std::vector<int32_t>& w, int32_t k,
       std::vector<int32_t>* o)
        : ptr(p), adj(a), wt(w), mark(k, 0), level(k, -1), out(o) {}

    // BFS inside subset `id` from s; returns nodes in BFS order, levels in `level`.
    void bfs(int32_t s, int32_t id, std::vector<int32_t>& q) {
        q.clear();
        q.push_back(s);
        level[s] = 0;
        for (size_t h = 0; h < q.size(); ++h) {
            int32_t x = q[h];
            for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e) {
                int32_t y = adj[e];
                if (mark[y] == id && level[y] < 0) {
                    level[y] = level[x] + 1;
                    q.push_back(y);
                }
            }
        }
    }
    void clear_levels(const std::vector<int32_t>& q) {
        for (int32_t x : q) level[x] = -1;
    }

    void run(std::vector<int32_t> nodes) {
        // iterative work list to avoid deep recursion: (nodes, phase) entries
        struct Work {
            std::vector<int32_t> nodes;
            std::vector<int32_t> sep;  // non-empty: emit after the two sides
            bool emit_sep;
        };
        std::vector<Work> stack;
        stack.push_back({std::move(nodes), {}, false});
        std::vector<int32_t> q, q2;
        while (!stack.empty()) {
            Work wk = std::move(stack.back());
            stack.pop_back();
            if (wk.emit_sep) {
                out->insert(out->end(), wk.sep.begin(), wk.sep.end());
                continue;
            }
            std::vector<int32_t>& S = wk.nodes;
            if (S.size() <= 2) {
                out->insert(out->end(), S.begin(), S.end());
                continue;
            }
            int32_t id = next_id++;
            for (int32_t x : S) mark[x] = id;
            // connected piece containing S[0]; other pieces are ordered separately
            bfs(S[0], id, q);
            if (q.size() < S.size()) {
                std::vector<int32_t> rest;
                for (int32_t x : S)
                    if (level[x] < 0) rest.push_back(x);
                std::vector<int32_t> piece = q;
                clear_levels(q);
                stack.push_back({std::move(rest), {}, false});
                stack.push_back({std::move(piece), {}, false});
                continue;
            }
            // pseudo-peripheral start: farthest node of two sweeps
            int32_t far = q.back();
            clear_levels(q);
            bfs(far, id, q);
            int32_t far2 = q.back();
            clear_levels(q);
            bfs(far2, id, q);
            int32_t hmax = level[q.back()];
            if (hmax < 2) {  // (nearly) a clique: no useful separator
                out->insert(out->end(), q.begin(), q.end());
                clear_levels(q);
                continue;
            }
            int64_t total = 0;
            for (int32_t x : q) total += wt[x];
            // level whose cumulative weight first reaches half
            std::vector<int64_t> lw(hmax + 1, 0);
            for (int32_t x : q) lw[level[x]] += wt[x];
            int64_t cum = 0;
            int32_t L = 1;
            for (int32_t l = 0; l <= hmax; ++l) {
                cum += lw[l];
                if (2 * cum >= total) {
                    L = l;
                    break;
                }
            }
            if (L < 1) L = 1;
            if (L > hmax - 1) L = hmax - 1;
            std::vector<int32_t> A, B, sep;
            for (int32_t x : q) {
                int32_t l = level[x];
                if (l < L) {
                    A.push_back(x);
                } else if (l > L) {
                    B.push_back(x);
                } else {
                    // keep in the separator only nodes adjacent to side B
                    bool touches_b = false;
                    for (int64_t e = ptr[x]; e < ptr[x + 1] && !touches_b; ++e) {
                        int32_t y = adj[e];
                        touches_b = mark[y] == id && level[y] == L + 1;
                    }
                    (touches_b ? sep : A).push_back(x);
                }
            }
            clear_levels(q);
            for (int32_t x : S) mark[x] = 0;
            stack.push_back({{}, std::move(sep), true});
            stack.push_back({std::move(B), {}, false});
            stack.push_back({std::move(A), {}, false});
        }
    }
};

// Nested dissection by id ranges: the node set is split at its weighted median id;
// the separator is the side (of the two) whose nodes adjacent to the other side weigh
// less.  Partitions numbered along a recursive bisection (recursive coordinate
// bisection, recursive graph bisection) get their own cut lines back this way.
void id_split_nd(const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj, const std::vector<int32_t>& wt,
                 int32_t k, std::vector<int32_t>* out) {
    std::vector<int32_t> side(k, 0);  // subset label during one split
    int32_t next = 1;
    struct Work {
        std::vector<int32_t> nodes;  // ascending ids
        std::vector<int32_t> sep;
        bool emit;
    };
    std::vector<Work> stack;
    {
        std::vector<int32_t> all(k);
        for (int32_t c = 0; c < k; ++c) all[c] = c;
        stack.push_back({std::move(all), {}, false});
    }
    while (!stack.empty()) {
        Work wk = std::move(stack.back());
        stack.pop_back();
        if (wk.emit) {
            out->insert(out->end(), wk.sep.begin(), wk.sep.end());
            continue;
        }
        std::vector<int32_t>& S = wk.nodes;
        if (S.size() <= 2) {
            out->insert(out->end(), S.begin(), S.end());
            continue;
        }
        int64_t total = 0;
        for (int32_t x : S) total += wt[x];
        int64_t cum = 0;
        size_t cut = 1;
        for (size_t i = 0; i < S.size(); ++i) {
            cum += wt[S[i]];
            if (2 * cum >= total) {
                cut = i + 1;
                break;
            }
        }
        if (cut >= S.size()) cut = S.size() - 1;
        const int32_t la = next++, lb = next++;
        for (size_t i = 0; i < S.size(); ++i) side[S[i]] = i < cut ? la : lb;
        std::vector<int32_t> sa, sb;  // nodes of each side adjacent to the other side
        int64_t wa = 0, wb = 0;
        for (int32_t x : S) {
            const int32_t other = side[x] == la ? lb : la;
            bool touches = false;
            for (int64_t e = ptr[x]; e < ptr[x + 1] && !touches; ++e) touches = side[adj[e]] == other;
            if (!touches) continue;
            if (side[x] == la) {
                sa.push_back(x);
                wa += wt[x];
            } else {
                sb.push_back(x);
                wb += wt[x];
            }
        }
        const bool use_a = wa <= wb;
        std::vector<int32_t>& sep = use_a ? sa : sb;
        for (int32_t x : sep) side[x] = 0;
        std::vector<int32_t> A, B;
        for (int32_t x : S) {
            if (side[x] == la) A.push_back(x);
            else if (side[x] == lb) B.push_back(x);
            side[x] = 0;
        }
        stack.push_back({{}, std::move(sep), true});
        stack.push_back({std::move(B), {}, false});
        stack.push_back({std::move(A), {}, false});
    }
}

// Symbolic cost of Floyd-Warshall with infinite-panel skipping, at component
// granularity: when component p's rows are the pivots, the finite rows are those of
// the components joined to p through components already eliminated, plus their
// uneliminated neighbours; the work is w(p) * (their weight)^2 / 2.
double fw_order_cost(const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj,
                     const std::vector<int32_t>& wt, const std::vector<int32_t>& order) {
    const int32_t k = (int32_t)order.size();
    std::vector<int32_t> parent(k), elim(k, 0);
    std::vector<int64_t> inner(k, 0), frontw(k, 0);
    std::vector<std::vector<int32_t>> front(k);  // sorted frontier (uneliminated neighbours)
    for (int32_t c = 0; c < k; ++c) parent[c] = c;
    auto find = [&](int32_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    double cost = 0.0;
    std::vector<int32_t> merged;
    for (int32_t p : order) {
        elim[p] = 1;
        int32_t rp = p;
        inner[rp] = wt[p];
        front[rp].clear();
        for (int64_t e = ptr[p]; e < ptr[p + 1]; ++e)
            if (!elim[adj[e]]) front[rp].push_back(adj[e]);
        std::sort(front[rp].begin(), front[rp].end());
        front[rp].erase(std::unique(front[rp].begin(), front[rp].end()), front[rp].end());
        for (int64_t e = ptr[p]; e < ptr[p + 1]; ++e) {
            int32_t q = adj[e];
            if (!elim[q] || q == p) continue;
            int32_t rq = find(q);
            rp = find(rp);
            if (rq == rp) continue;
            if (front[rq].size() > front[rp].size()) std::swap(rq, rp);
            parent[rq] = rp;
            inner[rp] += inner[rq];
            merged.clear();
            std::set_union(front[rp].begin(), front[rp].end(), front[rq].begin(), front[rq].end(),
                           std::back_inserter(merged));
            front[rp].swap(merged);
            std::vector<int32_t>().swap(front[rq]);
        }
        rp = find(rp);
        // drop eliminated nodes (p itself) from the frontier
        auto& F = front[rp];
        F.erase(std::remove_if(F.begin(), F.end(), [&](int32_t x) { return elim[x] != 0; }), F.end());
        int64_t fw = 0;
        for (int32_t x : F) fw += wt[x];
        const double reach = (double)(inner[rp] + fw);
        cost += (double)wt[p] * reach * reach * 0.5;
    }
    return cost;
}

// Vertex-level nested dissection of the boundary graph, following a bisection of the
// component set (rule 1: level structure, rule 2: id ranges).  At each split (A, B)
// the separator is the lighter of: the remaining boundary slots of A-components with an
// edge into a B-component, or the same for B.  Every path of the boundary graph between
// the two sides uses an edge of G between an A-component and a B-component, whose two
// ends are such slots, so either set separates (the clique edges stay inside one
// component, hence inside one side).  Slots: component-grouped numbering, slot_off[c]
// .. slot_off[c+1]-1 for component c in local order.  Emits every slot once.
// With nodes != NULL, the bisections of the top max_depth levels whose pieces hold at
// least min_slots slots are recorded as nodes (positions in *out): a node's slots are
// [begin, end), its own separator [sep_begin, end) after its two children.
void vertex_nd(int rule, int32_t k, const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj,
               const std::vector<int64_t>& slot_off, const std::vector<int64_t>& snb_ptr,
               const std::vector<int32_t>& snb, std::vector<int32_t>* out, int max_depth = 0,
               int64_t min_slots = 0, std::vector<NdNode>* nodes = nullptr) {
    const int64_t nslots = slot_off[k];
    std::vector<uint8_t> removed(nslots, 0);
    std::vector<int32_t> remain(k);
    for (int32_t c = 0; c < k; ++c) remain[c] = (int32_t)(slot_off[c + 1] - slot_off[c]);
    std::vector<int32_t> side(k, 0), level(k, -1);
    int32_t next = 1;
    auto emit_comp = [&](int32_t c) {
        for (int64_t sl = slot_off[c]; sl < slot_off[c + 1]; ++sl)
            if (!removed[sl]) {
                removed[sl] = 1;
                out->push_back((int32_t)sl);
            }
        remain[c] = 0;
    };
    struct Work {
        std::vector<int32_t> comps;  // ascending ids
        std::vector<int32_t> sep;    // slots to emit
        bool emit;
        int depth;
        int node;  // recorded node (-1: none)
    };
    std::vector<Work> stack;
    if (nodes) {
        nodes->clear();
        nodes->push_back(NdNode{});
    }
    {
        std::vector<int32_t> all(k);
        for (int32_t c = 0; c < k; ++c) all[c] = c;
        stack.push_back({std::move(all), {}, false, 0, nodes ? 0 : -1});
    }
    auto close_node = [&](int node, bool sep) {
        if (node < 0) return;
        NdNode& nd = (*nodes)[node];
        if (!sep) nd.sep_begin = (int64_t)out->size();
        nd.end = (int64_t)out->size();
    };
    std::vector<int32_t> q;
    while (!stack.empty()) {
        Work wk = std::move(stack.back());
        stack.pop_back();
        if (wk.emit) {
            if (wk.node >= 0) (*nodes)[wk.node].sep_begin = (int64_t)out->size();
            out->insert(out->end(), wk.sep.begin(), wk.sep.end());
            close_node(wk.node, true);
            continue;
        }
        if (wk.node >= 0) (*nodes)[wk.node].begin = (int64_t)out->size();
        std::vector<int32_t>& S = wk.comps;
        int64_t total = 0;
        for (int32_t c : S) total += remain[c];
        if (S.size() <= 1 || total == 0) {
            for (int32_t c : S) emit_comp(c);
            close_node(wk.node, false);
            continue;
        }
        const int32_t la = next++, lb = next++;
        bool ok = true;
        if (rule == 2) {
            int64_t cum = 0;
            size_t cut = S.size() - 1;
            for (size_t i = 0; i < S.size(); ++i) {
                cum += remain[S[i]];
                if (2 * cum >= total) {
                    cut = i + 1;
                    break;
                }
            }
            if (cut >= S.size()) cut = S.size() - 1;
            if (cut == 0) cut = 1;
            for (size_t i = 0; i < S.size(); ++i) side[S[i]] = i < cut ? la : lb;
        } else {
            for (int32_t c : S) side[c] = la;  // membership mark for the BFS
            auto bfs = [&](int32_t s0) {
                q.clear();
                q.push_back(s0);
                level[s0] = 0;
                for (size_t h = 0; h < q.size(); ++h) {
                    int32_t x = q[h];
                    for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e) {
                        int32_t y = adj[e];
                        if (side[y] == la && level[y] < 0) {
                            level[y] = level[x] + 1;
                            q.push_back(y);
                        }
                    }
                }
            };
            auto clear = [&]() {
                for (int32_t x : q) level[x] = -1;
            };
            bfs(S[0]);
            if (q.size() < S.size()) {  // disconnected: one piece against the rest
                for (int32_t c : S) side[c] = level[c] >= 0 ? la : lb;
                clear();
            } else {
                int32_t far = q.back();
                clear();
                bfs(far);
                int32_t far2 = q.back();
                clear();
                bfs(far2);
                const int32_t hmax = level[q.back()];
                if (hmax < 1) {
                    ok = false;
                    clear();
                } else {
                    std::vector<int64_t> lw(hmax + 1, 0);
                    for (int32_t x : q) lw[level[x]] += remain[x];
                    int64_t cum = 0;
                    int32_t L = 0;
                    for (int32_t l = 0; l <= hmax; ++l) {
                        cum += lw[l];
                        if (2 * cum >= total) {
                            L = l;
                            break;
                        }
                    }
                    if (L > hmax - 1) L = hmax - 1;
                    for (int32_t x : q) side[x] = level[x] <= L ? la : lb;
                    clear();
                }
            }
        }
        if (!ok) {
            for (int32_t c : S) {
                side[c] = 0;
                emit_comp(c);
            }
            close_node(wk.node, false);
            continue;
        }
        std::vector<int32_t> sa, sb;
        for (int32_t c : S) {
            const int32_t other = side[c] == la ? lb : la;
            std::vector<int32_t>& dst = side[c] == la ? sa : sb;
            for (int64_t sl = slot_off[c]; sl < slot_off[c + 1]; ++sl) {
                if (removed[sl]) continue;
                bool touches = false;
                for (int64_t e = snb_ptr[sl]; e < snb_ptr[sl + 1] && !touches; ++e) touches = side[snb[e]] == other;
                if (touches) dst.push_back((int32_t)sl);
            }
        }
        std::vector<int32_t>& sep = sa.size() <= sb.size() ? sa : sb;
        for (int32_t sl : sep) removed[sl] = 1;
        // remaining counts per component
        for (int32_t sl : sep) {
            int32_t c = (int32_t)(std::upper_bound(slot_off.begin(), slot_off.end(), (int64_t)sl) - slot_off.begin()) - 1;
            remain[c]--;
        }
        std::vector<int32_t> A, B;
        int64_t wa = 0, wb = 0;
        for (int32_t c : S) {
            (side[c] == la ? A : B).push_back(c);
            (side[c] == la ? wa : wb) += remain[c];
            side[c] = 0;
        }
        // record the two halves as nodes of their own when both are large enough
        int na = -1, nb2 = -1;
        if (wk.node >= 0 && wk.depth < max_depth && wa >= min_slots && wb >= min_slots) {
            na = (int)nodes->size();
            nodes->push_back(NdNode{});
            nb2 = (int)nodes->size();
            nodes->push_back(NdNode{});
            (*nodes)[na].parent = (*nodes)[nb2].parent = wk.node;
            (*nodes)[na].depth = (*nodes)[nb2].depth = wk.depth + 1;
            (*nodes)[wk.node].child[0] = na;
            (*nodes)[wk.node].child[1] = nb2;
        }
        stack.push_back({{}, std::move(sep), true, wk.depth, wk.node});
        stack.push_back({std::move(B), {}, false, wk.depth + 1, nb2});
        stack.push_back({std::move(A), {}, false, wk.depth + 1, na});
    }
}

}  // namespace

cudaError_t launch_emit_comp_pairs(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* part, int32_t k,
                                   uint32_t* keys, uint32_t* count, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_emit_comp_pairs<<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, part, (uint32_t)k, keys, nullptr, count);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_emit_slot_pairs(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* part,
                                   const int32_t* local, const int32_t* slot_off, int32_t* slots, int32_t* comps,
                                   uint32_t* count, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_emit_slot_pairs<<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, part, local, slot_off, slots, comps, count);
    count_launches(1);
    return cudaGetLastError();
}

void nested_dissection(int32_t k, const std::vector<int64_t>& adj_ptr, const std::vector<int32_t>& adj,
                       const std::vector<int32_t>& weight, std::vector<int32_t>* order) {
    order->clear();
    order->reserve(k);
    ND nd(adj_ptr, adj, weight, k, order);
    std::vector<int32_t> all(k);
    for (int32_t c = 0; c < k; ++c) all[c] = c;
    nd.run(std::move(all));
}

// Padded positions for the recorded bisections (see BgLayout): every node but the root
// starts at a multiple of the tile edge, and so does every split node's separator.
void aligned_layout(const std::vector<int32_t>& slot_order, const std::vector<NdNode>& nodes,
                    std::vector<int32_t>* bgpos, BgLayout* layout) {
    const int64_t ns = (int64_t)slot_order.size();
    std::vector<int64_t> starts;
    for (size_t i = 0; i < nodes.size(); ++i) {
        if (i != 0) starts.push_back(nodes[i].begin);
        if (nodes[i].child[0] >= 0) starts.push_back(nodes[i].sep_begin);
    }
    std::sort(starts.begin(), starts.end());
    starts.erase(std::unique(starts.begin(), starts.end()), starts.end());
    // pad[t] = padding before slot-order index t (t = ns: after the last slot)
    std::vector<int64_t> pad(ns + 1, 0);
    int64_t p = 0;
    size_t j = 0;
    for (int64_t t = 0; t <= ns; ++t) {
        while (j < starts.size() && starts[j] == t) {
            p += (kTile - (t + p) % kTile) % kTile;
            ++j;
        }
        pad[t] = p;
        if (t < ns) (*bgpos)[slot_order[t]] = (int32_t)(t + p);
    }
    layout->npad = ns + pad[ns];
    // block range of [a, b): from the (aligned) position of a to the end of slot b - 1
    auto blk_lo = [&](int64_t a) { return (int32_t)((a + pad[a]) / kTile); };
    auto blk_hi = [&](int64_t b) {
        if (b >= ns) return (int32_t)((layout->npad + kTile - 1) / kTile);
        return (int32_t)((b + pad[b]) / kTile);  // b starts aligned, or is a start of nothing
    };
    layout->tasks.clear();
    std::vector<int32_t> task_of(nodes.size(), -1);
    // post-order: children first
    std::vector<std::pair<int, bool>> st{{0, false}};
    while (!st.empty()) {
        auto [i, done] = st.back();
        st.pop_back();
        const NdNode& nd = nodes[i];
        const bool split = nd.child[0] >= 0;
        if (split && !done) {
            st.push_back({i, true});
            st.push_back({nd.child[1], false});
            st.push_back({nd.child[0], false});
            continue;
        }
        ElimTask tk;
        tk.lo = blk_lo(split ? nd.sep_begin : nd.begin);
        tk.hi = std::max(tk.lo, blk_hi(nd.end));
        tk.shared_from = tk.hi;
        if (split) {
            tk.deps.push_back(task_of[nd.child[0]]);
            tk.deps.push_back(task_of[nd.child[1]]);
        }
        task_of[i] = (int32_t)layout->tasks.size();
        layout->tasks.push_back(std::move(tk));
    }
}

spq_status boundary_order_host(int32_t k, const std::vector<int32_t>& nb, std::vector<uint32_t> hk,
                               const std::vector<int32_t>& hs, const std::vector<int32_t>& hcmp, spq_order ord,
                               std::vector<int32_t>* bgpos, int32_t* method, BgLayout* layout) {
    std::vector<int64_t> slot_off(k + 1, 0);
    for (int32_t c = 0; c < k; ++c) slot_off[c + 1] = slot_off[c] + nb[c];
    const int64_t nslots = slot_off[k];
    bgpos->resize(nslots);
    for (int64_t i = 0; i < nslots; ++i) (*bgpos)[i] = (int32_t)i;
    *method = 0;
    if (ord == SPQ_ORDER_ID || k < 4 || k > 65536 || hk.empty() || nslots == 0) return SPQ_OK;
    if (!std::is_sorted(hk.begin(), hk.end())) std::sort(hk.begin(), hk.end());
    hk.erase(std::unique(hk.begin(), hk.end()), hk.end());
    std::vector<int64_t> ptr(k + 1, 0);
    for (uint32_t key : hk) ptr[key / (uint32_t)k + 1]++;
    for (int32_t c = 0; c < k; ++c) ptr[c + 1] += ptr[c];
    std::vector<int32_t> adj(hk.size());
    for (size_t i = 0; i < hk.size(); ++i) adj[i] = (int32_t)(hk[i] % (uint32_t)k);  // sorted by source
    std::vector<int32_t> w(k);
    for (int32_t c = 0; c < k; ++c) w[c] = nb[c] > 0 ? nb[c] : 1;
    // candidates: id order, level-structure nested dissection, id-range nested
    // dissection of the components; keep the one of least symbolic cost
    std::vector<std::vector<int32_t>> cand(3);
    cand[0].resize(k);
    for (int32_t c = 0; c < k; ++c) cand[0][c] = c;
    nested_dissection(k, ptr, adj, w, &cand[1]);
    id_split_nd(ptr, adj, w, k, &cand[2]);
    const size_t first = (ord == SPQ_ORDER_AUTO) ? 0 : 1;
    size_t best = first;
    double best_cost = fw_order_cost(ptr, adj, w, cand[first]);
    for (size_t i = first + 1; i < cand.size(); ++i) {
        double c = fw_order_cost(ptr, adj, w, cand[i]);
        if (c < best_cost) {
            best_cost = c;
            best = i;
        }
    }
    *method = (int32_t)best;
    if (best == 0) return SPQ_OK;
    std::vector<int32_t> slot_order;
    slot_order.reserve(nslots);
    if (ord == SPQ_ORDER_DISSECTION) {
        for (int32_t c : cand[best])
            for (int64_t sl = slot_off[c]; sl < slot_off[c + 1]; ++sl) slot_order.push_back((int32_t)sl);
    } else {
        // per-slot neighbour components (counting sort by slot, then unique per slot)
        std::vector<int64_t> snb_ptr(nslots + 1, 0);
        for (int32_t sl : hs) snb_ptr[sl + 1]++;
        for (int64_t i = 0; i < nslots; ++i) snb_ptr[i + 1] += snb_ptr[i];
        std::vector<int32_t> snb(hs.size());
        std::vector<int64_t> fill(snb_ptr.begin(), snb_ptr.end() - 1);
        for (size_t i = 0; i < hs.size(); ++i) snb[fill[hs[i]]++] = hcmp[i];
        std::vector<int64_t> uptr(nslots + 1, 0);
        int64_t wpos = 0;
        for (int64_t sl = 0; sl < nslots; ++sl) {
            auto b = snb.begin() + snb_ptr[sl], en = snb.begin() + snb_ptr[sl + 1];
            std::sort(b, en);
            auto u = std::unique(b, en);
            uptr[sl] = wpos;
            for (auto it = b; it != u; ++it) snb[wpos++] = *it;
        }
        uptr[nslots] = wpos;
        std::vector<NdNode> nodes;
        // pieces of at least 16 tiles, layout->depth levels deep: up to 2^depth leaf runs
        // side by side (32 at the most: as many as a context has hardware work queues when
        // CUDA_DEVICE_MAX_CONNECTIONS is 32)
        vertex_nd((int)best, k, ptr, adj, slot_off, uptr, snb, &slot_order,
                  layout ? std::min(std::max(layout->depth, 0), kMaxRunDepth) : 0, 16 * kTile,
                  layout ? &nodes : nullptr);
        *method = (int32_t)best + 2;
        if ((int64_t)slot_order.size() != nslots) return SPQ_EINVAL;  // cannot happen: every slot is emitted once
        if (layout && nodes.size() > 1) {
            aligned_layout(slot_order, nodes, bgpos, layout);
            return SPQ_OK;
        }
    }
    if ((int64_t)slot_order.size() != nslots) return SPQ_EINVAL;  // cannot happen: every slot is emitted once
    for (int64_t i = 0; i < nslots; ++i) (*bgpos)[slot_order[i]] = (int32_t)i;
    return SPQ_OK;
}

spq_status boundary_pairs(int32_t n, int64_t m, const int64_t* d_rp, const int32_t* d_col, const int32_t* d_part,
                          const int32_t* d_local, const int32_t* d_slot_off, int32_t k, const std::vector<int32_t>& nb,
                          spq_order ord, cudaStream_t st, BoundaryPairs* out) {
    int64_t nslots = 0;
    for (int32_t c = 0; c < k; ++c) nslots += nb[c];
    out->want = false;
    const bool want = ord != SPQ_ORDER_ID && k >= 4;
    if (!want || k > 65536 || m == 0 || nslots == 0) return SPQ_OK;
    out->want = true;
    cudaError_t e = cudaSuccess;
    // ---- component adjacency (GPU emit, GPU radix sort, host unique) ----
    uint32_t *keys = nullptr, *vals = nullptr, *k1 = nullptr, *v1 = nullptr, *hist = nullptr, *cnt = nullptr;
    const int64_t hist_words = radix_hist_words(m);
    auto A = [&](uint32_t** p, size_t c) {
        if (e == cudaSuccess) e = scratch_alloc((void**)p, (c ? c : 1) * sizeof(uint32_t), st);
    };
    A(&keys, m);
    A(&vals, m);
    A(&k1, m);
    A(&v1, m);
    A(&hist, hist_words);
    A(&cnt, 1);
    uint32_t hc = 0;
    std::vector<uint32_t> hk;
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        k_emit_comp_pairs<<<(n + 255) / 256, 256, 0, st>>>(n, d_rp, d_col, d_part, (uint32_t)k, keys, vals, cnt);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    bool in_k1 = false;
    if (e == cudaSuccess && hc > 0) {
        int bits = 0;
        uint64_t mx = (uint64_t)k * (uint64_t)k - 1;
        while (bits < 64 && (mx >> bits)) ++bits;
        e = radix_sort_pairs(keys, vals, k1, v1, hist, hc, bits, &in_k1, st);
        hk.resize(hc);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hk.data(), in_k1 ? k1 : keys, hc * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    // ---- (slot, neighbour component) pairs for the vertex-level separators ----
    std::vector<int32_t> hs, hcmp;
    if (e == cudaSuccess && hc > 0 && ord != SPQ_ORDER_DISSECTION) {
        int32_t* ps = (int32_t*)k1;  // reuse: hc <= m words each
        int32_t* pc = (int32_t*)v1;
        e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st);
        if (e == cudaSuccess) {
            k_emit_slot_pairs<<<(n + 255) / 256, 256, 0, st>>>(n, d_rp, d_col, d_part, d_local, d_slot_off, ps, pc,
                                                                 cnt);
            count_launches(1);
            e = cudaGetLastError();
        }
        uint32_t hc2 = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc2, cnt, sizeof(hc2), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        hs.resize(hc2);
        hcmp.resize(hc2);
        if (e == cudaSuccess && hc2 > 0) e = cudaMemcpyAsync(hs.data(), ps, hc2 * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && hc2 > 0) e = cudaMemcpyAsync(hcmp.data(), pc, hc2 * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    uint32_t* ps[] = {keys, vals, k1, v1, hist, cnt};
    for (uint32_t* p : ps)
        if (p) cudaFreeAsync(p, st);
    if (e != cudaSuccess) return SPQ_ECUDA;
    out->hk = std::move(hk);
    out->hs = std::move(hs);
    out->hcmp = std::move(hcmp);
    return SPQ_OK;
}

spq_status boundary_order_from(int32_t k, const std::vector<int32_t>& nb, BoundaryPairs& bp, spq_order ord,
                               std::vector<int32_t>* bgpos, int32_t* method, BgLayout* layout) {
    int64_t nslots = 0;
    for (int32_t c = 0; c < k; ++c) nslots += nb[c];
    if (!bp.want) {
        bgpos->resize(nslots);
        for (int64_t i = 0; i < nslots; ++i) (*bgpos)[i] = (int32_t)i;
        *method = 0;
        return SPQ_OK;
    }
    return boundary_order_host(k, nb, std::move(bp.hk), bp.hs, bp.hcmp, ord, bgpos, method, layout);
}


}  // namespace spq

extern "C" int spq_component_order_host(int k, const long long* adj_ptr, const int* adj, const int* weight,
                                        int method, int* order_out, double* cost_out) {
    using namespace spq;
    if (k <= 0 || !adj_ptr || !weight || !order_out || method < 0 || method > 3) return -1;
    std::vector<int64_t> ptr(adj_ptr, adj_ptr + k + 1);
    std::vector<int32_t> ad(adj, adj + ptr[k]);
    std::vector<int32_t> w(weight, weight + k);
    std::vector<std::vector<int32_t>> cand(3);
    cand[0].resize(k);
    for (int32_t c = 0; c < k; ++c) cand[0][c] = c;
    nested_dissection(k, ptr, ad, w, &cand[1]);
    id_split_nd(ptr, ad, w, k, &cand[2]);
    double costs[3];
    for (int i = 0; i < 3; ++i) costs[i] = fw_order_cost(ptr, ad, w, cand[i]);
    int pick = method;
    if (method == 3) {
        pick = 0;
        for (int i = 1; i < 3; ++i)
            if (costs[i] < costs[pick]) pick = i;
    }
    for (int32_t c = 0; c < k; ++c) order_out[c] = cand[pick][c];
    if (cost_out)
        for (int i = 0; i < 3; ++i) cost_out[i] = costs[i];
    return pick;
}

extern "C" int spq_boundary_order_host(int k, const long long* adj_ptr, const int* adj, const long long* slot_off,
                                       const long long* snb_ptr, const int* snb, int rule, int* slot_order_out) {
    using namespace spq;
    if (k <= 0 || !adj_ptr || !slot_off || !snb_ptr || !slot_order_out || rule < 1 || rule > 2) return -1;
    std::vector<int64_t> ptr(adj_ptr, adj_ptr + k + 1);
    std::vector<int32_t> ad(adj, adj + ptr[k]);
    std::vector<int64_t> so(slot_off, slot_off + k + 1);
    const int64_t ns = so[k];
    std::vector<int64_t> sp(snb_ptr, snb_ptr + ns + 1);
    std::vector<int32_t> sn(snb, snb + sp[ns]);
    std::vector<int32_t> out;
    vertex_nd(rule, k, ptr, ad, so, sp, sn, &out);
    if ((int64_t)out.size() != ns) return -2;
    for (int64_t i = 0; i < ns; ++i) slot_order_out[i] = out[i];
    return 0;
}

extern "C" int spq_boundary_layout_host(int k, const long long* adj_ptr, const int* adj, const long long* slot_off,
                                        const long long* snb_ptr, const int* snb, int rule, int depth, int* bgpos_out,
                                        long long* npad_out, int* tasks_out, int cap_tasks) {
    using namespace spq;
    if (k <= 0 || !adj_ptr || !slot_off || !snb_ptr || !bgpos_out || !npad_out || rule < 1 || rule > 2 || depth < 0 ||
        depth > kMaxRunDepth)
        return -1;
    std::vector<int64_t> ptr(adj_ptr, adj_ptr + k + 1);
    std::vector<int32_t> ad(adj, adj + ptr[k]);
    std::vector<int64_t> so(slot_off, slot_off + k + 1);
    const int64_t ns = so[k];
    std::vector<int64_t> sp(snb_ptr, snb_ptr + ns + 1);
    std::vector<int32_t> sn(snb, snb + sp[ns]);
    std::vector<int32_t> out;
    std::vector<NdNode> nodes;
    vertex_nd(rule, k, ptr, ad, so, sp, sn, &out, depth, 16 * kTile, &nodes);
    if ((int64_t)out.size() != ns) return -2;
    std::vector<int32_t> bgpos(ns);
    BgLayout layout;
    if (nodes.size() > 1) {
        aligned_layout(out, nodes, &bgpos, &layout);
    } else {  // (no split: the slots packed, one run over every block row)
        for (int64_t i = 0; i < ns; ++i) bgpos[out[i]] = (int32_t)i;
        layout.npad = ns;
    }
    for (int64_t i = 0; i < ns; ++i) bgpos_out[i] = bgpos[i];
    *npad_out = layout.npad;
    const int nt = (int)layout.tasks.size();
    for (int t = 0; t < nt && t < cap_tasks && tasks_out; ++t) {
        const ElimTask& tk = layout.tasks[t];
        int* o = tasks_out + 5 * t;
        o[0] = tk.lo;
        o[1] = tk.hi;
        o[2] = tk.shared_from;
        o[3] = tk.deps.size() > 0 ? tk.deps[0] : -1;
        o[4] = tk.deps.size() > 1 ? tk.deps[1] : -1;
    }
    return nt;
}

namespace spq {

cudaError_t copy_table_out(bool to_i32, const void* src, int64_t rows, int64_t cols, int64_t ld, const int32_t* pos,
                           void* out, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const bool od = dev_ptr(out);
    uint32_t* dst = (uint32_t*)out;
    cudaError_t e = cudaSuccess;
    if (!od) e = scratch_alloc((void**)&dst, (size_t)(rows * cols) * 4, st);
    if (e != cudaSuccess) return e;
    int64_t blocks = rows < 65535 ? rows : 65535;
    if (pos) {
        if (to_i32)
            k_gather_out<true><<<(unsigned)blocks, 256, 0, st>>>((const uint32_t*)src, rows, ld, pos, dst);
        else
            k_gather_out<false><<<(unsigned)blocks, 256, 0, st>>>((const uint32_t*)src, rows, ld, pos, dst);
    } else if (to_i32) {
        k_copy_out<true><<<(unsigned)blocks, 256, 0, st>>>((const uint32_t*)src, rows, cols, ld, dst);
    } else {
        k_copy_out<false><<<(unsigned)blocks, 256, 0, st>>>((const uint32_t*)src, rows, cols, ld, dst);
    }
    count_launches(1);
    e = cudaGetLastError();
    if (!od) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dst, (size_t)(rows * cols) * 4, cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(dst, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace spq
