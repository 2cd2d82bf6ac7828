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
        vals[i] = 0u;
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

}  // namespace

void nested_dissection(int32_t k, const std::vector<int64_t>& adj_ptr, const std::vector<int32_t>& adj,
                       const std::vector<int32_t>& weight, std::vector<int32_t>* order) {
    order->clear();
    order->reserve(k);
    ND nd(adj_ptr, adj, weight, k, order);
    std::vector<int32_t> all(k);
    for (int32_t c = 0; c < k; ++c) all[c] = c;
    nd.run(std::move(all));
}

spq_status component_order(int32_t n, int64_t m, const int64_t* d_rp, const int32_t* d_col, const int32_t* d_part,
                           int32_t k, const std::vector<int32_t>& nb, spq_order ord, cudaStream_t st,
                           std::vector<int32_t>* order) {
    order->resize(k);
    for (int32_t c = 0; c < k; ++c) (*order)[c] = c;
    const bool want = ord == SPQ_ORDER_DISSECTION || (ord == SPQ_ORDER_AUTO && k >= 4);
    if (!want || k > 65536 || m == 0) return SPQ_OK;
    uint32_t *keys = nullptr, *vals = nullptr, *k1 = nullptr, *v1 = nullptr, *hist = nullptr, *cnt = nullptr;
    const int64_t hist_words = radix_hist_words(m);
    cudaError_t e = cudaSuccess;
    auto A = [&](uint32_t** p, size_t c) {
        if (e == cudaSuccess) e = cudaMallocAsync((void**)p, (c ? c : 1) * sizeof(uint32_t), st);
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
    uint32_t* ps[] = {keys, vals, k1, v1, hist, cnt};
    for (uint32_t* p : ps)
        if (p) cudaFreeAsync(p, st);
    if (e != cudaSuccess) return SPQ_ECUDA;
    hk.erase(std::unique(hk.begin(), hk.end()), hk.end());
    std::vector<int64_t> ptr(k + 1, 0);
    for (uint32_t key : hk) ptr[key / (uint32_t)k + 1]++;
    for (int32_t c = 0; c < k; ++c) ptr[c + 1] += ptr[c];
    std::vector<int32_t> adj(hk.size());
    for (size_t i = 0; i < hk.size(); ++i) adj[i] = (int32_t)(hk[i] % (uint32_t)k);  // sorted by source
    std::vector<int32_t> w(k);
    for (int32_t c = 0; c < k; ++c) w[c] = nb[c] > 0 ? nb[c] : 1;
    // candidates: id order, level-structure nested dissection, id-range nested
    // dissection; keep the one of least symbolic cost (ties: the earlier)
    std::vector<std::vector<int32_t>> cand(3);
    cand[0] = *order;
    nested_dissection(k, ptr, adj, w, &cand[1]);
    id_split_nd(ptr, adj, w, k, &cand[2]);
    const size_t first = ord == SPQ_ORDER_DISSECTION ? 1 : 0;
    size_t best = first;
    double best_cost = fw_order_cost(ptr, adj, w, cand[first]);
    for (size_t i = first + 1; i < cand.size(); ++i) {
        double c = fw_order_cost(ptr, adj, w, cand[i]);
        if (c < best_cost) {
            best_cost = c;
            best = i;
        }
    }
    *order = std::move(cand[best]);
    return SPQ_OK;
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

namespace spq {

cudaError_t copy_table_out(bool to_i32, const void* src, int64_t rows, int64_t cols, int64_t ld, void* out,
                           cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const bool od = dev_ptr(out);
    uint32_t* dst = (uint32_t*)out;
    cudaError_t e = cudaSuccess;
    if (!od) e = cudaMallocAsync((void**)&dst, (size_t)(rows * cols) * 4, st);
    if (e != cudaSuccess) return e;
    int64_t blocks = rows < 65535 ? rows : 65535;
    if (to_i32)
        k_copy_out<true><<<(unsigned)blocks, 256, 0, st>>>((const uint32_t*)src, rows, cols, ld, dst);
    else
        k_copy_out<false><<<(unsigned)blocks, 256, 0, st>>>((const uint32_t*)src, rows, cols, ld, dst);
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
