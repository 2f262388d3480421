// batch.cu -- tc_count_batch: G independent graphs counted as one disjoint union.
//
// Components never share edges, so the union's BFS levels, partition and
// intersections are exactly those of each graph on its own (each graph keeps
// its vertex order, so the canonical roots are the same).  Every triangle is
// credited to the graph owning its first vertex, so one pass over the union
// yields every per-graph count.  The union is built on the device by two
// gather kernels; then one count pipeline covers all graphs.
#include <algorithm>
#include <vector>

#include "pipeline.cuh"

namespace tc {

tc_status batch_arena_reserve(tc_ctx *ctx, size_t bytes);

namespace {

struct GraphDesc {
    const uint64_t *rp;
    const uint32_t *col;
    uint64_t sstart;
    uint32_t vstart;
    uint32_t pad;
};

template <class T>
__device__ __forceinline__ uint32_t last_le(const T *starts, uint32_t count, T x) {
    uint32_t a = 0, b = count;
    while (b - a > 1) {
        uint32_t m = (a + b) >> 1;
        if (starts[m] <= x) a = m; else b = m;
    }
    return a;
}

__global__ void k_union_rp(const GraphDesc *__restrict__ d, uint32_t G, const uint32_t *__restrict__ vstart,
                           uint32_t n_total, uint64_t S, uint64_t *__restrict__ rp) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n_total; v += stride) {
        if (v == n_total) {
            rp[v] = S;
            continue;
        }
        const uint32_t g = last_le<uint32_t>(vstart, G, (uint32_t)v);
        rp[v] = d[g].rp[v - d[g].vstart] + d[g].sstart;
    }
}

__global__ void k_union_col(const GraphDesc *__restrict__ d, uint32_t G, const unsigned long long *__restrict__ sstart,
                            uint64_t S, uint32_t *__restrict__ col) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += stride) {
        const uint32_t g = last_le<unsigned long long>(sstart, G, (unsigned long long)j);
        col[j] = d[g].col[j - d[g].sstart] + d[g].vstart;
    }
}

}  // namespace

tc_status count_batch(tc_ctx *ctx, uint32_t G, const tc_graph *const *graphs, uint64_t *counts) {
    cudaStream_t s = ctx->stream;
    // graphs small enough for one thread block go to the one-launch kernel
    // (graphs.cu), the others into one disjoint union through the pipeline
    const uint64_t small_cap = ctx->tune.batch_small_slots;
    std::vector<uint32_t> small, large;
    uint32_t nmax = 0;
    uint64_t smax = 0;
    for (uint32_t i = 0; i < G; ++i) {
        if (small_cap && small_graph_fits(graphs[i], small_cap)) {
            small.push_back(i);
            nmax = std::max(nmax, graphs[i]->n);
            smax = std::max(smax, graphs[i]->slots);
        } else {
            large.push_back(i);
        }
    }
    const uint32_t GL = (uint32_t)large.size();
    std::vector<GraphDesc> desc(GL);
    std::vector<uint32_t> vstart(GL + 1);
    std::vector<unsigned long long> sstart(GL + 1);
    uint64_t N = 0, S = 0;
    uint32_t max_deg = 0;
    for (uint32_t k = 0; k < GL; ++k) {
        const tc_graph *g = graphs[large[k]];
        vstart[k] = (uint32_t)N;
        sstart[k] = S;
        desc[k] = GraphDesc{g->rp, g->col, S, (uint32_t)N, 0};
        N += g->n;
        S += g->slots;
        max_deg = g->max_deg > max_deg ? g->max_deg : max_deg;
        if (N >= 0xFFFFFFFFull) return set_error(ctx, TC_ERR_INVALID, "batch has 2^32 - 1 or more vertices in total");
    }
    vstart[GL] = (uint32_t)N;
    sstart[GL] = S;
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    uint32_t small_blocks = 0;
    const size_t small_bytes =
        small.empty() ? 0 : r(small_graphs_bytes(ctx, std::max(nmax, 1u), std::max<uint64_t>(smax, 1), (uint32_t)small.size(),
                                                 &small_blocks));
    const size_t union_bytes = GL ? r(8 * (N + 1)) + r(4 * (S + 1)) + r(sizeof(GraphDesc) * GL) + r(4 * (GL + 1)) +
                                        r(8 * (GL + 1)) + r(8 * GL)
                                  : 0;
    const size_t need = r(8 * (size_t)G) + small_bytes + union_bytes + 4096;
    tc_status st = batch_arena_reserve(ctx, need);
    if (st != TC_OK) return st;
    Arena &a = ctx->batch_arena;
    a.reset();
    auto *d_all = a.take<unsigned long long>(G);
    char *small_scr = small_bytes ? a.take<char>(small_bytes) : nullptr;
    if (!d_all || (small_bytes && !small_scr)) return set_error(ctx, TC_ERR_OOM, "batch arena carve failed");
    TC_CUDA(ctx, cudaMemsetAsync(d_all, 0, 8ull * G, s));
    unsigned int *d_small_err = nullptr;
    if (!small.empty()) {
        st = count_small_graphs(ctx, graphs, small, d_all, small_scr, small_bytes, &d_small_err);
        if (st != TC_OK) return st;
    }
    std::vector<uint64_t> large_counts(GL);
    if (GL) {
        auto *rp = a.take<uint64_t>(N + 1);
        auto *col = a.take<uint32_t>(S + 1);
        auto *d_desc = a.take<GraphDesc>(GL);
        auto *d_vstart = a.take<uint32_t>(GL + 1);
        auto *d_sstart = a.take<unsigned long long>(GL + 1);
        auto *d_counts = a.take<unsigned long long>(GL);
        if (!rp || !col || !d_desc || !d_vstart || !d_sstart || !d_counts)
            return set_error(ctx, TC_ERR_OOM, "batch arena carve failed");
        TC_CUDA(ctx, cudaMemcpyAsync(d_desc, desc.data(), sizeof(GraphDesc) * GL, cudaMemcpyHostToDevice, s));
        TC_CUDA(ctx, cudaMemcpyAsync(d_vstart, vstart.data(), 4 * (GL + 1), cudaMemcpyHostToDevice, s));
        TC_CUDA(ctx, cudaMemcpyAsync(d_sstart, sstart.data(), 8 * (GL + 1), cudaMemcpyHostToDevice, s));
        TC_CUDA(ctx, cudaMemsetAsync(d_counts, 0, 8 * GL, s));
        const unsigned cap = (unsigned)ctx->num_sms * 16u;
        auto grid = [&](uint64_t w) {
            uint64_t b = (w + 255) / 256;
            return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
        };
        k_union_rp<<<grid(N + 1), 256, 0, s>>>(d_desc, GL, d_vstart, (uint32_t)N, S, rp);
        if (S) k_union_col<<<grid(S), 256, 0, s>>>(d_desc, GL, d_sstart, S, col);
        note_launch(ctx, S ? 2 : 1);
        TC_CUDA(ctx, cudaGetLastError());
        GraphView v;
        v.n = (uint32_t)N;
        v.slots = S;
        v.rp = rp;
        v.col = col;
        v.max_deg = max_deg;
        GroupSpec grp;
        grp.vertex_start = d_vstart;
        grp.n_groups = GL;
        grp.counts = d_counts;
        uint64_t total = 0;
        st = count_pipeline(ctx, v, nullptr, grp, &total, nullptr);
        if (st != TC_OK) return st;
        TC_CUDA(ctx, cudaMemcpyAsync(large_counts.data(), d_counts, 8ull * GL, cudaMemcpyDeviceToHost, s));
    }
    unsigned int small_err = 0;
    TC_CUDA(ctx, cudaMemcpyAsync(counts, d_all, 8ull * G, cudaMemcpyDeviceToHost, s));
    if (d_small_err) TC_CUDA(ctx, cudaMemcpyAsync(&small_err, d_small_err, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(ctx, cudaStreamSynchronize(s));
    for (uint32_t k = 0; k < GL; ++k) counts[large[k]] = large_counts[k];
    if (small_err) return set_error(ctx, TC_ERR_INVALID, "small-graph component step ran past its bound");
    return TC_OK;
}

}  // namespace tc
