// batch.cu -- tc_count_batch: G independent graphs counted as one disjoint union.
//
// Components never share edges, so the union's BFS levels, partition and
// intersections are exactly those of each graph on its own (each graph keeps
// its vertex order, so the canonical roots are the same).  Every triangle is
// credited to the graph owning its first vertex, so one pass over the union
// yields every per-graph count.  The union is built on the device by two
// gather kernels; then one count pipeline covers all graphs.
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
    std::vector<GraphDesc> desc(G);
    std::vector<uint32_t> vstart(G + 1);
    std::vector<unsigned long long> sstart(G + 1);
    uint64_t N = 0, S = 0;
    uint32_t max_deg = 0;
    for (uint32_t i = 0; i < G; ++i) {
        const tc_graph *g = graphs[i];
        vstart[i] = (uint32_t)N;
        sstart[i] = S;
        desc[i] = GraphDesc{g->rp, g->col, S, (uint32_t)N, 0};
        N += g->n;
        S += g->slots;
        max_deg = g->max_deg > max_deg ? g->max_deg : max_deg;
        if (N >= 0xFFFFFFFFull) return set_error(ctx, TC_ERR_INVALID, "batch has 2^32 - 1 or more vertices in total");
    }
    vstart[G] = (uint32_t)N;
    sstart[G] = S;
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = r(8 * (N + 1)) + r(4 * (S + 1)) + r(sizeof(GraphDesc) * G) + r(4 * (G + 1)) +
                        r(8 * (G + 1)) + r(8 * G) + 4096;
    tc_status st = batch_arena_reserve(ctx, need);
    if (st != TC_OK) return st;
    Arena &a = ctx->batch_arena;
    a.reset();
    auto *rp = a.take<uint64_t>(N + 1);
    auto *col = a.take<uint32_t>(S + 1);
    auto *d_desc = a.take<GraphDesc>(G);
    auto *d_vstart = a.take<uint32_t>(G + 1);
    auto *d_sstart = a.take<unsigned long long>(G + 1);
    auto *d_counts = a.take<unsigned long long>(G);
    if (!rp || !col || !d_desc || !d_vstart || !d_sstart || !d_counts)
        return set_error(ctx, TC_ERR_OOM, "batch arena carve failed");
    TC_CUDA(ctx, cudaMemcpyAsync(d_desc, desc.data(), sizeof(GraphDesc) * G, cudaMemcpyHostToDevice, s));
    TC_CUDA(ctx, cudaMemcpyAsync(d_vstart, vstart.data(), 4 * (G + 1), cudaMemcpyHostToDevice, s));
    TC_CUDA(ctx, cudaMemcpyAsync(d_sstart, sstart.data(), 8 * (G + 1), cudaMemcpyHostToDevice, s));
    TC_CUDA(ctx, cudaMemsetAsync(d_counts, 0, 8 * G, s));
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    auto grid = [&](uint64_t w) {
        uint64_t b = (w + 255) / 256;
        return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
    };
    k_union_rp<<<grid(N + 1), 256, 0, s>>>(d_desc, G, d_vstart, (uint32_t)N, S, rp);
    if (S) k_union_col<<<grid(S), 256, 0, s>>>(d_desc, G, d_sstart, S, col);
    TC_CUDA(ctx, cudaGetLastError());
    GraphView v;
    v.n = (uint32_t)N;
    v.slots = S;
    v.rp = rp;
    v.col = col;
    v.max_deg = max_deg;
    GroupSpec grp;
    grp.vertex_start = d_vstart;
    grp.n_groups = G;
    grp.counts = d_counts;
    uint64_t total = 0;
    st = count_pipeline(ctx, v, nullptr, grp, &total, nullptr);
    if (st != TC_OK) return st;
    TC_CUDA(ctx, cudaMemcpyAsync(counts, d_counts, 8 * G, cudaMemcpyDeviceToHost, s));
    TC_CUDA(ctx, cudaStreamSynchronize(s));
    return TC_OK;
}

}  // namespace tc
