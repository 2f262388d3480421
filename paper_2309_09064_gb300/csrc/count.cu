// count.cu -- one exact count: arena layout, stage sequence, readback, stats.
#include "pipeline.cuh"

namespace tc {

namespace {

__global__ void k_ctl_reset(Ctl *ctl) {
    // zero everything, then the min-reduction identity for the root key
    unsigned int *w = reinterpret_cast<unsigned int *>(ctl);
    for (unsigned i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) w[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) ctl->root_key = ~0ull;
}

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 64;
    while (p < x) p <<= 1;
    return p;
}

tc_status pull(tc_ctx *ctx) {
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TC_OK;
}

}  // namespace

// Bytes of scratch for a graph with n vertices, `slots` CSR slots and the
// given maximum degree.
size_t pipeline_bytes(const tc_ctx *ctx, uint32_t n, uint64_t slots, uint32_t max_deg, bool own_levels,
                      uint64_t *hub_slots, uint32_t *hub_blocks) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t n1 = (size_t)n + 1;
    size_t bytes = 0;
    bytes += 11 * r(4 * n1);                       // deg q0 q1 fdeg R parent hcnt scnt wlist blist ntask
    if (own_levels) bytes += r(4 * n1);            // L
    bytes += 3 * r(8 * n1);                        // fpref off2 tpref
    bytes += r(4 * (slots + 1));                   // adj2
    bytes += r(8 * scan_tmp_elems(n1 + 1));        // scan tiles
    *hub_slots = 0;
    *hub_blocks = 0;
    if (max_deg > ctx->tune.block_cap) {
        *hub_slots = next_pow2(2ull * max_deg);
        *hub_blocks = (uint32_t)ctx->num_sms;
        bytes += r(4ull * *hub_slots * *hub_blocks);
    }
    return bytes + 4096;
}

tc_status count_pipeline(tc_ctx *ctx, const GraphView &g, uint32_t *levels_out, const GroupSpec &groups,
                         uint64_t *triangles, tc_stats *stats) {
    const uint32_t n = g.n;
    cudaStream_t s = ctx->stream;
    uint64_t hub_slots = 0;
    uint32_t hub_blocks = 0;
    const size_t need = pipeline_bytes(ctx, n, g.slots, g.max_deg, levels_out == nullptr, &hub_slots, &hub_blocks);
    tc_status st = arena_reserve(ctx, need);
    if (st != TC_OK) return st;
    Arena &a = ctx->arena;
    a.reset();
    const size_t n1 = (size_t)n + 1;
    PipeBufs b;
    b.rp = g.rp;
    b.col = g.col;
    b.deg = a.take<uint32_t>(n1);
    b.L = levels_out ? levels_out : a.take<uint32_t>(n1);
    b.q0 = a.take<uint32_t>(n1);
    b.q1 = a.take<uint32_t>(n1);
    b.fdeg = a.take<uint32_t>(n1);
    b.R = a.take<uint32_t>(n1);
    b.parent = a.take<uint32_t>(n1);
    b.hcnt = a.take<uint32_t>(n1);
    b.scnt = a.take<uint32_t>(n1);
    b.wlist = a.take<uint32_t>(n1);
    b.blist = a.take<uint32_t>(n1);
    b.ntask = a.take<uint32_t>(n1);
    b.fpref = a.take<uint64_t>(n1);
    b.off2 = a.take<uint64_t>(n1);
    b.tpref = a.take<uint64_t>(n1);
    b.adj2 = a.take<uint32_t>(g.slots + 1);
    b.scan_tmp = a.take<uint64_t>(scan_tmp_elems(n1 + 1));
    b.hub_slots = hub_slots;
    b.hub_blocks = hub_blocks;
    if (hub_blocks) b.hub_tables = a.take<uint32_t>(hub_slots * hub_blocks);
    b.groups = groups;
    if (!b.deg || !b.L || !b.q0 || !b.q1 || !b.fdeg || !b.R || !b.parent || !b.hcnt || !b.scnt || !b.wlist ||
        !b.blist || !b.ntask || !b.fpref || !b.off2 || !b.tpref || !b.adj2 || !b.scan_tmp ||
        (hub_blocks && !b.hub_tables))
        return set_error(ctx, TC_ERR_OOM, "arena carve failed");

    ctx->launches = 0;
    ctx->isect_flags = 0;
    k_ctl_reset<<<1, 128, 0, s>>>(ctx->d_ctl);
    note_launch(ctx);
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[0], s));
    st = compute_levels(ctx, b, n, g.slots);
    if (st != TC_OK) return st;
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[1], s));
    st = build_rows(ctx, b, n);
    if (st != TC_OK) return st;
    st = pull(ctx);
    if (st != TC_OK) return st;
    const uint32_t nb = ctx->h_ctl->n_block_u;
    note_launch(ctx, scan_u32_to_u64(b.ntask, b.tpref, nb, b.scan_tmp, s));
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[2], s));
    st = intersect(ctx, b, n);
    if (st != TC_OK) return st;
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[3], s));
    st = pull(ctx);
    if (st != TC_OK) return st;
    const Ctl &h = *ctx->h_ctl;
    if (h.error) return set_error(ctx, TC_ERR_INVALID, "device-side check failed during the count");
    const uint64_t T = h.t_same + h.t_cross;
    if (triangles) *triangles = T;
    if (stats) {
        float t01 = 0, t12 = 0, t23 = 0;
        cudaEventElapsedTime(&t01, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&t12, ctx->ev[1], ctx->ev[2]);
        cudaEventElapsedTime(&t23, ctx->ev[2], ctx->ev[3]);
        stats->n = n;
        stats->m = g.slots / 2;
        stats->triangles = T;
        stats->t_same = h.t_same;
        stats->t_cross = h.t_cross;
        stats->horizontal_edges = h.e0;
        stats->levels = n ? (uint64_t)h.max_level + 1 : 0;
        stats->components = h.components;
        stats->probes = h.probes;
        stats->row2_slots = 0;
        uint64_t row2 = 0;
        if (n) {
            TC_CUDA(ctx, cudaMemcpyAsync(&row2, b.off2 + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
            TC_CUDA(ctx, cudaStreamSynchronize(s));
        }
        stats->row2_slots = row2;
        // Algorithmic bytes (4-byte ids, 8-byte offsets):
        //   levels: row_ptr 8(n+1) + col 4S + neighbour levels 4S + level writes 4n
        //   rows:   row_ptr 8(n+1) + col 4S + neighbour level and degree 8S
        //           + compacted rows 4*row2 + offsets/counts writes 16(n+1)
        //   intersections: hashed rows read once per u + probed rows per edge
        //   output: 8
        const uint64_t S = g.slots, N1 = (uint64_t)n + 1;
        const uint64_t lv = 8 * N1 + 4 * S + 4 * S + 4ull * n;
        const uint64_t rw = 8 * N1 + 4 * S + 8 * S + 4 * row2 + 16 * N1;
        uint64_t is = 0;
        for (int c = 0; c < 3; ++c) {
            stats->class_rows[c] = h.cls_rows[c];
            stats->class_probes[c] = h.cls_probes[c];
            stats->class_bytes[c] = 4ull * (h.cls_build[c] + h.cls_probes[c]);
            is += stats->class_bytes[c];
            stats->ms_class[c] = 0.f;
            if (ctx->isect_flags & (1u << c)) cudaEventElapsedTime(&stats->ms_class[c], ctx->ev[4 + c], ctx->ev[5 + c]);
        }
        stats->launches = ctx->launches;
        stats->reserved = 0;
        stats->isect_bytes = is;
        stats->alg_bytes = lv + rw + is + 8;
        stats->ms_levels = t01;
        stats->ms_mark = t12;
        stats->ms_isect = t23;
        stats->ms_total = t01 + t12 + t23;
    }
    return TC_OK;
}

}  // namespace tc
