// count.cu -- one exact count: arena layout, stage sequence, readback, stats.
#include <algorithm>
#include <cstdio>

#include "pipeline.cuh"

namespace tc {

namespace {

// t(x) = hits credited to x by id + hits credited to x's rank.
__global__ void k_vertex_finish(uint32_t n, const uint2 *__restrict__ lv, const unsigned long long *__restrict__ by_rank,
                                unsigned long long *__restrict__ by_id) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        by_id[x] += by_rank[lv[x].x];
}

__global__ void k_ctl_reset(Ctl *ctl) {
    // zero everything, then the min-reduction identity for the root key
    unsigned int *w = reinterpret_cast<unsigned int *>(ctl);
    for (unsigned i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) w[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) ctl->root_key = ~0ull;
}

tc_status pull(tc_ctx *ctx) {
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TC_OK;
}

}  // namespace

// Bytes of scratch for a graph with n vertices, `slots` CSR slots and the
// given maximum degree.
size_t pipeline_bytes(const tc_ctx *ctx, uint32_t n, uint64_t slots, uint32_t max_deg, bool own_levels, bool plain,
                      uint64_t *hub_words, uint32_t *hub_maps) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t n1 = (size_t)n + 1;
    const uint64_t rtiles = radix_tiles(n1);
    size_t bytes = 0;
    bytes += 21 * r(4 * n1);                       // deg q0 q1 fdeg R parent fcnt gcnt rank big huge lvp glo part rows[4] ntask[3]
    bytes += r(16 * n1);                           // vmeta
    bytes += r(4 * (slots / 2 / 256 + 2));         // chunk_row
    if (own_levels) bytes += r(4 * n1);            // L
    bytes += 8 * r(8 * n1);                        // fpref eoff tpref[3] lv rkeys0 rkeys1
    bytes += r(4 * (slots + 1));                   // adj2
    bytes += r(4 * (slots / 32 + 2));              // fence
    bytes += r(16 * (slots / 2 + 1));              // probe records: one per oriented G0 edge
    bytes += r(4 * (256 * rtiles + 1)) + r(8 * (256 * rtiles + 2));  // radix digit counts and offsets
    bytes += r(8 * scan_tmp_elems(std::max<uint64_t>(n1 + 1, 256 * rtiles + 2)));  // scan tiles
    bytes += r(8 * (slots / 2 + 1));               // task pool: at most one task per oriented G0 edge
    *hub_words = 0;
    *hub_maps = 0;
    if (max_deg > ctx->tune.block_cap) {
        *hub_words = ((((uint64_t)n + 31) / 32) + 31) & ~uint64_t(31);
        // plain counts run two hub groups at a time (isect.cu): two sets of bitmaps
        *hub_maps = ctx->tune.hub_group * (plain ? 2u : 1u);
        bytes += r(4ull * *hub_words * *hub_maps);
    }
    return bytes + 4096;
}

// Listing scratch (capacity `cap` triples in the caller's buffer): hit
// records of the tiny rows (at most one per vertex), one open-chunk state
// per warp that can be resident (64 per SM), an overflow area of one chunk
// per state (the open chunks can reach past the caller's buffer), the fill
// of every chunk, the compaction's two scans, rank -> id.
struct ListSizes {
    uint64_t tiny, states, ovf, nch, scratch, tmp;
};
ListSizes list_sizes(const tc_ctx *ctx, uint32_t n, uint64_t cap) {
    ListSizes z;
    z.tiny = (uint64_t)n + 2;
    z.states = (uint64_t)ctx->num_sms * 64;
    z.ovf = z.states * kListChunk;
    z.nch = (cap + z.ovf) / kListChunk + 1;
    z.scratch = list_compact_scratch(z.nch);
    z.tmp = scan_tmp_elems(std::max<uint64_t>(z.tiny, z.nch + 1));
    return z;
}
size_t list_bytes(const tc_ctx *ctx, uint32_t n, uint64_t cap) {
    const ListSizes z = list_sizes(ctx, n, cap);
    return 8 * z.tiny + 16 * z.states + 12 * z.ovf + 4 * z.nch + 8 * z.scratch + 8 * z.tmp +
           4ull * ((size_t)n + 1) + 8 * 256;
}

tc_status count_pipeline(tc_ctx *ctx, const GraphView &g, uint32_t *levels_out, const GroupSpec &groups,
                         uint64_t *triangles, tc_stats *stats, const uint32_t *levels_in, uint64_t *vertex_counts,
                         const ListSpec *list, bool alg3) {
    const uint32_t n = g.n;
    cudaStream_t s = ctx->stream;
    const uint32_t launches0 = ctx->launches;  // the context's running total before this call
    uint64_t hub_words = 0;
    uint32_t hub_maps = 0;
    const bool plain = !(vertex_counts || list || alg3);
    const size_t need = pipeline_bytes(ctx, n, g.slots, g.max_deg, levels_out == nullptr, plain, &hub_words, &hub_maps) +
                        (vertex_counts ? 8ull * ((size_t)n + 1) + 256 : 0) + (list ? list_bytes(ctx, n, list->capacity) : 0);
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
    b.fcnt = a.take<uint32_t>(n1);
    b.gcnt = a.take<uint32_t>(n1);
    b.rank = a.take<uint32_t>(n1);
    b.big = a.take<uint32_t>(n1);
    b.huge = a.take<uint32_t>(n1);
    b.glo = a.take<uint32_t>(n1);
    b.part = a.take<uint32_t>(n1);
    uint32_t *lvp = a.take<uint32_t>(n1);
    b.vmeta = a.take<uint4>(n1);
    b.chunk_row = a.take<uint32_t>(g.slots / 2 / 256 + 2);
    bool ok = b.deg && b.L && b.q0 && b.q1 && b.fdeg && b.R && b.parent && b.fcnt && b.gcnt && b.rank && b.big &&
              b.huge && b.glo && b.part && lvp && b.vmeta && b.chunk_row;
    // the split set serves the plain count; the per-vertex counts and the
    // listing are faster without it (their time goes to counters and output
    // writes, and the split's extra pieces cost more than its lookups save)
    ctx->split_R = plain ? g1_split_rank(ctx->tune) : 0u;
    b.rows[3] = a.take<uint32_t>(n1);
    ok = ok && b.rows[3];
    for (int c = 0; c < 3; ++c) {
        b.rows[c] = a.take<uint32_t>(n1);
        b.ntask[c] = a.take<uint32_t>(n1);
        b.tpref[c] = a.take<uint64_t>(n1);
        ok = ok && b.rows[c] && b.ntask[c] && b.tpref[c];
    }
    b.fpref = a.take<uint64_t>(n1);
    b.eoff = a.take<uint64_t>(n1);
    b.lv = a.take<uint2>(n1);
    b.rkeys0 = a.take<unsigned long long>(n1);
    b.rkeys1 = a.take<unsigned long long>(n1);
    const uint64_t rtiles = radix_tiles(n1);
    b.rcounts = a.take<uint32_t>(256 * rtiles + 1);
    b.roffs = a.take<uint64_t>(256 * rtiles + 2);
    b.adj2 = a.take<uint32_t>(g.slots + 1);
    b.fence = a.take<uint32_t>(g.slots / 32 + 2);
    b.slots = g.slots;
    b.erec_cap = g.slots / 2 + 1;
    b.erec = a.take<uint4>(b.erec_cap);
    b.scan_tmp = a.take<uint64_t>(scan_tmp_elems(std::max<uint64_t>(n1 + 1, 256 * rtiles + 2)));
    b.task_cap = g.slots / 2 + 1;
    b.task_pool = a.take<uint2>(b.task_cap);
    b.hub_words = hub_words;
    b.hub_sets = hub_maps > ctx->tune.hub_group ? 2u : 1u;
    if (hub_maps) b.hub_bits = a.take<uint32_t>(hub_words * hub_maps);
    b.groups = groups;
    if (vertex_counts) {
        b.vcount = reinterpret_cast<unsigned long long *>(vertex_counts);
        b.vcount_rank = a.take<unsigned long long>((size_t)n + 1);
        if (!b.vcount_rank) return set_error(ctx, TC_ERR_OOM, "arena carve failed");
        if (n) {
            TC_CUDA(ctx, cudaMemsetAsync(b.vcount, 0, 8ull * n, s));
            TC_CUDA(ctx, cudaMemsetAsync(b.vcount_rank, 0, 8ull * n, s));
        }
    }
    uint64_t *list_tmp = nullptr;
    unsigned long long *list_scratch = nullptr;
    if (list) {
        const ListSizes z = list_sizes(ctx, n, list->capacity);
        b.hits = a.take<unsigned long long>(z.tiny);
        b.wstate = a.take<ulonglong2>(z.states);
        b.wstate_len = z.states;
        b.ovf = a.take<uint32_t>(3 * z.ovf);
        b.ovf_cap = z.ovf;
        b.fills = a.take<uint32_t>(z.nch);
        b.nch = z.nch;
        list_scratch = a.take<unsigned long long>(z.scratch);
        list_tmp = a.take<uint64_t>(z.tmp);
        b.list_out = list->out;
        b.list_cap = list->capacity;
        if (ctx->opt.order == TC_ORDER_DEGREE && g.max_deg > 0) b.inv = a.take<uint32_t>(n1);
        if (!b.hits || !b.wstate || !b.ovf || !b.fills || !list_scratch || !list_tmp ||
            (ctx->opt.order == TC_ORDER_DEGREE && g.max_deg > 0 && !b.inv))
            return set_error(ctx, TC_ERR_OOM, "arena carve failed");
        TC_CUDA(ctx, cudaMemsetAsync(b.hits, 0, 8 * z.tiny, s));
        TC_CUDA(ctx, cudaMemsetAsync(b.wstate, 0, 16 * z.states, s));
    }
    ok = ok && b.fpref && b.eoff && b.lv && b.rkeys0 && b.rkeys1 && b.rcounts && b.roffs && b.adj2 && b.fence && b.erec &&
         b.scan_tmp && b.task_pool && (!hub_maps || b.hub_bits);
    if (!ok) return set_error(ctx, TC_ERR_OOM, "arena carve failed");

    k_ctl_reset<<<1, 128, 0, s>>>(ctx->d_ctl);
    note_launch(ctx);
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[0], s));
    st = levels_in ? given_levels(ctx, b, n, levels_in) : compute_levels(ctx, b, n, g.slots);
    if (st != TC_OK) return st;
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[1], s));
    // the packed 4-byte {rank, level} word needs ranks below 2^24 and levels below 255
    b.lvp = (n <= (1u << 24) && ctx->h_ctl->max_level < 255) ? lvp : nullptr;
    st = compute_ranks(ctx, b, n, g.max_deg);
    if (st != TC_OK) return st;
    Ctl counted{};                   // listing: the control block after phase 1
    unsigned long long list_tiny = 0;  // listing: triangles of the tiny rows
    if (alg3) {  // the comparison kernel: full neighbourhoods, no rows
        TC_CUDA(ctx, cudaEventRecord(ctx->ev[2], s));
        st = intersect_alg3(ctx, b, n, g.slots);
        if (st != TC_OK) return st;
        ctx->isect_flags = 0;
    } else {
        st = build_rows(ctx, b, n, g.max_deg);
        if (st != TC_OK) return st;
        st = pull(ctx);  // row counts per class
        if (st != TC_OK) return st;
        st = plan_scans(ctx, b);
        if (st != TC_OK) return st;
        st = pull(ctx);  // task counts per class
        if (st != TC_OK) return st;
        st = emit_tasks(ctx, b);
        if (st != TC_OK) return st;
        if (ctx->nshards > 1) {
            st = records_for_shard(ctx, b);
            if (st != TC_OK) return st;
        }
        TC_CUDA(ctx, cudaEventRecord(ctx->ev[2], s));
        b.list_phase = list ? 1 : 0;
        st = intersect(ctx, b, n);
        if (st != TC_OK) return st;
        if (list) {
            // Phase 1 wrote the triangles of the warp, block and hub classes
            // into chunks and counted those of the tiny rows; compact the
            // former into [0, T_big), then write the latter after them.
            const uint32_t n3 = ctx->h_ctl->n_rows[3];
            note_launch(ctx, scan_u64(reinterpret_cast<uint64_t *>(b.hits), reinterpret_cast<uint64_t *>(b.hits), n3,
                                      list_tmp, s));
            unsigned long long &t_tiny = list_tiny;
            TC_CUDA(ctx, cudaMemcpyAsync(&t_tiny, b.hits + n3, 8, cudaMemcpyDeviceToHost, s));
            st = pull(ctx);
            if (st != TC_OK) return st;
            counted = *ctx->h_ctl;
            const uint64_t T = counted.t_same + counted.t_cross;
            if (triangles) *triangles = T;
            if (counted.error && !(T > list->capacity && counted.error == 0x400u)) {
                char msg[96];
                std::snprintf(msg, sizeof msg, "device-side check failed during the count (code 0x%x)", counted.error);
                return set_error(ctx, TC_ERR_INVALID, msg);
            }
            if (T > list->capacity) return set_error(ctx, TC_ERR_CAPACITY, "listing: more triangles than capacity");
            if (t_tiny > T) return set_error(ctx, TC_ERR_INVALID, "listing: tiny-row records exceed the count");
            st = list_compact(ctx, b, T - t_tiny, counted.list_cursor, list_scratch,
                              reinterpret_cast<unsigned long long *>(list_tmp));
            if (st != TC_OK) return st;
            if (t_tiny) {
                b.list_phase = 2;
                b.tiny_base = T - t_tiny;
                st = intersect(ctx, b, n);
                if (st != TC_OK) return st;
            }
        }
    }  // Algorithm 4
    if (vertex_counts && n) {  // the third vertices were counted by rank
        k_vertex_finish<<<(unsigned)std::min<uint64_t>(((uint64_t)n + 255) / 256, (uint64_t)ctx->num_sms * 16), 256, 0,
                          s>>>(n, b.lv, b.vcount_rank, b.vcount);
        note_launch(ctx);
        TC_CUDA(ctx, cudaGetLastError());
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[3], s));
    st = pull(ctx);
    if (st != TC_OK) return st;
    if (list) {
        // phase 2 found the tiny rows' triangles again
        const Ctl &h2 = *ctx->h_ctl;
        if (!h2.error && h2.t_same + h2.t_cross != counted.t_same + counted.t_cross + list_tiny)
            return set_error(ctx, TC_ERR_INVALID, "listing pass of the tiny rows disagrees with the count");
        const unsigned err = h2.error;
        *ctx->h_ctl = counted;  // statistics of the listing pass
        ctx->h_ctl->error = err;
    }
    const Ctl &h = *ctx->h_ctl;
    if (h.error) {
        char msg[96];
        std::snprintf(msg, sizeof msg, "device-side check failed during the count (code 0x%x)", h.error);
        return set_error(ctx, TC_ERR_INVALID, msg);
    }
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
        // slots of the hashed and probed parts A and G1: every slot but F's
        const uint64_t row2 = g.slots - h.e0;
        stats->row2_slots = row2;
        // Algorithmic bytes (4-byte ids, 8-byte offsets):
        //   levels: row_ptr 8(n+1) + col 4S + neighbour levels 4S + level writes 4n
        //   rows:   row_ptr 8(n+1) + col 4S + neighbour rank and level 8S
        //           + rewritten rows 4S + |F|, |G1| writes 8n
        //   intersections: per hashed row its set and out-list 4(s(u) + |F(u)|),
        //           per oriented edge the probed range 4(|G1(v)| + p)
        //   output: 8
        const uint64_t S = g.slots, N1 = (uint64_t)n + 1;
        const uint64_t lv = 8 * N1 + 4 * S + 4 * S + 4ull * n;
        const uint64_t rw = alg3 ? 0 : 8 * N1 + 4 * S + 8 * S + 4 * S + 8ull * n;
        uint64_t is = 0;
        for (int c = 0; c < 4; ++c) {
            stats->class_rows[c] = h.cls_rows[c];
            stats->class_probes[c] = h.cls_probes[c];
            stats->class_bytes[c] = 4ull * (h.cls_build[c] + h.cls_probes[c]);
            stats->class_inserts[c] = h.cls_inserts[c];
            is += stats->class_bytes[c];
            stats->ms_class[c] = 0.f;
            // events: ev[4..7] bracket the warp, block and hub kernels, ev[8..9] the tiny one
            if (ctx->isect_flags & (1u << c)) {
                if (c < 3) cudaEventElapsedTime(&stats->ms_class[c], ctx->ev[4 + c], ctx->ev[5 + c]);
                else cudaEventElapsedTime(&stats->ms_class[3], ctx->ev[8], ctx->ev[9]);
            }
        }
        stats->launches = ctx->launches - launches0;
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
