// api.cu -- the C ABI: contexts, graphs, counting entry points.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "pipeline.cuh"

namespace tc {

tc_status set_error(tc_ctx *ctx, tc_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

tc_status cuda_error(tc_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    tc_status st = (e == cudaErrorMemoryAllocation) ? TC_ERR_OOM : TC_ERR_CUDA;
    return set_error(ctx, st, m);
}

cudaError_t device_alloc(tc_ctx *ctx, void **p, size_t bytes) {
    ++ctx->alloc_calls;
    if (ctx->fail_alloc_at && ctx->alloc_calls == ctx->fail_alloc_at) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;  // injected: nothing was allocated
    }
    return cudaMalloc(p, bytes);
}

cudaError_t graph_alloc(tc_ctx *ctx, void **p, size_t bytes, bool *pooled) {
    *pooled = false;
    if (!ctx->graph_pool) return device_alloc(ctx, p, bytes);
    ++ctx->alloc_calls;
    if (ctx->fail_alloc_at && ctx->alloc_calls == ctx->fail_alloc_at) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;  // injected: nothing was allocated
    }
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->graph_pool, ctx->stream);
    *pooled = e == cudaSuccess;
    return e;
}

void graph_free(tc_ctx *ctx, void *p, bool pooled) {
    if (!p) return;
    if (pooled) cudaFreeAsync(p, ctx->stream);
    else cudaFree(p);
}

// Grow-only device arena owned by the context.  Growing waits for the stream
// (earlier work may still read the old buffer), then replaces the buffer.
static tc_status reserve_in(tc_ctx *ctx, Arena &a, size_t bytes) {
    if (a.cap >= bytes) return TC_OK;
    TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (a.base) {
        cudaFree(a.base);
        a.base = nullptr;
        a.cap = 0;
    }
    size_t want = bytes + bytes / 8;
    if (device_alloc(ctx, (void **)&a.base, want) != cudaSuccess) {
        cudaGetLastError();
        if (device_alloc(ctx, (void **)&a.base, bytes) != cudaSuccess) {
            cudaGetLastError();
            a.base = nullptr;
            return set_error(ctx, TC_ERR_OOM, "device arena allocation of " + std::to_string(bytes) + " bytes failed");
        }
        want = bytes;
    }
    a.cap = want;
    a.off = 0;
    return TC_OK;
}

tc_status arena_reserve(tc_ctx *ctx, size_t bytes) { return reserve_in(ctx, ctx->arena, bytes); }
tc_status batch_arena_reserve(tc_ctx *ctx, size_t bytes) { return reserve_in(ctx, ctx->batch_arena, bytes); }

// Make ctx->device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static tc_status finish_graph(tc_ctx *ctx, tc_graph *g, int validate, tc_graph **out) {
    tc_status st = TC_OK;
    if (validate) {
        int ok = 0;
        st = validate_csr_device(ctx, g->n, g->rp, g->col, g->slots, &ok);
        if (st == TC_OK && !ok) st = set_error(ctx, TC_ERR_INVALID, "CSR is not a simple undirected graph "
                                                                  "(asymmetric, unsorted, self-loop, repeat or bad id)");
    }
    if (st == TC_OK) st = max_degree_device(ctx, g->n, g->rp, &g->max_deg);
    if (st != TC_OK) {
        tc_graph_free(g);
        return st;
    }
    *out = g;
    return TC_OK;
}

}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_create(tc_ctx **out, int device, const tc_options *opt) {
    if (!out) return TC_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    DeviceGuard guard(device);
    tc_ctx *ctx = new tc_ctx();
    ctx->device = device;
    if (opt) ctx->opt = *opt;
    if (ctx->opt.order != TC_ORDER_DEGREE && ctx->opt.order != TC_ORDER_ID) {
        delete ctx;
        return TC_ERR_INVALID;
    }
    if (!ctx->opt.max_queue) ctx->opt.max_queue = 65536;
    if (const char *f = std::getenv("TC_FAIL_ALLOC_AT")) ctx->fail_alloc_at = std::strtoull(f, nullptr, 10);
    bool ok = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess;
    if (ok && ctx->opt.stream) {
        ctx->stream = (cudaStream_t)ctx->opt.stream;
    } else if (ok) {
        ok = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) == cudaSuccess;
        ctx->stream = ctx->own_stream;
    }
    ok = ok && cudaMalloc(&ctx->d_ctl, sizeof(Ctl)) == cudaSuccess;
    ok = ok && cudaMallocHost(&ctx->h_ctl, sizeof(Ctl)) == cudaSuccess;
    for (int i = 0; ok && i < 10; ++i) ok = cudaEventCreate(&ctx->ev[i]) == cudaSuccess;
    if (ok) {
        // graph arrays come from a pool that keeps freed memory, so a user who makes
        // and frees a graph per request does not pay cudaMalloc / cudaFree each time
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&ctx->graph_pool, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(ctx->graph_pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            ctx->graph_pool = nullptr;  // fall back to cudaMalloc
        }
    }
    if (!ok) {
        cudaGetLastError();
        tc_destroy(ctx);
        return TC_ERR_CUDA;
    }
    *out = ctx;
    return TC_OK;
}

tc_status tc_destroy(tc_ctx *ctx) {
    if (!ctx) return TC_ERR_INVALID;
    serve_shutdown(ctx);
    DeviceGuard guard(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->side_stream) cudaStreamSynchronize(ctx->side_stream);  // hub groups read the arena
    if (ctx->arena.base) cudaFree(ctx->arena.base);
    if (ctx->batch_arena.base) cudaFree(ctx->batch_arena.base);
    if (ctx->d_ctl) cudaFree(ctx->d_ctl);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    for (int i = 0; i < 10; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < 2; ++i)
        if (ctx->side_ev[i]) cudaEventDestroy(ctx->side_ev[i]);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    if (ctx->graph_pool) cudaMemPoolDestroy(ctx->graph_pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return TC_OK;
}

const char *tc_last_error(const tc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tc_status tc_set_stream(tc_ctx *ctx, void *stream) {
    if (!ctx) return TC_ERR_INVALID;
    DeviceGuard guard(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->side_stream) {  // made again on first use, with the new stream's priority
        cudaStreamSynchronize(ctx->side_stream);
        cudaStreamDestroy(ctx->side_stream);
        ctx->side_stream = nullptr;
    }
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    if (!ctx->stream) {
        if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(ctx, TC_ERR_CUDA, "stream creation failed");
        ctx->stream = ctx->own_stream;
    }
    return TC_OK;
}

tc_status tc_get_tuning(const tc_ctx *ctx, tc_tuning *out) {
    if (!ctx || !out) return TC_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    const Tuning &t = ctx->tune;
    out->warp_cap = t.warp_cap;
    out->block_cap = t.block_cap;
    out->task_work = t.task_work;
    out->warps_per_block = t.warps_per_block;
    out->block_threads = t.block_threads;
    out->warp_task_work = t.warp_task_work;
    out->hub_task_work = t.hub_task_work;
    out->max_v = t.max_v;
    out->hub_group = t.hub_group;
    out->hub_filter_log2 = t.hub_filter_log2;
    out->hub_threads = t.hub_threads;
    out->tiny_cap = t.tiny_cap;
    out->table_kind = t.table_kind;
    out->flat_cap = t.flat_cap;
    out->block_bits_log2 = t.block_bits_log2;
    out->batch_small_slots = t.batch_small_slots;
    return TC_OK;
}

tc_status tc_set_tuning(tc_ctx *ctx, const tc_tuning *t) {
    if (!ctx || !t) return TC_ERR_INVALID;
    Tuning nt;
    nt.warp_cap = t->warp_cap;
    nt.block_cap = t->block_cap;
    nt.task_work = t->task_work;
    nt.warps_per_block = t->warps_per_block;
    nt.block_threads = t->block_threads;
    nt.warp_task_work = t->warp_task_work;
    nt.hub_task_work = t->hub_task_work;
    nt.max_v = t->max_v;
    nt.hub_group = t->hub_group;
    nt.hub_filter_log2 = t->hub_filter_log2;
    nt.hub_threads = t->hub_threads;
    nt.tiny_cap = t->tiny_cap;
    nt.table_kind = t->table_kind;
    nt.flat_cap = t->flat_cap;
    nt.block_bits_log2 = t->block_bits_log2;
    nt.batch_small_slots = t->batch_small_slots;
    const size_t smem_limit = 227 * 1024;
    auto threads_ok = [](uint32_t x) { return x >= 64 && x <= 1024 && x % 32 == 0; };
    if (nt.warp_cap < 1 || nt.warp_cap > 4096 || nt.block_cap < nt.warp_cap || nt.block_cap > 16384 ||
        nt.task_work < 1 || nt.warp_task_work < 1 || nt.hub_task_work < 1 || nt.warps_per_block < 1 ||
        nt.warps_per_block > 8 || !threads_ok(nt.block_threads) || !threads_ok(nt.hub_threads) || nt.max_v < 64 ||
        nt.max_v > 4096 || nt.hub_group < 1 || nt.hub_group > 64 || nt.hub_filter_log2 < 10 ||
        nt.hub_filter_log2 > 20 || nt.tiny_cap > 64 || nt.table_kind > 1 || nt.flat_cap > 4096 ||
        (nt.block_bits_log2 != 0 && (nt.block_bits_log2 < 10 || nt.block_bits_log2 > 20)) || warp_kernel_smem(nt) > smem_limit || block_kernel_smem(nt) > smem_limit ||
        hub_kernel_smem(nt) > smem_limit)
        return set_error(ctx, TC_ERR_INVALID, "tuning out of range");
    ctx->tune = nt;
    return TC_OK;
}

tc_status tc_arena_bytes(const tc_ctx *ctx, uint64_t *bytes) {
    if (!ctx || !bytes) return TC_ERR_INVALID;
    *bytes = ctx->arena.cap + ctx->batch_arena.cap;
    return TC_OK;
}

tc_status tc_graph_from_csr(tc_ctx *ctx, uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int where,
                            int flags, tc_graph **out) {
    if (!ctx || !out || !row_ptr || n == 0xFFFFFFFFu) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (where != TC_HOST && where != TC_DEVICE) return set_error(ctx, TC_ERR_INVALID, "bad `where`");
    if (where == TC_HOST && (flags & TC_BORROW)) return set_error(ctx, TC_ERR_INVALID, "TC_BORROW needs device arrays");
    *out = nullptr;
    DeviceGuard guard(ctx->device);
    uint64_t slots = 0;
    if (where == TC_HOST) {
        slots = row_ptr[n];
    } else {
        TC_CUDA(ctx, cudaMemcpyAsync(&slots, row_ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
        TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (slots && !col) return set_error(ctx, TC_ERR_INVALID, "col is NULL");
    tc_graph *g = new tc_graph();
    g->ctx = ctx;
    g->n = n;
    g->slots = slots;
    if (flags & TC_BORROW) {
        g->rp = const_cast<uint64_t *>(row_ptr);
        g->col = const_cast<uint32_t *>(col);
        g->owned = false;
    } else {
        g->owned = true;
        bool p1 = false, p2 = false;
        const cudaError_t e1 = graph_alloc(ctx, (void **)&g->rp, sizeof(uint64_t) * ((size_t)n + 1), &p1);
        const cudaError_t e2 =
            e1 == cudaSuccess ? graph_alloc(ctx, (void **)&g->col, sizeof(uint32_t) * (size_t)(slots + 1), &p2) : e1;
        g->pooled = p1;  // both come from the same source
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cudaGetLastError();
            tc_graph_free(g);
            return set_error(ctx, TC_ERR_OOM, "graph allocation failed");
        }
        const cudaMemcpyKind kind = where == TC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        cudaError_t e = cudaMemcpyAsync(g->rp, row_ptr, sizeof(uint64_t) * ((size_t)n + 1), kind, ctx->stream);
        if (e == cudaSuccess && slots)
            e = cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * (size_t)slots, kind, ctx->stream);
        if (e != cudaSuccess) {
            tc_graph_free(g);
            return cuda_error(ctx, e, "graph copy");
        }
    }
    return finish_graph(ctx, g, flags & TC_VALIDATE, out);
}

tc_status tc_build_csr(tc_ctx *ctx, uint32_t n, uint64_t n_tuples, const uint32_t *src, const uint32_t *dst,
                       int where, tc_graph **out) {
    if (!ctx || !out || n == 0xFFFFFFFFu || (n_tuples && (!src || !dst)))
        return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (where != TC_HOST && where != TC_DEVICE) return set_error(ctx, TC_ERR_INVALID, "bad `where`");
    *out = nullptr;
    DeviceGuard guard(ctx->device);
    const uint32_t *ds = src, *dd = dst;
    uint32_t *tmp = nullptr;
    if (where == TC_HOST && n_tuples) {
        if (device_alloc(ctx, (void **)&tmp, sizeof(uint32_t) * 2 * (size_t)n_tuples) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, TC_ERR_OOM, "tuple upload allocation failed");
        }
        cudaMemcpyAsync(tmp, src, sizeof(uint32_t) * n_tuples, cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(tmp + n_tuples, dst, sizeof(uint32_t) * n_tuples, cudaMemcpyHostToDevice, ctx->stream);
        ds = tmp;
        dd = tmp + n_tuples;
    }
    uint64_t *rp = nullptr;
    uint32_t *col = nullptr;
    uint64_t slots = 0;
    bool pooled = false;
    tc_status st = build_csr_device(ctx, n, n_tuples, ds, dd, &rp, &col, &slots, &pooled);
    if (tmp) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(tmp);
    }
    if (st != TC_OK) return st;
    tc_graph *g = new tc_graph();
    g->ctx = ctx;
    g->n = n;
    g->slots = slots;
    g->rp = rp;
    g->col = col;
    g->pooled = pooled;
    g->owned = true;
    return finish_graph(ctx, g, 0, out);
}

tc_status tc_graph_info(const tc_graph *g, uint32_t *n, uint64_t *slots, const uint64_t **d_row_ptr,
                        const uint32_t **d_col) {
    if (!g) return TC_ERR_INVALID;
    if (n) *n = g->n;
    if (slots) *slots = g->slots;
    if (d_row_ptr) *d_row_ptr = g->rp;
    if (d_col) *d_col = g->col;
    return TC_OK;
}

tc_status tc_graph_copy_out(tc_ctx *ctx, const tc_graph *g, uint64_t *row_ptr, uint32_t *col, int where) {
    if (!ctx || !g || !row_ptr || (g->slots && !col)) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (where != TC_HOST && where != TC_DEVICE) return set_error(ctx, TC_ERR_INVALID, "bad `where`");
    DeviceGuard guard(ctx->device);
    const cudaMemcpyKind kind = where == TC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    TC_CUDA(ctx, cudaMemcpyAsync(row_ptr, g->rp, sizeof(uint64_t) * ((size_t)g->n + 1), kind, ctx->stream));
    if (g->slots) TC_CUDA(ctx, cudaMemcpyAsync(col, g->col, sizeof(uint32_t) * g->slots, kind, ctx->stream));
    TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TC_OK;
}

tc_status tc_validate(tc_ctx *ctx, const tc_graph *g, int *ok) {
    if (!ctx || !g || !ok) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    DeviceGuard guard(ctx->device);
    return validate_csr_device(ctx, g->n, g->rp, g->col, g->slots, ok);
}

tc_status tc_graph_free(tc_graph *g) {
    if (!g) return TC_ERR_INVALID;
    if (g->owned) {
        DeviceGuard guard(g->ctx->device);
        if (g->ctx->stream) cudaStreamSynchronize(g->ctx->stream);  // its last use on the context is done
        graph_free(g->ctx, g->rp, g->pooled);
        graph_free(g->ctx, g->col, g->pooled);
    }
    delete g;
    return TC_OK;
}

tc_status tc_count_levels(tc_ctx *ctx, const tc_graph *g, uint32_t *d_levels, uint64_t *triangles,
                          tc_stats *stats) {
    if (!ctx || !g) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (g->ctx != ctx && g->ctx->device != ctx->device)
        return set_error(ctx, TC_ERR_INVALID, "graph lives on another device");
    DeviceGuard guard(ctx->device);
    GraphView v;
    v.n = g->n;
    v.slots = g->slots;
    v.rp = g->rp;
    v.col = g->col;
    v.max_deg = g->max_deg;
    GroupSpec none;
    return count_pipeline(ctx, v, d_levels, none, triangles, stats);
}

tc_status tc_count_with_levels(tc_ctx *ctx, const tc_graph *g, const uint32_t *d_levels, uint64_t *triangles,
                               tc_stats *stats) {
    if (!ctx || !g || (g->n && !d_levels)) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (g->ctx != ctx && g->ctx->device != ctx->device)
        return set_error(ctx, TC_ERR_INVALID, "graph lives on another device");
    DeviceGuard guard(ctx->device);
    GraphView v;
    v.n = g->n;
    v.slots = g->slots;
    v.rp = g->rp;
    v.col = g->col;
    v.max_deg = g->max_deg;
    GroupSpec none;
    return count_pipeline(ctx, v, nullptr, none, triangles, stats, d_levels);
}

tc_status tc_count_vertices(tc_ctx *ctx, const tc_graph *g, uint64_t *d_counts, uint64_t *triangles,
                            tc_stats *stats) {
    if (!ctx || !g || (g->n && !d_counts)) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (g->ctx != ctx && g->ctx->device != ctx->device)
        return set_error(ctx, TC_ERR_INVALID, "graph lives on another device");
    DeviceGuard guard(ctx->device);
    GraphView v;
    v.n = g->n;
    v.slots = g->slots;
    v.rp = g->rp;
    v.col = g->col;
    v.max_deg = g->max_deg;
    GroupSpec none;
    return count_pipeline(ctx, v, nullptr, none, triangles, stats, nullptr, d_counts);
}

tc_status tc_list_triangles(tc_ctx *ctx, const tc_graph *g, uint32_t *d_triples, uint64_t capacity,
                            uint64_t *triangles, tc_stats *stats) {
    if (!ctx || !g || (capacity && !d_triples) || capacity > (UINT64_MAX / 12))
        return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (g->ctx != ctx && g->ctx->device != ctx->device)
        return set_error(ctx, TC_ERR_INVALID, "graph lives on another device");
    DeviceGuard guard(ctx->device);
    GraphView v;
    v.n = g->n;
    v.slots = g->slots;
    v.rp = g->rp;
    v.col = g->col;
    v.max_deg = g->max_deg;
    GroupSpec none;
    ListSpec list;
    list.out = d_triples;
    list.capacity = capacity;
    return count_pipeline(ctx, v, nullptr, none, triangles, stats, nullptr, nullptr, &list);
}

tc_status tc_count_alg3(tc_ctx *ctx, const tc_graph *g, uint64_t *triangles, tc_stats *stats) {
    if (!ctx || !g) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    if (g->ctx != ctx && g->ctx->device != ctx->device)
        return set_error(ctx, TC_ERR_INVALID, "graph lives on another device");
    DeviceGuard guard(ctx->device);
    GraphView v;
    v.n = g->n;
    v.slots = g->slots;
    v.rp = g->rp;
    v.col = g->col;
    v.max_deg = g->max_deg;
    GroupSpec none;
    return count_pipeline(ctx, v, nullptr, none, triangles, stats, nullptr, nullptr, nullptr, true);
}

tc_status tc_count(tc_ctx *ctx, const tc_graph *g, uint64_t *triangles, tc_stats *stats) {
    return tc_count_levels(ctx, g, nullptr, triangles, stats);
}

tc_status tc_selftest_barrier(tc_ctx *ctx, uint32_t timeout_ms) {
    if (!ctx || timeout_ms == 0 || timeout_ms > 10000) return set_error(ctx, TC_ERR_INVALID, "bad timeout");
    DeviceGuard guard(ctx->device);
    return selftest_barrier(ctx, timeout_ms);
}

tc_status tc_count_shard(tc_ctx *ctx, const tc_graph *g, uint32_t shard, uint32_t nshards, uint64_t *partial,
                         tc_stats *stats) {
    if (!ctx || nshards == 0 || shard >= nshards) return set_error(ctx, TC_ERR_INVALID, "bad shard");
    ctx->shard = shard;
    ctx->nshards = nshards;
    const tc_status st = tc_count_levels(ctx, g, nullptr, partial, stats);
    ctx->shard = 0;
    ctx->nshards = 1;
    return st;
}

tc_status tc_count_batch(tc_ctx *ctx, uint32_t G, const tc_graph *const *graphs, uint64_t *counts) {
    if (!ctx || (G && (!graphs || !counts))) return set_error(ctx, TC_ERR_INVALID, "bad argument");
    for (uint32_t i = 0; i < G; ++i)
        if (!graphs[i] || graphs[i]->ctx->device != ctx->device)
            return set_error(ctx, TC_ERR_INVALID, "null graph or graph on another device");
    if (G == 0) return TC_OK;
    DeviceGuard guard(ctx->device);
    return count_batch(ctx, G, graphs, counts);
}

}  // extern "C"
