// isect.cu -- hashed intersections of the compacted rows over every oriented
// horizontal edge u -> v (Algorithm 4 with Algorithm 2 on G0), and the
// reduction of the counts into 64-bit totals.
//
// As in the paper's hashed loop, the row of u (the endpoint that comes first
// in the working order, i.e. the higher-degree one under the degree order) is
// put in a hash set once, and the rows of all its horizontal out-neighbours v
// are probed against it: the cost per edge is the length of v's row, at most
// min(d(u), d(v)).  Rows are split by the size s(u) of the hashed row:
//   warp class   s(u) <= warp_cap : one warp per u, table in the warp's slice
//                                   of shared memory;
//   block class  s(u) <= block_cap: one block per task (a slice of u's
//                                   out-edges), table in shared memory;
//   hub class    larger           : one block per task, table in a
//                                   block-private region of global memory.
// Tables use open addressing with linear probing at load factor <= 1/2.
#include "pipeline.cuh"

namespace tc {
namespace {

struct Acc {
    unsigned long long same = 0, cross = 0, probes = 0;
};

template <bool kShared>
__device__ __forceinline__ uint32_t tab_load(const uint32_t *tab, uint32_t slot) {
    if (kShared) return tab[slot];
    return __ldcg(tab + slot);
}

// Insert the distinct ids row[0..len) with `nthreads` cooperating threads
// (thread index `t`).
__device__ __forceinline__ void table_insert(uint32_t *tab, uint32_t shift, uint32_t mask, const uint32_t *row,
                                             uint32_t len, uint32_t t, uint32_t nthreads) {
    for (uint32_t j = t; j < len; j += nthreads) {
        const uint32_t w = row[j];
        uint32_t slot = hash_slot(w, shift);
        while (atomicCAS(tab + slot, kEmpty, w) != kEmpty) slot = (slot + 1) & mask;
    }
}

template <bool kShared>
__device__ __forceinline__ bool table_has(const uint32_t *tab, uint32_t shift, uint32_t mask, uint32_t w) {
    uint32_t slot = hash_slot(w, shift);
    for (;;) {
        const uint32_t k = tab_load<kShared>(tab, slot);
        if (k == w) return true;
        if (k == kEmpty) return false;
        slot = (slot + 1) & mask;
    }
}

// Probe the rows of v = H(u)[k] for k in [k_lo, k_hi) with one warp.  Lanes
// fetch the metadata of 32 out-neighbours at a time; then the warp walks each
// row, lanes striding over its entries.  An entry at position j of row(v) is a
// G0 triangle when j < |H(v)|, else a cross-level triangle.
template <bool kShared>
__device__ __forceinline__ void probe_slice(const uint32_t *tab, uint32_t shift, uint32_t mask,
                                            const uint32_t *__restrict__ hrow, uint32_t k_lo, uint32_t k_hi,
                                            uint32_t k_step, const uint64_t *__restrict__ off2,
                                            const uint32_t *__restrict__ adj2, const uint32_t *__restrict__ hcnt,
                                            Acc &acc) {
    const unsigned lane = lane_id();
    for (uint32_t k0 = k_lo; k0 < k_hi; k0 += k_step) {
        const uint32_t k = k0 + lane;
        uint64_t vb = 0;
        uint32_t vs = 0, vh = 0;
        if (k < k_hi && lane < k_step) {
            const uint32_t v = hrow[k];
            vb = off2[v];
            vs = (uint32_t)(off2[v + 1] - vb);
            vh = hcnt[v];
        }
        const uint32_t cnt = min(32u, min(k_step, k_hi - k0));
        for (uint32_t t = 0; t < cnt; ++t) {
            const uint64_t b = __shfl_sync(0xFFFFFFFFu, vb, t);
            const uint32_t len = __shfl_sync(0xFFFFFFFFu, vs, t);
            const uint32_t hv = __shfl_sync(0xFFFFFFFFu, vh, t);
            acc.probes += len;
            for (uint32_t j = lane; j < len; j += 32) {
                const uint32_t w = adj2[b + j];
                if (table_has<kShared>(tab, shift, mask, w)) {
                    if (j < hv) ++acc.same; else ++acc.cross;
                }
            }
        }
    }
}

__device__ __forceinline__ uint32_t table_size_for(uint32_t len, uint32_t min_size) {
    uint32_t ts = min_size;
    while (ts < 2 * len) ts <<= 1;
    return ts;
}

__device__ __forceinline__ uint32_t group_of(const GroupSpec &g, uint32_t u) {
    uint32_t a = 0, b = g.n_groups;
    while (b - a > 1) {
        uint32_t m = (a + b) >> 1;
        if (g.vertex_start[m] <= u) a = m; else b = m;
    }
    return a;
}

// Reduce a warp's counters into the control block (class c: 0 warp, 1 block, 2 hub).
__device__ __forceinline__ void flush(Acc &acc, Ctl *ctl, int c, unsigned long long build_elems,
                                      unsigned long long rows) {
    const unsigned long long s = warp_sum(acc.same), x = warp_sum(acc.cross), p = warp_sum(acc.probes);
    if (lane_id() == 0) {
        if (s) atomicAdd(&ctl->t_same, s);
        if (x) atomicAdd(&ctl->t_cross, x);
        if (p) {
            atomicAdd(&ctl->probes, p);
            atomicAdd(&ctl->cls_probes[c], p);
        }
        if (build_elems) atomicAdd(&ctl->cls_build[c], build_elems);
        if (rows) atomicAdd(&ctl->cls_rows[c], rows);
    }
}

// Warp class: one warp per row u, dynamically scheduled.
__global__ void k_isect_warp(const uint32_t *__restrict__ wlist, const uint64_t *__restrict__ off2,
                             const uint32_t *__restrict__ adj2, const uint32_t *__restrict__ hcnt, Ctl *ctl,
                             uint32_t table_slots, GroupSpec groups) {
    extern __shared__ uint32_t smem[];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t *tab = smem + (size_t)warp * table_slots;
    const uint32_t nw = ctl->n_warp_u;
    Acc acc;
    unsigned long long build = 0, rows = 0;
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(&ctl->warp_next, 1u);
        i = __shfl_sync(0xFFFFFFFFu, i, 0);
        if (i >= nw) break;
        const uint32_t u = wlist[i];
        const uint64_t ub = off2[u];
        const uint32_t su = (uint32_t)(off2[u + 1] - ub);
        const uint32_t hu = hcnt[u];
        const uint32_t ts = table_size_for(su, 64);
        const uint32_t shift = __clz(ts) + 1, mask = ts - 1;
        for (uint32_t j = lane; j < ts; j += 32) tab[j] = kEmpty;
        __syncwarp();
        table_insert(tab, shift, mask, adj2 + ub, su, lane, 32);
        __syncwarp();
        build += su;
        ++rows;
        const unsigned long long before = acc.same + acc.cross;
        probe_slice<true>(tab, shift, mask, adj2 + ub, 0, hu, 32, off2, adj2, hcnt, acc);
        if (groups.n_groups) {
            const unsigned long long found = warp_sum(acc.same + acc.cross - before);
            if (lane == 0 && found) atomicAdd(&groups.counts[group_of(groups, u)], found);
        }
        __syncwarp();
    }
    flush(acc, ctl, 0, lane == 0 ? build : 0, lane == 0 ? rows : 0);
}

// Block and hub classes: one block per task (u, slice t of nt).
template <bool kShared>
__global__ void k_isect_block(const uint32_t *__restrict__ blist, const uint32_t *__restrict__ ntask,
                              const unsigned long long *__restrict__ tpref, const uint64_t *__restrict__ off2,
                              const uint32_t *__restrict__ adj2, const uint32_t *__restrict__ hcnt, Ctl *ctl,
                              uint32_t block_cap, uint32_t *hub_tables, uint64_t hub_slots, GroupSpec groups) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t s_task[4];
    __shared__ unsigned long long s_found;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t nb = ctl->n_block_u;
    const unsigned long long total = tpref[nb];
    uint32_t *tab = kShared ? smem : hub_tables + (size_t)blockIdx.x * hub_slots;
    Acc acc;
    unsigned long long build = 0, tasks = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long k = atomicAdd(&ctl->block_next, 1u);
            uint32_t i = 0xFFFFFFFFu;
            if (k < total) {
                uint32_t a = 0, b = nb;
                while (b - a > 1) {
                    uint32_t m = (a + b) >> 1;
                    if (tpref[m] <= k) a = m; else b = m;
                }
                i = a;
            }
            s_task[0] = i;
            s_task[1] = i != 0xFFFFFFFFu ? (uint32_t)(k - tpref[i]) : 0;
            s_found = 0;
        }
        __syncthreads();
        const uint32_t i = s_task[0];
        if (i == 0xFFFFFFFFu) break;
        const uint32_t u = blist[i];
        const uint32_t su = (uint32_t)(off2[u + 1] - off2[u]);
        // this block class takes rows above or below block_cap, per instantiation
        const bool mine = kShared ? su <= block_cap : su > block_cap;
        if (mine) {
            const uint32_t t = s_task[1], nt = ntask[i];
            const uint64_t ub = off2[u];
            const uint32_t hu = hcnt[u];
            const uint32_t k_lo = (uint32_t)((uint64_t)t * hu / nt), k_hi = (uint32_t)((uint64_t)(t + 1) * hu / nt);
            const uint32_t ts = table_size_for(su, 64);
            const uint32_t shift = __clz(ts) + 1, mask = ts - 1;
            for (uint32_t j = threadIdx.x; j < ts; j += blockDim.x) tab[j] = kEmpty;
            if (!kShared) __threadfence_block();
            __syncthreads();
            table_insert(tab, shift, mask, adj2 + ub, su, threadIdx.x, blockDim.x);
            if (!kShared) __threadfence_block();
            __syncthreads();
            if (threadIdx.x == 0) {
                if (t == 0) build += su;
                ++tasks;
            }
            const unsigned long long before = acc.same + acc.cross;
            // warps take 32-edge chunks of the slice in turn
            for (uint32_t c0 = k_lo + warp * 32; c0 < k_hi; c0 += nwarps * 32)
                probe_slice<kShared>(tab, shift, mask, adj2 + ub, c0, min(c0 + 32, k_hi), 32, off2, adj2, hcnt, acc);
            if (groups.n_groups) {
                const unsigned long long found = warp_sum(acc.same + acc.cross - before);
                if (lane == 0 && found) atomicAdd(&s_found, found);
            }
        }
        __syncthreads();
        if (mine && groups.n_groups && threadIdx.x == 0 && s_found)
            atomicAdd(&groups.counts[group_of(groups, u)], s_found);
    }
    flush(acc, ctl, kShared ? 1 : 2, threadIdx.x == 0 ? build : 0, threadIdx.x == 0 ? tasks : 0);
}

}  // namespace

tc_status intersect(tc_ctx *ctx, PipeBufs &b, uint32_t n) {
    cudaStream_t s = ctx->stream;
    const Tuning &tu = ctx->tune;
    const Ctl &h = *ctx->h_ctl;  // pulled after build_rows
    auto *tpref = reinterpret_cast<const unsigned long long *>(b.tpref);
    // ev[4..7] bracket the warp, block and hub kernels
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[4], s));
    if (h.n_warp_u) {
        const uint32_t slots = [&] {
            uint32_t t = 64;
            while (t < 2 * tu.warp_cap) t <<= 1;
            return t;
        }();
        const size_t smem = (size_t)tu.warps_per_block * slots * sizeof(uint32_t);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_isect_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect_warp, 32 * tu.warps_per_block, smem));
        if (per_sm < 1) per_sm = 1;
        unsigned grid = (unsigned)(ctx->num_sms * per_sm);
        const unsigned need = (h.n_warp_u + tu.warps_per_block - 1) / tu.warps_per_block;
        if (grid > need) grid = need;
        k_isect_warp<<<grid, 32 * tu.warps_per_block, smem, s>>>(b.wlist, b.off2, b.adj2, b.hcnt, ctx->d_ctl, slots,
                                                                  b.groups);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[5], s));
    bool hub = false;
    if (h.n_block_u) {
        const uint32_t slots = [&] {
            uint32_t t = 64;
            while (t < 2 * tu.block_cap) t <<= 1;
            return t;
        }();
        const size_t smem = (size_t)slots * sizeof(uint32_t);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_isect_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect_block<true>, tu.block_threads, smem));
        if (per_sm < 1) per_sm = 1;
        k_isect_block<true><<<(unsigned)(ctx->num_sms * per_sm), tu.block_threads, smem, s>>>(
            b.blist, b.ntask, tpref, b.off2, b.adj2, b.hcnt, ctx->d_ctl, tu.block_cap, nullptr, 0, b.groups);
        note_launch(ctx);
        hub = h.max_s2 > tu.block_cap;
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[6], s));
    if (hub) {
        {
            TC_CUDA(ctx, cudaMemsetAsync(&ctx->d_ctl->block_next, 0, sizeof(unsigned), s));
            k_isect_block<false><<<b.hub_blocks, tu.block_threads, 0, s>>>(
                b.blist, b.ntask, tpref, b.off2, b.adj2, b.hcnt, ctx->d_ctl, tu.block_cap, b.hub_tables, b.hub_slots,
                b.groups);
            note_launch(ctx);
        }
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[7], s));
    ctx->isect_flags = (h.n_warp_u ? 1u : 0u) | (h.n_block_u ? 2u : 0u) | (hub ? 4u : 0u);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
