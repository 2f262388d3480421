// isect.cu -- hashed intersections of the compacted rows over every oriented
// horizontal edge u -> v (Algorithm 4 with Algorithm 2 on G0), and the
// reduction of the counts into 64-bit totals.
//
// As in the paper's hashed loop, the row of u (the endpoint that comes first
// in the working order, the higher-degree one under the degree order) is put
// in a set once, and the rows of its horizontal out-neighbours v are probed
// against it; the cost per edge is |row(v)| <= min(d(u), d(v)).  Rows are
// split by the size s(u) of the hashed row, and every row's out-edges are cut
// into tasks of bounded probe work:
//   warp class  s(u) <= warp_cap : one warp per task, open-addressing table in
//                                  the warp's slice of shared memory;
//   block class s(u) <= block_cap: one block per task, table in shared memory;
//   hub class   larger           : hub rows are taken `hub_group` at a time,
//                                  each gets an n-bit bitmap in global memory
//                                  (L2-resident while its group runs) and all
//                                  SMs probe the group's tasks against them.
// Probing is flattened: the rows of a batch of v's are viewed as one list and
// every lane keeps kUnroll independent loads in flight.
#include <algorithm>

#include "pipeline.cuh"

namespace tc {
namespace {

constexpr int kUnroll = 8;                 // elements in flight per lane
constexpr uint32_t kChunk = 32 * kUnroll;  // elements per warp step

struct Acc {
    unsigned long long same = 0, cross = 0, probes = 0;
};

// ---------------------------------------------------------------------------- set representations

struct SmemTable {  // open addressing, linear probing, load factor <= 1/2
    uint32_t *tab;
    uint32_t shift, mask;
    __device__ __forceinline__ bool has(uint32_t w) const {
        uint32_t slot = hash_slot(w, shift);
        for (;;) {
            const uint32_t k = tab[slot];
            if (k == w) return true;
            if (k == kEmpty) return false;
            slot = (slot + 1) & mask;
        }
    }
};

struct GlobalBitmap {  // one bit per vertex id, read-only while probing
    const uint32_t *bits;
    __device__ __forceinline__ bool has(uint32_t w) const { return (__ldg(bits + (w >> 5)) >> (w & 31)) & 1u; }
};

__device__ __forceinline__ uint32_t table_size_for(uint32_t len) {
    uint32_t ts = 64;
    while (ts < 2 * len) ts <<= 1;
    return ts;
}

// Size a shared table for len ids and clear it (threads t of nthreads).
__device__ __forceinline__ SmemTable clear_table(uint32_t *tab, uint32_t len, uint32_t t, uint32_t nthreads) {
    const uint32_t ts = table_size_for(len);
    SmemTable T{tab, (uint32_t)__clz(ts) + 1u, ts - 1u};
    for (uint32_t j = t; j < ts; j += nthreads) tab[j] = kEmpty;
    return T;
}

// Insert the distinct ids row[0..len) (after a barrier following clear_table).
__device__ __forceinline__ void fill_table(const SmemTable &T, const uint32_t *__restrict__ row, uint32_t len,
                                           uint32_t t, uint32_t nthreads) {
    for (uint32_t j = t; j < len; j += nthreads) {
        const uint32_t w = row[j];
        uint32_t slot = hash_slot(w, T.shift);
        while (atomicCAS(T.tab + slot, kEmpty, w) != kEmpty) slot = (slot + 1) & T.mask;
    }
}

// ---------------------------------------------------------------------------- flattened probing

// Probe the flattened list of `nv` rows described by pre[0..nv] (exclusive
// prefix of lengths, pre[nv] = total), rb[] (row starts in adj2) and rh[]
// (|H(v)|), all in shared memory.  The warp takes chunks c_begin,
// c_begin + c_step, ... of kChunk elements.  An element at position j of
// row(v) is a G0 triangle when j < |H(v)|, otherwise cross-level.
template <class Set>
__device__ __forceinline__ void probe_flat(const Set &set, const uint32_t *__restrict__ adj2,
                                           const uint32_t *pre, const unsigned long long *rb, const uint32_t *rh,
                                           uint32_t nv, uint32_t c_begin, uint32_t c_step, Acc &acc) {
    const unsigned lane = lane_id();
    const uint32_t total = pre[nv];
    for (uint32_t f0 = c_begin * kChunk; f0 < total; f0 += c_step * kChunk) {
        // row holding this lane's first element: largest t with pre[t] <= f
        const uint32_t f = f0 + lane;
        uint32_t t = 0;
        if (f < total) {
            uint32_t a = 0, b = nv;
            while (b - a > 1) {
                const uint32_t m = (a + b) >> 1;
                if (pre[m] <= f) a = m; else b = m;
            }
            t = a;
        }
        uint32_t lo = pre[t], hi = pre[t + 1];
        unsigned long long base = rb[t];
        uint32_t hv = rh[t];
        uint32_t w[kUnroll];
        bool cls[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int i = 0; i < kUnroll; ++i) {
            const uint32_t fi = f0 + (uint32_t)i * 32u + lane;
            ok[i] = fi < total;
            w[i] = 0;
            cls[i] = false;
            if (ok[i]) {
                while (fi >= hi) {  // advance to the row holding fi; fi < total = pre[nv] bounds t < nv
                    ++t;
                    lo = hi;
                    hi = pre[t + 1];
                    base = rb[t];
                    hv = rh[t];
                }
                const uint32_t j = fi - lo;
                w[i] = adj2[base + j];
                cls[i] = j < hv;
            }
        }
#pragma unroll
        for (int i = 0; i < kUnroll; ++i) {
            if (ok[i] && set.has(w[i])) {
                if (cls[i]) ++acc.same; else ++acc.cross;
            }
        }
    }
    if (lane == 0 && c_begin == 0) acc.probes += total;
}

// Block-wide exclusive scan of len[0..nv) into pre[0..nv]; all threads of the
// block call it; ends with a barrier.
__device__ __forceinline__ void block_scan_lengths(const uint32_t *len, uint32_t *pre, uint32_t nv) {
    __shared__ uint32_t warp_tot[32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t per = (nv + blockDim.x - 1) / blockDim.x;  // items per thread (contiguous)
    const uint32_t beg = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (beg + i < nv) sum += len[beg + i];
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nwarps ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= (unsigned)o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    uint32_t run = (warp ? warp_tot[warp - 1] : 0u) + x - sum;
    for (uint32_t i = 0; i < per; ++i) {
        if (beg + i < nv) {
            pre[beg + i] = run;
            run += len[beg + i];
        }
    }
    if (threadIdx.x == 0) pre[nv] = warp_tot[nwarps - 1];
    __syncthreads();
}

__device__ __forceinline__ uint32_t group_of(const GroupSpec &g, uint32_t u) {
    uint32_t a = 0, b = g.n_groups;
    while (b - a > 1) {
        const uint32_t m = (a + b) >> 1;
        if (g.vertex_start[m] <= u) a = m; else b = m;
    }
    return a;
}

// Reduce a warp's counters into the control block (class c: 0 warp, 1 block, 2 hub).
__device__ __forceinline__ void flush(const Acc &acc, Ctl *ctl, int c, unsigned long long build_elems,
                                      unsigned long long tasks) {
    const unsigned long long s = warp_sum(acc.same), x = warp_sum(acc.cross), p = warp_sum(acc.probes);
    if (lane_id() == 0) {
        if (s) atomicAdd(&ctl->t_same, s);
        if (x) atomicAdd(&ctl->t_cross, x);
        if (p) {
            atomicAdd(&ctl->probes, p);
            atomicAdd(&ctl->cls_probes[c], p);
        }
        if (build_elems) atomicAdd(&ctl->cls_build[c], build_elems);
        if (tasks) atomicAdd(&ctl->cls_rows[c], tasks);
    }
}

// ---------------------------------------------------------------------------- warp class

struct WarpMeta {
    unsigned long long b[32];
    uint32_t pre[33];
    uint32_t h[32];
    uint32_t pad[3];
};

__global__ void __launch_bounds__(1024) k_isect_warp(const uint2 *__restrict__ tasks, const uint32_t *__restrict__ rows,
                                                    const uint32_t *__restrict__ ntask,
                                                    const uint64_t *__restrict__ off2, const uint32_t *__restrict__ adj2,
                                                    const uint32_t *__restrict__ hcnt, Ctl *ctl, uint32_t table_slots,
                                                    GroupSpec groups) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    WarpMeta *meta = reinterpret_cast<WarpMeta *>(smem_raw) + warp;
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem_raw + sizeof(WarpMeta) * nwarps) + (size_t)warp * table_slots;
    const unsigned long long ntasks = ctl->n_tasks[0];
    Acc acc;
    unsigned long long build = 0, done = 0;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(&ctl->task_next[0], 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= ntasks) break;
        const uint2 task = tasks[k];
        const uint32_t u = rows[task.x], nt = ntask[task.x];
        const uint64_t ub = off2[u];
        const uint32_t su = (uint32_t)(off2[u + 1] - ub);
        const uint32_t hu = hcnt[u];
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * hu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * hu / nt);
        const SmemTable T = clear_table(tab, su, lane, 32);
        __syncwarp();
        fill_table(T, adj2 + ub, su, lane, 32);
        __syncwarp();
        if (task.y == 0) build += su;
        ++done;
        const unsigned long long before = acc.same + acc.cross;
        for (uint32_t k0 = k_lo; k0 < k_hi; k0 += 32) {
            const uint32_t kk = k0 + lane;
            uint32_t len = 0, hv = 0;
            unsigned long long b = 0;
            if (kk < k_hi) {
                const uint32_t v = adj2[ub + kk];
                b = off2[v];
                len = (uint32_t)(off2[v + 1] - b);
                hv = hcnt[v];
            }
            uint32_t x = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= (unsigned)o) x += y;
            }
            meta->pre[lane + 1] = x;
            if (lane == 0) meta->pre[0] = 0;
            meta->b[lane] = b;
            meta->h[lane] = hv;
            __syncwarp();
            const uint32_t nv = min(32u, k_hi - k0);
            probe_flat(T, adj2, meta->pre, meta->b, meta->h, nv, 0, 1, acc);
            __syncwarp();
        }
        if (groups.n_groups) {
            const unsigned long long found = warp_sum(acc.same + acc.cross - before);
            if (lane == 0 && found) atomicAdd(&groups.counts[group_of(groups, u)], found);
        }
        __syncwarp();
    }
    flush(acc, ctl, 0, lane == 0 ? build : 0, lane == 0 ? done : 0);
}

// ---------------------------------------------------------------------------- block and hub classes

// Per-task shared metadata of up to max_v out-neighbours.
struct SliceSmem {
    unsigned long long *b;
    uint32_t *h, *len, *pre;
};

__device__ __forceinline__ SliceSmem carve_slice(unsigned char *p, uint32_t max_v) {
    SliceSmem s;
    s.b = reinterpret_cast<unsigned long long *>(p);
    s.h = reinterpret_cast<uint32_t *>(p + 8ull * max_v);
    s.len = s.h + max_v;
    s.pre = s.len + max_v;
    return s;
}

__host__ __device__ constexpr size_t slice_smem_bytes(uint32_t max_v) { return 8ull * max_v + 12ull * max_v + 16; }

// Load the metadata of v = hrow[k], k in [k_lo, k_hi), and scan the lengths.
__device__ __forceinline__ uint32_t load_slice(const SliceSmem &S, const uint32_t *__restrict__ hrow, uint32_t k_lo,
                                               uint32_t k_hi, const uint64_t *__restrict__ off2,
                                               const uint32_t *__restrict__ hcnt) {
    const uint32_t nv = k_hi - k_lo;
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
        const uint32_t v = hrow[k_lo + i];
        const unsigned long long b = off2[v];
        S.b[i] = b;
        S.len[i] = (uint32_t)(off2[v + 1] - b);
        S.h[i] = hcnt[v];
    }
    __syncthreads();
    block_scan_lengths(S.len, S.pre, nv);
    return nv;
}

// Thread 0 takes the next task index of class c; all threads see it.
__device__ __forceinline__ bool next_task(Ctl *ctl, int c, unsigned long long first, unsigned long long last,
                                          const uint2 *tasks, uint2 *s_task) {
    if (threadIdx.x == 0) {
        const unsigned long long k = first + atomicAdd(&ctl->task_next[c], 1u);
        s_task[0] = k < last ? tasks[k] : make_uint2(0xFFFFFFFFu, 0u);
    }
    __syncthreads();
    return s_task[0].x != 0xFFFFFFFFu;
}

__global__ void __launch_bounds__(1024) k_isect_block(const uint2 *__restrict__ tasks, const uint32_t *__restrict__ rows,
                                                      const uint32_t *__restrict__ ntask,
                                                      const uint64_t *__restrict__ off2,
                                                      const uint32_t *__restrict__ adj2,
                                                      const uint32_t *__restrict__ hcnt, Ctl *ctl, uint32_t max_v,
                                                      GroupSpec groups) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint2 s_task[1];
    __shared__ unsigned long long s_found;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const SliceSmem S = carve_slice(smem_raw, max_v);
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem_raw + ((slice_smem_bytes(max_v) + 15) & ~size_t(15)));
    const unsigned long long ntasks = ctl->n_tasks[1];
    Acc acc;
    unsigned long long build = 0, done = 0;
    for (;;) {
        if (threadIdx.x == 0) s_found = 0;
        if (!next_task(ctl, 1, 0, ntasks, tasks, s_task)) break;
        const uint2 task = s_task[0];
        const uint32_t u = rows[task.x], nt = ntask[task.x];
        const uint64_t ub = off2[u];
        const uint32_t su = (uint32_t)(off2[u + 1] - ub);
        const uint32_t hu = hcnt[u];
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * hu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * hu / nt);
        const SmemTable T = clear_table(tab, su, threadIdx.x, blockDim.x);
        const uint32_t nv = load_slice(S, adj2 + ub, k_lo, k_hi, off2, hcnt);  // has barriers after the clear
        fill_table(T, adj2 + ub, su, threadIdx.x, blockDim.x);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (task.y == 0) build += su;
            ++done;
        }
        const unsigned long long before = acc.same + acc.cross;
        probe_flat(T, adj2, S.pre, S.b, S.h, nv, warp, nwarps, acc);
        if (groups.n_groups) {
            const unsigned long long found = warp_sum(acc.same + acc.cross - before);
            if (lane == 0 && found) atomicAdd(&s_found, found);
        }
        __syncthreads();
        if (groups.n_groups && threadIdx.x == 0 && s_found) atomicAdd(&groups.counts[group_of(groups, u)], s_found);
    }
    flush(acc, ctl, 1, threadIdx.x == 0 ? build : 0, threadIdx.x == 0 ? done : 0);
}

// Set the bits of hub rows rows[i0 .. i0+g) into bitmaps bits + r * words.
__global__ void k_hub_set(const uint32_t *__restrict__ rows, uint32_t i0, uint32_t g,
                          const uint64_t *__restrict__ off2, const uint32_t *__restrict__ adj2, uint32_t *bits,
                          uint64_t words) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t r = 0; r < g; ++r) {
        const uint32_t u = rows[i0 + r];
        const uint64_t b = off2[u], e = off2[u + 1];
        uint32_t *bm = bits + (uint64_t)r * words;
        for (uint64_t j = b + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < e; j += stride) {
            const uint32_t w = adj2[j];
            atomicOr(bm + (w >> 5), 1u << (w & 31));
        }
    }
}

// Probe the tasks [first, last) of the hub rows with row index in
// [i0, i0 + hub_group) against their bitmaps.
__global__ void __launch_bounds__(1024) k_isect_hub(const uint2 *__restrict__ tasks, unsigned long long first,
                                                    unsigned long long last, const uint32_t *__restrict__ rows,
                                                    const uint32_t *__restrict__ ntask, uint32_t i0,
                                                    const uint64_t *__restrict__ off2, const uint32_t *__restrict__ adj2,
                                                    const uint32_t *__restrict__ hcnt, Ctl *ctl, const uint32_t *bits,
                                                    uint64_t words, uint32_t max_v, GroupSpec groups) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint2 s_task[1];
    __shared__ unsigned long long s_found;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const SliceSmem S = carve_slice(smem_raw, max_v);
    Acc acc;
    unsigned long long build = 0, done = 0;
    for (;;) {
        if (threadIdx.x == 0) s_found = 0;
        if (!next_task(ctl, 2, first, last, tasks, s_task)) break;
        const uint2 task = s_task[0];
        const uint32_t u = rows[task.x], nt = ntask[task.x];
        const uint64_t ub = off2[u];
        const uint32_t hu = hcnt[u];
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * hu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * hu / nt);
        const GlobalBitmap B{bits + (uint64_t)(task.x - i0) * words};
        const uint32_t nv = load_slice(S, adj2 + ub, k_lo, k_hi, off2, hcnt);
        if (threadIdx.x == 0) {
            if (task.y == 0) build += (uint32_t)(off2[u + 1] - ub);
            ++done;
        }
        const unsigned long long before = acc.same + acc.cross;
        probe_flat(B, adj2, S.pre, S.b, S.h, nv, warp, nwarps, acc);
        if (groups.n_groups) {
            const unsigned long long found = warp_sum(acc.same + acc.cross - before);
            if (lane == 0 && found) atomicAdd(&s_found, found);
        }
        __syncthreads();
        if (groups.n_groups && threadIdx.x == 0 && s_found) atomicAdd(&groups.counts[group_of(groups, u)], s_found);
    }
    flush(acc, ctl, 2, threadIdx.x == 0 ? build : 0, threadIdx.x == 0 ? done : 0);
}

uint32_t pow2_at_least(uint64_t x) {
    uint32_t t = 64;
    while (t < x) t <<= 1;
    return t;
}

}  // namespace

size_t warp_kernel_smem(const Tuning &tu) {
    return (size_t)tu.warps_per_block * (sizeof(WarpMeta) + 4ull * pow2_at_least(2ull * tu.warp_cap));
}
size_t block_kernel_smem(const Tuning &tu) {
    return ((slice_smem_bytes(tu.max_v) + 15) & ~size_t(15)) + 4ull * pow2_at_least(2ull * tu.block_cap);
}
size_t hub_kernel_smem(const Tuning &tu) { return slice_smem_bytes(tu.max_v); }

tc_status intersect(tc_ctx *ctx, PipeBufs &b, uint32_t n) {
    (void)n;
    cudaStream_t s = ctx->stream;
    const Tuning &tu = ctx->tune;
    const Ctl &h = *ctx->h_ctl;  // pulled after planning
    // ev[4..7] bracket the warp, block and hub kernels
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[4], s));
    if (h.n_tasks[0]) {
        const uint32_t slots = pow2_at_least(2ull * tu.warp_cap);
        const size_t smem = warp_kernel_smem(tu);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_isect_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect_warp, 32 * tu.warps_per_block, smem));
        if (per_sm < 1) per_sm = 1;
        uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
        const uint64_t need = (h.n_tasks[0] + tu.warps_per_block - 1) / tu.warps_per_block;
        if (grid > need) grid = need;
        k_isect_warp<<<(unsigned)grid, 32 * tu.warps_per_block, smem, s>>>(b.tasks[0], b.rows[0], b.ntask[0], b.off2,
                                                                            b.adj2, b.hcnt, ctx->d_ctl, slots, b.groups);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[5], s));
    if (h.n_tasks[1]) {
        const size_t smem = block_kernel_smem(tu);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_isect_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect_block, tu.block_threads, smem));
        if (per_sm < 1) per_sm = 1;
        uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
        if (grid > h.n_tasks[1]) grid = h.n_tasks[1];
        k_isect_block<<<(unsigned)grid, tu.block_threads, smem, s>>>(b.tasks[1], b.rows[1], b.ntask[1], b.off2, b.adj2,
                                                                     b.hcnt, ctx->d_ctl, tu.max_v, b.groups);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[6], s));
    const uint32_t nh = h.n_rows[2];
    if (nh) {
        // task ranges of the hub rows: the host walks the groups
        std::vector<unsigned long long> pref(nh + 1);
        TC_CUDA(ctx, cudaMemcpyAsync(pref.data(), b.tpref[2], 8ull * (nh + 1), cudaMemcpyDeviceToHost, s));
        TC_CUDA(ctx, cudaStreamSynchronize(s));
        const size_t smem = hub_kernel_smem(tu);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_isect_hub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect_hub, tu.hub_threads, smem));
        if (per_sm < 1) per_sm = 1;
        for (uint32_t i0 = 0; i0 < nh; i0 += tu.hub_group) {
            const uint32_t g = std::min<uint32_t>(tu.hub_group, nh - i0);
            TC_CUDA(ctx, cudaMemsetAsync(b.hub_bits, 0, 4ull * b.hub_words * g, s));
            TC_CUDA(ctx, cudaMemsetAsync(&ctx->d_ctl->task_next[2], 0, sizeof(unsigned), s));
            k_hub_set<<<(unsigned)ctx->num_sms * 4u, 256, 0, s>>>(b.rows[2], i0, g, b.off2, b.adj2, b.hub_bits,
                                                                 b.hub_words);
            const unsigned long long first = pref[i0], last = pref[i0 + g];
            uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
            if (grid > last - first) grid = last - first;
            k_isect_hub<<<(unsigned)grid, tu.hub_threads, smem, s>>>(b.tasks[2], first, last, b.rows[2], b.ntask[2], i0,
                                                                     b.off2, b.adj2, b.hcnt, ctx->d_ctl, b.hub_bits,
                                                                     b.hub_words, tu.max_v, b.groups);
            note_launch(ctx, 2);
        }
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[7], s));
    ctx->isect_flags = (h.n_tasks[0] ? 1u : 0u) | (h.n_tasks[1] ? 2u : 0u) | (nh ? 4u : 0u);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
