// rows.cu -- partition of E into E0 / E1, orientation of E0 by the working
// order, and compaction into one row per vertex (Algorithm 4, partition loop).
//
// For every vertex x the compacted row is  [ H(x) | G1(x) ]  with
//   H(x)  = { y in N(x) : L(y) == L(x), x precedes y }   (G0, oriented)
//   G1(x) = { y in N(x) : L(y) != L(x) }                 (level-spanning)
// each part ascending (the CSR row order is kept).  Because L(u) == L(v) on a
// horizontal edge u -> v, a common element w of row(u) and row(v) lies in
// H(u) and H(v) when L(w) == L(u) (a triangle inside G0, counted once at its
// first edge: Algorithm 2 on G0) and in G1(u) and G1(v) otherwise (a triangle
// with exactly one horizontal edge: the hashed G1 loop of Algorithm 4).  So
// one intersection per horizontal edge counts both kinds, and the position of
// w in row(v) (below or above |H(v)|) tells which kind it is.
#include "pipeline.cuh"

namespace tc {
namespace {

// Each lane owns one vertex x; rows of degree <= kSmallRow are handled by
// their lane alone (sequential, in order), larger rows by the whole warp one
// at a time (lanes stride over the row, ballots keep the order).
constexpr uint32_t kSmallRow = 32;

// Level and degree of a neighbour, either from the two arrays or from one
// packed word (level << 24 | degree) when every level is < 255 and every
// degree < 2^24: one random 4-byte read instead of two.
struct LevelDeg {
    const uint32_t *L, *deg, *packed;
    __device__ __forceinline__ void get(uint32_t y, uint32_t &ly, uint32_t &dy) const {
        if (packed) {
            const uint32_t p = packed[y];
            ly = p >> 24;
            dy = p & 0xFFFFFFu;
        } else {
            ly = L[y];
            dy = 0xFFFFFFFFu;  // loaded on demand
        }
    }
    __device__ __forceinline__ uint32_t degree(uint32_t y, uint32_t dy) const { return packed ? dy : deg[y]; }
};

__device__ __forceinline__ bool is_h(uint32_t x, uint32_t dx, uint32_t lx, uint32_t y, const LevelDeg &ld,
                                     uint32_t order, bool *is_g) {
    uint32_t ly, dy;
    ld.get(y, ly, dy);
    if (ly != lx) {
        *is_g = true;
        return false;
    }
    *is_g = false;
    return precedes(x, dx, y, ld.degree(y, dy), order);
}

__global__ void k_pack_level_deg(uint32_t n, const uint32_t *__restrict__ L, const uint32_t *__restrict__ deg,
                                 uint32_t *__restrict__ packed) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        packed[v] = (L[v] << 24) | deg[v];
}

__global__ void k_row_count(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                            const uint32_t *__restrict__ deg, const uint32_t *__restrict__ L, LevelDeg ld,
                            uint32_t *__restrict__ hcnt, uint32_t *__restrict__ scnt, Ctl *ctl, uint32_t order) {
    __shared__ unsigned long long s_e0;
    if (threadIdx.x == 0) s_e0 = 0;
    __syncthreads();
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_round = ((uint64_t)n + 31) & ~uint64_t(31);
    unsigned long long e0 = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_round; x += stride) {
        const bool valid = x < n;
        const uint32_t dx = valid ? deg[x] : 0;
        const uint32_t lx = valid ? L[x] : 0;
        const uint64_t b = valid ? rp[x] : 0;
        uint32_t h = 0, g = 0;
        if (dx <= kSmallRow) {
            for (uint32_t j = 0; j < dx; ++j) {
                bool isg;
                if (is_h((uint32_t)x, dx, lx, col[b + j], ld, order, &isg)) ++h;
                g += isg;
            }
        }
        unsigned big = __ballot_sync(0xFFFFFFFFu, dx > kSmallRow);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t bx = (uint32_t)__shfl_sync(0xFFFFFFFFu, (unsigned long long)x, src);
            const uint32_t bd = __shfl_sync(0xFFFFFFFFu, dx, src);
            const uint32_t bl = __shfl_sync(0xFFFFFFFFu, lx, src);
            const uint64_t bb = __shfl_sync(0xFFFFFFFFu, b, src);
            uint32_t hh = 0, gg = 0;
            for (uint32_t j = lane; j < bd; j += 32) {
                bool isg;
                if (is_h(bx, bd, bl, col[bb + j], ld, order, &isg)) ++hh;
                gg += isg;
            }
            hh = warp_sum(hh);
            gg = warp_sum(gg);
            if ((int)lane == src) {
                h = hh;
                g = gg;
            }
        }
        if (valid) {
            hcnt[x] = h;
            scnt[x] = h + g;
            e0 += h;
        }
    }
    e0 = warp_sum(e0);
    if (lane == 0 && e0) atomicAdd(&s_e0, e0);
    __syncthreads();
    if (threadIdx.x == 0 && s_e0) atomicAdd(&ctl->e0, s_e0);
}

__global__ void k_row_fill(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                           const uint32_t *__restrict__ deg, const uint32_t *__restrict__ L, LevelDeg ld,
                           const uint32_t *__restrict__ hcnt, const uint64_t *__restrict__ off2,
                           uint32_t *__restrict__ adj2, uint32_t order) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_round = ((uint64_t)n + 31) & ~uint64_t(31);
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_round; x += stride) {
        const bool valid = x < n;
        const uint32_t dx = valid ? deg[x] : 0;
        const uint32_t lx = valid ? L[x] : 0;
        const uint64_t b = valid ? rp[x] : 0;
        const uint64_t base = valid && dx ? off2[x] : 0;
        const uint32_t hx = valid && dx ? hcnt[x] : 0;
        if (dx <= kSmallRow) {
            uint32_t hp = 0, gp = 0;
            for (uint32_t j = 0; j < dx; ++j) {
                const uint32_t y = col[b + j];
                bool isg;
                if (is_h((uint32_t)x, dx, lx, y, ld, order, &isg)) adj2[base + hp++] = y;
                else if (isg) adj2[base + hx + gp++] = y;
            }
        }
        unsigned big = __ballot_sync(0xFFFFFFFFu, dx > kSmallRow);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t bx = (uint32_t)__shfl_sync(0xFFFFFFFFu, (unsigned long long)x, src);
            const uint32_t bd = __shfl_sync(0xFFFFFFFFu, dx, src);
            const uint32_t bl = __shfl_sync(0xFFFFFFFFu, lx, src);
            const uint64_t bb = __shfl_sync(0xFFFFFFFFu, b, src);
            const uint64_t bbase = __shfl_sync(0xFFFFFFFFu, base, src);
            const uint32_t bh = __shfl_sync(0xFFFFFFFFu, hx, src);
            uint32_t hp = 0, gp = 0;
            for (uint32_t j0 = 0; j0 < bd; j0 += 32) {
                const uint32_t j = j0 + lane;
                bool isH = false, isG = false;
                uint32_t y = 0;
                if (j < bd) {
                    y = col[bb + j];
                    isH = is_h(bx, bd, bl, y, ld, order, &isG);
                }
                const unsigned mh = __ballot_sync(0xFFFFFFFFu, isH);
                const unsigned mg = __ballot_sync(0xFFFFFFFFu, isG);
                if (isH) adj2[bbase + hp + __popc(mh & lt)] = y;
                if (isG) adj2[bbase + bh + gp + __popc(mg & lt)] = y;
                hp += __popc(mh);
                gp += __popc(mg);
            }
        }
    }
}

// Rows with at least one oriented horizontal edge are the hashed side of the
// intersections; split them by the size s(u) of their compacted row:
// class 3 (tiny) s <= tiny_cap and degree <= 4 tiny_cap, class 0 (warp)
// s <= warp_cap, class 1 (block) s <= block_cap, class 2 (hub).
// The lists are built by a stable scan, so they (and the task lists made from
// them) are in vertex order on every run: shards of a count agree on them.
__global__ void k_class_flags(uint32_t n, const uint32_t *__restrict__ hcnt, const uint32_t *__restrict__ scnt,
                              const uint32_t *__restrict__ deg, uint32_t *__restrict__ cls, Ctl *ctl,
                              uint32_t warp_cap, uint32_t block_cap, uint32_t tiny_cap) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned my_max = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        uint32_t c = 4;  // no oriented horizontal edge: nothing to intersect
        if (hcnt[x] > 0) {
            const uint32_t s = scnt[x];
            c = s <= warp_cap ? 0u : (s <= block_cap ? 1u : 2u);
            if (s <= tiny_cap && deg[x] <= 4 * tiny_cap) c = 3;
            if (c == 1 || c == 2) my_max = s > my_max ? s : my_max;
        }
        cls[x] = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned y = __shfl_xor_sync(0xFFFFFFFFu, my_max, o);
        my_max = y > my_max ? y : my_max;
    }
    if (lane_id() == 0 && my_max) atomicMax(&ctl->max_s2, my_max);
}

__global__ void k_class_indicator(uint32_t n, const uint32_t *__restrict__ cls, uint32_t c, uint32_t *__restrict__ ind) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) ind[x] = cls[x] == c;
}

__global__ void k_class_scatter(uint32_t n, const uint32_t *__restrict__ cls, uint32_t c,
                                const unsigned long long *__restrict__ pos, uint32_t *__restrict__ rows,
                                unsigned int *__restrict__ n_rows) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        if (cls[x] == c) rows[pos[x]] = (uint32_t)x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_rows = (unsigned int)pos[n];
}

// Split every hashed row u of class c into tasks (contiguous slices of H(u))
// of about `target` probes: work(u) = sum of s(v) over v in H(u),
// ntask = ceil(work(u) / max(task_work, min_mult * s(u))), at least
// ceil(|H(u)| / max_v) (shared-memory metadata of one task), at most |H(u)|.
__global__ void k_plan(const uint32_t *__restrict__ rows, const unsigned int *__restrict__ n_rows,
                       const uint64_t *__restrict__ off2, const uint32_t *__restrict__ adj2,
                       const uint32_t *__restrict__ hcnt, const uint32_t *__restrict__ scnt,
                       uint32_t *__restrict__ ntask, uint32_t task_work, uint32_t min_mult, uint32_t max_v) {
    const unsigned lane = lane_id();
    const uint32_t nr = *n_rows;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nr; i += warps) {
        const uint32_t u = rows[i];
        const uint64_t b = off2[u];
        const uint32_t hu = hcnt[u];
        unsigned long long work = 0;
        for (uint32_t k = lane; k < hu; k += 32) work += scnt[adj2[b + k]];
        work = warp_sum(work);
        if (lane == 0) {
            const unsigned long long su = scnt[u];
            const unsigned long long floor_t = (unsigned long long)min_mult * su;
            const unsigned long long target = floor_t > task_work ? floor_t : task_work;
            unsigned long long nt = (work + target - 1) / target;
            const unsigned long long by_v = (hu + max_v - 1) / max_v;
            if (nt < by_v) nt = by_v;
            if (nt < 1) nt = 1;
            if (nt > hu) nt = hu;
            ntask[i] = (uint32_t)nt;
        }
    }
}

__global__ void k_task_totals(Ctl *ctl, const unsigned long long *__restrict__ p0,
                              const unsigned long long *__restrict__ p1, const unsigned long long *__restrict__ p2) {
    ctl->n_tasks[0] = p0[ctl->n_rows[0]];
    ctl->n_tasks[1] = p1[ctl->n_rows[1]];
    ctl->n_tasks[2] = p2[ctl->n_rows[2]];
}

__global__ void k_emit(const uint32_t *__restrict__ ntask, const unsigned long long *__restrict__ tpref, uint32_t nr,
                       uint2 *__restrict__ tasks) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        const unsigned long long base = tpref[i];
        const uint32_t nt = ntask[i];
        for (uint32_t t = 0; t < nt; ++t) tasks[base + t] = make_uint2(i, t);
    }
}

unsigned grid_for(uint64_t work, unsigned threads, unsigned cap) {
    uint64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

tc_status build_rows(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint32_t max_deg) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    const uint32_t order = ctx->opt.order;
    const Tuning &tu = ctx->tune;
    if (n == 0) return TC_OK;
    // pack (level, degree) into one word when both fit (q0 is free after the levels)
    LevelDeg ld{b.L, b.deg, nullptr};
    uint32_t launches = 0;
    if (ctx->h_ctl->max_level < 255 && max_deg < (1u << 24)) {
        k_pack_level_deg<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.L, b.deg, b.q0);
        ld.packed = b.q0;
        ++launches;
    }
    k_row_count<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.rp, b.col, b.deg, b.L, ld, b.hcnt, b.scnt, ctx->d_ctl,
                                                      order);
    launches += 1 + scan_u32_to_u64(b.scnt, b.off2, n, b.scan_tmp, s);
    k_row_fill<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.rp, b.col, b.deg, b.L, ld, b.hcnt, b.off2, b.adj2, order);
    // fdeg and R are free after the levels: class of every vertex, 0/1 indicator
    k_class_flags<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.hcnt, b.scnt, b.deg, b.fdeg, ctx->d_ctl, tu.warp_cap,
                                                        tu.block_cap, tu.tiny_cap);
    launches += 2;
    for (uint32_t c = 0; c < 4; ++c) {
        k_class_indicator<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.fdeg, c, b.R);
        launches += 2 + scan_u32_to_u64(b.R, b.fpref, n, b.scan_tmp, s);
        k_class_scatter<<<grid_for(n, 256, cap), 256, 0, s>>>(
            n, b.fdeg, c, reinterpret_cast<const unsigned long long *>(b.fpref), b.rows[c], &ctx->d_ctl->n_rows[c]);
    }
    const uint32_t work[3] = {tu.warp_task_work, tu.task_work, tu.hub_task_work};
    const uint32_t mult[3] = {1, 2, 2};
    const uint32_t maxv[3] = {0xFFFFFFFFu, tu.max_v, tu.max_v};
    for (int c = 0; c < 3; ++c) {
        k_plan<<<grid_for((uint64_t)n * 32, 256, cap), 256, 0, s>>>(b.rows[c], &ctx->d_ctl->n_rows[c], b.off2, b.adj2,
                                                                    b.hcnt, b.scnt, b.ntask[c], work[c], mult[c],
                                                                    maxv[c]);
        ++launches;
    }
    note_launch(ctx, launches);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

// After the host has read n_rows: scan the task counts, publish the totals.
tc_status plan_scans(tc_ctx *ctx, const PipeBufs &b) {
    cudaStream_t s = ctx->stream;
    uint32_t launches = 1;
    for (int c = 0; c < 3; ++c)
        launches += scan_u32_to_u64(b.ntask[c], b.tpref[c], ctx->h_ctl->n_rows[c], b.scan_tmp, s);
    k_task_totals<<<1, 1, 0, s>>>(ctx->d_ctl, reinterpret_cast<const unsigned long long *>(b.tpref[0]),
                                  reinterpret_cast<const unsigned long long *>(b.tpref[1]),
                                  reinterpret_cast<const unsigned long long *>(b.tpref[2]));
    note_launch(ctx, launches);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

tc_status emit_tasks(tc_ctx *ctx, PipeBufs &b) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    uint64_t off = 0;
    for (int c = 0; c < 3; ++c) {
        b.tasks[c] = b.task_pool + off;
        off += ctx->h_ctl->n_tasks[c];
    }
    if (off > b.task_cap) return set_error(ctx, TC_ERR_OOM, "task list exceeds its bound");
    for (int c = 0; c < 3; ++c) {
        const uint32_t nr = ctx->h_ctl->n_rows[c];
        if (!nr) continue;
        k_emit<<<grid_for(nr, 256, cap), 256, 0, s>>>(b.ntask[c], reinterpret_cast<const unsigned long long *>(b.tpref[c]),
                                                     nr, b.tasks[c]);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
