// csr.cu -- building, checking and measuring the input CSR on the device.
//
// tc_build_csr: tuples (a, b) -> 64-bit keys (a << 32 | b) and (b << 32 | a)
// for a != b -> stable LSD radix sort (8-bit digits, only the digits that
// can be nonzero) -> drop repeated keys -> col = low halves, row_ptr from the
// run boundaries of the high halves.  The result is the paper's input format:
// symmetric, loop-free, duplicate-free, rows ascending.
#include <algorithm>

#include "pipeline.cuh"

namespace tc {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr uint64_t kRsTile = (uint64_t)kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void k_make_keys(uint64_t t, const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst, uint32_t n,
                            unsigned long long *__restrict__ keys, Ctl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t_round = (t + 31) & ~uint64_t(31);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < t_round; i += stride) {
        uint32_t a = 0, b = 0;
        bool keep = false;
        if (i < t) {
            a = src[i];
            b = dst[i];
            if (a >= n || b >= n) ctl->error = 1;
            else keep = a != b;
        }
        // two keys per kept tuple: count them in pairs
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
        uint64_t base = 0;
        if (mask) {
            const unsigned leader = __ffs(mask) - 1;
            if (lane_id() == leader) base = (uint64_t)atomicAdd(&ctl->visited_edges, 2ull * __popc(mask));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
        }
        if (keep) {
            const uint64_t slot = base + 2u * __popc(mask & ((1u << lane_id()) - 1u));
            keys[slot] = ((unsigned long long)a << 32) | b;
            keys[slot + 1] = ((unsigned long long)b << 32) | a;
        }
    }
}

// Per-tile digit histograms, digit-major: counts[d * nblocks + block].
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const unsigned long long *__restrict__ keys, uint64_t count,
                                                        int shift, uint32_t *__restrict__ counts, uint32_t nblocks) {
    __shared__ uint32_t h[kRsWarps][256];
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const unsigned warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int i = 0; i < kRsItems; ++i) {
        const uint64_t j = base + (uint64_t)i * kRsThreads + threadIdx.x;
        if (j < count) atomicAdd(&h[warp][(keys[j] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kRsThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) s += h[w][d];
        counts[(uint64_t)d * nblocks + blockIdx.x] = s;
    }
}

// Stable scatter: keys of a tile are taken round by round (round i holds
// entries base + i*256 + t), so input order is (round, thread).  A key's rank
// among equal digits = keys of that digit in earlier rounds + in earlier
// warps of this round + in earlier lanes of its warp.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const unsigned long long *__restrict__ in,
                                                           unsigned long long *__restrict__ out, uint64_t count,
                                                           int shift, const unsigned long long *__restrict__ offs,
                                                           uint32_t nblocks) {
    __shared__ uint32_t running[256];
    __shared__ uint32_t wc[kRsWarps][256];
    __shared__ unsigned long long start[256];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += kRsThreads) {
        running[d] = 0;
        start[d] = offs[(uint64_t)d * nblocks + blockIdx.x];
    }
    const uint64_t base = (uint64_t)blockIdx.x * kRsTile;
    for (int i = 0; i < kRsItems; ++i) {
        for (int k = threadIdx.x; k < kRsWarps * 256; k += kRsThreads) (&wc[0][0])[k] = 0;
        __syncthreads();
        const uint64_t j = base + (uint64_t)i * kRsThreads + threadIdx.x;
        const bool valid = j < count;
        unsigned long long key = valid ? in[j] : 0ull;
        const uint32_t d = valid ? (uint32_t)((key >> shift) & 0xFF) : 256u + lane;  // invalid lanes: unique tags
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t in_warp = __popc(peers & ((1u << lane) - 1u));
        if (valid && in_warp == 0) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t before = running[d] + in_warp;
            for (unsigned w = 0; w < warp; ++w) before += wc[w][d];
            out[start[d] + before] = key;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < 256; dd += kRsThreads) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) s += wc[w][dd];
            running[dd] += s;
        }
        __syncthreads();
    }
}

__global__ void k_unique_flags(const unsigned long long *__restrict__ keys, uint64_t count, uint32_t *__restrict__ flag) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_compact(const unsigned long long *__restrict__ keys, uint64_t count,
                          const uint32_t *__restrict__ flag, const unsigned long long *__restrict__ pos,
                          uint32_t *__restrict__ col, uint32_t *__restrict__ src32) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        if (!flag[i]) continue;
        const unsigned long long k = keys[i];
        col[pos[i]] = (uint32_t)k;
        src32[pos[i]] = (uint32_t)(k >> 32);
    }
}

// row_ptr[v] = first position p with src32[p] >= v (U = number of slots).
__global__ void k_rowptr(const uint32_t *__restrict__ src32, uint64_t U, uint32_t n, uint64_t *__restrict__ rp) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= U; p += stride) {
        const uint64_t lo = p == 0 ? 0 : (uint64_t)src32[p - 1] + 1;   // first v whose start is p
        const uint64_t hi = p == U ? (uint64_t)n : (uint64_t)src32[p];  // last such v
        if (p == 0) {
            for (uint64_t v = 0; v <= hi && v <= n; ++v) rp[v] = 0;
        } else {
            for (uint64_t v = lo; v <= hi && v <= n; ++v) rp[v] = p;
        }
    }
}

__global__ void k_empty_rowptr(uint32_t n, uint64_t *__restrict__ rp) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) rp[v] = 0;
}

// Well-formedness: monotone row_ptr ending at `slots`, ids < n, rows strictly
// ascending (no repeats), no self-loops, and every (v, w) has its (w, v).
__global__ void k_validate(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                           uint64_t slots, Ctl *ctl) {
    const unsigned lane = lane_id();
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint64_t b = rp[v], e = rp[v + 1];
        if (e < b || e > slots || (v == 0 && b != 0) || (v + 1 == n && e != slots)) {
            if (lane == 0) ctl->error = 1;
            continue;
        }
        for (uint64_t j = b + lane; j < e; j += 32) {
            const uint32_t w = col[j];
            bool bad = w >= n || w == v || (j > b && col[j - 1] >= w);
            if (!bad) {
                uint64_t lo = rp[w], hi = rp[w + 1];
                if (hi > slots || lo > hi) {  // w's own row is malformed: never read outside col
                    ctl->error = 1;
                    continue;
                }
                bool found = false;
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    const uint32_t x = col[mid];
                    if (x == v) { found = true; break; }
                    if (x < v) lo = mid + 1; else hi = mid;
                }
                bad = !found;
            }
            if (bad) ctl->error = 1;
        }
    }
}

__global__ void k_max_deg(uint32_t n, const uint64_t *__restrict__ rp, Ctl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned m = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint64_t d = rp[v + 1] - rp[v];
        const unsigned dd = d > 0xFFFFFFFFull ? 0xFFFFFFFFu : (unsigned)d;
        m = dd > m ? dd : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
        m = y > m ? y : m;
    }
    if (lane_id() == 0 && m) atomicMax(&ctl->max_s2, m);
}

__global__ void k_ctl_zero(Ctl *ctl) {
    unsigned int *w = reinterpret_cast<unsigned int *>(ctl);
    for (unsigned i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) w[i] = 0;
}

unsigned grid_for(uint64_t work, unsigned threads, unsigned cap) {
    uint64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

tc_status pull(tc_ctx *ctx) {
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TC_OK;
}

}  // namespace

uint64_t radix_tiles(uint64_t count) { return (count + kRsTile - 1) / kRsTile; }

uint32_t radix_sort_u64(unsigned long long **cur, unsigned long long **alt, uint64_t count, const int *shifts,
                        int nshifts, uint32_t *counts, uint64_t *coffs, uint64_t *tmp, cudaStream_t s) {
    if (count < 2) return 0;
    const uint32_t nblk = (uint32_t)radix_tiles(count);
    uint32_t launches = 0;
    for (int i = 0; i < nshifts; ++i) {
        k_rs_hist<<<nblk, kRsThreads, 0, s>>>(*cur, count, shifts[i], counts, nblk);
        launches += 2 + scan_u32_to_u64(counts, coffs, 256ull * nblk, tmp, s);
        k_rs_scatter<<<nblk, kRsThreads, 0, s>>>(*cur, *alt, count, shifts[i],
                                                 reinterpret_cast<const unsigned long long *>(coffs), nblk);
        std::swap(*cur, *alt);
    }
    return launches;
}

tc_status build_csr_device(tc_ctx *ctx, uint32_t n, uint64_t t, const uint32_t *d_src, const uint32_t *d_dst,
                           uint64_t **rp_out, uint32_t **col_out, uint64_t *slots_out, bool *pooled_out) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    const uint64_t K = 2 * t;  // upper bound on keys
    const uint64_t nblk_max = (K + kRsTile - 1) / kRsTile;
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = 2 * r(8 * (K + 1)) + r(4 * (K + 1)) + r(8 * (K + 2)) + r(4 * (K + 1)) +
                        r(4 * (256 * nblk_max + 1)) + r(8 * (256 * nblk_max + 2)) +
                        r(8 * scan_tmp_elems(std::max<uint64_t>(K, 256 * nblk_max) + 2)) + 4096;
    tc_status st = arena_reserve(ctx, need);
    if (st != TC_OK) return st;
    Arena &a = ctx->arena;
    a.reset();
    auto *k0 = a.take<unsigned long long>(K + 1);
    auto *k1 = a.take<unsigned long long>(K + 1);
    auto *flag = a.take<uint32_t>(K + 1);
    auto *pos = a.take<uint64_t>(K + 2);
    auto *src32 = a.take<uint32_t>(K + 1);
    auto *counts = a.take<uint32_t>(256 * nblk_max + 1);
    auto *coffs = a.take<uint64_t>(256 * nblk_max + 2);
    auto *tmp = a.take<uint64_t>(scan_tmp_elems(std::max<uint64_t>(K, 256 * nblk_max) + 2));
    if (!k0 || !k1 || !flag || !pos || !src32 || !counts || !coffs || !tmp)
        return set_error(ctx, TC_ERR_OOM, "arena carve failed (build_csr)");

    k_ctl_zero<<<1, 128, 0, s>>>(ctx->d_ctl);
    if (t) k_make_keys<<<grid_for(t, 256, cap), 256, 0, s>>>(t, d_src, d_dst, n, k0, ctx->d_ctl);
    TC_CUDA(ctx, cudaGetLastError());
    st = pull(ctx);
    if (st != TC_OK) return st;
    if (ctx->h_ctl->error) return set_error(ctx, TC_ERR_INVALID, "tc_build_csr: a tuple names a vertex id >= n");
    const uint64_t nk = ctx->h_ctl->visited_edges;  // keys written (2 per kept tuple)

    // significant bits of an id: the radix passes cover [0, B) and [32, 32 + B)
    int B = 0;
    while (B < 32 && (1ull << B) < n) ++B;
    std::vector<int> shifts;
    for (int sh = 0; sh < B; sh += 8) shifts.push_back(sh);
    for (int sh = 0; sh < B; sh += 8) shifts.push_back(32 + sh);
    unsigned long long *cur = k0, *alt = k1;
    radix_sort_u64(&cur, &alt, nk, shifts.data(), (int)shifts.size(), counts, coffs, tmp, s);
    uint64_t *rp = nullptr;
    uint32_t *col = nullptr;
    uint64_t U = 0;
    if (nk) {
        k_unique_flags<<<grid_for(nk, 256, cap), 256, 0, s>>>(cur, nk, flag);
        scan_u32_to_u64(flag, pos, nk, tmp, s);
        TC_CUDA(ctx, cudaMemcpyAsync(&U, pos + nk, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        TC_CUDA(ctx, cudaStreamSynchronize(s));
    }
    bool pooled = false, pooled2 = false;
    if (graph_alloc(ctx, (void **)&rp, sizeof(uint64_t) * ((size_t)n + 1), &pooled) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, TC_ERR_OOM, "tc_build_csr: row_ptr allocation failed");
    }
    if (graph_alloc(ctx, (void **)&col, sizeof(uint32_t) * (size_t)(U + 1), &pooled2) != cudaSuccess) {
        cudaGetLastError();
        graph_free(ctx, rp, pooled);
        return set_error(ctx, TC_ERR_OOM, "tc_build_csr: col allocation failed");
    }
    *pooled_out = pooled;
    if (U) {
        k_compact<<<grid_for(nk, 256, cap), 256, 0, s>>>(cur, nk, flag, reinterpret_cast<const unsigned long long *>(pos),
                                                        col, src32);
        k_rowptr<<<grid_for(U + 1, 256, cap), 256, 0, s>>>(src32, U, n, rp);
    } else {
        k_empty_rowptr<<<grid_for((uint64_t)n + 1, 256, cap), 256, 0, s>>>(n, rp);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        graph_free(ctx, rp, pooled);
        graph_free(ctx, col, pooled2);
        return cuda_error(ctx, e, "tc_build_csr kernels");
    }
    *rp_out = rp;
    *col_out = col;
    *slots_out = U;
    return TC_OK;
}

tc_status validate_csr_device(tc_ctx *ctx, uint32_t n, const uint64_t *rp, const uint32_t *col, uint64_t slots,
                              int *ok) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    k_ctl_zero<<<1, 128, 0, s>>>(ctx->d_ctl);
    if (n) k_validate<<<grid_for((uint64_t)n * 32, 256, cap), 256, 0, s>>>(n, rp, col, slots, ctx->d_ctl);
    TC_CUDA(ctx, cudaGetLastError());
    tc_status st = pull(ctx);
    if (st != TC_OK) return st;
    *ok = ctx->h_ctl->error == 0 && (n > 0 || slots == 0);
    return TC_OK;
}

tc_status max_degree_device(tc_ctx *ctx, uint32_t n, const uint64_t *rp, uint32_t *max_deg) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    k_ctl_zero<<<1, 128, 0, s>>>(ctx->d_ctl);
    if (n) k_max_deg<<<grid_for(n, 256, cap), 256, 0, s>>>(n, rp, ctx->d_ctl);
    TC_CUDA(ctx, cudaGetLastError());
    tc_status st = pull(ctx);
    if (st != TC_OK) return st;
    *max_deg = ctx->h_ctl->max_s2;
    return TC_OK;
}

}  // namespace tc
