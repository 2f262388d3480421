// rank.cu -- position of every vertex in the working order (Sec. II, last
// paragraph: vertices re-ordered by decreasing degree).
//
// The intersections compare and hash vertices by their rank, the position in
// the working order: under the degree order (BaderD) vertices sorted by
// decreasing degree, ties by ascending id; under the id order (Bader) the id
// itself.  Using ranks as the stored values is the relabelling the paper
// charges as preprocessing, applied to the rows the intersections read; the
// CSR input is never rewritten.
//
// The degree order is one stable LSD radix sort of 64-bit keys
// (max_deg - deg(x)) << 32 | x over the digits of the high half only: the keys
// start in id order and every pass is stable, so equal degrees stay in id
// order.  Then rank[x] = position of x's key.
#include "pipeline.cuh"

namespace tc {
namespace {

__global__ void k_rank_keys(uint32_t n, const uint32_t *__restrict__ deg, uint32_t max_deg,
                            unsigned long long *__restrict__ keys) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        keys[x] = ((unsigned long long)(max_deg - deg[x]) << 32) | x;
}

// rank[x] = position of x's key; inv (nullable) gets the inverse, the id at
// every position (the listing maps ranks found by the intersections back).
__global__ void k_rank_scatter(uint32_t n, const unsigned long long *__restrict__ keys, uint32_t *__restrict__ rank,
                               uint32_t *__restrict__ inv) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t x = (uint32_t)(keys[i] & 0xFFFFFFFFull);
        rank[x] = (uint32_t)i;
        if (inv) inv[i] = x;
    }
}

// lv[x] = {rank(x), L(x)}: one 8-byte read gives both for a neighbour; and,
// when n <= 2^24 and every level is below 255, lvp[x] = rank(x) << 8 | L(x):
// one 4-byte read (half the bytes, so the array stays in L2 for longer).
__global__ void k_pack_rank_level(uint32_t n, const uint32_t *__restrict__ rank, const uint32_t *__restrict__ L,
                                  uint2 *__restrict__ lv, uint32_t *__restrict__ lvp) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const uint32_t r = rank ? rank[x] : (uint32_t)x, l = L[x];
        lv[x] = make_uint2(r, l);
        if (lvp) lvp[x] = (r << 8) | l;
    }
}

unsigned grid_for(uint64_t work, unsigned threads, unsigned cap) {
    uint64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

tc_status compute_ranks(tc_ctx *ctx, PipeBufs &b, uint32_t n, uint32_t max_deg) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    if (n == 0) return TC_OK;
    uint32_t launches = 0;
    const uint32_t *rank = nullptr;
    if (ctx->opt.order == TC_ORDER_DEGREE && max_deg > 0) {
        k_rank_keys<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.deg, max_deg, b.rkeys0);
        int shifts[4], ns = 0;
        for (int sh = 0; sh < 32 && (max_deg >> sh) != 0; sh += 8) shifts[ns++] = 32 + sh;
        unsigned long long *cur = b.rkeys0, *alt = b.rkeys1;
        launches += 1 + radix_sort_u64(&cur, &alt, n, shifts, ns, b.rcounts, b.roffs, b.scan_tmp, s);
        k_rank_scatter<<<grid_for(n, 256, cap), 256, 0, s>>>(n, cur, b.rank, b.inv);
        ++launches;
        rank = b.rank;
        b.order = cur;
    }
    k_pack_rank_level<<<grid_for(n, 256, cap), 256, 0, s>>>(n, rank, b.L, b.lv, b.lvp);
    note_launch(ctx, launches + 1);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
