// alg3.cu -- Algorithm 3 (cover-edge triangle counting) as a comparison
// kernel for Algorithm 4.
//
// Algorithm 3 walks the same horizontal edges as Algorithm 4 but intersects
// the FULL neighbourhoods: for every edge u -> v with L(u) == L(v) and u
// before v in the working order, every common neighbour w counts when it
// lies on another level, or on the same level and after v (Sec. III: a
// triangle with three horizontal edges is found from its first edge only, a
// triangle with one horizontal edge from that edge).  Same result and the
// same t_same / t_cross split as Algorithm 4, with more work per edge: the
// sets are all of N(u) and N(v) instead of the prefix sets of Algorithm 2
// and the level-spanning parts.  It reads the CSR as given (rows sorted by
// id) and the {rank, level} words of the count's rank stage; there is no
// row rewriting.
//
// One warp per 32 consecutive CSR slots (taken from a shared counter): every
// lane finds the row of its slot by binary search over row_ptr and tests its
// edge; the warp then takes the qualifying edges one by one, the lanes
// sharing the shorter row, each element looked up by binary search in the
// longer row.
#include "pipeline.cuh"

namespace tc {
namespace {

constexpr long long kAlg3WatchdogCycles = 20000000000ll;  // about 10 s of SM clock
constexpr unsigned kAlg3Watchdog = 0x80u;                 // same code as the intersection kernels' watchdog

// First index i in [lo, hi) with a[i] >= x (hi if none); a sorted ascending.
__device__ __forceinline__ uint64_t lower_bound_u32(const uint32_t *__restrict__ a, uint64_t lo, uint64_t hi,
                                                    uint32_t x) {
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_alg3(uint32_t n, const uint64_t *__restrict__ rp,
                                              const uint32_t *__restrict__ col, const uint2 *__restrict__ lv,
                                              uint64_t slots, Ctl *ctl) {
    const unsigned lane = lane_id();
    unsigned long long same = 0, cross = 0, probes = 0, e0 = 0;
    const long long t_start = clock64();
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) {
            c = atomicAdd(&ctl->task_next[0], 1u);
            if (clock64() - t_start > kAlg3WatchdogCycles) {
                atomicOr(&ctl->error, kAlg3Watchdog);
                c = ~0ull;
            }
        }
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        if (c == ~0ull || c * 32ull >= slots) break;
        const uint64_t j = c * 32ull + lane;
        bool q = false;
        uint32_t u = 0, v = 0;
        uint2 lu = make_uint2(0, 0), lw = make_uint2(0, 0);
        if (j < slots) {
            uint32_t a = 0, b = n;  // largest u with rp[u] <= j
            while (b - a > 1) {
                const uint32_t m = (a + b) >> 1;
                if (rp[m] <= j) a = m;
                else b = m;
            }
            u = a;
            v = col[j];
            lu = lv[u];
            lw = lv[v];
            q = lu.y == lw.y && lu.x < lw.x;  // horizontal, u before v
        }
        unsigned mask = __ballot_sync(0xFFFFFFFFu, q);
        e0 += lane == 0 ? (unsigned long long)__popc(mask) : 0ull;
        while (mask) {
            const int t = __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t ut = __shfl_sync(0xFFFFFFFFu, u, t);
            const uint32_t vt = __shfl_sync(0xFFFFFFFFu, v, t);
            const uint32_t level = __shfl_sync(0xFFFFFFFFu, lu.y, t);
            const uint32_t rank_v = __shfl_sync(0xFFFFFFFFu, lw.x, t);
            const uint64_t ub = rp[ut], ue = rp[ut + 1], vb = rp[vt], ve = rp[vt + 1];
            const bool u_short = ue - ub <= ve - vb;
            const uint64_t sb = u_short ? ub : vb, se = u_short ? ue : ve;
            const uint64_t lb = u_short ? vb : ub, le = u_short ? ve : ue;
            if (lane == 0) probes += (se - sb) + (le - lb);
            for (uint64_t i = sb + lane; i < se; i += 32) {
                const uint32_t x = __ldg(col + i);
                const uint64_t p = lower_bound_u32(col, lb, le, x);
                if (p < le && __ldg(col + p) == x) {
                    const uint2 l = lv[x];
                    if (l.y != level) ++cross;
                    else if (rank_v < l.x) ++same;
                }
            }
        }
    }
    same = warp_sum(same);
    cross = warp_sum(cross);
    probes = warp_sum(probes);
    e0 = warp_sum(e0);
    if (lane == 0) {
        if (same) atomicAdd(&ctl->t_same, same);
        if (cross) atomicAdd(&ctl->t_cross, cross);
        if (probes) {
            atomicAdd(&ctl->probes, probes);
            atomicAdd(&ctl->cls_probes[0], probes);
        }
        if (e0) atomicAdd(&ctl->e0, e0);
    }
}

}  // namespace

tc_status intersect_alg3(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots) {
    if (slots == 0 || n == 0) return TC_OK;
    cudaStream_t s = ctx->stream;
    int per_sm = 0;
    TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_alg3, 256, 0));
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
    const uint64_t need = (slots + 32 * 8 - 1) / (32 * 8);
    if (grid > need) grid = need;
    TC_CUDA(ctx, cudaMemsetAsync(ctx->d_ctl->task_next, 0, sizeof(ctx->d_ctl->task_next), s));
    k_alg3<<<(unsigned)grid, 256, 0, s>>>(n, b.rp, b.col, b.lv, slots, ctx->d_ctl);
    note_launch(ctx);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
