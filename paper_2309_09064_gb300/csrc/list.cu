// list.cu -- compaction of a one-pass triangle listing (tc_list_triangles).
//
// The warp, block and hub classes write their triangles into chunks of
// kListChunk positions, each warp filling one chunk at a time from a global
// cursor (isect.cu).  Every chunk is full except the ones still open when the
// pass ends (at most one per warp state).  With t_big triangles written this
// way, positions [0, t_big) must end up holding all of them: the gaps below
// t_big (the unfilled tails of open chunks) are exactly as many as the
// triangles written at or past t_big, and the k-th such triangle moves into
// the k-th gap.  Sources and destinations never overlap, so one parallel
// copy does it.
#include "pipeline.cuh"

namespace tc {
namespace {

constexpr unsigned kGuardCompact = 0x800u;  // a compaction index fell outside the triple buffers

__device__ __forceinline__ uint32_t *triple_ptr(uint32_t *out, unsigned long long cap, uint32_t *ovf,
                                                unsigned long long ovf_cap, unsigned long long p) {
    if (p < cap) return out + 3 * p;
    p -= cap;
    return p < ovf_cap ? ovf + 3 * p : nullptr;
}

// Record the fill of every chunk still open: a state {next position, room}
// with room > 0 is the chunk ending at next + room.
__global__ void k_list_close(const ulonglong2 *__restrict__ wstate, unsigned long long len, uint32_t *fills,
                             unsigned long long nch, Ctl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const ulonglong2 st = wstate[i];
        if (st.y == 0) continue;
        const unsigned long long id = (st.x + st.y) / kListChunk - 1;
        if (id < nch) fills[id] = kListChunk - (uint32_t)st.y;
        else atomicOr(&ctl->error, kGuardCompact);
    }
}

// Chunk c covers [c K, (c+1) K) (K = kListChunk) and holds triangles in
// [c K, c K + fill).  holes[c] = its unfilled positions below t_big,
// src[c] = its triangles at or past t_big.
__global__ void k_list_gaps(const uint32_t *__restrict__ fills, unsigned long long nchunks,
                            unsigned long long t_big, unsigned long long *holes, unsigned long long *src) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += stride) {
        const unsigned long long start = c * kListChunk, filled = start + fills[c];
        const unsigned long long hi = start + kListChunk < t_big ? start + kListChunk : t_big;
        const unsigned long long lo = start > t_big ? start : t_big;
        holes[c] = hi > filled ? hi - filled : 0;
        src[c] = filled > lo ? filled - lo : 0;
    }
}

// One warp per chunk with triangles at or past t_big: source k (global
// index by the scan sp) goes to gap k, found by binary search of the gaps'
// scan hp (largest chunk c' with hp[c'] <= k).
__global__ void k_list_move(const unsigned long long *__restrict__ hp, const unsigned long long *__restrict__ sp,
                            const uint32_t *__restrict__ fills, unsigned long long nchunks, unsigned long long t_big,
                            uint32_t *out, unsigned long long cap, uint32_t *ovf, unsigned long long ovf_cap,
                            Ctl *ctl) {
    const unsigned lane = lane_id();
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
        const unsigned long long s0 = sp[c], ns = sp[c + 1] - s0;
        if (ns == 0) continue;
        const unsigned long long first = c * kListChunk > t_big ? c * kListChunk : t_big;
        for (unsigned long long j = lane; j < ns; j += 32) {
            const unsigned long long k = s0 + j;
            unsigned long long a = 0, b = nchunks;  // hp[a] <= k < hp[b]
            while (b - a > 1) {
                const unsigned long long m = (a + b) >> 1;
                if (hp[m] <= k) a = m;
                else b = m;
            }
            const unsigned long long dst = a * kListChunk + fills[a] + (k - hp[a]);
            uint32_t *d = triple_ptr(out, cap, ovf, ovf_cap, dst);
            const uint32_t *q = triple_ptr(out, cap, ovf, ovf_cap, first + j);
            if (!d || !q || dst >= t_big) {
                atomicOr(&ctl->error, kGuardCompact);
                continue;
            }
            d[0] = q[0];
            d[1] = q[1];
            d[2] = q[2];
        }
    }
}

unsigned blocks_for(uint64_t work, unsigned threads, unsigned cap) {
    uint64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace

size_t list_compact_scratch(unsigned long long nch) { return 2 * ((size_t)nch + 1); }

tc_status list_compact(tc_ctx *ctx, const PipeBufs &b, unsigned long long t_big, unsigned long long g_end,
                       unsigned long long *scratch, unsigned long long *scan_tmp) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    if (g_end % kListChunk) return set_error(ctx, TC_ERR_INVALID, "listing: chunk cursor not on a chunk boundary");
    const unsigned long long nchunks = g_end / kListChunk;
    if (nchunks > b.nch) return set_error(ctx, TC_ERR_INVALID, "listing: more chunks than the chunk table holds");
    k_list_close<<<blocks_for(b.wstate_len, 256, cap), 256, 0, s>>>(b.wstate, b.wstate_len, b.fills, b.nch,
                                                                    ctx->d_ctl);
    note_launch(ctx);
    if (nchunks == 0) {
        TC_CUDA(ctx, cudaGetLastError());
        return TC_OK;
    }
    unsigned long long *holes = scratch, *src = scratch + (b.nch + 1);
    k_list_gaps<<<blocks_for(nchunks, 256, cap), 256, 0, s>>>(b.fills, nchunks, t_big, holes, src);
    note_launch(ctx);
    note_launch(ctx, scan_u64(reinterpret_cast<uint64_t *>(holes), reinterpret_cast<uint64_t *>(holes), nchunks,
                              reinterpret_cast<uint64_t *>(scan_tmp), s));
    note_launch(ctx, scan_u64(reinterpret_cast<uint64_t *>(src), reinterpret_cast<uint64_t *>(src), nchunks,
                              reinterpret_cast<uint64_t *>(scan_tmp), s));
    unsigned long long tot[2] = {0, 0};
    TC_CUDA(ctx, cudaMemcpyAsync(&tot[0], holes + nchunks, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(ctx, cudaMemcpyAsync(&tot[1], src + nchunks, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(ctx, cudaStreamSynchronize(s));
    if (tot[0] != tot[1]) return set_error(ctx, TC_ERR_INVALID, "listing: written triangles disagree with the count");
    if (tot[0]) {
        k_list_move<<<blocks_for(32 * nchunks, 256, cap), 256, 0, s>>>(holes, src, b.fills, nchunks, t_big,
                                                                      b.list_out, b.list_cap, b.ovf, b.ovf_cap,
                                                                      ctx->d_ctl);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
