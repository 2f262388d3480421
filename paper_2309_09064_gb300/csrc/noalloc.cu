// noalloc.cu -- tc_count_noalloc: an exact count that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// count: code running inside another allocator's callback, a memory pool that
// has already handed out the whole device, or an environment that forbids
// cudaMalloc after start-up.  For them this entry point runs the same method
// as tc_count (BFS levels from each component's first vertex in the working
// order, E0/E1 partition, degree orientation, hashed intersections) in ONE
// thread block, with all scratch in a fixed array in device global memory that
// is declared at file scope below.  The caller passes the inputs and the
// output; the library calls no cudaMalloc, cudaFree or other allocating
// routine on this path.
//
// Limits: n <= kMaxN vertices and row_ptr[n] <= kMaxSlots CSR slots.  The
// array (about 5.8 MB) belongs to every GPU that loads the library until the
// process exits.  All calls share it, so calls that overlap on the GPU (two
// streams, two threads) race and give wrong results; serialise them.  The
// array keeps the last call's contents; the kernel itself resets everything
// it reads before use.
//
// Set-up: the first call on a device looks up the device address of the
// array (cudaGetSymbolAddress, with that device current) and caches it; make
// that first call outside any stream capture.
#include <mutex>

#include "pipeline.cuh"

namespace tc {
namespace {

constexpr uint32_t kMaxN = 65536;
constexpr uint64_t kMaxSlots = 1u << 20;
constexpr int kThreads = 512;                    // 16 warps
constexpr uint32_t kBitmapWords = kMaxN / 32;    // one n-bit set per warp in shared memory

struct NoAllocScratch {
    uint32_t deg[kMaxN];
    uint32_t L[kMaxN];
    uint32_t q[2][kMaxN];
    uint32_t hcnt[kMaxN];
    uint32_t off[kMaxN + 1];
    uint32_t adj2[kMaxSlots];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long v, unsigned long long *red) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = y < v ? y : v;
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long m = ~0ull;
    for (unsigned w = 0; w < (blockDim.x >> 5); ++w) m = red[w] < m ? red[w] : m;
    return m;
}

// Whole count in one block.  out[0] = T, out[1] = triangles inside G0,
// out[2] = cross-level triangles, out[3] = nonzero if the input exceeded the
// limits (then nothing else was written).
__global__ void __launch_bounds__(kThreads, 1) k_count_noalloc(NoAllocScratch *S, const uint64_t *__restrict__ rp,
                                                               const uint32_t *__restrict__ col, uint32_t n,
                                                               uint32_t order, unsigned long long *out) {
    extern __shared__ uint32_t bitmaps[];  // 16 warps x kBitmapWords
    __shared__ unsigned long long red[32];
    __shared__ unsigned int s_cnt[2];
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (n > kMaxN || rp[n] > kMaxSlots) {
        if (tid == 0) {
            out[0] = out[1] = out[2] = 0;
            out[3] = 1;
        }
        return;
    }
    // degrees; isolated vertices are their own roots at level 0
    for (uint32_t v = tid; v < n; v += blockDim.x) {
        const uint32_t d = (uint32_t)(rp[v + 1] - rp[v]);
        S->deg[v] = d;
        S->L[v] = d ? kUnvisited : 0u;
    }
    __syncthreads();
    // BFS from the first unvisited vertex in the working order, until none is left
    for (;;) {
        unsigned long long best = ~0ull;
        for (uint32_t v = tid; v < n; v += blockDim.x)
            if (S->L[v] == kUnvisited) {
                const unsigned long long k = order_key(v, S->deg[v], order);
                best = k < best ? k : best;
            }
        best = block_min_u64(best, red);
        if (best == ~0ull) break;
        const uint32_t root = (uint32_t)(best & 0xFFFFFFFFull);
        if (tid == 0) {
            S->L[root] = 0;
            S->q[0][0] = root;
            s_cnt[0] = 1;
        }
        __syncthreads();
        uint32_t cur = 0, level = 0;
        for (;;) {
            const uint32_t fcount = s_cnt[cur];
            if (fcount == 0) break;
            if (tid == 0) s_cnt[cur ^ 1] = 0;
            __syncthreads();
            for (uint32_t i = warp; i < fcount; i += nwarps) {
                const uint32_t v = S->q[cur][i];
                for (uint64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) {
                    const uint32_t w = col[j];
                    if (S->L[w] == kUnvisited && atomicCAS(&S->L[w], kUnvisited, level + 1) == kUnvisited)
                        S->q[cur ^ 1][atomicAdd(&s_cnt[cur ^ 1], 1u)] = w;
                }
            }
            __syncthreads();
            cur ^= 1;
            ++level;
        }
        __syncthreads();
    }
    // rows [H(x) | G1(x)]: counts, exclusive scan, fill (warp per vertex, ballot order)
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t x = warp; x < n; x += nwarps) {
        const uint32_t dx = S->deg[x], lx = S->L[x];
        uint32_t h = 0, g = 0;
        for (uint64_t j = rp[x] + lane; j < rp[x + 1]; j += 32) {
            const uint32_t y = col[j];
            if (S->L[y] != lx) ++g;
            else if (precedes(x, dx, y, S->deg[y], order)) ++h;
        }
        h = warp_sum(h);
        g = warp_sum(g);
        if (lane == 0) {
            S->hcnt[x] = h;
            S->off[x] = h + g;
        }
    }
    __syncthreads();
    if (tid == 0) {  // serial scan: n <= 65536, once per call
        uint32_t run = 0;
        for (uint32_t x = 0; x < n; ++x) {
            const uint32_t c = S->off[x];
            S->off[x] = run;
            run += c;
        }
        S->off[n] = run;
    }
    __syncthreads();
    for (uint32_t x = warp; x < n; x += nwarps) {
        const uint32_t dx = S->deg[x], lx = S->L[x];
        const uint32_t base = S->off[x], hx = S->hcnt[x];
        uint32_t hp = 0, gp = 0;
        for (uint64_t j0 = rp[x]; j0 < rp[x + 1]; j0 += 32) {
            const uint64_t j = j0 + lane;
            bool isH = false, isG = false;
            uint32_t y = 0;
            if (j < rp[x + 1]) {
                y = col[j];
                if (S->L[y] != lx) isG = true;
                else isH = precedes(x, dx, y, S->deg[y], order);
            }
            const unsigned mh = __ballot_sync(0xFFFFFFFFu, isH), mg = __ballot_sync(0xFFFFFFFFu, isG);
            if (isH) S->adj2[base + hp + __popc(mh & lt)] = y;
            if (isG) S->adj2[base + hx + gp + __popc(mg & lt)] = y;
            hp += __popc(mh);
            gp += __popc(mg);
        }
    }
    // intersections: each warp owns an n-bit set in shared memory
    uint32_t *bm = bitmaps + (size_t)warp * kBitmapWords;
    for (uint32_t j = lane; j < kBitmapWords; j += 32) bm[j] = 0u;
    __syncthreads();
    unsigned long long same = 0, cross = 0;
    for (uint32_t u = warp; u < n; u += nwarps) {
        const uint32_t hu = S->hcnt[u];
        if (hu == 0) continue;
        const uint32_t ub = S->off[u], ue = S->off[u + 1];
        for (uint32_t j = ub + lane; j < ue; j += 32) atomicOr(bm + (S->adj2[j] >> 5), 1u << (S->adj2[j] & 31));
        __syncwarp();
        for (uint32_t k = 0; k < hu; ++k) {
            const uint32_t v = S->adj2[ub + k];
            const uint32_t vb = S->off[v], ve = S->off[v + 1], hv = S->hcnt[v];
            for (uint32_t j = vb + lane; j < ve; j += 32) {
                const uint32_t w = S->adj2[j];
                if ((bm[w >> 5] >> (w & 31)) & 1u) {
                    if (j - vb < hv) ++same; else ++cross;
                }
            }
        }
        __syncwarp();
        for (uint32_t j = ub + lane; j < ue; j += 32) bm[S->adj2[j] >> 5] = 0u;
        __syncwarp();
    }
    same = warp_sum(same);
    cross = warp_sum(cross);
    __syncthreads();
    if (lane == 0) {
        red[warp] = same;
        red[16 + warp] = cross;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long s = 0, c = 0;
        for (unsigned w = 0; w < nwarps; ++w) {
            s += red[w];
            c += red[16 + w];
        }
        out[0] = s + c;
        out[1] = s;
        out[2] = c;
        out[3] = 0;
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};
bool g_smem_set[kMaxDevices] = {};

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_count_noalloc(const uint64_t *d_row_ptr, const uint32_t *d_col, uint32_t n, uint64_t slots,
                                      uint32_t order, uint64_t *d_out, void *stream) {
    if (!d_row_ptr || !d_out || (slots && !d_col)) return TC_ERR_INVALID;
    if (n > kMaxN || slots > kMaxSlots) return TC_ERR_INVALID;  // beyond the fixed scratch array
    if (order != TC_ORDER_DEGREE && order != TC_ORDER_ID) return TC_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TC_ERR_CUDA;
    NoAllocScratch *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return TC_ERR_CUDA;
            }
            g_scratch_ptr[dev] = static_cast<NoAllocScratch *>(p);
        }
        if (!g_smem_set[dev]) {
            if (cudaFuncSetAttribute(k_count_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(16 * kBitmapWords * sizeof(uint32_t))) != cudaSuccess) {
                cudaGetLastError();
                return TC_ERR_CUDA;
            }
            g_smem_set[dev] = true;
        }
        S = g_scratch_ptr[dev];
    }
    k_count_noalloc<<<1, kThreads, 16 * kBitmapWords * sizeof(uint32_t), (cudaStream_t)stream>>>(
        S, d_row_ptr, d_col, n, order, reinterpret_cast<unsigned long long *>(d_out));
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
