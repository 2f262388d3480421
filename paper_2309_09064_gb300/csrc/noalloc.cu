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
// array (about 5.8 MB) lives in this file's device code.  The CUDA driver
// loads device code lazily by default, so the array is allocated on a device
// when the first call on that device looks up its address (or, with eager
// module loading, when the library is loaded); from then on it stays until
// the process exits.  All calls share it, so calls that overlap on the GPU
// (two streams, two threads) race and give wrong results; serialise them.
// The array keeps the last call's contents; the kernel itself resets
// everything it reads before use.
//
// Set-up: the first call on a device looks up the device address of the
// array (cudaGetSymbolAddress, with that device current), which loads the
// device code and allocates the array, and caches it; make that first call
// at start-up (a call with n = 0 is enough) and outside any stream capture.
//
// Roots: each component's root is its first vertex in the working order,
// found for all components at once -- components by union-find (hooking the
// larger root index under the smaller), then the smallest order key of each
// component by an atomic minimum -- and one BFS runs from all roots
// together.  The cost is O(n + m) work and one barrier per BFS level of the
// deepest component, however many components there are.
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

// 32-bit working-order key for n <= 65536 (degrees < 65536): smaller key =
// earlier vertex.  Degree order: decreasing degree, ties by ascending id.
__device__ __forceinline__ uint32_t key32(uint32_t v, uint32_t d, uint32_t order) {
    return order == TC_ORDER_DEGREE ? ((0xFFFFu - d) << 16) | v : v;
}

__device__ __forceinline__ uint32_t vload(const uint32_t *p) { return *(const volatile uint32_t *)p; }

// Root of x's tree in the union-find forest par (par[v] <= v, roots point to
// themselves), halving the path on the way.  Every step moves to a smaller
// index, so the walk ends within n steps.
__device__ __forceinline__ uint32_t uf_find(uint32_t *par, uint32_t x) {
    uint32_t p = vload(par + x);
    while (p != x) {
        const uint32_t gp = vload(par + p);
        if (gp != p) *(volatile uint32_t *)(par + x) = gp;
        x = p;
        p = gp;
    }
    return x;
}

// Join the trees of x and y: the larger root is hooked under the smaller
// one by compare-and-swap.  A failed swap means that root was just hooked
// by another thread, which can happen at most n - 1 times in all, so the
// loop is bounded by n retries; past it *bad is set (never expected).
__device__ __forceinline__ void uf_union(uint32_t *par, uint32_t x, uint32_t y, uint32_t n, unsigned int *bad) {
    for (uint32_t it = 0; it <= n; ++it) {
        const uint32_t rx = uf_find(par, x), ry = uf_find(par, y);
        if (rx == ry) return;
        const uint32_t hi = rx > ry ? rx : ry, lo = rx > ry ? ry : rx;
        if (atomicCAS(par + hi, hi, lo) == hi) return;
        x = hi;
        y = lo;
    }
    atomicOr(bad, 1u);
}

// Exclusive scan of a[0..n) in place with one block (a[n] = total).
__device__ __forceinline__ void block_scan_excl(uint32_t *a, uint32_t n, uint32_t *warp_tot) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t beg = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (beg + i < n) sum += a[beg + i];
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
        if (beg + i < n) {
            const uint32_t c = a[beg + i];
            a[beg + i] = run;
            run += c;
        }
    }
    if (threadIdx.x == 0) a[n] = warp_tot[nwarps - 1];
    __syncthreads();
}

// Whole count in one block.  out[0] = T, out[1] = triangles inside G0,
// out[2] = cross-level triangles, out[3] = 0 on success, 1 if the input
// exceeded the limits (nothing else was written), 2 if the component step
// ran past its bound (never expected; the counts are then 0).
__global__ void __launch_bounds__(kThreads, 1) k_count_noalloc(NoAllocScratch *S, const uint64_t *__restrict__ rp,
                                                               const uint32_t *__restrict__ col, uint32_t n,
                                                               uint32_t order, unsigned long long *out) {
    extern __shared__ uint32_t bitmaps[];  // 16 warps x kBitmapWords
    __shared__ unsigned long long red[32];
    __shared__ uint32_t warp_tot[32];
    __shared__ unsigned int s_cnt[2];
    __shared__ unsigned int s_bad;
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (n > kMaxN || rp[n] > kMaxSlots) {
        if (tid == 0) {
            out[0] = out[1] = out[2] = 0;
            out[3] = 1;
        }
        return;
    }
    uint32_t *par = S->hcnt;     // union-find forest (the row counts reuse it later)
    uint32_t *minkey = S->q[1];  // smallest order key of each component, at its root (then a frontier)
    if (tid == 0) {
        s_bad = 0;
        s_cnt[0] = 0;
    }
    // degrees; isolated vertices are their own roots at level 0
    for (uint32_t v = tid; v < n; v += blockDim.x) {
        const uint32_t d = (uint32_t)(rp[v + 1] - rp[v]);
        S->deg[v] = d;
        S->L[v] = d ? kUnvisited : 0u;
        par[v] = v;
        minkey[v] = 0xFFFFFFFFu;
    }
    __syncthreads();
    // components: one union per edge x < y (a warp per vertex)
    for (uint32_t x = warp; x < n; x += nwarps)
        for (uint64_t j = rp[x] + lane; j < rp[x + 1]; j += 32) {
            const uint32_t y = col[j];
            if (y > x) uf_union(par, x, y, n, &s_bad);
        }
    __syncthreads();
    for (uint32_t v = tid; v < n; v += blockDim.x)
        if (S->deg[v]) {
            const uint32_t r = uf_find(par, v);
            atomicMin(minkey + r, key32(v, S->deg[v], order));
        }
    __syncthreads();
    // roots: the vertex holding its component's smallest key; all start one BFS
    for (uint32_t v = tid; v < n; v += blockDim.x)
        if (S->deg[v] && minkey[uf_find(par, v)] == key32(v, S->deg[v], order)) {
            S->L[v] = 0;
            S->q[0][atomicAdd(&s_cnt[0], 1u)] = v;
        }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            out[0] = out[1] = out[2] = 0;
            out[3] = 2;
        }
        return;
    }
    {
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
    }
    __syncthreads();
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
    block_scan_excl(S->off, n, warp_tot);
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
    // The launch's own status (not cudaGetLastError, which would also report
    // and clear an earlier, unrelated error of the process).
    unsigned long long *out = reinterpret_cast<unsigned long long *>(d_out);
    void *args[] = {&S, (void *)&d_row_ptr, (void *)&d_col, &n, &order, &out};
    const cudaError_t e = cudaLaunchKernel((const void *)k_count_noalloc, dim3(1), dim3(kThreads), args,
                                           16 * kBitmapWords * sizeof(uint32_t), (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the error this launch recorded
        return TC_ERR_CUDA;
    }
    return TC_OK;
}
