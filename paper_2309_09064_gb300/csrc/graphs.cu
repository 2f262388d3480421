// graphs.cu -- many small graphs counted in one launch, one thread block per
// graph at a time (the batched form of the counter).
//
// A persistent grid takes the graphs of a batch from a shared counter,
// largest first, and runs the whole method on each with one block: degrees;
// components by union-find and each component's first vertex in the working
// order as its BFS root; one level-synchronous BFS from all roots; rows
// [H(x) | G1(x)] (H(x): horizontal neighbours that x precedes, G1(x): the
// level-spanning ones); then, for every horizontal edge u -> v, the elements
// of v's row found in u's row.  A hit in H(v) is a triangle on one level
// (counted once, at the edge between its two earlier vertices: Algorithm 2's
// forward count on G0 with the static oriented sets), a hit in G1(v) a
// triangle with exactly one horizontal edge (counted once, at that edge:
// Algorithm 4's hashed loop); a hit across the two parts is impossible
// (different levels).  u's row is a bitmap of n bits in the warp's slice of
// shared memory, so graphs have at most kSmallN vertices.  The probed rows of
// 32 out-neighbours at a time are walked as one flat sequence, every lane
// busy however short the rows are.
//
// One launch (plus the copies of its descriptors and results) counts any
// number of such graphs: no host synchronisation inside the batch, no
// per-graph launches.  Larger graphs take the union pipeline (batch.cu).
#include <algorithm>
#include <numeric>

#include "pipeline.cuh"

namespace tc {

namespace {

constexpr int kGWarps = 8;
constexpr int kGThreads = 32 * kGWarps;

struct SmallGraph {
    const uint64_t *rp;
    const uint32_t *col;
    uint32_t n;
    uint32_t out;  // position of its count
};

// 32-bit working-order key (n <= 65536, so degrees < 65536): smaller key =
// earlier vertex.  Degree order: decreasing degree, ties by ascending id.
__device__ __forceinline__ uint32_t gkey(uint32_t v, uint32_t d, uint32_t order) {
    return order == TC_ORDER_DEGREE ? ((0xFFFFu - d) << 16) | v : v;
}

__device__ __forceinline__ uint32_t gload(const uint32_t *p) { return *(const volatile uint32_t *)p; }

// Union-find root of x with path halving (par[v] <= v; each step moves to a
// smaller index, so the walk ends).
__device__ __forceinline__ uint32_t gfind(uint32_t *par, uint32_t x) {
    uint32_t p = gload(par + x);
    while (p != x) {
        const uint32_t gp = gload(par + p);
        if (gp != p) *(volatile uint32_t *)(par + x) = gp;
        x = p;
        p = gp;
    }
    return x;
}

// Hook the larger root under the smaller.  A failed swap means that root was
// hooked by another thread meanwhile (at most n - 1 hooks in all), so n + 1
// tries always suffice; past them *bad is set.
__device__ __forceinline__ void gunion(uint32_t *par, uint32_t x, uint32_t y, uint32_t n, unsigned int *bad) {
    for (uint32_t it = 0; it <= n; ++it) {
        const uint32_t rx = gfind(par, x), ry = gfind(par, y);
        if (rx == ry) return;
        const uint32_t hi = rx > ry ? rx : ry, lo = rx > ry ? ry : rx;
        if (atomicCAS(par + hi, hi, lo) == hi) return;
        x = hi;
        y = lo;
    }
    atomicOr(bad, 1u);
}

// Exclusive scan of a[0..n) in place by the block (a[n] = total).
__device__ __forceinline__ void gscan(uint32_t *a, uint32_t n, uint32_t *warp_tot) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
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
        uint32_t t = lane < (unsigned)kGWarps ? warp_tot[lane] : 0u;
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
    if (threadIdx.x == 0) a[n] = warp_tot[kGWarps - 1];
    __syncthreads();
}

// One graph with the whole block.  Scratch (global, this block's slice):
// deg, L, q0, q1, h (union-find forest first, then |H(x)|) of nmax words,
// off of nmax + 1, adj2 of the graph's slots.  Returns T (thread 0), or
// ~0 if the component step ran past its bound (never expected).
__device__ __forceinline__ unsigned long long count_one(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col, uint32_t n,
                                        uint32_t order, uint32_t *deg, uint32_t *L, uint32_t *q0, uint32_t *q1,
                                        uint32_t *h, uint32_t *off, uint32_t *adj2, uint32_t *bm_all,
                                        uint32_t bm_words) {
    __shared__ uint32_t warp_tot[32];
    __shared__ unsigned int s_cnt[2], s_bad, s_next;
    __shared__ unsigned long long s_tot;
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (tid == 0) {
        s_bad = 0;
        s_cnt[0] = 0;
        s_next = 0;
        s_tot = 0;
    }
    for (uint32_t v = tid; v < n; v += blockDim.x) {
        const uint32_t d = (uint32_t)(rp[v + 1] - rp[v]);
        deg[v] = d;
        L[v] = d ? kUnvisited : 0u;  // isolated vertices: their own roots, level 0
        h[v] = v;
        q1[v] = 0xFFFFFFFFu;
    }
    __syncthreads();
    for (uint32_t x = warp; x < n; x += kGWarps)
        for (uint64_t j = rp[x] + lane; j < rp[x + 1]; j += 32) {
            const uint32_t y = col[j];
            if (y > x) gunion(h, x, y, n, &s_bad);
        }
    __syncthreads();
    for (uint32_t v = tid; v < n; v += blockDim.x)
        if (deg[v]) atomicMin(q1 + gfind(h, v), gkey(v, deg[v], order));
    __syncthreads();
    for (uint32_t v = tid; v < n; v += blockDim.x)
        if (deg[v] && q1[gfind(h, v)] == gkey(v, deg[v], order)) {
            L[v] = 0;
            q0[atomicAdd(&s_cnt[0], 1u)] = v;
        }
    __syncthreads();
    if (s_bad) return ~0ull;
    for (uint32_t cur = 0, level = 0;; cur ^= 1, ++level) {
        const uint32_t fcount = s_cnt[cur];
        if (fcount == 0) break;
        if (tid == 0) s_cnt[cur ^ 1] = 0;
        __syncthreads();
        const uint32_t *qc = cur ? q1 : q0;
        uint32_t *qn = cur ? q0 : q1;
        for (uint32_t i = warp; i < fcount; i += kGWarps) {
            const uint32_t v = qc[i];
            for (uint64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) {
                const uint32_t w = col[j];
                if (L[w] == kUnvisited && atomicCAS(&L[w], kUnvisited, level + 1) == kUnvisited)
                    qn[atomicAdd(&s_cnt[cur ^ 1], 1u)] = w;
            }
        }
        __syncthreads();
    }
    // rows [H(x) | G1(x)]: lengths, scan, fill (a warp per vertex, ballot order)
    for (uint32_t x = warp; x < n; x += kGWarps) {
        const uint32_t dx = deg[x], lx = L[x];
        uint32_t hh = 0, g = 0;
        for (uint64_t j = rp[x] + lane; j < rp[x + 1]; j += 32) {
            const uint32_t y = col[j];
            if (L[y] != lx) ++g;
            else if (precedes(x, dx, y, deg[y], order)) ++hh;
        }
        hh = warp_sum(hh);
        g = warp_sum(g);
        if (lane == 0) {
            h[x] = hh;
            off[x] = hh + g;
        }
    }
    __syncthreads();
    gscan(off, n, warp_tot);
    for (uint32_t x = warp; x < n; x += kGWarps) {
        const uint32_t dx = deg[x], lx = L[x];
        const uint32_t base = off[x], hx = h[x];
        uint32_t hp = 0, gp = 0;
        for (uint64_t j0 = rp[x]; j0 < rp[x + 1]; j0 += 32) {
            const uint64_t j = j0 + lane;
            bool isH = false, isG = false;
            uint32_t y = 0;
            if (j < rp[x + 1]) {
                y = col[j];
                if (L[y] != lx) isG = true;
                else isH = precedes(x, dx, y, deg[y], order);
            }
            const unsigned mh = __ballot_sync(0xFFFFFFFFu, isH), mg = __ballot_sync(0xFFFFFFFFu, isG);
            if (isH) adj2[base + hp + __popc(mh & lt)] = y;
            if (isG) adj2[base + hx + gp + __popc(mg & lt)] = y;
            hp += __popc(mh);
            gp += __popc(mg);
        }
    }
    __syncthreads();
    // intersections: warps take hashed vertices u from a shared counter; u's
    // row becomes bits of the warp's bitmap; the rows of 32 out-neighbours at
    // a time are probed as one flat sequence
    uint32_t *bm = bm_all + (size_t)warp * bm_words;
    unsigned long long same = 0, cross = 0;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(&s_next, 1u);
        u = __shfl_sync(0xFFFFFFFFu, u, 0);
        if (u >= n) break;
        const uint32_t hu = h[u];
        if (hu == 0) continue;
        const uint32_t ub = off[u], ue = off[u + 1];
        for (uint32_t j = ub + lane; j < ue; j += 32) {
            const uint32_t w = adj2[j];
            atomicOr(bm + (w >> 5), 1u << (w & 31u));
        }
        __syncwarp();
        for (uint32_t k0 = 0; k0 < hu; k0 += 32) {
            const uint32_t k = k0 + lane;
            uint32_t vb = 0, vlen = 0, vh = 0;
            if (k < hu) {
                const uint32_t v = adj2[ub + k];
                vb = off[v];
                vlen = off[v + 1] - vb;
                vh = h[v];
            }
            uint32_t incl = vlen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= (unsigned)o) incl += y;
            }
            const uint32_t excl = incl - vlen;
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            for (uint32_t p0 = 0; p0 < total; p0 += 32) {
                const uint32_t p = p0 + lane;
                // owner: the last lane r with excl_r <= p (ranges of length 0 are skipped by it)
                uint32_t r = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, r + step);
                    if (e <= p) r += step;
                }
                const uint32_t er = __shfl_sync(0xFFFFFFFFu, excl, r);
                const uint32_t br = __shfl_sync(0xFFFFFFFFu, vb, r);
                const uint32_t hr = __shfl_sync(0xFFFFFFFFu, vh, r);
                if (p < total) {
                    const uint32_t j = p - er;
                    const uint32_t w = adj2[br + j];
                    if ((bm[w >> 5] >> (w & 31u)) & 1u) {
                        if (j < hr) ++same;
                        else ++cross;
                    }
                }
            }
        }
        __syncwarp();
        for (uint32_t j = ub + lane; j < ue; j += 32) bm[adj2[j] >> 5] = 0u;
        __syncwarp();
    }
    const unsigned long long t = warp_sum(same + cross);
    if (lane == 0 && t) atomicAdd(&s_tot, t);
    __syncthreads();
    const unsigned long long T = s_tot;
    __syncthreads();  // s_tot and the other shared words are reset by the next graph's thread 0
    return T;
}

// Persistent: blocks take graphs in the order `order_idx` (largest first).
// counts[g.out] gets T of each graph; err gets 1 if a component step failed.
__global__ void __launch_bounds__(kGThreads) k_count_graphs(const SmallGraph *__restrict__ gs,
                                                            const uint32_t *__restrict__ order_idx, uint32_t G,
                                                            unsigned int *next, uint32_t *scratch,
                                                            unsigned long long words_per_block, uint32_t nmax,
                                                            uint32_t bm_words, uint32_t order,
                                                            unsigned long long *counts, unsigned int *err) {
    extern __shared__ uint32_t gbm[];  // kGWarps bitmaps of bm_words words
    __shared__ unsigned int s_i;
    for (uint32_t j = threadIdx.x; j < kGWarps * bm_words; j += blockDim.x) gbm[j] = 0u;
    uint32_t *base = scratch + (size_t)blockIdx.x * words_per_block;
    uint32_t *deg = base, *L = deg + nmax, *q0 = L + nmax, *q1 = q0 + nmax, *h = q1 + nmax, *off = h + nmax;
    uint32_t *adj2 = off + nmax + 1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_i = atomicAdd(next, 1u);
        __syncthreads();
        if (s_i >= G) break;
        const SmallGraph g = gs[order_idx[s_i]];
        const unsigned long long T = count_one(g.rp, g.col, g.n, order, deg, L, q0, q1, h, off, adj2, gbm, bm_words);
        if (threadIdx.x == 0) {
            if (T == ~0ull) {
                atomicOr(err, 1u);
                counts[g.out] = 0;
            } else {
                counts[g.out] = T;
            }
        }
    }
}

}  // namespace

bool small_graph_fits(const tc_graph *g, uint64_t max_slots) { return g->n <= kSmallN && g->slots <= max_slots; }

size_t small_graphs_bytes(const tc_ctx *ctx, uint32_t nmax, uint64_t smax, uint32_t G, uint32_t *blocks) {
    const size_t smem = 4ull * kGWarps * ((nmax + 31) / 32);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_graphs, kGThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    *blocks = std::min<uint32_t>(G, (uint32_t)(ctx->num_sms * per_sm));
    const uint64_t words = 6ull * nmax + 1 + smax;
    return (size_t)(*blocks) * ((words * 4 + 255) & ~255ull) + sizeof(SmallGraph) * (size_t)G + 4ull * (G + 2) + 256;
}

// Count graphs[i] for i in idx (all small: small_graph_fits) into d_counts[i]
// (device), on the context's stream; no synchronisation.  scratch: bytes from
// small_graphs_bytes.  *d_err gets the device word that is 1 if a graph's
// component step failed (its count is then 0).
tc_status count_small_graphs(tc_ctx *ctx, const tc_graph *const *graphs, const std::vector<uint32_t> &idx,
                             unsigned long long *d_counts, char *scratch, size_t scratch_bytes, unsigned int **d_err) {
    cudaStream_t s = ctx->stream;
    const uint32_t G = (uint32_t)idx.size();
    if (G == 0) return TC_OK;
    std::vector<SmallGraph> gs(G);
    uint32_t nmax = 1;
    uint64_t smax = 1;
    for (uint32_t i = 0; i < G; ++i) {
        const tc_graph *g = graphs[idx[i]];
        gs[i] = SmallGraph{g->rp, g->col, g->n, idx[i]};
        nmax = std::max(nmax, g->n);
        smax = std::max<uint64_t>(smax, g->slots);
    }
    std::vector<uint32_t> order(G);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        return graphs[idx[a]]->slots > graphs[idx[b]]->slots;  // largest first
    });
    uint32_t blocks = 0;
    const size_t need = small_graphs_bytes(ctx, nmax, smax, G, &blocks);
    if (need > scratch_bytes) return set_error(ctx, TC_ERR_OOM, "small-graph scratch too small");
    const unsigned long long words = (((6ull * nmax + 1 + smax) * 4 + 255) & ~255ull) / 4;
    uint32_t *d_scr = reinterpret_cast<uint32_t *>(scratch);
    auto *d_gs = reinterpret_cast<SmallGraph *>(scratch + (size_t)blocks * words * 4);
    auto *d_order = reinterpret_cast<uint32_t *>(d_gs + G);
    auto *d_next = reinterpret_cast<unsigned int *>(d_order + G);  // then the error word
    *d_err = d_next + 1;
    TC_CUDA(ctx, cudaMemcpyAsync(d_gs, gs.data(), sizeof(SmallGraph) * G, cudaMemcpyHostToDevice, s));
    TC_CUDA(ctx, cudaMemcpyAsync(d_order, order.data(), 4ull * G, cudaMemcpyHostToDevice, s));
    TC_CUDA(ctx, cudaMemsetAsync(d_next, 0, 8, s));
    const uint32_t bm_words = (nmax + 31) / 32;
    const size_t smem = 4ull * kGWarps * bm_words;
    TC_CUDA(ctx, cudaFuncSetAttribute(k_count_graphs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_count_graphs<<<blocks, kGThreads, smem, s>>>(d_gs, d_order, G, d_next, d_scr, words, nmax, bm_words,
                                                   ctx->opt.order, d_counts, d_next + 1);
    note_launch(ctx);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
