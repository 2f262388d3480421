// levels.cu -- degrees, canonical BFS roots and BFS levels (Algorithm 4, BFS loop).
//
// Algorithm 4 starts a BFS from every vertex still unvisited, taking vertices in
// the working order, so every component's root is its first vertex in that order
// (degree order: highest degree, then lowest id).  On the GPU:
//   1. k_init computes degrees, gives isolated vertices level 0 (each is its
//      own root) and finds the globally first non-isolated vertex;
//   2. a direction-optimising frontier BFS (top-down with edge-balanced
//      expansion, bottom-up when the frontier is large) levels its component;
//   3. the vertices still unvisited form the other components: min-key
//      hooking with pointer jumping finds each one's first vertex, and a
//      multi-source BFS from those roots levels them.
// BFS distances are unique given the roots, so L matches the serial
// algorithm exactly whatever the thread schedule.
#include <algorithm>

#include "pipeline.cuh"

namespace tc {
namespace {

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        v = y < v ? y : v;
    }
    return v;
}

__global__ void k_init(uint32_t n, const uint64_t *__restrict__ rp, uint32_t *__restrict__ deg,
                       uint32_t *__restrict__ L, Ctl *ctl, uint32_t order) {
    __shared__ unsigned int s_iso;
    __shared__ unsigned long long s_key;
    if (threadIdx.x == 0) {
        s_iso = 0;
        s_key = ~0ull;
    }
    __syncthreads();
    unsigned long long best = ~0ull;
    unsigned iso = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t d = (uint32_t)(rp[v + 1] - rp[v]);
        deg[v] = d;
        if (d == 0) {
            L[v] = 0;
            ++iso;
        } else {
            L[v] = kUnvisited;
            unsigned long long k = order_key((uint32_t)v, d, order);
            best = k < best ? k : best;
        }
    }
    best = warp_min_u64(best);
    iso = warp_sum(iso);
    if (lane_id() == 0) {
        atomicMin(&s_key, best);
        atomicAdd(&s_iso, iso);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_key != ~0ull) atomicMin(&ctl->root_key, s_key);
        if (s_iso) {
            atomicAdd(&ctl->visited, s_iso);
            atomicAdd(&ctl->components, s_iso);
        }
    }
}

// Seed the BFS with the globally first non-isolated vertex (if any).
__global__ void k_seed(const uint32_t *__restrict__ deg, uint32_t *__restrict__ L, uint32_t *__restrict__ q,
                       Ctl *ctl, int cur) {
    unsigned long long key = ctl->root_key;
    if (key == ~0ull) return;
    uint32_t r = (uint32_t)(key & 0xFFFFFFFFull);
    L[r] = 0;
    q[0] = r;
    ctl->fr_count[cur] = 1;
    ctl->fr_edges[cur] = deg[r];
    ctl->visited += 1;
    ctl->visited_edges += deg[r];
    ctl->components += 1;
}

__global__ void k_gather_deg(const uint32_t *__restrict__ q, uint32_t count, const uint32_t *__restrict__ deg,
                             uint32_t *__restrict__ out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) out[i] = deg[q[i]];
}

constexpr int kTdThreads = 256;
constexpr int kTdItems = 8;
constexpr uint64_t kTdTile = (uint64_t)kTdThreads * kTdItems;

// Top-down step with edge-balanced expansion: the frontier's adjacency lists
// are viewed as one concatenated list (fpref = exclusive prefix of frontier
// degrees); each block takes tiles of kTdTile consecutive entries.
__global__ void __launch_bounds__(kTdThreads) k_td(const uint32_t *__restrict__ q, uint32_t fcount,
                                                   const unsigned long long *__restrict__ fpref,
                                                   const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                                   const uint32_t *__restrict__ deg, uint32_t *__restrict__ L,
                                                   uint32_t *__restrict__ qn, Ctl *ctl, uint32_t level, int nxt) {
    __shared__ uint32_t s_lo, s_hi;
    __shared__ unsigned long long s_edges;
    const unsigned long long total = fpref[fcount];
    unsigned long long edges = 0;
    for (unsigned long long t0 = (unsigned long long)blockIdx.x * kTdTile; t0 < total;
         t0 += (unsigned long long)gridDim.x * kTdTile) {
        const unsigned long long t1 = t0 + kTdTile < total ? t0 + kTdTile : total;
        if (threadIdx.x == 0) {
            // frontier slots holding entries t0 and t1-1: largest i with fpref[i] <= x
            uint32_t a = 0, b = fcount;
            while (b - a > 1) {
                uint32_t m = (a + b) >> 1;
                if (fpref[m] <= t0) a = m; else b = m;
            }
            s_lo = a;
            b = fcount;
            while (b - a > 1) {
                uint32_t m = (a + b) >> 1;
                if (fpref[m] <= t1 - 1) a = m; else b = m;
            }
            s_hi = a;
        }
        __syncthreads();
        const uint32_t lo = s_lo, hi = s_hi;
        __syncthreads();
#pragma unroll 1
        for (int it = 0; it < kTdItems; ++it) {
            const unsigned long long e = t0 + (unsigned long long)it * kTdThreads + threadIdx.x;
            bool claim = false;
            uint32_t w = 0;
            if (e < t1) {
                uint32_t a = lo, b = hi + 1;
                while (b - a > 1) {
                    uint32_t m = (a + b) >> 1;
                    if (fpref[m] <= e) a = m; else b = m;
                }
                const uint32_t v = q[a];
                w = col[rp[v] + (e - fpref[a])];
                if (L[w] == kUnvisited && atomicCAS(&L[w], kUnvisited, level + 1) == kUnvisited) claim = true;
            }
            uint32_t slot = warp_append(claim, &ctl->fr_count[nxt]);
            if (claim) {
                qn[slot] = w;
                edges += deg[w];
            }
        }
    }
    edges = warp_sum(edges);
    if (threadIdx.x == 0) s_edges = 0;
    __syncthreads();
    if (lane_id() == 0 && edges) atomicAdd(&s_edges, edges);
    __syncthreads();
    if (threadIdx.x == 0 && s_edges) atomicAdd(&ctl->fr_edges[nxt], s_edges);
}

// Bottom-up step: every unvisited vertex looks for a neighbour on `level`.
__global__ void k_bu(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                     const uint32_t *__restrict__ deg, uint32_t *__restrict__ L, uint32_t *__restrict__ qn, Ctl *ctl,
                     uint32_t level, int nxt) {
    __shared__ unsigned long long s_edges;
    if (threadIdx.x == 0) s_edges = 0;
    __syncthreads();
    unsigned long long edges = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_round = ((uint64_t)n + 31) & ~uint64_t(31);
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_round; v += stride) {
        bool found = false;
        if (v < n && L[v] == kUnvisited) {
            const uint64_t b = rp[v], e = rp[v + 1];
            for (uint64_t j = b; j < e; ++j) {
                if (L[col[j]] == level) {
                    found = true;
                    break;
                }
            }
            if (found) L[v] = level + 1;
        }
        uint32_t slot = warp_append(found, &ctl->fr_count[nxt]);
        if (found) {
            qn[slot] = (uint32_t)v;
            edges += deg[v];
        }
    }
    edges = warp_sum(edges);
    if (lane_id() == 0 && edges) atomicAdd(&s_edges, edges);
    __syncthreads();
    if (threadIdx.x == 0 && s_edges) atomicAdd(&ctl->fr_edges[nxt], s_edges);
}

__global__ void k_collect_unvisited(uint32_t n, const uint32_t *__restrict__ L, uint32_t *__restrict__ R, Ctl *ctl) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_round = ((uint64_t)n + 31) & ~uint64_t(31);
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_round; v += stride) {
        bool un = v < n && L[v] == kUnvisited;
        uint32_t slot = warp_append(un, &ctl->n_residual);
        if (un) R[slot] = (uint32_t)v;
    }
}

__global__ void k_cc_init(const uint32_t *__restrict__ R, uint32_t nr, uint32_t *__restrict__ parent) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) parent[R[i]] = R[i];
}

// Follow parent pointers to the root.  Pointers always lead to a vertex with a
// smaller key, so the walk ends; the bound only guards against a corrupted
// array and raises the error flag.
__device__ __forceinline__ uint32_t find_root(const uint32_t *parent, uint32_t x, uint32_t n, Ctl *ctl) {
    for (uint32_t it = 0; it <= n; ++it) {
        uint32_t p = parent[x];
        if (p == x) return x;
        x = p;
    }
    ctl->error = 2;
    return x;
}

// Hooking: for every edge joining two trees, attach the root with the larger
// working-order key under the root with the smaller one.
__global__ void k_cc_hook(const uint32_t *__restrict__ R, uint32_t nr, uint32_t n, const uint64_t *__restrict__ rp,
                          const uint32_t *__restrict__ col, const uint32_t *__restrict__ deg, uint32_t *parent,
                          Ctl *ctl, uint32_t order) {
    const uint32_t stride = gridDim.x * blockDim.x;
    bool changed = false;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        const uint32_t v = R[i];
        for (uint64_t j = rp[v]; j < rp[v + 1]; ++j) {
            const uint32_t w = col[j];
            if (w < v) continue;  // each undirected edge once
            uint32_t rv = find_root(parent, v, n, ctl), rw = find_root(parent, w, n, ctl);
            if (rv == rw) continue;
            unsigned long long kv = order_key(rv, deg[rv], order), kw = order_key(rw, deg[rw], order);
            uint32_t hi = kv < kw ? rw : rv, lo = kv < kw ? rv : rw;
            atomicCAS(&parent[hi], hi, lo);
            changed = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, changed) && lane_id() == 0) ctl->changed = 1;
}

__global__ void k_cc_compress(const uint32_t *__restrict__ R, uint32_t nr, uint32_t n, uint32_t *parent, Ctl *ctl) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        const uint32_t v = R[i];
        parent[v] = find_root(parent, v, n, ctl);
    }
}

__global__ void k_cc_roots(const uint32_t *__restrict__ R, uint32_t nr, const uint32_t *__restrict__ parent,
                           const uint32_t *__restrict__ deg, uint32_t *__restrict__ L, uint32_t *__restrict__ q,
                           Ctl *ctl, int cur) {
    __shared__ unsigned long long s_edges;
    if (threadIdx.x == 0) s_edges = 0;
    __syncthreads();
    unsigned long long edges = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t nr_round = (nr + 31) & ~31u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr_round; i += stride) {
        bool root = false;
        uint32_t v = 0;
        if (i < nr) {
            v = R[i];
            root = parent[v] == v;
        }
        uint32_t slot = warp_append(root, &ctl->fr_count[cur]);
        if (root) {
            L[v] = 0;
            q[slot] = v;
            edges += deg[v];
        }
    }
    edges = warp_sum(edges);
    if (lane_id() == 0 && edges) atomicAdd(&s_edges, edges);
    __syncthreads();
    if (threadIdx.x == 0 && s_edges) atomicAdd(&ctl->fr_edges[cur], s_edges);
}

__global__ void k_count_roots(Ctl *ctl, int cur) {
    ctl->components += ctl->fr_count[cur];
    ctl->visited += ctl->fr_count[cur];
    ctl->visited_edges += ctl->fr_edges[cur];
}

__global__ void k_reset_next(Ctl *ctl, int nxt) {
    ctl->fr_count[nxt] = 0;
    ctl->fr_edges[nxt] = 0;
    ctl->bar_count = 0;  // a persistent launch may follow: its barriers count from zero
}

__global__ void k_after_level(Ctl *ctl, int nxt, uint32_t level) {
    ctl->visited += ctl->fr_count[nxt];
    ctl->visited_edges += ctl->fr_edges[nxt];
    if (ctl->fr_count[nxt]) ctl->max_level = level + 1 > ctl->max_level ? level + 1 : ctl->max_level;
}

// Grid-wide barrier for the persistent BFS (all blocks are co-resident: the
// kernel is launched cooperatively).  The arrival counter only grows within
// a launch (the host zeroes it before each launch): barrier k of the launch
// is passed once the counter reaches (k + 1) x nblocks, so an arriving block
// adds one and waits for that count, with no generation word to reset.  A
// wait gives up after `timeout_cycles` of clock time, raises the error flag
// and returns false, so the kernel ends and the host reads TC_ERR_TIMEOUT.
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, unsigned nblocks, unsigned k, long long timeout_cycles) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *count = &ctl->bar_count;
        const unsigned target = (k + 1) * nblocks;
        __threadfence();  // this block's frontier writes before its arrival
        atomicAdd(&ctl->bar_count, 1u);
        int ok = 1;
        const long long t0 = clock64();
        while (*count < target) {
            if (clock64() - t0 > timeout_cycles) {
                ctl->error = 4;
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Persistent top-down BFS for small frontiers (high-diameter graphs): one
// launch runs level after level, one grid barrier per level, until the
// frontier is empty or leaves [min_f, max_f] x [0, max_e], or its mean
// degree passes max_avg (a high-degree vertex would hold up the one warp
// that expands it; the edge-balanced kernel spreads it over the GPU); then
// the host takes over again.  A frontier vertex of degree <= 32 is expanded
// by a group of G lanes (G = the threads the grid has per frontier vertex,
// a power of two up to 32; one thread when the frontier is large); larger
// rows by the whole warp, one at a time.  Counter slots rotate mod 3 (level L reads
// slot s, writes s+1, and s+2 is cleared for level L+1); queues alternate.
__global__ void __launch_bounds__(512) k_bfs_persist(uint32_t *__restrict__ q0, uint32_t *__restrict__ q1,
                                                     const uint64_t *__restrict__ rp,
                                                     const uint32_t *__restrict__ col,
                                                     const uint32_t *__restrict__ deg, uint32_t *L, Ctl *ctl,
                                                     uint32_t slot, uint32_t queue, uint32_t level, uint32_t max_f,
                                                     unsigned long long max_e, uint32_t min_f, uint32_t max_avg) {
    const unsigned lane = lane_id();
    const unsigned gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    volatile unsigned *vcount = ctl->fr_count;
    volatile unsigned long long *vedges = ctl->fr_edges;
    // levels this launch adds (written once at the end by block 0, thread 0)
    unsigned int add_visited = 0;
    unsigned long long add_edges = 0;
    uint32_t start_level = level;
    unsigned bar_k = 0;  // barriers passed in this launch
    for (;;) {
        const uint32_t fcount = vcount[slot];
        const unsigned long long fedges = vedges[slot];
        if (fcount == 0 || fcount > max_f || fedges > max_e || fcount < min_f ||
            fedges > (unsigned long long)fcount * max_avg)
            break;
        const uint32_t s1 = slot == 2 ? 0 : slot + 1, s2 = s1 == 2 ? 0 : s1 + 1;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->fr_count[s2] = 0;
            ctl->fr_edges[s2] = 0;
        }
        const uint32_t *q = queue ? q1 : q0;
        uint32_t *qn = queue ? q0 : q1;
        unsigned long long edges = 0;
        const uint32_t nthreads = nwarps * 32u, gtid = gwarp * 32u + lane;
        // Lanes per frontier vertex: as many as the grid has to spare (a power
        // of two up to 32), so that the neighbours of a small frontier are
        // visited in parallel rather than one after another by one thread.
        uint32_t G = 1;
        while (G < 32 && (unsigned long long)fcount * (G * 2) <= nthreads) G <<= 1;
        const uint32_t sub = lane & (G - 1), ngroups = nthreads / G, vt = gtid / G;
        for (uint32_t r0 = 0; r0 < fcount; r0 += ngroups) {
            const uint32_t i = r0 + vt;
            const bool valid = i < fcount;
            const uint32_t v = valid ? q[i] : 0u;
            const uint64_t b = valid ? rp[v] : 0, e = valid ? rp[v + 1] : 0;
            const bool small = e - b <= 32;
            if (G == 1) {
                if (small) {
                    for (uint64_t j = b; j < e; ++j) {
                        const uint32_t w = col[j];
                        if (L[w] == kUnvisited && atomicCAS(&L[w], kUnvisited, level + 1) == kUnvisited) {
                            qn[atomicAdd(&ctl->fr_count[s1], 1u)] = w;
                            edges += deg[w];
                        }
                    }
                }
            } else {  // the G lanes of a group take their vertex's neighbours in turn
                const uint32_t d = valid && small ? (uint32_t)(e - b) : 0u;
                const uint32_t kmax = __reduce_max_sync(0xFFFFFFFFu, (d + G - 1) / G);
                for (uint32_t k = 0; k < kmax; ++k) {
                    const uint32_t j = k * G + sub;
                    bool claim = false;
                    uint32_t w = 0, dw = 0;
                    if (j < d) {
                        w = col[b + j];
                        dw = deg[w];  // read beside L[w], not after the claim
                        claim = L[w] == kUnvisited && atomicCAS(&L[w], kUnvisited, level + 1) == kUnvisited;
                    }
                    const uint32_t pos = warp_append(claim, &ctl->fr_count[s1]);
                    if (claim) {
                        qn[pos] = w;
                        edges += dw;
                    }
                }
            }
            unsigned big = __ballot_sync(0xFFFFFFFFu, valid && !small && sub == 0);
            while (big) {
                const int src = __ffs(big) - 1;
                big &= big - 1;
                const uint64_t bb = __shfl_sync(0xFFFFFFFFu, b, src), be = __shfl_sync(0xFFFFFFFFu, e, src);
                for (uint64_t j0 = bb; j0 < be; j0 += 32) {
                    const uint64_t j = j0 + lane;
                    bool claim = false;
                    uint32_t w = 0;
                    if (j < be) {
                        w = col[j];
                        claim = L[w] == kUnvisited && atomicCAS(&L[w], kUnvisited, level + 1) == kUnvisited;
                    }
                    const uint32_t pos = warp_append(claim, &ctl->fr_count[s1]);
                    if (claim) {
                        qn[pos] = w;
                        edges += deg[w];
                    }
                }
            }
        }
        edges = warp_sum(edges);
        if (lane == 0 && edges) atomicAdd(&ctl->fr_edges[s1], edges);
        if (!grid_barrier(ctl, gridDim.x, bar_k++, 4000000000ll)) return;  // ~2 s at 2 GHz
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            add_visited += vcount[s1];
            add_edges += vedges[s1];
        }
        slot = s1;
        queue ^= 1u;
        ++level;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->p_slot = slot;
        ctl->p_queue = queue;
        ctl->p_level = level;
        ctl->visited += add_visited;
        ctl->visited_edges += add_edges;
        // the last level that received vertices: the final frontier's level if it is
        // non-empty, else the one before
        const uint32_t last = vcount[slot] ? level : level - 1;
        if (level > start_level && last > ctl->max_level) ctl->max_level = last;
    }
}

// Self-test of the bounded wait: the barrier expects one more block than the
// grid has, so no generation change ever comes and every block times out.
__global__ void k_barrier_selftest(Ctl *ctl, long long timeout_cycles) {
    grid_barrier(ctl, gridDim.x + 1, 0, timeout_cycles);
}

unsigned grid_for(uint64_t work, unsigned threads, unsigned cap) {
    uint64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

constexpr uint32_t kPersistMaxF = 32768;          // frontier vertices (whole-grid mode)
constexpr unsigned long long kPersistMaxE = 65536;  // frontier edges
constexpr uint32_t kPersistMaxAvg = 256;            // mean frontier degree

// Levels given by the caller: degrees, a copy of the levels, their maximum,
// and the check that makes the count exact with them -- every edge joins
// vertices whose levels differ by at most one (then a triangle's levels are
// {l, l, l} or {l, l, l +- 1}: exactly three or exactly one horizontal edge).
// Lanes own rows of degree <= 32, whole warps take the longer rows.
__global__ void k_given_levels(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                               const uint32_t *__restrict__ given, uint32_t *__restrict__ deg,
                               uint32_t *__restrict__ L, Ctl *ctl) {
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_round = ((uint64_t)n + 31) & ~uint64_t(31);
    unsigned bad = 0, top = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_round; x += stride) {
        const bool valid = x < n;
        const uint64_t b = valid ? rp[x] : 0;
        const uint32_t d = valid ? (uint32_t)(rp[x + 1] - b) : 0;
        const uint32_t lx = valid ? given[x] : 0;
        if (valid) {
            deg[x] = d;
            L[x] = lx;
            top = lx > top ? lx : top;
        }
        if (valid && d <= 32)
            for (uint32_t j = 0; j < d; ++j) {
                const uint32_t ly = given[col[b + j]];
                bad |= (ly > lx ? ly - lx : lx - ly) > 1u;
            }
        unsigned pending = __ballot_sync(0xFFFFFFFFu, valid && d > 32);
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1;
            const uint64_t bb = __shfl_sync(0xFFFFFFFFu, b, src);
            const uint32_t bd = __shfl_sync(0xFFFFFFFFu, d, src);
            const uint32_t bl = __shfl_sync(0xFFFFFFFFu, lx, src);
            for (uint32_t j = lane; j < bd; j += 32) {
                const uint32_t ly = given[col[bb + j]];
                bad |= (ly > bl ? ly - bl : bl - ly) > 1u;
            }
        }
    }
    bad = __any_sync(0xFFFFFFFFu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned y = __shfl_xor_sync(0xFFFFFFFFu, top, o);
        top = y > top ? y : top;
    }
    if (lane == 0) {
        if (bad) atomicOr(&ctl->error, 0x200u);
        if (top) atomicMax(&ctl->max_level, top);
    }
}

}  // namespace

// Pull the control block to the host (synchronises the stream).
static tc_status pull_ctl(tc_ctx *ctx) {
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    TC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return TC_OK;
}

// Level-synchronous BFS from the frontier in queue `queue`, counter slot
// `slot` (levels 0 .. start_level already assigned).  Per level the host
// chooses top-down (edge-balanced) or bottom-up (Beamer et al.'s edge/vertex
// heuristics); runs of small frontiers go to the persistent kernel.
static tc_status bfs_loop(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots, uint32_t start_level,
                          uint32_t slot, uint32_t queue) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    uint32_t level = start_level;
    bool bottom_up = false;
    tc_status st = pull_ctl(ctx);
    if (st != TC_OK) return st;
    uint32_t fcount = ctx->h_ctl->fr_count[slot];
    unsigned long long fedges = ctx->h_ctl->fr_edges[slot];
    uint32_t prev_count = 0;
    int persist_blocks = -1;
    while (fcount > 0) {
        const unsigned long long unexplored = slots - ctx->h_ctl->visited_edges;
        if (!bottom_up && fedges > unexplored / 14 && fcount > 64) bottom_up = true;
        else if (bottom_up && fcount < n / 24 && fcount < prev_count) bottom_up = false;
        const uint32_t nxt = slot == 2 ? 0 : slot + 1;
        if (!bottom_up && fcount <= kPersistMaxF && fedges <= kPersistMaxE &&
            fedges <= (unsigned long long)fcount * kPersistMaxAvg) {
            if (persist_blocks < 0) {
                int per_sm = 0;
                TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_persist, 512, 0));
                // enough threads for the largest frontier it takes, no more: fewer
                // blocks make the per-level grid barrier cheaper
                persist_blocks = std::min<int>(std::max(1, std::min(per_sm, 1)) * ctx->num_sms,
                                               (int)((kPersistMaxF + 511) / 512));
            }
            k_reset_next<<<1, 1, 0, s>>>(ctx->d_ctl, (int)nxt);
            uint32_t *q0 = b.q0, *q1 = b.q1;
            const uint64_t *rp = b.rp;
            const uint32_t *col = b.col, *deg = b.deg;
            uint32_t *L = b.L;
            Ctl *ctl = ctx->d_ctl;
            uint32_t a_slot = slot, a_queue = queue, a_level = level;
            uint32_t a_max_f = kPersistMaxF, a_min_f = 0, a_max_avg = kPersistMaxAvg;
            unsigned long long a_max_e = kPersistMaxE;
            void *args[] = {&q0, &q1, &rp, &col, &deg, &L, &ctl, &a_slot, &a_queue, &a_level, &a_max_f, &a_max_e,
                            &a_min_f, &a_max_avg};
            TC_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_bfs_persist, dim3(persist_blocks), dim3(512),
                                                     args, 0, s));
            note_launch(ctx, 2);
            st = pull_ctl(ctx);
            if (st != TC_OK) return st;
            if (ctx->h_ctl->error == 4) return set_error(ctx, TC_ERR_TIMEOUT, "persistent BFS barrier timed out");
            slot = ctx->h_ctl->p_slot;
            queue = ctx->h_ctl->p_queue;
            level = ctx->h_ctl->p_level;
            prev_count = fcount;
            fcount = ctx->h_ctl->fr_count[slot];
            fedges = ctx->h_ctl->fr_edges[slot];
            continue;  // the frontier is empty or too large for the persistent kernel
        }
        uint32_t *q = queue ? b.q1 : b.q0;
        uint32_t *qn = queue ? b.q0 : b.q1;
        k_reset_next<<<1, 1, 0, s>>>(ctx->d_ctl, (int)nxt);
        note_launch(ctx, 2);  // reset + after-level bookkeeping
        if (bottom_up) {
            k_bu<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.rp, b.col, b.deg, b.L, qn, ctx->d_ctl, level, (int)nxt);
            note_launch(ctx);
        } else if (fedges > 0) {
            k_gather_deg<<<grid_for(fcount, 256, cap), 256, 0, s>>>(q, fcount, b.deg, b.fdeg);
            note_launch(ctx, 2 + scan_u32_to_u64(b.fdeg, b.fpref, fcount, b.scan_tmp, s));
            k_td<<<grid_for((fedges + kTdTile - 1) / kTdTile, 1, cap), kTdThreads, 0, s>>>(
                q, fcount, reinterpret_cast<const unsigned long long *>(b.fpref), b.rp, b.col, b.deg, b.L, qn,
                ctx->d_ctl, level, (int)nxt);
        }
        k_after_level<<<1, 1, 0, s>>>(ctx->d_ctl, (int)nxt, level);
        TC_CUDA(ctx, cudaGetLastError());
        st = pull_ctl(ctx);
        if (st != TC_OK) return st;
        prev_count = fcount;
        fcount = ctx->h_ctl->fr_count[nxt];
        fedges = ctx->h_ctl->fr_edges[nxt];
        slot = nxt;
        queue ^= 1u;
        ++level;
    }
    return TC_OK;
}

tc_status selftest_barrier(tc_ctx *ctx, uint32_t timeout_ms) {
    cudaStream_t s = ctx->stream;
    TC_CUDA(ctx, cudaMemsetAsync(ctx->d_ctl, 0, sizeof(Ctl), s));
    Ctl *ctl = ctx->d_ctl;
    long long cycles = (long long)timeout_ms * 2000000ll;  // clock64 ticks at about 2 GHz
    void *args[] = {&ctl, &cycles};
    TC_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(ctx->num_sms), dim3(64), args, 0, s));
    tc_status st = pull_ctl(ctx);
    if (st != TC_OK) return st;
    if (ctx->h_ctl->error == 4) return set_error(ctx, TC_ERR_TIMEOUT, "device wait timed out (self-test)");
    return set_error(ctx, TC_ERR_CUDA, "self-test barrier did not time out");
}

tc_status given_levels(tc_ctx *ctx, const PipeBufs &b, uint32_t n, const uint32_t *levels_in) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    if (n == 0) return TC_OK;
    k_given_levels<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.rp, b.col, levels_in, b.deg, b.L, ctx->d_ctl);
    note_launch(ctx);
    TC_CUDA(ctx, cudaGetLastError());
    tc_status st = pull_ctl(ctx);
    if (st != TC_OK) return st;
    if (ctx->h_ctl->error & 0x200u)
        return set_error(ctx, TC_ERR_INVALID, "given levels differ by more than one across an edge");
    return TC_OK;
}

tc_status compute_levels(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    if (n == 0) return TC_OK;
    k_init<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.rp, b.deg, b.L, ctx->d_ctl, ctx->opt.order);
    k_seed<<<1, 1, 0, s>>>(b.deg, b.L, b.q0, ctx->d_ctl, 0);
    note_launch(ctx, 2);
    TC_CUDA(ctx, cudaGetLastError());
    tc_status st = bfs_loop(ctx, b, n, slots, 0, 0, 0);
    if (st != TC_OK) return st;
    if (ctx->h_ctl->visited >= n) return TC_OK;

    // Remaining components: min-key roots by hooking, then a multi-source BFS.
    k_collect_unvisited<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.L, b.R, ctx->d_ctl);
    note_launch(ctx);
    st = pull_ctl(ctx);
    if (st != TC_OK) return st;
    const uint32_t nr = ctx->h_ctl->n_residual;
    if (nr == 0) return TC_OK;
    k_cc_init<<<grid_for(nr, 256, cap), 256, 0, s>>>(b.R, nr, b.parent);
    note_launch(ctx);
    for (int round = 0;; ++round) {
        TC_CUDA(ctx, cudaMemsetAsync(&ctx->d_ctl->changed, 0, sizeof(unsigned), s));
        k_cc_hook<<<grid_for(nr, 256, cap), 256, 0, s>>>(b.R, nr, n, b.rp, b.col, b.deg, b.parent, ctx->d_ctl,
                                                         ctx->opt.order);
        k_cc_compress<<<grid_for(nr, 256, cap), 256, 0, s>>>(b.R, nr, n, b.parent, ctx->d_ctl);
        note_launch(ctx, 2);
        TC_CUDA(ctx, cudaGetLastError());
        st = pull_ctl(ctx);
        if (st != TC_OK) return st;
        if (ctx->h_ctl->error) return set_error(ctx, TC_ERR_INVALID, "connected-components walk did not end");
        if (!ctx->h_ctl->changed) break;
        if (round > 64) return set_error(ctx, TC_ERR_TIMEOUT, "connected components did not converge");
    }
    k_reset_next<<<1, 1, 0, s>>>(ctx->d_ctl, 0);
    k_cc_roots<<<grid_for(nr, 256, cap), 256, 0, s>>>(b.R, nr, b.parent, b.deg, b.L, b.q0, ctx->d_ctl, 0);
    k_count_roots<<<1, 1, 0, s>>>(ctx->d_ctl, 0);
    note_launch(ctx, 3);
    TC_CUDA(ctx, cudaGetLastError());
    return bfs_loop(ctx, b, n, slots, 0, 0, 0);
}

}  // namespace tc
