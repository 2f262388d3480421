// tc_internal.cuh -- internal types and device helpers of libtc (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tc.h"

namespace tc {

constexpr uint32_t kUnvisited = 0xFFFFFFFFu;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// ----------------------------------------------------------------------------- tuning
// Class boundaries of the intersection stage by the size s(u) = |A(u)| +
// |G1(u)| of the hashed set of the earlier endpoint u of a horizontal edge.
struct Tuning {
    uint32_t warp_cap = 768;         // s(u) <= warp_cap: warp tasks, per-warp smem table
    uint32_t block_cap = 13107;      // s(u) <= block_cap: block tasks, smem table; larger: hub tasks
    uint32_t task_work = 4194304;    // target probes per block task (at least 2 s(u))
    uint32_t warps_per_block = 8;    // warp-class kernel: warps per block
    uint32_t block_threads = 1024;   // block-class kernel threads
    uint32_t warp_task_work = 65536; // target probes per warp task
    uint32_t hub_task_work = 2097152; // target probes per hub task
    uint32_t max_v = 2048;           // out-neighbours per block / hub task (shared-memory metadata)
    uint32_t hub_group = 32;         // hub rows sharing one launch (one L2-resident bitmap each)
    uint32_t hub_threads = 1024;     // hub kernel threads
    uint32_t hub_filter_log2 = 20;   // hub prefilter bits (log2)
    uint32_t tiny_cap = 16;          // s(u) <= tiny_cap and deg(u) <= 4 tiny_cap: thread-per-row merges (0: off)
    uint32_t table_kind = 0;         // warp/block-class sets: 0 two-choice cuckoo tables, 1 bucketed tables
    uint32_t flat_cap = 128;         // warp class: probe ranges shorter than this are concatenated across lanes
    uint32_t block_bits_log2 = 20;   // block class (cuckoo): ranks below 2^k in a shared bitmap (0: off)
    uint32_t batch_small_slots = 0;  // batches: graphs this small counted a block each in one launch (0: off)
};

// Control block in device memory: counters the kernels update and the host
// reads back between launches.
struct Ctl {
    unsigned long long root_key;     // smallest working-order key among non-isolated vertices
    unsigned long long t_same;       // triangles wholly inside G0
    unsigned long long t_cross;      // triangles with one horizontal edge
    unsigned long long e0;           // |E0|
    unsigned long long probes;       // probed elements
    unsigned long long cls_probes[4];   // per intersection class (warp, block, hub, tiny)
    unsigned long long cls_build[4];    // hashed-row elements per class (each row once)
    unsigned long long cls_rows[4];     // tasks (warp, block, hub) / rows (tiny) per class
    unsigned long long cls_inserts[4];  // table / prefilter inserts actually done (rebuilds included)
    unsigned long long fr_edges[3];  // sum of degrees per frontier slot
    unsigned long long visited_edges;
    unsigned int fr_count[3];        // frontier sizes per slot (slots rotate in the persistent BFS)
    unsigned int visited;            // vertices with a level
    unsigned int max_level;
    unsigned int components;         // BFS roots
    unsigned int changed;            // CC hooking made progress
    unsigned int n_residual;
    unsigned int n_rows[4];          // rows per intersection class (warp, block, hub, tiny)
    unsigned int task_next[4];       // dynamic scheduling counters per class (3: odd hub groups)
    unsigned long long n_tasks[3];   // tasks per class
    unsigned int error;              // nonzero: a device-side check failed
    unsigned int max_s2;             // largest hashed row among block-class rows / max degree
    unsigned int p_slot, p_queue, p_level;  // where the persistent BFS stopped
    unsigned int bar_count, bar_spare;      // arrivals at the persistent BFS's grid barriers (this launch)
    unsigned int n_big;              // rows whose A part the block sorter sorts
    unsigned int n_huge;             // rows of very high degree filled by a block each
    unsigned int n_part;             // rows whose level-spanning part k_g1_split splits
    unsigned int fill_next;          // k_row_fill: next chunk of 32 vertices a warp takes
    unsigned int huge_next;          // k_row_fill_huge: next listed row a block takes
    unsigned int sort_next;          // k_sort_big: next listed row a block takes
    unsigned int split_next;         // k_g1_split: next listed row a block takes
    unsigned int pad[2];
    unsigned long long list_cursor;  // listing: next free chunk position
};

// ----------------------------------------------------------------------------- arena
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    void reset() { off = 0; }
    template <class T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        T *p = reinterpret_cast<T *>(base + off);
        off += bytes;
        return p;
    }
};

}  // namespace tc

struct tc_graph {
    tc_ctx *ctx;
    uint32_t n;
    uint64_t slots;    // row_ptr[n] = 2m
    uint64_t *rp;      // device
    uint32_t *col;     // device
    uint32_t max_deg;
    bool owned;
    bool pooled = false;  // rp/col come from the context's graph pool (stream-ordered free)
};

struct ServeState;  // serve.cu

struct tc_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    tc_options opt{};
    tc::Tuning tune{};
    tc::Arena arena;
    tc::Arena batch_arena;   // union CSR of tc_count_batch
    cudaMemPool_t graph_pool = nullptr;  // graph arrays: freed memory stays in the pool for the next graph
    tc::Ctl *d_ctl = nullptr;
    tc::Ctl *h_ctl = nullptr;   // pinned
    cudaEvent_t ev[10] = {};
    cudaStream_t side_stream = nullptr;  // hub groups of odd index, beside `stream` (made on first use)
    cudaEvent_t side_ev[2] = {};         // fork and join of the side stream
    uint32_t launches = 0;    // kernels launched on this context so far (a call reports its own difference)
    uint32_t isect_flags = 0; // which intersection kernels the last count launched (1 warp, 2 block, 4 hub)
    uint32_t shard = 0, nshards = 1;  // intersection tasks of this count: share `shard` of `nshards`
    uint32_t split_R = 0;             // this count's split rank (block-class bitmap; 0: none)
    uint64_t alloc_calls = 0;         // device allocations made by this context
    uint64_t fail_alloc_at = 0;       // fault injection: fail this allocation (1-based; 0 = never)
    std::string err;
    ServeState *serve = nullptr;
};

namespace tc {

// ----------------------------------------------------------------------------- host helpers
tc_status set_error(tc_ctx *ctx, tc_status st, const std::string &msg);
tc_status cuda_error(tc_ctx *ctx, cudaError_t e, const char *what);
tc_status arena_reserve(tc_ctx *ctx, size_t bytes);
// cudaMalloc through the context (counts calls; honours the injected failure).
cudaError_t device_alloc(tc_ctx *ctx, void **p, size_t bytes);
// Graph arrays: from the context's memory pool, stream-ordered on its stream
// (plain cudaMalloc when the pool could not be made); *pooled says which.
cudaError_t graph_alloc(tc_ctx *ctx, void **p, size_t bytes, bool *pooled);
void graph_free(tc_ctx *ctx, void *p, bool pooled);

// Launch bookkeeping: every kernel launch site calls this once per launch.
inline void note_launch(tc_ctx *ctx, uint32_t k = 1) { ctx->launches += k; }

#define TC_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return tc::cuda_error((ctx), _e, #call); \
    } while (0)

// Exclusive scan of `count` uint32 values into uint64 out[count + 1]
// (out[count] = total).  tmp needs scan_tmp_elems(count) uint64 entries.
// Returns the number of kernels launched.
size_t scan_tmp_elems(uint64_t count);
uint32_t scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t count, uint64_t *tmp, cudaStream_t s);
// Same for uint64 inputs.
uint32_t scan_u64(const uint64_t *in, uint64_t *out, uint64_t count, uint64_t *tmp, cudaStream_t s);

// Stable LSD radix sort of `count` 64-bit keys over the 8-bit digits starting
// at shifts[0..nshifts) (least significant first); *cur holds the keys and on
// return the sorted keys (the two buffers are swapped once per pass).  counts
// needs 256 * radix_tiles(count) + 1 entries, coffs two more, tmp
// scan_tmp_elems(256 * radix_tiles(count) + 1).  Returns the kernels launched.
uint64_t radix_tiles(uint64_t count);
uint32_t radix_sort_u64(unsigned long long **cur, unsigned long long **alt, uint64_t count, const int *shifts,
                        int nshifts, uint32_t *counts, uint64_t *coffs, uint64_t *tmp, cudaStream_t s);

// Pipeline entry (count.cu).  levels_out: device uint32[n] or nullptr.
// group_of / n_groups / group_counts: optional per-group accumulation
// (batched counting of a disjoint union): group_vertex_start is a device
// uint32[n_groups + 1] of first vertex ids, group_counts a device uint64[n_groups].
struct GroupSpec {
    const uint32_t *vertex_start = nullptr;
    uint32_t n_groups = 0;
    unsigned long long *counts = nullptr;
};
struct GraphView {
    uint32_t n = 0;
    uint64_t slots = 0;
    const uint64_t *rp = nullptr;
    const uint32_t *col = nullptr;
    uint32_t max_deg = 0;
};
// Triangle listing: room for `capacity` triples at `out` (device).
struct ListSpec {
    uint32_t *out = nullptr;
    uint64_t capacity = 0;
};
tc_status count_pipeline(tc_ctx *ctx, const GraphView &g, uint32_t *levels_out, const GroupSpec &groups,
                         uint64_t *triangles, tc_stats *stats, const uint32_t *levels_in = nullptr,
                         uint64_t *vertex_counts = nullptr, const ListSpec *list = nullptr, bool alg3 = false);
size_t pipeline_bytes(const tc_ctx *ctx, uint32_t n, uint64_t slots, uint32_t max_deg, bool own_levels, bool plain,
                      uint64_t *hub_words, uint32_t *hub_maps);

// CSR construction / validation (csr.cu)
tc_status build_csr_device(tc_ctx *ctx, uint32_t n, uint64_t t, const uint32_t *d_src,
                           const uint32_t *d_dst, uint64_t **rp_out, uint32_t **col_out,
                           uint64_t *slots_out, bool *pooled_out);
tc_status validate_csr_device(tc_ctx *ctx, uint32_t n, const uint64_t *rp, const uint32_t *col,
                              uint64_t slots, int *ok);
tc_status max_degree_device(tc_ctx *ctx, uint32_t n, const uint64_t *rp, uint32_t *max_deg);
// Batched counting of G graphs as one disjoint union (batch.cu).
tc_status count_batch(tc_ctx *ctx, uint32_t G, const tc_graph *const *graphs, uint64_t *counts);

// Shared-memory bytes of the intersection kernels under a tuning (isect.cu)
size_t warp_kernel_smem(const Tuning &tu);
size_t block_kernel_smem(const Tuning &tu);
size_t hub_kernel_smem(const Tuning &tu);

// Serving (serve.cu)
void serve_shutdown(tc_ctx *ctx);

// ----------------------------------------------------------------------------- device helpers
#ifdef __CUDACC__
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Working-order key: smaller key = earlier vertex.  Degree order (BaderD):
// decreasing degree, ties by ascending id.  Id order (Bader): the id.
__device__ __forceinline__ unsigned long long order_key(uint32_t v, uint32_t deg, uint32_t order) {
    return order == TC_ORDER_DEGREE ? ((unsigned long long)(0xFFFFFFFFu - deg) << 32) | v
                                    : (unsigned long long)v;
}

// x precedes y in the working order
__device__ __forceinline__ bool precedes(uint32_t x, uint32_t dx, uint32_t y, uint32_t dy, uint32_t order) {
    if (order == TC_ORDER_DEGREE) return dx > dy || (dx == dy && x < y);
    return x < y;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Append `pred` items to a global list with one atomic per warp (all lanes of
// the warp must call it).  Returns this lane's slot (valid where pred).
__device__ __forceinline__ uint32_t warp_append(bool pred, unsigned int *counter) {
    unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    uint32_t base = 0;
    if (mask) {
        unsigned leader = __ffs(mask) - 1;
        if (lane_id() == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
    }
    return base + __popc(mask & ((1u << lane_id()) - 1u));
}

// Knuth multiplicative hashing: the top log2(table size) bits of w * 2654435761
// (shift = 32 - log2(table size), table size >= 2).
__device__ __forceinline__ uint32_t hash_slot(uint32_t w, uint32_t shift) {
    return (w * 2654435761u) >> shift;
}
#endif

}  // namespace tc
