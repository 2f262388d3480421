// pipeline.cuh -- device buffers and stage entry points of one count.
#pragma once

#include "tc_internal.cuh"

namespace tc {

// Listing: output slots a warp takes at a time (see isect.cu).
constexpr uint32_t kListChunk = 2048;

// All scratch of one count, carved from the context arena.  Sizes: n vertices,
// S = row_ptr[n] CSR slots.
struct PipeBufs {
    // input (read-only)
    const uint64_t *rp = nullptr;   // [n+1]
    const uint32_t *col = nullptr;  // [S]
    // levels stage
    uint32_t *deg = nullptr;        // [n]   degrees
    uint32_t *L = nullptr;          // [n]   BFS levels
    uint32_t *q0 = nullptr;         // [n]   frontier queues
    uint32_t *q1 = nullptr;         // [n]
    uint32_t *fdeg = nullptr;       // [n]   frontier degrees
    uint64_t *fpref = nullptr;      // [n+1] their exclusive prefix
    uint32_t *R = nullptr;          // [n]   unvisited vertices after the first BFS
    uint32_t *parent = nullptr;     // [n]   hooking forest
    // ranks (position in the working order)
    uint32_t *rank = nullptr;       // [n]   (degree order only; the id order uses the id)
    uint2 *lv = nullptr;            // [n]   {rank, level}
    uint32_t *lvp = nullptr;        // [n]   rank << 8 | level (only when n <= 2^24 and levels < 255)
    unsigned long long *rkeys0 = nullptr, *rkeys1 = nullptr;  // [n] radix-sort keys
    const unsigned long long *order = nullptr;  // [n] the sorted keys: the vertex of rank i in their low half
                                                //       (null under the id order: rank = id)
    uint32_t *rcounts = nullptr;    // radix digit counts per tile
    uint64_t *roffs = nullptr;      // their scan
    // partition / orientation / rows: every vertex keeps its CSR slots
    // [rp[x], rp[x+1]) rewritten as [ F(x) | A(x) | G1(x) ]
    uint32_t *fcnt = nullptr;       // [n]   |F(x)|  horizontal out-neighbours (ids)
    uint32_t *gcnt = nullptr;       // [n]   |G1(x)| level-spanning neighbours (ranks)
    uint32_t *adj2 = nullptr;       // [S]   the rewritten rows; A(x) (ranks) is descending
    uint32_t *fence = nullptr;      // [S/32] every 32nd slot of adj2 (searches in long A parts)
    uint64_t slots = 0;             // S
    uint32_t *big = nullptr;        // [n]   rows whose A part the block sorter sorts
    uint32_t *huge = nullptr;       // [n]   rows of very high degree (filled by a block each)
    uint4 *vmeta = nullptr;         // [n]   {A start lo, A start hi, |A(x)|, |G1(x)|}
    uint32_t *glo = nullptr;        // [n]   ranks of G1(x) below the split rank, placed first (kNoSplit: not split)
    uint32_t *part = nullptr;       // [n]   rows whose G1 part k_g1_split splits
    uint32_t *chunk_row = nullptr;  // first row of every chunk of kRecChunk probe records
    uint64_t *eoff = nullptr;       // [n+1] exclusive prefix of fcnt: first probe record of x
    uint4 *erec = nullptr;          // [|E0|] probe record per oriented horizontal edge u -> v:
                                    //        {start lo, start hi, length, split}
    uint64_t erec_cap = 0;
    // intersection planning, per class c (0 warp, 1 block, 2 hub)
    uint32_t *rows[4] = {};         // [n]   rows u of class c (0 warp, 1 block, 2 hub, 3 tiny)
    uint32_t *ntask[3] = {};        // [n]   tasks per row
    uint64_t *tpref[3] = {};        // [n+1] exclusive prefix of ntask
    uint2 *tasks[3] = {};           // {row index i, slice t} per task (carved after planning)
    uint2 *task_pool = nullptr;     // capacity task_cap
    uint64_t task_cap = 0;
    uint32_t *hub_bits = nullptr;   // hub_group bitmaps of hub_words words each (indexed by rank)
    uint64_t hub_words = 0;
    uint32_t hub_sets = 1;          // 2: two groups' bitmaps, hub groups alternate between two streams
    uint64_t *scan_tmp = nullptr;
    // batched counting of a disjoint union
    GroupSpec groups;
    // per-vertex triangle counts (tc_count_vertices): by id (the caller's
    // array) and by rank (scratch); null otherwise
    unsigned long long *vcount = nullptr;
    unsigned long long *vcount_rank = nullptr;
    // listing (tc_list_triangles).  Phase 1: the tiny class counts and
    // records its rows' hits (hits), the other classes write their triangles
    // into chunks; phase 2: the tiny class writes at tiny_base + its scanned
    // offsets.  Triple positions run through list_out (list_cap triples),
    // then the overflow area (ovf_cap triples).
    int list_phase = 0;
    unsigned long long *hits = nullptr;       // [rows of the tiny class + 1]
    uint32_t *list_out = nullptr;
    unsigned long long list_cap = 0;
    uint32_t *ovf = nullptr;
    unsigned long long ovf_cap = 0;
    uint32_t *fills = nullptr;                // [nch] filled slots per chunk
    unsigned long long nch = 0;
    ulonglong2 *wstate = nullptr;             // [wstate_len] open chunk of every warp
    unsigned long long wstate_len = 0;
    unsigned long long tiny_base = 0;
    uint32_t *inv = nullptr;                  // [n] rank -> id (null under the id order)
};

// Ranks below this value are kept in the block class's shared bitmap, and
// the rows stage puts them first in every level-spanning part (0: no split).
// A count uses it for the plain count only (ctx->split_R); the per-vertex
// counts and the listing keep their shared memory for their own staging.
inline uint32_t g1_split_rank(const Tuning &tu) {
    return (tu.table_kind == 0 && tu.block_bits_log2) ? (1u << tu.block_bits_log2) : 0u;
}
constexpr uint32_t kNoSplit = 0xFFFFFFFFu;  // glo[x]: G1(x) was not split
// Out-edges per hub task: with a split rank the hub kernel's shared memory also
// holds the low-rank bitmap, so its tasks take at most 1024 records to leave
// room for a larger prefilter (the planner and the kernel use the same value).
inline uint32_t hub_max_v(const Tuning &tu, uint32_t R) { return (R && tu.max_v > 1024) ? 1024u : tu.max_v; }
constexpr size_t kSmemLimitBytes = 227 * 1024;  // shared memory one block may opt into on sm_103a
// Cuckoo slots per table of the block class and the most ranks at or above
// R one block-class set may hold (R = 0: no split, the whole set).
uint32_t block_units_for(const Tuning &tu, uint32_t R);
uint32_t block_hi_cap(const Tuning &tu, uint32_t R);

// Batched form, one thread block per graph (graphs.cu): graphs of at most
// kSmallN vertices and max_slots CSR slots.
constexpr uint32_t kSmallN = 65536;
bool small_graph_fits(const tc_graph *g, uint64_t max_slots);
// Scratch bytes for G such graphs of at most nmax vertices and smax slots;
// *blocks gets the grid.
size_t small_graphs_bytes(const tc_ctx *ctx, uint32_t nmax, uint64_t smax, uint32_t G, uint32_t *blocks);
// Count graphs[i], i in idx, into d_counts[i] (device) on the context's
// stream, one launch, no synchronisation.
tc_status count_small_graphs(tc_ctx *ctx, const tc_graph *const *graphs, const std::vector<uint32_t> &idx,
                             unsigned long long *d_counts, char *scratch, size_t scratch_bytes,
                             unsigned int **d_err);

tc_status compute_levels(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots);
// levels supplied by the caller (device uint32[n]): copied into b.L after the
// check that they differ by at most one across every edge (TC_ERR_INVALID if not)
tc_status given_levels(tc_ctx *ctx, const PipeBufs &b, uint32_t n, const uint32_t *levels_in);
tc_status selftest_barrier(tc_ctx *ctx, uint32_t timeout_ms);
// rank of every vertex in the working order, packed with its level (lv)
tc_status compute_ranks(tc_ctx *ctx, PipeBufs &b, uint32_t n, uint32_t max_deg);
// Listing: close the open chunks, then move the triangles written past the
// first t_big positions into the gaps below it (list.cu).  g_end = the chunk
// cursor after the listing pass.
tc_status list_compact(tc_ctx *ctx, const PipeBufs &b, unsigned long long t_big, unsigned long long g_end,
                       unsigned long long *scratch, unsigned long long *scan_tmp);
size_t list_compact_scratch(unsigned long long nch);
// Algorithm 3 over the CSR as given, after the levels and ranks (alg3.cu).
tc_status intersect_alg3(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots);
// partition, orientation, compaction, classification and per-class task counts
tc_status build_rows(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint32_t max_deg);
// scans of the per-class task counts (after the host has read the row counts)
tc_status plan_scans(tc_ctx *ctx, const PipeBufs &b);
// task emission (after the host knows the task totals)
tc_status emit_tasks(tc_ctx *ctx, PipeBufs &b);
// a count split into shards: the probe records of this shard's tasks only
tc_status records_for_shard(tc_ctx *ctx, const PipeBufs &b);
tc_status intersect(tc_ctx *ctx, PipeBufs &b, uint32_t n);

}  // namespace tc
