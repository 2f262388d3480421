// pipeline.cuh -- device buffers and stage entry points of one count.
#pragma once

#include "tc_internal.cuh"

namespace tc {

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
    // partition / orientation / compaction
    uint32_t *hcnt = nullptr;       // [n]   |G0 out-list(x)|
    uint32_t *scnt = nullptr;       // [n]   |G0 out-list(x)| + |G1(x)|
    uint64_t *off2 = nullptr;       // [n+1] offsets of the compacted rows
    uint32_t *adj2 = nullptr;       // [S]   rows [G0 out-list | G1 list], each part ascending
    // intersection planning, per class c (0 warp, 1 block, 2 hub)
    uint32_t *rows[4] = {};         // [n]   rows u of class c (0 warp, 1 block, 2 hub, 3 tiny)
    uint32_t *ntask[3] = {};        // [n]   tasks per row
    uint64_t *tpref[3] = {};        // [n+1] exclusive prefix of ntask
    uint2 *tasks[3] = {};           // {row index i, slice t} per task (carved after planning)
    uint2 *task_pool = nullptr;     // capacity task_cap
    uint64_t task_cap = 0;
    uint32_t *hub_bits = nullptr;   // hub_group bitmaps of hub_words words each
    uint64_t hub_words = 0;
    uint64_t *scan_tmp = nullptr;
    // batched counting of a disjoint union
    GroupSpec groups;
};

tc_status compute_levels(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots);
tc_status selftest_barrier(tc_ctx *ctx, uint32_t timeout_ms);
// partition, orientation, compaction, classification and per-class task counts
tc_status build_rows(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint32_t max_deg);
// scans of the per-class task counts (after the host has read the row counts)
tc_status plan_scans(tc_ctx *ctx, const PipeBufs &b);
// task emission (after the host knows the task totals)
tc_status emit_tasks(tc_ctx *ctx, PipeBufs &b);
tc_status intersect(tc_ctx *ctx, PipeBufs &b, uint32_t n);

}  // namespace tc
