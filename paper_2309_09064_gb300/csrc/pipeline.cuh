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
    // intersection planning
    uint32_t *wlist = nullptr;      // [n]   warp-class rows u
    uint32_t *blist = nullptr;      // [n]   block-class rows u
    uint32_t *ntask = nullptr;      // [n]   tasks per block-class row
    uint64_t *tpref = nullptr;      // [n+1] exclusive prefix of ntask
    uint32_t *hub_tables = nullptr; // global tables for rows too large for shared memory
    uint64_t hub_slots = 0;         // slots per hub table
    uint32_t hub_blocks = 0;        // number of hub tables
    uint64_t *scan_tmp = nullptr;
    // batched counting of a disjoint union
    GroupSpec groups;
};

tc_status compute_levels(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint64_t slots);
tc_status build_rows(tc_ctx *ctx, const PipeBufs &b, uint32_t n);
tc_status intersect(tc_ctx *ctx, PipeBufs &b, uint32_t n);

}  // namespace tc
