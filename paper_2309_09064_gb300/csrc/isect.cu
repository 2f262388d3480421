// isect.cu -- hashed intersections over every oriented horizontal edge
// u -> v (Algorithm 4 with Algorithm 2 on G0), and the reduction of the
// counts into 64-bit totals.
//
// As in the paper's hashed loops, u (the endpoint that comes first in the
// working order, the higher-degree one under the degree order) is put in a
// set once -- its A(u) and G1(u), as ranks -- and for every v in F(u) the
// range of v's slots that k_plan recorded is probed against it: the elements
// of A(v) ranked below u (Algorithm 2's intersection A(u) & A(v) at edge
// (u, v): a triangle inside G0, found once, at the edge between its two later
// vertices) and all of G1(v) (Algorithm 4's hashed loop: a triangle with
// exactly one horizontal edge, found once, at that edge).  A common element
// of G1(u) and A(v) or of A(u) and G1(v) is impossible (different levels), so
// one set and one probe range serve both counts; the position of a hit in the
// range (below or above the record's split) says which kind it is.
//
// Rows are split by the size s(u) = |A(u)| + |G1(u)| of the set, and every
// row's out-edges are cut into tasks (contiguous slices of F(u)) of bounded
// probe work:
//   warp class  s(u) <= warp_cap : one warp per task, bucketed hash table in
//                                  the warp's slice of shared memory;
//   block class s(u) <= block_cap: one block per task, bucketed hash table in
//                                  shared memory;
//   hub class   larger           : hub rows are taken `hub_group` at a time,
//                                  each gets an n-bit bitmap (by rank) in
//                                  global memory (L2-resident while its group
//                                  runs); a block keeps a shared-memory
//                                  prefilter of its set so that only
//                                  prefilter-positive probes read the bitmap;
//   tiny class  s(u) <= tiny_cap (|G1(u)| <= 8) : one thread per row, sorted merges / scans.
// Within a task, warps take probe ranges dynamically and walk each range
// with every lane holding several independent loads.  A block keeps its table
// (or prefilter) when its next task belongs to the same row.
#include <algorithm>

#include "pipeline.cuh"

namespace tc {
namespace {


struct Acc {
    unsigned long long same = 0, cross = 0, probes = 0;
};

// What the kernels do with the triangles they find, besides counting them
// (template parameter kM of the kernels):
//   kM = 1, per-vertex counts (tc_count_vertices): every triangle adds one to
//     each of its three vertices -- the hashed vertex u and the probed vertex
//     v by id (tid), the third vertex w by rank (trank, the value found in the
//     probe range; mapped back to ids after the count);
//   kM = 2, listing (tc_list_triangles): every triangle is written as
//     (u, v, w) in vertex ids.  The warp, block and hub classes write in one
//     pass into chunks of kListChunk slots that every warp takes from a global
//     cursor as it fills them (a compaction after the pass closes the gaps
//     the last, partly filled chunks leave); the tiny class writes at exact
//     offsets (off: the scan of its rows' hits, recorded in task_hits by an
//     earlier counting launch), after the others.
struct VertexOut {
    unsigned long long *tid = nullptr;
    unsigned long long *trank = nullptr;
    unsigned long long *priv = nullptr;        // shared: block-private counts of the ranks below kPrivRanks
    uint32_t *out = nullptr;                   // listing: triples, room for cap of them
    unsigned long long cap = 0;
    uint32_t *ovf = nullptr;                   // listing: overflow triples (positions cap .. cap + ovf_cap)
    unsigned long long ovf_cap = 0;
    unsigned long long *cursor = nullptr;      // listing: next free chunk position
    uint32_t *fills = nullptr;                 // listing: filled slots of every full chunk (nch chunks)
    unsigned long long nch = 0;
    ulonglong2 *wstate = nullptr;              // listing: open chunk {next position, room} of every warp
    unsigned long long wstate_len = 0;
    unsigned int *err = nullptr;
    const uint32_t *inv = nullptr;             // listing: rank -> id (null: ranks are ids)
    const unsigned long long *off = nullptr;   // listing, tiny class: output offset of every row
    unsigned long long base = 0;               // listing, tiny class: where the tiny triangles start
    unsigned long long *task_hits = nullptr;   // tiny counting launch of a listing: hits of every row
};

constexpr unsigned kGuardList = 0x400u;  // a listing write fell outside its room

// Where triple position p lives: the caller's buffer, then the overflow
// area; null past both (the caller's capacity was too small).
__device__ __forceinline__ uint32_t *triple_at(const VertexOut &vo, unsigned long long p) {
    if (p < vo.cap) return vo.out + 3 * p;
    p -= vo.cap;
    return p < vo.ovf_cap ? vo.ovf + 3 * p : nullptr;
}

__device__ __forceinline__ void put_triple(const VertexOut &vo, unsigned long long p, uint32_t u, uint32_t v,
                                           uint32_t w) {
    uint32_t *t = triple_at(vo, p);
    if (!t) {
        atomicOr(vo.err, kGuardList);
        return;
    }
    t[0] = u;
    t[1] = v;
    t[2] = vo.inv ? vo.inv[w] : w;
}

// Listing state of one warp (all lanes hold the same values): its open
// chunk -- next free position and the slots left in it (0: none) -- and the
// vertices of the current range; or, for one thread of the tiny class, its
// exact slots [base, end) and cursor.
struct ListCtx {
    unsigned long long pos = 0;
    uint32_t room = 0;
    uint32_t u = 0, v = 0;
    uint32_t *stage = nullptr;  // the warp's shared staging area (kStageSlots ids, then as many vertices)
    unsigned long long base = 0, end = 0;
    uint32_t local = 0;
};

// Hits of one warp step staged in shared memory before they are written:
// at most 32 lanes x 8 unrolled elements.
constexpr uint32_t kStageSlots = 256;

__device__ __forceinline__ void load_list_state(const VertexOut &vo, ListCtx &lc, unsigned long long gw) {
    if (gw < vo.wstate_len) {
        const ulonglong2 st = vo.wstate[gw];
        lc.pos = st.x;
        lc.room = (uint32_t)st.y;
    } else {
        atomicOr(vo.err, kGuardList);
    }
}

__device__ __forceinline__ void store_list_state(const VertexOut &vo, const ListCtx &lc, unsigned long long gw) {
    if (lane_id() == 0 && gw < vo.wstate_len) vo.wstate[gw] = make_ulonglong2(lc.pos, lc.room);
}

// One triangle (u, v, third vertex by rank w) at the thread's own cursor
// (one thread per row: the tiny class).
__device__ __forceinline__ void emit_one(const VertexOut &vo, ListCtx &lc, uint32_t w) {
    const unsigned long long o = lc.base + lc.local++;
    if (o >= lc.end) {
        atomicOr(vo.err, kGuardList);
        return;
    }
    put_triple(vo, o, lc.u, lc.v, w);
}

// Write the hits of one warp step, element-major: the hits of element i of
// all lanes are consecutive, one ballot per element placing them.  With a
// stage (block and hub classes) the lanes first put them in shared memory,
// then write them out with every lane busy, consecutive lanes writing
// consecutive rows; without one (the warp class, whose steps come from
// short ranges) each lane writes its own.  They go to the rest of the warp's
// open chunk and, past its end, to a new chunk taken from the global cursor
// (a step never fills a whole chunk); a chunk that fills up records its
// fill.  With kPerElemV the probed vertex differs per element (vr[i], the
// concatenated path); otherwise it is lc.v.
template <int U, bool kPerElemV, bool kStage>
__device__ __forceinline__ void emit_step(const bool (&hit)[U], const uint32_t (&w)[U], const uint32_t (&vr)[U],
                                          const VertexOut &vo, ListCtx &lc) {
    static_assert(32 * U <= kStageSlots, "a warp step must fit in the stage");
    static_assert(32 * U < kListChunk, "a warp step must fit in one fresh chunk");
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;  // lanes before this one
    unsigned m[U];
    uint32_t total = 0;
#pragma unroll
    for (int i = 0; i < U; ++i) {
        m[i] = __ballot_sync(0xFFFFFFFFu, hit[i]);
        total += __popc(m[i]);
    }
    if (total == 0) return;
    if (!kStage && total <= lc.room && lc.pos + lc.room <= vo.cap) {
        // no stage (the warp class): each lane writes its own hits
        uint32_t *dst = vo.out + 3 * lc.pos;
        uint32_t k = 0;
#pragma unroll
        for (int i = 0; i < U; ++i) {
            if (hit[i]) {
                uint32_t *t = dst + 3 * (k + __popc(m[i] & below));
                t[0] = lc.u;
                t[1] = kPerElemV ? vr[i] : lc.v;
                t[2] = vo.inv ? vo.inv[w[i]] : w[i];
            }
            k += __popc(m[i]);
        }
        lc.pos += total;
        lc.room -= total;
        if (lc.room == 0) {
            if (lane == 0) {
                const unsigned long long id = lc.pos / kListChunk - 1;
                if (id < vo.nch) vo.fills[id] = kListChunk;
            }
            lc.pos = 0;
        }
        return;
    }
    if (!kStage) {  // rare (a chunk boundary, the overflow area): one position at a time
        unsigned long long fresh = 0;
        if (total > lc.room) {
            if (lane == 0) fresh = atomicAdd(vo.cursor, (unsigned long long)kListChunk);
            fresh = __shfl_sync(0xFFFFFFFFu, fresh, 0);
        }
        uint32_t k = 0;
#pragma unroll
        for (int i = 0; i < U; ++i) {
            if (hit[i]) {
                const uint32_t kk = k + __popc(m[i] & below);
                put_triple(vo, kk < lc.room ? lc.pos + kk : fresh + (kk - lc.room), lc.u, kPerElemV ? vr[i] : lc.v,
                           w[i]);
            }
            k += __popc(m[i]);
        }
        if (total < lc.room) {
            lc.pos += total;
            lc.room -= total;
        } else {
            if (lc.room && lane == 0) {
                const unsigned long long id = (lc.pos + lc.room) / kListChunk - 1;
                if (id < vo.nch) vo.fills[id] = kListChunk;
            }
            const uint32_t spill = total - lc.room;
            lc.pos = spill ? fresh + spill : 0;
            lc.room = spill ? kListChunk - spill : 0;
        }
        return;
    }
    uint32_t k = 0;
#pragma unroll
    for (int i = 0; i < U; ++i) {
        if (hit[i]) {
            const uint32_t kk = k + __popc(m[i] & below);
            lc.stage[kk] = w[i];
            if constexpr (kPerElemV) lc.stage[kStageSlots + kk] = vr[i];
        }
        k += __popc(m[i]);
    }
    __syncwarp();
    if (total <= lc.room && lc.pos + lc.room <= vo.cap) {  // the open chunk takes it, in the caller's buffer
        uint32_t *dst = vo.out + 3 * lc.pos;
        for (uint32_t j = lane; j < total; j += 32) {
            const uint32_t x = lc.stage[j];
            uint32_t *t = dst + 3 * j;
            t[0] = lc.u;
            t[1] = kPerElemV ? lc.stage[kStageSlots + j] : lc.v;
            t[2] = vo.inv ? vo.inv[x] : x;
        }
    } else {
        unsigned long long fresh = 0;
        if (total > lc.room) {
            if (lane == 0) fresh = atomicAdd(vo.cursor, (unsigned long long)kListChunk);
            fresh = __shfl_sync(0xFFFFFFFFu, fresh, 0);
        }
        for (uint32_t j = lane; j < total; j += 32)
            put_triple(vo, j < lc.room ? lc.pos + j : fresh + (j - lc.room), lc.u,
                       kPerElemV ? lc.stage[kStageSlots + j] : lc.v, lc.stage[j]);
        if (total < lc.room) {
            lc.pos += total;
            lc.room -= total;
        } else {
            if (lc.room && lane == 0) {  // the open chunk is full
                const unsigned long long id = (lc.pos + lc.room) / kListChunk - 1;
                if (id < vo.nch) vo.fills[id] = kListChunk;
            }
            const uint32_t spill = total - lc.room;
            lc.pos = spill ? fresh + spill : 0;
            lc.room = spill ? kListChunk - spill : 0;
        }
        __syncwarp();
        return;
    }
    __syncwarp();  // the stage is read before the next step refills it
    if (total < lc.room) {
        lc.pos += total;
        lc.room -= total;
    } else {  // total == room: the open chunk is full
        if (lane == 0) {
            const unsigned long long id = (lc.pos + lc.room) / kListChunk - 1;
            if (id < vo.nch) vo.fills[id] = kListChunk;
        }
        lc.pos = 0;
        lc.room = 0;
    }
}

// The highest-ranked vertices (the largest degrees) close the most
// triangles; their counts are kept per block in shared memory and added to
// trank once per block, so the global atomics on them do not serialise.
constexpr uint32_t kPrivRanks = 1024;

__device__ __forceinline__ void credit_rank(const VertexOut &vo, uint32_t w) {
    if (w < kPrivRanks) atomicAdd(vo.priv + w, 1ull);
    else atomicAdd(vo.trank + w, 1ull);
}

template <int U>
__device__ __forceinline__ void credit_third(const bool (&hit)[U], const uint32_t (&w)[U], const VertexOut &vo) {
#pragma unroll
    for (int i = 0; i < U; ++i)
        if (hit[i]) credit_rank(vo, w[i]);
}

// Zero the block-private counts (all threads; ends with a barrier) / add them
// to the global ones (all threads; starts with a barrier).
__device__ __forceinline__ void priv_begin(const VertexOut &vo) {
    for (uint32_t i = threadIdx.x; i < kPrivRanks; i += blockDim.x) vo.priv[i] = 0;
    __syncthreads();
}
__device__ __forceinline__ void priv_end(const VertexOut &vo) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kPrivRanks; i += blockDim.x)
        if (vo.priv[i]) atomicAdd(vo.trank + i, vo.priv[i]);
}

// ---------------------------------------------------------------------------- set representations

// Bucketed open addressing: buckets of four 32-bit slots read with one 128-bit
// shared load, linear probing over buckets.  Inserts fill a bucket's slots in
// order (each insert tries slot 0, 1, 2, 3 with compare-and-swap), so a bucket
// whose last slot is empty ends every probe sequence that reaches it: a key
// sits in the first bucket, from its home, that had room when it was inserted.
struct BucketTable {
    static constexpr int kUnroll = 8;  // ids in flight per lane
    static constexpr int kBatch = 4;   // lookups resolved together
    static constexpr uint32_t kPad = kEmpty;  // probe padding (lookups reject it)
    static constexpr bool kFineTail = false;
    uint4 *bk;
    uint32_t shift, mask;  // home bucket = hash >> shift; mask = buckets - 1
    unsigned int *err;     // device error word: a walk longer than the table sets kGuardTable
};

// Guard codes OR-ed into the control block's error word when a loop whose
// length depends on the data runs past its bound (the loop then stops and
// the count reports an error instead of spinning).
constexpr unsigned kGuardInsert = 0x10u;    // table insert found no free slot
constexpr unsigned kGuardTable = 0x20u;     // table probe walked the whole table
constexpr unsigned kGuardWalk = 0x40u;      // concatenated ranges walked past the last range
constexpr unsigned kGuardWatchdog = 0x80u;  // a kernel ran past its time limit
constexpr long long kWatchdogCycles = 20000000000ll;  // about 10 s of SM clock

// Buckets for len keys: at most `cap` buckets, at least len / 2 (load factor
// <= 1/2), preferably len (load factor <= 1/4); a power of two >= 16.
__device__ __forceinline__ uint32_t buckets_for(uint32_t len, uint32_t cap) {
    uint32_t nb = 16;
    while (nb < len && nb < cap) nb <<= 1;
    return nb;
}

__device__ __forceinline__ BucketTable clear_table(uint4 *bk, uint32_t len, uint32_t cap, uint32_t t,
                                                   uint32_t nthreads, unsigned int *err) {
    const uint32_t nb = buckets_for(len, cap);
    BucketTable T{bk, (uint32_t)__clz(nb) + 1u, nb - 1u, err};
    const uint4 e = make_uint4(kEmpty, kEmpty, kEmpty, kEmpty);
    for (uint32_t j = t; j < nb; j += nthreads) bk[j] = e;
    return T;
}

__device__ __forceinline__ void table_insert(const BucketTable &T, uint32_t w) {
    uint32_t b = hash_slot(w, T.shift);
    for (uint32_t step = 0; step <= T.mask; ++step) {
        uint32_t *s = reinterpret_cast<uint32_t *>(T.bk + b);
        if (atomicCAS(s + 0, kEmpty, w) == kEmpty || atomicCAS(s + 1, kEmpty, w) == kEmpty ||
            atomicCAS(s + 2, kEmpty, w) == kEmpty || atomicCAS(s + 3, kEmpty, w) == kEmpty)
            return;
        b = (b + 1) & T.mask;
    }
    atomicOr(T.err, kGuardInsert);
}

__device__ __forceinline__ void fill_table(const BucketTable &T, const uint32_t *__restrict__ row, uint32_t len,
                                           uint32_t t, uint32_t nthreads) {
    for (uint32_t j = t; j < len; j += nthreads) table_insert(T, row[j]);
}

// Continue the probe sequence of w past its full home bucket (rare).
__device__ __forceinline__ bool table_find_rest(const BucketTable &T, uint32_t home, uint32_t w) {
    uint32_t bb = home;
    for (uint32_t step = 0; step < T.mask; ++step) {
        bb = (bb + 1) & T.mask;
        const uint4 r = T.bk[bb];
        if (r.x == w || r.y == w || r.z == w || r.w == w) return true;
        if (r.w == kEmpty) return false;
    }
    atomicOr(T.err, kGuardTable);
    return false;
}

// One multiplicative hash into 2^k bits (fshift = 32 - k): the shared filters
// of the block and hub classes.
__device__ __forceinline__ uint32_t filter_bit(uint32_t w, uint32_t fshift) { return (w * 0x85EBCA6Bu) >> fshift; }

__device__ __forceinline__ bool filter_test(const uint32_t *filter, uint32_t w, uint32_t fshift) {
    const uint32_t f = filter_bit(w, fshift);
    return (filter[f >> 5] >> (f & 31)) & 1u;
}

// Block rows: two-choice cuckoo hashing.  Every key sits in T0[h0(w)] or in
// T1[h1(w)] (one 32-bit slot each; h = top bits of w times an odd
// multiplier), so a lookup is two independent 32-bit shared loads and two
// compares, with no branch.  The tables hold at most 0.4 keys per slot; a key
// that finds no place after kCuckooIters displacements goes to a small
// stash, which lookups read only when it is not empty (a block-wide
// condition).  If the stash overflows, the table is rebuilt with the next
// pair of multipliers.
constexpr uint32_t kNone = 0xFFFFFFFEu;  // probe padding: never a rank (n <= 2^32 - 2), never stored
constexpr int kCuckooIters = 64;
constexpr uint32_t kStash = 64;
constexpr int kCuckooAttempts = 4;
__device__ __constant__ uint32_t kCuckooMul[2 * kCuckooAttempts] = {
    0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu, 0x165667B1u, 0xD3A2646Du, 0xFD7046C5u, 0xB55A4F09u};

struct CuckooTable {
    static constexpr int kUnroll = 8;
    static constexpr int kBatch = 8;
    static constexpr uint32_t kPad = kNone;
    static constexpr bool kFineTail = false;
    uint32_t *t;            // 2m slots: T0 = t[0, m), T1 = t[m, 2m)
    const uint32_t *stash;  // shared, nstash entries
    uint32_t m, shift;      // m slots per table, shift = 32 - log2 m
    uint32_t k0, k1;        // multipliers of this build
    uint32_t nstash;
    uint32_t a0, a1;        // shared-window byte addresses of T0 and T1 (lookups use 32-bit addressing)
};

// 32-bit load from the shared window at byte address addr.
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint32_t shared_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 32-bit load from the shared window at byte address addr when p holds;
// otherwise `other` (no shared-memory access: the lane takes no part in it).
__device__ __forceinline__ uint32_t lds_u32_if(bool p, uint32_t addr, uint32_t other) {
    uint32_t v = other;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.shared.u32 %0, [%1];\n\t}"
        : "+r"(v)
        : "r"(addr), "r"((uint32_t)p));
    return v;
}

// Block rows with a split set: the ranks of the set below R sit in a direct
// bitmap (bit w of R / 32 shared words), the others in the cuckoo table.
// The probed ids are mostly low ranks (high-degree vertices appear in many
// rows), so most lookups read one bitmap word -- one shared load, and lanes
// whose ranks share a word read it together -- instead of two random table
// slots.  The rows stage puts the low ranks of every level-spanning part
// first, so a warp step mostly lies wholly below R (bitmap only) or wholly
// above it (table only); a step that straddles R does both, lane by lane.
struct SplitSet {
    static constexpr int kUnroll = 8;
    static constexpr int kBatch = 8;
    static constexpr uint32_t kPad = kNone;  // probe padding: a "low" lane in the vote, never a hit
    static constexpr bool kFineTail = false;
    CuckooTable C;  // ranks >= R
    uint32_t bm;    // shared-window byte address of the bitmap
    uint32_t R;     // ranks below R are in the bitmap (a power of two, or 0: none)
};

// The bitmap part of a split set alone: probe pieces whose ids are all below
// R (the low part of a range the rows stage split) need one shared load per
// id.  Tail steps clamp the padding's word index and reject it.
struct BitmapSet {
    static constexpr int kUnroll = 8;
    static constexpr int kBatch = 8;
    static constexpr uint32_t kPad = kNone;
    static constexpr bool kFineTail = false;
    uint32_t bm;  // shared-window byte address of the bitmap
    uint32_t R;   // its size in bits
};

// Hub rows: shared prefilter (2^hub_filter_log2 bits) in front of the exact
// n-bit bitmap (by rank) in global memory.
struct HubSet {
    static constexpr int kUnroll = 8;  // ids in flight per lane
    static constexpr int kBatch = 8;   // prefilter tests, then all bitmap loads together
    static constexpr uint32_t kPad = kEmpty;  // probe padding (lookups reject it)
    static constexpr bool kFineTail = true;   // bitmap lookups go to L2: skip padding work
    const uint32_t *filter;  // shared
    const uint32_t *bits;    // global, read-only while probing
    uint32_t fshift;
};

// A hub set split at R: ids below R in the shared low bitmap, the others
// behind the prefilter (which then holds only the set's ids >= R) in the L2
// bitmap.  For probe pieces of ranges whose split is unknown.
struct HubMixSet {
    static constexpr int kUnroll = 4;  // rare pieces: fewer registers held
    static constexpr int kBatch = 4;
    static constexpr uint32_t kPad = kEmpty;
    static constexpr bool kFineTail = true;
    HubSet H;
    uint32_t bm;  // shared-window byte address of the low bitmap
    uint32_t R;
};

// Probe one batch of N elements against the bucket table: first buckets for
// all, then the rare continuation for those whose home bucket was full.
template <int N>
__device__ __forceinline__ void lookup_batch(const BucketTable &T, const uint32_t (&w)[N], bool (&hit)[N]) {
    uint4 q[N];
    uint32_t home[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        home[i] = hash_slot(w[i], T.shift);
        q[i] = T.bk[home[i]];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        hit[i] = q[i].x == w[i] || q[i].y == w[i] || q[i].z == w[i] || q[i].w == w[i];
        if (!hit[i] && q[i].w != kEmpty && w[i] != kEmpty) hit[i] = table_find_rest(T, home[i], w[i]);
        hit[i] = hit[i] && w[i] != kEmpty;
    }
}

// Both candidate slots of all N elements, then the compares; the stash only
// when it is not empty.
template <int N>
__device__ __forceinline__ void lookup_batch(const CuckooTable &C, const uint32_t (&w)[N], bool (&hit)[N]) {
    uint32_t a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        a[i] = lds_u32(C.a0 + (((w[i] * C.k0) >> C.shift) << 2));
        b[i] = lds_u32(C.a1 + (((w[i] * C.k1) >> C.shift) << 2));
    }
#pragma unroll
    for (int i = 0; i < N; ++i) hit[i] = a[i] == w[i] || b[i] == w[i];
    if (C.nstash) {
        for (uint32_t k = 0; k < C.nstash; ++k) {
            const uint32_t x = C.stash[k];
#pragma unroll
            for (int i = 0; i < N; ++i) hit[i] = hit[i] || x == w[i];
        }
    }
}

// Prefilter for all N elements, then the exact bitmap word for the positive
// ones (predicated loads, all in flight together).
template <int N>
__device__ __forceinline__ void lookup_batch(const HubSet &H, const uint32_t (&w)[N], bool (&hit)[N]) {
    bool pos[N];
#pragma unroll
    for (int i = 0; i < N; ++i) pos[i] = w[i] != kEmpty && filter_test(H.filter, w[i], H.fshift);
    uint32_t word[N];
#pragma unroll
    for (int i = 0; i < N; ++i) word[i] = pos[i] ? __ldg(H.bits + (w[i] >> 5)) : 0u;
#pragma unroll
    for (int i = 0; i < N; ++i) hit[i] = pos[i] && ((word[i] >> (w[i] & 31)) & 1u);
}

template <int N>
__device__ __forceinline__ void lookup_batch(const HubMixSet &M, const uint32_t (&w)[N], bool (&hit)[N]) {
    bool lo[N], pos[N];
    uint32_t x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        lo[i] = w[i] < M.R;
        const uint32_t f = filter_bit(w[i], M.H.fshift);
        // low ids read their bitmap word, the others their prefilter word
        x[i] = lds_u32(lo[i] ? M.bm + ((w[i] >> 5) << 2) : shared_addr(M.H.filter) + ((f >> 5) << 2));
        pos[i] = !lo[i] && w[i] != kEmpty && ((x[i] >> (f & 31u)) & 1u);
    }
    uint32_t word[N];
#pragma unroll
    for (int i = 0; i < N; ++i) word[i] = pos[i] ? __ldg(M.H.bits + (w[i] >> 5)) : 0u;
#pragma unroll
    for (int i = 0; i < N; ++i)
        hit[i] = lo[i] ? ((x[i] >> (w[i] & 31u)) & 1u) != 0u : (pos[i] && ((word[i] >> (w[i] & 31u)) & 1u));
}

// ---------------------------------------------------------------------------- probing

// Count the hits of one step of U x 32 positions starting at j0 into same /
// cross: the split (end of the A part) is the same for the whole warp, and
// most steps lie wholly on one side of it.
template <int U>
__device__ __forceinline__ void count_step(const bool (&hit)[U], uint32_t j0, uint32_t split, uint32_t lane,
                                           uint32_t &same, uint32_t &cross) {
    uint32_t c = 0;
    if (j0 + 32u * U <= split) {
#pragma unroll
        for (int i = 0; i < U; ++i) c += hit[i];
        same += c;
    } else if (j0 >= split) {
#pragma unroll
        for (int i = 0; i < U; ++i) c += hit[i];
        cross += c;
    } else {
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const bool in_a = j0 + (uint32_t)i * 32u + lane < split;
            same += hit[i] && in_a;
            cross += hit[i] && !in_a;
        }
    }
}

template <int U, bool kTail = false, class Set>
__device__ __forceinline__ void lookup_step(const Set &set, const uint32_t (&w)[U], bool (&hit)[U]) {
    constexpr int B = Set::kBatch < U ? Set::kBatch : U;
    static_assert(U % B == 0, "the unroll must be a multiple of the lookup batch");
#pragma unroll
    for (int half = 0; half < U; half += B) {
        uint32_t ww[B];
        bool hh[B];
#pragma unroll
        for (int i = 0; i < B; ++i) ww[i] = w[half + i];
        lookup_batch(set, ww, hh);
#pragma unroll
        for (int i = 0; i < B; ++i) hit[half + i] = hh[i];
    }
}

// One warp step against a split set: a vote picks the bitmap alone (every
// lane's ids below R, padding included), the table alone (every id at or
// above R), or both, lane by lane.  The stash holds only ranks >= R.
template <int U, bool kTail = false>
__device__ __forceinline__ void lookup_step(const BitmapSet &B, const uint32_t (&w)[U], bool (&hit)[U]) {
    uint32_t x[U];
    if constexpr (kTail) {
#pragma unroll
        for (int i = 0; i < U; ++i) x[i] = lds_u32(B.bm + (((w[i] < B.R ? w[i] : 0u) >> 5) << 2));
#pragma unroll
        for (int i = 0; i < U; ++i) hit[i] = w[i] < B.R && ((x[i] >> (w[i] & 31u)) & 1u);
    } else {
#pragma unroll
        for (int i = 0; i < U; ++i) x[i] = lds_u32(B.bm + ((w[i] >> 5) << 2));
#pragma unroll
        for (int i = 0; i < U; ++i) hit[i] = (x[i] >> (w[i] & 31u)) & 1u;
    }
}

template <int U, bool kTail = false>
__device__ __forceinline__ void lookup_step(const SplitSet &S, const uint32_t (&w)[U], bool (&hit)[U]) {
    bool lo_all = true, hi_all = true;
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const bool lo = w[i] < S.R;
        lo_all = lo_all && (lo || w[i] == SplitSet::kPad);
        hi_all = hi_all && !lo;
    }
    lo_all = __all_sync(0xFFFFFFFFu, lo_all);
    hi_all = __all_sync(0xFFFFFFFFu, hi_all);
    if (lo_all) {
        uint32_t x[U];
#pragma unroll
        for (int i = 0; i < U; ++i) x[i] = lds_u32(S.bm + (((w[i] < S.R ? w[i] : 0u) >> 5) << 2));
#pragma unroll
        for (int i = 0; i < U; ++i) hit[i] = w[i] < S.R && ((x[i] >> (w[i] & 31u)) & 1u);
        return;
    }
    if (hi_all) {
        lookup_step<U>(S.C, w, hit);
        return;
    }
    uint32_t a[U], c[U];
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const bool lo = w[i] < S.R;
        a[i] = lds_u32(lo ? S.bm + ((w[i] >> 5) << 2) : S.C.a0 + (((w[i] * S.C.k0) >> S.C.shift) << 2));
        c[i] = lds_u32_if(!lo, S.C.a1 + (((w[i] * S.C.k1) >> S.C.shift) << 2), kEmpty);
    }
#pragma unroll
    for (int i = 0; i < U; ++i)
        hit[i] = w[i] < S.R ? (((a[i] >> (w[i] & 31u)) & 1u) != 0u) : (a[i] == w[i] || c[i] == w[i]);
    if (S.C.nstash) {
        for (uint32_t k = 0; k < S.C.nstash; ++k) {
            const uint32_t x = S.C.stash[k];
#pragma unroll
            for (int i = 0; i < U; ++i) hit[i] = hit[i] || x == w[i];
        }
    }
}

// Positions [j_lo, j_hi) of one probe range adj2[b ..] with one warp: full
// steps of U x 32 positions (U loads in flight per lane, no bounds checks),
// then the ragged end in one bounds-checked step of U x 32 positions, or in
// steps of 64 positions (kFineTail: pays where lookups are expensive);
// positions below `split` are the A part.
template <int U, bool kFineTail = false, int kM = 0, bool kStage = false, bool kHalfTail = true, class Set>
__device__ __forceinline__ uint32_t probe_row(const Set &set, const uint32_t *__restrict__ adj2, unsigned long long b,
                                              uint32_t j_lo, uint32_t j_hi, uint32_t split, Acc &acc,
                                              const VertexOut &vo = VertexOut{}, ListCtx *lc = nullptr) {
    const unsigned lane = lane_id();
    const uint32_t *row = adj2 + b + lane;
    uint32_t same = 0, cross = 0;
    uint32_t j0 = j_lo;
    for (; j0 + 32u * U <= j_hi; j0 += 32u * U) {
        uint32_t w[U];
        bool hit[U];
#pragma unroll
        for (int i = 0; i < U; ++i) w[i] = __ldg(row + j0 + (uint32_t)i * 32u);
        lookup_step<U>(set, w, hit);
        if constexpr (kM == 1) credit_third<U>(hit, w, vo);
        if constexpr (kM == 2) emit_step<U, false, kStage>(hit, w, w, vo, *lc);
        count_step<U>(hit, j0, split, lane, same, cross);
    }
    constexpr int T = kFineTail ? 2 : U;
    constexpr int H = (kHalfTail && T >= 8) ? T / 2 : T;  // a ragged end of at most half a step takes a half step
    constexpr int Q = (kHalfTail && T >= 8) ? T / 4 : T;  // of at most a quarter step, a quarter step
    if (Q < H && j0 < j_hi && j_hi - j0 <= 32u * Q) {
        uint32_t w[Q];
        bool hit[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t j = j0 + (uint32_t)i * 32u;
            w[i] = j + lane < j_hi ? __ldg(row + j) : Set::kPad;
        }
        lookup_step<Q, true>(set, w, hit);
        if constexpr (kM == 1) credit_third<Q>(hit, w, vo);
        if constexpr (kM == 2) emit_step<Q, false, kStage>(hit, w, w, vo, *lc);
        count_step<Q>(hit, j0, split, lane, same, cross);
        j0 = j_hi;
    }
    if (H < T && j0 < j_hi && j_hi - j0 <= 32u * H) {
        uint32_t w[H];
        bool hit[H];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const uint32_t j = j0 + (uint32_t)i * 32u;
            w[i] = j + lane < j_hi ? __ldg(row + j) : Set::kPad;
        }
        lookup_step<H, true>(set, w, hit);
        if constexpr (kM == 1) credit_third<H>(hit, w, vo);
        if constexpr (kM == 2) emit_step<H, false, kStage>(hit, w, w, vo, *lc);
        count_step<H>(hit, j0, split, lane, same, cross);
        j0 = j_hi;
    }
    for (; j0 < j_hi; j0 += 32u * T) {
        uint32_t w[T];
        bool hit[T];
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const uint32_t j = j0 + (uint32_t)i * 32u;
            w[i] = j + lane < j_hi ? __ldg(row + j) : Set::kPad;
        }
        lookup_step<T, true>(set, w, hit);
        if constexpr (kM == 1) credit_third<T>(hit, w, vo);
        if constexpr (kM == 2) emit_step<T, false, kStage>(hit, w, w, vo, *lc);
        count_step<T>(hit, j0, split, lane, same, cross);
    }
    acc.same += same;
    acc.cross += cross;
    return same + cross;  // this lane's hits (the caller credits the probed vertex)
}

// Short probe ranges, concatenated: range r covers positions
// [pre[r], pre[r+1]) of one flat sequence (ranges of length 0 allowed,
// pre[nv] = total), starts at adj2[b[r]] and has its A part below split[r].
// One warp probes positions [q_lo, q_hi) (q_hi <= total) with every lane busy
// however short the ranges are: each lane finds the range of its first
// position by binary search and then walks forward.
template <int U, int kM = 0, class Set>
__device__ __forceinline__ void probe_flat(const Set &set, const uint32_t *__restrict__ adj2,
                                           const unsigned long long *sb, const uint32_t *spre,
                                           const uint32_t *ssplit, const uint32_t *sv, uint32_t nv, uint32_t q_lo,
                                           uint32_t q_hi, Acc &acc, unsigned int *err,
                                           const VertexOut &vo = VertexOut{}, ListCtx *lc = nullptr) {
    const unsigned lane = lane_id();
    const uint32_t q0 = min(q_lo + lane, q_hi - 1);
    uint32_t r = 0, e = nv;  // largest r < nv with pre[r] <= q0
    while (e - r > 1) {
        const uint32_t m = (r + e) >> 1;
        if (spre[m] <= q0) r = m; else e = m;
    }
    uint32_t lo = spre[r], hi = spre[r + 1];
    unsigned long long base = sb[r] - lo;
    uint32_t split = lo + ssplit[r];
    uint32_t same = 0, cross = 0;
    for (uint32_t j0 = q_lo; j0 < q_hi; j0 += 32u * U) {
        uint32_t w[U], vr[U];
        bool in_a[U], hit[U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const uint32_t q = j0 + (uint32_t)i * 32u + lane;
            bool valid = q < q_hi;
            if (valid) {
                while (q >= hi) {
                    if (r + 1 >= nv) {  // past the last range: inconsistent prefix
                        atomicOr(err, kGuardWalk);
                        valid = false;
                        break;
                    }
                    ++r;
                    lo = hi;
                    hi = spre[r + 1];
                    base = sb[r] - lo;
                    split = lo + ssplit[r];
                }
            }
            w[i] = valid ? __ldg(adj2 + base + q) : Set::kPad;
            in_a[i] = q < split;
            if constexpr (kM != 0) vr[i] = sv[r];
        }
        lookup_step<U>(set, w, hit);
        if constexpr (kM == 2) emit_step<U, true, false>(hit, w, vr, vo, *lc);
#pragma unroll
        for (int i = 0; i < U; ++i) {
            same += hit[i] && in_a[i];
            cross += hit[i] && !in_a[i];
            if constexpr (kM == 1) {
                if (hit[i]) {
                    credit_rank(vo, w[i]);
                    atomicAdd(vo.tid + vr[i], 1ull);
                }
            }
        }
    }
    acc.same += same;
    acc.cross += cross;
}

__device__ __forceinline__ uint32_t group_of(const GroupSpec &g, uint32_t u) {
    uint32_t a = 0, b = g.n_groups;
    while (b - a > 1) {
        const uint32_t m = (a + b) >> 1;
        if (g.vertex_start[m] <= u) a = m; else b = m;
    }
    return a;
}

// Reduce a warp's counters into the control block (class c: 0 warp, 1 block, 2 hub, 3 tiny).
__device__ __forceinline__ void flush(const Acc &acc, Ctl *ctl, int c, unsigned long long build_elems,
                                      unsigned long long tasks) {
    const unsigned long long s = warp_sum(acc.same), x = warp_sum(acc.cross), p = warp_sum(acc.probes);
    if (lane_id() == 0) {
        if (s) atomicAdd(&ctl->t_same, s);
        if (x) atomicAdd(&ctl->t_cross, x);
        if (p) {
            atomicAdd(&ctl->probes, p);
            atomicAdd(&ctl->cls_probes[c], p);
        }
        if (build_elems) atomicAdd(&ctl->cls_build[c], build_elems);
        if (tasks) atomicAdd(&ctl->cls_rows[c], tasks);
    }
}

__device__ __forceinline__ unsigned long long rec_start(const uint4 &r) {
    return ((unsigned long long)r.y << 32) | r.x;
}

// Long probe ranges are walked in kSeg pieces, one warp each.  In the warp
// class, ranges shorter than flat_cap (a tuning knob) are concatenated
// (probe_flat) so that every lane has work.
constexpr uint32_t kSeg = 2048;

// Build the cuckoo table of a hashed set row[0..s) (all threads of a block,
// or of a warp, call it): clear 2m slots, insert every key by displacement, stash the keys
// that found no place; rebuild with the next multipliers if the stash
// overflowed.  m = the smallest power of two >= 1.25 s (at most m_cap): at
// most 0.4 keys per slot.
struct CuckooShared {
    uint32_t stash[kStash];
    unsigned int nstash;
};

__device__ __forceinline__ void cuckoo_insert(const CuckooTable &C, uint32_t key, CuckooShared *cs) {
    uint32_t which = 0, pos = (key * C.k0) >> C.shift;
    for (int it = 0; it < kCuckooIters; ++it) {
        const uint32_t old = atomicExch(C.t + which * C.m + pos, key);
        if (old == kEmpty) return;
        key = old;
        which ^= 1u;
        pos = (key * (which ? C.k1 : C.k0)) >> C.shift;
    }
    const unsigned k = atomicAdd(&cs->nstash, 1u);
    if (k < kStash) cs->stash[k] = key;
}

__device__ __forceinline__ uint32_t cuckoo_slots_for(uint32_t s, uint32_t m_cap) {
    uint32_t m = 64;
    while (m < s + s / 4 && m < m_cap) m <<= 1;
    return m;
}

// Block-wide build (all threads of the block call it).  With a bitmap bm of
// R bits (R > 0), keys below R set their bit there instead (the bitmap is
// cleared first) and only the others enter the table.
__device__ __forceinline__ CuckooTable cuckoo_build(uint32_t *t, uint32_t m_cap, const uint32_t *__restrict__ row,
                                                    uint32_t s, CuckooShared *cs, unsigned int *err,
                                                    uint32_t *bm = nullptr, uint32_t R = 0, uint32_t table_keys = 0) {
    const uint32_t m = cuckoo_slots_for(R ? table_keys : s, m_cap);
    CuckooTable C{t, cs->stash, m, (uint32_t)__clz(m) + 1u, 0, 0, 0, shared_addr(t), shared_addr(t + m)};
    for (uint32_t j = threadIdx.x; j < (R >> 5); j += blockDim.x) bm[j] = 0u;
    for (int attempt = 0; attempt < kCuckooAttempts; ++attempt) {
        C.k0 = kCuckooMul[2 * attempt];
        C.k1 = kCuckooMul[2 * attempt + 1];
        for (uint32_t j = threadIdx.x; j < 2 * m; j += blockDim.x) t[j] = kEmpty;
        if (threadIdx.x == 0) cs->nstash = 0;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < s; j += blockDim.x) {
            const uint32_t key = row[j];
            if (key < R) atomicOr(bm + (key >> 5), 1u << (key & 31u));
            else cuckoo_insert(C, key, cs);
        }
        __syncthreads();
        const unsigned ns = cs->nstash;
        __syncthreads();  // everyone has read it before a rebuild clears it
        if (ns <= kStash) {
            C.nstash = ns;
            return C;
        }
    }
    if (threadIdx.x == 0) atomicOr(err, kGuardInsert);  // keys were dropped: the count reports an error
    C.nstash = kStash;
    return C;
}

// Warp-wide build (all lanes of the warp call it).
__device__ __forceinline__ CuckooTable warp_cuckoo_build(uint32_t *t, uint32_t m_cap, const uint32_t *__restrict__ row,
                                                         uint32_t s, CuckooShared *cs, unsigned int *err) {
    const unsigned lane = lane_id();
    const uint32_t m = cuckoo_slots_for(s, m_cap);
    CuckooTable C{t, cs->stash, m, (uint32_t)__clz(m) + 1u, 0, 0, 0, shared_addr(t), shared_addr(t + m)};
    for (int attempt = 0; attempt < kCuckooAttempts; ++attempt) {
        C.k0 = kCuckooMul[2 * attempt];
        C.k1 = kCuckooMul[2 * attempt + 1];
        for (uint32_t j = lane; j < 2 * m; j += 32) t[j] = kEmpty;
        if (lane == 0) cs->nstash = 0;
        __syncwarp();
        for (uint32_t j = lane; j < s; j += 32) cuckoo_insert(C, row[j], cs);
        __syncwarp();
        const unsigned ns = cs->nstash;
        __syncwarp();
        if (ns <= kStash) {
            C.nstash = ns;
            return C;
        }
    }
    if (lane == 0) atomicOr(err, kGuardInsert);
    C.nstash = kStash;
    return C;
}

// ---------------------------------------------------------------------------- warp class

// Per-warp shared metadata of the 32 probe records a warp holds at a time.
struct WarpMeta {
    unsigned long long b[32];
    uint32_t pre[33];
    uint32_t split[32];
    uint32_t v[32];  // probed vertex of each range (per-vertex counts only)
};
constexpr size_t kWarpMetaBytes = (sizeof(WarpMeta) + 15) & ~size_t(15);

// Shared memory of one warp: its set (cuckoo table and stash, or buckets),
// then the metadata of the 32 records it holds.
__host__ __device__ constexpr size_t warp_set_bytes(bool cuckoo, uint32_t units) {
    return cuckoo ? ((8ull * units + sizeof(CuckooShared) + 15) & ~15ull) : 16ull * units;
}

template <bool kCuckoo, int kM>
__global__ void __launch_bounds__(256, 3) k_isect_warp(const uint2 *__restrict__ tasks, const uint32_t *__restrict__ rows,
                                                     const uint32_t *__restrict__ ntask,
                                                     const uint64_t *__restrict__ rp,
                                                     const uint32_t *__restrict__ adj2,
                                                     const uint32_t *__restrict__ fcnt,
                                                     const uint64_t *__restrict__ eoff,
                                                     const uint4 *__restrict__ erec, Ctl *ctl, uint32_t table_units,
                                                     uint32_t flat_cap, unsigned long long first,
                                                     unsigned long long last, GroupSpec groups, VertexOut vo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const size_t set_bytes = warp_set_bytes(kCuckoo, table_units);
    unsigned char *mine = smem_raw + (size_t)warp * (set_bytes + kWarpMetaBytes);
    WarpMeta *meta = reinterpret_cast<WarpMeta *>(mine + set_bytes);
    CuckooShared *cs = reinterpret_cast<CuckooShared *>(mine + 8ull * table_units);
    Acc acc;
    unsigned long long build = 0, done = 0, inserts = 0;
    uint32_t cur_row = 0xFFFFFFFFu;
    BucketTable T{reinterpret_cast<uint4 *>(mine), 0, 0, &ctl->error};
    CuckooTable C{reinterpret_cast<uint32_t *>(mine), cs->stash, 64, 26, 0, 0, 0, 0, 0};
    if constexpr (kM == 1) {
        vo.priv = reinterpret_cast<unsigned long long *>(smem_raw + (size_t)(blockDim.x >> 5) *
                                                                         (set_bytes + kWarpMetaBytes));
        priv_begin(vo);
    }
    ListCtx lc;
    const unsigned long long gw = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if constexpr (kM == 2) load_list_state(vo, lc, gw);  // no stage: lanes write their own hits
    const long long t_start = clock64();
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) {
            k = first + atomicAdd(&ctl->task_next[0], 1u);
            if (clock64() - t_start > kWatchdogCycles) {
                atomicOr(&ctl->error, kGuardWatchdog);
                k = last;
            }
        }
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= last) break;
        const uint2 task = tasks[k];
        const uint32_t u = rows[task.x], nt = ntask[task.x];
        const uint32_t fu = fcnt[u];
        const uint64_t hb = rp[u] + fu;
        const uint32_t su = (uint32_t)(rp[u + 1] - hb);
        const uint4 *rec = erec + eoff[u];
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * fu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * fu / nt);
        lc.u = u;
        if (task.x != cur_row) {  // tasks of one row reuse its table
            __syncwarp();
            if constexpr (kCuckoo) {
                C = warp_cuckoo_build(C.t, table_units, adj2 + hb, su, cs, &ctl->error);
            } else {
                T = clear_table(T.bk, su, table_units, lane, 32, &ctl->error);
                __syncwarp();
                fill_table(T, adj2 + hb, su, lane, 32);
                __syncwarp();
            }
            cur_row = task.x;
            inserts += su;
        }
        if (task.y == 0) build += su + fu;
        ++done;
        const unsigned long long before = acc.same + acc.cross;
        for (uint32_t k0 = k_lo; k0 < k_hi; k0 += 32) {
            const uint32_t kk = k0 + lane;
            uint4 r = make_uint4(0, 0, 0, 0);
            uint32_t vid = 0;
            if (kk < k_hi) {
                r = rec[kk];
                if constexpr (kM != 0) vid = adj2[hb - fu + kk];
            }
            acc.probes += r.z;
            const unsigned long long b = rec_start(r);
            // long ranges: the whole warp on each in turn
            const bool longr = r.z >= flat_cap;
            unsigned lm = __ballot_sync(0xFFFFFFFFu, longr);
            while (lm) {
                const int t = __ffs(lm) - 1;
                lm &= lm - 1;
                const unsigned long long bt = __shfl_sync(0xFFFFFFFFu, b, t);
                const uint32_t lt = __shfl_sync(0xFFFFFFFFu, r.z, t);
                const uint32_t ht = __shfl_sync(0xFFFFFFFFu, r.w, t);
                uint32_t got;
                if constexpr (kM == 2) lc.v = __shfl_sync(0xFFFFFFFFu, vid, t);
                if constexpr (kCuckoo)
                    got = probe_row<CuckooTable::kUnroll, false, kM, false, false>(C, adj2, bt, 0, lt, ht, acc, vo, &lc);
                else
                    got = probe_row<BucketTable::kUnroll, false, kM, false, false>(T, adj2, bt, 0, lt, ht, acc, vo, &lc);
                if constexpr (kM == 1) {
                    got = warp_sum(got);
                    const uint32_t vt = __shfl_sync(0xFFFFFFFFu, vid, t);
                    if (lane == 0 && got) atomicAdd(vo.tid + vt, (unsigned long long)got);
                }
            }
            // short ranges: concatenated
            const uint32_t sl = longr ? 0u : r.z;
            uint32_t incl = sl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= (unsigned)o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (total) {
                meta->b[lane] = b;
                meta->pre[lane] = incl - sl;
                meta->split[lane] = r.w;
                meta->v[lane] = vid;
                if (lane == 31) meta->pre[32] = total;
                __syncwarp();
                if constexpr (kCuckoo)
                    probe_flat<CuckooTable::kUnroll, kM>(C, adj2, meta->b, meta->pre, meta->split, meta->v, 32, 0,
                                                         total, acc, &ctl->error, vo, &lc);
                else
                    probe_flat<BucketTable::kUnroll, kM>(T, adj2, meta->b, meta->pre, meta->split, meta->v, 32, 0,
                                                         total, acc, &ctl->error, vo, &lc);
                __syncwarp();
            }
        }
        if (groups.n_groups || kM == 1) {
            const unsigned long long found = warp_sum(acc.same + acc.cross - before);
            if (lane == 0 && found) {
                if (groups.n_groups) atomicAdd(&groups.counts[group_of(groups, u)], found);
                if constexpr (kM == 1) atomicAdd(vo.tid + u, found);
            }
        }
    }
    flush(acc, ctl, 0, lane == 0 ? build : 0, lane == 0 ? done : 0);
    if (lane == 0 && inserts) atomicAdd(&ctl->cls_inserts[0], inserts);
    if constexpr (kM == 1) priv_end(vo);
    if constexpr (kM == 2) store_list_state(vo, lc, gw);
}

// ---------------------------------------------------------------------------- tiny class

// Size of the intersection of a[0..na) (shared, column `stride` apart) and
// b[0..nb) (global), both descending: two-pointer merge.
template <int kM>
__device__ __forceinline__ uint32_t merge_count_desc(const uint32_t *a, uint32_t stride, uint32_t na,
                                                     const uint32_t *__restrict__ b, uint32_t nb,
                                                     const VertexOut &vo, ListCtx &lc) {
    uint32_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        const uint32_t x = a[i * stride], y = __ldg(b + j);
        c += x == y;
        if constexpr (kM == 1)
            if (x == y) credit_rank(vo, y);
        if constexpr (kM == 2)
            if (x == y) emit_one(vo, lc, y);
        i += x >= y;
        j += y >= x;
    }
    return c;
}

// Size of the intersection of a[0..na) (shared, column `stride` apart) and
// b[0..nb) (global), in any order: every pair compared (na <= tiny_cap).
template <int kM>
__device__ __forceinline__ uint32_t scan_count(const uint32_t *a, uint32_t stride, uint32_t na,
                                               const uint32_t *__restrict__ b, uint32_t nb, const VertexOut &vo,
                                               ListCtx &lc) {
    uint32_t c = 0;
    for (uint32_t j = 0; j < nb; ++j) {
        const uint32_t y = __ldg(b + j);
        uint32_t cy = 0;
        for (uint32_t i = 0; i < na; ++i) cy += a[i * stride] == y;
        c += cy;
        if constexpr (kM == 1)
            if (cy) credit_rank(vo, y);
        if constexpr (kM == 2)
            if (cy) emit_one(vo, lc, y);
    }
    return c;
}

// Tiny class: one thread per row u (s(u) <= tiny_cap, deg(u) <= 4 tiny_cap,
// so every v in F(u), which comes later in the working order, has at most
// 4 tiny_cap neighbours too; and |G1(u)| <= 8, see k_class_flags).  A(u) and G1(u) are copied to a shared column;
// for every v in F(u) the A parts (both descending) are merged -- only
// elements ranked below u can match, since A(u) holds no other -- and the G1
// parts compared pairwise.
template <int kM>
__global__ void __launch_bounds__(256) k_isect_tiny(const uint32_t *__restrict__ rows, uint32_t lo, uint32_t hi,
                                                    const uint64_t *__restrict__ rp,
                                                    const uint32_t *__restrict__ adj2,
                                                    const uint32_t *__restrict__ fcnt,
                                                    const uint32_t *__restrict__ gcnt, Ctl *ctl, uint32_t tiny_cap,
                                                    GroupSpec groups, VertexOut vo) {
    extern __shared__ uint32_t srow[];  // tiny_cap x blockDim, column per thread
    uint32_t *mine = srow + threadIdx.x;
    const uint32_t stride = blockDim.x;
    if constexpr (kM == 1) {
        vo.priv = reinterpret_cast<unsigned long long *>(srow + (size_t)tiny_cap * blockDim.x);
        priv_begin(vo);
    }
    Acc acc;
    unsigned long long build = 0, done = 0;
    const uint32_t total = (uint32_t)((uint64_t)gridDim.x * blockDim.x);
    for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += total) {
        const uint32_t u = rows[i];
        const uint64_t ub = rp[u];
        const uint32_t fu = fcnt[u], gu = gcnt[u];
        const uint32_t su = (uint32_t)(rp[u + 1] - ub) - fu, au = su - gu;
        for (uint32_t k = 0; k < su; ++k) mine[k * stride] = __ldg(adj2 + ub + fu + k);  // A(u) then G1(u)
        uint32_t same = 0, cross = 0;
        unsigned long long probes = 0;
        ListCtx lc;
        if constexpr (kM == 2) {
            lc.base = vo.base + vo.off[i];
            lc.end = vo.base + vo.off[i + 1];
            lc.u = u;
        }
        for (uint32_t k = 0; k < fu; ++k) {
            const uint32_t v = __ldg(adj2 + ub + k);
            lc.v = v;
            const uint64_t vb = rp[v], ve = rp[v + 1];
            const uint32_t fv = fcnt[v], gv = gcnt[v];
            const uint32_t av = (uint32_t)(ve - vb) - fv - gv;
            const uint32_t sv = merge_count_desc<kM>(mine, stride, au, adj2 + vb + fv, av, vo, lc);
            const uint32_t cv = scan_count<kM>(mine + au * stride, stride, gu, adj2 + (ve - gv), gv, vo, lc);
            same += sv;
            cross += cv;
            if constexpr (kM == 1)
                if (sv + cv) atomicAdd(vo.tid + v, (unsigned long long)(sv + cv));
            probes += av + gv;
        }
        acc.same += same;
        acc.cross += cross;
        acc.probes += probes;
        build += su + fu;
        ++done;
        if (groups.n_groups && same + cross) atomicAdd(&groups.counts[group_of(groups, u)], (unsigned long long)(same + cross));
        if constexpr (kM == 1)
            if (same + cross) atomicAdd(vo.tid + u, (unsigned long long)(same + cross));
        if (vo.task_hits) vo.task_hits[i] = same + cross;
        if constexpr (kM == 2)
            if (lc.base + lc.local != lc.end) atomicOr(vo.err, kGuardList);
    }
    const unsigned long long b = warp_sum(build), d = warp_sum(done);
    flush(acc, ctl, 3, lane_id() == 0 ? b : 0, lane_id() == 0 ? d : 0);
    if constexpr (kM == 1) priv_end(vo);
}

// ---------------------------------------------------------------------------- block and hub classes

// Per-task shared metadata of up to max_v probe records: start, length and
// split of each range, and seg = exclusive prefix of their kSeg-piece counts.
// Warps take pieces one at a time, so no long range holds up the block.
struct SliceSmem {
    unsigned long long *b;
    uint32_t *len, *h, *seg, *v;  // v: probed vertex of each range (per-vertex counts and listing only)
    uint32_t *q;                  // split sets: end of the range's ids below the split rank (kNoSplit: unknown)
};

__device__ __forceinline__ SliceSmem carve_slice(unsigned char *p, uint32_t max_v) {
    SliceSmem s;
    s.b = reinterpret_cast<unsigned long long *>(p);
    s.len = reinterpret_cast<uint32_t *>(p + 8ull * max_v);
    s.h = s.len + max_v;
    s.seg = s.h + max_v;
    s.v = s.seg + max_v + 1;
    s.q = s.v + max_v;
    return s;
}

__host__ __device__ constexpr size_t slice_smem_bytes(uint32_t max_v) { return (28ull * max_v + 4 + 15) & ~15ull; }

// Pieces of one probe range: kSeg positions each; a split range (q known) is
// cut into its low part [0, q) and its high part [q, len) separately.
__device__ __forceinline__ uint32_t range_pieces(uint32_t len, uint32_t q) {
    if (q == kNoSplit) return (len + kSeg - 1) / kSeg;
    return (q + kSeg - 1) / kSeg + (len - q + kSeg - 1) / kSeg;
}

// Block-wide exclusive scan of the piece counts of ranges 0..nv-1 into
// seg[0..nv]; all threads of the block call it; ends with a barrier.
__device__ __forceinline__ void scan_segments(const uint32_t *len, uint32_t *seg, uint32_t nv,
                                              const uint32_t *q = nullptr) {
    __shared__ uint32_t warp_tot[32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t per = (nv + blockDim.x - 1) / blockDim.x;  // ranges per thread (contiguous)
    const uint32_t beg = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (beg + i < nv) sum += q ? range_pieces(len[beg + i], q[beg + i]) : (len[beg + i] + kSeg - 1) / kSeg;
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
        if (beg + i < nv) {
            seg[beg + i] = run;
            run += q ? range_pieces(len[beg + i], q[beg + i]) : (len[beg + i] + kSeg - 1) / kSeg;
        }
    }
    if (threadIdx.x == 0) seg[nv] = warp_tot[nwarps - 1];
    __syncthreads();
}

// Load the probe records of edges k in [k_lo, k_hi) of one row (no barrier),
// and with per-vertex counts or listing the probed vertices (F of the row, at
// frow).
template <int kM, bool kSplit = false>
__device__ __forceinline__ void load_slice(const SliceSmem &S, const uint4 *__restrict__ rec, uint32_t k_lo,
                                           uint32_t k_hi, const uint32_t *__restrict__ frow,
                                           const uint32_t *__restrict__ glo = nullptr, bool tail_lo = false) {
    for (uint32_t i = threadIdx.x; i < k_hi - k_lo; i += blockDim.x) {
        const uint4 r = rec[k_lo + i];
        S.b[i] = rec_start(r);
        S.len[i] = r.z;
        S.h[i] = r.w;
        if constexpr (kM != 0 || kSplit) {
            const uint32_t v = frow[k_lo + i];
            if constexpr (kM != 0) S.v[i] = v;
            if constexpr (kSplit) {
                // the range is [A tail | G1 low | G1 high]: its ids below the split rank
                // end after G1's low part when the A tail (ranks below u's) is low too
                const uint32_t gl = glo[v];
                S.q[i] = (tail_lo && gl != kNoSplit) ? r.w + gl : kNoSplit;
            }
        }
    }
}

// Warps take the slice's pieces in batches of up to 32 (shared counter): the
// lanes of a warp locate the pieces of a batch in parallel (one binary search
// each over seg), then the warp walks them one by one.  The batch shrinks for
// small slices so that every warp of the block still gets work.
template <int kM = 0, class Set>
__device__ __forceinline__ void probe_slice(const Set &set, const SliceSmem &S, uint32_t nv,
                                            const uint32_t *__restrict__ adj2, unsigned int *next, Acc &acc,
                                            const VertexOut &vo, ListCtx &lc) {
    const unsigned lane = lane_id();
    const uint32_t total = S.seg[nv];
    const uint32_t nwarps = blockDim.x >> 5;
    uint32_t batch = total / (4 * nwarps);
    batch = batch < 1 ? 1 : (batch > 32 ? 32 : batch);
    for (;;) {
        uint32_t g0 = 0;
        if (lane == 0) g0 = atomicAdd(next, batch);
        g0 = __shfl_sync(0xFFFFFFFFu, g0, 0);
        if (g0 >= total) break;
        const uint32_t cnt = min(batch, total - g0);
        {   // guided: later grabs take fewer pieces, so the warps finish the task together
            uint32_t nb = (total - g0 - cnt) / (4 * nwarps);
            batch = nb < 1 ? 1 : (nb < batch ? nb : batch);
        }
        unsigned long long b = 0;
        uint32_t j_lo = 0, j_hi = 0, h = 0, vid = 0;
        if (lane < cnt) {
            const uint32_t g = g0 + lane;
            uint32_t a = 0, e = nv;  // range of piece g: largest t with seg[t] <= g
            while (e - a > 1) {
                const uint32_t m = (a + e) >> 1;
                if (S.seg[m] <= g) a = m; else e = m;
            }
            j_lo = (g - S.seg[a]) * kSeg;
            j_hi = min(S.len[a], j_lo + kSeg);
            b = S.b[a];
            h = S.h[a];
            if constexpr (kM != 0) vid = S.v[a];
            acc.probes += j_hi - j_lo;
        }
        for (uint32_t t = 0; t < cnt; ++t) {
            const unsigned long long bt = __shfl_sync(0xFFFFFFFFu, b, t);
            const uint32_t lo = __shfl_sync(0xFFFFFFFFu, j_lo, t);
            const uint32_t hi = __shfl_sync(0xFFFFFFFFu, j_hi, t);
            const uint32_t ht = __shfl_sync(0xFFFFFFFFu, h, t);
            if constexpr (kM == 2) lc.v = __shfl_sync(0xFFFFFFFFu, vid, t);
            uint32_t got = probe_row<Set::kUnroll, Set::kFineTail, kM, true>(set, adj2, bt, lo, hi, ht, acc, vo, &lc);
            if constexpr (kM == 1) {
                got = warp_sum(got);
                const uint32_t vt = __shfl_sync(0xFFFFFFFFu, vid, t);
                if (lane == 0 && got) atomicAdd(vo.tid + vt, (unsigned long long)got);
            }
        }
    }
}

// Ask L2 for the lines of positions [lo, hi) of the range at adj2[b]: one
// 128-byte line per lane (at most 32 lines, i.e. a whole 512-position piece
// with room to spare).  No registers wait on it; the walk's loads then find
// the lines in L2 instead of DRAM.
__device__ __forceinline__ void prefetch_piece(const uint32_t *adj2, unsigned long long b, uint32_t lo, uint32_t hi) {
    const unsigned lane = lane_id();
    const uint32_t *p0 = adj2 + b + lo;
    const uint32_t *line = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(p0) & ~uintptr_t(127)) +
                           32u * lane;
    if (hi > lo && line < adj2 + b + hi) asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
}

// probe_slice for a split set: a piece of a split range lies wholly in its
// low part (bitmap lookups only) or wholly in its high part (cuckoo table
// only); pieces of ranges whose split is unknown take both, lane by lane.
// Low pieces go to `low` (the bitmap), high pieces to `high`, pieces of
// ranges with no known split to `mix` (a set that answers for any id).
template <int kM = 0, bool kPrefetch = false, class LowSet, class HighSet, class MixSet>
__device__ __forceinline__ void probe_slice_split(const LowSet &low, const HighSet &high, const MixSet &mix,
                                                  const SliceSmem &S, uint32_t nv, const uint32_t *__restrict__ adj2,
                                                  unsigned int *next, Acc &acc, const VertexOut &vo, ListCtx &lc) {
    const unsigned lane = lane_id();
    const uint32_t total = S.seg[nv];
    const uint32_t nwarps = blockDim.x >> 5;
    uint32_t batch = total / (4 * nwarps);
    batch = batch < 1 ? 1 : (batch > 32 ? 32 : batch);
    for (;;) {
        uint32_t g0 = 0;
        if (lane == 0) g0 = atomicAdd(next, batch);
        g0 = __shfl_sync(0xFFFFFFFFu, g0, 0);
        if (g0 >= total) break;
        const uint32_t cnt = min(batch, total - g0);
        {   // guided: later grabs take fewer pieces, so the warps finish the task together
            uint32_t nb = (total - g0 - cnt) / (4 * nwarps);
            batch = nb < 1 ? 1 : (nb < batch ? nb : batch);
        }
        unsigned long long b = 0;
        uint32_t j_lo = 0, j_hi = 0, h = 0, vid = 0, kind = 0;  // kind: 0 both, 1 low part, 2 high part
        if (lane < cnt) {
            const uint32_t g = g0 + lane;
            uint32_t a = 0, e = nv;  // range of piece g: largest t with seg[t] <= g
            while (e - a > 1) {
                const uint32_t m = (a + e) >> 1;
                if (S.seg[m] <= g) a = m; else e = m;
            }
            uint32_t l = g - S.seg[a];
            const uint32_t len = S.len[a], q = S.q[a];
            if (q == kNoSplit) {
                j_lo = l * kSeg;
                j_hi = min(len, j_lo + kSeg);
            } else {
                const uint32_t nlo = (q + kSeg - 1) / kSeg;
                if (l < nlo) {
                    j_lo = l * kSeg;
                    j_hi = min(q, j_lo + kSeg);
                    kind = 1;
                } else {
                    l -= nlo;
                    j_lo = q + l * kSeg;
                    j_hi = min(len, j_lo + kSeg);
                    kind = 2;
                }
            }
            b = S.b[a];
            h = S.h[a];
            if constexpr (kM != 0) vid = S.v[a];
            acc.probes += j_hi - j_lo;
        }
        for (uint32_t t = 0; t < cnt; ++t) {
            const unsigned long long bt = __shfl_sync(0xFFFFFFFFu, b, t);
            const uint32_t lo = __shfl_sync(0xFFFFFFFFu, j_lo, t);
            const uint32_t hi = __shfl_sync(0xFFFFFFFFu, j_hi, t);
            const uint32_t ht = __shfl_sync(0xFFFFFFFFu, h, t);
            const uint32_t kt = __shfl_sync(0xFFFFFFFFu, kind, t);
            if constexpr (kPrefetch) {  // the next piece of the batch to L2 while this one is walked
                const uint32_t tn = t + 1 < cnt ? t + 1 : t;
                const unsigned long long bn = __shfl_sync(0xFFFFFFFFu, b, tn);
                const uint32_t ln = __shfl_sync(0xFFFFFFFFu, j_lo, tn), hn = __shfl_sync(0xFFFFFFFFu, j_hi, tn);
                if (t + 1 < cnt) prefetch_piece(adj2, bn, ln, hn);
            }
            if constexpr (kM == 2) lc.v = __shfl_sync(0xFFFFFFFFu, vid, t);
            uint32_t got;
            if (kt == 1)
                got = probe_row<LowSet::kUnroll, LowSet::kFineTail, kM, true>(low, adj2, bt, lo, hi, ht, acc, vo, &lc);
            else if (kt == 2)
                got = probe_row<HighSet::kUnroll, HighSet::kFineTail, kM, true>(high, adj2, bt, lo, hi, ht, acc, vo, &lc);
            else
                got = probe_row<MixSet::kUnroll, MixSet::kFineTail, kM, true>(mix, adj2, bt, lo, hi, ht, acc, vo, &lc);
            if constexpr (kM == 1) {
                got = warp_sum(got);
                const uint32_t vt = __shfl_sync(0xFFFFFFFFu, vid, t);
                if (lane == 0 && got) atomicAdd(vo.tid + vt, (unsigned long long)got);
            }
        }
    }
}

struct TaskSmem {
    uint2 task;
    unsigned int next;
    unsigned int pad;
    unsigned long long found;
    unsigned long long chunk_pos, chunk_end;  // this block's current run of consecutive tasks
};

// Thread 0 takes the next task of class c in [first, last): blocks grab runs
// of `chunk` consecutive tasks, so the tasks of one row mostly stay on one
// block and its table is built once.  All threads see the task.
__device__ __forceinline__ bool next_task(Ctl *ctl, int c, unsigned long long first, unsigned long long last,
                                          unsigned long long chunk, const uint2 *tasks, TaskSmem *ts,
                                          long long t_start) {
    __syncthreads();  // everyone is done with the previous task
    if (threadIdx.x == 0) {
        if (clock64() - t_start > kWatchdogCycles) {
            atomicOr(&ctl->error, kGuardWatchdog);
            ts->task = make_uint2(0xFFFFFFFFu, 0u);
        } else {
            if (ts->chunk_pos >= ts->chunk_end) {
                const unsigned long long k = first + (unsigned long long)atomicAdd(&ctl->task_next[c], 1u) * chunk;
                ts->chunk_pos = k;
                ts->chunk_end = k + chunk < last ? k + chunk : last;
            }
            const unsigned long long k = ts->chunk_pos++;
            ts->task = k < ts->chunk_end ? tasks[k] : make_uint2(0xFFFFFFFFu, 0u);
        }
        ts->next = 0;
        ts->found = 0;
    }
    __syncthreads();
    return ts->task.x != 0xFFFFFFFFu;
}

// End of a block's task: the triangles it found (this thread's share is
// `mine`) go to the group counts and to the hashed vertex's count.
template <int kM>
__device__ __forceinline__ void finish_task(unsigned long long mine, const GroupSpec &groups, const VertexOut &vo,
                                            TaskSmem &ts, uint32_t u) {
    if (groups.n_groups || kM == 1) {
        const unsigned long long found = warp_sum(mine);
        if (lane_id() == 0 && found) atomicAdd(&ts.found, found);
        __syncthreads();
        if (threadIdx.x == 0 && ts.found) {
            if (groups.n_groups) atomicAdd(&groups.counts[group_of(groups, u)], ts.found);
            if constexpr (kM == 1) atomicAdd(vo.tid + u, ts.found);
        }
    }
}

__device__ __forceinline__ void init_task_smem(TaskSmem *ts) {
    if (threadIdx.x == 0) {
        ts->chunk_pos = 0;
        ts->chunk_end = 0;
    }
}

// Block class.  The hashed set lives in shared memory: a cuckoo table
// (kSet = 0), the bucketed table (kSet = 1), or a split set (kSet = 2: ranks
// below split_R in a bitmap placed after the cuckoo table, the rest in it).
template <int kSet, int kM>
__global__ void __launch_bounds__(1024, 1) k_isect_block(const uint2 *__restrict__ tasks, const uint32_t *__restrict__ rows,
                                                      const uint32_t *__restrict__ ntask,
                                                      const uint64_t *__restrict__ rp,
                                                      const uint32_t *__restrict__ adj2,
                                                      const uint32_t *__restrict__ fcnt,
                                                      const uint64_t *__restrict__ eoff,
                                                      const uint4 *__restrict__ erec, Ctl *ctl, uint32_t max_v,
                                                      uint32_t table_units, uint32_t split_R,
                                                      const uint32_t *__restrict__ glo,
                                                      const uint32_t *__restrict__ gcnt,
                                                      const uint2 *__restrict__ lv, unsigned long long chunk,
                                                      unsigned long long first, unsigned long long last,
                                                      GroupSpec groups, VertexOut vo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TaskSmem ts;
    __shared__ CuckooShared cs;
    const unsigned lane = lane_id();
    constexpr bool kCuckoo = kSet != 1;
    const SliceSmem S = carve_slice(smem_raw, max_v);
    unsigned char *tab = smem_raw + slice_smem_bytes(max_v);
    uint32_t *bmp = reinterpret_cast<uint32_t *>(tab + (kCuckoo ? 8ull : 16ull) * table_units);
    unsigned char *after = tab + (kCuckoo ? 8ull : 16ull) * table_units + (kSet == 2 ? split_R / 8 : 0u);
    Acc acc;
    unsigned long long build = 0, done = 0, inserts = 0;
    uint32_t cur_row = 0xFFFFFFFFu;
    CuckooTable C{reinterpret_cast<uint32_t *>(tab), cs.stash, 64, 26, 0, 0, 0, 0, 0};
    BucketTable T{reinterpret_cast<uint4 *>(tab), 0, 0, &ctl->error};
    if constexpr (kM == 1) {
        vo.priv = reinterpret_cast<unsigned long long *>(after);
        priv_begin(vo);
    }
    init_task_smem(&ts);
    ListCtx lc;
    const unsigned long long gw = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if constexpr (kM == 2) {
        lc.stage = reinterpret_cast<uint32_t *>(after) + (size_t)(threadIdx.x >> 5) * kStageSlots;
        load_list_state(vo, lc, gw);
    }
    const long long t_start = clock64();
    while (next_task(ctl, 1, first, last, chunk, tasks, &ts, t_start)) {
        const uint2 task = ts.task;
        const uint32_t u = rows[task.x], nt = ntask[task.x];
        const uint32_t fu = fcnt[u];
        const uint64_t hb = rp[u] + fu;
        const uint32_t su = (uint32_t)(rp[u + 1] - hb);
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * fu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * fu / nt);
        const bool rebuild = task.x != cur_row;
        if constexpr (!kCuckoo)
            if (rebuild) T = clear_table(T.bk, su, table_units, threadIdx.x, blockDim.x, &ctl->error);
        // split set: u's own A part holds ranks below u's, all low when u is ranked below split_R
        const bool tail_lo = kSet == 2 && lv[u].x <= split_R;
        load_slice<kM, kSet == 2>(S, erec + eoff[u], k_lo, k_hi, adj2 + (hb - fu), glo, tail_lo);
        __syncthreads();
        scan_segments(S.len, S.seg, k_hi - k_lo, kSet == 2 ? S.q : nullptr);
        if (rebuild) {
            if constexpr (kSet == 2) {
                const uint32_t g = gcnt[u], gl = glo[u];
                const uint32_t hi_keys = (gl == kNoSplit ? g : g - gl) + (tail_lo ? 0u : su - g);
                C = cuckoo_build(C.t, table_units, adj2 + hb, su, &cs, &ctl->error, bmp, split_R, hi_keys);
            } else if constexpr (kCuckoo) {
                C = cuckoo_build(C.t, table_units, adj2 + hb, su, &cs, &ctl->error);
            } else {
                fill_table(T, adj2 + hb, su, threadIdx.x, blockDim.x);
                __syncthreads();
            }
            cur_row = task.x;
            if (threadIdx.x == 0) inserts += su;
        }
        if (threadIdx.x == 0) {
            if (task.y == 0) build += su + fu;
            ++done;
        }
        const unsigned long long before = acc.same + acc.cross;
        lc.u = u;
        if constexpr (kSet == 2) {
            const SplitSet SS{C, shared_addr(bmp), split_R};
            probe_slice_split<kM>(BitmapSet{SS.bm, split_R}, C, SS, S, k_hi - k_lo, adj2, &ts.next, acc, vo, lc);
        }
        else if constexpr (kCuckoo) probe_slice<kM>(C, S, k_hi - k_lo, adj2, &ts.next, acc, vo, lc);
        else probe_slice<kM>(T, S, k_hi - k_lo, adj2, &ts.next, acc, vo, lc);
        finish_task<kM>(acc.same + acc.cross - before, groups, vo, ts, u);
    }
    flush(acc, ctl, 1, threadIdx.x == 0 ? build : 0, threadIdx.x == 0 ? done : 0);
    if (threadIdx.x == 0 && inserts) atomicAdd(&ctl->cls_inserts[1], inserts);
    if constexpr (kM == 1) priv_end(vo);
    if constexpr (kM == 2) store_list_state(vo, lc, gw);
}

// Set the bits of the hashed sets of hub rows rows[i0 .. i0+g) into bitmaps
// bits + r * words (bit index = rank).
__global__ void k_hub_set(const uint32_t *__restrict__ rows, uint32_t i0, uint32_t g,
                          const uint64_t *__restrict__ rp, const uint32_t *__restrict__ fcnt,
                          const uint32_t *__restrict__ adj2, uint32_t *bits, uint64_t words) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t r = 0; r < g; ++r) {
        const uint32_t u = rows[i0 + r];
        const uint64_t b = rp[u] + fcnt[u], e = rp[u + 1];
        uint32_t *bm = bits + (uint64_t)r * words;
        for (uint64_t j = b + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < e; j += stride) {
            const uint32_t w = adj2[j];
            atomicOr(bm + (w >> 5), 1u << (w & 31));
        }
    }
}

// Probe the tasks [first, last) of the hub rows with row index in
// [i0, i0 + hub_group) against their bitmaps.
// With kSplit (split_R > 0), the ranks of the set below split_R sit in an
// exact shared bitmap after the prefilter, which then holds only the others:
// the low pieces of split probe ranges are answered in shared memory, high
// pieces take the prefilter and the L2 bitmap, pieces of unsplit ranges
// (HubMixSet) either, id by id.
template <int kM, bool kSplit = false>
__global__ void __launch_bounds__(1024, 1) k_isect_hub(const uint2 *__restrict__ tasks, unsigned long long first,
                                                    unsigned long long last, const uint32_t *__restrict__ rows,
                                                    const uint32_t *__restrict__ ntask, uint32_t i0,
                                                    const uint64_t *__restrict__ rp, const uint32_t *__restrict__ adj2,
                                                    const uint32_t *__restrict__ fcnt,
                                                    const uint64_t *__restrict__ eoff, const uint4 *__restrict__ erec,
                                                    Ctl *ctl, const uint32_t *bits, uint64_t words, uint32_t max_v,
                                                    unsigned long long chunk, uint32_t filter_log2, GroupSpec groups,
                                                    VertexOut vo, uint32_t split_R = 0, const uint32_t *__restrict__ glo = nullptr,
                                                    const uint2 *__restrict__ lv = nullptr, int ctr = 2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TaskSmem ts;
    const unsigned lane = lane_id();
    const SliceSmem S = carve_slice(smem_raw, max_v);
    uint32_t *filter = reinterpret_cast<uint32_t *>(smem_raw + slice_smem_bytes(max_v));
    const uint32_t filter_words = 1u << (filter_log2 - 5);
    const uint32_t fshift = 32u - filter_log2;
    uint32_t *lowbm = filter + filter_words;                             // kSplit: split_R bits
    uint32_t *after = lowbm + (kSplit ? (split_R >> 5) : 0u);            // per-vertex counters or listing stage
    if constexpr (kM == 1) {
        vo.priv = reinterpret_cast<unsigned long long *>(after);
        priv_begin(vo);
    }
    Acc acc;
    unsigned long long build = 0, done = 0, inserts = 0;
    uint32_t cur_row = 0xFFFFFFFFu;
    init_task_smem(&ts);
    ListCtx lc;
    const unsigned long long gw = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if constexpr (kM == 2) {
        lc.stage = after + (size_t)(threadIdx.x >> 5) * kStageSlots;
        load_list_state(vo, lc, gw);
    }
    const long long t_start = clock64();
    while (next_task(ctl, ctr, first, last, chunk, tasks, &ts, t_start)) {
        const uint2 task = ts.task;
        const uint32_t u = rows[task.x], nt = ntask[task.x];
        const uint32_t fu = fcnt[u];
        const uint64_t hb = rp[u] + fu;
        const uint32_t su = (uint32_t)(rp[u + 1] - hb);
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * fu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * fu / nt);
        const bool rebuild = task.x != cur_row;
        if (rebuild) {
            for (uint32_t j = threadIdx.x; j < filter_words; j += blockDim.x) filter[j] = 0u;
            if constexpr (kSplit)
                for (uint32_t j = threadIdx.x; j < (split_R >> 5); j += blockDim.x) lowbm[j] = 0u;
        }
        bool tail_lo = false;
        if constexpr (kSplit) tail_lo = lv[u].x <= split_R;
        load_slice<kM, kSplit>(S, erec + eoff[u], k_lo, k_hi, adj2 + (hb - fu), glo, tail_lo);
        __syncthreads();
        scan_segments(S.len, S.seg, k_hi - k_lo, kSplit ? S.q : nullptr);
        if (rebuild) {
            for (uint32_t j = threadIdx.x; j < su; j += blockDim.x) {
                const uint32_t w = adj2[hb + j];
                if (kSplit && w < split_R) {  // low ids: the exact bitmap only
                    atomicOr(lowbm + (w >> 5), 1u << (w & 31u));
                } else {
                    const uint32_t f = filter_bit(w, fshift);
                    atomicOr(filter + (f >> 5), 1u << (f & 31));
                }
            }
            __syncthreads();
            cur_row = task.x;
            if (threadIdx.x == 0) inserts += su;
        }
        if (threadIdx.x == 0) {
            if (task.y == 0) build += su + fu;
            ++done;
        }
        const HubSet H{filter, bits + (uint64_t)(task.x - i0) * words, fshift};
        const unsigned long long before = acc.same + acc.cross;
        lc.u = u;
        if constexpr (kSplit)
            // the hub's probe ranges mostly come from DRAM: their next piece is prefetched into L2
            probe_slice_split<kM, true>(BitmapSet{shared_addr(lowbm), split_R}, H,
                                        HubMixSet{H, shared_addr(lowbm), split_R}, S, k_hi - k_lo, adj2, &ts.next,
                                        acc, vo, lc);
        else
            probe_slice<kM>(H, S, k_hi - k_lo, adj2, &ts.next, acc, vo, lc);
        finish_task<kM>(acc.same + acc.cross - before, groups, vo, ts, u);
    }
    flush(acc, ctl, 2, threadIdx.x == 0 ? build : 0, threadIdx.x == 0 ? done : 0);
    if (threadIdx.x == 0 && inserts) atomicAdd(&ctl->cls_inserts[2], inserts);
    if constexpr (kM == 1) priv_end(vo);
    if constexpr (kM == 2) store_list_state(vo, lc, gw);
}

uint32_t pow2_at_least(uint64_t x, uint32_t lo) {
    uint32_t t = lo;
    while (t < x) t <<= 1;
    return t;
}

}  // namespace

// Shared-memory sets of the warp and block classes (table_kind 0: cuckoo
// slots per table, >= 1.25 x the class cap; 1: buckets, load <= 1/2).
uint32_t warp_table_units(const Tuning &tu) {
    return tu.table_kind == 0 ? pow2_at_least((uint64_t)tu.warp_cap + tu.warp_cap / 4, 64)
                              : pow2_at_least((tu.warp_cap + 1) / 2, 16);
}
uint32_t block_table_units(const Tuning &tu) {
    return tu.table_kind == 0 ? pow2_at_least((uint64_t)tu.block_cap + tu.block_cap / 4, 64)
                              : pow2_at_least((tu.block_cap + 1) / 2, 16);
}
size_t warp_kernel_smem(const Tuning &tu) {
    return (size_t)tu.warps_per_block * (warp_set_bytes(tu.table_kind == 0, warp_table_units(tu)) + kWarpMetaBytes);
}
// With a split rank R the cuckoo table shares shared memory with the R-bit
// bitmap: the largest power-of-two table that fits beside it (and the task
// metadata), at most the size the class cap needs.
uint32_t block_units_for(const Tuning &tu, uint32_t R) {
    const uint32_t full = block_table_units(tu);
    if (!R || tu.table_kind != 0) return full;
    const size_t fixed = slice_smem_bytes(tu.max_v) + R / 8 + 2048;  // 2 KB: static shared memory and margin
    uint32_t m = full;
    while (m > 64 && fixed + 8ull * m > kSmemLimitBytes) m >>= 1;
    return m;
}
uint32_t block_hi_cap(const Tuning &tu, uint32_t R) {
    const uint32_t m = block_units_for(tu, R);
    return R ? (uint32_t)((uint64_t)m * 4 / 5) : tu.block_cap;
}
size_t block_kernel_smem(const Tuning &tu) {
    const uint32_t R = g1_split_rank(tu);
    return slice_smem_bytes(tu.max_v) + (tu.table_kind == 0 ? 8ull : 16ull) * block_units_for(tu, R) + R / 8;
}
size_t hub_kernel_smem(const Tuning &tu) { return slice_smem_bytes(tu.max_v) + (1ull << tu.hub_filter_log2) / 8; }

// Shared memory one block may opt into on sm_103a.
constexpr size_t kSmemLimit = kSmemLimitBytes;

tc_status intersect(tc_ctx *ctx, PipeBufs &b, uint32_t n) {
    (void)n;
    cudaStream_t s = ctx->stream;
    const Tuning &tu = ctx->tune;
    // what the kernels do with the triangles: 0 count, 1 per-vertex counts,
    // 2 listing (phase 1: the tiny class counts and records, the others
    // write; phase 2: the tiny class writes, the others do not run)
    const int mode = b.vcount ? 1 : (b.list_phase ? 2 : 0);
    VertexOut vo{b.vcount, b.vcount_rank};
    vo.out = b.list_out;
    vo.cap = b.list_cap;
    vo.ovf = b.ovf;
    vo.ovf_cap = b.ovf_cap;
    vo.cursor = &ctx->d_ctl->list_cursor;
    vo.fills = b.fills;
    vo.nch = b.nch;
    vo.wstate = b.wstate;
    vo.wstate_len = b.wstate_len;
    vo.err = &ctx->d_ctl->error;
    vo.inv = b.inv;
    const Ctl &h = *ctx->h_ctl;  // pulled after planning
    const size_t priv = mode == 1 ? 8ull * kPrivRanks : 0;
    // warps of a listing launch: at most one open chunk state each
    auto list_grid = [&](uint64_t grid, uint32_t warps_per_block) {
        if (mode == 2 && grid * warps_per_block > b.wstate_len) grid = b.wstate_len / warps_per_block;
        return grid;
    };
    // ev[4..7] bracket the warp, block and hub kernels
    // tiny rows: one thread each (this count's share of them)
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[8], s));
    const uint32_t nt3 = h.n_rows[3];
    const uint32_t lo3 = (uint32_t)((uint64_t)nt3 * ctx->shard / ctx->nshards);
    const uint32_t hi3 = (uint32_t)((uint64_t)nt3 * (ctx->shard + 1) / ctx->nshards);
    if (hi3 > lo3) {
        const int tmode = b.list_phase == 1 ? 0 : mode;
        const size_t smem = 4ull * tu.tiny_cap * 256 + priv;
        auto tiny = tmode == 0 ? k_isect_tiny<0> : tmode == 1 ? k_isect_tiny<1> : k_isect_tiny<2>;
        TC_CUDA(ctx, cudaFuncSetAttribute(tiny, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const uint32_t grid = std::min<uint32_t>((hi3 - lo3 + 255) / 256, (uint32_t)ctx->num_sms * 8u);
        VertexOut vt = vo;
        if (b.list_phase == 1) vt.task_hits = b.hits;
        if (b.list_phase == 2) {
            vt.off = b.hits;
            vt.base = b.tiny_base;
        }
        tiny<<<grid, 256, smem, s>>>(b.rows[3], lo3, hi3, b.rp, b.adj2, b.fcnt, b.gcnt, ctx->d_ctl, tu.tiny_cap,
                                     b.groups, vt);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[9], s));
    if (b.list_phase == 2) {  // the other classes wrote in phase 1
        ctx->isect_flags |= hi3 > lo3 ? 8u : 0u;
        TC_CUDA(ctx, cudaGetLastError());
        return TC_OK;
    }
    // this count's share of every class's task list (all of it unless sharded)
    auto share = [&](unsigned long long total, unsigned long long *lo, unsigned long long *hi) {
        *lo = total * ctx->shard / ctx->nshards;
        *hi = total * (ctx->shard + 1) / ctx->nshards;
    };
    unsigned long long lo0, hi0, lo1, hi1, lo2, hi2;
    share(h.n_tasks[0], &lo0, &hi0);
    share(h.n_tasks[1], &lo1, &hi1);
    share(h.n_tasks[2], &lo2, &hi2);
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[4], s));
    if (hi0 > lo0) {
        const size_t smem = warp_kernel_smem(tu) + priv;
        if (smem > kSmemLimit) return set_error(ctx, TC_ERR_INVALID, "tuning leaves no shared memory for this mode");
        auto kern = tu.table_kind == 0
                        ? (mode == 0 ? k_isect_warp<true, 0> : mode == 1 ? k_isect_warp<true, 1> : k_isect_warp<true, 2>)
                        : (mode == 0 ? k_isect_warp<false, 0>
                                     : mode == 1 ? k_isect_warp<false, 1> : k_isect_warp<false, 2>);
        TC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * tu.warps_per_block, smem));
        if (per_sm < 1) per_sm = 1;
        uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
        const uint64_t need = (hi0 - lo0 + tu.warps_per_block - 1) / tu.warps_per_block;
        if (grid > need) grid = need;
        grid = list_grid(grid, tu.warps_per_block);
        kern<<<(unsigned)grid, 32 * tu.warps_per_block, smem, s>>>(b.tasks[0], b.rows[0], b.ntask[0], b.rp, b.adj2,
                                                                   b.fcnt, b.eoff, b.erec, ctx->d_ctl,
                                                                   warp_table_units(tu), tu.flat_cap, lo0, hi0,
                                                                   b.groups, vo);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[5], s));
    if (hi1 > lo1) {
        // split set (plain counts only): the bitmap sits after the cuckoo table
        const size_t extra = priv + (mode == 2 ? 4ull * kStageSlots * (tu.block_threads / 32) : 0);
        const uint32_t split_R = ctx->split_R;
        const uint32_t units = block_units_for(tu, split_R);
        const size_t smem =
            slice_smem_bytes(tu.max_v) + (tu.table_kind == 0 ? 8ull : 16ull) * units + split_R / 8 + extra;
        if (smem > kSmemLimit) return set_error(ctx, TC_ERR_INVALID, "tuning leaves no shared memory for this mode");
        auto kern = tu.table_kind == 1 ? (mode == 0   ? k_isect_block<1, 0>
                                          : mode == 1 ? k_isect_block<1, 1>
                                                      : k_isect_block<1, 2>)
                    : split_R         ? k_isect_block<2, 0>  // split sets serve plain counts only
                                      : (mode == 0   ? k_isect_block<0, 0>
                                          : mode == 1 ? k_isect_block<0, 1>
                                                      : k_isect_block<0, 2>);
        TC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tu.block_threads, smem));
        if (per_sm < 1) per_sm = 1;
        uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
        if (grid > hi1 - lo1) grid = hi1 - lo1;
        grid = list_grid(grid, tu.block_threads / 32);
        // runs of about 1/64 of a block's share of the tasks: with the rows in the working order the
        // last runs hold the smallest tasks, and short runs let the blocks finish close together
        const unsigned long long chunk = std::max<unsigned long long>(1, (hi1 - lo1) / (grid * 64));
        kern<<<(unsigned)grid, tu.block_threads, smem, s>>>(b.tasks[1], b.rows[1], b.ntask[1], b.rp, b.adj2, b.fcnt,
                                                            b.eoff, b.erec, ctx->d_ctl, tu.max_v, units, split_R,
                                                            b.glo, b.gcnt, b.lv, chunk, lo1, hi1, b.groups, vo);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[6], s));
    const uint32_t nh = hi2 > lo2 ? h.n_rows[2] : 0;
    if (nh) {
        // task ranges of the hub rows: the host walks the groups
        std::vector<unsigned long long> pref(nh + 1);
        TC_CUDA(ctx, cudaMemcpyAsync(pref.data(), b.tpref[2], 8ull * (nh + 1), cudaMemcpyDeviceToHost, s));
        TC_CUDA(ctx, cudaStreamSynchronize(s));
        // split (plain counts): the prefilter shrinks to make room for the low-rank bitmap
        const uint32_t split_R = ctx->split_R;
        const uint32_t hmax_v = hub_max_v(tu, split_R);
        uint32_t filter_log2 = tu.hub_filter_log2;
        while (split_R && filter_log2 > 10 &&
               slice_smem_bytes(hmax_v) + (1ull << filter_log2) / 8 + split_R / 8 + 2048 > kSmemLimit)
            --filter_log2;
        const size_t smem = slice_smem_bytes(hmax_v) + (1ull << filter_log2) / 8 + split_R / 8 + priv +
                            (mode == 2 ? 4ull * kStageSlots * (tu.hub_threads / 32) : 0);
        if (smem > kSmemLimit) return set_error(ctx, TC_ERR_INVALID, "tuning leaves no shared memory for this mode");
        auto hub = split_R ? k_isect_hub<0, true>
                           : mode == 0 ? k_isect_hub<0> : mode == 1 ? k_isect_hub<1> : k_isect_hub<2>;
        TC_CUDA(ctx, cudaFuncSetAttribute(hub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        TC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hub, tu.hub_threads, smem));
        if (per_sm < 1) per_sm = 1;
        // Plain counts with two sets of bitmaps: groups alternate between the
        // context's stream and a side stream, each with its own bitmaps and task
        // counter, so that a group's last tasks overlap the next group's start.
        // (Per-vertex counts and listing keep one stream: their per-warp output
        // state is indexed by the warp's place in the grid.)
        const bool two = mode == 0 && b.hub_sets == 2 && nh > tu.hub_group;
        if (two) {
            if (!ctx->side_stream) {
                int prio = 0;
                TC_CUDA(ctx, cudaStreamGetPriority(s, &prio));
                TC_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->side_stream, cudaStreamNonBlocking, prio));
                for (int i = 0; i < 2; ++i)
                    if (!ctx->side_ev[i])
                        TC_CUDA(ctx, cudaEventCreateWithFlags(&ctx->side_ev[i], cudaEventDisableTiming));
            }
            TC_CUDA(ctx, cudaEventRecord(ctx->side_ev[0], s));
            TC_CUDA(ctx, cudaStreamWaitEvent(ctx->side_stream, ctx->side_ev[0], 0));
        }
        uint32_t gi = 0;
        for (uint32_t i0 = 0; i0 < nh; i0 += tu.hub_group) {
            const uint32_t g = std::min<uint32_t>(tu.hub_group, nh - i0);
            const unsigned long long first = std::max<unsigned long long>(pref[i0], lo2);
            const unsigned long long last = std::min<unsigned long long>(pref[i0 + g], hi2);
            if (first >= last) continue;  // none of this group's tasks is in this shard
            const bool side = two && (gi++ & 1u);
            cudaStream_t gs = side ? ctx->side_stream : s;
            uint32_t *bits = b.hub_bits + (side ? b.hub_words * tu.hub_group : 0ull);
            const int ctr = side ? 3 : 2;
            TC_CUDA(ctx, cudaMemsetAsync(bits, 0, 4ull * b.hub_words * g, gs));
            TC_CUDA(ctx, cudaMemsetAsync(&ctx->d_ctl->task_next[ctr], 0, sizeof(unsigned), gs));
            k_hub_set<<<(unsigned)ctx->num_sms * 4u, 256, 0, gs>>>(b.rows[2], i0, g, b.rp, b.fcnt, b.adj2, bits,
                                                                  b.hub_words);
            uint64_t grid = (uint64_t)ctx->num_sms * per_sm;
            if (grid > last - first) grid = last - first;
            grid = list_grid(grid, tu.hub_threads / 32);
            const unsigned long long chunk = std::max<unsigned long long>(1, (last - first) / (grid * 8));
            hub<<<(unsigned)grid, tu.hub_threads, smem, gs>>>(b.tasks[2], first, last, b.rows[2], b.ntask[2], i0,
                                                                      b.rp, b.adj2, b.fcnt, b.eoff, b.erec, ctx->d_ctl,
                                                                      bits, b.hub_words, hmax_v, chunk, filter_log2,
                                                                      b.groups, vo, split_R, b.glo, b.lv, ctr);
            note_launch(ctx, 2);
        }
        if (two) {  // the context's stream waits for the side stream's groups
            TC_CUDA(ctx, cudaEventRecord(ctx->side_ev[1], ctx->side_stream));
            TC_CUDA(ctx, cudaStreamWaitEvent(s, ctx->side_ev[1], 0));
        }
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[7], s));
    ctx->isect_flags = (hi0 > lo0 ? 1u : 0u) | (hi1 > lo1 ? 2u : 0u) | (nh ? 4u : 0u) | (hi3 > lo3 ? 8u : 0u);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
