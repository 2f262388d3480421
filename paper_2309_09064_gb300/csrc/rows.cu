// rows.cu -- partition of E into E0 / E1, orientation of E0 by the working
// order, and the rows the intersections read (Algorithm 4, partition loop).
//
// Every vertex x keeps its CSR slots [rp[x], rp[x+1]); they are rewritten as
//     [ F(x) | A(x) | G1(x) ]
//   F(x)  = { y ~ x : L(y) == L(x), x precedes y }  horizontal out-neighbours, as vertex ids
//   A(x)  = { y ~ x : L(y) == L(x), y precedes x }  horizontal in-neighbours, as ranks, descending
//   G1(x) = { y ~ x : L(y) != L(x) }                level-spanning neighbours, as ranks
// (rank = position in the working order).  G1(x) holds its ranks below
// g1_lo first (g1_lo = 2^block_bits_log2, 0: no split): the block class keeps
// those ranks of its sets in a direct bitmap, so a probe range whose steps lie
// wholly below (or wholly above) g1_lo takes one kind of lookup per step.
// The split is kept where it is cheap -- rows of up to 32 neighbours (a lane's
// buffer column), level-spanning parts of up to kWarpA ranks (the warp's
// buffer) and the block-filled rows -- and otherwise left out (the lookups do
// not depend on it).  A(x) is the set Algorithm 2 has
// built for x once every row before x's is done.  For a horizontal edge u -> v
// the intersections hash A(u) and G1(u) and probe the elements of A(v) ranked
// below u -- which in descending order are the last ones of A(v) -- and all of
// G1(v): one contiguous range at the end of v's slots.  k_records finds, for
// every oriented edge, where that range starts (a binary search for rank(u) in
// A(v)) and writes a probe record {start, length, split}.
#include "pipeline.cuh"

namespace tc {
namespace {

constexpr uint32_t kSmallRow = 32;    // rows of degree <= 32: one lane each
constexpr uint32_t kWarpA = 1024;     // A parts up to this size: sorted by the warp in shared memory
constexpr uint32_t kSortCap = 32768;  // A parts up to this size: sorted (larger: k_sort_big); beyond: unsorted
constexpr uint32_t kHugeRow = 8192;   // rows of higher degree: one block each (k_row_fill_huge)
constexpr int kFillThreads = 256;
constexpr uint32_t kFillAhead = 8;   // neighbours of a lane-owned row read ahead together

// Sort buf[0..P) ascending (P a power of two) with one warp: bitonic network.
__device__ __forceinline__ void warp_bitonic(uint32_t *buf, uint32_t P) {
    const unsigned lane = lane_id();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < P; i += 32) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const uint32_t a = buf[i], c = buf[l];
                    if ((a > c) == ((i & k) == 0)) {
                        buf[i] = c;
                        buf[l] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ uint32_t pow2_ceil(uint32_t a) {
    uint32_t p = 1;
    while (p < a) p <<= 1;
    return p;
}

// One pass over every CSR row: F from the front, G1 from the back, A through
// shared memory (sorted there) into the slots between them.  Rows of degree
// <= 32 belong to one lane, which keeps A sorted by insertion in its own
// column of the warp's buffer; longer rows are done by the whole warp, lanes
// striding over the row and ballots keeping the order; their A part is sorted
// in the warp's buffer when it fits, else written in CSR order and sorted
// later by k_sort_big (or left unsorted beyond kSortCap).
// Rank and level of a vertex: from the packed 4-byte word (rank << 8 |
// level) when there is one, else from the {rank, level} pair.
template <bool kPacked>
__device__ __forceinline__ uint2 rank_level(const uint2 *__restrict__ lv, const uint32_t *__restrict__ lvp, uint32_t y) {
    if constexpr (kPacked) {
        const uint32_t p = lvp[y];
        return make_uint2(p >> 8, p & 0xFFu);
    } else {
        return lv[y];
    }
}

template <bool kPacked>
__global__ void __launch_bounds__(kFillThreads) k_row_fill(uint32_t n, const uint64_t *__restrict__ rp,
                                                           const uint32_t *__restrict__ col,
                                                           const uint2 *__restrict__ lv,
                                                           const uint32_t *__restrict__ lvp, uint32_t *__restrict__ adj2,
                                                           uint32_t *__restrict__ fcnt, uint32_t *__restrict__ gcnt,
                                                           uint4 *__restrict__ vmeta, uint32_t *__restrict__ big,
                                                           uint32_t *__restrict__ huge, Ctl *ctl, uint32_t g1_lo,
                                                           uint32_t *__restrict__ glo, uint32_t *__restrict__ part) {
    __shared__ uint32_t sbuf[kFillThreads / 32][kWarpA];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t *buf = sbuf[warp];
    // warps take chunks of 32 vertices from a counter: rows of very different lengths even out
    const uint64_t chunks = ((uint64_t)n + 31) / 32;
    for (;;) {
        unsigned int c = 0;
        if (lane == 0) c = atomicAdd(&ctl->fill_next, 1u);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        if (c >= chunks) break;
        const uint64_t x = (uint64_t)c * 32 + lane;
        const bool valid = x < n;
        const uint64_t b = valid ? rp[x] : 0;
        const uint32_t dx = valid ? (uint32_t)(rp[x + 1] - b) : 0;
        const uint2 me = valid ? rank_level<kPacked>(lv, lvp, (uint32_t)x) : make_uint2(0, 0);
        if (valid && dx <= kSmallRow) {
            uint32_t fp = 0, gp = 0, ap = 0, gl = 0;  // gl: level-spanning ranks below g1_lo (column top)
            for (uint32_t j0 = 0; j0 < dx; j0 += kFillAhead) {
                // the ids and their rank/level words of kFillAhead neighbours in
                // flight together, then the neighbours in order
                uint32_t y[kFillAhead];
                uint2 q[kFillAhead];
#pragma unroll
                for (uint32_t t = 0; t < kFillAhead; ++t) y[t] = j0 + t < dx ? col[b + j0 + t] : 0u;
#pragma unroll
                for (uint32_t t = 0; t < kFillAhead; ++t)
                    q[t] = j0 + t < dx ? rank_level<kPacked>(lv, lvp, y[t]) : make_uint2(0, 0);
#pragma unroll
                for (uint32_t t = 0; t < kFillAhead; ++t) {
                    if (j0 + t >= dx) break;
                    if (q[t].y != me.y) {
                        // below g1_lo: kept at the top of the column (A fills it from the
                        // bottom; together they hold at most dx <= 32 ranks)
                        if (q[t].x < g1_lo) buf[(kSmallRow - 1 - gl++) * 32 + lane] = q[t].x;
                        else adj2[b + dx - 1 - gp++] = q[t].x;
                    } else if (me.x < q[t].x) {
                        adj2[b + fp++] = y[t];
                    } else {  // insert into the lane's column, descending
                        uint32_t i = ap++;
                        while (i > 0 && buf[(i - 1) * 32 + lane] < q[t].x) {
                            buf[i * 32 + lane] = buf[(i - 1) * 32 + lane];
                            --i;
                        }
                        buf[i * 32 + lane] = q[t].x;
                    }
                }
            }
            for (uint32_t i = 0; i < ap; ++i) adj2[b + fp + i] = buf[i * 32 + lane];
            for (uint32_t i = 0; i < gl; ++i) adj2[b + fp + ap + i] = buf[(kSmallRow - 1 - i) * 32 + lane];
            gp += gl;
            fcnt[x] = fp;
            gcnt[x] = gp;
            glo[x] = gl;
            const uint64_t as = b + fp;
            vmeta[x] = make_uint4((uint32_t)as, (uint32_t)(as >> 32), ap, gp);
        }
        __syncwarp();
        // rows of degree above kHugeRow go to k_row_fill_huge (a block each)
        const unsigned huge_m = __ballot_sync(0xFFFFFFFFu, valid && dx > kHugeRow);
        if (valid && dx > kHugeRow) huge[atomicAdd(&ctl->n_huge, 1u)] = (uint32_t)x;
        unsigned pending = __ballot_sync(0xFFFFFFFFu, valid && dx > kSmallRow) & ~huge_m;
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1;
            const uint32_t bx = (uint32_t)__shfl_sync(0xFFFFFFFFu, (unsigned long long)x, src);
            const uint32_t bd = __shfl_sync(0xFFFFFFFFu, dx, src);
            const uint64_t bb = __shfl_sync(0xFFFFFFFFu, b, src);
            const uint32_t brx = __shfl_sync(0xFFFFFFFFu, me.x, src);
            const uint32_t blx = __shfl_sync(0xFFFFFFFFu, me.y, src);
            uint32_t fp = 0, gp = 0, ap = 0;
            for (uint32_t j0 = 0; j0 < bd; j0 += 32) {
                const uint32_t j = j0 + lane;
                bool isF = false, isG = false, isA = false;
                uint32_t y = 0, ry = 0;
                if (j < bd) {
                    y = col[bb + j];
                    const uint2 q = rank_level<kPacked>(lv, lvp, y);
                    ry = q.x;
                    if (q.y != blx) isG = true;
                    else if (brx < ry) isF = true;
                    else isA = true;
                }
                const unsigned mF = __ballot_sync(0xFFFFFFFFu, isF);
                const unsigned mG = __ballot_sync(0xFFFFFFFFu, isG);
                const unsigned mA = __ballot_sync(0xFFFFFFFFu, isA);
                if (isF) adj2[bb + fp + __popc(mF & lt)] = y;
                if (isG) adj2[bb + bd - 1 - (gp + __popc(mG & lt))] = ry;
                if (isA) {
                    const uint32_t pos = ap + __popc(mA & lt);
                    if (pos < kWarpA) buf[pos] = ry;
                }
                fp += __popc(mF);
                gp += __popc(mG);
                ap += __popc(mA);
            }
            __syncwarp();
            if (ap <= kWarpA) {
                const uint32_t P = pow2_ceil(ap);
                for (uint32_t i = ap + lane; i < P; i += 32) buf[i] = kEmpty;
                __syncwarp();
                warp_bitonic(buf, P);
                for (uint32_t i = lane; i < ap; i += 32) adj2[bb + fp + i] = buf[ap - 1 - i];
            } else {  // A in CSR order now; sorted by k_sort_big if it is not too long
                uint32_t apos = 0;
                for (uint32_t j0 = 0; j0 < bd; j0 += 32) {
                    const uint32_t j = j0 + lane;
                    bool isA = false;
                    uint32_t ry = 0;
                    if (j < bd) {
                        const uint2 q = rank_level<kPacked>(lv, lvp, col[bb + j]);
                        ry = q.x;
                        isA = q.y == blx && ry < brx;
                    }
                    const unsigned mA = __ballot_sync(0xFFFFFFFFu, isA);
                    if (isA) adj2[bb + fp + apos + __popc(mA & lt)] = ry;
                    apos += __popc(mA);
                }
                if (lane == 0 && ap <= kSortCap) big[atomicAdd(&ctl->n_big, 1u)] = bx;
            }
            __syncwarp();
            uint32_t row_glo = 0;
            if (g1_lo && gp > kWarpA) {  // split by k_g1_split (a block each)
                if (lane == 0) part[atomicAdd(&ctl->n_part, 1u)] = bx;
                row_glo = kNoSplit;
            } else if (g1_lo && gp > 0) {
                // G1 (written from the back) through the warp's buffer, back in place
                // with its ranks below g1_lo first
                const uint64_t gb = bb + bd - gp;
                uint32_t nlo = 0;
                for (uint32_t i = lane; i < gp; i += 32) {
                    const uint32_t r = adj2[gb + i];
                    buf[i] = r;
                    nlo += r < g1_lo;
                }
                nlo = warp_sum(nlo);
                __syncwarp();
                uint32_t lp = 0, hp = 0;
                for (uint32_t i0 = 0; i0 < gp; i0 += 32) {
                    const uint32_t i = i0 + lane;
                    const uint32_t r = i < gp ? buf[i] : 0u;
                    const bool lo = i < gp && r < g1_lo, hi = i < gp && r >= g1_lo;
                    const unsigned ml = __ballot_sync(0xFFFFFFFFu, lo), mh = __ballot_sync(0xFFFFFFFFu, hi);
                    if (lo) adj2[gb + lp + __popc(ml & lt)] = r;
                    if (hi) adj2[gb + nlo + hp + __popc(mh & lt)] = r;
                    lp += __popc(ml);
                    hp += __popc(mh);
                }
                __syncwarp();
                row_glo = nlo;
            }
            if (lane == 0) {
                fcnt[bx] = fp;
                gcnt[bx] = gp;
                glo[bx] = row_glo;
                const uint64_t as = bb + fp;
                vmeta[bx] = make_uint4((uint32_t)as, (uint32_t)(as >> 32), ap, gp);
            }
        }
    }
}

// Rows of degree above kHugeRow, one block each (persistent over the list the
// fill kernel built): a counting pass, then a writing pass over chunks of
// blockDim neighbours whose positions come from the warps' ballots and a
// prefix over the warps in order, so every part keeps CSR order and every
// run writes the same rows (a count split into shards recomputes the rows
// on each shard, and its tasks are slices of F(u): the shards must agree on
// its order).  A is listed for k_sort_big (or left unsorted beyond kSortCap).
template <bool kPacked>
__global__ void __launch_bounds__(1024) k_row_fill_huge(const uint32_t *__restrict__ huge, Ctl *ctl,
                                                        const uint64_t *__restrict__ rp,
                                                        const uint32_t *__restrict__ col,
                                                        const uint2 *__restrict__ lv,
                                                        const uint32_t *__restrict__ lvp, uint32_t *__restrict__ adj2,
                                                        uint32_t *__restrict__ fcnt, uint32_t *__restrict__ gcnt,
                                                        uint4 *__restrict__ vmeta, uint32_t *__restrict__ big,
                                                        uint32_t g1_lo, uint32_t *__restrict__ glo) {
    __shared__ unsigned int cnt[4], base[4];
    __shared__ unsigned int wcnt[32][4];  // this chunk's F, G1 (high), A, G1 (low) per warp
    __shared__ unsigned int s_i;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t nh = ctl->n_huge;
    for (;;) {  // blocks take rows from a counter (their degrees differ by orders of magnitude)
        if (threadIdx.x == 0) s_i = atomicAdd(&ctl->huge_next, 1u);
        __syncthreads();
        const uint32_t i = s_i;
        __syncthreads();
        if (i >= nh) break;
        const uint32_t x = huge[i];
        const uint64_t b = rp[x];
        const uint32_t d = (uint32_t)(rp[x + 1] - b);
        const uint2 me = rank_level<kPacked>(lv, lvp, x);
        if (threadIdx.x < 4) cnt[threadIdx.x] = base[threadIdx.x] = 0;
        __syncthreads();
        uint32_t f = 0, g = 0, gl = 0;
        for (uint32_t j = threadIdx.x; j < d; j += blockDim.x) {
            const uint2 q = rank_level<kPacked>(lv, lvp, col[b + j]);
            if (q.y != me.y) {
                ++g;
                gl += q.x < g1_lo;
            } else if (me.x < q.x) {
                ++f;
            }
        }
        f = warp_sum(f);
        g = warp_sum(g);
        gl = warp_sum(gl);
        if (lane == 0) {
            atomicAdd(&cnt[0], f);
            atomicAdd(&cnt[1], g);
            atomicAdd(&cnt[3], gl);
        }
        __syncthreads();
        const uint32_t F = cnt[0], G = cnt[1], A = d - F - G;
        for (uint32_t j0 = 0; j0 < d; j0 += blockDim.x) {  // every thread takes part in every chunk
            const uint32_t j = j0 + threadIdx.x;
            bool isF = false, isG = false, isA = false, isL = false;
            uint32_t y = 0, ry = 0;
            if (j < d) {
                y = col[b + j];
                const uint2 q = rank_level<kPacked>(lv, lvp, y);
                ry = q.x;
                if (q.y != me.y) {
                    isL = ry < g1_lo;  // level-spanning, below g1_lo: right after A
                    isG = !isL;
                } else if (me.x < ry) {
                    isF = true;
                } else {
                    isA = true;
                }
            }
            const unsigned mF = __ballot_sync(0xFFFFFFFFu, isF);
            const unsigned mG = __ballot_sync(0xFFFFFFFFu, isG);
            const unsigned mA = __ballot_sync(0xFFFFFFFFu, isA);
            const unsigned mL = __ballot_sync(0xFFFFFFFFu, isL);
            if (lane == 0) {
                wcnt[warp][0] = __popc(mF);
                wcnt[warp][1] = __popc(mG);
                wcnt[warp][2] = __popc(mA);
                wcnt[warp][3] = __popc(mL);
            }
            __syncthreads();
            uint32_t pF = base[0], pG = base[1], pA = base[2], pL = base[3];
            for (unsigned w = 0; w < warp; ++w) {
                pF += wcnt[w][0];
                pG += wcnt[w][1];
                pA += wcnt[w][2];
                pL += wcnt[w][3];
            }
            if (isF) adj2[b + pF + __popc(mF & lt)] = y;
            if (isA) adj2[b + F + pA + __popc(mA & lt)] = ry;
            if (isL) adj2[b + F + A + pL + __popc(mL & lt)] = ry;
            if (isG) adj2[b + d - 1 - (pG + __popc(mG & lt))] = ry;
            __syncthreads();
            if (threadIdx.x < 4) {
                uint32_t t = 0;
                for (unsigned w = 0; w < nwarps; ++w) t += wcnt[w][threadIdx.x];
                base[threadIdx.x] += t;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            fcnt[x] = F;
            gcnt[x] = G;
            glo[x] = cnt[3];
            const uint64_t as = b + F;
            vmeta[x] = make_uint4((uint32_t)as, (uint32_t)(as >> 32), A, G);
            if (A > 1 && A <= kSortCap) big[atomicAdd(&ctl->n_big, 1u)] = x;
        }
        __syncthreads();
    }
}

// Level-spanning parts of more than kWarpA ranks in warp-filled rows (at most
// kHugeRow): one block per listed row stages the part in shared memory and
// writes it back with its ranks below g1_lo first, each side in its former
// order (positions from the warps' ballots and a prefix over the warps).
__global__ void __launch_bounds__(1024) k_g1_split(const uint32_t *__restrict__ part, Ctl *ctl,
                                                   const uint64_t *__restrict__ rp, const uint32_t *__restrict__ gcnt,
                                                   uint32_t *__restrict__ adj2, uint32_t g1_lo,
                                                   uint32_t *__restrict__ glo) {
    extern __shared__ uint32_t sg[];  // kHugeRow ranks
    __shared__ unsigned int wcnt[32][2], base[2], nlo;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    __shared__ unsigned int s_i;
    const uint32_t np = ctl->n_part;
    for (;;) {  // blocks take rows from a counter
        if (threadIdx.x == 0) s_i = atomicAdd(&ctl->split_next, 1u);
        __syncthreads();
        const uint32_t i = s_i;
        __syncthreads();
        if (i >= np) break;
        const uint32_t x = part[i];
        const uint32_t g = gcnt[x];
        if (threadIdx.x == 0) {
            base[0] = base[1] = 0;
            nlo = 0;
        }
        __syncthreads();
        if (g > kHugeRow) {  // not a row the fill kernel listed: leave it unsplit
            if (threadIdx.x == 0) glo[x] = kNoSplit;
            continue;
        }
        const uint64_t gb = rp[x + 1] - g;
        uint32_t c = 0;
        for (uint32_t j = threadIdx.x; j < g; j += blockDim.x) {
            const uint32_t r = adj2[gb + j];
            sg[j] = r;
            c += r < g1_lo;
        }
        c = warp_sum(c);
        if (lane == 0) atomicAdd(&nlo, c);
        __syncthreads();
        const uint32_t L = nlo;
        for (uint32_t j0 = 0; j0 < g; j0 += blockDim.x) {
            const uint32_t j = j0 + threadIdx.x;
            const uint32_t r = j < g ? sg[j] : 0u;
            const bool lo = j < g && r < g1_lo, hi = j < g && r >= g1_lo;
            const unsigned ml = __ballot_sync(0xFFFFFFFFu, lo), mh = __ballot_sync(0xFFFFFFFFu, hi);
            if (lane == 0) {
                wcnt[warp][0] = __popc(ml);
                wcnt[warp][1] = __popc(mh);
            }
            __syncthreads();
            uint32_t pl = base[0], ph = base[1];
            for (unsigned w = 0; w < warp; ++w) {
                pl += wcnt[w][0];
                ph += wcnt[w][1];
            }
            if (lo) adj2[gb + pl + __popc(ml & lt)] = r;
            if (hi) adj2[gb + L + ph + __popc(mh & lt)] = r;
            __syncthreads();
            if (threadIdx.x < 2) {
                uint32_t t = 0;
                for (unsigned w = 0; w < nwarps; ++w) t += wcnt[w][threadIdx.x];
                base[threadIdx.x] += t;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) glo[x] = L;
        __syncthreads();
    }
}

// A parts longer than kWarpA (and at most kSortCap): one block per row sorts
// it in shared memory (bitonic, padded with kEmpty) and writes it back
// descending.  Persistent: blocks stride over the list the fill kernel built.
__global__ void __launch_bounds__(1024) k_sort_big(const uint32_t *__restrict__ big, Ctl *ctl,
                                                   const uint64_t *__restrict__ rp, const uint32_t *__restrict__ fcnt,
                                                   const uint32_t *__restrict__ gcnt, uint32_t *__restrict__ adj2) {
    extern __shared__ uint32_t sb[];  // kSortCap words
    __shared__ unsigned int s_i;
    const uint32_t nb = ctl->n_big;
    for (;;) {  // blocks take rows from a counter (the parts differ in length by 32x)
        if (threadIdx.x == 0) s_i = atomicAdd(&ctl->sort_next, 1u);
        __syncthreads();
        const uint32_t i = s_i;
        __syncthreads();
        if (i >= nb) break;
        const uint32_t x = big[i];
        const uint64_t b = rp[x] + fcnt[x];
        const uint32_t a = (uint32_t)(rp[x + 1] - b) - gcnt[x];
        if (a > kSortCap) {  // not a row the fill kernel listed: report, leave it
            if (threadIdx.x == 0) atomicOr(&ctl->error, 0x100u);
            continue;
        }
        const uint32_t P = pow2_ceil(a);
        for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) sb[t] = t < a ? adj2[b + t] : kEmpty;
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
                    const uint32_t l = t ^ j;
                    if (l > t) {
                        const uint32_t p = sb[t], q = sb[l];
                        if ((p > q) == ((t & k) == 0)) {
                            sb[t] = q;
                            sb[l] = p;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t t = threadIdx.x; t < a; t += blockDim.x) adj2[b + t] = sb[a - 1 - t];
        __syncthreads();
    }
}

// Rows with at least one oriented horizontal edge are the hashed side of the
// intersections; split them by the size s(u) = |A(u)| + |G1(u)| of the hashed
// set: class 3 (tiny) s <= tiny_cap and degree <= 4 tiny_cap, class 0 (warp)
// s <= warp_cap, class 1 (block) s <= block_cap, class 2 (hub).
// The lists are built by a stable scan, so they (and the task lists made from
// them) are in vertex order on every run: shards of a count agree on them.
// The tiny class compares the level-spanning parts pairwise (|G1(u)| x
// |G1(v)| per edge), so it takes only rows whose G1 part is short.
constexpr uint32_t kTinyG = 8;

// With a split rank R the block class also needs the set's ranks at or above
// R (the ones its cuckoo table holds) to number at most hi_cap: G1's high part,
// and all of A(x) when x itself is ranked at or above R (A holds ranks below
// x's); a G1 part left unsplit counts whole.
__global__ void k_class_flags(uint32_t n, const uint32_t *__restrict__ fcnt, const uint32_t *__restrict__ gcnt,
                              const uint32_t *__restrict__ deg, uint32_t *__restrict__ cls, Ctl *ctl,
                              uint32_t warp_cap, uint32_t block_cap, uint32_t tiny_cap, uint32_t R, uint32_t hi_cap,
                              const uint32_t *__restrict__ glo, const uint2 *__restrict__ lv) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned my_max = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        uint32_t c = 4;  // no oriented horizontal edge: nothing to intersect
        const uint32_t f = fcnt[x];
        if (f > 0) {
            const uint32_t s = deg[x] - f;
            bool fits = s <= block_cap;
            if (R && fits && s > warp_cap) {
                const uint32_t g = gcnt[x], gl = glo[x];
                const uint32_t hi = (gl == kNoSplit ? g : g - gl) + (lv[x].x >= R ? s - g : 0u);
                fits = hi <= hi_cap;
            }
            c = s <= warp_cap ? 0u : (fits ? 1u : 2u);
            if (s <= tiny_cap && deg[x] <= 4 * tiny_cap && gcnt[x] <= kTinyG) c = 3;
            if (c == 1 || c == 2) my_max = s > my_max ? s : my_max;
        }
        cls[x] = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned y = __shfl_xor_sync(0xFFFFFFFFu, my_max, o);
        my_max = y > my_max ? y : my_max;
    }
    if (lane_id() == 0 && my_max) atomicMax(&ctl->max_s2, my_max);
}

// The rows of every class are listed in the working order (order[i] = the
// vertex of rank i, the sorted rank keys; null: the identity): the largest
// hashed sets come first and the task lists end with the smallest tasks, so
// the blocks that claim the last runs of tasks finish close together.
__device__ __forceinline__ uint32_t vertex_at(const unsigned long long *order, uint64_t i) {
    return order ? (uint32_t)(order[i] & 0xFFFFFFFFull) : (uint32_t)i;
}

__global__ void k_class_indicator(uint32_t n, const uint32_t *__restrict__ cls, uint32_t c, uint32_t *__restrict__ ind,
                                  const unsigned long long *__restrict__ order) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        ind[i] = cls[vertex_at(order, i)] == c;
}

__global__ void k_class_scatter(uint32_t n, const uint32_t *__restrict__ cls, uint32_t c,
                                const unsigned long long *__restrict__ pos, uint32_t *__restrict__ rows,
                                unsigned int *__restrict__ n_rows, const unsigned long long *__restrict__ order) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t x = vertex_at(order, i);
        if (cls[x] == c) rows[pos[i]] = x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_rows = (unsigned int)pos[n];
}

// Probe records are made edge-parallel: the oriented edges u -> v are
// numbered e = eoff[u] + k (v = F(u)[k]) and cut into chunks of kRecChunk;
// chunk_row[c] is the row holding edge c * kRecChunk.
constexpr uint32_t kRecChunk = 256;
constexpr uint32_t kRecLinear = 16;  // A parts up to this size are counted, not searched

__global__ void k_chunk_rows(uint32_t n, const uint64_t *__restrict__ eoff, uint32_t *__restrict__ chunk_row) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const uint64_t lo = eoff[u], hi = eoff[u + 1];
        for (uint64_t c = (lo + kRecChunk - 1) / kRecChunk; c * kRecChunk < hi; ++c) chunk_row[c] = (uint32_t)u;
    }
}

// Every 32nd slot of the rewritten rows, kept compact: fence[k] = adj2[32 k].
// A search in a long sorted A part runs over its fences first (one 128-byte
// line holds 32 of them, and the array stays in L2), then inside the one
// 128-byte line of adj2 left.
__global__ void k_fence(const uint32_t *__restrict__ adj2, uint64_t slots, uint32_t *__restrict__ fence) {
    const uint64_t nf = (slots + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += stride) fence[k] = adj2[32 * k];
}

// The interval [*lo, *hi) of positions of the descending run adj2[as, as + av)
// that holds its first element below r, from a binary search over the run's
// fences: at most 32 positions (all positions when the run holds no fence).
__device__ __forceinline__ void fence_search(const uint32_t *__restrict__ fence, uint64_t as, uint32_t av, uint32_t r,
                                             uint32_t *lo, uint32_t *hi) {
    const uint64_t k0 = (as + 31) / 32, kend = (as + av + 31) / 32;  // fences at 32 k in [as, as + av)
    uint64_t flo = k0, fhi = kend > k0 ? kend : k0;
    while (flo < fhi) {
        const uint64_t mid = (flo + fhi) >> 1;
        if (fence[mid] < r) fhi = mid; else flo = mid + 1;
    }
    *lo = flo > k0 ? (uint32_t)(32 * (flo - 1) - as + 1) : 0u;  // fence flo - 1 holds a rank >= r
    *hi = flo < kend ? (uint32_t)(32 * flo - as) : av;          // fence flo holds one below r
}

// For every oriented edge u -> v: the number p of elements of A(v) ranked
// below u (binary search in the descending A(v), over its fences first; all
// of A(v) when it was left unsorted), and the probe record {start, length = |G1(v)| + p, split = p}
// of the range at the end of v's slots.  One warp per chunk; every lane walks
// from the chunk's first row to the rows of its own edges, and runs the
// binary searches of kRecBatch edges in lockstep (independent loads in
// flight).  Block 0 also publishes |E0| = eoff[n].
constexpr int kRecBatch = 2;

__global__ void k_records(uint32_t n, const uint64_t *__restrict__ eoff, const uint32_t *__restrict__ chunk_row,
                          const uint64_t *__restrict__ rp, const uint32_t *__restrict__ adj2,
                          const uint2 *__restrict__ lv, const uint4 *__restrict__ vmeta, uint4 *__restrict__ erec,
                          Ctl *ctl, const uint32_t *__restrict__ fence) {
    const unsigned lane = lane_id();
    const uint64_t E = eoff[n];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->e0 = E;
    const uint64_t chunks = (E + kRecChunk - 1) / kRecChunk;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < chunks; c += warps) {
        const uint64_t e_lo = c * kRecChunk, e_hi = min(E, e_lo + kRecChunk);
        uint32_t u = chunk_row[c];
        uint64_t u_lo = eoff[u], u_hi = eoff[u + 1], fb = rp[u];
        uint32_t ru = lv[u].x;
        for (uint64_t e0 = e_lo + lane; e0 < e_hi; e0 += 32 * kRecBatch) {
            uint32_t r[kRecBatch], lo[kRecBatch], hi[kRecBatch], av[kRecBatch], gv[kRecBatch];
            uint64_t as[kRecBatch];
            bool ok[kRecBatch];
#pragma unroll
            for (int i = 0; i < kRecBatch; ++i) {
                const uint64_t e = e0 + 32ull * i;
                ok[i] = e < e_hi;
                uint32_t v = 0;
                if (ok[i]) {
                    while (e >= u_hi) {  // rows of no edge have u_lo == u_hi and are skipped
                        ++u;
                        u_lo = u_hi;
                        u_hi = eoff[u + 1];
                        fb = rp[u];
                        ru = lv[u].x;
                    }
                    v = adj2[fb + (e - u_lo)];
                }
                r[i] = ru;
                const uint4 m = ok[i] ? vmeta[v] : make_uint4(0, 0, 0, 0);
                as[i] = ((uint64_t)m.y << 32) | m.x;
                av[i] = m.z;
                gv[i] = m.w;
                lo[i] = 0;
                hi[i] = av[i] <= kSortCap ? av[i] : 0;  // unsorted A: no search, p = |A(v)|
                if (av[i] <= kRecLinear) {  // short A: count the ranks >= r, all loads at once
                    uint32_t c = 0;
#pragma unroll
                    for (uint32_t j = 0; j < kRecLinear; ++j) c += j < av[i] && adj2[as[i] + j] >= r[i];
                    lo[i] = hi[i] = c;
                }
            }
            // long sorted A parts: over the fences first, in lockstep
            uint64_t flo[kRecBatch], fhi[kRecBatch], fk0[kRecBatch], fend[kRecBatch];
#pragma unroll
            for (int i = 0; i < kRecBatch; ++i) {
                fk0[i] = (as[i] + 31) / 32;
                fend[i] = (as[i] + av[i] + 31) / 32;
                const bool use = hi[i] > lo[i] + 32;
                flo[i] = fk0[i];
                fhi[i] = use ? fend[i] : fk0[i];
            }
            for (int step = 0; step < 17; ++step) {
                bool any = false;
#pragma unroll
                for (int i = 0; i < kRecBatch; ++i) {
                    if (flo[i] < fhi[i]) {
                        const uint64_t mid = (flo[i] + fhi[i]) >> 1;
                        if (fence[mid] < r[i]) fhi[i] = mid; else flo[i] = mid + 1;
                        any = true;
                    }
                }
                if (!any) break;
            }
#pragma unroll
            for (int i = 0; i < kRecBatch; ++i) {
                if (hi[i] > lo[i] + 32) {  // the one line left between two fences
                    const uint32_t l = flo[i] > fk0[i] ? (uint32_t)(32 * (flo[i] - 1) - as[i] + 1) : 0u;
                    const uint32_t h = flo[i] < fend[i] ? (uint32_t)(32 * flo[i] - as[i]) : av[i];
                    lo[i] = l;
                    hi[i] = h;
                }
            }
            // first position holding a rank below r, all searches in lockstep
            for (int step = 0; step < 17; ++step) {
                bool any = false;
#pragma unroll
                for (int i = 0; i < kRecBatch; ++i) {
                    if (lo[i] < hi[i]) {
                        const uint32_t mid = (lo[i] + hi[i]) >> 1;
                        if (adj2[as[i] + mid] < r[i]) hi[i] = mid; else lo[i] = mid + 1;
                        any = true;
                    }
                }
                if (!any) break;
            }
#pragma unroll
            for (int i = 0; i < kRecBatch; ++i) {
                if (!ok[i]) continue;
                const uint32_t p = av[i] <= kSortCap ? av[i] - lo[i] : av[i];
                const uint64_t start = as[i] + av[i] - p;
                erec[e0 + 32ull * i] = make_uint4((uint32_t)start, (uint32_t)(start >> 32), gv[i] + p, p);
            }
        }
    }
}

// Cut the out-edges of every row u of class c (one warp each) into tasks
// (contiguous slices of F(u)) of about `target` probes: work(u) = sum of the
// record lengths, ntask = ceil(work(u) / max(task_work, min_mult * s(u))), at
// least ceil(|F(u)| / max_v) (shared-memory metadata of one task), at most
// |F(u)|.
// With est (a count split into shards), the work of an edge u -> v is taken
// as |A(v)| + |G1(v)| (the probe range at most), read from v's descriptor:
// the plan then needs no probe record, and every shard builds the records of
// its own tasks only.
__global__ void k_plan(const uint32_t *__restrict__ rows, const unsigned int *__restrict__ n_rows,
                       const uint64_t *__restrict__ rp, const uint32_t *__restrict__ fcnt,
                       const uint64_t *__restrict__ eoff, const uint4 *__restrict__ erec,
                       uint32_t *__restrict__ ntask, uint32_t task_work, uint32_t min_mult, uint32_t max_v,
                       bool est, const uint32_t *__restrict__ adj2, const uint4 *__restrict__ vmeta) {
    const unsigned lane = lane_id();
    const uint32_t nr = *n_rows;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nr; i += warps) {
        const uint32_t u = rows[i];
        const uint32_t fu = fcnt[u];
        const uint4 *rec = erec + eoff[u];
        unsigned long long w0 = 0, w1 = 0, w2 = 0, w3 = 0;
        uint32_t k = lane;
        if (est) {
            const uint32_t *f = adj2 + rp[u];  // F(u): the probed vertices
            for (; k < fu; k += 32) {
                const uint4 m = vmeta[f[k]];
                w0 += (unsigned long long)m.z + m.w;
            }
        } else {
            for (; k + 96 < fu; k += 128) {  // four independent loads in flight
                w0 += rec[k].z;
                w1 += rec[k + 32].z;
                w2 += rec[k + 64].z;
                w3 += rec[k + 96].z;
            }
            for (; k < fu; k += 32) w0 += rec[k].z;
        }
        const unsigned long long work = warp_sum(w0 + w1 + w2 + w3);
        if (lane == 0) {
            const unsigned long long su = (rp[u + 1] - rp[u]) - fu;
            const unsigned long long floor_t = (unsigned long long)min_mult * su;
            const unsigned long long target = floor_t > task_work ? floor_t : task_work;
            unsigned long long nt = (work + target - 1) / target;
            const unsigned long long by_v = (fu + max_v - 1) / max_v;
            if (nt < by_v) nt = by_v;
            if (nt < 1) nt = 1;
            if (nt > fu) nt = fu;
            ntask[i] = (uint32_t)nt;
        }
    }
}

__global__ void k_e0(uint32_t n, const uint64_t *__restrict__ eoff, Ctl *ctl) { ctl->e0 = eoff[n]; }

// The probe records of the edges of tasks [first, last) of one class only (a
// shard's share): one warp per task, one edge per lane, the same record as
// k_records (p = the elements of the descending A(v) ranked below u, by a
// binary search; all of A(v) when it was left unsorted).
__global__ void k_records_tasks(const uint2 *__restrict__ tasks, unsigned long long first, unsigned long long last,
                                const uint32_t *__restrict__ rows, const uint32_t *__restrict__ ntask,
                                const uint64_t *__restrict__ rp, const uint32_t *__restrict__ fcnt,
                                const uint64_t *__restrict__ eoff, const uint32_t *__restrict__ adj2,
                                const uint2 *__restrict__ lv, const uint4 *__restrict__ vmeta,
                                uint4 *__restrict__ erec, const uint32_t *__restrict__ fence) {
    const unsigned lane = lane_id();
    const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long t = first + (((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < last;
         t += warps) {
        const uint2 task = tasks[t];
        const uint32_t u = rows[task.x], nt = ntask[task.x], fu = fcnt[u];
        const uint32_t k_lo = (uint32_t)((uint64_t)task.y * fu / nt), k_hi = (uint32_t)((uint64_t)(task.y + 1) * fu / nt);
        const uint32_t ru = lv[u].x;
        const uint64_t fb = rp[u], e_base = eoff[u];
        for (uint32_t k = k_lo + lane; k < k_hi; k += 32) {
            const uint32_t v = adj2[fb + k];
            const uint4 m = vmeta[v];
            const uint64_t as = ((uint64_t)m.y << 32) | m.x;
            const uint32_t av = m.z;
            uint32_t p = av;  // an unsorted A part is probed whole
            if (av <= kSortCap) {
                uint32_t lo = 0, hi = av;  // first position holding a rank below u's
                if (av > 32) fence_search(fence, as, av, ru, &lo, &hi);
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (adj2[as + mid] < ru) hi = mid; else lo = mid + 1;
                }
                p = av - lo;
            }
            const uint64_t start = as + av - p;
            erec[e_base + k] = make_uint4((uint32_t)start, (uint32_t)(start >> 32), m.w + p, p);
        }
    }
}

__global__ void k_task_totals(Ctl *ctl, const unsigned long long *__restrict__ p0,
                              const unsigned long long *__restrict__ p1, const unsigned long long *__restrict__ p2) {
    ctl->n_tasks[0] = p0[ctl->n_rows[0]];
    ctl->n_tasks[1] = p1[ctl->n_rows[1]];
    ctl->n_tasks[2] = p2[ctl->n_rows[2]];
}

__global__ void k_emit(const uint32_t *__restrict__ ntask, const unsigned long long *__restrict__ tpref, uint32_t nr,
                       uint2 *__restrict__ tasks) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        const unsigned long long base = tpref[i];
        const uint32_t nt = ntask[i];
        for (uint32_t t = 0; t < nt; ++t) tasks[base + t] = make_uint2(i, t);
    }
}

unsigned grid_for(uint64_t work, unsigned threads, unsigned cap) {
    uint64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

tc_status build_rows(tc_ctx *ctx, const PipeBufs &b, uint32_t n, uint32_t max_deg) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    const Tuning &tu = ctx->tune;
    if (n == 0) return TC_OK;
    uint32_t launches = 1;
    const uint32_t g1_lo = ctx->split_R;
    if (b.lvp)
        k_row_fill<true><<<grid_for(n, kFillThreads, cap), kFillThreads, 0, s>>>(
            n, b.rp, b.col, b.lv, b.lvp, b.adj2, b.fcnt, b.gcnt, b.vmeta, b.big, b.huge, ctx->d_ctl, g1_lo, b.glo,
            b.part);
    else
        k_row_fill<false><<<grid_for(n, kFillThreads, cap), kFillThreads, 0, s>>>(
            n, b.rp, b.col, b.lv, b.lvp, b.adj2, b.fcnt, b.gcnt, b.vmeta, b.big, b.huge, ctx->d_ctl, g1_lo, b.glo,
            b.part);
    if (max_deg > kHugeRow) {
        if (b.lvp)
            k_row_fill_huge<true><<<(unsigned)ctx->num_sms, 1024, 0, s>>>(b.huge, ctx->d_ctl, b.rp, b.col, b.lv, b.lvp,
                                                                         b.adj2, b.fcnt, b.gcnt, b.vmeta, b.big, g1_lo,
                                                                         b.glo);
        else
            k_row_fill_huge<false><<<(unsigned)ctx->num_sms, 1024, 0, s>>>(b.huge, ctx->d_ctl, b.rp, b.col, b.lv, b.lvp,
                                                                          b.adj2, b.fcnt, b.gcnt, b.vmeta, b.big,
                                                                          g1_lo, b.glo);
        ++launches;
    }
    if (g1_lo && max_deg > kWarpA) {
        const int smem = (int)(4 * kHugeRow);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_g1_split, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_g1_split<<<(unsigned)ctx->num_sms, 1024, smem, s>>>(b.part, ctx->d_ctl, b.rp, b.gcnt, b.adj2, g1_lo, b.glo);
        ++launches;
    }
    if (max_deg > kWarpA) {
        const int smem = (int)(4 * kSortCap);
        TC_CUDA(ctx, cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_sort_big<<<(unsigned)ctx->num_sms, 1024, smem, s>>>(b.big, ctx->d_ctl, b.rp, b.fcnt, b.gcnt, b.adj2);
        ++launches;
    }
    k_fence<<<cap, 256, 0, s>>>(b.adj2, b.slots, b.fence);
    ++launches;
    launches += scan_u32_to_u64(b.fcnt, b.eoff, n, b.scan_tmp, s);
    // a count split into shards builds each shard's records after planning (records_for_shard)
    const bool sharded = ctx->nshards > 1;
    if (sharded) {
        k_e0<<<1, 1, 0, s>>>(n, b.eoff, ctx->d_ctl);
    } else {
        k_chunk_rows<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.eoff, b.chunk_row);
        k_records<<<cap, 256, 0, s>>>(n, b.eoff, b.chunk_row, b.rp, b.adj2, b.lv, b.vmeta, b.erec, ctx->d_ctl,
                                      b.fence);
    }
    // fdeg and R are free after the levels: class of every vertex, 0/1 indicator
    k_class_flags<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.fcnt, b.gcnt, b.deg, b.fdeg, ctx->d_ctl, tu.warp_cap,
                                                        tu.block_cap, tu.tiny_cap, g1_lo, block_hi_cap(tu, g1_lo),
                                                        b.glo, b.lv);
    launches += sharded ? 2 : 3;
    // class lists in the working order; a count split into shards keeps the vertex order, in which
    // contiguous slices of a task list carry about equal work (in the working order the first
    // shard would get every large task)
    const unsigned long long *order = sharded ? nullptr : b.order;
    for (uint32_t c = 0; c < 4; ++c) {
        k_class_indicator<<<grid_for(n, 256, cap), 256, 0, s>>>(n, b.fdeg, c, b.R, order);
        launches += 2 + scan_u32_to_u64(b.R, b.fpref, n, b.scan_tmp, s);
        k_class_scatter<<<grid_for(n, 256, cap), 256, 0, s>>>(
            n, b.fdeg, c, reinterpret_cast<const unsigned long long *>(b.fpref), b.rows[c], &ctx->d_ctl->n_rows[c],
            order);
    }
    const uint32_t work[3] = {tu.warp_task_work, tu.task_work, tu.hub_task_work};
    const uint32_t mult[3] = {1, 2, 2};
    const uint32_t maxv[3] = {0xFFFFFFFFu, tu.max_v, hub_max_v(tu, g1_lo)};
    for (int c = 0; c < 3; ++c) {
        k_plan<<<grid_for((uint64_t)n * 32, 256, cap), 256, 0, s>>>(b.rows[c], &ctx->d_ctl->n_rows[c], b.rp, b.fcnt,
                                                                    b.eoff, b.erec, b.ntask[c], work[c], mult[c],
                                                                    maxv[c], sharded, b.adj2, b.vmeta);
        ++launches;
    }
    note_launch(ctx, launches);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

// After the host has read n_rows: scan the task counts, publish the totals.
tc_status plan_scans(tc_ctx *ctx, const PipeBufs &b) {
    cudaStream_t s = ctx->stream;
    uint32_t launches = 1;
    for (int c = 0; c < 3; ++c)
        launches += scan_u32_to_u64(b.ntask[c], b.tpref[c], ctx->h_ctl->n_rows[c], b.scan_tmp, s);
    k_task_totals<<<1, 1, 0, s>>>(ctx->d_ctl, reinterpret_cast<const unsigned long long *>(b.tpref[0]),
                                  reinterpret_cast<const unsigned long long *>(b.tpref[1]),
                                  reinterpret_cast<const unsigned long long *>(b.tpref[2]));
    note_launch(ctx, launches);
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

// A count split into shards: the probe records of this shard's tasks
// (share ctx->shard of ctx->nshards of every class's task list, as the
// intersections take them), after the tasks are emitted.
tc_status records_for_shard(tc_ctx *ctx, const PipeBufs &b) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    for (int c = 0; c < 3; ++c) {
        const unsigned long long total = ctx->h_ctl->n_tasks[c];
        const unsigned long long lo = total * ctx->shard / ctx->nshards;
        const unsigned long long hi = total * (ctx->shard + 1) / ctx->nshards;
        if (hi <= lo) continue;
        k_records_tasks<<<grid_for((hi - lo) * 32, 256, cap), 256, 0, s>>>(b.tasks[c], lo, hi, b.rows[c], b.ntask[c],
                                                                           b.rp, b.fcnt, b.eoff, b.adj2, b.lv,
                                                                           b.vmeta, b.erec, b.fence);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

tc_status emit_tasks(tc_ctx *ctx, PipeBufs &b) {
    cudaStream_t s = ctx->stream;
    const unsigned cap = (unsigned)ctx->num_sms * 16u;
    uint64_t off = 0;
    for (int c = 0; c < 3; ++c) {
        b.tasks[c] = b.task_pool + off;
        off += ctx->h_ctl->n_tasks[c];
    }
    if (off > b.task_cap) return set_error(ctx, TC_ERR_OOM, "task list exceeds its bound");
    for (int c = 0; c < 3; ++c) {
        const uint32_t nr = ctx->h_ctl->n_rows[c];
        if (!nr) continue;
        k_emit<<<grid_for(nr, 256, cap), 256, 0, s>>>(b.ntask[c], reinterpret_cast<const unsigned long long *>(b.tpref[c]),
                                                     nr, b.tasks[c]);
        note_launch(ctx);
    }
    TC_CUDA(ctx, cudaGetLastError());
    return TC_OK;
}

}  // namespace tc
