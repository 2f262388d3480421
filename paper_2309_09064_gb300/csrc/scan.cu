// scan.cu -- device exclusive prefix sums (reduce, scan of tile sums, scan of tiles).
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr uint64_t kTile = (uint64_t)kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ unsigned long long block_exclusive(unsigned long long v, unsigned long long *total) {
    __shared__ unsigned long long warp_tot[32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= (unsigned)o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long before = warp ? warp_tot[warp - 1] : 0ull;
    *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const T *in, uint64_t count, unsigned long long *sums) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t j = base + (uint64_t)i * kScanThreads + threadIdx.x;
        if (j < count) s += in[j];
    }
    unsigned long long tot;
    block_exclusive<T>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// In-place exclusive scan of nb tile sums by one block, chunk by chunk.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(unsigned long long *sums, uint64_t nb) {
    unsigned long long carry = 0;
    for (uint64_t c = 0; c < nb; c += kTile) {
        unsigned long long v[kScanItems];
        unsigned long long s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            uint64_t j = c + (uint64_t)threadIdx.x * kScanItems + i;
            v[i] = j < nb ? sums[j] : 0ull;
            s += v[i];
        }
        unsigned long long tot;
        unsigned long long ex = block_exclusive<unsigned long long>(s, &tot);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            uint64_t j = c + (uint64_t)threadIdx.x * kScanItems + i;
            if (j < nb) sums[j] = carry + ex;
            ex += v[i];
        }
        carry += tot;
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const T *in, unsigned long long *out, uint64_t count,
                                                              const unsigned long long *sums) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kScanItems;
    unsigned long long v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t j = base + i;
        v[i] = j < count ? (unsigned long long)in[j] : 0ull;
        s += v[i];
    }
    unsigned long long tot;
    unsigned long long ex = block_exclusive<T>(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t j = base + i;
        if (j < count) out[j] = ex;
        ex += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = sums[blockIdx.x] + tot;
}

__global__ void k_zero_total(unsigned long long *out) { out[0] = 0ull; }

template <class T>
uint32_t scan_impl(const T *in, uint64_t *out, uint64_t count, uint64_t *tmp, cudaStream_t s) {
    if (count == 0) {
        k_zero_total<<<1, 1, 0, s>>>(reinterpret_cast<unsigned long long *>(out));
        return 1;
    }
    const uint64_t nb = (count + kTile - 1) / kTile;
    auto *sums = reinterpret_cast<unsigned long long *>(tmp);
    auto *o = reinterpret_cast<unsigned long long *>(out);
    k_tile_sums<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, count, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb);
    k_scan_tiles<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, o, count, sums);
    return 3;
}

}  // namespace

size_t scan_tmp_elems(uint64_t count) { return (size_t)((count + kTile - 1) / kTile + 1); }

uint32_t scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t count, uint64_t *tmp, cudaStream_t s) {
    return scan_impl<uint32_t>(in, out, count, tmp, s);
}

uint32_t scan_u64(const uint64_t *in, uint64_t *out, uint64_t count, uint64_t *tmp, cudaStream_t s) {
    return scan_impl<unsigned long long>(reinterpret_cast<const unsigned long long *>(in), out, count, tmp, s);
}

}  // namespace tc
