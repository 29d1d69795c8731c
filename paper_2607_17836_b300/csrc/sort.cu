// K7: counting sort of one species by cell (row-major cell id j * n + i).
//
// Particles that are neighbours in memory then sit in neighbouring cells, so
// the gathers of a warp hit the same few cache lines of the snapshot pair.
// The order inside a cell is whatever the atomics give; nothing downstream
// depends on it (each particle's step is independent of the others, and
// the statistics are reduced in original-index order).
//
//   k_sort_count   : rank[p] = atomicAdd(&bins[key], 1), key = the particle's
//                    tile of 2^shift x 2^shift cells (shift tunable)
//   scan (3 kernels): bins -> exclusive prefix sums (offsets)
//   k_sort_scatter : buffer cur^1 at bins[key] + rank[p] <- buffer cur at p;
//                    then cur flips (in the device species table too, so a
//                    captured step graph follows the swap)
#include "common.cuh"

namespace el {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;  // 4096 bins per block

// Re-binning key of a cell: row-major index of its tile of 2^shift x 2^shift
// cells (shift = 0: the cell itself).
__device__ __forceinline__ uint32_t bin_key(uint32_t c, int log2n, int shift) {
    uint32_t i = (c & 0xffffu) >> shift, j = (c >> 16) >> shift;
    return (j << (log2n - shift)) | i;
}

__global__ void k_sort_count(const uint32_t* __restrict__ cell, int64_t np, int log2n, int shift,
                             uint32_t* __restrict__ bins, uint32_t* __restrict__ rank) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    rank[p] = atomicAdd(bins + bin_key(cell[p], log2n, shift), 1u);
}

// Exclusive scan of one tile of kScanTile values in place; the tile total
// goes to sums[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(uint32_t* __restrict__ data,
                                                            int64_t count,
                                                            uint32_t* __restrict__ sums) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        v[k] = (base + k < count) ? data[base + k] : 0u;
        local += v[k];
    }
    // inclusive scan of the per-thread totals within the warp
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    uint32_t prefix = (warp > 0 ? warp_tot[warp - 1] : 0u) + (x - local);
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        if (base + k < count) data[base + k] = prefix;
        prefix += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = warp_tot[31];
}

__global__ void k_scan_add(uint32_t* __restrict__ data, int64_t count,
                           const uint32_t* __restrict__ sums) {
    int64_t q = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t add = sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; k++)
        if (q + k < count) data[q + k] += add;
}

__global__ void k_sort_scatter(const uint32_t* __restrict__ cell0, const float2* __restrict__ off0,
                               const float2* __restrict__ vel0, const int2* __restrict__ img0,
                               const uint32_t* __restrict__ id0, const uint32_t* __restrict__ rank,
                               const uint32_t* __restrict__ offsets, int64_t np, int log2n,
                               int shift, int inertial, uint32_t* __restrict__ cell1, float2* __restrict__ off1,
                               float2* __restrict__ vel1, int2* __restrict__ img1,
                               uint32_t* __restrict__ id1, SpeciesDev* __restrict__ table,
                               int new_cur) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) table->cur = new_cur;  // read only by later launches
    if (p >= np) return;
    uint32_t c = cell0[p];
    uint32_t d = offsets[bin_key(c, log2n, shift)] + rank[p];
    cell1[d] = c;
    off1[d] = off0[p];
    if (inertial) vel1[d] = vel0[p];
    img1[d] = img0[p];
    id1[d] = id0[p];
}

}  // namespace

// Exclusive scan of `count` (<= kScanTile^2) values in place.
static el_status exclusive_scan(el_flow* f, uint32_t* data, int64_t count) {
    int64_t tiles = (count + kScanTile - 1) / kScanTile;
    if (tiles > kScanTile) return fail(f, EL_EINVAL, "scan of %lld values too large", (long long)count);
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, f->stream>>>(data, count, f->bin_sums);
    EL_LAUNCHED(f);
    if (tiles > 1) {
        k_scan_tile<<<1, kScanThreads, 0, f->stream>>>(f->bin_sums, tiles, f->bin_sums + kScanTile);
        EL_LAUNCHED(f);
        k_scan_add<<<(unsigned)tiles, kScanThreads, 0, f->stream>>>(data, count, f->bin_sums);
        EL_LAUNCHED(f);
    }
    return EL_OK;
}

el_status particles_sort(el_flow* f, int s) {
    Species& sp = f->sp[s];
    if (sp.np < 2) return EL_OK;
    const int T = 256;
    const int a = sp.cur, b = sp.cur ^ 1;
    int inertial = sp.st > 0.0 ? 1 : 0;
    const int shift = f->sort_shift;
    const int64_t nbins = (int64_t)f->n2 >> (2 * shift);
    EL_CUDA_OK(f, cudaMemsetAsync(f->bins, 0, (size_t)nbins * sizeof(uint32_t), f->stream));
    k_sort_count<<<blocks_for(sp.np, T), T, 0, f->stream>>>(sp.cell[a], sp.np, f->log2n, shift,
                                                            f->bins, sp.rank);
    EL_LAUNCHED(f);
    EL_TRY(exclusive_scan(f, f->bins, nbins));
    k_sort_scatter<<<blocks_for(sp.np, T), T, 0, f->stream>>>(
        sp.cell[a], sp.off[a], sp.vel[a], sp.img[a], sp.id[a], sp.rank, f->bins, sp.np, f->log2n,
        shift, inertial, sp.cell[b], sp.off[b], sp.vel[b], sp.img[b], sp.id[b], f->table + s, b);
    EL_LAUNCHED(f);
    sp.cur = b;
    f->h_table[s].cur = b;
    return EL_OK;
}

}  // namespace el
