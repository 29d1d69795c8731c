// K6: the particle step (Secs. 2.2, 2.3, 3.3, 3.4; Algorithm 1): one RK4 step
// of every species (Eq. 12 tracers, Eq. 14 inertial) in one launch, between
// fluid levels n and n+1, fused with the gathers (Eqs. 15-22), the time blend
// (Eqs. 23-24) and the wrap/carry write-back of the split-precision state
// (cell, FP32 offset, int32 image; see particles.cu).
#include "common.cuh"
#include "stages.cuh"

#include <algorithm>

namespace el {
namespace {

constexpr int kRK4MaxThreads = 512;
// Blocks of kRK4MaxThreads per SM the kernels are compiled for, which caps
// their registers (2 -> 64, 3 -> 40): occupancy hides the two dependent
// memory round trips of a particle (state, then stencil).
#ifndef EL_RK4_BILINEAR_MIN_BLOCKS
#define EL_RK4_BILINEAR_MIN_BLOCKS 3
#endif
#ifndef EL_RK4_CUBIC_MIN_BLOCKS
#define EL_RK4_CUBIC_MIN_BLOCKS 1
#endif
// The cubic kernels' register caps, EL_RK4_CUBIC_MAXNREG and
// EL_RK4_SHARED_MAXNREG, are in stages.cuh (the batched kernels take them too).
// EL_GATHER_AUTO takes the warp-shared patch from this many particles per
// cell (of the densest species) on.  Measured (Catmull-Rom, St = 1): 1 per
// cell (1024^2, 1M a species) registers 0.110 ms, shared 0.175 ms; 4 per
// cell (2048^2, 16M) 0.434 / 0.383 ms; 16 per cell (1024^2, 16M) 0.395 /
// 0.344 ms.
#ifndef EL_RK4_SHARED_DENSITY
#define EL_RK4_SHARED_DENSITY 2.0
#endif

struct RK4Args {
    const float4* snap;
    const float2* psi;        // streamfunction pair (tracer_velocity = 1), else nullptr
    const SpeciesDev* table;  // device-resident: the sort flips `cur` there
    int n, log2n;
    float dt, h;              // h = dt * n / (2 pi): grid units per unit velocity
    unsigned block_begin[kMaxSpecies];
    KinArgs kin;              // EL_ANALYTIC only: the prescribed field at the stage times
    uint32_t* check;          // EL_CHECK_BOUNDS builds: the flow's violation words
    int prefetch;             // particles ahead whose state a block prefetches into L2 (0: none)
};

// The species of block b: the largest k with block_begin[k] <= b (ascending;
// slots past the last species hold UINT_MAX), by a three-step binary search.
__device__ __forceinline__ int species_of(const unsigned (&begin)[kMaxSpecies], unsigned b) {
    static_assert(kMaxSpecies == 8, "three halvings");
    int s = 0;
    if (b >= begin[s + 4]) s += 4;
    if (b >= begin[s + 2]) s += 2;
    if (b >= begin[s + 1]) s += 1;
    return s;
}

// K6: one RK4 step of every species in one launch (blocks are split between
// species by block_begin), between levels n and n+1 (rk4_particle).  One
// block per run of particles: at the register cap that gives 75 % occupancy
// a grid-stride loop over runs measured 15-18 % slower (more spills, and a
// block no longer retires between runs).
//
// SHARED (cubic schemes only): the warp-shared stencil patch (PatchStencil)
// instead of each thread's register copy of its cell's stencil; the same
// arithmetic on the same values, so the same bits.
//
// BESIDE (bilinear only): the instantiation launched beside the fluid branch
// of the overlapped step, which carries the bilinear carve-out preference
// (EL_SMEM_CARVEOUT_BILINEAR); the particle-only step (a single step, the
// last step of a call) launches the other, which keeps the driver's choice
// and with it the larger L1.  The same code, so the same bits.
template <int SCHEME, bool PSI, bool SHARED, bool BESIDE = false>
__global__ void __launch_bounds__(kRK4MaxThreads, SCHEME == 0 ? EL_RK4_BILINEAR_MIN_BLOCKS : EL_RK4_CUBIC_MIN_BLOCKS)
    __maxnreg__(SHARED ? EL_RK4_SHARED_MAXNREG : (SCHEME == 1 || SCHEME == 2 ? EL_RK4_CUBIC_MAXNREG : 128))
    k_rk4(const __grid_constant__ RK4Args a) {
    const int s = species_of(a.block_begin, blockIdx.x);
    const SpeciesDev& sd = a.table[s];
    const int first = (int)(blockIdx.x - a.block_begin[s]) * (int)blockDim.x;
    prefetch_state(sd, first, a.prefetch);
    const int p = first + (int)threadIdx.x;
    const bool active = p < sd.np;
#if EL_CHECK_BOUNDS
    if (active) {
        const uint32_t c = sd.cell[sd.cur][p];
        const float2 o = sd.off[sd.cur][p];
        const bool bad = (c & 0xffffu) >= (uint32_t)a.n || (c >> 16) >= (uint32_t)a.n ||
                         !(o.x >= 0.f && o.x < 1.f) || !(o.y >= 0.f && o.y < 1.f);
        if (bad && atomicAdd(a.check, 1u) == 0u) {
            a.check[1] = (uint32_t)p;
            a.check[2] = (uint32_t)s;
        }
    }
#endif
    if constexpr (SHARED) {
        // warp-shared stencils: every lane of the warp takes part
        static_assert(SCHEME == 1 || SCHEME == 2, "the shared patch serves the cubic schemes");
        extern __shared__ float2 el_patch[];
        if (PSI && !sd.inertial) {  // the streamfunction path (the same for the whole block)
            if (active) rk4_psi_tracer<SCHEME>(a.psi, a.n, a.log2n, a.h, sd, p);
            return;
        }
        rk4_particle_coop<SCHEME>(a.snap, a.n, a.log2n, a.dt, a.h, sd, p, active,
                                  el_patch + (threadIdx.x >> 5) * (3 * kPatchCap));
    } else {
        if (!active) return;
        rk4_particle<SCHEME, PSI>(a.snap, a.psi, a.n, a.log2n, a.dt, a.h, sd, p, &a.kin);
    }
}
}  // namespace

bool rk4_shared_gather(int interp, int gather, double density) {
    if (interp != EL_CATMULL_ROM && interp != EL_BSPLINE) return false;
    return gather == EL_GATHER_SHARED || (gather == EL_GATHER_AUTO && density >= EL_RK4_SHARED_DENSITY);
}

// Dynamic shared memory of a particle-step block of `threads` threads: the
// warps' stencil patches with the shared gather, none otherwise.
size_t rk4_patch_bytes(bool shared, int threads) {
    return shared ? (size_t)(threads / 32) * 3 * kPatchCap * sizeof(float2) : 0;
}

// Allow the shared-gather kernels the dynamic shared memory of 512-thread
// blocks (above the 48 KiB default) on the current device.
template <int SCHEME, bool PSI>
static cudaError_t rk4_allow_smem() {
    return cudaFuncSetAttribute(k_rk4<SCHEME, PSI, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rk4_patch_bytes(true, kRK4MaxThreads));
}

// Launch attributes of the flow's particle kernels, set when the flow is
// created (outside any stream capture) on its device.
template <int SCHEME>
static cudaError_t rk4_set_carveout() {
    if constexpr (SCHEME == 0) {
        constexpr int cv = EL_SMEM_CARVEOUT_BILINEAR;
        cudaError_t e = set_carveout(k_rk4<0, false, false, true>, cv);
        if (e == cudaSuccess) e = set_carveout(k_rk4<0, true, false, true>, cv);
        return e;
    }
    constexpr int cv = EL_SMEM_CARVEOUT_CUBIC;
    cudaError_t e = set_carveout(k_rk4<SCHEME, false, false>, cv);
    if (e == cudaSuccess) e = set_carveout(k_rk4<SCHEME, true, false>, cv);
    if constexpr (SCHEME == 1 || SCHEME == 2) {
        if (e == cudaSuccess) e = set_carveout(k_rk4<SCHEME, false, true>, cv);
        if (e == cudaSuccess) e = set_carveout(k_rk4<SCHEME, true, true>, cv);
    }
    return e;
}

el_status rk4_prepare(el_flow* f) {
    if (f->d.interp == EL_CATMULL_ROM) {
        EL_CUDA_OK(f, (rk4_allow_smem<1, false>()));
        EL_CUDA_OK(f, (rk4_allow_smem<1, true>()));
        EL_CUDA_OK(f, rk4_set_carveout<1>());
    } else if (f->d.interp == EL_BSPLINE) {
        EL_CUDA_OK(f, (rk4_allow_smem<2, false>()));
        EL_CUDA_OK(f, (rk4_allow_smem<2, true>()));
        EL_CUDA_OK(f, rk4_set_carveout<2>());
    } else if (f->d.interp == EL_BILINEAR) {
        EL_CUDA_OK(f, rk4_set_carveout<0>());
    }
    return EL_OK;
}

// Resident blocks of k_rk4 on the whole GPU at the flow's block size.
template <int SCHEME, bool PSI, bool SHARED>
static int rk4_wave_blocks(int threads) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rk4<SCHEME, PSI, SHARED>, threads,
                                                  rk4_patch_bytes(SHARED, threads));
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

// The prefetch distance of k_rk4 in particles, cached per block size and
// gather: EL_RK4_PREFETCH_WAVES resident waves (SMs x resident blocks), a
// whole number of blocks.
static int rk4_prefetch_distance(el_flow* f, bool shared) {
    const int T = f->rk4_threads;
    const int key = T + (shared ? 1024 : 0);
    if (f->prefetch_threads == key) return f->prefetch_particles;
    int wave = 0;
    const bool psi = f->psi_plane >= 0;
    switch (f->d.interp) {
        case EL_BILINEAR:
            wave = psi ? rk4_wave_blocks<0, true, false>(T) : rk4_wave_blocks<0, false, false>(T);
            break;
        case EL_CATMULL_ROM:
            wave = shared ? (psi ? rk4_wave_blocks<1, true, true>(T) : rk4_wave_blocks<1, false, true>(T))
                          : (psi ? rk4_wave_blocks<1, true, false>(T) : rk4_wave_blocks<1, false, false>(T));
            break;
        case EL_BSPLINE:
            wave = shared ? (psi ? rk4_wave_blocks<2, true, true>(T) : rk4_wave_blocks<2, false, true>(T))
                          : (psi ? rk4_wave_blocks<2, true, false>(T) : rk4_wave_blocks<2, false, false>(T));
            break;
        default: wave = rk4_wave_blocks<3, false, false>(T); break;
    }
    f->prefetch_particles = (int)((double)wave * EL_RK4_PREFETCH_WAVES + 0.5) * T;
    f->prefetch_threads = key;
    return f->prefetch_particles;
}

// K6 for every species of the flow in one launch, step number `step`
// (levels step and step + 1: pair snap[step % 2]); `beside`: launched beside
// the fluid branch (the bilinear kernel's carve-out variant).
el_status particles_step_all(el_flow* f, int64_t step, bool beside) {
    NvtxRange range("particles_step");
    RK4Args a{};
    a.snap = f->snap[step % 2];
    a.psi = f->psi_plane >= 0 ? f->psi[step % 2] : nullptr;
    a.table = f->table;
    a.check = f->check;
    a.n = f->n;
    a.log2n = f->log2n;
    a.dt = (float)f->d.dt;
    a.h = (float)(f->d.dt * (double)f->n / kTwoPi);
    double density = 0.0;  // particles per cell of the densest species
    for (int s = 0; s < f->d.max_species; s++)
        density = std::max(density, (double)f->sp[s].np / (double)f->n2);
    const bool shared = rk4_shared_gather(f->d.interp, f->gather, density);
    a.prefetch = rk4_prefetch_distance(f, shared);
    unsigned blocks = 0;
    int ns = 0;
    for (int s = 0; s < f->d.max_species; s++) {
        // every slot up to the last non-empty one takes part (empty ones get no blocks)
        a.block_begin[s] = blocks;
        blocks += f->sp[s].np > 0 ? blocks_for(f->sp[s].np, f->rk4_threads) : 0;
        if (f->sp[s].np > 0) ns = s + 1;
    }
    if (ns == 0) return EL_OK;
    // empty slots share block_begin with the next slot, so the last slot with
    // a given block_begin (the non-empty one) wins the select in the kernel;
    // slots past max_species are never selected
    for (int s = f->d.max_species; s < kMaxSpecies; s++) a.block_begin[s] = 0xffffffffu;
    const int T = f->rk4_threads;
    const size_t smem = rk4_patch_bytes(shared, T);
    cudaStream_t st = f->stream;
    const bool psi = f->psi_plane >= 0;
    if (f->d.interp == EL_ANALYTIC) {
        a.kin = kinematic_stage_args(f, step);
        k_rk4<3, false, false><<<blocks, T, 0, st>>>(a);
    } else if (f->d.interp == EL_BILINEAR) {
        if (beside) {
            if (psi) k_rk4<0, true, false, true><<<blocks, T, 0, st>>>(a);
            else k_rk4<0, false, false, true><<<blocks, T, 0, st>>>(a);
        } else {
            if (psi) k_rk4<0, true, false><<<blocks, T, 0, st>>>(a);
            else k_rk4<0, false, false><<<blocks, T, 0, st>>>(a);
        }
    } else if (f->d.interp == EL_CATMULL_ROM) {
        if (shared) {
            if (psi) k_rk4<1, true, true><<<blocks, T, smem, st>>>(a);
            else k_rk4<1, false, true><<<blocks, T, smem, st>>>(a);
        } else {
            if (psi) k_rk4<1, true, false><<<blocks, T, 0, st>>>(a);
            else k_rk4<1, false, false><<<blocks, T, 0, st>>>(a);
        }
    } else {
        if (shared) {
            if (psi) k_rk4<2, true, true><<<blocks, T, smem, st>>>(a);
            else k_rk4<2, false, true><<<blocks, T, smem, st>>>(a);
        } else {
            if (psi) k_rk4<2, true, false><<<blocks, T, 0, st>>>(a);
            else k_rk4<2, false, false><<<blocks, T, 0, st>>>(a);
        }
    }
    EL_LAUNCHED(f);
    return EL_OK;
}

}  // namespace el
