// Internal declarations shared by the translation units of libelpath.so.
// Nothing here is part of the public ABI (include/elpath.h).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/elpath.h"

namespace el {

constexpr int kMaxSpecies = EL_MAX_SPECIES;
constexpr int kBoxes = 64;          // clustering-index box grid (kBoxes x kBoxes)
constexpr int kRedBlocks = 512;     // fixed grid of the FP64 reductions (fixed order)
constexpr int kRedThreads = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// EL_CHECK_BOUNDS=1 builds a debug library whose particle kernel checks each
// particle's split state (cell indices below n, offsets in [0, 1)) before
// its step and counts violations in a device word (no trap); el_get_stats
// then reports them as EL_ESTATE.
#ifndef EL_CHECK_BOUNDS
#define EL_CHECK_BOUNDS 0
#endif

// Device-resident descriptor of one species, read by the particle step.
// `cur` selects the current buffer of each pair; the sort flips it on the
// device, so a captured step graph stays valid across re-binning.
struct SpeciesDev {
    uint32_t* cell[2];
    float2* off[2];
    float2* vel[2];
    int2* img[2];
    int np;
    int cur;
    int inertial;
    float inv_st;
};

// One particle species (host view).  Structure-of-arrays in two buffers
// (cur = current, cur ^ 1 = the sort's target, also used as staging).
struct Species {
    int cur = 0;
    int64_t np = 0;
    int64_t cap = 0;
    double st = 0.0;
    uint32_t* cell[2] = {nullptr, nullptr};  // i | j << 16
    float2* off[2] = {nullptr, nullptr};     // in-cell offset, [0, 1)^2
    float2* vel[2] = {nullptr, nullptr};     // particle velocity (inertial only)
    int2* img[2] = {nullptr, nullptr};       // periodic image count per axis
    uint32_t* id[2] = {nullptr, nullptr};    // original index
    double2* x0 = nullptr;                   // reference position, indexed by id
    uint32_t* rank = nullptr;                // sort scratch
};

}  // namespace el

struct el_batch;

struct el_flow {
    el_flow_desc d{};
    cudaStream_t stream = nullptr;
    int device = 0;

    // geometry
    int n = 0, nh = 0, log2n = 0;
    size_t n2 = 0, nmodes = 0;
    int nplanes = 4;         // u, v, wx, wy [, prefiltered cu, cv] [, psi stencil]
    int stencil_plane = 0;   // plane holding the u the particle stencil weights
    int psi_plane = -1;      // plane of the streamfunction stencil field, or -1

    // workspace carve-out
    char* ws = nullptr;
    size_t ws_bytes = 0;

    // fluid state (device)
    float2* what = nullptr;   // omega-hat, half spectrum [ky][kx], n x (n/2+1)
    float2* what_lo = nullptr;  // low part of omega-hat (compensated storage)
    float2* hist = nullptr;   // AB2 history
    float2* nhat = nullptr;   // nonlinear term of the latest level
    float2* spec = nullptr;   // nplanes half spectra (C2R input)
    float* phys = nullptr;    // nplanes physical planes (C2R output)
    float* nl = nullptr;      // physical nonlinear term (R2C input)
    float4* snap[2] = {nullptr, nullptr};  // level pairs: snap[k % 2] = levels (k, k+1) per node
    float2* psi[2] = {nullptr, nullptr};   // streamfunction level pairs (tracer_velocity = 1)
    float2* aux_spec = nullptr;
    float* aux_phys = nullptr;
    double* stage64 = nullptr;  // n^2 doubles: host <-> device field staging
    float2* ex = nullptr;     // exp(-nu kx^2 dt) as (hi, lo) floats, kx = 0..n/2
    float2* ey = nullptr;     // exp(-nu ky^2 dt) as (hi, lo) floats, row index 0..n-1
    float2* twiddle = nullptr;  // exp(-2 pi i m / n), m < n (the fused step's transforms)
    bool fused = false;         // the fluid step runs the fused kernels (fused_fluid.cu)
    float* pre_x = nullptr;   // spline prefilter 3/(2 + cos(k dx)) per kx
    float* pre_y = nullptr;   // ... per row index
    el::SpeciesDev* table = nullptr;  // device copy of h_table
    el::SpeciesDev h_table[el::kMaxSpecies] = {};
    uint32_t* check = nullptr;    // EL_CHECK_BOUNDS builds: violations, first particle, its species
    unsigned long long* bad_input = nullptr;  // first bad index of an uploaded particle set
    double* red = nullptr;        // reduction partials
    double* red_out = nullptr;    // reduced scalars (device)
    unsigned long long* boxes = nullptr;  // kBoxes^2 counters
    uint32_t* bins = nullptr;     // n^2 sort bins
    uint32_t* bin_sums = nullptr; // scan block sums
    void* fft_work = nullptr;
    char* pool = nullptr;         // particle pool
    size_t pool_bytes = 0, pool_used = 0;

    cufftHandle plan_c2r = 0, plan_r2c = 0, plan_c2r1 = 0;
    bool plans_made = false;

    el::Species sp[el::kMaxSpecies];

    int64_t step = 0;          // coupled steps taken
    int rk4_threads = 256;     // threads per block of the particle step (tunable)
    int gather = EL_GATHER_AUTO;  // cubic schemes' stencil gather (tunable)
    int prefetch_threads = 0;  // block size (and gather, + 1024) the cached prefetch distance is for
    int prefetch_particles = 0;
    int sort_shift = 0;        // re-binning key: tiles of 2^sort_shift cells per side
    el_batch* batch = nullptr; // the batch this flow is a member of, if any
    int fft_pool = -1, fft_slot = -1;  // its slot in one of the batch's FFT pools, if any
    float2* nhat_cur = nullptr;        // N-hat while it lives in that slot (else nhat)
    cudaStream_t own_stream = nullptr;  // stream given at creation (restored on batch removal)
    int64_t since_sort = 0;
    int64_t launches = 0;

    // captured graphs, one per step parity: the fluid step alone, the
    // particle step alone, and particles(n) alongside fluid(n + 1)
    cudaGraphExec_t g_fluid[2] = {}, g_part[2] = {}, g_both[2] = {};
    int64_t k_fluid[2] = {}, k_part[2] = {}, k_both[2] = {};
    cudaStream_t side = nullptr;       // second branch of the overlapped step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    int kinematic = 0;         // 1: the prescribed field of Sec. 5.2 replaces the solver
    el_kinematic kin{};

    std::string err;
};

namespace el {

// NVTX range over a host-side stage of the library (shown by profilers; a
// no-op when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- launch helpers -------------------------------------------------------
inline unsigned blocks_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

el_status fail(el_flow* f, el_status s, const char* fmt, ...);

// Preferred shared-memory carve-out (percent of the SM's unified L1 / shared
// memory) of the particle kernels (bilinear; cubic schemes) and of the fused
// fluid kernels, single-flow and batched; -1 leaves it to the driver.  An SM
// changes its split only when it is empty, so the fluid branch's blocks start
// beside running particle blocks only where the particle kernel left a
// carve-out large enough for them.  Single flow, 1024^2 with 4 x 1M bilinear
// particles, coupled step: 75 / 75 (a 196 KB carve-out) 0.0745 ms against
// 0.0771 ms with the driver's choice; 65 / 65 0.0756, 50 / 50 0.0757, 75 / 65
// 0.0765, 100 / 100 slower (the particle kernel alone loses ~5 % at 75, from
// fewer L1 hits; the overlap gains more).  The cubic kernels lean on L1 for
// their gathers: 2048^2 shear layer (16M Catmull-Rom, patch gather) particle
// launch 0.383 ms with the driver's choice against 0.411 ms at 75, coupled
// step 0.493-0.501 ms with only the fluid kernels at 75 against 0.521-0.530
// with both.
#ifndef EL_SMEM_CARVEOUT_BILINEAR
#define EL_SMEM_CARVEOUT_BILINEAR 75
#endif
#ifndef EL_SMEM_CARVEOUT_CUBIC
#define EL_SMEM_CARVEOUT_CUBIC -1
#endif
#ifndef EL_SMEM_CARVEOUT_FLUID
#define EL_SMEM_CARVEOUT_FLUID 75
#endif
template <class K>
inline cudaError_t set_carveout(K* kernel, int percent) {
    return percent < 0 ? cudaSuccess
                       : cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, percent);
}

#define EL_CUDA_OK(f, call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ::el::fail((f), EL_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                              __FILE__, __LINE__);                                       \
    } while (0)

#define EL_LAUNCHED(f)                                                                   \
    do {                                                                                 \
        (f)->launches++;                                                                 \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess)                                                           \
            return ::el::fail((f), EL_ECUDA, "kernel launch: %s (%s:%d)",                \
                              cudaGetErrorString(e_), __FILE__, __LINE__);               \
    } while (0)

#define EL_TRY(call)                      \
    do {                                  \
        el_status s_ = (call);            \
        if (s_ != EL_OK) return s_;       \
    } while (0)

// ---- fluid (fluid.cu) -------------------------------------------------------
struct SpecArgs;
el_status fluid_init(el_flow* f, const double* omega0_host);
el_status fluid_step(el_flow* f, int64_t step);   // K5+K1, C2R, K3, R2C
el_status fluid_diagnostics(el_flow* f);          // E, Z, P -> red_out[0..2]
// ---- prescribed kinematic flow (kinematic.cu) --------------------------------------
struct KinArgs;
KinArgs kinematic_stage_args(const el_flow* f, int64_t step);  // the field at RK4 stage times
el_status kinematic_level(el_flow* f, int64_t m, bool setup);  // level m into its pair
el_status kinematic_get_field(el_flow* f, int which, double* host_nn);  // omega, u, v at t_n
void kinematic_diagnostics(const el_flow* f, double* e3);  // exact E, Z, P
el_status fluid_refresh_planes(el_flow* f);       // physical planes of the current level
el_status fluid_get_field(el_flow* f, int which, double* host_nn);
// ---- the fused 1024^2 / 2048^2 fluid step (fused_fluid.cu) ----------------------------
bool fused_fluid_supported(const el_flow* f);
el_status fused_fluid_prepare(el_flow* f);
el_status fluid_step_fused(el_flow* f, const SpecArgs& a, int64_t step);
struct FusedMember;
// The fused step of `count` batched flows of grid n with `planes`
// inverse-transform planes (device records d_members), each at its step
// counter + `ahead`; twiddle: the n-entry table of any of them.
cudaError_t fused_fluid_batch(cudaStream_t s, const FusedMember* d_members, int count, int n, int planes,
                              int ahead, const float2* twiddle);
cudaError_t fused_fluid_batch_prepare(int n, int planes);

// ---- flow descriptors (api.cu) ----------------------------------------------------
const char* flow_desc_problem(const el_flow_desc* d);  // nullptr when the descriptor is valid
int flow_planes(const el_flow_desc& d);                // spectral planes of the inverse FFT

// ---- particles (particles.cu; the RK4 step in rk4.cu) ----------------------------
el_status particles_set(el_flow* f, int s, int64_t np, double st, const double* xy,
                        const double* vxy);
el_status particles_step_all(el_flow* f, int64_t step, bool beside);  // K6 (rk4.cu), every species in one launch
// K6 with the warp-shared stencil patch?  For scheme `interp` under setting
// `gather`, with `density` = the largest particles-per-cell of a species (rk4.cu).
bool rk4_shared_gather(int interp, int gather, double density);
size_t rk4_patch_bytes(bool shared, int threads);  // dynamic shared memory of a K6 block (rk4.cu)
el_status rk4_prepare(el_flow* f);                 // K6 launch attributes, at flow creation (rk4.cu)
el_status particles_get(el_flow* f, int s, double* xy, double* vxy);
// msd x, msd y, cluster, <dx^4>, <dy^4> (the squared displacements' second moments)
el_status particles_stats_into(el_flow* f, int s, double* out5);
el_status sample_velocity(el_flow* f, int64_t np, const double* d_xy, double theta, double* d_uv);

void drop_graphs(el_flow* f);                     // api.cu
// Would species of np[k] particles (k < max_species) all fit the particle pool?
bool species_fit(const el_flow* f, const int64_t* np);
// Room for np particles in slot s (a slot keeps room it already has).
bool carve_species_slot(el_flow* f, int s, int64_t np);
// Rebuild slot s's entry of the device species table from the host view.
el_status particles_restore_table(el_flow* f, int s);


// ---- sort (sort.cu) -------------------------------------------------------------
el_status particles_sort(el_flow* f, int s);      // K7

// ---- reductions (reduce.cu) ---------------------------------------------------------
// Means of `count` consecutive double2 values, summed in a fixed order, into out2 (device).
el_status reduce_double2(el_flow* f, const double2* in, int64_t count, double* out2);

}  // namespace el
