// Batched engine: many independent simulations (flows of any grid size,
// species mix, scheme and step count) advanced together.  One coupled step of
// the batch is one captured CUDA graph:
//
//   k_batch_spectral  (persistent, every member's modes)   AB2 + velocity planes
//   cuFFT C2R per member, on forked branches (they run concurrently)
//   k_batch_nonlinear (persistent, every member's nodes)   nonlinear term + snapshot
//   cuFFT R2C per member, on forked branches
//     (members in a slot of an FFT pool: one batched C2R and one batched R2C
//     per pool instead, over the pool's contiguous slots)
//   k_batch_rk4<S,G>  (every member's species) RK4 particle step, one launch
//                     per scheme and stencil gather present
//   k_batch_advance                                        per-member step counters
//
// Members whose fluid step is the fused one (fused_fluid.cu)
// take no part in the spectral, cuFFT and nonlinear stages: the fused
// kernels advance all of them at once (one launch of each of the four per
// plane count present, the member in the grid's last dimension).
//
// The per-element arithmetic is the single-flow kernels' (stages.cuh), so a
// member's results do not depend on what else is in the batch.  Each member
// keeps its own step counter on the device (members join and leave at any
// step), so the same graph serves every step until the membership changes.
// Re-binning runs per member, outside the graph, when it is due.
#include "common.cuh"
#include "stages.cuh"
#include "tune.cuh"

#include <algorithm>
#include <cstdarg>
#include <string>
#include <vector>

namespace el {

// Fluid and particle parameters of one member, device-resident.
struct MemberDev {
    SpecArgs spec;          // arrays and constants of k_spectral (first from `step`)
    const float4* phys4;
    float4* nl4;
    float4* snap[2];        // level pairs: snap[k % 2] = levels (k, k+1)
    float2* psi[2];         // streamfunction level pairs, or nullptr
    unsigned long long n4;  // n^2 / 4
    int stencil_plane, psi_plane, n, log2n, scheme;
    float dt, h;
    long long step;
};

struct BatchArgs {
    MemberDev* members;
    const int* spec_begin;            // task prefix sums, nmembers + 1
    const int* nl_begin;
    const int* rk_begin;              // nentries + 1
    const int* rk_member;             // member of each (member, species) entry
    const SpeciesDev* const* rk_sp;   // that member's device species descriptor
    int nmembers, nentries;
    int spec_tasks, nl_tasks, rk_tasks;
    // entries grouped by class c = 2 scheme + gather (gather 1: the
    // warp-shared patch): entries [rk_class_entry[c], rk_class_entry[c + 1]),
    // their tasks [rk_class_task[c], rk_class_task[c + 1]), and the class's
    // state-prefetch distance in particles
    int rk_class_entry[7], rk_class_task[7], rk_prefetch[6];
};

namespace {

constexpr int kBSpecThreads = 128;
constexpr int kBNlThreads = 256;
constexpr int kSideStreams = 4;
constexpr int kRkClasses = 6;  // (scheme, gather) classes of the particle entries

// Largest k in [0, count) with begin[k] <= t (begin ascending, begin[0] = 0).
__device__ __forceinline__ int owner_of(const int* __restrict__ begin, int count, int t) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ __forceinline__ int spec_chunks(int n) {
    int c = (n / 2) / kBSpecThreads;
    return c < 1 ? 1 : c;
}

// `ahead` = 1: the fluid step one past each member's step counter (the
// fluid branch of the overlapped step), 0: the step at the counter.
__global__ void __launch_bounds__(kBSpecThreads) k_batch_spectral(const __grid_constant__ BatchArgs b,
                                                                  int ahead) {
    for (int t = blockIdx.x; t < b.spec_tasks; t += gridDim.x) {
        const int m = owner_of(b.spec_begin, b.nmembers, t);
        const MemberDev& md = b.members[m];
        const int local = t - b.spec_begin[m];
        const int chunks = spec_chunks(md.n);
        const int j = local / chunks, i = (local - j * chunks) * kBSpecThreads + threadIdx.x;
        SpecArgs a = md.spec;
        a.first = md.step + ahead == 0;
        if (i < md.n / 2) {
            spectral_mode<true>(a, i, j);
            if (i == 0) spectral_mode<true>(a, md.n / 2, j);
        }
    }
}

__global__ void __launch_bounds__(kBNlThreads) k_batch_nonlinear(const __grid_constant__ BatchArgs b,
                                                                   int ahead) {
    for (int t = blockIdx.x; t < b.nl_tasks; t += gridDim.x) {
        const int m = owner_of(b.nl_begin, b.nmembers, t);
        const MemberDev& md = b.members[m];
        const size_t i = (size_t)(t - b.nl_begin[m]) * kBNlThreads + threadIdx.x;
        const size_t n2 = 4 * md.n4;
        const long long lv = md.step + 1 + ahead;  // the level this step produces
        if (i < n2)
            nonlinear_node(reinterpret_cast<const float*>(md.phys4), reinterpret_cast<float*>(md.nl4),
                           md.snap[lv % 2], md.snap[(lv + 1) % 2], nullptr, n2, i,
                           md.stencil_plane, md.psi_plane, md.psi[lv % 2], md.psi[(lv + 1) % 2],
                           nullptr);
    }
}

// K6 for task t (a run of one entry's particles) of class c = 2 SCHEME +
// SHARED; the class's entries are [rk_class_entry[c], rk_class_entry[c + 1]).
// SHARED: the warp-shared stencil patch of the cubic schemes (as k_rk4).
template <int SCHEME, bool SHARED>
__device__ __forceinline__ void batch_rk4_task(const BatchArgs& b, int c, int t, int prefetch) {
    const int e0 = b.rk_class_entry[c];
    const int e = e0 + owner_of(b.rk_begin + e0, b.rk_class_entry[c + 1] - e0, t);
    const MemberDev& md = b.members[b.rk_member[e]];
    const SpeciesDev& sd = *b.rk_sp[e];
    const int first = (t - b.rk_begin[e]) * (int)blockDim.x;
    prefetch_state(sd, first, prefetch);
    const int p = first + (int)threadIdx.x;
    const int k = (int)(md.step % 2);
    if constexpr (SHARED) {
        // warp-shared stencils (as in the single-flow kernel): every lane of
        // the warp takes part; the branches are block-uniform
        extern __shared__ float2 el_patch[];
        const bool active = p < sd.np;
        if (md.psi_plane >= 0 && !sd.inertial) {
            if (active) rk4_psi_tracer<SCHEME>(md.psi[k], md.n, md.log2n, md.h, sd, p);
            return;
        }
        rk4_particle_coop<SCHEME>(md.snap[k], md.n, md.log2n, md.dt, md.h, sd, p, active,
                                  el_patch + (threadIdx.x >> 5) * (3 * kPatchCap));
        return;
    }
    if (p >= sd.np) return;
    if (md.psi_plane >= 0)
        rk4_particle<SCHEME, true>(md.snap[k], md.psi[k], md.n, md.log2n, md.dt, md.h, sd, p);
    else
        rk4_particle<SCHEME, false>(md.snap[k], nullptr, md.n, md.log2n, md.dt, md.h, sd, p);
}

// K6 for every entry of one (scheme, gather) class, with the single-flow
// kernel's register caps (stages.cuh).  The cubic classes: one block per task
// with the L2 state prefetch, as in the single-flow kernel (a grid-stride loop
// costs the capped kernels spills; persistent, a batch of one ran 1.2-1.5x
// slower than the flow alone).  The bilinear class (40 registers): a
// persistent grid of one resident wave looping over the tasks, without the
// prefetch; one block per task slowed the 64-member ensemble step, whose
// particle launch runs beside the fluid branch, from 0.910 to 0.977 ms.
template <int SCHEME, bool SHARED>
__global__ void __launch_bounds__(512, SCHEME == 0 ? 3 : 1)
    __maxnreg__(SHARED ? EL_RK4_SHARED_MAXNREG : (SCHEME == 1 || SCHEME == 2 ? EL_RK4_CUBIC_MAXNREG : 128))
    k_batch_rk4(const __grid_constant__ BatchArgs b) {
    constexpr int c = 2 * SCHEME + (SHARED ? 1 : 0);
    if constexpr (SCHEME == 0) {
        for (int t = b.rk_class_task[c] + (int)blockIdx.x; t < b.rk_class_task[c + 1]; t += gridDim.x)
            batch_rk4_task<SCHEME, SHARED>(b, c, t, 0);
    } else {
        batch_rk4_task<SCHEME, SHARED>(b, c, b.rk_class_task[c] + (int)blockIdx.x, b.rk_prefetch[c]);
    }
}

__global__ void k_batch_advance(MemberDev* members, int nmembers) {
    for (int m = threadIdx.x; m < nmembers; m += blockDim.x) members[m].step += 1;
}

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace
}  // namespace el

using namespace el;

// An FFT pool: caller-provided memory holding the transient transform
// buffers of `slots` members of one class (grid n, inverse-FFT planes P) one
// after another, so that one cuFFT plan transforms every slot at once (cuFFT's
// time per plane falls steeply with the batch count).  Slot s: spectral
// planes spec + s P nmodes, physical planes phys + s P n^2, nonlinear term
// nl + s n^2, its transform nhat + s nmodes (N-hat is carried from one step
// to the next, so it moves into the slot when the member joins and back to
// the member when it leaves).
struct FftPool {
    int n = 0, planes = 0, slots = 0;
    size_t nmodes = 0, n2 = 0;
    float2* spec = nullptr;
    float* phys = nullptr;
    float* nl = nullptr;
    float2* nhat = nullptr;
    void* work = nullptr;
    size_t work_bytes = 0;
    // plans over the first k slots, k = 1..slots (0: not made yet); members
    // take the lowest free slot, and the transforms cover slots [0, k) with
    // k one past the highest occupied slot
    std::vector<cufftHandle> c2r, r2c;
    std::vector<el_flow*> member;  // occupant of each slot (nullptr: free)
    int span() const {
        int k = 0;
        for (int i = 0; i < slots; i++)
            if (member[i]) k = i + 1;
        return k;
    }
};

struct el_batch {
    cudaStream_t stream = nullptr;
    std::vector<FftPool> pools;
    int max_members = 0;
    std::vector<el_flow*> members;
    // device tables (in the caller's workspace)
    MemberDev* d_members = nullptr;
    int* d_spec_begin = nullptr;
    int* d_nl_begin = nullptr;
    int* d_rk_begin = nullptr;
    int* d_rk_member = nullptr;
    const SpeciesDev** d_rk_sp = nullptr;
    FusedMember* d_fused = nullptr;
    // host copies (kept alive while their upload may be pending)
    std::vector<MemberDev> h_members;
    std::vector<int> h_spec_begin, h_nl_begin, h_rk_begin, h_rk_member;
    std::vector<const SpeciesDev*> h_rk_sp;
    // fused members' records, grouped by class c = 4 g + planes - 4 with g the
    // grid (n = 128 << g, g < kFusedGrids): records [fused_begin[c], fused_begin[c + 1])
    static constexpr int kFusedGrids = 5;
    std::vector<FusedMember> h_fused;
    int fused_begin[4 * kFusedGrids + 1] = {};
    const float2* fused_twiddle[kFusedGrids] = {};  // the n-entry table of a member of each grid
    BatchArgs args{};
    int grid_spec = 0, grid_nl = 0;
    unsigned grid_bilinear = 1;  // the persistent bilinear particle grid (one resident wave)
    bool tables_valid = false;
    // one coupled step of every member in three captured forms (fluid of
    // step s, particles of s alongside fluid of s + 1, particles of the last
    // step); the fluid branch runs at the highest stream priority
    cudaGraphExec_t graph[3] = {};
    int64_t graph_kernels[3] = {};
    cudaStream_t fluid = nullptr;
    cudaEvent_t f_fork = nullptr, f_join = nullptr;
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kSideStreams] = {};
    int sms = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

el_status bfail(el_batch* b, el_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return s;
}

#define BT_CUDA(b, call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail((b), EL_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));         \
    } while (0)

size_t table_bytes(int max_members) {
    size_t m = (size_t)max_members, e = m * kMaxSpecies;
    return align_up(m * sizeof(MemberDev)) + 2 * align_up((m + 1) * sizeof(int)) +
           2 * align_up((e + 1) * sizeof(int)) + align_up(e * sizeof(void*)) +
           align_up(m * sizeof(FusedMember));
}

MemberDev member_of(const el_batch* b, el_flow* f) {
    MemberDev md{};
    SpecArgs& a = md.spec;
    a.what = f->what;
    a.what_lo = f->what_lo;
    a.hist = f->hist;
    a.nhat = f->nhat;
    a.spec = f->spec;
    a.ex = f->ex;
    a.ey = f->ey;
    a.pre_x = f->pre_x;
    a.pre_y = f->pre_y;
    a.n = f->n;
    a.nh = f->nh;
    a.nplanes = f->nplanes;
    a.spline = f->stencil_plane != 0;
    a.psi_plane = f->psi_plane;
    a.mode = f->d.ab2_mode;
    a.first = 0;
    a.nmodes = f->nmodes;
    a.scale = 1.0f / (float)f->n2;
    a.dt = (float)f->d.dt;
    a.nu = (float)f->d.nu;
    md.phys4 = reinterpret_cast<const float4*>(f->phys);
    md.nl4 = reinterpret_cast<float4*>(f->nl);
    for (int k = 0; k < 2; k++) {
        md.snap[k] = f->snap[k];
        md.psi[k] = f->psi[k];
    }
    md.psi_plane = f->psi_plane;
    md.n4 = f->n2 / 4;
    md.stencil_plane = f->stencil_plane;
    md.n = f->n;
    md.log2n = f->log2n;
    md.scheme = f->d.interp;
    md.dt = (float)f->d.dt;
    md.h = (float)(f->d.dt * (double)f->n / kTwoPi);
    md.step = f->step;
    if (f->fft_pool >= 0) {  // its transform buffers live in a pool slot
        const FftPool& p = b->pools[f->fft_pool];
        const size_t k = (size_t)f->fft_slot;
        a.spec = p.spec + k * p.planes * p.nmodes;
        a.nhat = p.nhat + k * p.nmodes;
        md.phys4 = reinterpret_cast<const float4*>(p.phys + k * p.planes * p.n2);
        md.nl4 = reinterpret_cast<float4*>(p.nl + k * p.n2);
    }
    return md;
}

void ensure_prefix_plans(el_batch* b, FftPool& p, int k);

// Rebuild and upload the member tables, and size the persistent grids.
el_status rebuild_tables(el_batch* b) {
    const int M = (int)b->members.size();
    b->h_members.clear();
    b->h_spec_begin.assign(1, 0);
    b->h_nl_begin.assign(1, 0);
    b->h_rk_begin.assign(1, 0);
    b->h_rk_member.clear();
    b->h_rk_sp.clear();
    int rk_threads = 256;
    for (int m = 0; m < M; m++) {
        el_flow* f = b->members[m];
        rk_threads = f->rk4_threads;  // one block size for the whole batch
        b->h_members.push_back(member_of(b, f));
        const bool own = !f->fused;  // the spectral and nonlinear stages' members
        b->h_spec_begin.push_back(b->h_spec_begin.back() + (own ? f->n * spec_chunks(f->n) : 0));
        b->h_nl_begin.push_back(b->h_nl_begin.back() +
                                (own ? (int)((f->n2 + kBNlThreads - 1) / kBNlThreads) : 0));
    }
    // the fused members' records, grouped by grid and plane count
    b->h_fused.clear();
    for (int g = 0; g < el_batch::kFusedGrids; g++) b->fused_twiddle[g] = nullptr;
    for (int c = 0; c < 4 * el_batch::kFusedGrids; c++) {
        const int n = 128 << (c / 4), planes = 4 + (c & 3);
        b->fused_begin[c] = (int)b->h_fused.size();
        for (int m = 0; m < M; m++) {
            el_flow* f = b->members[m];
            if (!f->fused || f->n != n || f->nplanes != planes) continue;
            FusedMember fm{};
            fm.spec = b->h_members[m].spec;
            fm.S = f->spec;
            fm.G = reinterpret_cast<float2*>(f->phys);
            fm.H = reinterpret_cast<float2*>(f->nl);
            fm.nhat = f->nhat;
            for (int k = 0; k < 2; k++) {
                fm.snap[k] = f->snap[k];
                fm.psi[k] = f->psi[k];
            }
            fm.step = &b->d_members[m].step;
            fm.psi_plane = f->psi_plane;
            b->h_fused.push_back(fm);
            b->fused_twiddle[c / 4] = f->twiddle;  // the same table in every flow of the grid
        }
        if (b->h_fused.size() > (size_t)b->fused_begin[c])
            BT_CUDA(b, fused_fluid_batch_prepare(n, planes));
    }
    b->fused_begin[4 * el_batch::kFusedGrids] = (int)b->h_fused.size();
    BatchArgs& a = b->args;
    for (int m = 0; m < M; m++)
        if (b->members[m]->rk4_threads != rk_threads)
            return bfail(b, EL_EINVAL, "batch members must share one rk4 block size");
    // the (member, species) entries, class by class; each entry's own
    // density picks its gather (a sparse member beside a dense one keeps its
    // register stencils)
    for (int c = 0; c < kRkClasses; c++) {
        a.rk_class_entry[c] = (int)b->h_rk_member.size();
        a.rk_class_task[c] = b->h_rk_begin.back();
        for (int m = 0; m < M; m++) {
            el_flow* f = b->members[m];
            if (f->d.interp < 0 || f->d.interp > 2) continue;
            for (int s = 0; s < f->d.max_species; s++) {
                if (f->sp[s].np == 0) continue;
                const bool shared = rk4_shared_gather(f->d.interp, f->gather,
                                                      (double)f->sp[s].np / (double)f->n2);
                if (2 * f->d.interp + (shared ? 1 : 0) != c) continue;
                b->h_rk_member.push_back(m);
                b->h_rk_sp.push_back(f->table + s);
                b->h_rk_begin.push_back(b->h_rk_begin.back() +
                                        (int)((f->sp[s].np + rk_threads - 1) / rk_threads));
            }
        }
    }
    a.rk_class_entry[kRkClasses] = (int)b->h_rk_member.size();
    a.rk_class_task[kRkClasses] = b->h_rk_begin.back();
    a.members = b->d_members;
    a.spec_begin = b->d_spec_begin;
    a.nl_begin = b->d_nl_begin;
    a.rk_begin = b->d_rk_begin;
    a.rk_member = b->d_rk_member;
    a.rk_sp = b->d_rk_sp;
    a.nmembers = M;
    a.nentries = (int)b->h_rk_member.size();
    a.spec_tasks = b->h_spec_begin.back();
    a.nl_tasks = b->h_nl_begin.back();
    a.rk_tasks = b->h_rk_begin.back();
    if (M > 0) {
        BT_CUDA(b, cudaMemcpyAsync(b->d_members, b->h_members.data(), sizeof(MemberDev) * M,
                                   cudaMemcpyHostToDevice, b->stream));
        BT_CUDA(b, cudaMemcpyAsync(b->d_spec_begin, b->h_spec_begin.data(), sizeof(int) * (M + 1),
                                   cudaMemcpyHostToDevice, b->stream));
        BT_CUDA(b, cudaMemcpyAsync(b->d_nl_begin, b->h_nl_begin.data(), sizeof(int) * (M + 1),
                                   cudaMemcpyHostToDevice, b->stream));
    }
    if (!b->h_fused.empty())
        BT_CUDA(b, cudaMemcpyAsync(b->d_fused, b->h_fused.data(), sizeof(FusedMember) * b->h_fused.size(),
                                   cudaMemcpyHostToDevice, b->stream));
    if (a.nentries > 0) {
        BT_CUDA(b, cudaMemcpyAsync(b->d_rk_begin, b->h_rk_begin.data(),
                                   sizeof(int) * (a.nentries + 1), cudaMemcpyHostToDevice, b->stream));
        BT_CUDA(b, cudaMemcpyAsync(b->d_rk_member, b->h_rk_member.data(), sizeof(int) * a.nentries,
                                   cudaMemcpyHostToDevice, b->stream));
        BT_CUDA(b, cudaMemcpyAsync((void*)b->d_rk_sp, b->h_rk_sp.data(),
                                   sizeof(void*) * a.nentries, cudaMemcpyHostToDevice, b->stream));
    }
    // persistent grids: as many blocks as fit on the GPU at once (capped by the work)
    int occ = 0;
    BT_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_spectral, kBSpecThreads, 0));
    b->grid_spec = std::max(1, std::min(a.spec_tasks, occ * b->sms));
    BT_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_nonlinear, kBNlThreads, 0));
    b->grid_nl = std::max(1, std::min(a.nl_tasks, occ * b->sms));
    // each class's prefetch distance (EL_RK4_PREFETCH_WAVES resident waves;
    // the cubic classes) and the bilinear class's persistent grid
    void (*rk_kernels[kRkClasses])(BatchArgs) = {k_batch_rk4<0, false>, nullptr,
                                                  k_batch_rk4<1, false>, k_batch_rk4<1, true>,
                                                  k_batch_rk4<2, false>, k_batch_rk4<2, true>};
    for (int c = 0; c < kRkClasses; c++) {
        a.rk_prefetch[c] = 0;
        if (a.rk_class_task[c + 1] == a.rk_class_task[c] || !rk_kernels[c]) continue;
        const size_t smem = rk4_patch_bytes(c & 1, rk_threads);
        if (smem > 0)
            BT_CUDA(b, cudaFuncSetAttribute(rk_kernels[c], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)rk4_patch_bytes(true, 512)));
        BT_CUDA(b, set_carveout(rk_kernels[c], c < 2 ? EL_SMEM_CARVEOUT_BILINEAR : EL_SMEM_CARVEOUT_CUBIC));
        BT_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rk_kernels[c], rk_threads, smem));
        const int wave = std::max(1, occ) * b->sms;
        if (c == 0) b->grid_bilinear = (unsigned)wave;
        else a.rk_prefetch[c] = (int)((double)wave * EL_RK4_PREFETCH_WAVES + 0.5) * rk_threads;
    }
    for (FftPool& p : b->pools) ensure_prefix_plans(b, p, p.span());
    b->tables_valid = true;
    return EL_OK;
}

// cuFFT of every member on forked branches of the capture (from `origin`).
el_status fork_ffts(el_batch* b, cudaStream_t origin, bool c2r) {
    BT_CUDA(b, cudaEventRecord(b->fork_ev, origin));
    for (int k = 0; k < kSideStreams; k++) BT_CUDA(b, cudaStreamWaitEvent(b->side[k], b->fork_ev, 0));
    size_t branch = 0;
    for (FftPool& p : b->pools) {
        const int k = p.span();
        if (k == 0) continue;
        const int use = p.c2r[k] ? k : p.slots;  // a prefix plan, else the full one
        cudaStream_t s = b->side[branch++ % kSideStreams];
        cufftHandle plan = c2r ? p.c2r[use] : p.r2c[use];
        if (cufftSetStream(plan, s) != CUFFT_SUCCESS) return bfail(b, EL_ECUFFT, "cufftSetStream");
        cufftResult r = c2r ? cufftExecC2R(plan, reinterpret_cast<cufftComplex*>(p.spec), p.phys)
                            : cufftExecR2C(plan, p.nl, reinterpret_cast<cufftComplex*>(p.nhat));
        if (r != CUFFT_SUCCESS) return bfail(b, EL_ECUFFT, "cuFFT exec (pool) failed (%d)", (int)r);
    }
    for (size_t m = 0; m < b->members.size(); m++) {
        el_flow* f = b->members[m];
        if (f->fft_pool >= 0 || f->fused) continue;
        cudaStream_t s = b->side[branch++ % kSideStreams];
        cufftHandle plan = c2r ? f->plan_c2r : f->plan_r2c;
        if (cufftSetStream(plan, s) != CUFFT_SUCCESS) return bfail(b, EL_ECUFFT, "cufftSetStream");
        cufftResult r = c2r ? cufftExecC2R(plan, reinterpret_cast<cufftComplex*>(f->spec), f->phys)
                            : cufftExecR2C(plan, f->nl, reinterpret_cast<cufftComplex*>(f->nhat));
        if (r != CUFFT_SUCCESS) return bfail(b, EL_ECUFFT, "cuFFT exec failed (%d)", (int)r);
    }
    for (int k = 0; k < kSideStreams; k++) {
        BT_CUDA(b, cudaEventRecord(b->join_ev[k], b->side[k]));
        BT_CUDA(b, cudaStreamWaitEvent(origin, b->join_ev[k], 0));
    }
    return EL_OK;
}

// The fluid step (every member) on stream s: the fused members' kernels,
// then for the others the spectral stage, C2R, nonlinear stage and level
// pair, R2C.
el_status enqueue_fluid(el_batch* b, cudaStream_t s, int ahead) {
    const BatchArgs& a = b->args;
    for (int c = 0; c < 4 * el_batch::kFusedGrids; c++) {
        const int count = b->fused_begin[c + 1] - b->fused_begin[c];
        if (count == 0) continue;
        BT_CUDA(b, fused_fluid_batch(s, b->d_fused + b->fused_begin[c], count, 128 << (c / 4),
                                     4 + (c & 3), ahead, b->fused_twiddle[c / 4]));
        b->launches += 4;
    }
    if (a.spec_tasks == 0) return EL_OK;  // every member is fused
    k_batch_spectral<<<b->grid_spec, kBSpecThreads, 0, s>>>(a, ahead);
    b->launches++;
    EL_TRY(fork_ffts(b, s, true));
    k_batch_nonlinear<<<b->grid_nl, kBNlThreads, 0, s>>>(a, ahead);
    b->launches++;
    return fork_ffts(b, s, false);
}

// The particle step (every member, one launch per scheme present) and the
// per-member step counters.
el_status enqueue_particles(el_batch* b) {
    const BatchArgs& a = b->args;
    if (a.rk_tasks > 0) {
        const int threads = b->members.empty() ? 256 : b->members[0]->rk4_threads;
        const size_t smem = rk4_patch_bytes(true, threads);
        auto tasks = [&](int c) { return (unsigned)(a.rk_class_task[c + 1] - a.rk_class_task[c]); };
        if (tasks(0)) k_batch_rk4<0, false><<<std::min(tasks(0), b->grid_bilinear), threads, 0, b->stream>>>(a);
        if (tasks(2)) k_batch_rk4<1, false><<<tasks(2), threads, 0, b->stream>>>(a);
        if (tasks(3)) k_batch_rk4<1, true><<<tasks(3), threads, smem, b->stream>>>(a);
        if (tasks(4)) k_batch_rk4<2, false><<<tasks(4), threads, 0, b->stream>>>(a);
        if (tasks(5)) k_batch_rk4<2, true><<<tasks(5), threads, smem, b->stream>>>(a);
        for (int c = 0; c < kRkClasses; c++) b->launches += tasks(c) > 0;
    }
    return EL_OK;
}

enum { kBatchFluid = 0, kBatchOverlap = 1, kBatchLast = 2 };

el_status capture_body(el_batch* b, int kind) {
    const BatchArgs& a = b->args;
    if (kind == kBatchFluid) {
        EL_TRY(enqueue_fluid(b, b->stream, 0));
    } else {
        if (kind == kBatchOverlap) {  // fluid of s + 1 on a forked, high-priority branch
            BT_CUDA(b, cudaEventRecord(b->f_fork, b->stream));
            BT_CUDA(b, cudaStreamWaitEvent(b->fluid, b->f_fork, 0));
            EL_TRY(enqueue_fluid(b, b->fluid, 1));
        }
        EL_TRY(enqueue_particles(b));
        if (kind == kBatchOverlap) {
            BT_CUDA(b, cudaEventRecord(b->f_join, b->fluid));
            BT_CUDA(b, cudaStreamWaitEvent(b->stream, b->f_join, 0));
        }
        k_batch_advance<<<1, 256, 0, b->stream>>>(b->d_members, a.nmembers);
        b->launches++;
    }
    BT_CUDA(b, cudaGetLastError());
    return EL_OK;
}

el_status build_batch_graph(el_batch* b, int kind) {
    if (b->graph[kind]) {
        cudaGraphExecDestroy(b->graph[kind]);
        b->graph[kind] = nullptr;
    }
    int64_t before = b->launches;
    cudaGraph_t g = nullptr;
    BT_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    el_status s = capture_body(b, kind);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    for (el_flow* f : b->members) {  // plans back on the batch stream
        cufftSetStream(f->plan_c2r, b->stream);
        cufftSetStream(f->plan_r2c, b->stream);
    }
    for (FftPool& p : b->pools)
        for (int k = 1; k <= p.slots; k++) {
            if (p.c2r[k]) cufftSetStream(p.c2r[k], b->stream);
            if (p.r2c[k]) cufftSetStream(p.r2c[k], b->stream);
        }
    if (s != EL_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return bfail(b, EL_ECUDA, "batch capture: %s", cudaGetErrorString(e));
    // kernel nodes keep the priority of the stream they were captured on
    e = cudaGraphInstantiate(&b->graph[kind], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, EL_ECUDA, "batch graph: %s", cudaGetErrorString(e));
    b->graph_kernels[kind] = b->launches - before;
    b->launches = before;
    return EL_OK;
}

el_status launch_graph(el_batch* b, int kind) {
    if (!b->graph[kind]) EL_TRY(build_batch_graph(b, kind));
    BT_CUDA(b, cudaGraphLaunch(b->graph[kind], b->stream));
    b->launches += b->graph_kernels[kind];
    return EL_OK;
}

// Byte offsets of a pool's arrays and its total size for (n, planes, slots)
// and a cuFFT work area of `work` bytes.
struct PoolLayout {
    size_t spec, phys, nl, nhat, work, total;
};

PoolLayout pool_layout(int n, int planes, int slots, size_t work) {
    const size_t nm = (size_t)n * (n / 2 + 1), n2 = (size_t)n * n, k = (size_t)slots;
    PoolLayout l{};
    l.spec = 0;
    l.phys = l.spec + align_up(k * planes * nm * sizeof(float2));
    l.nl = l.phys + align_up(k * planes * n2 * sizeof(float));
    l.nhat = l.nl + align_up(k * n2 * sizeof(float));
    l.work = l.nhat + align_up(k * nm * sizeof(float2));
    l.total = l.work + align_up(work);
    return l;
}

// The pool's two plans (C2R over slots x planes, R2C over slots), with the
// work area left to the caller; `work` = the larger of their work areas.
cufftResult pool_plans(int n, int planes, int slots, cufftHandle* c2r, cufftHandle* r2c, size_t* work) {
    int dims[2] = {n, n};
    size_t w0 = 0, w1 = 0;
    cufftResult r;
    *c2r = *r2c = 0;
    if ((r = cufftCreate(c2r)) != CUFFT_SUCCESS) return r;
    if ((r = cufftCreate(r2c)) != CUFFT_SUCCESS) return r;
    cufftSetAutoAllocation(*c2r, 0);
    cufftSetAutoAllocation(*r2c, 0);
    if ((r = cufftMakePlanMany(*c2r, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, slots * planes,
                               &w0)) != CUFFT_SUCCESS)
        return r;
    if ((r = cufftMakePlanMany(*r2c, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, slots, &w1)) !=
        CUFFT_SUCCESS)
        return r;
    *work = std::max(w0, w1);
    return CUFFT_SUCCESS;
}

// Put a joining member into a free slot of a pool of its class, if any;
// its N-hat moves into the slot (stream-ordered on the batch stream).  On a
// failed copy the member and the pool are left as they were.
el_status pool_join(el_batch* b, el_flow* f) {
    if (f->fused) return EL_OK;  // its transforms are the fused kernels'
    for (size_t q = 0; q < b->pools.size(); q++) {
        FftPool& p = b->pools[q];
        if (p.n != f->n || p.planes != f->nplanes) continue;
        for (int k = 0; k < p.slots; k++) {
            if (p.member[k]) continue;
            float2* slot_nhat = p.nhat + (size_t)k * p.nmodes;
            BT_CUDA(b, cudaMemcpyAsync(slot_nhat, f->nhat, p.nmodes * sizeof(float2),
                                       cudaMemcpyDeviceToDevice, b->stream));
            p.member[k] = f;  // after the copy was accepted
            f->fft_pool = (int)q;
            f->fft_slot = k;
            f->nhat_cur = slot_nhat;
            return EL_OK;
        }
    }
    return EL_OK;
}

// A leaving member takes its N-hat back from its slot and frees it.
el_status pool_leave(el_batch* b, el_flow* f) {
    if (f->fft_pool < 0) return EL_OK;
    FftPool& p = b->pools[f->fft_pool];
    BT_CUDA(b, cudaMemcpyAsync(f->nhat, f->nhat_cur, p.nmodes * sizeof(float2),
                               cudaMemcpyDeviceToDevice, b->stream));
    BT_CUDA(b, cudaStreamSynchronize(b->stream));
    p.member[f->fft_slot] = nullptr;
    f->fft_pool = f->fft_slot = -1;
    f->nhat_cur = nullptr;
    return EL_OK;
}

// The plans over the first k slots of pool p, made (outside any capture)
// when first needed; left unmade if they would need more work area than the
// pool has (the full plan, sized with the pool, serves then).
void ensure_prefix_plans(el_batch* b, FftPool& p, int k) {
    if (k <= 0 || p.c2r[k]) return;
    cufftHandle c2r = 0, r2c = 0;
    size_t work = 0;
    cufftResult r = pool_plans(p.n, p.planes, k, &c2r, &r2c, &work);
    if (r == CUFFT_SUCCESS && work <= p.work_bytes) {
        r = cufftSetWorkArea(c2r, p.work);
        if (r == CUFFT_SUCCESS) r = cufftSetWorkArea(r2c, p.work);
        if (r == CUFFT_SUCCESS) r = cufftSetStream(c2r, b->stream);
        if (r == CUFFT_SUCCESS) r = cufftSetStream(r2c, b->stream);
        if (r == CUFFT_SUCCESS) {
            p.c2r[k] = c2r;
            p.r2c[k] = r2c;
            return;
        }
    }
    if (c2r) cufftDestroy(c2r);
    if (r2c) cufftDestroy(r2c);
}

void invalidate(el_batch* b) {
    b->tables_valid = false;
    for (cudaGraphExec_t& g : b->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

}  // namespace

namespace el {
// Called when a member's particles or tuning change.
void batch_member_changed(el_batch* b) {
    if (b) invalidate(b);
}
}  // namespace el

extern "C" {

size_t el_batch_workspace_bytes(int32_t max_members) {
    if (max_members <= 0 || max_members > 4096) return 0;
    return table_bytes(max_members);
}

size_t el_batch_fft_pool_bytes(const el_flow_desc* desc, int32_t slots) {
    if (flow_desc_problem(desc) || slots < 1 || slots > 4096) return 0;
    const int planes = flow_planes(*desc);
    cufftHandle c2r = 0, r2c = 0;
    size_t work = 0;
    const cufftResult r = pool_plans(desc->n, planes, slots, &c2r, &r2c, &work);
    if (c2r) cufftDestroy(c2r);
    if (r2c) cufftDestroy(r2c);
    if (r != CUFFT_SUCCESS) return 0;
    return pool_layout(desc->n, planes, slots, work).total;
}

el_status el_batch_add_fft_pool(el_batch* b, const el_flow_desc* desc, int32_t slots,
                                void* dev_workspace, size_t bytes) {
    if (!b || !desc) return EL_EINVAL;
    if (const char* why = flow_desc_problem(desc)) return bfail(b, EL_EINVAL, "%s", why);
    if (slots < 1 || slots > 4096) return bfail(b, EL_EINVAL, "slots out of range");
    if (!dev_workspace || (uintptr_t)dev_workspace % kAlign)
        return bfail(b, EL_EINVAL, "pool memory NULL or not 256-byte aligned");
    FftPool p;
    p.n = desc->n;
    p.planes = flow_planes(*desc);
    p.slots = slots;
    p.nmodes = (size_t)p.n * (p.n / 2 + 1);
    p.n2 = (size_t)p.n * p.n;
    size_t work = 0;
    cufftHandle full_c2r = 0, full_r2c = 0;
    cufftResult r = pool_plans(p.n, p.planes, slots, &full_c2r, &full_r2c, &work);
    const PoolLayout l = pool_layout(p.n, p.planes, slots, work);
    if (r == CUFFT_SUCCESS && bytes < l.total) {
        cufftDestroy(full_c2r);
        cufftDestroy(full_r2c);
        return bfail(b, EL_ENOMEM, "pool memory has %zu bytes, needs %zu", bytes, l.total);
    }
    char* base = static_cast<char*>(dev_workspace);
    p.spec = reinterpret_cast<float2*>(base + l.spec);
    p.phys = reinterpret_cast<float*>(base + l.phys);
    p.nl = reinterpret_cast<float*>(base + l.nl);
    p.nhat = reinterpret_cast<float2*>(base + l.nhat);
    p.work = base + l.work;
    p.work_bytes = work;
    if (r == CUFFT_SUCCESS) r = cufftSetWorkArea(full_c2r, p.work);
    if (r == CUFFT_SUCCESS) r = cufftSetWorkArea(full_r2c, p.work);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(full_c2r, b->stream);
    if (r == CUFFT_SUCCESS) r = cufftSetStream(full_r2c, b->stream);
    if (r != CUFFT_SUCCESS) {
        if (full_c2r) cufftDestroy(full_c2r);
        if (full_r2c) cufftDestroy(full_r2c);
        return bfail(b, EL_ECUFFT, "pool plans failed (%d)", (int)r);
    }
    // free slots inside the transformed span hold zeros until first used
    cudaError_t e = cudaMemsetAsync(base, 0, l.work, b->stream);
    if (e != cudaSuccess) {
        cufftDestroy(full_c2r);
        cufftDestroy(full_r2c);
        return bfail(b, EL_ECUDA, "pool clear: %s", cudaGetErrorString(e));
    }
    p.c2r.assign((size_t)slots + 1, 0);
    p.r2c.assign((size_t)slots + 1, 0);
    p.c2r[slots] = full_c2r;
    p.r2c[slots] = full_r2c;
    p.member.assign((size_t)slots, nullptr);
    b->pools.push_back(std::move(p));
    invalidate(b);
    return EL_OK;
}

el_status el_batch_create(int32_t max_members, void* dev_workspace, size_t bytes,
                          void* cuda_stream, el_batch** out) {
    if (!out) return EL_EINVAL;
    *out = nullptr;
    if (max_members <= 0 || max_members > 4096) return fail(nullptr, EL_EINVAL, "max_members out of range");
    if (!dev_workspace || (uintptr_t)dev_workspace % kAlign)
        return fail(nullptr, EL_EINVAL, "batch workspace NULL or not 256-byte aligned");
    if (bytes < table_bytes(max_members))
        return fail(nullptr, EL_ENOMEM, "batch workspace has %zu bytes, needs %zu", bytes,
                    table_bytes(max_members));
    el_batch* b = new (std::nothrow) el_batch();
    if (!b) return fail(nullptr, EL_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->max_members = max_members;
    char* p = (char*)dev_workspace;
    size_t m = (size_t)max_members, e = m * kMaxSpecies, off = 0;
    auto take = [&](size_t n) { char* r = p + off; off += align_up(n); return r; };
    b->d_members = (MemberDev*)take(m * sizeof(MemberDev));
    b->d_spec_begin = (int*)take((m + 1) * sizeof(int));
    b->d_nl_begin = (int*)take((m + 1) * sizeof(int));
    b->d_rk_begin = (int*)take((e + 1) * sizeof(int));
    b->d_rk_member = (int*)take((e + 1) * sizeof(int));
    b->d_rk_sp = (const SpeciesDev**)take(e * sizeof(void*));
    b->d_fused = (FusedMember*)take(m * sizeof(FusedMember));
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    int lo_prio = 0, hi_prio = 0;
    if (err == cudaSuccess) err = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    for (int k = 0; k < kSideStreams && err == cudaSuccess; k++)
        err = cudaStreamCreateWithPriority(&b->side[k], cudaStreamNonBlocking, hi_prio);
    if (err == cudaSuccess) err = cudaStreamCreateWithPriority(&b->fluid, cudaStreamNonBlocking, hi_prio);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->f_fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->f_join, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    for (int k = 0; k < kSideStreams && err == cudaSuccess; k++)
        err = cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming);
    if (err != cudaSuccess) {
        el_batch_destroy(b);
        return fail(nullptr, EL_ECUDA, "batch create: %s", cudaGetErrorString(err));
    }
    *out = b;
    return EL_OK;
}

el_status el_batch_add(el_batch* b, el_flow* f) {
    if (!b || !f) return EL_EINVAL;
    if (f->batch) return bfail(b, EL_ESTATE, "flow already belongs to a batch");
    if (f->kinematic) return bfail(b, EL_EINVAL, "kinematic flows step alone");
    if ((int)b->members.size() >= b->max_members) return bfail(b, EL_EINVAL, "batch is full");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != f->device) return bfail(b, EL_EINVAL, "flow lives on another device");
    BT_CUDA(b, cudaStreamSynchronize(f->stream));
    // a pool slot first: if moving N-hat into it fails, nothing has changed
    EL_TRY(pool_join(b, f));
    if (!b->members.empty() && b->members[0]->rk4_threads != f->rk4_threads)
        f->rk4_threads = b->members[0]->rk4_threads;
    if (!b->members.empty()) f->gather = b->members[0]->gather;  // one setting per batch
    f->own_stream = f->stream;
    f->stream = b->stream;
    cufftSetStream(f->plan_c2r, b->stream);
    cufftSetStream(f->plan_r2c, b->stream);
    cufftSetStream(f->plan_c2r1, b->stream);
    f->batch = b;
    b->members.push_back(f);
    invalidate(b);
    return EL_OK;
}

el_status el_batch_remove(el_batch* b, el_flow* f) {
    if (!b || !f) return EL_EINVAL;
    auto it = std::find(b->members.begin(), b->members.end(), f);
    if (it == b->members.end()) return bfail(b, EL_EINVAL, "flow is not a member");
    BT_CUDA(b, cudaStreamSynchronize(b->stream));
    EL_TRY(pool_leave(b, f));
    b->members.erase(it);
    f->stream = f->own_stream;
    cufftSetStream(f->plan_c2r, f->stream);
    cufftSetStream(f->plan_r2c, f->stream);
    cufftSetStream(f->plan_c2r1, f->stream);
    f->batch = nullptr;
    drop_graphs(f);  // its own graphs were captured before it joined
    invalidate(b);
    return EL_OK;
}

el_status el_batch_step(el_batch* b, int32_t nsteps) {
    if (!b) return EL_EINVAL;
    NvtxRange range("el_batch_step");
    if (nsteps < 0) return bfail(b, EL_EINVAL, "nsteps < 0");
    if (b->members.empty()) return EL_OK;
    if (!b->tables_valid) EL_TRY(rebuild_tables(b));
    if (nsteps == 0) return EL_OK;
    // As in el_step_coupled, the fluid runs one step ahead inside the call:
    // fluid of s0, then particles of s alongside fluid of s + 1, then the
    // particles of the last step; every member ends at the same level.
    EL_TRY(launch_graph(b, kBatchFluid));
    for (int32_t k = 0; k < nsteps; k++) {
        for (el_flow* f : b->members) {
            if (f->d.sort_every > 0 && f->since_sort >= f->d.sort_every) {
                for (int s = 0; s < f->d.max_species; s++) {
                    el_status st = particles_sort(f, s);
                    if (st != EL_OK) return bfail(b, st, "re-binning: %s", f->err.c_str());
                }
                f->since_sort = 0;
            }
        }
        EL_TRY(launch_graph(b, k + 1 < nsteps ? kBatchOverlap : kBatchLast));
        for (el_flow* f : b->members) {
            f->step++;
            f->since_sort++;
        }
    }
    return EL_OK;
}

el_status el_batch_autotune(el_batch* b, int32_t trial_steps, el_tuning* best);

int32_t el_batch_size(const el_batch* b) { return b ? (int32_t)b->members.size() : 0; }

int64_t el_batch_kernel_launches(const el_batch* b) { return b ? b->launches : 0; }

const char* el_batch_last_error(const el_batch* b) { return b ? b->err.c_str() : ""; }

el_status el_batch_destroy(el_batch* b) {
    if (!b) return EL_EINVAL;
    if (b->stream || !b->members.empty()) cudaStreamSynchronize(b->stream);
    while (!b->members.empty()) el_batch_remove(b, b->members.back());
    for (FftPool& p : b->pools)
        for (int k = 1; k <= p.slots; k++) {
            if (p.c2r[k]) cufftDestroy(p.c2r[k]);
            if (p.r2c[k]) cufftDestroy(p.r2c[k]);
        }
    for (cudaGraphExec_t g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    for (int k = 0; k < kSideStreams; k++) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->fluid) cudaStreamDestroy(b->fluid);
    if (b->f_fork) cudaEventDestroy(b->f_fork);
    if (b->f_join) cudaEventDestroy(b->f_join);
    delete b;
    return EL_OK;
}

}  // extern "C"

namespace {

el_status batch_apply(el_batch* b, const el_tuning& t) {
    for (el_flow* f : b->members) {
        f->rk4_threads = t.rk4_threads;
        f->gather = t.gather;
        f->d.sort_every = t.sort_every;
        f->sort_shift = std::min(t.sort_shift, std::max(0, f->log2n - 2));
    }
    invalidate(b);
    return EL_OK;
}

}  // namespace

// Same search as el_autotune, one setting for every member.
extern "C" el_status el_batch_autotune(el_batch* b, int32_t trial_steps, el_tuning* best_out) {
    if (!b || !best_out) return EL_EINVAL;
    if (trial_steps < 1) return bfail(b, EL_EINVAL, "trial_steps must be >= 1");
    if (b->members.empty()) return bfail(b, EL_ESTATE, "empty batch");
    el_flow* f0 = b->members[0];
    el_tuning start{f0->rk4_threads, f0->d.sort_every, f0->sort_shift, f0->gather, 0.0};
    int nmin = f0->n;
    bool cubic = false;
    for (el_flow* f : b->members) {
        nmin = std::min(nmin, f->n);
        cubic = cubic || f->d.interp == EL_CATMULL_ROM || f->d.interp == EL_BSPLINE;
    }
    auto step = [b](int n) { return el_batch_step(b, n); };
    auto apply = [b](el_tuning t) { return batch_apply(b, t); };
    auto sort_all = [b]() -> el_status {
        for (el_flow* f : b->members) {
            for (int s = 0; s < f->d.max_species; s++) EL_TRY(particles_sort(f, s));
            f->since_sort = 0;
        }
        return EL_OK;
    };
    return autotune_model(step, apply, sort_all, b->stream, start, trial_steps, best_out, nmin, cubic);
}
