// The C ABI of include/elpath.h: argument checks, the workspace layout,
// cuFFT plans, the captured step graph and the coupled step of Algorithm 1.
#include "common.cuh"
#include "tune.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

namespace el {

void batch_member_changed(el_batch* b);

void fluid_tables(const el_flow_desc& d, std::vector<float2>& ex, std::vector<float2>& ey,
                  std::vector<float>& px, std::vector<float>& py);

namespace {

thread_local std::string g_create_error;

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

const char* check_desc(const el_flow_desc* d) {
    if (!d) return "desc is NULL";
    if (!is_pow2(d->n) || d->n < 16 || d->n > 4096) return "n must be a power of two in [16, 4096]";
    if (d->interp < 0 || d->interp > 3) return "interp must be 0, 1, 2 or 3";
    if (d->interp == EL_ANALYTIC && d->tracer_velocity)
        return "EL_ANALYTIC evaluates the velocity itself: tracer_velocity must be 0";
    if (!std::isfinite(d->nu) || d->nu < 0.0) return "nu must be finite and >= 0";
    if (!std::isfinite(d->dt) || d->dt <= 0.0) return "dt must be finite and > 0";
    if (d->ab2_mode != 0 && d->ab2_mode != 1) return "ab2_mode must be 0 or 1";
    if (d->bspline_prefilter != 0 && d->bspline_prefilter != 1) return "bspline_prefilter must be 0 or 1";
    if (d->max_species < 0 || d->max_species > EL_MAX_SPECIES) return "max_species out of range";
    if (d->max_particles < 0 || d->max_particles > ((int64_t)1 << 31)) return "max_particles out of range";
    if (d->max_particles > 0 && d->max_species == 0) return "max_particles > 0 needs max_species > 0";
    if (d->sort_every < 0) return "sort_every must be >= 0";
    if (d->tracer_velocity != 0 && d->tracer_velocity != 1) return "tracer_velocity must be 0 or 1";
    return nullptr;
}

int planes_of(const el_flow_desc& d) {
    return 4 + ((d.interp == EL_BSPLINE && d.bspline_prefilter) ? 2 : 0) + (d.tracer_velocity ? 1 : 0);
}

// Bytes one species of np particles takes from the pool: 12 arrays, each
// 256-byte aligned.  The sort block (index 1 of each pair) is carved as one
// contiguous run of at least 32 * np bytes, which also serves as staging.
size_t species_bytes(int64_t np) {
    size_t n = (size_t)np;
    size_t a = align_up(n * 4) + align_up(n * 8) + align_up(n * 8) + align_up(n * 8) + align_up(n * 4);
    return 2 * a + align_up(n * 16) + align_up(n * 4);
}

// cuFFT work-area bytes for (n, planes), cached.
std::mutex g_fft_mutex;
std::map<std::pair<int, int>, size_t> g_fft_bytes;

cufftResult make_plans(int n, int planes, cufftHandle* c2r, cufftHandle* r2c, cufftHandle* c2r1,
                       size_t* work) {
    int dims[2] = {n, n};
    size_t w0 = 0, w1 = 0, w2 = 0;
    cufftResult r;
    *c2r = *r2c = *c2r1 = 0;
    if ((r = cufftCreate(c2r)) != CUFFT_SUCCESS) return r;
    if ((r = cufftCreate(r2c)) != CUFFT_SUCCESS) return r;
    if ((r = cufftCreate(c2r1)) != CUFFT_SUCCESS) return r;
    cufftSetAutoAllocation(*c2r, 0);
    cufftSetAutoAllocation(*r2c, 0);
    cufftSetAutoAllocation(*c2r1, 0);
    if ((r = cufftMakePlanMany(*c2r, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, planes, &w0)) !=
        CUFFT_SUCCESS)
        return r;
    if ((r = cufftMakePlanMany(*r2c, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1, &w1)) !=
        CUFFT_SUCCESS)
        return r;
    if ((r = cufftMakePlanMany(*c2r1, 2, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1, &w2)) !=
        CUFFT_SUCCESS)
        return r;
    *work = std::max(w0, std::max(w1, w2));
    return CUFFT_SUCCESS;
}

void destroy_plans(cufftHandle a, cufftHandle b, cufftHandle c) {
    if (a) cufftDestroy(a);
    if (b) cufftDestroy(b);
    if (c) cufftDestroy(c);
}

bool fft_work_bytes(int n, int planes, size_t* out) {
    std::lock_guard<std::mutex> g(g_fft_mutex);
    auto key = std::make_pair(n, planes);
    auto it = g_fft_bytes.find(key);
    if (it != g_fft_bytes.end()) {
        *out = it->second;
        return true;
    }
    cufftHandle a, b, c;
    size_t w = 0;
    cufftResult r = make_plans(n, planes, &a, &b, &c, &w);
    destroy_plans(a, b, c);
    if (r != CUFFT_SUCCESS) return false;
    g_fft_bytes[key] = w;
    *out = w;
    return true;
}

// The workspace layout.  With base == nullptr only the size is computed.
size_t carve(const el_flow_desc& d, size_t fft_bytes, el_flow* f, char* base) {
    size_t cur = 0;
    auto take = [&](size_t bytes) -> char* {
        size_t o = align_up(cur);
        cur = o + bytes;
        return base ? base + o : nullptr;
    };
    size_t n = (size_t)d.n, nh = n / 2 + 1, n2 = n * n, nm = n * nh;
    int planes = planes_of(d);
    char* what = take(nm * 8);
    char* what_lo = take(nm * 8);
    char* hist = take(nm * 8);
    char* nhat = take(nm * 8);
    char* spec = take((size_t)planes * nm * 8);
    char* phys = take((size_t)planes * n2 * 4);
    char* nl = take(n2 * 4);
    char* snap0 = take(n2 * 16);
    char* snap1 = take(n2 * 16);
    char* psi0 = d.tracer_velocity ? take(n2 * 8) : nullptr;
    char* psi1 = d.tracer_velocity ? take(n2 * 8) : nullptr;
    char* aux_spec = take(nm * 8);
    char* aux_phys = take(n2 * 4);
    char* stage64 = take(n2 * 8);
    char* ex = take(nh * 8);
    char* ey = take(n * 8);
    char* px = take(nh * 4);
    char* py = take(n * 4);
    char* twiddle = take(n * 8);
    char* table = take(sizeof(SpeciesDev) * kMaxSpecies);
    char* check = take(4 * sizeof(uint32_t));
    char* bad_input = take(sizeof(unsigned long long));
    char* red = take((size_t)kRedBlocks * 3 * 8);
    char* red_out = take(64 * 8);
    char* boxes = take((size_t)kBoxes * kBoxes * 8);
    bool parts = d.max_particles > 0;
    char* bins = parts ? take(n2 * 4) : nullptr;
    char* bin_sums = parts ? take((4096 + 64) * 4) : nullptr;
    char* fft = take(fft_bytes);
    size_t pool_bytes = parts ? species_bytes(d.max_particles) + (size_t)d.max_species * 12 * kAlign : 0;
    char* pool = take(pool_bytes);
    if (f) {
        f->what = (float2*)what;
        f->what_lo = (float2*)what_lo;
        f->hist = (float2*)hist;
        f->nhat = (float2*)nhat;
        f->spec = (float2*)spec;
        f->phys = (float*)phys;
        f->nl = (float*)nl;
        f->snap[0] = (float4*)snap0;
        f->snap[1] = (float4*)snap1;
        f->psi[0] = (float2*)psi0;
        f->psi[1] = (float2*)psi1;
        f->aux_spec = (float2*)aux_spec;
        f->aux_phys = (float*)aux_phys;
        f->stage64 = (double*)stage64;
        f->ex = (float2*)ex;
        f->ey = (float2*)ey;
        f->pre_x = (float*)px;
        f->pre_y = (float*)py;
        f->twiddle = (float2*)twiddle;
        f->table = (SpeciesDev*)table;
        f->check = (uint32_t*)check;
        f->bad_input = (unsigned long long*)bad_input;
        f->red = (double*)red;
        f->red_out = (double*)red_out;
        f->boxes = (unsigned long long*)boxes;
        f->bins = (uint32_t*)bins;
        f->bin_sums = (uint32_t*)bin_sums;
        f->fft_work = fft;
        f->pool = pool;
        f->pool_bytes = pool_bytes;
        f->pool_used = 0;
    }
    return align_up(cur);
}

// Give species slot s room for np particles from the pool.
bool carve_species(el_flow* f, Species& sp, int64_t np) {
    if (np <= sp.cap) return true;
    size_t need = species_bytes(np);
    size_t start = align_up(f->pool_used);
    if (start + need > f->pool_bytes) return false;
    char* base = f->pool + start;
    size_t cur = 0;
    auto take = [&](size_t bytes) -> char* {
        size_t o = align_up(cur);
        cur = o + bytes;
        return base + o;
    };
    size_t n = (size_t)np;
    for (int k = 0; k < 2; k++) {
        sp.cell[k] = (uint32_t*)take(n * 4);
        sp.off[k] = (float2*)take(n * 8);
        sp.vel[k] = (float2*)take(n * 8);
        sp.img[k] = (int2*)take(n * 8);
        sp.id[k] = (uint32_t*)take(n * 4);
    }
    sp.x0 = (double2*)take(n * 16);
    sp.rank = (uint32_t*)take(n * 4);
    f->pool_used = start + align_up(cur);
    sp.cap = np;
    return true;
}

enum { kFluidStep = 0, kParticleStep = 1, kOverlapStep = 2 };

// Enqueue one piece of Algorithm 1 on the flow's stream: the fluid step n ->
// n+1, the particle step between levels n and n+1, or the particle step of n
// on a forked branch alongside the fluid step of n+1.  The two are
// independent: particles of step n read the level pair (n, n+1); the fluid
// step of n+1 only reads that pair's second half and writes pair (n+1, n+2).
#ifndef EL_FLUID_BRANCH_PRIORITY
#define EL_FLUID_BRANCH_PRIORITY 1
#endif

el_status enqueue_step(el_flow* f, int kind, int64_t step) {
    if (kind == kFluidStep) return fluid_step(f, step);
    if (kind == kParticleStep) return particles_step_all(f, step, false);
    EL_CUDA_OK(f, cudaEventRecord(f->ev_fork, f->stream));
    EL_CUDA_OK(f, cudaStreamWaitEvent(f->side, f->ev_fork, 0));
    cudaStream_t main = f->stream;
#if EL_FLUID_BRANCH_PRIORITY
    // The fluid chain (several short kernels) goes on the high-priority side
    // branch, so its blocks are dispatched as soon as the particle kernel's
    // blocks free an SM instead of after the particle kernel.
    EL_TRY(particles_step_all(f, step, true));
    f->stream = f->side;
    cufftSetStream(f->plan_c2r, f->side);
    cufftSetStream(f->plan_r2c, f->side);
    el_status s = fluid_step(f, step + 1);
    cufftSetStream(f->plan_c2r, main);
    cufftSetStream(f->plan_r2c, main);
    f->stream = main;
    EL_TRY(s);
#else
    f->stream = f->side;
    el_status s = particles_step_all(f, step, true);
    f->stream = main;
    EL_TRY(s);
    EL_TRY(fluid_step(f, step + 1));
#endif
    EL_CUDA_OK(f, cudaEventRecord(f->ev_join, f->side));
    EL_CUDA_OK(f, cudaStreamWaitEvent(f->stream, f->ev_join, 0));
    return EL_OK;
}

cudaGraphExec_t* graph_slot(el_flow* f, int kind, int phase, int64_t** count) {
    if (kind == kFluidStep) {
        *count = &f->k_fluid[phase];
        return &f->g_fluid[phase];
    }
    if (kind == kParticleStep) {
        *count = &f->k_part[phase];
        return &f->g_part[phase];
    }
    *count = &f->k_both[phase];
    return &f->g_both[phase];
}

// Capture `kind` for step parity `phase` (a step >= 1 with that parity: the
// first, forward-Euler fluid step always runs by direct launches).
el_status build_graph(el_flow* f, int kind, int phase) {
    int64_t* count = nullptr;
    cudaGraphExec_t* slot = graph_slot(f, kind, phase, &count);
    if (*slot) {
        cudaGraphExecDestroy(*slot);
        *slot = nullptr;
    }
    int64_t before = f->launches;
    cudaGraph_t g = nullptr;
    EL_CUDA_OK(f, cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal));
    el_status s = enqueue_step(f, kind, 2 + phase);
    cudaError_t e = cudaStreamEndCapture(f->stream, &g);
    if (s != EL_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(f, EL_ECUDA, "stream capture: %s", cudaGetErrorString(e));
    // kernel nodes keep the priority of the stream they were captured on
    e = cudaGraphInstantiate(slot, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(f, EL_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    *count = f->launches - before;
    f->launches = before;  // nothing ran yet; replays add the count each
    return EL_OK;
}

// Kinematic flows pass the step's time to their kernels as arguments, so
// they run by direct launches.
bool graphs_enabled(const el_flow* f) {
    static const bool no_graph = std::getenv("ELPATH_NO_GRAPH") != nullptr;
    return f->stream != nullptr && !no_graph && !f->kinematic;
}

el_status run_step(el_flow* f, int kind, int64_t step) {
    if (!graphs_enabled(f) || (kind == kFluidStep && step == 0)) return enqueue_step(f, kind, step);
    int phase = (int)(step % 2);
    int64_t* count = nullptr;
    cudaGraphExec_t* slot = graph_slot(f, kind, phase, &count);
    if (!*slot) EL_TRY(build_graph(f, kind, phase));
    EL_CUDA_OK(f, cudaGraphLaunch(*slot, f->stream));
    f->launches += *count;
    return EL_OK;
}

el_status maybe_sort(el_flow* f) {
    if (f->d.sort_every > 0 && f->since_sort >= f->d.sort_every) {
        NvtxRange range("rebin");
        for (int s = 0; s < f->d.max_species; s++) EL_TRY(particles_sort(f, s));
        f->since_sort = 0;
    }
    return EL_OK;
}

}  // namespace

bool species_fit(const el_flow* f, const int64_t* np) {
    size_t used = f->pool_used;
    for (int k = 0; k < f->d.max_species; k++) {
        if (np[k] <= f->sp[k].cap) continue;
        used = align_up(used) + species_bytes(np[k]);
        if (used > f->pool_bytes) return false;
    }
    return true;
}

bool carve_species_slot(el_flow* f, int s, int64_t np) { return carve_species(f, f->sp[s], np); }

const char* flow_desc_problem(const el_flow_desc* d) { return check_desc(d); }

int flow_planes(const el_flow_desc& d) { return planes_of(d); }

void drop_graphs(el_flow* f) {
    for (int k = 0; k < 2; k++) {
        cudaGraphExec_t* gs[3] = {&f->g_fluid[k], &f->g_part[k], &f->g_both[k]};
        for (cudaGraphExec_t* g : gs) {
            if (*g) cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    }
}

el_status fail(el_flow* f, el_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (f)
        f->err = buf;
    else
        g_create_error = buf;
    return s;
}

}  // namespace el

using namespace el;

extern "C" {

size_t el_workspace_bytes(const el_flow_desc* desc) {
    if (check_desc(desc)) return 0;
    size_t fft = 0;
    if (!fft_work_bytes(desc->n, planes_of(*desc), &fft)) return 0;
    return carve(*desc, fft, nullptr, nullptr);
}

}  // extern "C"

// Both creation calls: a solved flow from omega0, or (kin != NULL) the
// prescribed kinematic flow.
static el_status create_flow(const el_flow_desc* desc, const double* omega0, const el_kinematic* kin,
                             void* dev_workspace, size_t workspace_bytes, void* cuda_stream,
                             el_flow** out) {
    NvtxRange range("el_create_flow");
    if (!out) return fail(nullptr, EL_EINVAL, "out is NULL");
    *out = nullptr;
    if (const char* why = check_desc(desc)) return fail(nullptr, EL_EINVAL, "%s", why);
    if (!kin && desc->interp == EL_ANALYTIC)
        return fail(nullptr, EL_EINVAL, "EL_ANALYTIC needs a kinematic flow (el_create_kinematic)");
    if (kin) {
        const bool ok = std::isfinite(kin->alpha) && std::isfinite(kin->k) && std::isfinite(kin->eps) &&
                        std::isfinite(kin->omega) && std::isfinite(kin->phi) && kin->k >= 1.0 &&
                        kin->k == std::floor(kin->k) && 3.0 * kin->k < desc->n;
        if (!ok) return fail(nullptr, EL_EINVAL, "kinematic parameters: finite, k an integer in [1, n/3)");
    } else if (!omega0) {
        return fail(nullptr, EL_EINVAL, "omega0 is NULL");
    }
    if (!dev_workspace) return fail(nullptr, EL_EINVAL, "workspace is NULL");
    if ((uintptr_t)dev_workspace % kAlign) return fail(nullptr, EL_EINVAL, "workspace not 256-byte aligned");
    for (size_t q = 0, nn = omega0 ? (size_t)desc->n * desc->n : 0; q < nn; q++)
        if (!std::isfinite(omega0[q])) return fail(nullptr, EL_EINVAL, "omega0 has a non-finite value");
    size_t fft = 0;
    if (!fft_work_bytes(desc->n, planes_of(*desc), &fft))
        return fail(nullptr, EL_ECUFFT, "cuFFT plan creation failed for n=%d", desc->n);
    size_t need = carve(*desc, fft, nullptr, nullptr);
    if (workspace_bytes < need)
        return fail(nullptr, EL_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);

    el_flow* f = new (std::nothrow) el_flow();
    if (!f) return fail(nullptr, EL_ENOMEM, "host allocation failed");
    f->d = *desc;
    if (kin) {
        f->kinematic = 1;
        f->kin = *kin;
    }
    f->stream = (cudaStream_t)cuda_stream;
    f->own_stream = f->stream;
    cudaGetDevice(&f->device);
    f->n = desc->n;
    f->nh = desc->n / 2 + 1;
    f->log2n = 0;
    while ((1 << f->log2n) < f->n) f->log2n++;
    f->n2 = (size_t)f->n * f->n;
    f->nmodes = (size_t)f->n * f->nh;
    f->nplanes = planes_of(*desc);
    f->stencil_plane = (desc->interp == EL_BSPLINE && desc->bspline_prefilter) ? 4 : 0;
    f->psi_plane = desc->tracer_velocity ? f->nplanes - 1 : -1;
    f->ws = (char*)dev_workspace;
    f->ws_bytes = workspace_bytes;
    carve(*desc, fft, f, f->ws);

    auto bail = [&](el_status s) {
        g_create_error = f->err;
        destroy_plans(f->plan_c2r, f->plan_r2c, f->plan_c2r1);
        if (f->side) cudaStreamDestroy(f->side);
        if (f->ev_fork) cudaEventDestroy(f->ev_fork);
        if (f->ev_join) cudaEventDestroy(f->ev_join);
        delete f;
        return s;
    };
    if (f->stream) {
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        cudaError_t es = cudaStreamCreateWithPriority(&f->side, cudaStreamNonBlocking,
                                                      EL_FLUID_BRANCH_PRIORITY ? hi_prio : lo_prio);
        if (es == cudaSuccess) es = cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming);
        if (es == cudaSuccess) es = cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming);
        if (es != cudaSuccess) {
            fail(f, EL_ECUDA, "side stream: %s", cudaGetErrorString(es));
            return bail(EL_ECUDA);
        }
    }
    size_t w = 0;
    cufftResult r = make_plans(f->n, f->nplanes, &f->plan_c2r, &f->plan_r2c, &f->plan_c2r1, &w);
    if (r != CUFFT_SUCCESS || w > fft) {
        fail(f, EL_ECUFFT, "cuFFT plan creation failed (%d)", (int)r);
        return bail(EL_ECUFFT);
    }
    cufftHandle plans[3] = {f->plan_c2r, f->plan_r2c, f->plan_c2r1};
    for (cufftHandle p : plans) {
        if (cufftSetWorkArea(p, f->fft_work) != CUFFT_SUCCESS || cufftSetStream(p, f->stream) != CUFFT_SUCCESS) {
            fail(f, EL_ECUFFT, "cuFFT work area / stream binding failed");
            return bail(EL_ECUFFT);
        }
    }
    f->plans_made = true;

    std::vector<float2> ex, ey;
    std::vector<float> px, py;
    fluid_tables(*desc, ex, ey, px, py);
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpyAsync(f->ex, ex.data(), ex.size() * 8, cudaMemcpyHostToDevice, f->stream);
    e = e ? e : cudaMemcpyAsync(f->ey, ey.data(), ey.size() * 8, cudaMemcpyHostToDevice, f->stream);
    e = e ? e : cudaMemcpyAsync(f->pre_x, px.data(), px.size() * 4, cudaMemcpyHostToDevice, f->stream);
    e = e ? e : cudaMemcpyAsync(f->pre_y, py.data(), py.size() * 4, cudaMemcpyHostToDevice, f->stream);
    if (e != cudaSuccess) {
        fail(f, EL_ECUDA, "table upload: %s", cudaGetErrorString(e));
        return bail(EL_ECUDA);
    }
    std::vector<float2> tw;
    if (fused_fluid_supported(f)) {
        // exp(-2 pi i m / n) in FP64, rounded once
        tw.resize((size_t)f->n);
        for (int m = 0; m < f->n; m++) {
            const double t = kTwoPi * (double)m / (double)f->n;
            tw[m] = make_float2((float)std::cos(t), (float)-std::sin(t));
        }
        e = cudaMemcpyAsync(f->twiddle, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, f->stream);
        if (e != cudaSuccess) {
            fail(f, EL_ECUDA, "twiddle upload: %s", cudaGetErrorString(e));
            return bail(EL_ECUDA);
        }
        el_status fs = fused_fluid_prepare(f);
        if (fs != EL_OK) return bail(fs);
        f->fused = true;
    }
    e = cudaMemsetAsync(f->check, 0, 4 * sizeof(uint32_t), f->stream);
    if (e != cudaSuccess) {
        fail(f, EL_ECUDA, "check word: %s", cudaGetErrorString(e));
        return bail(EL_ECUDA);
    }
    el_status s = kin ? kinematic_level(f, 0, true) : fluid_init(f, omega0);
    if (s != EL_OK) return bail(s);
    s = rk4_prepare(f);
    if (s != EL_OK) return bail(s);
    e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) {
        fail(f, EL_ECUDA, "create: %s", cudaGetErrorString(e));
        return bail(EL_ECUDA);
    }
    *out = f;
    return EL_OK;
}

extern "C" {

el_status el_create_flow(const el_flow_desc* desc, const double* omega0, void* dev_workspace,
                         size_t workspace_bytes, void* cuda_stream, el_flow** out) {
    return create_flow(desc, omega0, nullptr, dev_workspace, workspace_bytes, cuda_stream, out);
}

el_status el_create_kinematic(const el_flow_desc* desc, const el_kinematic* kin, void* dev_workspace,
                              size_t workspace_bytes, void* cuda_stream, el_flow** out) {
    if (!kin) {
        if (out) *out = nullptr;
        return fail(nullptr, EL_EINVAL, "kin is NULL");
    }
    return create_flow(desc, nullptr, kin, dev_workspace, workspace_bytes, cuda_stream, out);
}

el_status el_set_particles(el_flow* f, int32_t species, int64_t np, double st, const double* xy,
                           const double* vxy) {
    if (!f) return EL_EINVAL;
    NvtxRange range("el_set_particles");
    if (species < 0 || species >= f->d.max_species)
        return fail(f, EL_EINVAL, "species %d outside [0, %d)", species, f->d.max_species);
    if (np < 0 || np > f->d.max_particles) return fail(f, EL_EINVAL, "np %lld out of range", (long long)np);
    if (!std::isfinite(st) || st < 0.0) return fail(f, EL_EINVAL, "st must be finite and >= 0");
    if (f->d.interp == EL_ANALYTIC && st > 0.0)
        return fail(f, EL_EINVAL, "EL_ANALYTIC flows take tracers (st = 0) only");
    if (np > 0 && !xy) return fail(f, EL_EINVAL, "xy is NULL");
    Species& sp = f->sp[species];
    // Positions (finite, |x| <= 1e9) and velocities (finite) are checked on
    // the device, on the staged copy, before anything of the slot changes.
    // Capacity carved for this call is host bookkeeping only, handed back if
    // the check refuses the data, so a refused call changes nothing.
    const Species kept = sp;
    const size_t kept_used = f->pool_used;
    if (!carve_species(f, sp, np))
        return fail(f, EL_EINVAL, "particle capacity exhausted (max_particles=%lld)",
                    (long long)f->d.max_particles);
    const el_status placed = particles_set(f, species, np, st, xy, vxy);
    if (placed == EL_EINVAL) {
        sp = kept;
        f->pool_used = kept_used;
    }
    if (placed != EL_OK) return placed;
    // The captured step graphs read the species table on the device; what
    // they bake in is each species' block range and the gather choice, both
    // set by the particle counts, so new particles in the same numbers keep
    // them (no re-capture on the next step).
    if (kept.np != np) {
        drop_graphs(f);
        batch_member_changed(f->batch);
    }
    if (f->d.sort_every > 0) f->since_sort = f->d.sort_every;  // bin the new particles first
    return EL_OK;
}

// Algorithm 1 for nsteps steps.  The fluid runs one step ahead inside the
// call: particles of step n and the fluid step of n+1 go on two branches of
// one graph and overlap on the device; the call ends with both at the same
// level, so every other call sees a consistent state.
el_status el_step_coupled(el_flow* f, int32_t nsteps) {
    if (!f) return EL_EINVAL;
    NvtxRange range("el_step_coupled");
    if (f->batch) return fail(f, EL_ESTATE, "flow belongs to a batch: step it with el_batch_step");
    if (nsteps < 0) return fail(f, EL_EINVAL, "nsteps < 0");
    if (nsteps == 0) return EL_OK;
    const bool overlap = graphs_enabled(f) && f->side;
    const int64_t n0 = f->step;
    EL_TRY(maybe_sort(f));
    EL_TRY(run_step(f, kFluidStep, n0));
    for (int64_t s = n0; s < n0 + nsteps; s++) {
        const bool last = s == n0 + nsteps - 1;
        if (last) {
            EL_TRY(run_step(f, kParticleStep, s));
        } else if (overlap) {
            EL_TRY(run_step(f, kOverlapStep, s));
        } else {
            EL_TRY(run_step(f, kParticleStep, s));
            EL_TRY(run_step(f, kFluidStep, s + 1));
        }
        f->step = s + 1;
        f->since_sort++;
        if (!last) EL_TRY(maybe_sort(f));
    }
    return EL_OK;
}

el_status el_get_stats(el_flow* f, el_stats* out) {
    if (!f || !out) return EL_EINVAL;
    NvtxRange range("el_get_stats");
    if (!f->kinematic) EL_TRY(fluid_diagnostics(f));
    int ns = f->d.max_species;
    for (int s = 0; s < ns; s++)
        if (f->sp[s].np > 0) EL_TRY(particles_stats_into(f, s, f->red_out + 3 + 5 * s));
    double host[3 + 5 * EL_MAX_SPECIES] = {0};
    EL_CUDA_OK(f, cudaMemcpyAsync(host, f->red_out, sizeof(double) * (3 + 5 * ns), cudaMemcpyDeviceToHost,
                                  f->stream));
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    if (EL_CHECK_BOUNDS) {
        uint32_t chk[4] = {0, 0, 0, 0};
        EL_CUDA_OK(f, cudaMemcpy(chk, f->check, sizeof chk, cudaMemcpyDeviceToHost));
        if (chk[0] != 0)
            return fail(f, EL_ESTATE,
                        "particle state invariant violated %u times (first: particle %u of species %u)",
                        chk[0], chk[1], chk[2]);
    }
    if (f->kinematic) kinematic_diagnostics(f, host);
    *out = el_stats{};
    out->t = (double)f->step * f->d.dt;
    out->step = f->step;
    out->energy = host[0];
    out->enstrophy = host[1];
    out->palinstrophy = host[2];
    bool finite = std::isfinite(host[0]) && std::isfinite(host[1]) && std::isfinite(host[2]);
    for (int s = 0; s < ns; s++) {
        out->np[s] = f->sp[s].np;
        if (f->sp[s].np == 0) continue;
        const double* h = host + 3 + 5 * s;
        out->msd[s][0] = h[0];
        out->msd[s][1] = h[1];
        out->cluster[s] = h[2];
        // standard error of the mean squared displacement per axis: the
        // sample variance of the squared displacements over np particles,
        // np / (np - 1) (<d^4> - <d^2>^2), divided by np
        const double np = (double)f->sp[s].np;
        for (int a = 0; a < 2; a++) {
            const double var = np > 1.0 ? std::max(0.0, h[3 + a] - h[a] * h[a]) / (np - 1.0) : 0.0;
            out->msd_sem[s][a] = std::sqrt(var);
            out->diffusivity[s][a] = out->t > 0.0 ? h[a] / (2.0 * out->t) : 0.0;
        }
        finite = finite && std::isfinite(h[0]) && std::isfinite(h[1]);
    }
    out->finite = finite ? 1 : 0;
    if (!finite) return fail(f, EL_ENONFINITE, "non-finite diagnostics at step %lld", (long long)f->step);
    return EL_OK;
}

el_status el_get_particles(el_flow* f, int32_t species, double* xy, double* vxy) {
    if (!f) return EL_EINVAL;
    if (species < 0 || species >= f->d.max_species)
        return fail(f, EL_EINVAL, "species %d outside [0, %d)", species, f->d.max_species);
    return particles_get(f, species, xy, vxy);
}

el_status el_get_field(el_flow* f, int32_t which, double* host_nn) {
    if (!f || !host_nn) return EL_EINVAL;
    if (which < 0 || which > 4) return fail(f, EL_EINVAL, "which must be 0..4");
    return fluid_get_field(f, which, host_nn);
}

el_status el_sample_velocity(el_flow* f, int64_t np, const double* d_xy, double theta, double* d_uv) {
    if (!f) return EL_EINVAL;
    if (np < 0 || (np > 0 && (!d_xy || !d_uv))) return fail(f, EL_EINVAL, "bad sample arrays");
    if (!(theta >= 0.0 && theta <= 1.0)) return fail(f, EL_EINVAL, "theta must be in [0, 1]");
    if (f->d.interp == EL_ANALYTIC) return fail(f, EL_EINVAL, "EL_ANALYTIC has no grid interpolant");
    return sample_velocity(f, np, d_xy, theta, d_uv);
}

el_status el_profile_step(el_flow* f, double* stage_ms, int32_t nstage) {
    if (!f || !stage_ms) return EL_EINVAL;
    if (f->batch) return fail(f, EL_ESTATE, "flow belongs to a batch");
    if (nstage < 3) return fail(f, EL_EINVAL, "nstage must be >= 3");
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; k++) EL_CUDA_OK(f, cudaEventCreate(&ev[k]));
    el_status st = EL_OK;
    bool sorted = false;
    cudaEventRecord(ev[0], f->stream);
    if (f->d.sort_every > 0 && f->since_sort >= f->d.sort_every) {
        for (int s = 0; s < f->d.max_species && st == EL_OK; s++) st = particles_sort(f, s);
        f->since_sort = 0;
        sorted = true;
    }
    cudaEventRecord(ev[1], f->stream);
    if (st == EL_OK) st = fluid_step(f, f->step);
    cudaEventRecord(ev[2], f->stream);
    // the particle kernel the overlapped step runs (its carve-out variant)
    if (st == EL_OK) st = particles_step_all(f, f->step, true);
    cudaEventRecord(ev[3], f->stream);
    cudaError_t e = cudaStreamSynchronize(f->stream);
    if (st == EL_OK && e != cudaSuccess) st = fail(f, EL_ECUDA, "profile: %s", cudaGetErrorString(e));
    if (st == EL_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[1], ev[2]);
        stage_ms[0] = ms;
        cudaEventElapsedTime(&ms, ev[2], ev[3]);
        stage_ms[1] = ms;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        stage_ms[2] = sorted ? ms : 0.0;
        f->step++;
        f->since_sort++;
    }
    for (int k = 0; k < 4; k++) cudaEventDestroy(ev[k]);
    return st;
}

int64_t el_kernel_launches(const el_flow* f) { return f ? f->launches : 0; }

int32_t el_flow_fused(const el_flow* f) { return f && f->fused ? 1 : 0; }

el_status el_get_tuning(const el_flow* f, el_tuning* out) {
    if (!f || !out) return EL_EINVAL;
    out->rk4_threads = f->rk4_threads;
    out->sort_every = f->d.sort_every;
    out->sort_shift = f->sort_shift;
    out->gather = f->gather;
    out->ms_per_step = 0.0;
    return EL_OK;
}

el_status el_set_tuning(el_flow* f, const el_tuning* t) {
    if (!f || !t) return EL_EINVAL;
    if (t->rk4_threads < 64 || t->rk4_threads > 512 || t->rk4_threads % 32)
        return fail(f, EL_EINVAL, "rk4_threads must be a multiple of 32 in [64, 512]");
    if (t->sort_every < 0) return fail(f, EL_EINVAL, "sort_every must be >= 0");
    if (t->sort_shift < 0 || t->sort_shift > 4 || (1 << t->sort_shift) > f->n / 4)
        return fail(f, EL_EINVAL, "sort_shift out of range");
    if (t->gather < EL_GATHER_AUTO || t->gather > EL_GATHER_SHARED)
        return fail(f, EL_EINVAL, "gather must be EL_GATHER_AUTO, _REGISTERS or _SHARED");
    f->rk4_threads = t->rk4_threads;
    f->gather = t->gather;
    f->d.sort_every = t->sort_every;
    f->sort_shift = t->sort_shift;
    drop_graphs(f);
    batch_member_changed(f->batch);
    return EL_OK;
}

el_status el_autotune(el_flow* f, int32_t trial_steps, el_tuning* best) {
    if (!f || !best) return EL_EINVAL;
    NvtxRange range("el_autotune");
    if (f->batch) return fail(f, EL_ESTATE, "flow belongs to a batch: use el_batch_autotune");
    if (trial_steps < 1) return fail(f, EL_EINVAL, "trial_steps must be >= 1");
    el_tuning start{};
    el_get_tuning(f, &start);
    auto step = [f](int n) { return el_step_coupled(f, n); };
    auto apply = [f](el_tuning t) { return el_set_tuning(f, &t); };
    auto sort_all = [f]() -> el_status {
        for (int s = 0; s < f->d.max_species; s++) EL_TRY(particles_sort(f, s));
        f->since_sort = 0;
        return EL_OK;
    };
    const bool cubic = f->d.interp == EL_CATMULL_ROM || f->d.interp == EL_BSPLINE;
    return autotune_model(step, apply, sort_all, f->stream, start, trial_steps, best, f->n, cubic);
}

el_status el_destroy_flow(el_flow* f) {
    if (!f) return EL_EINVAL;
    if (f->batch) el_batch_remove(f->batch, f);
    cudaStreamSynchronize(f->stream);
    drop_graphs(f);
    destroy_plans(f->plan_c2r, f->plan_r2c, f->plan_c2r1);
    if (f->side) cudaStreamDestroy(f->side);
    if (f->ev_fork) cudaEventDestroy(f->ev_fork);
    if (f->ev_join) cudaEventDestroy(f->ev_join);
    delete f;
    return EL_OK;
}

const char* el_last_error(const el_flow* f) {
    if (!f) return g_create_error.c_str();
    return f->err.c_str();
}

}  // extern "C"
