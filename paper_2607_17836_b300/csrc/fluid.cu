// Pseudospectral vorticity solver (Sec. 3.1): the pointwise kernels around
// cuFFT's transforms.  Half spectrum [ky][kx], kx = 0..n/2, ky = j for
// j < n/2 and j - n otherwise; physical arrays [j][i].  One step:
//
//   K5+K1 k_spectral<true> : 2/3 rule + AB2 update of omega-hat (Eqs. 9, 10),
//                            then from the new omega-hat: u-hat, v-hat
//                            (Eqs. 5, 6), i kx omega-hat, i ky omega-hat
//                            (Eq. 4), scaled by 1/n^2 (the inverse
//                            normalisation of Sec. 3.1), and for the B-spline
//                            scheme the prefiltered spline coefficients
//   cuFFT C2R (batched)    : the planes to physical space
//   K3 k_nonlinear         : N = u d(omega)/dx + v d(omega)/dy (Eq. 7), and the
//                            level pair (n, n+1) the particle step reads
//   cuFFT R2C              : N-hat (Eq. 8)
//
// Modes are addressed by a 2-D grid (blockIdx.y = row j), so no thread
// divides by n/2 + 1.
#include "common.cuh"
#include "stages.cuh"

#include <cmath>
#include <vector>

namespace el {
namespace {

constexpr int kSpecThreads = 128;

// Threads cover kx = 0..n/2-1 of row blockIdx.y; the thread of kx = 0 also
// takes the Nyquist column kx = n/2.
template <bool ADVANCE>
__global__ void __launch_bounds__(kSpecThreads) k_spectral(const __grid_constant__ SpecArgs a) {
    const int i = blockIdx.x * kSpecThreads + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= a.n / 2) return;
    spectral_mode<ADVANCE>(a, i, j);
    if (i == 0) spectral_mode<ADVANCE>(a, a.n / 2, j);
}

// N and the level pair of the new level at every node (nonlinear_node).
__global__ void k_nonlinear(const float* __restrict__ phys, float* __restrict__ nl,
                            const float4* __restrict__ src, float4* __restrict__ dst,
                            float4* __restrict__ other, size_t n2, int stencil_plane,
                            int psi_plane, const float2* __restrict__ psi_src,
                            float2* __restrict__ psi_dst, float2* __restrict__ psi_other) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    nonlinear_node(phys, nl, src, dst, other, n2, i, stencil_plane, psi_plane, psi_src, psi_dst,
                   psi_other);
}

// Initial projection: mean removed, 2/3 rule (Sec. 3.1).
__global__ void k_project(const float2* __restrict__ src, float2* __restrict__ what, int n, int nh) {
    const int i = blockIdx.x * kSpecThreads + threadIdx.x, j = blockIdx.y;
    if (i >= nh) return;
    const size_t q = (size_t)j * nh + i;
    const int ky = wavenumber_row(j, n), kx = i;
    const bool keep = kept(kx, ky, n) && !(kx == 0 && ky == 0);
    what[q] = keep ? src[q] : make_float2(0.f, 0.f);
}

__global__ void k_d2f(const double* __restrict__ src, float* __restrict__ dst, size_t count) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count) dst[q] = (float)src[q];
}

__global__ void k_f2d(const float* __restrict__ src, double* __restrict__ dst, size_t count,
                      int stride, int offset) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count) dst[q] = (double)src[q * stride + offset];
}

// omega-hat / n^2 into the auxiliary spectrum (for the physical vorticity).
__global__ void k_scaled_copy(const float2* __restrict__ src, float2* __restrict__ dst,
                              size_t nmodes, float scale) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nmodes) dst[q] = make_float2(src[q].x * scale, src[q].y * scale);
}

// FP64 partial sums over the half spectrum for E, Z, P (Parseval).  Modes
// with 0 < kx < n/2 stand for themselves and their conjugates (weight 2).
__global__ void __launch_bounds__(kRedThreads) k_spec_diag(const float2* __restrict__ what, int n,
                                                           int nh, size_t nmodes,
                                                           double* __restrict__ partial) {
    double se = 0.0, sz = 0.0, sp = 0.0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nmodes;
         q += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(q / nh), i = (int)(q - (size_t)j * nh);
        int ky = wavenumber_row(j, n), kx = i;
        double k2 = (double)kx * kx + (double)ky * ky;
        double wgt = (i == 0 || i == n / 2) ? 1.0 : 2.0;
        double a = (double)what[q].x, b = (double)what[q].y;
        double m = wgt * (a * a + b * b);
        sz += m;
        sp += k2 * m;
        se += k2 > 0.0 ? m / k2 : 0.0;
    }
    __shared__ double sh[3][kRedThreads / 32];
    double v[3] = {se, sz, sp};
    for (int c = 0; c < 3; c++) {
        double x = v[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++) {
            double x = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) x += sh[c][w];
            partial[(size_t)blockIdx.x * 3 + c] = x;
        }
    }
}

// Sum of the block partials in a fixed tree (one block of kRedThreads).
__global__ void __launch_bounds__(kRedThreads) k_spec_diag_final(const double* __restrict__ partial,
                                                                 int nblocks, double scale,
                                                                 double* __restrict__ out) {
    __shared__ double sh[3][kRedThreads / 32];
    for (int c = 0; c < 3; c++) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) x += partial[(size_t)b * 3 + c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0.0;
        for (int w = 0; w < kRedThreads / 32; w++) x += sh[threadIdx.x][w];
        out[threadIdx.x] = x * scale;
    }
}

}  // namespace

static el_status fft_exec_c2r(el_flow* f, cufftHandle plan, float2* in, float* out) {
    cufftResult r = cufftExecC2R(plan, reinterpret_cast<cufftComplex*>(in), out);
    if (r != CUFFT_SUCCESS) return fail(f, EL_ECUFFT, "cufftExecC2R failed (%d)", (int)r);
    return EL_OK;
}

static el_status fft_exec_r2c(el_flow* f, float* in, float2* out) {
    cufftResult r = cufftExecR2C(f->plan_r2c, in, reinterpret_cast<cufftComplex*>(out));
    if (r != CUFFT_SUCCESS) return fail(f, EL_ECUFFT, "cufftExecR2C failed (%d)", (int)r);
    return EL_OK;
}

static SpecArgs spec_args(el_flow* f, int first) {
    SpecArgs a{};
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
    a.first = first;
    a.nmodes = f->nmodes;
    a.scale = 1.0f / (float)f->n2;
    a.dt = (float)f->d.dt;
    a.nu = (float)f->d.nu;
    return a;
}

// Planes -> physical fields, nonlinear term, the pair (m-1, m) of the new
// level m (pair (k, k+1) is snap[k % 2]), N-hat.
static el_status finish_rhs(el_flow* f, int64_t m, bool setup) {
    const int T = 256;
    EL_TRY(fft_exec_c2r(f, f->plan_c2r, f->spec, f->phys));
    float4* dst = f->snap[(m + 1) % 2];        // pair (m-1, m)
    const float4* src = f->snap[m % 2];        // pair (m-2, m-1): level m-1 in its second half
    k_nonlinear<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(
        f->phys, f->nl, setup ? nullptr : src, dst, setup ? f->snap[m % 2] : nullptr, f->n2,
        f->stencil_plane, f->psi_plane, setup ? nullptr : f->psi[m % 2], f->psi[(m + 1) % 2],
        setup ? f->psi[m % 2] : nullptr);
    EL_LAUNCHED(f);
    EL_TRY(fft_exec_r2c(f, f->nl, f->nhat));
    return EL_OK;
}

static dim3 spec_grid(el_flow* f) {
    return dim3((unsigned)((f->n / 2 + kSpecThreads - 1) / kSpecThreads), (unsigned)f->n);
}

el_status fluid_init(el_flow* f, const double* omega0_host) {
    const int T = 256;
    double* stage = f->stage64;
    EL_CUDA_OK(f, cudaMemcpyAsync(stage, omega0_host, f->n2 * sizeof(double),
                                  cudaMemcpyHostToDevice, f->stream));
    k_d2f<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(stage, f->nl, f->n2);
    EL_LAUNCHED(f);
    EL_TRY(fft_exec_r2c(f, f->nl, f->nhat));
    k_project<<<dim3((unsigned)((f->nh + kSpecThreads - 1) / kSpecThreads), (unsigned)f->n),
                kSpecThreads, 0, f->stream>>>(f->nhat, f->what, f->n, f->nh);
    EL_LAUNCHED(f);
    EL_CUDA_OK(f, cudaMemsetAsync(f->hist, 0, f->nmodes * sizeof(float2), f->stream));
    EL_CUDA_OK(f, cudaMemsetAsync(f->what_lo, 0, f->nmodes * sizeof(float2), f->stream));
    k_spectral<false><<<spec_grid(f), kSpecThreads, 0, f->stream>>>(spec_args(f, 0));
    EL_LAUNCHED(f);
    return finish_rhs(f, 0, true);
}

// Fluid n -> n+1 for step number n = `step`.
el_status fluid_step(el_flow* f, int64_t step) {
    NvtxRange range("fluid_step");
    if (f->kinematic) return kinematic_level(f, step + 1, false);
    if (f->fused) return fluid_step_fused(f, spec_args(f, step == 0), step);
    k_spectral<true><<<spec_grid(f), kSpecThreads, 0, f->stream>>>(spec_args(f, step == 0));
    EL_LAUNCHED(f);
    return finish_rhs(f, step + 1, false);
}

// The physical planes (u, v, ...) of the current level from omega-hat,
// without touching N-hat or the level pairs (after a state was loaded).
el_status fluid_refresh_planes(el_flow* f) {
    if (f->kinematic) return EL_OK;  // nothing spectral to rebuild
    k_spectral<false><<<spec_grid(f), kSpecThreads, 0, f->stream>>>(spec_args(f, 0));
    EL_LAUNCHED(f);
    return fft_exec_c2r(f, f->plan_c2r, f->spec, f->phys);
}

el_status fluid_diagnostics(el_flow* f) {
    k_spec_diag<<<kRedBlocks, kRedThreads, 0, f->stream>>>(f->what, f->n, f->nh, f->nmodes, f->red);
    EL_LAUNCHED(f);
    double nn = (double)f->n2;
    k_spec_diag_final<<<1, kRedThreads, 0, f->stream>>>(f->red, kRedBlocks, 0.5 / (nn * nn),
                                                        f->red_out);
    EL_LAUNCHED(f);
    return EL_OK;
}

el_status fluid_get_field(el_flow* f, int which, double* host_nn) {
    if (f->kinematic && which <= 2) return kinematic_get_field(f, which, host_nn);
    const int T = 256;
    double* out = f->stage64;
    if (which == 0) {
        k_scaled_copy<<<blocks_for((int64_t)f->nmodes, T), T, 0, f->stream>>>(
            f->what, f->aux_spec, f->nmodes, 1.0f / (float)f->n2);
        EL_LAUNCHED(f);
        EL_TRY(fft_exec_c2r(f, f->plan_c2r1, f->aux_spec, f->aux_phys));
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(f->aux_phys, out, f->n2, 1, 0);
    } else if (which == 1 || which == 2) {
        // physical planes 0/1 hold u, v of the current level (the fused step
        // does not write them: rebuild them from omega-hat first)
        if (f->fused) EL_TRY(fluid_refresh_planes(f));
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(f->phys + (which - 1) * f->n2,
                                                                   out, f->n2, 1, 0);
    } else {
        // stencil field of the current level n: second half of pair (n-1, n)
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(
            reinterpret_cast<const float*>(f->snap[(f->step + 1) % 2]), out, f->n2, 4,
            2 + (which - 3));
    }
    EL_LAUNCHED(f);
    EL_CUDA_OK(f, cudaMemcpyAsync(host_nn, out, f->n2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  f->stream));
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    return EL_OK;
}

// Host-side FP64 tables: the 1-D integrating factors exp(-nu k^2 dt) as
// float pairs (hi, lo), and the spline prefilter factors 3 / (2 + cos k dx).
void fluid_tables(const el_flow_desc& d, std::vector<float2>& ex, std::vector<float2>& ey,
                  std::vector<float>& px, std::vector<float>& py) {
    int n = d.n, nh = n / 2 + 1;
    ex.resize(nh);
    px.resize(nh);
    ey.resize(n);
    py.resize(n);
    double dxg = kTwoPi / n;
    auto pair = [](double v) {
        float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    for (int i = 0; i < nh; i++) {
        double k = i;
        ex[i] = pair(std::exp(-d.nu * k * k * d.dt));
        px[i] = (float)(3.0 / (2.0 + std::cos(k * dxg)));
    }
    for (int j = 0; j < n; j++) {
        double k = j < n / 2 ? j : j - n;
        ey[j] = pair(std::exp(-d.nu * k * k * d.dt));
        py[j] = (float)(3.0 / (2.0 + std::cos(k * dxg)));
    }
}

}  // namespace el
