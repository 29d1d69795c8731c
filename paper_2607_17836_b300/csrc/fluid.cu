// Pseudospectral vorticity solver (Sec. 3.1): the pointwise kernels around
// cuFFT's transforms.  Half spectrum [ky][kx], kx = 0..n/2, ky = j for
// j < n/2 and j - n otherwise; physical arrays [j][i].
//
//   K1 k_spec_velocity : omega-hat -> u-hat, v-hat (Eqs. 5, 6), i kx omega-hat,
//                        i ky omega-hat (Eq. 4), scaled by 1/n^2 (the inverse
//                        normalisation of Sec. 3.1), plus prefiltered spline
//                        coefficients of u, v for the B-spline scheme
//   cuFFT C2R (batched): the planes to physical space
//   K3 k_nonlinear     : N = u d(omega)/dx + v d(omega)/dy (Eq. 7), and the
//                        new time level of the particle snapshot
//   cuFFT R2C          : N-hat (Eq. 8)
//   K5 k_ab2           : 2/3 rule + AB2 update (Eqs. 9, 10)
#include "common.cuh"

#include <cmath>
#include <vector>

namespace el {
namespace {

__device__ __forceinline__ int wavenumber_row(int j, int n) { return j < n / 2 ? j : j - n; }

// 2/3 rule: keep iff 3|kx| < n and 3|ky| < n.
__device__ __forceinline__ bool kept(int kx, int ky, int n) {
    return 3 * abs(kx) < n && 3 * abs(ky) < n;
}

__global__ void k_spec_velocity(const float2* __restrict__ what, float2* __restrict__ spec, int n,
                                int nh, size_t nmodes, float scale, int nplanes,
                                const float* __restrict__ pre_x, const float* __restrict__ pre_y) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nmodes) return;
    int j = (int)(q / nh), i = (int)(q - (size_t)j * nh);
    int ky = wavenumber_row(j, n), kx = i;
    float dkx = (i == n / 2) ? 0.f : (float)kx;   // Nyquist: zero derivative
    float dky = (j == n / 2) ? 0.f : (float)ky;
    float k2 = (float)(kx * kx + ky * ky);
    float2 w = what[q];
    w.x *= scale;
    w.y *= scale;
    float ik2 = k2 > 0.f ? 1.f / k2 : 0.f;        // psi-hat(0) = 0
    float2 psi = make_float2(w.x * ik2, w.y * ik2);
    float2 uh = make_float2(-dky * psi.y, dky * psi.x);   // u-hat = i ky psi-hat
    float2 vh = make_float2(dkx * psi.y, -dkx * psi.x);   // v-hat = -i kx psi-hat
    spec[q] = uh;
    spec[nmodes + q] = vh;
    spec[2 * nmodes + q] = make_float2(-dkx * w.y, dkx * w.x);   // i kx omega-hat
    spec[3 * nmodes + q] = make_float2(-dky * w.y, dky * w.x);   // i ky omega-hat
    if (nplanes == 6) {
        // Interpolating cubic-spline coefficients: (c_{i-1} + 4 c_i + c_{i+1})/6 = f_i
        // is diagonal in Fourier space with factor (2 + cos k dx)/3 per axis.
        float p = pre_x[i] * pre_y[j];
        spec[4 * nmodes + q] = make_float2(uh.x * p, uh.y * p);
        spec[5 * nmodes + q] = make_float2(vh.x * p, vh.y * p);
    }
}

// N = u wx + v wy at every node; the stencil field of the new level goes to
// half `h` of the snapshot pair: h = (step + 1) & 1, or both halves at set-up.
__global__ void k_nonlinear(const float* __restrict__ phys, float* __restrict__ nl,
                            float2* __restrict__ snap2, size_t n2, int stencil_plane,
                            const int64_t* __restrict__ d_step, int both) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n2) return;
    float u = phys[q], v = phys[n2 + q], wx = phys[2 * n2 + q], wy = phys[3 * n2 + q];
    nl[q] = fmaf(u, wx, v * wy);
    float2 s = stencil_plane == 0 ? make_float2(u, v)
                                  : make_float2(phys[4 * n2 + q], phys[5 * n2 + q]);
    if (both) {
        snap2[2 * q] = s;
        snap2[2 * q + 1] = s;
    } else {
        int h = (int)((*d_step + 1) & 1);
        snap2[2 * q + h] = s;
    }
}

// Error-free FP32 transformations (double-float arithmetic).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Dealias N-hat and advance omega-hat by one AB2 step (Eqs. 9, 10).
// omega-hat is held as an unevaluated sum w = w_hi + w_lo of two floats: a
// single float would round the small per-step change (the viscous decay is
// only nu k^2 dt of w) the same way step after step and drift by up to half
// an ulp per step; the pair keeps about 44 bits.  Only w_hi feeds the
// transforms.
// mode 0 (integrating factor): E = exp(-nu k^2 dt) = ex[kx] * ey[ky], the 1-D
//   factors computed on the host in FP64 and held as float pairs;
//   w <- E w - dt (3/2 E N - 1/2 E^2 H), H <- N.
// mode 1 (Eq. 10 as printed): R = -N - nu k^2 w; w <- w + dt (3/2 R - 1/2 H), H <- R.
// The first step (step == 0) is forward Euler in either mode.
__global__ void k_ab2(float2* __restrict__ what, float2* __restrict__ what_lo,
                      float2* __restrict__ hist, const float2* __restrict__ nhat, int n, int nh,
                      size_t nmodes, const float2* __restrict__ ex, const float2* __restrict__ ey,
                      float dt, float nu, int mode, const int64_t* __restrict__ d_step) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nmodes) return;
    int j = (int)(q / nh), i = (int)(q - (size_t)j * nh);
    int ky = wavenumber_row(j, n), kx = i;
    bool first = (*d_step == 0);
    float2 N = kept(kx, ky, n) ? nhat[q] : make_float2(0.f, 0.f);
    float2 w = what[q], wl = what_lo[q];
    float2 inc, hi_part;  // new w = hi_part + (lo terms) + inc
    float2 lo;
    if (mode == 0) {
        // E = Eh + El from the float pairs (two-product of the hi parts)
        float2 a = ex[i], b = ey[j];
        float Eh = a.x * b.x;
        float El = fmaf(a.x, b.x, -Eh) + fmaf(a.x, b.y, a.y * b.x);
        float E2 = Eh * Eh;
        float2 H = first ? make_float2(0.f, 0.f) : hist[q];
        float c1 = first ? dt : 1.5f * dt, c2 = first ? 0.f : 0.5f * dt * E2;
        // E * (w_hi + w_lo) - c1 E N + c2 H
        float px = Eh * w.x, py = Eh * w.y;
        float ex_ = fmaf(Eh, w.x, -px), ey_ = fmaf(Eh, w.y, -py);
        inc = make_float2(fmaf(c2, H.x, -c1 * Eh * N.x), fmaf(c2, H.y, -c1 * Eh * N.y));
        hi_part = make_float2(px, py);
        lo = make_float2(ex_ + fmaf(El, w.x, Eh * wl.x), ey_ + fmaf(El, w.y, Eh * wl.y));
        hist[q] = N;
    } else {
        float nuk2 = nu * (float)(kx * kx + ky * ky);
        float2 R = make_float2(-N.x - nuk2 * w.x, -N.y - nuk2 * w.y);
        if (first) {
            inc = make_float2(dt * R.x, dt * R.y);
        } else {
            float2 H = hist[q];
            inc = make_float2(dt * (1.5f * R.x - 0.5f * H.x), dt * (1.5f * R.y - 0.5f * H.y));
        }
        hi_part = w;
        lo = wl;
        hist[q] = R;
    }
    float sx, ex2, sy, ey2;
    two_sum(hi_part.x, lo.x + inc.x, sx, ex2);
    two_sum(hi_part.y, lo.y + inc.y, sy, ey2);
    what[q] = make_float2(sx, sy);
    what_lo[q] = make_float2(ex2, ey2);
}

// Initial projection: mean removed, 2/3 rule (Sec. 3.1).
__global__ void k_project(const float2* __restrict__ src, float2* __restrict__ what, int n, int nh,
                          size_t nmodes) {
    size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nmodes) return;
    int j = (int)(q / nh), i = (int)(q - (size_t)j * nh);
    int ky = wavenumber_row(j, n), kx = i;
    bool keep = kept(kx, ky, n) && !(kx == 0 && ky == 0);
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
__global__ void k_spec_diag(const float2* __restrict__ what, int n, int nh, size_t nmodes,
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

__global__ void k_step_increment(int64_t* d_step) { *d_step += 1; }

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

// Velocity planes, nonlinear term and snapshot of the current omega-hat.
static el_status rhs_from_what(el_flow* f, int both_halves) {
    const int T = 256;
    k_spec_velocity<<<blocks_for((int64_t)f->nmodes, T), T, 0, f->stream>>>(
        f->what, f->spec, f->n, f->nh, f->nmodes, 1.0f / (float)f->n2, f->nplanes, f->pre_x,
        f->pre_y);
    EL_LAUNCHED(f);
    EL_TRY(fft_exec_c2r(f, f->plan_c2r, f->spec, f->phys));
    k_nonlinear<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(
        f->phys, f->nl, reinterpret_cast<float2*>(f->snap), f->n2, f->stencil_plane, f->d_step,
        both_halves);
    EL_LAUNCHED(f);
    EL_TRY(fft_exec_r2c(f, f->nl, f->nhat));
    return EL_OK;
}

el_status fluid_init(el_flow* f, const double* omega0_host) {
    const int T = 256;
    double* stage = f->stage64;
    EL_CUDA_OK(f, cudaMemcpyAsync(stage, omega0_host, f->n2 * sizeof(double),
                                  cudaMemcpyHostToDevice, f->stream));
    k_d2f<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(stage, f->nl, f->n2);
    EL_LAUNCHED(f);
    EL_TRY(fft_exec_r2c(f, f->nl, f->nhat));
    k_project<<<blocks_for((int64_t)f->nmodes, T), T, 0, f->stream>>>(f->nhat, f->what, f->n,
                                                                      f->nh, f->nmodes);
    EL_LAUNCHED(f);
    EL_CUDA_OK(f, cudaMemsetAsync(f->hist, 0, f->nmodes * sizeof(float2), f->stream));
    EL_CUDA_OK(f, cudaMemsetAsync(f->what_lo, 0, f->nmodes * sizeof(float2), f->stream));
    EL_CUDA_OK(f, cudaMemsetAsync(f->d_step, 0, sizeof(int64_t), f->stream));
    EL_TRY(rhs_from_what(f, 1));
    return EL_OK;
}

el_status fluid_step(el_flow* f) {
    const int T = 256;
    k_ab2<<<blocks_for((int64_t)f->nmodes, T), T, 0, f->stream>>>(
        f->what, f->what_lo, f->hist, f->nhat, f->n, f->nh, f->nmodes, f->ex, f->ey,
        (float)f->d.dt, (float)f->d.nu, f->d.ab2_mode, f->d_step);
    EL_LAUNCHED(f);
    return rhs_from_what(f, 0);
}

el_status step_increment(el_flow* f) {
    k_step_increment<<<1, 1, 0, f->stream>>>(f->d_step);
    EL_LAUNCHED(f);
    return EL_OK;
}

el_status fluid_diagnostics(el_flow* f) {
    k_spec_diag<<<kRedBlocks, kRedThreads, 0, f->stream>>>(f->what, f->n, f->nh, f->nmodes, f->red);
    EL_LAUNCHED(f);
    double nn = (double)f->n2;
    k_spec_diag_final<<<1, kRedThreads, 0, f->stream>>>(f->red, kRedBlocks, 0.5 / (nn * nn), f->red_out);
    EL_LAUNCHED(f);
    return EL_OK;
}

el_status fluid_get_field(el_flow* f, int which, double* host_nn) {
    const int T = 256;
    double* out = f->stage64;
    if (which == 0) {
        k_scaled_copy<<<blocks_for((int64_t)f->nmodes, T), T, 0, f->stream>>>(
            f->what, f->aux_spec, f->nmodes, 1.0f / (float)f->n2);
        EL_LAUNCHED(f);
        EL_TRY(fft_exec_c2r(f, f->plan_c2r1, f->aux_spec, f->aux_phys));
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(f->aux_phys, out, f->n2, 1, 0);
    } else if (which == 1 || which == 2) {
        // physical planes 0/1 hold u, v of the current level
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(f->phys + (which - 1) * f->n2,
                                                                   out, f->n2, 1, 0);
    } else {
        // stencil field of the current level: half (step & 1) of the snapshot pair
        int h = (int)(f->step & 1);
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(
            reinterpret_cast<const float*>(f->snap), out, f->n2, 4, 2 * h + (which - 3));
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
