// The prescribed kinematic flow of Sec. 5.2 (time-periodic oscillating
// Taylor-Green eddies) in place of the spectral solver:
//
//   psi = (alpha / k) sin(k [x - eps sin(omega t)]) sin(k [y - eps sin(omega t + phi)]),
//   u = alpha sin(k [x - ...]) cos(k [y - ...]),  v = -alpha cos(k [x - ...]) sin(k [y - ...]).
//
// A "fluid step" writes the field of level m at t = m dt into the level pair
// (m-1, m) (and the streamfunction pair), exactly as the solver's nonlinear
// kernel does, so the particle step, every interpolant and both tracer paths
// run unchanged.  For the prefiltered B-spline the stencil holds the
// interpolating spline coefficients: each factor of the field is a single
// Fourier mode of wavenumber k, and the coefficient condition
// (c_{i-1} + 4 c_i + c_{i+1}) / 6 = f_i maps such a mode to itself times
// P(k) = 3 / (2 + cos(k dx)), so the coefficients are the field times P(k)^2.
#include "common.cuh"
#include "interp.cuh"

#include <cmath>

namespace el {
namespace {

// Level m of the field at every node (one node per thread).
__global__ void k_kinematic_level(int n, int log2n, int kw, float alpha, float dk, float sxv,
                                  float syv, float coef, float psi_coef,
                                  const float4* __restrict__ src, float4* __restrict__ dst,
                                  float4* __restrict__ other, const float2* __restrict__ psi_src,
                                  float2* __restrict__ psi_dst, float2* __restrict__ psi_other) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)n * n) return;
    const int mask = n - 1;
    const int i = (int)(q & mask), j = (int)(q >> log2n);
    float snx, csx, sny, csy;
    sincosf(fmaf(dk, (float)((kw * i) & mask), -sxv), &snx, &csx);
    sincosf(fmaf(dk, (float)((kw * j) & mask), -syv), &sny, &csy);
    const float u = coef * alpha * snx * csy, v = -coef * alpha * csx * sny;
    if (src) {
        const float4 o = src[q];
        dst[q] = make_float4(o.z, o.w, u, v);
    } else {
        dst[q] = make_float4(u, v, u, v);
        other[q] = make_float4(u, v, u, v);
    }
    if (psi_dst) {
        const float ps = psi_coef * snx * sny;
        if (psi_src) {
            psi_dst[q] = make_float2(psi_src[q].y, ps);
        } else {
            psi_dst[q] = make_float2(ps, ps);
            psi_other[q] = make_float2(ps, ps);
        }
    }
}

// omega (which = 0), u (1) or v (2) of the field at time t, FP64, [j][i].
__global__ void k_kinematic_field(int n, int which, double alpha, double k, double sxv, double syv,
                                  double* __restrict__ out) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)n * n) return;
    const int i = (int)(q % n), j = (int)(q / n);
    const double dx = kTwoPi / n;
    double snx, csx, sny, csy;
    sincos(k * (i * dx) - sxv, &snx, &csx);
    sincos(k * (j * dx) - syv, &sny, &csy);
    double r;
    if (which == 0)
        r = 2.0 * alpha * k * snx * sny;  // omega = -laplacian(psi) = 2 k^2 psi
    else if (which == 1)
        r = alpha * snx * csy;
    else
        r = -alpha * csx * sny;
    out[q] = r;
}

}  // namespace

// Phase shifts k eps sin(omega t) and k eps sin(omega t + phi) at t, FP64.
static void kinematic_shifts(const el_flow* f, double t, double& sx, double& sy) {
    const el_kinematic& k = f->kin;
    sx = k.k * k.eps * std::sin(k.omega * t);
    sy = k.k * k.eps * std::sin(k.omega * t + k.phi);
}

KinArgs kinematic_stage_args(const el_flow* f, int64_t step) {
    KinArgs a{};
    a.alpha = (float)f->kin.alpha;
    a.dk = (float)(kTwoPi / f->n);
    a.kw = (int)f->kin.k;
    a.mask = f->n - 1;
    const double t0 = (double)step * f->d.dt;
    const double c[3] = {0.0, 0.5, 1.0};  // stage times t_n, t_n + dt/2, t_n + dt
    for (int s = 0; s < 3; s++) {
        double sx, sy;
        kinematic_shifts(f, t0 + c[s] * f->d.dt, sx, sy);
        a.sx[s] = (float)sx;
        a.sy[s] = (float)sy;
    }
    return a;
}

// Level m into pair (m-1, m) = snap[(m + 1) % 2]; at set-up level 0 fills
// both halves of both pairs.
el_status kinematic_level(el_flow* f, int64_t m, bool setup) {
    const int T = 256;
    double sx, sy;
    kinematic_shifts(f, (double)m * f->d.dt, sx, sy);
    const bool spline = f->stencil_plane != 0;
    const double kdx = f->kin.k * kTwoPi / f->n;
    const double pk = 3.0 / (2.0 + std::cos(kdx));
    const double coef = spline ? pk * pk : 1.0;
    const bool psi = f->psi_plane >= 0;
    k_kinematic_level<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(
        f->n, f->log2n, (int)f->kin.k, (float)f->kin.alpha, (float)(kTwoPi / f->n), (float)sx,
        (float)sy, (float)coef, (float)(coef * f->kin.alpha / f->kin.k),
        setup ? nullptr : f->snap[m % 2], f->snap[(m + 1) % 2], setup ? f->snap[m % 2] : nullptr,
        (psi && !setup) ? f->psi[m % 2] : nullptr, psi ? f->psi[(m + 1) % 2] : nullptr,
        (psi && setup) ? f->psi[m % 2] : nullptr);
    EL_LAUNCHED(f);
    return EL_OK;
}

el_status kinematic_get_field(el_flow* f, int which, double* host_nn) {
    const int T = 256;
    double sx, sy;
    kinematic_shifts(f, (double)f->step * f->d.dt, sx, sy);
    k_kinematic_field<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(
        f->n, which, f->kin.alpha, f->kin.k, sx, sy, f->stage64);
    EL_LAUNCHED(f);
    EL_CUDA_OK(f, cudaMemcpyAsync(host_nn, f->stage64, f->n2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  f->stream));
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    return EL_OK;
}

// Domain means of the field (exact for the grid too when n > 2k):
// E = alpha^2 / 4, Z = alpha^2 k^2 / 2, P = alpha^2 k^4.
void kinematic_diagnostics(const el_flow* f, double* e3) {
    const double a2 = f->kin.alpha * f->kin.alpha, k2 = f->kin.k * f->kin.k;
    e3[0] = 0.25 * a2;
    e3[1] = 0.5 * a2 * k2;
    e3[2] = a2 * k2 * k2;
}

}  // namespace el
