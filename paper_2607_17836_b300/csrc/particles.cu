// Lagrangian particles (Secs. 2.2, 2.3, 3.2, 3.3; Algorithm 1).
//
// State per particle, split precision: cell (i, j) packed i | j << 16, the
// FP32 offset in the cell in [0, 1)^2, and an int32 periodic image count per
// axis; the unwrapped position is 2 pi * img + (2 pi / n) * (cell + offset).
// Inertial particles also carry their FP32 velocity.  RK4 works in grid
// units relative to the cell origin, so every stage position is a small
// number whatever the particle's distance from the origin, and the carry
// into cell and image is exact integer arithmetic.
//
//   K6 k_rk4       : in rk4.cu
//   K9 k_init      : FP64 positions -> split state; zero-slip velocity
//   k_unsplit      : split state -> FP64 unwrapped positions, original order
//   k_msd / k_box  : per-particle terms of the statistics
#include "common.cuh"
#include "stages.cuh"

#include <algorithm>

namespace el {
namespace {

// FP64 position -> (cell, offset, image), Sec. 3.2: mapped periodically onto
// [0, 2 pi); a point on a node belongs to the cell on its right.
__device__ __forceinline__ void split_position(double x, int n, int& cell, float& off, int& image) {
    const double inv_two_pi = 1.0 / kTwoPi;  // folded at compile time: no division here
    double k = floor(x * inv_two_pi);
    double xw = fma(-kTwoPi, k, x);
    double s = xw * ((double)n * inv_two_pi);
    double c = floor(s);
    float o = (float)(s - c);
    int ci = (int)c, im = (int)k;
    if (o >= 1.0f) {
        o = 0.0f;
        ci += 1;
    }
    while (ci >= n) {
        ci -= n;
        im += 1;
    }
    while (ci < 0) {
        ci += n;
        im -= 1;
    }
    cell = ci;
    off = o;
    image = im;
}

template <int SCHEME>
__device__ float2 fluid_at_dispatch(const float4* snap, int n, int ci, int cj, float ox, float oy,
                                    float wa, float wb) {
    return fluid_at<SCHEME>(snap, n, ci, cj, ox, oy, wa, wb);
}

__device__ float2 fluid_at_scheme(int scheme, const float4* snap, int n, int ci, int cj, float ox,
                                  float oy, float wa, float wb) {
    if (scheme == 0) return fluid_at_dispatch<0>(snap, n, ci, cj, ox, oy, wa, wb);
    if (scheme == 1) return fluid_at_dispatch<1>(snap, n, ci, cj, ox, oy, wa, wb);
    return fluid_at_dispatch<2>(snap, n, ci, cj, ox, oy, wa, wb);
}

// The smallest index of an uploaded value that set_particles refuses: a
// position that is not finite or beyond 1e9 in magnitude (index into xy), else
// a velocity that is not finite (index into vxy, tagged kBadVelocity); the
// word stays all ones when every value is good.
constexpr unsigned long long kBadVelocity = 1ull << 62;

__global__ void k_check_inputs(const double* __restrict__ xy, const double* __restrict__ vxy,
                               int64_t count, unsigned long long* __restrict__ first_bad) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (!(fabs(xy[q]) <= 1e9)) atomicMin(first_bad, (unsigned long long)q);
        if (vxy && !isfinite(vxy[q])) atomicMin(first_bad, kBadVelocity | (unsigned long long)q);
    }
}

// K9: split-precision state from FP64 positions; velocity from vxy, or zero
// slip (the interpolated fluid velocity of the current level: the second
// half of the pair `snap`).
__global__ void k_init(const double* __restrict__ xy, const double* __restrict__ vxy, int64_t np,
                       int n, int scheme, int inertial, const float4* __restrict__ snap,
                       uint32_t* __restrict__ cell, float2* __restrict__ off,
                       float2* __restrict__ vel, int2* __restrict__ img, uint32_t* __restrict__ id,
                       double2* __restrict__ x0) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double x = xy[2 * p], y = xy[2 * p + 1];
    int ci, cj, ix, iy;
    float ox, oy;
    split_position(x, n, ci, ox, ix);
    split_position(y, n, cj, oy, iy);
    cell[p] = (uint32_t)ci | ((uint32_t)cj << 16);
    off[p] = make_float2(ox, oy);
    img[p] = make_int2(ix, iy);
    id[p] = (uint32_t)p;
    x0[p] = make_double2(x, y);
    if (inertial) {
        if (vxy) {
            vel[p] = make_float2((float)vxy[2 * p], (float)vxy[2 * p + 1]);
        } else {
            vel[p] = fluid_at_scheme(scheme, snap, n, ci, cj, ox, oy, 0.0f, 1.0f);
        }
    }
}

__device__ __forceinline__ double2 unwrapped(uint32_t c, float2 o, int2 m, double dx) {
    double x = kTwoPi * (double)m.x + dx * ((double)(c & 0xffffu) + (double)o.x);
    double y = kTwoPi * (double)m.y + dx * ((double)(c >> 16) + (double)o.y);
    return make_double2(x, y);
}

__global__ void k_unsplit(const uint32_t* __restrict__ cell, const float2* __restrict__ off,
                          const float2* __restrict__ vel, const int2* __restrict__ img,
                          const uint32_t* __restrict__ id, int64_t np, double dx, int inertial,
                          double2* __restrict__ xy_out, double2* __restrict__ v_out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    uint32_t k = id[p];
    xy_out[k] = unwrapped(cell[p], off[p], img[p], dx);
    float2 v = inertial ? vel[p] : make_float2(0.f, 0.f);
    v_out[k] = make_double2((double)v.x, (double)v.y);
}

// Squared displacement per particle, stored by original index so that the
// fixed-order reduction that follows does not depend on the sort order.
__global__ void k_msd(const uint32_t* __restrict__ cell, const float2* __restrict__ off,
                      const int2* __restrict__ img, const uint32_t* __restrict__ id,
                      const double2* __restrict__ x0, int64_t np, double dx,
                      double2* __restrict__ out, double2* __restrict__ out2) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    uint32_t k = id[p];
    double2 x = unwrapped(cell[p], off[p], img[p], dx);
    double2 r = x0[k];
    double ddx = x.x - r.x, ddy = x.y - r.y;
    const double sx = ddx * ddx, sy = ddy * ddy;
    out[k] = make_double2(sx, sy);          // squared displacement per axis
    out2[k] = make_double2(sx * sx, sy * sy);  // its square (for the standard error)
}

// Particle counts on the kBoxes x kBoxes box grid (integer atomics: exact).
// With n >= kBoxes every box is a block of whole cells (integer shift);
// coarser grids split cells, done exactly in FP64 (power-of-two scale).
__global__ void k_box(const uint32_t* __restrict__ cell, const float2* __restrict__ off, int64_t np,
                      int n, int log2n, unsigned long long* __restrict__ boxes) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    uint32_t c = cell[p];
    int bx, by;
    if (n >= kBoxes) {
        int sh = log2n - 6;  // kBoxes = 2^6
        bx = (int)(c & 0xffffu) >> sh;
        by = (int)(c >> 16) >> sh;
    } else {
        float2 o = off[p];
        double scale = (double)kBoxes / (double)n;
        bx = (int)(((double)(c & 0xffffu) + (double)o.x) * scale);
        by = (int)(((double)(c >> 16) + (double)o.y) * scale);
        bx = bx > kBoxes - 1 ? kBoxes - 1 : bx;
        by = by > kBoxes - 1 ? kBoxes - 1 : by;
    }
    atomicAdd(boxes + by * kBoxes + bx, 1ull);
}

// Var(n)/mean(n) - 1 from the integer box counts: one block of 1024 threads,
// integer sums (exact, so the order does not matter), then FP64 on one thread.
__global__ void __launch_bounds__(1024) k_cluster_final(const unsigned long long* __restrict__ boxes,
                                                        double* __restrict__ out) {
    __shared__ unsigned long long s1w[32], s2w[32];
    unsigned long long s1 = 0, s2 = 0;
    for (int b = threadIdx.x; b < kBoxes * kBoxes; b += blockDim.x) {
        unsigned long long c = boxes[b];
        s1 += c;
        s2 += c * c;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s1w[threadIdx.x >> 5] = s1;
        s2w[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s1 = s2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            s1 += s1w[w];
            s2 += s2w[w];
        }
        double B = (double)(kBoxes * kBoxes);
        double mean = (double)s1 / B;
        double var = (double)s2 / B - mean * mean;
        *out = mean > 0.0 ? var / mean - 1.0 : 0.0;
    }
}

// Sampling hook: the gather of K6 at arbitrary FP64 points.
__global__ void k_sample(const double* __restrict__ xy, int64_t np, int n, int scheme, float wa,
                         float wb, const float4* __restrict__ snap, double* __restrict__ uv) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int ci, cj, ix, iy;
    float ox, oy;
    split_position(xy[2 * p], n, ci, ox, ix);
    split_position(xy[2 * p + 1], n, cj, oy, iy);
    float2 u = fluid_at_scheme(scheme, snap, n, ci, cj, ox, oy, wa, wb);
    uv[2 * p] = (double)u.x;
    uv[2 * p + 1] = (double)u.y;
}

}  // namespace

static el_status upload_table(el_flow* f) {
    EL_CUDA_OK(f, cudaMemcpyAsync(f->table, f->h_table, sizeof(SpeciesDev) * kMaxSpecies,
                                  cudaMemcpyHostToDevice, f->stream));
    return EL_OK;
}

// Stage, check and place np particles (EL_EINVAL, with nothing of the slot
// changed, when the staged values are refused).
el_status particles_set(el_flow* f, int s, int64_t np, double st, const double* xy,
                        const double* vxy) {
    Species& sp = f->sp[s];
    const int T = 256;
    const int cur = sp.cur;
    // staging in the other (sort) buffer: 32 B per particle
    double* stage = reinterpret_cast<double*>(sp.cell[cur ^ 1]);
    EL_CUDA_OK(f, cudaMemcpyAsync(stage, xy, (size_t)np * 2 * sizeof(double),
                                  cudaMemcpyHostToDevice, f->stream));
    const double* d_vxy = nullptr;
    if (vxy && st > 0.0) {
        EL_CUDA_OK(f, cudaMemcpyAsync(stage + 2 * np, vxy, (size_t)np * 2 * sizeof(double),
                                      cudaMemcpyHostToDevice, f->stream));
        d_vxy = stage + 2 * np;
    }
    if (np > 0) {
        // the staged values, before anything of the species changes
        unsigned long long first = 0;
        EL_CUDA_OK(f, cudaMemsetAsync(f->bad_input, 0xff, sizeof first, f->stream));
        const int64_t cnt = 2 * np;
        const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(cnt, T), 4096);
        k_check_inputs<<<grid, T, 0, f->stream>>>(stage, d_vxy, cnt, f->bad_input);
        EL_LAUNCHED(f);
        EL_CUDA_OK(f, cudaMemcpyAsync(&first, f->bad_input, sizeof first, cudaMemcpyDeviceToHost,
                                      f->stream));
        EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
        if (first != ~0ull) {
            if (first & kBadVelocity)
                return fail(f, EL_EINVAL, "vxy[%lld] is not finite", (long long)(first & ~kBadVelocity));
            return fail(f, EL_EINVAL, "xy[%lld] is not finite or beyond 1e9", (long long)first);
        }
    }
    if (np > 0) {
        k_init<<<blocks_for(np, T), T, 0, f->stream>>>(
            stage, d_vxy, np, f->n, f->d.interp, st > 0.0 ? 1 : 0, f->snap[(f->step + 1) % 2],
            sp.cell[cur], sp.off[cur], sp.vel[cur], sp.img[cur], sp.id[cur], sp.x0);
        EL_LAUNCHED(f);
    }
    sp.np = np;
    sp.st = st;
    EL_TRY(particles_restore_table(f, s));
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    return EL_OK;
}

el_status particles_restore_table(el_flow* f, int s) {
    const Species& sp = f->sp[s];
    SpeciesDev& d = f->h_table[s];
    for (int k = 0; k < 2; k++) {
        d.cell[k] = sp.cell[k];
        d.off[k] = sp.off[k];
        d.vel[k] = sp.vel[k];
        d.img[k] = sp.img[k];
    }
    d.np = (int)sp.np;
    d.cur = sp.cur;
    d.inertial = sp.st > 0.0 ? 1 : 0;
    d.inv_st = sp.st > 0.0 ? (float)(1.0 / sp.st) : 0.0f;
    return upload_table(f);
}


el_status particles_get(el_flow* f, int s, double* xy, double* vxy) {
    Species& sp = f->sp[s];
    const int T = 256;
    const int cur = sp.cur;
    double2* out_xy = reinterpret_cast<double2*>(sp.cell[cur ^ 1]);
    double2* out_v = out_xy + sp.np;
    if (sp.np > 0) {
        k_unsplit<<<blocks_for(sp.np, T), T, 0, f->stream>>>(
            sp.cell[cur], sp.off[cur], sp.vel[cur], sp.img[cur], sp.id[cur], sp.np, kTwoPi / f->n,
            sp.st > 0.0 ? 1 : 0, out_xy, out_v);
        EL_LAUNCHED(f);
        if (xy)
            EL_CUDA_OK(f, cudaMemcpyAsync(xy, out_xy, (size_t)sp.np * sizeof(double2),
                                          cudaMemcpyDeviceToHost, f->stream));
        if (vxy)
            EL_CUDA_OK(f, cudaMemcpyAsync(vxy, out_v, (size_t)sp.np * sizeof(double2),
                                          cudaMemcpyDeviceToHost, f->stream));
    }
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    return EL_OK;
}

// Mean-square displacement (out3[0], out3[1]) and clustering index (out3[2])
// of species s, into device memory.
el_status particles_stats_into(el_flow* f, int s, double* out5) {
    Species& sp = f->sp[s];
    const int T = 256;
    const int cur = sp.cur;
    // the sort buffer holds 32 bytes per particle: both term arrays fit
    double2* terms = reinterpret_cast<double2*>(sp.cell[cur ^ 1]);
    double2* terms2 = terms + sp.np;
    k_msd<<<blocks_for(sp.np, T), T, 0, f->stream>>>(sp.cell[cur], sp.off[cur], sp.img[cur],
                                                     sp.id[cur], sp.x0, sp.np, kTwoPi / f->n, terms,
                                                     terms2);
    EL_LAUNCHED(f);
    EL_TRY(reduce_double2(f, terms, sp.np, out5));
    EL_TRY(reduce_double2(f, terms2, sp.np, out5 + 3));
    double* out3 = out5;
    EL_CUDA_OK(f, cudaMemsetAsync(f->boxes, 0, sizeof(unsigned long long) * kBoxes * kBoxes,
                                  f->stream));
    k_box<<<blocks_for(sp.np, T), T, 0, f->stream>>>(sp.cell[cur], sp.off[cur], sp.np, f->n,
                                                     f->log2n, f->boxes);
    EL_LAUNCHED(f);
    k_cluster_final<<<1, 1024, 0, f->stream>>>(f->boxes, out3 + 2);
    EL_LAUNCHED(f);
    return EL_OK;
}

el_status sample_velocity(el_flow* f, int64_t np, const double* d_xy, double theta, double* d_uv) {
    if (np == 0) return EL_OK;
    const int T = 256;
    // pair (n-1, n): previous level first, current level second
    float th = (float)theta;
    k_sample<<<blocks_for(np, T), T, 0, f->stream>>>(d_xy, np, f->n, f->d.interp, 1.0f - th, th,
                                                      f->snap[(f->step + 1) % 2], d_uv);
    EL_LAUNCHED(f);
    return EL_OK;
}

}  // namespace el

namespace el {

// Clustering index from kBoxes^2 box counts, on a caller-chosen stream; used
// where no flow exists.
cudaError_t launch_cluster_final(cudaStream_t stream, const unsigned long long* boxes,
                                 double* out) {
    k_cluster_final<<<1, 1024, 0, stream>>>(boxes, out);
    return cudaGetLastError();
}

}  // namespace el
