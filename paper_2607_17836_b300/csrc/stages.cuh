// Per-element bodies of the step kernels, shared by the single-flow kernels
// (fluid.cu, rk4.cu) and the batched kernels (batch.cu), so that a
// simulation advanced alone or inside a batch does the same arithmetic.
#pragma once

#include "common.cuh"
#include "interp.cuh"

#ifndef EL_STREAMING_STATE
#define EL_STREAMING_STATE 1
#endif

// Register caps of the cubic schemes' particle kernels (single-flow k_rk4 and
// batched k_batch_rk4).  Register-cached stencils: 96 (4-8 B of spills) fits
// 5 blocks of 128 threads per SM against 4 at their natural 120, 8-10 %
// faster at 1024^2 (4 and 16 particles per cell); 80 spills 250 B and is
// slower.  Warp-shared stencils (PatchStencil: nothing large stays in
// registers): 56, measured against 48 and 64 at 16 particles per cell.
#ifndef EL_RK4_CUBIC_MAXNREG
#define EL_RK4_CUBIC_MAXNREG 96
#endif
#ifndef EL_RK4_SHARED_MAXNREG
#define EL_RK4_SHARED_MAXNREG 56
#endif
// The L2 prefetch distance of the particle kernels in resident waves (SMs x
// resident blocks).  Measured at 1024^2: 0.5, 1 and 2 waves time alike, 4-5 %
// faster than no prefetch for every scheme and particle count.
#ifndef EL_RK4_PREFETCH_WAVES
#define EL_RK4_PREFETCH_WAVES 1.0
#endif

#if EL_STREAMING_STATE
#define EL_STATE_LD(ptr) __ldcs(ptr)
#define EL_STATE_ST(ptr, v) __stcs(ptr, v)
#else
#define EL_STATE_LD(ptr) (*(ptr))
#define EL_STATE_ST(ptr, v) (*(ptr) = (v))
#endif

namespace el {

__device__ __forceinline__ int wavenumber_row(int j, int n) { return j < n / 2 ? j : j - n; }

// 2/3 rule: keep iff 3|kx| < n and 3|ky| < n.
__device__ __forceinline__ bool kept(int kx, int ky, int n) {
    return 3 * abs(kx) < n && 3 * abs(ky) < n;
}

// Error-free FP32 sum (double-float arithmetic).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

struct SpecArgs {
    float2* what;       // omega-hat, high part
    float2* what_lo;    // omega-hat, low part
    float2* hist;       // AB2 history
    const float2* nhat; // N-hat of the current level
    float2* spec;       // nplanes output half spectra
    const float2* ex;   // exp(-nu kx^2 dt) as (hi, lo)
    const float2* ey;   // exp(-nu ky^2 dt) as (hi, lo)
    const float* pre_x;
    const float* pre_y;
    int n, nh, nplanes, mode, first;
    int spline;         // 1: write prefiltered cu, cv to planes 4, 5
    int psi_plane;      // plane of the streamfunction stencil field, or -1
    size_t nmodes;
    float scale, dt, nu;
};

// One batched flow's fused 1024^2 fluid step (fused_fluid.cu), device-resident:
// everything but what depends on the step number, which the kernels derive
// from the member's step counter on the device.
struct FusedMember {
    SpecArgs spec;            // its `first` is set on the device
    float2* S;                // planes before the column transforms
    float2* G;                // after them
    float2* H;                // N after the row transforms
    float2* nhat;             // N-hat (read by the AB2 update, then written)
    float4* snap[2];          // level pairs: snap[k % 2] = levels (k, k+1)
    float2* psi[2];           // streamfunction pairs, or nullptr
    const long long* step;    // the member's step counter
    int psi_plane;
};

// AB2 update (when ADVANCE) and the spectral velocity / gradient planes of
// the resulting omega-hat.
//
// omega-hat is held as an unevaluated sum w_hi + w_lo of two floats: one
// float would round the small per-step change (the viscous decay is only
// nu k^2 dt of w) the same way step after step and drift by up to half an
// ulp per step; the pair keeps about 44 bits.  Only w_hi feeds the planes.
// mode 0 (integrating factor): E = exp(-nu k^2 dt) = ex[kx] * ey[ky] (the 1-D
//   factors computed on the host in FP64, held as float pairs);
//   w <- E w - dt (3/2 E N - 1/2 E^2 H), H <- N.
// mode 1 (Eq. 10 as printed): R = -N - nu k^2 w; w <- w + dt (3/2 R - 1/2 H), H <- R.
// The first step is forward Euler in either mode.
// What the AB2 update of one mode reads.
struct ModeIn {
    float2 w, N, wl, H, ea, eb;
};

// The loads of the AB2 update of mode (i, j) (row-major index q), all issued
// together.
__device__ __forceinline__ ModeIn load_mode(const SpecArgs& a, int i, int j, size_t q) {
    const float2* __restrict__ nhat = a.nhat;
    const float2* __restrict__ hist_in = a.hist;
    const float2* __restrict__ lo_in = a.what_lo;
    ModeIn in;
    in.w = a.what[q];
    in.N = nhat[q];
    in.wl = lo_in[q];
    in.H = make_float2(0.f, 0.f);
    in.ea = in.H;
    in.eb = in.H;
    if (!a.first) in.H = hist_in[q];
    if (a.mode == 0) {
        in.ea = a.ex[i];
        in.eb = a.ey[j];
    }
    return in;
}

// The AB2 update of mode (i, j) from its loaded inputs: writes the new
// omega-hat (both parts) and history, returns the new high part.
__device__ __forceinline__ float2 advance_loaded(const SpecArgs& a, int i, int j, size_t q, const ModeIn& in) {
    const int n = a.n;
    const int kx = i, ky = wavenumber_row(j, n);
    const bool keep = kept(kx, ky, n);
    float2 w = in.w, N = in.N;
    const float2 wl = in.wl, H = in.H, ea = in.ea, eb = in.eb;
    if (!keep) N = make_float2(0.f, 0.f);
    const float dt = a.dt;
    float2 inc, hi, lo, hist_out;
    if (a.mode == 0) {
        float Eh = ea.x * eb.x;  // E = Eh + El (two-product of the hi parts)
        float El = fmaf(ea.x, eb.x, -Eh) + fmaf(ea.x, eb.y, ea.y * eb.x);
        float E2 = Eh * Eh;
        float c1 = a.first ? dt : 1.5f * dt, c2 = a.first ? 0.f : 0.5f * dt * E2;
        float px = Eh * w.x, py = Eh * w.y;
        hi = make_float2(px, py);
        lo = make_float2(fmaf(Eh, w.x, -px) + fmaf(El, w.x, Eh * wl.x),
                         fmaf(Eh, w.y, -py) + fmaf(El, w.y, Eh * wl.y));
        inc = make_float2(fmaf(c2, H.x, -c1 * Eh * N.x), fmaf(c2, H.y, -c1 * Eh * N.y));
        hist_out = N;
    } else {
        // Eq. 10 with every rounding written out (fmaf where one rounding is
        // meant, __fmul_rn where a product rounds by itself): nothing is left
        // for the compiler to contract, so every kernel that inlines this
        // update (one flow or a batch) rounds it the same way
        const float nuk2 = __fmul_rn(a.nu, (float)(kx * kx + ky * ky));
        const float2 R = make_float2(fmaf(-nuk2, w.x, -N.x), fmaf(-nuk2, w.y, -N.y));
        inc = a.first ? make_float2(__fmul_rn(dt, R.x), __fmul_rn(dt, R.y))
                      : make_float2(__fmul_rn(dt, fmaf(1.5f, R.x, __fmul_rn(-0.5f, H.x))),
                                    __fmul_rn(dt, fmaf(1.5f, R.y, __fmul_rn(-0.5f, H.y))));
        hi = w;
        lo = wl;
        hist_out = R;
    }
    float sx, exx, sy, eyy;
    two_sum(hi.x, lo.x + inc.x, sx, exx);
    two_sum(hi.y, lo.y + inc.y, sy, eyy);
    w = make_float2(sx, sy);
    a.hist[q] = hist_out;
    a.what[q] = w;
    a.what_lo[q] = make_float2(exx, eyy);
    return w;
}

// The AB2 update of mode (i, j) (row-major index q), reading N-hat, the low
// part and the history and writing the new omega-hat (both parts) and
// history; returns the new high part.
__device__ __forceinline__ float2 advance_mode(const SpecArgs& a, int i, int j, size_t q) {
    return advance_loaded(a, i, j, q, load_mode(a, i, j, q));
}

// Plane `p` of the spectral planes of omega-hat w (high part) at mode (i, j):
// 0 u-hat = i ky psi-hat, 1 v-hat = -i kx psi-hat (Eqs. 5, 6; psi-hat = w/k^2,
// psi-hat(0) = 0), 2 i kx w, 3 i ky w (Eq. 4), then with the spline prefilter
// 4, 5 = u-hat, v-hat times the prefilter factor pre_x[i] pre_y[j], and
// psi_plane = psi-hat (times the same factor with the prefilter), all scaled
// by 1/n^2 (the inverse transform's normalisation).
__device__ __forceinline__ float2 plane_value(const SpecArgs& a, int p, int i, int j, float2 w) {
    const int n = a.n;
    const int kx = i, ky = wavenumber_row(j, n);
    const float dkx = (i == n / 2) ? 0.f : (float)kx;  // Nyquist: zero derivative
    const float dky = (j == n / 2) ? 0.f : (float)ky;
    const float k2 = (float)(kx * kx + ky * ky);
    w.x *= a.scale;
    w.y *= a.scale;
    if (p == 2) return make_float2(-dkx * w.y, dkx * w.x);
    if (p == 3) return make_float2(-dky * w.y, dky * w.x);
    const float ik2 = k2 > 0.f ? 1.f / k2 : 0.f;
    const float2 psi = make_float2(w.x * ik2, w.y * ik2);
    const float pf = (a.spline && p >= 4) ? a.pre_x[i] * a.pre_y[j] : 1.0f;
    if (p == a.psi_plane) return make_float2(psi.x * pf, psi.y * pf);
    if (p == 0 || p == 4) {
        const float2 uh = make_float2(-dky * psi.y, dky * psi.x);
        return p == 0 ? uh : make_float2(uh.x * pf, uh.y * pf);
    }
    const float2 vh = make_float2(dkx * psi.y, -dkx * psi.x);
    return p == 1 ? vh : make_float2(vh.x * pf, vh.y * pf);
}

// AB2 update (when ADVANCE) and the spectral velocity / gradient planes of
// the resulting omega-hat.
//
// omega-hat is held as an unevaluated sum w_hi + w_lo of two floats: one
// float would round the small per-step change (the viscous decay is only
// nu k^2 dt of w) the same way step after step and drift by up to half an
// ulp per step; the pair keeps about 44 bits.  Only w_hi feeds the planes.
// mode 0 (integrating factor): E = exp(-nu k^2 dt) = ex[kx] * ey[ky] (the 1-D
//   factors computed on the host in FP64, held as float pairs);
//   w <- E w - dt (3/2 E N - 1/2 E^2 H), H <- N.
// mode 1 (Eq. 10 as printed): R = -N - nu k^2 w; w <- w + dt (3/2 R - 1/2 H), H <- R.
// The first step is forward Euler in either mode.
template <bool ADVANCE>
__device__ __forceinline__ void spectral_mode(const SpecArgs& a, int i, int j) {
    const size_t q = (size_t)j * a.nh + i;
    const float2 w = ADVANCE ? advance_mode(a, i, j, q) : a.what[q];
    const size_t m = a.nmodes;
    float2* __restrict__ spec = a.spec;
    spec[q] = plane_value(a, 0, i, j, w);
    spec[m + q] = plane_value(a, 1, i, j, w);
    spec[2 * m + q] = plane_value(a, 2, i, j, w);
    spec[3 * m + q] = plane_value(a, 3, i, j, w);
    if (a.spline) {
        spec[4 * m + q] = plane_value(a, 4, i, j, w);
        spec[5 * m + q] = plane_value(a, 5, i, j, w);
    }
    if (a.psi_plane >= 0) spec[(size_t)a.psi_plane * m + q] = plane_value(a, a.psi_plane, i, j, w);
}

// N = u wx + v wy at node i (Eq. 7), and node i's level pair (m-1, m) of the
// new level m: `dst` = (level m-1 read from the second half of `src`, level
// m), one full 16-byte store.  At set-up (src == nullptr) level 0 fills both
// halves of `dst` and of `other`, so no pair ever holds uninitialised values
// (a blend weight of 0 times a NaN left in reused memory is NaN).  The n2
// floats of each physical plane follow one another in `phys`.  One node per
// thread: scalar plane loads, the pair loads and stores contiguous across the
// warp (11.7 -> 9.2 us at 1024^2 against four nodes per thread).
__device__ __forceinline__ void nonlinear_node(const float* __restrict__ phys,
                                               float* __restrict__ nl,
                                               const float4* __restrict__ src,
                                               float4* __restrict__ dst,
                                               float4* __restrict__ other, size_t n2, size_t i,
                                               int stencil_plane, int psi_plane,
                                               const float2* __restrict__ psi_src,
                                               float2* __restrict__ psi_dst,
                                               float2* __restrict__ psi_other) {
    float u = phys[i], v = phys[n2 + i];
    const float wx = phys[2 * n2 + i], wy = phys[3 * n2 + i];
    nl[i] = fmaf(u, wx, v * wy);
    if (stencil_plane != 0) {
        u = phys[4 * n2 + i];
        v = phys[5 * n2 + i];
    }
    if (src) {
        const float4 old = src[i];
        dst[i] = make_float4(old.z, old.w, u, v);
    } else {
        const float4 both = make_float4(u, v, u, v);
        dst[i] = both;
        other[i] = both;
    }
    if (psi_plane >= 0) {  // the streamfunction stencil field, same pair layout (scalar)
        const float pk = phys[(size_t)psi_plane * n2 + i];
        if (src) {
            psi_dst[i] = make_float2(psi_src[i].y, pk);
        } else {
            psi_dst[i] = make_float2(pk, pk);
            psi_other[i] = make_float2(pk, pk);
        }
    }
}

// Carry an offset that left [0, 1) into the cell index and the image count.
__device__ __forceinline__ void carry_axis(float x, int c, int log2n, float& off, int& cell,
                                           int& dimg) {
    float fl = floorf(x);
    float o = x - fl;
    int k = (int)fl;
    if (o >= 1.0f) {  // x - floor(x) rounded up to 1 for x just below an integer
        o = 0.0f;
        k += 1;
    }
    int c2 = c + k;
    dimg = c2 >> log2n;              // floor division by n
    cell = c2 & ((1 << log2n) - 1);  // the remainder, in [0, n)
    off = o;
}

// A particle between the load of its state and stencil and its update.
template <int SCHEME>
struct ParticleRK4 {
    int p, ci, cj;
    float2 o, v;
    Stencil<SCHEME> st;
};

// The particle state (streamed once per step: evict-first loads keep the
// caches for the level pair the gathers re-read).
template <int SCHEME>
__device__ __forceinline__ void rk4_load_state(const SpeciesDev& sd, int p, ParticleRK4<SCHEME>& q) {
    const int cur = sd.cur;
    const uint32_t c = EL_STATE_LD(sd.cell[cur] + p);
    q.p = p;
    q.ci = (int)(c & 0xffffu);
    q.cj = (int)(c >> 16);
    q.o = EL_STATE_LD(sd.off[cur] + p);
    q.v = sd.inertial ? EL_STATE_LD(sd.vel[cur] + p) : make_float2(0.f, 0.f);
}

// One RK4 step (Eq. 12 tracers, Eq. 14 inertial) between levels n and n+1,
// read from their level pair `snap`, of a particle whose state and stencil
// are loaded: stage 1 (theta = 0) and stage 4 (theta = 1) read one half of
// each node without blending.  All (x, y) and (u, v) arithmetic is on float
// pairs (one paired FP32 instruction per two lanes of work).  h = dt * n /
// (2 pi): grid units per unit velocity.  Writes the new state.
//
// G supplies the fluid velocity at the stages: first_stage<THETA>(o) in the
// particle's own cell, to_mid() after it, at<THETA>(snap, n, ci, cj, l) at
// grid-unit position l relative to cell (ci, cj) (Stencil: a register cache
// of one cell's nodes; PatchStencil: a warp's shared-memory patch).
template <class G>
__device__ __forceinline__ void rk4_update(const float4* __restrict__ snap, int n, int log2n, float dt,
                                           float h, const SpeciesDev& sd, int p, int ci, int cj,
                                           float2 o, float2 vel, G& st) {
    const int cur = sd.cur;
    const float2 h2 = make_float2(0.5f * h, 0.5f * h), h1 = make_float2(h, h);
    const float2 two = make_float2(2.0f, 2.0f);
    float2 np2;
    if (!sd.inertial) {
        // Eq. 12, stages at t, t + dt/2, t + dt/2, t + dt (theta = 0, 1/2, 1/2, 1)
        float2 k1 = st.template first_stage<0>(o);
        st.to_mid();
        float2 k2 = st.template at<1>(snap, n, ci, cj, __ffma2_rn(h2, k1, o));
        float2 k3 = st.template at<1>(snap, n, ci, cj, __ffma2_rn(h2, k2, o));
        float2 k4 = st.template at<2>(snap, n, ci, cj, __ffma2_rn(h1, k3, o));
        float2 sum = __fadd2_rn(__ffma2_rn(two, __fadd2_rn(k2, k3), k1), k4);
        const float h6 = h * (1.0f / 6.0f);
        np2 = __ffma2_rn(make_float2(h6, h6), sum, o);
    } else {
        // Eq. 14: x and v jointly; stage s has x_s = x + c_s dt v_{s-1},
        // v_s = v + c_s dt a_{s-1}, a_s = (u(x_s, t_s) - v_s) / St (Eq. 13).
        const float2 ist = make_float2(sd.inv_st, sd.inv_st);
        const float2 d2 = make_float2(0.5f * dt, 0.5f * dt), d1 = make_float2(dt, dt);
        const float2 v = vel;
        float2 u1 = st.template first_stage<0>(o);
        st.to_mid();
        float2 a1 = __fmul2_rn(fsub2(u1, v), ist);
        float2 v2 = __ffma2_rn(d2, a1, v);
        float2 u2 = st.template at<1>(snap, n, ci, cj, __ffma2_rn(h2, v, o));
        float2 a2 = __fmul2_rn(fsub2(u2, v2), ist);
        float2 v3 = __ffma2_rn(d2, a2, v);
        float2 u3 = st.template at<1>(snap, n, ci, cj, __ffma2_rn(h2, v2, o));
        float2 a3 = __fmul2_rn(fsub2(u3, v3), ist);
        float2 v4 = __ffma2_rn(d1, a3, v);
        float2 u4 = st.template at<2>(snap, n, ci, cj, __ffma2_rn(h1, v3, o));
        float2 a4 = __fmul2_rn(fsub2(u4, v4), ist);
        const float h6 = h * (1.0f / 6.0f), d6 = dt * (1.0f / 6.0f);
        float2 sx = __fadd2_rn(__ffma2_rn(two, __fadd2_rn(v2, v3), v), v4);
        float2 sa = __fadd2_rn(__ffma2_rn(two, __fadd2_rn(a2, a3), a1), a4);
        np2 = __ffma2_rn(make_float2(h6, h6), sx, o);
        EL_STATE_ST(sd.vel[cur] + p, __ffma2_rn(make_float2(d6, d6), sa, v));
    }
    float ox, oy;
    int ni, nj, dix, diy;
    carry_axis(np2.x, ci, log2n, ox, ni, dix);
    carry_axis(np2.y, cj, log2n, oy, nj, diy);
    EL_STATE_ST(sd.cell[cur] + p, (uint32_t)ni | ((uint32_t)nj << 16));
    EL_STATE_ST(sd.off[cur] + p, make_float2(ox, oy));
    if (dix | diy) {  // crossed the periodic boundary: rare read-modify-write
        int2* imgp = sd.img[cur];
        int2 m = imgp[p];
        imgp[p] = make_int2(m.x + dix, m.y + diy);
    }
}

template <int SCHEME>
__device__ __forceinline__ void rk4_finish(const float4* __restrict__ snap, int n, int log2n, float dt,
                                           float h, const SpeciesDev& sd, ParticleRK4<SCHEME>& q) {
    rk4_update(snap, n, log2n, dt, h, sd, q.p, q.ci, q.cj, q.o, q.v, q.st);
}

// Tracers driven by the streamfunction (tracer_velocity = 1, Eq. 11): the
// streamfunction at (x +- dx, y) and (x, y +- dy), each interpolated in space
// and time, and centred differences; the neighbours sit one grid unit away,
// so they share the offsets.
template <int SCHEME>
__device__ __forceinline__ void rk4_psi_tracer(const float2* __restrict__ psi, int n, int log2n,
                                               float h, const SpeciesDev& sd, int p) {
    const int cur = sd.cur;
    const uint32_t c = EL_STATE_LD(sd.cell[cur] + p);
    const int ci = (int)(c & 0xffffu), cj = (int)(c >> 16);
    const float2 o = EL_STATE_LD(sd.off[cur] + p);
    const float2 h2 = make_float2(0.5f * h, 0.5f * h), h1 = make_float2(h, h);
    const float2 two = make_float2(2.0f, 2.0f);
    const float inv2d = (float)n * (float)(1.0 / (4.0 * 3.14159265358979323846));
    float2 k1 = psi_velocity<SCHEME, 0>(psi, n, ci, cj, o, inv2d);
    float2 k2 = psi_velocity<SCHEME, 1>(psi, n, ci, cj, __ffma2_rn(h2, k1, o), inv2d);
    float2 k3 = psi_velocity<SCHEME, 1>(psi, n, ci, cj, __ffma2_rn(h2, k2, o), inv2d);
    float2 k4 = psi_velocity<SCHEME, 2>(psi, n, ci, cj, __ffma2_rn(h1, k3, o), inv2d);
    float2 sum = __fadd2_rn(__ffma2_rn(two, __fadd2_rn(k2, k3), k1), k4);
    const float h6 = h * (1.0f / 6.0f);
    const float2 np2 = __ffma2_rn(make_float2(h6, h6), sum, o);
    float ox, oy;
    int ni, nj, dix, diy;
    carry_axis(np2.x, ci, log2n, ox, ni, dix);
    carry_axis(np2.y, cj, log2n, oy, nj, diy);
    EL_STATE_ST(sd.cell[cur] + p, (uint32_t)ni | ((uint32_t)nj << 16));
    EL_STATE_ST(sd.off[cur] + p, make_float2(ox, oy));
    if (dix | diy) {
        int2* imgp = sd.img[cur];
        int2 m = imgp[p];
        imgp[p] = make_int2(m.x + dix, m.y + diy);
    }
}

// One RK4 step of particle p of species sd for the cubic schemes, with the
// warp's stencils shared through shared memory (PatchStencil).  Every lane of
// the warp calls this; lanes with active = false (past the species' end) only
// help load the patch.  `region`: the warp's 3 * kPatchCap float2 of shared
// memory.
template <int SCHEME>
__device__ __forceinline__ void rk4_particle_coop(const float4* __restrict__ snap, int n, int log2n,
                                                  float dt, float h, const SpeciesDev& sd, int p,
                                                  bool active, float2* __restrict__ region) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (act == 0) return;  // the same on every lane
    int ci = 0, cj = 0;
    float2 o = make_float2(0.f, 0.f), v = o;
    if (active) {
        const int cur = sd.cur;
        const uint32_t c = EL_STATE_LD(sd.cell[cur] + p);
        ci = (int)(c & 0xffffu);
        cj = (int)(c >> 16);
        o = EL_STATE_LD(sd.off[cur] + p);
        if (sd.inertial) v = EL_STATE_LD(sd.vel[cur] + p);
    }
    PatchStencil<SCHEME> st;
    patch_setup(st, region, snap, n, ci, cj, active, act);
    if (active) rk4_update(snap, n, log2n, dt, h, sd, p, ci, cj, o, v, st);
}

// One RK4 step of particle p of species sd between levels n and n+1 (the
// streamfunction path for tracers when PSI).
template <int SCHEME, bool PSI>
__device__ __forceinline__ void rk4_particle(const float4* __restrict__ snap,
                                             const float2* __restrict__ psi, int n, int log2n,
                                             float dt, float h, const SpeciesDev& sd, int p,
                                             const KinArgs* kin = nullptr) {
    if (PSI && !sd.inertial) {
        rk4_psi_tracer<SCHEME>(psi, n, log2n, h, sd, p);
        return;
    }
    ParticleRK4<SCHEME> q;
    rk4_load_state(sd, p, q);
    q.st.bind(kin);  // the prescribed field of EL_ANALYTIC; unused by the grid schemes
    q.st.load(snap, n, q.ci, q.cj);
    rk4_finish(snap, n, log2n, dt, h, sd, q);
}

// Bulk prefetch into L2 of the state of the block `ahead` particles later in
// the same species (its cell, offset and velocity rows), issued by thread 0.
// The state stream is latency-bound: a block that waits on its own loads and
// then on its L2 gathers keeps few HBM requests in flight, so the block about
// one resident wave earlier asks for them.  Only whole 16-byte units inside
// [q0, np) are prefetched (start aligned: q0 is a multiple of the block size,
// the arrays 256-byte aligned); a prefetch changes no data and waits for
// nothing.
__device__ __forceinline__ void prefetch_state(const SpeciesDev& sd, int first, int ahead) {
    const int q0 = first + ahead;
    if (threadIdx.x != 0 || ahead <= 0 || q0 >= sd.np) return;
    const unsigned cnt = (unsigned)min((int)blockDim.x, sd.np - q0);
    const unsigned b4 = (cnt * 4u) & ~15u, b8 = (cnt * 8u) & ~15u;
    const int cur = sd.cur;
    if (b4) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sd.cell[cur] + q0), "r"(b4) : "memory");
    if (b8) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sd.off[cur] + q0), "r"(b8) : "memory");
    if (b8 && sd.inertial)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(sd.vel[cur] + q0), "r"(b8) : "memory");
}

}  // namespace el
