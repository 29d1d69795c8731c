// Per-element bodies of the step kernels, shared by the single-flow kernels
// (fluid.cu, particles.cu) and the batched kernels (batch.cu), so that a
// simulation advanced alone or inside a batch does the same arithmetic.
#pragma once

#include "common.cuh"
#include "interp.cuh"

#ifndef EL_STREAMING_STATE
#define EL_STREAMING_STATE 1
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
    cell = c2 - (dimg << log2n);
    off = o;
}

// One RK4 step of particle p of species sd (Eq. 12 tracers, Eq. 14 inertial)
// between levels n and n+1, read from their level pair `snap`: stage 1
// (theta = 0) and stage 4 (theta = 1) read one half of each node without
// blending.  All (x, y) and (u, v) arithmetic is on float pairs (one paired
// FP32 instruction per two lanes of work).  h = dt * n / (2 pi): grid units
// per unit velocity.
template <int SCHEME, bool PSI>
__device__ __forceinline__ void rk4_particle(const float4* __restrict__ snap,
                                             const float2* __restrict__ psi, int n, int log2n,
                                             float dt, float h, const SpeciesDev& sd, int p) {
    const int cur = sd.cur;
    uint32_t* __restrict__ cellp = sd.cell[cur];
    float2* __restrict__ offp = sd.off[cur];
    // the particle state is streamed once per step: evict-first loads and
    // stores keep the caches for the level pair the gathers re-read
    const uint32_t c = EL_STATE_LD(cellp + p);
    const int ci = (int)(c & 0xffffu), cj = (int)(c >> 16);
    const float2 o = EL_STATE_LD(offp + p);
    Stencil<SCHEME> st;
    st.load(snap, n, ci, cj);
    const float2 h2 = make_float2(0.5f * h, 0.5f * h), h1 = make_float2(h, h);
    const float2 two = make_float2(2.0f, 2.0f);
    float2 np2;
    float2 vnew = make_float2(0.f, 0.f);
    const bool inertial = sd.inertial;
    if (PSI && !inertial) {
        // Eq. 11: the streamfunction at (x +- dx, y) and (x, y +- dy), each
        // interpolated in space and time, and centred differences; the
        // neighbours sit one grid unit away, so they share the offsets.
        const float inv2d = (float)n * (float)(1.0 / (4.0 * 3.14159265358979323846));
        float2 k1 = psi_velocity<SCHEME, 0>(psi, n, ci, cj, o, inv2d);
        float2 k2 = psi_velocity<SCHEME, 1>(psi, n, ci, cj, __ffma2_rn(h2, k1, o), inv2d);
        float2 k3 = psi_velocity<SCHEME, 1>(psi, n, ci, cj, __ffma2_rn(h2, k2, o), inv2d);
        float2 k4 = psi_velocity<SCHEME, 2>(psi, n, ci, cj, __ffma2_rn(h1, k3, o), inv2d);
        float2 sum = __fadd2_rn(__ffma2_rn(two, __fadd2_rn(k2, k3), k1), k4);
        const float h6 = h * (1.0f / 6.0f);
        np2 = __ffma2_rn(make_float2(h6, h6), sum, o);
    } else if (!inertial) {
        // Eq. 12, stages at t, t + dt/2, t + dt/2, t + dt (theta = 0, 1/2, 1/2, 1)
        float2 k1 = st.template first_stage<0>(o);
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
        float2* __restrict__ velp = sd.vel[cur];
        const float2 v = EL_STATE_LD(velp + p);
        float2 u1 = st.template first_stage<0>(o);
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
        vnew = __ffma2_rn(make_float2(d6, d6), sa, v);
        EL_STATE_ST(velp + p, vnew);
    }
    float ox, oy;
    int ni, nj, dix, diy;
    carry_axis(np2.x, ci, log2n, ox, ni, dix);
    carry_axis(np2.y, cj, log2n, oy, nj, diy);
    EL_STATE_ST(cellp + p, (uint32_t)ni | ((uint32_t)nj << 16));
    EL_STATE_ST(offp + p, make_float2(ox, oy));
    if (dix | diy) {  // crossed the periodic boundary: rare read-modify-write
        int2* imgp = sd.img[cur];
        int2 m = imgp[p];
        imgp[p] = make_int2(m.x + dix, m.y + diy);
    }
}

}  // namespace el
