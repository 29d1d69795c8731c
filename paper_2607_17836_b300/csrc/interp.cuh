// Device-side spatial + temporal interpolation of the fluid velocity
// (Sec. 3.4, Eqs. 15-24), shared by the particle step and the sampling hook.
//
// The field is a level pair: per node a float4 (u_n, v_n, u_n+1, v_n+1)
// holding two consecutive time levels, so one 16-byte load fetches both.  A
// node's value at a stage is wa * (u_n, v_n) + wb * (u_n+1, v_n+1) (Eq. 23).
// Blending the nodes before the spatial weights is the same linear map as
// Eq. 23 applied to the two spatially interpolated values.
#pragma once

#include <cuda_runtime.h>

namespace el {

// Catmull-Rom weights (Eq. 19), nodes i-1, i, i+1, i+2.
__device__ __forceinline__ void weights_catmull_rom(float s, float w[4]) {
    w[0] = s * fmaf(s, fmaf(-0.5f, s, 1.0f), -0.5f);
    w[1] = fmaf(s * s, fmaf(1.5f, s, -2.5f), 1.0f);
    w[2] = s * fmaf(s, fmaf(-1.5f, s, 2.0f), 0.5f);
    w[3] = s * s * fmaf(0.5f, s, -0.5f);
}

// Cubic B-spline weights (Eq. 22), nodes i-1, i, i+1, i+2.
__device__ __forceinline__ void weights_bspline(float s, float w[4]) {
    float r = 1.0f - s;
    w[0] = r * r * r * (1.0f / 6.0f);
    w[1] = fmaf(s * s, fmaf(0.5f, s, -1.0f), 2.0f / 3.0f);
    w[2] = fmaf(s, fmaf(s, fmaf(-0.5f, s, 0.5f), 0.5f), 1.0f / 6.0f);
    w[3] = s * s * s * (1.0f / 6.0f);
}

__device__ __forceinline__ float4 node_ld(const float4* __restrict__ snap, int idx) {
    return __ldg(snap + idx);
}

// Velocity at grid-unit position (ci + lx, cj + ly), lx, ly any small reals:
// the containing cell is (ci + floor(lx), cj + floor(ly)) wrapped
// periodically (n a power of two), the offsets lx - floor(lx), ly - floor(ly).
// SCHEME: 0 bilinear (Eq. 16), 1 Catmull-Rom (Eq. 18), 2 B-spline (Eq. 21).
template <int SCHEME>
__device__ __forceinline__ float2 fluid_at(const float4* __restrict__ snap, int n, int ci, int cj,
                                           float lx, float ly, float wa, float wb) {
    const int m = n - 1;
    float flx = floorf(lx), fly = floorf(ly);
    int i = ci + (int)flx, j = cj + (int)fly;
    float sx = lx - flx, sy = ly - fly;
    if (SCHEME == 0) {
        int i0 = i & m, i1 = (i + 1) & m;
        int r0 = (j & m) * n, r1 = ((j + 1) & m) * n;
        float4 a = node_ld(snap, r0 + i0), b = node_ld(snap, r0 + i1);
        float4 c = node_ld(snap, r1 + i0), d = node_ld(snap, r1 + i1);
        float au = fmaf(wa, a.x, wb * a.z), av = fmaf(wa, a.y, wb * a.w);
        float bu = fmaf(wa, b.x, wb * b.z), bv = fmaf(wa, b.y, wb * b.w);
        float cu = fmaf(wa, c.x, wb * c.z), cv = fmaf(wa, c.y, wb * c.w);
        float du = fmaf(wa, d.x, wb * d.z), dv = fmaf(wa, d.y, wb * d.w);
        // Eq. 16 as two lerps per axis
        float lo_u = fmaf(sx, bu - au, au), hi_u = fmaf(sx, du - cu, cu);
        float lo_v = fmaf(sx, bv - av, av), hi_v = fmaf(sx, dv - cv, cv);
        return make_float2(fmaf(sy, hi_u - lo_u, lo_u), fmaf(sy, hi_v - lo_v, lo_v));
    } else {
        float wx[4], wy[4];
        if (SCHEME == 1) {
            weights_catmull_rom(sx, wx);
            weights_catmull_rom(sy, wy);
        } else {
            weights_bspline(sx, wx);
            weights_bspline(sy, wy);
        }
        int ii[4];
#pragma unroll
        for (int a = 0; a < 4; a++) ii[a] = (i + a - 1) & m;
        float u = 0.f, v = 0.f;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            int row = ((j + b - 1) & m) * n;
            float ru = 0.f, rv = 0.f;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                float4 t = node_ld(snap, row + ii[a]);
                ru = fmaf(wx[a], fmaf(wa, t.x, wb * t.z), ru);
                rv = fmaf(wx[a], fmaf(wa, t.y, wb * t.w), rv);
            }
            u = fmaf(wy[b], ru, u);
            v = fmaf(wy[b], rv, v);
        }
        return make_float2(u, v);
    }
}

// a - b on float pairs: one paired subtraction, rounded to nearest per lane
// (no constant pair (-1, -1) to keep in registers, as b * -1 + a would need).
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 x, y, d;\n\t"
        "mov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "sub.rn.f32x2 d, x, y;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 pair(float x) { return make_float2(x, x); }

// Catmull-Rom (Eq. 19) weights for the x and y offsets at once:
// w[k] = (w_k(sx), w_k(sy)), nodes i-1, i, i+1, i+2.
__device__ __forceinline__ void catmull_rom_weights2(float2 s, float2 w[4]) {
    w[0] = __fmul2_rn(s, __ffma2_rn(s, __ffma2_rn(pair(-0.5f), s, pair(1.0f)), pair(-0.5f)));
    w[1] = __ffma2_rn(__fmul2_rn(s, s), __ffma2_rn(pair(1.5f), s, pair(-2.5f)), pair(1.0f));
    w[2] = __fmul2_rn(s, __ffma2_rn(s, __ffma2_rn(pair(-1.5f), s, pair(2.0f)), pair(0.5f)));
    w[3] = __fmul2_rn(__fmul2_rn(s, s), __ffma2_rn(pair(0.5f), s, pair(-0.5f)));
}

// Cubic B-spline (Eq. 22) weights of one offset s, nodes i-1, i, i+1, i+2.
__device__ __forceinline__ void bspline_weights1(float s, float w[4]) {
    const float r = 1.0f - s;
    w[0] = (r * r) * (r * (1.0f / 6.0f));
    w[1] = fmaf(s * s, fmaf(0.5f, s, -1.0f), 2.0f / 3.0f);
    w[2] = fmaf(s, fmaf(s, fmaf(-0.5f, s, 0.5f), 0.5f), 1.0f / 6.0f);
    w[3] = (s * s) * (s * (1.0f / 6.0f));
}

// The weights of both axes as the pairs the paired FMAs take:
// wx[a] = (w_a(sx), w_a(sx)), wy[b] = (w_b(sy), w_b(sy)); the particle
// kernels' register and shared gathers both use these (so the two give the
// same bits).  Measured at 16M particles, 1024^2, against the other form
// of each: Catmull-Rom formed by paired FMAs on (sx, sy) is 1 % faster than
// by scalars; the B-spline weights formed as scalars (constant operands as
// immediates) are 4 % faster than paired, and leave the B-spline kernels
// without register spills.
template <int SCHEME>
__device__ __forceinline__ void cubic_weight_pairs(float2 s, float2 wx[4], float2 wy[4]) {
    if (SCHEME == 1) {
        float2 w[4];
        catmull_rom_weights2(s, w);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            wx[k] = pair(w[k].x);
            wy[k] = pair(w[k].y);
        }
    } else {
        float ax[4], ay[4];
        bspline_weights1(s.x, ax);
        bspline_weights1(s.y, ay);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            wx[k] = pair(ax[k]);
            wy[k] = pair(ay[k]);
        }
    }
}

// The prescribed kinematic velocity of Sec. 5.2 at the three RK4 stage
// times (t_n, t_n + dt/2, t_n + dt): u = alpha sin(k x - sx) cos(k y - sy),
// v = -alpha cos(k x - sx) sin(k y - sy), with sx = k eps sin(omega t) and
// sy = k eps sin(omega t + phi) computed on the host in FP64.
struct KinArgs {
    float alpha;         // peak speed
    float dk;            // 2 pi / n: radians per grid unit at unit wavenumber
    float sx[3], sy[3];  // phase shifts at the stage times
    int kw;              // integer wavenumber k
    int mask;            // n - 1
};

// Register-resident copy of the W x W stencil nodes (both time levels) of
// one cell.  A particle moves a fraction of a cell per step, so its four RK4
// stages nearly always fall in the cell of the previous stage: the stencil is
// loaded once and re-used, and only a stage that crosses into another cell
// fetches again.  (ci, cj) are the cell's unwrapped indices; addresses wrap.
// THETA: 0 = level n, 1 = mid-way (theta = 1/2), 2 = level n+1 (Eq. 23).
template <int SCHEME>
struct Stencil {
    static constexpr int W = SCHEME == 0 ? 2 : 4;
    static constexpr int O = SCHEME == 0 ? 0 : -1;  // first node relative to the cell
    int ci, cj;
    float4 v[W * W];

    __device__ __forceinline__ void bind(const KinArgs*) {}

    __device__ __forceinline__ void load(const float4* __restrict__ snap, int n, int i, int j) {
        const int m = n - 1;
#pragma unroll
        for (int b = 0; b < W; b++) {
            int row = ((j + O + b) & m) * n;
#pragma unroll
            for (int a = 0; a < W; a++) v[b * W + a] = node_ld(snap, row + ((i + O + a) & m));
        }
        ci = i;
        cj = j;
    }

    // After the first stage, the (x, y) half of each node is replaced by the
    // SUM of the two levels, which both mid-way stages read (computed once,
    // the same values as forming it per stage); the (z, w) half, level n+1,
    // stays for the last stage.
    __device__ __forceinline__ void to_mid() {
#pragma unroll
        for (int k = 0; k < W * W; k++) {
            const float2 m = __fadd2_rn(make_float2(v[k].x, v[k].y), make_float2(v[k].z, v[k].w));
            v[k].x = m.x;
            v[k].y = m.y;
        }
    }

    // Node value at the stage time: THETA = 0 level n (before to_mid), 1 the
    // SUM of the two levels (after to_mid; the factor 1/2 is applied once to
    // the interpolated value), 2 level n+1.
    template <int THETA>
    __device__ __forceinline__ float2 node(int k) const {
        const float4& t = v[k];
        return THETA == 2 ? make_float2(t.z, t.w) : make_float2(t.x, t.y);
    }

    template <int THETA>
    __device__ __forceinline__ float2 eval(float2 s) const {
        float2 r;
        if (SCHEME == 0) {
            // Eq. 16 as two lerps in x and one in y
            const float2 a = node<THETA>(0), b = node<THETA>(1);
            const float2 c = node<THETA>(2), d = node<THETA>(3);
            const float2 sx = pair(s.x), sy = pair(s.y);
            const float2 lo = __ffma2_rn(sx, fsub2(b, a), a);
            const float2 hi = __ffma2_rn(sx, fsub2(d, c), c);
            r = __ffma2_rn(sy, fsub2(hi, lo), lo);
        } else {
            float2 wx[4], wy[4];
            cubic_weight_pairs<SCHEME>(s, wx, wy);
            r = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 4; b++) {
                float2 row = __fmul2_rn(wx[0], node<THETA>(b * 4));
#pragma unroll
                for (int a = 1; a < 4; a++) row = __ffma2_rn(wx[a], node<THETA>(b * 4 + a), row);
                r = __ffma2_rn(wy[b], row, r);
            }
        }
        if (THETA == 1) r = __fmul2_rn(r, pair(0.5f));
        return r;
    }

    // Stage 1: the particle's own cell, offsets o in [0, 1).
    template <int THETA>
    __device__ __forceinline__ float2 first_stage(float2 o) const {
        return eval<THETA>(o);
    }

    // Fluid velocity at grid-unit position (ci0 + l.x, cj0 + l.y), stages in
    // RK4 order (first_stage, to_mid, THETA 1, 1, 2).  For the
    // bilinear scheme the common case, a stage inside the cached cell
    // (ci0, cj0), skips the floor: there floor(l) = 0 and l - 0 = l exactly
    // (measured 5 % faster for bilinear, 5 % slower for the cubic schemes,
    // whose register budget it upsets).
    template <int THETA>
    __device__ __forceinline__ float2 at(const float4* __restrict__ snap, int n, int ci0, int cj0,
                                         float2 l) {
        float2 s = l;
        // 0 <= l < 1 on both axes as one unsigned compare of the bit
        // patterns: non-negative floats order like their bits, below 1.0f's,
        // and any sign bit (or NaN) makes the pattern larger
        const bool home = SCHEME == 0 && ci == ci0 && cj == cj0 &&
                          max(__float_as_uint(l.x), __float_as_uint(l.y)) < 0x3f800000u;
        if (!home) {
            const float flx = floorf(l.x), fly = floorf(l.y);
            const int i = ci0 + (int)flx, j = cj0 + (int)fly;
            if (i != ci || j != cj) {
                load(snap, n, i, j);
                if (THETA == 1) to_mid();
            }
            s = fsub2(l, make_float2(flx, fly));
        }
        return eval<THETA>(s);
    }
};

// Warp-shared stencils of the cubic schemes (Eqs. 18-22).  After re-binning
// the 32 particles of a warp sit in a few neighbouring cells, so their 4 x 4
// stencils overlap: the warp loads the union of them once (one node per lane
// per pass) into its own region of shared memory, and every stage of every
// lane reads its 16 nodes from there.  Nothing is held in registers between
// stages, which leaves room for more resident warps than a per-thread register
// copy of the 16 level pairs (64 registers) would.
//
// The patch covers the warp's cells plus one cell on every side, so a stage
// that moves one cell away (the common crossing) still finds its stencil; a
// stage further away, or a warp whose cells spread over more than kPatchCap
// nodes, gathers from the level pair in global memory instead.  Each node is
// stored three times, as the value each stage time reads: level n (stage 1),
// the SUM of the two levels (stages 2 and 3, times 1/2 after the sum over the
// stencil) and level n+1 (stage 4); the values and the order of the
// arithmetic are the register cache's, so both give the same bits.
constexpr int kPatchCap = 192;  // nodes of one warp's patch

template <int SCHEME>
struct PatchStencil {
    const float2* lv;    // the warp's patch: [0, cap) level n, [cap, 2 cap) sum, [2 cap, 3 cap) level n+1
    int w;               // patch width (nodes per row)
    int base;            // patch index of the first node of the particle's own cell's stencil
    bool patch;          // the patch holds the warp's stencils
    const float4* snap;  // the level pair (for stencils outside the patch)
    int n, ci, cj;       // grid size, the particle's cell

    __device__ __forceinline__ void to_mid() {}

    template <int THETA>
    __device__ __forceinline__ float2 first_stage(float2 o) const {
        return eval<THETA>(0, 0, o);
    }

    template <int THETA>
    __device__ __forceinline__ float2 at(const float4* __restrict__, int, int, int, float2 l) const {
        const float flx = floorf(l.x), fly = floorf(l.y);
        return eval<THETA>((int)flx, (int)fly, fsub2(l, make_float2(flx, fly)));
    }

    // Value of the node at THETA (0: level n, 1: the level sum, 2: level n+1)
    // from its level pair.
    template <int THETA>
    __device__ __forceinline__ static float2 pick(float4 t) {
        return THETA == 0 ? make_float2(t.x, t.y)
                          : (THETA == 2 ? make_float2(t.z, t.w)
                                        : __fadd2_rn(make_float2(t.x, t.y), make_float2(t.z, t.w)));
    }

    // The stencil of cell (ci + fi, cj + fj) at offsets s, THETA as in Stencil::eval.
    template <int THETA>
    __device__ __forceinline__ float2 eval(int fi, int fj, float2 s) const {
        float2 wx[4], wy[4];
        cubic_weight_pairs<SCHEME>(s, wx, wy);
        float2 r = make_float2(0.f, 0.f);
        if (patch && (unsigned)(fi + 1) <= 2u && (unsigned)(fj + 1) <= 2u) {
            const float2* q = lv + THETA * kPatchCap + base + fj * w + fi;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const float2* qr = q + b * w;
                float2 row = __fmul2_rn(wx[0], qr[0]);
#pragma unroll
                for (int a = 1; a < 4; a++) row = __ffma2_rn(wx[a], qr[a], row);
                r = __ffma2_rn(wy[b], row, r);
            }
        } else {
            const int m = n - 1;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const float4* rp = snap + ((cj + fj - 1 + b) & m) * n;
                float2 row = __fmul2_rn(wx[0], pick<THETA>(node_ld(rp, (ci + fi - 1) & m)));
#pragma unroll
                for (int a = 1; a < 4; a++)
                    row = __ffma2_rn(wx[a], pick<THETA>(node_ld(rp, (ci + fi - 1 + a) & m)), row);
                r = __ffma2_rn(wy[b], row, r);
            }
        }
        if (THETA == 1) r = __fmul2_rn(r, pair(0.5f));
        return r;
    }
};

// Set up the warp's patch: every lane of the warp calls this (inactive lanes
// too, with active = false); at least one lane is active.  The cells are
// taken relative to the first active lane's, as signed distances modulo n
// (any representative works: node indices wrap), and the patch spans the
// warp's cells plus one cell each side, plus the stencil's reach (one node
// before the cell, two after).  `region` is the warp's 3 * kPatchCap float2
// of shared memory; the previous contents may still be read by lanes of an
// earlier particle, so the warp synchronises before overwriting them.
template <int SCHEME>
__device__ __forceinline__ void patch_setup(PatchStencil<SCHEME>& st, float2* __restrict__ region,
                                            const float4* __restrict__ snap, int n, int ci, int cj,
                                            bool active, unsigned act) {
    const unsigned full = 0xffffffffu;
    const int src = __ffs(act) - 1;
    const int ri = __shfl_sync(full, ci, src), rj = __shfl_sync(full, cj, src);
    const int m = n - 1, half = n >> 1;
    const int di = active ? ((ci - ri + half) & m) - half : 0;
    const int dj = active ? ((cj - rj + half) & m) - half : 0;
    const int imin = __reduce_min_sync(full, di), imax = __reduce_max_sync(full, di);
    const int jmin = __reduce_min_sync(full, dj), jmax = __reduce_max_sync(full, dj);
    const int w = imax - imin + 6, h = jmax - jmin + 6;
    st.lv = region;
    st.w = w;
    st.base = (dj - jmin + 1) * w + (di - imin + 1);
    st.patch = w * h <= kPatchCap;  // the same on every lane
    st.snap = snap;
    st.n = n;
    st.ci = ci;
    st.cj = cj;
    __syncwarp();
    if (st.patch) {
        const int oi = ri + imin - 2, oj = rj + jmin - 2;
        // row of patch index k: floor((k + 1/2) / w), exact in FP32 here
        // (k < kPatchCap, so the quotient is >= 1/(2 kPatchCap) from an integer)
        const float inv_w = 1.0f / (float)w;
        for (int k = (int)(threadIdx.x & 31); k < w * h; k += 32) {
            const int r = (int)(((float)k + 0.5f) * inv_w);
            const int c = k - r * w;
            const float4 t = node_ld(snap, ((oj + r) & m) * n + ((oi + c) & m));
            region[k] = make_float2(t.x, t.y);
            region[kPatchCap + k] = __fadd2_rn(make_float2(t.x, t.y), make_float2(t.z, t.w));
            region[2 * kPatchCap + k] = make_float2(t.z, t.w);
        }
        __syncwarp();
    }
}

// EL_ANALYTIC: the kinematic field itself at the particle (no grid, no
// stencil); THETA selects the stage time.  The integer part of k x in grid
// units is reduced modulo n exactly before the phase is formed.
template <>
struct Stencil<3> {
    const KinArgs* kin;
    int ci, cj;

    __device__ __forceinline__ void bind(const KinArgs* k) { kin = k; }
    __device__ __forceinline__ void to_mid() {}
    __device__ __forceinline__ void load(const float4*, int, int i, int j) {
        ci = i;
        cj = j;
    }
    template <int THETA>
    __device__ __forceinline__ float2 value(int i, int j, float2 l) const {
        const float fx = (float)((kin->kw * i) & kin->mask) + (float)kin->kw * l.x;
        const float fy = (float)((kin->kw * j) & kin->mask) + (float)kin->kw * l.y;
        float snx, csx, sny, csy;
        sincosf(fmaf(kin->dk, fx, -kin->sx[THETA]), &snx, &csx);
        sincosf(fmaf(kin->dk, fy, -kin->sy[THETA]), &sny, &csy);
        return make_float2(kin->alpha * snx * csy, -kin->alpha * csx * sny);
    }
    template <int THETA>
    __device__ __forceinline__ float2 first_stage(float2 o) const {
        return value<THETA>(ci, cj, o);
    }
    template <int THETA>
    __device__ __forceinline__ float2 at(const float4*, int, int ci0, int cj0, float2 l) {
        return value<THETA>(ci0, cj0, l);
    }
};

// Scalar field (the streamfunction) stored as level pairs (f_n, f_n+1) per
// node: its value in cell (i, j) (unwrapped) at offsets (sx, sy), at the
// stage time THETA (0: level n, 1: mid-way, 2: level n+1).
template <int SCHEME, int THETA>
__device__ __forceinline__ float scalar_at(const float2* __restrict__ f, int n, int i, int j,
                                           float sx, float sy) {
    const int m = n - 1;
    auto lv = [&](int idx) {
        const float2 t = __ldg(f + idx);
        return THETA == 0 ? t.x : (THETA == 2 ? t.y : 0.5f * (t.x + t.y));
    };
    if (SCHEME == 0) {
        const int i0 = i & m, i1 = (i + 1) & m, r0 = (j & m) * n, r1 = ((j + 1) & m) * n;
        const float a = lv(r0 + i0), b = lv(r0 + i1), c = lv(r1 + i0), d = lv(r1 + i1);
        const float lo = fmaf(sx, b - a, a), hi = fmaf(sx, d - c, c);
        return fmaf(sy, hi - lo, lo);
    } else {
        float wx[4], wy[4];
        if (SCHEME == 1) {
            weights_catmull_rom(sx, wx);
            weights_catmull_rom(sy, wy);
        } else {
            weights_bspline(sx, wx);
            weights_bspline(sy, wy);
        }
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int row = ((j + b - 1) & m) * n;
            float r = 0.f;
#pragma unroll
            for (int a = 0; a < 4; a++) r = fmaf(wx[a], lv(row + ((i + a - 1) & m)), r);
            acc = fmaf(wy[b], r, acc);
        }
        return acc;
    }
}

// Tracer velocity from the streamfunction (Eq. 11) at grid-unit position
// (ci + l.x, cj + l.y): u = (psi(x, y+dy) - psi(x, y-dy)) / 2dy,
// v = -(psi(x+dx, y) - psi(x-dx, y)) / 2dx, inv2d = 1 / (2 dx).
template <int SCHEME, int THETA>
__device__ __forceinline__ float2 psi_velocity(const float2* __restrict__ psi, int n, int ci, int cj,
                                               float2 l, float inv2d) {
    const float flx = floorf(l.x), fly = floorf(l.y);
    const int i = ci + (int)flx, j = cj + (int)fly;
    const float sx = l.x - flx, sy = l.y - fly;
    const float pe = scalar_at<SCHEME, THETA>(psi, n, i + 1, j, sx, sy);
    const float pw = scalar_at<SCHEME, THETA>(psi, n, i - 1, j, sx, sy);
    const float pn = scalar_at<SCHEME, THETA>(psi, n, i, j + 1, sx, sy);
    const float ps = scalar_at<SCHEME, THETA>(psi, n, i, j - 1, sx, sy);
    return make_float2((pn - ps) * inv2d, (pw - pe) * inv2d);
}

}  // namespace el
