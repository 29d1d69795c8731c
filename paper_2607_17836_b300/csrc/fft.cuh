// The pseudospectral fluid step (Sec. 3.1) as two fused passes, each a batch
// of 1-D FFTs done in shared memory:
//
//   column pass, per tile of tc half-spectrum columns kx < n/2:
//     forward FFT along y of the x-transformed nonlinear term  -> N-hat (Eq. 8)
//     2/3 rule + AB2 update of omega-hat (Eqs. 9, 10)
//     for every plane (u-hat, v-hat, i kx omega-hat, i ky omega-hat, spline
//     coefficients, streamfunction; Eqs. 4-6): its spectrum from the new
//     omega-hat, inverse FFT along y, stored in row space [p][y][kx]
//   row pass, per grid row y:
//     inverse real FFT along x of every plane -> u, v, d(omega)/dx, ... on the row
//     N = u d(omega)/dx + v d(omega)/dy (Eq. 7) and the level pair the
//     particle step reads
//     forward real FFT along x of N, stored for the next column pass
//
// The Nyquist column kx = n/2 is outside the 2/3 rule, so omega-hat, N-hat
// and every plane are identically zero there: the column pass skips it and
// the planes keep the zeros written at creation.
//
// Each 1-D transform is a self-sorting (Stockham) mixed-radix FFT: passes of
// radix 16 while at least four bits of the length remain, then one pass of
// radix 2, 4 or 8.  A pass reads R elements j + r L/R of a sequence, scales
// element r by W_{Ns R}^{(j mod Ns) r}, takes an R-point DFT in registers and
// writes it to (j div Ns) Ns R + (j mod Ns) + r Ns, where Ns is the product
// of the earlier radices (the formulation of Govindaraju et al., SC 2008).
// Passes run in place: every thread holds the 16 values of its group(s) in
// registers across a barrier.  The R-point DFTs are radix-2
// decimation-in-frequency networks with the output permutation resolved at
// compile time.  Shared-memory index i is stored at i + i/16, which keeps the
// stride-16 writes of the first pass free of bank conflicts.  Both directions
// are unnormalised; the 1/n^2 of the inverse is folded into the plane spectra.
// A real transform of length n runs as a complex one of length n/2 on
// (x_2m + i x_2m+1) with the even/odd split of its spectrum.
// Twiddle tables are computed on the host in FP64 (fft_twiddles).
#pragma once

#include "stages.cuh"

#include <vector>

namespace el {

// ---- radix schedule and twiddle tables --------------------------------------

struct FftSchedule {
    int npass;
    int log2r[12];
};

__host__ __device__ __forceinline__ FftSchedule fft_schedule(int log2l) {
    FftSchedule s{};
    int l = log2l;
    while (l >= 4) {
        s.log2r[s.npass++] = 4;
        l -= 4;
    }
    if (l > 0) s.log2r[s.npass++] = l;
    return s;
}

// Table of a length-2^log2l transform: for every pass p >= 1 (Ns = product of
// the earlier radices, R its own), entries (r - 1) Ns + q = exp(-2 pi i q r /
// (Ns R)), r = 1..R-1, q = 0..Ns-1, one pass after the other.  L - R_0 entries.
void fft_twiddles(int log2l, std::vector<float2>& out);

// ---- complex helpers -------------------------------------------------------

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// Twiddle load through the read-only path.  The asm is volatile so that the
// compiler does not hoist the loads of every pass out of an enclosing loop
// and keep them all live in registers.
__device__ __forceinline__ float2 ld_twiddle(const float2* p) {
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// Padded length of one sequence of 2^log2l elements in shared memory (+4
// staggers the sequences of a tile across banks).
__host__ __device__ __forceinline__ int fft_seq_stride(int log2l) {
    const int l = 1 << log2l;
    return l + (l >> 4) + 4;
}

// exp(-2 pi i m / 16), m = 0..7 (m a compile-time constant after unrolling).
__device__ __forceinline__ float2 w16(int m) {
    constexpr float c1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float s1 = 0.38268343236508977173f;  // sin(pi/8)
    constexpr float h = 0.70710678118654752440f;   // cos(pi/4)
    switch (m) {
        case 1: return make_float2(c1, -s1);
        case 2: return make_float2(h, -h);
        case 3: return make_float2(s1, -c1);
        case 5: return make_float2(-s1, -c1);
        case 6: return make_float2(-h, -h);
        case 7: return make_float2(-c1, -s1);
        default: return make_float2(1.f, 0.f);
    }
}

__host__ __device__ constexpr int bitrev_c(int k, int bits) {
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((k >> b) & 1) << (bits - 1 - b);
    return r;
}

// In-register R-point DFT (R = 2, 4, 8, 16), natural order in and out;
// DIR = -1 forward, +1 inverse (unnormalised).
template <int LOG2R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
    constexpr int R = 1 << LOG2R;
#pragma unroll
    for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * span) {
#pragma unroll
            for (int k = 0; k < span; k++) {
                const float2 a = v[b + k], c = v[b + k + span];
                v[b + k] = cadd(a, c);
                const float2 d = csub(a, c);
                const int m = k * (8 / span);  // W_{2 span}^k = W_16^m
                if (m == 0) {
                    v[b + k + span] = d;
                } else if (m == 4) {           // times -i (forward) or +i (inverse)
                    v[b + k + span] = DIR < 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
                } else {
                    const float2 w = w16(m);
                    v[b + k + span] = cmul(d, DIR < 0 ? w : conjf2(w));
                }
            }
        }
    }
    float2 t[R];
#pragma unroll
    for (int k = 0; k < R; k++) t[k] = v[bitrev_c(k, LOG2R)];
#pragma unroll
    for (int k = 0; k < R; k++) v[k] = t[k];
}

// One in-place Stockham pass of radix 2^LOG2R over nseq sequences of length
// 2^log2l at buf + s * sstride.  Needs blockDim.x * 16 >= nseq * 2^log2l.
// Called by every thread of the block; ends with a barrier.
template <int LOG2R, int DIR>
__device__ __forceinline__ void fft_pass(float2* __restrict__ buf, int log2l, int log2ns, int nseq,
                                         int sstride, const float2* __restrict__ tw) {
    constexpr int R = 1 << LOG2R, G = 16 / R;
    // The scalars pass through an empty asm so that the compiler cannot
    // treat anything of this pass as invariant in an enclosing loop: hoisting
    // it would keep the indices of every pass of every transform live at once.
    int tid = threadIdx.x, bd = blockDim.x;
    asm volatile("" : "+r"(tid), "+r"(bd), "+r"(log2l), "+r"(log2ns), "+r"(nseq), "+r"(sstride));
    const int log2g = log2l - LOG2R;  // groups per sequence: L / R
    const int total = nseq << log2g;
    const int gmask = (1 << log2g) - 1, nsmask = (1 << log2ns) - 1;
    float2 v[G][R];
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int t = tid + g * bd;
        if (t < total) {
            const float2* b = buf + (t >> log2g) * sstride;
            const int j = t & gmask;
#pragma unroll
            for (int r = 0; r < R; r++) v[g][r] = b[pidx(j + (r << log2g))];
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int t = tid + g * bd;
        if (t < total) {
            const int j = t & gmask, q = j & nsmask;
            if (log2ns > 0) {
#pragma unroll
                for (int r = 1; r < R; r++) {
                    const float2 w = ld_twiddle(tw + ((r - 1) << log2ns) + q);
                    v[g][r] = cmul(v[g][r], DIR < 0 ? w : conjf2(w));
                }
            }
            dft<LOG2R, DIR>(v[g]);
            float2* b = buf + (t >> log2g) * sstride;
            const int d = ((j >> log2ns) << (log2ns + LOG2R)) + q;
#pragma unroll
            for (int r = 0; r < R; r++) b[pidx(d + (r << log2ns))] = v[g][r];
        }
    }
    __syncthreads();
}

// Full transform of nseq sequences of length 2^log2l (natural order in and
// out): floor(log2l / 4) passes of radix 16, then one of radix 2^REM, REM =
// log2l mod 4 (a template argument: a runtime choice among the remainder
// passes makes the compiler keep the registers of all of them at once).
template <int DIR, int REM>
__device__ __forceinline__ void fft_smem(float2* buf, int log2l, int nseq, int sstride,
                                         const float2* __restrict__ tw) {
    int log2ns = 0, off = 0;
    const int n16 = log2l >> 2;
#pragma unroll 1
    for (int p = 0; p < n16; p++) {
        fft_pass<4, DIR>(buf, log2l, log2ns, nseq, sstride, tw + off);
        if (p > 0) off += 15 << log2ns;
        log2ns += 4;
    }
    if (REM > 0) fft_pass<(REM > 0 ? REM : 1), DIR>(buf, log2l, log2ns, nseq, sstride, tw + off);
}

// ---- the two passes ------------------------------------------------------------

// Everything the column pass of one flow reads and writes.
struct ColArgs {
    float2* what;            // omega-hat, high part, column-major [kx][j] (n per column)
    float2* what_lo;         // low part (compensated storage)
    float2* hist;            // AB2 history
    const float2* nrow;      // N transformed along x, [y][pitch]
    float2* planes;          // output planes in row space, [p][y][pitch]
    const float2* ex;        // exp(-nu kx^2 dt) as (hi, lo)
    const float2* ey;        // exp(-nu ky^2 dt) as (hi, lo), row index j
    const float* pre_x;      // spline prefilter 3 / (2 + cos k dx)
    const float* pre_y;
    const float2* tw;        // fft_twiddles(log2n)
    size_t pstride;          // n * pitch
    int n, log2n, pitch, nplanes, log2tc;
    int mode;
    int spline, psi_plane;
    float scale, dt, nu;
};

// Spectrum of plane p at mode (kx, j) from w (omega-hat already scaled by
// 1/n^2): 0 u-hat = i ky psi-hat, 1 v-hat = -i kx psi-hat (Eqs. 5, 6; psi-hat
// = w / k^2, psi-hat(0) = 0), 2 i kx w, 3 i ky w (Eq. 4), 4/5 the interpolating
// cubic-spline coefficients of u/v (if spline), psi_plane the streamfunction
// stencil field.  The Nyquist row j = n/2 takes no derivative.  The spline
// condition (c_{i-1} + 4 c_i + c_{i+1}) / 6 = f_i is diagonal in Fourier
// space, factor (2 + cos k dx) / 3 per axis.
__device__ __forceinline__ float2 plane_value(const ColArgs& a, int p, float2 w, int kx, int j) {
    const int n = a.n, ky = wavenumber_row(j, n);
    const float fkx = (float)kx;
    const float fky = (j == n / 2) ? 0.f : (float)ky;
    const float k2 = (float)(kx * kx + ky * ky);
    const float ik2 = k2 > 0.f ? 1.f / k2 : 0.f;
    const float2 psi = make_float2(w.x * ik2, w.y * ik2);
    const float pf = a.spline ? a.pre_x[kx] * a.pre_y[j] : 1.0f;
    if (p == a.psi_plane) return make_float2(psi.x * pf, psi.y * pf);
    switch (p) {
        case 0: return make_float2(-fky * psi.y, fky * psi.x);
        case 1: return make_float2(fkx * psi.y, -fkx * psi.x);
        case 2: return make_float2(-fkx * w.y, fkx * w.x);
        case 3: return make_float2(-fky * w.y, fky * w.x);
        case 4: return make_float2(-fky * psi.y * pf, fky * psi.x * pf);
        default: return make_float2(fkx * psi.y * pf, -fkx * psi.x * pf);
    }
}

// AB2 update of one mode (q in the column-major arrays), N the unmasked
// N-hat.  omega-hat is held as an unevaluated sum w_hi + w_lo of two floats:
// one float would round the small per-step change (the viscous decay is only
// nu k^2 dt of w) the same way step after step; the pair keeps about 44 bits.
// mode 0 (integrating factor): E = exp(-nu k^2 dt) = ex[kx] ey[ky] as a
//   double-float; w <- E w - dt (3/2 E N - 1/2 E^2 H), H <- N.
// mode 1 (Eq. 10 as printed): R = -N - nu k^2 w; w <- w + dt (3/2 R - 1/2 H), H <- R.
// The first step is forward Euler in either mode.  Returns the new w_hi.
__device__ __forceinline__ float2 ab2_update(const ColArgs& a, size_t q, int kx, int j, float2 N,
                                             int first) {
    const int n = a.n, ky = wavenumber_row(j, n);
    if (!kept(kx, ky, n)) N = make_float2(0.f, 0.f);
    const float2 w = a.what[q], wl = a.what_lo[q];
    const float2 H = first ? make_float2(0.f, 0.f) : a.hist[q];
    const float dt = a.dt;
    float2 inc, hi, lo, hist_out;
    if (a.mode == 0) {
        const float2 ea = a.ex[kx], eb = a.ey[j];
        const float Eh = ea.x * eb.x;
        const float El = fmaf(ea.x, eb.x, -Eh) + fmaf(ea.x, eb.y, ea.y * eb.x);
        const float E2 = Eh * Eh;
        const float c1 = first ? dt : 1.5f * dt, c2 = first ? 0.f : 0.5f * dt * E2;
        const float px = Eh * w.x, py = Eh * w.y;
        hi = make_float2(px, py);
        lo = make_float2(fmaf(Eh, w.x, -px) + fmaf(El, w.x, Eh * wl.x),
                         fmaf(Eh, w.y, -py) + fmaf(El, w.y, Eh * wl.y));
        inc = make_float2(fmaf(c2, H.x, -c1 * Eh * N.x), fmaf(c2, H.y, -c1 * Eh * N.y));
        hist_out = N;
    } else {
        const float nuk2 = a.nu * (float)(kx * kx + ky * ky);
        const float2 R = make_float2(-N.x - nuk2 * w.x, -N.y - nuk2 * w.y);
        inc = first ? make_float2(dt * R.x, dt * R.y)
                      : make_float2(dt * (1.5f * R.x - 0.5f * H.x), dt * (1.5f * R.y - 0.5f * H.y));
        hi = w;
        lo = wl;
        hist_out = R;
    }
    float sx, exx, sy, eyy;
    two_sum(hi.x, lo.x + inc.x, sx, exx);
    two_sum(hi.y, lo.y + inc.y, sy, eyy);
    a.hist[q] = hist_out;
    a.what[q] = make_float2(sx, sy);
    a.what_lo[q] = make_float2(exx, eyy);
    return make_float2(sx, sy);
}

// Threads a column-pass block needs: 16 values per thread.
__host__ __device__ __forceinline__ int col_threads(int n, int log2tc) {
    const int t = (n << log2tc) / 16;
    return t < 32 ? 32 : t;
}
__host__ __device__ __forceinline__ int col_tiles(int n, int log2tc) { return (n / 2) >> log2tc; }
// The transform buffer and the new omega-hat of the tile.
__host__ __device__ __forceinline__ size_t col_smem_bytes(int log2n, int log2tc) {
    return 2 * (size_t)fft_seq_stride(log2n) * ((size_t)1 << log2tc) * sizeof(float2);
}

// Column pass of tile `tile` (columns tile * tc .. tile * tc + tc - 1);
// first = forward Euler, advance = 0 only builds the planes of the current
// omega-hat (set-up).  REM = log2(n) mod 4.
template <int REM>
__device__ __forceinline__ void column_tile(const ColArgs& a, int first, int advance, int tile,
                                            float2* sm) {
    int tid = threadIdx.x, bd = blockDim.x;
    asm volatile("" : "+r"(tid), "+r"(bd));  // not invariant in a persistent caller's loop
    const int n = a.n, log2n = a.log2n, log2tc = a.log2tc, tc = 1 << log2tc;
    const int ss = fft_seq_stride(log2n);
    const int c0 = tile << log2tc;
    const int total = n << log2tc;
    float2* wb = sm + tc * ss;  // omega-hat / n^2 of the tile's modes
    if (advance) {
#pragma unroll 2
        for (int e = tid; e < total; e += bd) {
            const int t = e & (tc - 1), y = e >> log2tc;
            sm[t * ss + pidx(y)] = a.nrow[(size_t)y * a.pitch + c0 + t];
        }
        __syncthreads();
        fft_smem<-1, REM>(sm, log2n, tc, ss, a.tw);
    }
#pragma unroll 2
    for (int e = tid; e < total; e += bd) {
        const int t = e >> log2n, j = e & (n - 1), kx = c0 + t;
        const size_t q = (size_t)kx * n + j;
        const int i = t * ss + pidx(j);
        float2 w = advance ? ab2_update(a, q, kx, j, sm[i], first) : a.what[q];
        wb[i] = make_float2(w.x * a.scale, w.y * a.scale);
    }
    for (int p = 0; p < a.nplanes; p++) {
        __syncthreads();  // the new omega-hat is complete; the previous plane is stored
#pragma unroll 2
        for (int e = tid; e < total; e += bd) {
            const int t = e >> log2n, j = e & (n - 1);
            const int i = t * ss + pidx(j);
            sm[i] = plane_value(a, p, wb[i], c0 + t, j);
        }
        __syncthreads();
        fft_smem<1, REM>(sm, log2n, tc, ss, a.tw);
        float2* out = a.planes + (size_t)p * a.pstride;
#pragma unroll 2
        for (int e = tid; e < total; e += bd) {
            const int t = e & (tc - 1), y = e >> log2tc;
            out[(size_t)y * a.pitch + c0 + t] = sm[t * ss + pidx(y)];
        }
    }
    __syncthreads();
}

// Everything the row pass of one flow reads and writes.
struct RowArgs {
    const float2* planes;    // [p][y][pitch] from the column pass
    float2* nrow;            // output: N transformed along x, [y][pitch]
    const float2* tw;        // fft_twiddles(log2n - 1)
    const float2* wn;        // exp(-2 pi i k / n), k = 0..n/2
    size_t pstride;
    int n, log2n, pitch, nplanes, stencil_plane, psi_plane;
};

// The level pairs one row pass produces (level m).
struct RowLevel {
    const float4* snap_src;  // pair (m-2, m-1): level m-1 in its second half
    float4* snap_dst;        // pair (m-1, m)
    float4* snap_other;      // set-up only: the other pair, also filled with level 0
    const float2* psi_src;   // the same for the streamfunction (or nullptr)
    float2* psi_dst;
    float2* psi_other;
    int setup;
};

// Columns per column-pass tile: 4 up to n = 1024, then 2, then 1 (the
// tile's shared memory stays the same).
__host__ __device__ __forceinline__ int col_log2tc(int n) { return n <= 1024 ? 2 : (n == 2048 ? 1 : 0); }
// Largest shared memory any flow's passes take (n <= 4096, up to 7 planes):
// the kernels' limit is raised to it once, so flows of different sizes
// never lower it under one another.
constexpr int kMaxPlanes = 7;
size_t max_col_smem_bytes();
size_t max_row_smem_bytes();

ColArgs column_args(const el_flow* f);                // fluid.cu
RowArgs row_args(const el_flow* f);
RowLevel row_level(const el_flow* f, int64_t m, bool setup);  // producing level m

// At most 512 threads; the planes' transforms then run in groups.
__host__ __device__ __forceinline__ int row_threads(int n, int nplanes) {
    int t = nplanes * (n / 2) / 16;
    t = (t + 31) / 32 * 32;
    return t < 32 ? 32 : (t > 512 ? 512 : t);
}
__host__ __device__ __forceinline__ size_t row_smem_bytes(int log2n, int nplanes) {
    return (size_t)fft_seq_stride(log2n - 1) * nplanes * sizeof(float2);
}

// Row pass of grid row y.  The level pair (m-1, m) is written as one full
// 16-byte store per node: (level m-1 read from the second half of the source
// pair, level m).  At set-up level 0 fills both halves of both pairs, so no
// pair ever holds uninitialised values.  REM = log2(n / 2) mod 4.
template <int REM>
__device__ __forceinline__ void row_pass(const RowArgs& a, const RowLevel& lv, int y, float2* sm) {
    int tid = threadIdx.x, bd = blockDim.x;
    asm volatile("" : "+r"(tid), "+r"(bd));  // not invariant in a persistent caller's loop
    const int n = a.n, h = n / 2, log2h = a.log2n - 1;
    const int ss = fft_seq_stride(log2h);
    const int np = a.nplanes;
    // inverse real FFT, step 1: Z_k = (X_k + conj X_{h-k}) + i W^-k (X_k - conj X_{h-k})
#pragma unroll 2
    for (int e = tid; e < np * h; e += bd) {
        const int p = e >> log2h, k = e & (h - 1);
        const float2* row = a.planes + (size_t)p * a.pstride + (size_t)y * a.pitch;
        const float2 xk = row[k], xm = conjf2(row[h - k]);
        const float2 s = cadd(xk, xm);
        const float2 wd = cmul(csub(xk, xm), conjf2(a.wn[k]));
        sm[p * ss + pidx(k)] = make_float2(s.x - wd.y, s.y + wd.x);
    }
    __syncthreads();
    const int per = (bd * 16) >> log2h;  // sequences one transform call covers
    for (int p0 = 0; p0 < np; p0 += per)
        fft_smem<1, REM>(sm + p0 * ss, log2h, np - p0 < per ? np - p0 : per, ss, a.tw);
    // nodes 2m (real parts) and 2m + 1 (imaginary parts)
#pragma unroll 1
    for (int m = tid; m < h; m += bd) {
        const int im = pidx(m);
        const float2 u = sm[im], v = sm[ss + im], wx = sm[2 * ss + im], wy = sm[3 * ss + im];
        float2 su = u, sv = v;
        if (a.stencil_plane != 0) {
            su = sm[a.stencil_plane * ss + im];
            sv = sm[(a.stencil_plane + 1) * ss + im];
        }
        const size_t node = (size_t)y * n + 2 * m;
        if (lv.setup) {
            const float4 l0 = make_float4(su.x, sv.x, su.x, sv.x), l1 = make_float4(su.y, sv.y, su.y, sv.y);
            lv.snap_dst[node] = l0;
            lv.snap_dst[node + 1] = l1;
            lv.snap_other[node] = l0;
            lv.snap_other[node + 1] = l1;
        } else {
            const float4 o0 = lv.snap_src[node], o1 = lv.snap_src[node + 1];
            lv.snap_dst[node] = make_float4(o0.z, o0.w, su.x, sv.x);
            lv.snap_dst[node + 1] = make_float4(o1.z, o1.w, su.y, sv.y);
        }
        if (a.psi_plane >= 0) {
            const float2 ps = sm[a.psi_plane * ss + im];
            if (lv.setup) {
                lv.psi_dst[node] = make_float2(ps.x, ps.x);
                lv.psi_dst[node + 1] = make_float2(ps.y, ps.y);
                lv.psi_other[node] = make_float2(ps.x, ps.x);
                lv.psi_other[node + 1] = make_float2(ps.y, ps.y);
            } else {
                lv.psi_dst[node] = make_float2(lv.psi_src[node].y, ps.x);
                lv.psi_dst[node + 1] = make_float2(lv.psi_src[node + 1].y, ps.y);
            }
        }
        // this thread alone reads and writes index m of sequence 0
        sm[im] = make_float2(fmaf(u.x, wx.x, v.x * wy.x), fmaf(u.y, wx.y, v.y * wy.y));
    }
    __syncthreads();
    fft_smem<-1, REM>(sm, log2h, 1, ss, a.tw);
    // forward real FFT, last step: X_k = (Z_k + conj Z_{h-k}) / 2 + W^k (Z_k - conj Z_{h-k}) / 2i
    float2* out = a.nrow + (size_t)y * a.pitch;
#pragma unroll 2
    for (int k = tid; k <= h; k += bd) {
        const float2 zk = sm[pidx(k & (h - 1))], zm = conjf2(sm[pidx((h - k) & (h - 1))]);
        const float2 ev = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
        const float2 od = make_float2(0.5f * (zk.y - zm.y), -0.5f * (zk.x - zm.x));
        out[k] = cadd(ev, cmul(od, a.wn[k]));
    }
    __syncthreads();
}

}  // namespace el
