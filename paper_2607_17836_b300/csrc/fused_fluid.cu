// The pseudospectral step (Sec. 3.1, Eqs. 4-10) as four kernels of our own
// instead of the pointwise kernels around cuFFT's 2-D transforms, for one
// flow or for every member of a batch on the same grid at once (the member in
// the grid's last dimension; OneFlow / Members below).  The kernels below are
// written out for 1024^2 (one warp per 1024-point transform); 2048^2 runs
// each 2048-point transform on a warp pair, 256^2 and 512^2 on lane groups.
// Only the modes the 2/3 rule keeps are ever nonzero (the initial field is
// projected, N-hat is masked every step), so every transform is pruned to
// them: at 1024^2, 342 of the 513 columns kx and 683 of the 1024 rows ky.
//
//   k_fused_advance    : the AB2 update of the kept modes (advance_mode) in
//                        32 x 32 tiles, and every spectral plane of the new
//                        omega-hat (plane_value) written transposed, S[p][kx][j]
//   k_fused_columns<P> : one warp per plane and kept column: the inverse
//                        transform along y (1024 points) into G[p][kx][y]
//   k_fused_rows<P>    : one warp per row y: the planes' inverse real
//                        transforms along x, two real planes per complex
//                        transform (u + i v, wx + i wy, ...), the nonlinear
//                        term N = u wx + v wy (Eq. 7), the level pair (n, n+1)
//                        the particle step reads, and the forward transform of
//                        N along x, kept columns only, into H[kx][y]
//   k_fused_nhat       : one warp per kept column: the forward transform of
//                        H along y, kept rows only, into N-hat (Eq. 8)
//
// The state between steps is the cuFFT path's: omega-hat (high and low
// parts), the AB2 history, N-hat and the level pairs; the physical planes
// are not written (fluid_get_field rebuilds them when asked).  Every global
// access is coalesced: the row-major state is read along kx and the
// transposes go through shared memory.
//
// Every transform is 1024 = 32 x 32 points held by one warp, 32 per lane:
// lane l holds elements l + 32 i in register i.  A 32-point DFT over each
// lane's registers (radix-2, decimation in frequency, compile-time
// twiddles), the twiddles exp(+-2 pi i l k1 / 1024) from a per-block
// shared-memory table, a transpose through shared memory (row pitch 33:
// conflict-free), and a 32-point DFT over the lanes' values leave X[l + 32 k]
// in register k of lane l: the same layout as the input.
#include "common.cuh"
#include "stages.cuh"

#include <cstdlib>


namespace el {
namespace {

constexpr int kFN = 1024;         // grid size of the fused step
constexpr int kFKC = 342;         // kept columns: kx in [0, 342) (3 kx < 1024)
constexpr int kFKCP = 344;        // kept columns padded: rows of the intermediate arrays
constexpr int kTP = 33;           // row pitch (float2) of a warp's transpose buffer
constexpr int kTB = 32 * kTP;     // float2 in a warp's transpose buffer
constexpr int kRowWarps = 4;      // rows (warps) per block of k_fused_rows
constexpr int kNhatWarps = 4;     // columns (warps) per block of k_fused_nhat

// cos(2 pi m / 32) for m = 0..8.
__host__ __device__ constexpr float cos32_q(int m) {
    return m == 0   ? 1.0f
           : m == 1 ? 0.980785280403230449126f
           : m == 2 ? 0.923879532511286756128f
           : m == 3 ? 0.831469612302545237079f
           : m == 4 ? 0.707106781186547524401f
           : m == 5 ? 0.555570233019602224743f
           : m == 6 ? 0.382683432365089771728f
           : m == 7 ? 0.195090322016128267848f
                    : 0.0f;
}

// d * exp(DIR 2 pi i m / 32) for m in [0, 16) (a compile-time constant once
// the loops that call it are unrolled).
template <int DIR>
__device__ __forceinline__ float2 rot32(float2 d, int m) {
    if (m == 0) return d;
    if (m == 8) return DIR > 0 ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    const float c = m < 8 ? cos32_q(m) : -cos32_q(16 - m);
    const float sn = m < 8 ? cos32_q(8 - m) : cos32_q(m - 8);
    const float s = DIR > 0 ? sn : -sn;
    return make_float2(fmaf(d.x, c, -d.y * s), fmaf(d.x, s, d.y * c));
}

__host__ __device__ constexpr int bitrev5(int k) {
    return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

// v[k] <- sum_n v[n] exp(DIR 2 pi i n k / 32), in registers.
template <int DIR>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
#pragma unroll
    for (int M = 32; M >= 2; M >>= 1) {
#pragma unroll
        for (int g = 0; g < 32; g += M) {
#pragma unroll
            for (int j = 0; j < M / 2; j++) {
                const float2 a = v[g + j], b = v[g + j + M / 2];
                v[g + j] = __fadd2_rn(a, b);
                v[g + j + M / 2] = rot32<DIR>(fsub2(a, b), j * (32 / M));
            }
        }
    }
    float2 t[32];
#pragma unroll
    for (int k = 0; k < 32; k++) t[k] = v[bitrev5(k)];
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = t[k];
}

// The 1024-point transform of the warp's 32 x 32 values (see the file
// comment).  tw2[k1 * 32 + l] = exp(-2 pi i l k1 / 1024); tb: this warp's
// transpose buffer.
template <int DIR>
__device__ __forceinline__ void fft1024(float2 (&v)[32], float2* __restrict__ tb,
                                        const float2* __restrict__ tw2, int lane) {
    dft32<DIR>(v);
#pragma unroll
    for (int k1 = 1; k1 < 32; k1++) {
        float2 t = tw2[k1 * 32 + lane];
        if (DIR > 0) t.y = -t.y;
        const float2 x = v[k1];
        v[k1] = make_float2(fmaf(x.x, t.x, -x.y * t.y), fmaf(x.x, t.y, x.y * t.x));
    }
#pragma unroll
    for (int k1 = 0; k1 < 32; k1++) tb[k1 * kTP + lane] = v[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 32; n2++) v[n2] = tb[lane * kTP + n2];
    __syncwarp();
    dft32<DIR>(v);
}

// v[k] <- sum_n v[n] exp(DIR 2 pi i n k / L) for L in {2, 4, 8, 16}, in
// registers (radix-2, decimation in frequency, as dft32).
template <int L>
__host__ __device__ constexpr int bitrev_l(int k) {
    int r = 0;
    for (int b = 1, t = L >> 1; b < L; b <<= 1, t >>= 1)
        if (k & b) r |= t;
    return r;
}
template <int DIR, int L>
__device__ __forceinline__ void dftL(float2 (&v)[L]) {
#pragma unroll
    for (int M = L; M >= 2; M >>= 1) {
#pragma unroll
        for (int g = 0; g < L; g += M) {
#pragma unroll
            for (int j = 0; j < M / 2; j++) {
                const float2 a = v[g + j], b = v[g + j + M / 2];
                v[g + j] = __fadd2_rn(a, b);
                v[g + j + M / 2] = rot32<DIR>(fsub2(a, b), j * (32 / M));
            }
        }
    }
    float2 t[L];
#pragma unroll
    for (int k = 0; k < L; k++) t[k] = v[bitrev_l<L>(k)];
#pragma unroll
    for (int k = 0; k < L; k++) v[k] = t[k];
}

// The N = 32 M-point transform (M in {4, 8, 16}) held by a group of M lanes
// (gl = lane % M; a warp holds 32 / M groups), 32 values per lane: lane gl
// holds x[gl + M i] in register i on entry and X[gl + M i] on exit.  A
// 32-point DFT over each lane's registers, the twiddles exp(DIR 2 pi i gl k1
// / N) from the block's table twg[k1 M + gl], a transpose through the
// group's buffer tbg (32 rows of M + 1), and 32 / M DFTs of M points over the
// group's lanes (fft1024 is the case M = 32).
template <int DIR, int M>
__device__ __forceinline__ void fft_group(float2 (&v)[32], float2* __restrict__ tbg,
                                          const float2* __restrict__ twg, int gl) {
    dft32<DIR>(v);
#pragma unroll
    for (int k1 = 1; k1 < 32; k1++) {
        float2 t = twg[k1 * M + gl];
        if (DIR > 0) t.y = -t.y;
        const float2 x = v[k1];
        v[k1] = make_float2(fmaf(x.x, t.x, -x.y * t.y), fmaf(x.x, t.y, x.y * t.x));
    }
#pragma unroll
    for (int k1 = 0; k1 < 32; k1++) tbg[k1 * (M + 1) + gl] = v[k1];
    __syncwarp();
    constexpr int J = 32 / M;
#pragma unroll
    for (int j = 0; j < J; j++) {
        float2 w[M];
#pragma unroll
        for (int l = 0; l < M; l++) w[l] = tbg[(gl + M * j) * (M + 1) + l];
        dftL<DIR, M>(w);
#pragma unroll
        for (int k2 = 0; k2 < M; k2++) v[j + J * k2] = w[k2];  // X[gl + M j + 32 k2]
    }
    __syncwarp();
}

// The block's table for fft_group from the N-entry table exp(-2 pi i m / N):
// twg[k1 M + gl] = exp(-2 pi i gl k1 / N) (NT threads).
template <int M, int NT>
__device__ __forceinline__ void load_twiddles_group(float2* __restrict__ twg, const float2* __restrict__ tw) {
    constexpr int E = 32 * M, passes = (E + NT - 1) / NT;
    float2 t[passes];
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < E) t[k] = tw[(e % M) * (e / M)];
    }
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < E) twg[e] = t[k];
    }
}

// The block's twiddle table from the 1024-entry table exp(-2 pi i m / 1024)
// (NT threads; every load of a thread issued before its stores).
template <int NT>
__device__ __forceinline__ void load_twiddles(float2* __restrict__ tw2, const float2* __restrict__ tw) {
    constexpr int passes = (1024 + NT - 1) / NT;
    float2 t[passes];
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < 1024) t[k] = tw[(e & 31) * (e >> 5)];
    }
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < 1024) tw2[e] = t[k];
    }
}

// The kept rows of a column, indexed r in [0, 683): j = r (r < 342) or
// r + 341 (ky = j - 1024 in [-341, -1]).
constexpr int kFKR = 683;
__device__ __forceinline__ int kept_row(int r) { return r < kFKC ? r : r + (kFN - kFKR); }
__device__ __forceinline__ bool row_is_kept(int j) { return j < kFKC || j >= kFN - kFKR + kFKC; }

constexpr int kTile = 32;  // KA's tiles: 32 kept rows x 32 columns

// The kept spectrum of an N^2 grid (2/3 rule): columns kx < KC, rows ky in
// [-(KC - 1), KC - 1], i.e. KR = 2 KC - 1 rows j = ky mod N; the
// intermediate arrays hold KCP >= KC columns of N values.
template <int N>
struct Geo;
template <>
struct Geo<1024> {
    static constexpr int KC = kFKC, KCP = kFKCP, KR = kFKR;
};
template <>
struct Geo<2048> {
    static constexpr int KC = 683, KCP = 688, KR = 1365;
};
template <>
struct Geo<128> {
    static constexpr int KC = 43, KCP = 48, KR = 85;
};
template <>
struct Geo<256> {
    static constexpr int KC = 86, KCP = 88, KR = 171;
};
template <>
struct Geo<512> {
    static constexpr int KC = 171, KCP = 176, KR = 341;
};
template <int N>
__device__ __forceinline__ int kept_row_n(int r) {
    return r < Geo<N>::KC ? r : r + (N - Geo<N>::KR);
}
template <int N>
__device__ __forceinline__ bool row_kept_n(int j) {
    return j < Geo<N>::KC || j >= N - Geo<N>::KR + Geo<N>::KC;
}

// ---- 2048-point transforms on a warp pair -----------------------------------
// A 2048-point transform is two 1024-point ones (fft1024) joined by one
// radix-2 step, the two halves on the two warps of a pair (half = 0: A,
// 1: B), which exchange them through their transpose buffers (free once
// fft1024 returns) under a named barrier of the pair.  With W = exp(DIR 2 pi
// i / 2048):
//   decimation in time (the inverse transforms here): A transforms the even
//     samples x[2m] (E), B the odd ones x[2m+1] (O); X[k] = E[k] + W^k O[k],
//     X[k + 1024] = E[k] - W^k O[k]: A ends with X[lane + 32 i], B with
//     X[1024 + lane + 32 i];
//   decimation in frequency (the forward ones): from x[n] and x[n + 1024],
//     A transforms x[n] + x[n + 1024] into X[2k], B (x[n] - x[n + 1024]) W^n
//     into X[2k + 1], k = lane + 32 i.
// Twiddles: tw2 as for fft1024, and comb[n] = exp(-2 pi i n / 2048), n < 1024.

// The block's tables from the 2048-entry table exp(-2 pi i m / 2048) (NT
// threads; every load of a thread issued before its stores).
template <int NT>
__device__ __forceinline__ void load_twiddles2k(float2* __restrict__ tw2, float2* __restrict__ comb,
                                                const float2* __restrict__ tw) {
    constexpr int passes = (2048 + NT - 1) / NT;
    float2 t[passes];
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < 1024) t[k] = tw[2 * ((e & 31) * (e >> 5))];  // exp(-2 pi i l k1 / 1024)
        else if (e < 2048) t[k] = tw[e - 1024];
    }
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < 1024) tw2[e] = t[k];
        else if (e < 2048) comb[e - 1024] = t[k];
    }
}

// Barrier of the warp pair `pair` (named barriers 1..15; 0 is __syncthreads).
__device__ __forceinline__ void pair_sync(int pair) {
    asm volatile("bar.sync %0, 64;" ::"r"(pair + 1) : "memory");
}

__device__ __forceinline__ float2 cmul(float2 x, float2 t) {
    return make_float2(fmaf(x.x, t.x, -x.y * t.y), fmaf(x.x, t.y, x.y * t.x));
}
template <int DIR>
__device__ __forceinline__ float2 comb_w(const float2* __restrict__ comb, int n) {
    float2 t = comb[n];
    if (DIR > 0) t.y = -t.y;
    return t;
}

// Decimation in time (see above): v holds this warp's parity of the input on
// entry, its half of the output on exit.
template <int DIR>
__device__ __forceinline__ void fft2048_dit(float2 (&v)[32], float2* __restrict__ tb, const float2* __restrict__ tb_other,
                                            const float2* __restrict__ tw2, const float2* __restrict__ comb,
                                            int lane, int half, int pair) {
    fft1024<DIR>(v, tb, tw2, lane);
    if (half) {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = cmul(v[i], comb_w<DIR>(comb, lane + 32 * i));
    }
#pragma unroll
    for (int i = 0; i < 32; i++) tb[lane + 32 * i] = v[i];  // E (A) or W^k O (B)
    pair_sync(pair);
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const float2 o = tb_other[lane + 32 * i];
        v[i] = half ? fsub2(o, v[i]) : __fadd2_rn(v[i], o);
    }
    pair_sync(pair);  // the partner is done reading this warp's buffer
}

// Decimation in frequency from both halves of the input (lo = x[n], hi =
// x[n + 1024], n = lane + 32 i): v ends with X[2k + half].
template <int DIR>
__device__ __forceinline__ void fft2048_dif(float2 (&v)[32], const float2 (&lo)[32], const float2 (&hi)[32],
                                            float2* __restrict__ tb, const float2* __restrict__ tw2,
                                            const float2* __restrict__ comb, int lane, int half) {
#pragma unroll
    for (int i = 0; i < 32; i++)
        v[i] = half ? cmul(fsub2(lo[i], hi[i]), comb_w<DIR>(comb, lane + 32 * i)) : __fadd2_rn(lo[i], hi[i]);
    fft1024<DIR>(v, tb, tw2, lane);
}

// The arguments of one flow's fused step (RowArgs: those of k_fused_rows).
struct RowArgs {
    const float2* G;        // [P][kFKCP][kFN] planes after the column transforms
    float2* H;              // [kFKCP][kFN] N after the row transform (kept columns)
    const float2* tw;       // exp(-2 pi i m / 1024), m < 1024
    const float4* src;      // level pair (m-2, m-1)
    float4* dst;            // level pair (m-1, m)
    const float2* psi_src;  // streamfunction pairs, or nullptr
    float2* psi_dst;
    int psi_plane;
};

// Where a launch's flows come from.  OneFlow: one flow, every argument
// computed on the host (in the kernels' parameter space).  Members: batched
// flows (device records, one per grid slice: blockIdx.z of KA, blockIdx.y of
// the others), the step-dependent arguments derived from each member's step
// counter + `ahead`, as the batched spectral and nonlinear kernels do.
struct OneFlow {
    SpecArgs a;
    RowArgs r;
    float2* S;
    float2* G;
    float2* nhat;
    __device__ __forceinline__ const SpecArgs& spec(int) const { return a; }
    __device__ __forceinline__ float2* planes_s(int) const { return S; }
    __device__ __forceinline__ float2* planes_g(int) const { return G; }
    __device__ __forceinline__ const RowArgs& rows(int) const { return r; }
    __device__ __forceinline__ const float2* h(int) const { return r.H; }
    __device__ __forceinline__ float2* nhat_out(int) const { return nhat; }
};

struct Members {
    const FusedMember* m;
    const float2* tw;
    int ahead;
    __device__ __forceinline__ long long step(int k) const { return *m[k].step + ahead; }
    __device__ __forceinline__ SpecArgs spec(int k) const {
        SpecArgs a = m[k].spec;
        a.first = step(k) == 0;
        return a;
    }
    __device__ __forceinline__ float2* planes_s(int k) const { return m[k].S; }
    __device__ __forceinline__ float2* planes_g(int k) const { return m[k].G; }
    __device__ __forceinline__ RowArgs rows(int k) const {
        const FusedMember& f = m[k];
        const long long lv = step(k) + 1;  // the level this step produces
        RowArgs r;
        r.G = f.G;
        r.H = f.H;
        r.tw = tw;
        r.src = f.snap[lv % 2];        // pair (lv-2, lv-1)
        r.dst = f.snap[(lv + 1) % 2];  // pair (lv-1, lv)
        r.psi_src = f.psi_plane >= 0 ? f.psi[lv % 2] : nullptr;
        r.psi_dst = f.psi_plane >= 0 ? f.psi[(lv + 1) % 2] : nullptr;
        r.psi_plane = f.psi_plane;
        return r;
    }
    __device__ __forceinline__ const float2* h(int k) const { return m[k].H; }
    __device__ __forceinline__ float2* nhat_out(int k) const { return m[k].nhat; }
};

// KA: the AB2 update of a 32 x 32 tile of kept modes (rows r0.., columns
// kx0..), read and written in the row-major state (32 consecutive kx per
// warp), then each spectral plane of the new omega-hat written transposed,
// S[p][kx][j], through a shared-memory tile (32 consecutive j per warp).
// Block: 32 x 8 threads; blockIdx.z: the flow.
template <int N, int P, class Src>
__global__ void __launch_bounds__(256) k_fused_advance(const __grid_constant__ Src src) {
    using Gm = Geo<N>;
    const auto& a = src.spec(blockIdx.z);
    float2* __restrict__ S = src.planes_s(blockIdx.z);
    __shared__ float2 tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int kx0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
    const int kx = kx0 + tx;
    ModeIn in[kTile / 8];
#pragma unroll
    for (int m = 0; m < kTile / 8; m++) {  // every load first
        const int r = r0 + ty + 8 * m, j = kept_row_n<N>(r);
        if (r < Gm::KR && kx < Gm::KC) in[m] = load_mode(a, kx, j, (size_t)j * a.nh + kx);
    }
#pragma unroll
    for (int m = 0; m < kTile / 8; m++) {
        const int r = r0 + ty + 8 * m, j = kept_row_n<N>(r);
        float2 w = make_float2(0.f, 0.f);
        if (r < Gm::KR && kx < Gm::KC) w = advance_loaded(a, kx, j, (size_t)j * a.nh + kx, in[m]);
        tile[ty + 8 * m][tx] = w;
    }
    __syncthreads();
    const int r = r0 + tx;
    if (r >= Gm::KR) return;  // no barrier follows
    const int j = kept_row_n<N>(r);
#pragma unroll
    for (int m = 0; m < kTile / 8; m++) {
        const int kx = kx0 + ty + 8 * m;
        if (kx >= Gm::KC) break;
        const float2 w = tile[tx][ty + 8 * m];
#pragma unroll
        for (int p = 0; p < P; p++) S[((size_t)p * Gm::KCP + kx) * N + j] = plane_value(a, p, kx, j, w);
    }
}

// KB: the inverse transform along y of plane p, column kx (warp p of block
// kx): S[p][kx][j] for the kept rows (zero elsewhere, never read) into
// G[p][kx][y].  Block: P warps; blockIdx.y: the flow.
template <int P, class Src>
__global__ void __launch_bounds__(P * 32) k_fused_columns(const __grid_constant__ Src src,
                                                          const float2* __restrict__ tw) {
    const float2* __restrict__ S = src.planes_s(blockIdx.y);
    float2* __restrict__ G = src.planes_g(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* tw2 = sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tb = sm + 1024 + warp * kTB;
    load_twiddles<P * 32>(tw2, tw);
    __syncthreads();
    const size_t col = ((size_t)warp * kFKCP + blockIdx.x) * kFN;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int j = lane + 32 * i;
        v[i] = row_is_kept(j) ? S[col + j] : make_float2(0.f, 0.f);
    }
    fft1024<1>(v, tb, tw2, lane);
#pragma unroll
    for (int i = 0; i < 32; i++) G[col + lane + 32 * i] = v[i];
}


constexpr int kRowPitch = kFKCP;  // float2 per staged row of a plane in KC

// KC's staging of one plane's x-spectrum (kept columns) of the block's
// kRowWarps rows: buf[yy][kx] = G[p][kx][y0 + yy].  Each warp reads 8
// columns x 4 rows (32-byte runs); every load of a thread is issued before
// its stores.
constexpr int kStageElems = kFKC * kRowWarps;
constexpr int kStagePasses = (kStageElems + kRowWarps * 32 - 1) / (kRowWarps * 32);
__device__ __forceinline__ void stage_plane(float2* __restrict__ buf, const float2* __restrict__ G, int p,
                                            int y0) {
    static_assert(kRowWarps == 4, "kx = e / 4, yy = e % 4");
    float2 t[kStagePasses];
#pragma unroll
    for (int k = 0; k < kStagePasses; k++) {
        const int e = threadIdx.x + k * kRowWarps * 32;
        if (e < kStageElems) t[k] = G[((size_t)p * kFKCP + (e >> 2)) * kFN + y0 + (e & 3)];
    }
#pragma unroll
    for (int k = 0; k < kStagePasses; k++) {
        const int e = threadIdx.x + k * kRowWarps * 32;
        if (e < kStageElems) buf[(e & 3) * kRowPitch + (e >> 2)] = t[k];
    }
}

__device__ __forceinline__ void stage_rows(float2* __restrict__ buf, const float2* __restrict__ G, int p0,
                                           int p1, int y0) {
    stage_plane(buf, G, p0, y0);
    if (p1 >= 0) stage_plane(buf + kRowWarps * kRowPitch, G, p1, y0);
}

// The same staging of planes p0 and p1 split in two: the loads into
// registers (issued early, in flight while the warp transforms), then the
// stores into the staging buffer (once every warp is done reading it).
struct Staged {
    float2 t[2][kStagePasses];
};
__device__ __forceinline__ void stage_load(Staged& st, const float2* __restrict__ G, int p0, int p1, int y0) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int p = q == 0 ? p0 : p1;
#pragma unroll
        for (int k = 0; k < kStagePasses; k++) {
            const int e = threadIdx.x + k * kRowWarps * 32;
            if (e < kStageElems) st.t[q][k] = G[((size_t)p * kFKCP + (e >> 2)) * kFN + y0 + (e & 3)];
        }
    }
}
__device__ __forceinline__ void stage_store(const Staged& st, float2* __restrict__ buf) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
#pragma unroll
        for (int k = 0; k < kStagePasses; k++) {
            const int e = threadIdx.x + k * kRowWarps * 32;
            if (e < kStageElems) buf[(q * kRowWarps + (e & 3)) * kRowPitch + (e >> 2)] = st.t[q][k];
        }
    }
}

// dst[x] = (src[x].z, src[x].w, new[x]) for the row's 1024 nodes (lane +
// 32 i holds new value v[i]): the read-modify-write of the level pair in
// batches of 8 loads per lane, the next batch's loads issued before the
// current batch is stored.
__device__ __forceinline__ void write_pair_row(const float4* __restrict__ src, float4* __restrict__ dst,
                                               const float2 (&v)[32], int lane) {
    float4 cur[8], nxt[8];
#pragma unroll
    for (int k = 0; k < 8; k++) cur[k] = src[lane + 32 * k];
#pragma unroll
    for (int b = 0; b < 4; b++) {
        if (b < 3) {
#pragma unroll
            for (int k = 0; k < 8; k++) nxt[k] = src[lane + 32 * (8 * (b + 1) + k)];
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int i = 8 * b + k;
            dst[lane + 32 * i] = make_float4(cur[k].z, cur[k].w, v[i].x, v[i].y);
        }
        if (b < 3) {
#pragma unroll
            for (int k = 0; k < 8; k++) cur[k] = nxt[k];
        }
    }
}

// The complex row sequence z[k] = A[k] + i B[k] of two real planes (staged
// in `buf` for this warp's row), for register k = lane + 32 i: kept columns,
// their mirror images (Hermitian symmetry of a real plane's spectrum) for
// k > 1024 - 342, zero between.  The kx = 0 value of a real plane is real.
__device__ __forceinline__ void row_pair(float2 (&v)[32], const float2* __restrict__ bufA,
                                         const float2* __restrict__ bufB, int lane) {
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int k = lane + 32 * i;
        float2 z = make_float2(0.f, 0.f);
        if (k < kFKC || k > kFN - kFKC) {
            const int kk = k < kFKC ? k : kFN - k;
            float2 A = bufA[kk];
            float2 B = bufB ? bufB[kk] : make_float2(0.f, 0.f);
            if (kk == 0) {
                A.y = 0.f;
                B.y = 0.f;
            }
            z = k < kFKC ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
        }
        v[i] = z;
    }
}

// KC: rows y0 .. y0 + kRowWarps - 1 (one per warp): the planes' inverse real
// transforms along x, two real planes per complex transform, the nonlinear
// term N = u wx + v wy (Eq. 7), the level pair (and streamfunction pair),
// and the forward transform of N along x into H[kx][y] (kept columns,
// written in 32-byte runs through the staging buffer).  blockIdx.y: the flow.
template <int P, class Src>
__global__ void __launch_bounds__(kRowWarps * 32) k_fused_rows(const __grid_constant__ Src src) {
    const auto& r = src.rows(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* tw2 = sm;
    float2* buf = sm + 1024;  // 2 planes x kRowWarps rows x kRowPitch
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tb = buf + 2 * kRowWarps * kRowPitch + warp * (kTB + 1024);
    float2* hold = tb + kTB;  // (wx, wy) of the row: element lane + 32 i at [32 i + lane]
    float2* mine0 = buf + warp * kRowPitch;
    float2* mine1 = buf + (kRowWarps + warp) * kRowPitch;
    const int y0 = blockIdx.x * kRowWarps, y = y0 + warp;
    load_twiddles<kRowWarps * 32>(tw2, r.tw);
    stage_rows(buf, r.G, 2, 3, y0);
    Staged next;
    stage_load(next, r.G, 0, 1, y0);  // in flight during the first transform
    __syncthreads();
    float2 v[32];
    row_pair(v, mine0, mine1, lane);  // wx + i wy
    fft1024<1>(v, tb, tw2, lane);
#pragma unroll
    for (int i = 0; i < 32; i++) hold[32 * i + lane] = v[i];
    __syncthreads();
    stage_store(next, buf);
    __syncthreads();
    row_pair(v, mine0, mine1, lane);  // u + i v
    fft1024<1>(v, tb, tw2, lane);
    float nl[32];
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const float2 g = hold[32 * i + lane];
        nl[i] = fmaf(v[i].x, g.x, v[i].y * g.y);  // Eq. 7
    }
    if (P == 6 || P == 7) {  // the level pair holds the spline coefficients
        __syncthreads();
        stage_rows(buf, r.G, 4, 5, y0);
        __syncthreads();
        row_pair(v, mine0, mine1, lane);
        fft1024<1>(v, tb, tw2, lane);
    }
    write_pair_row(r.src + (size_t)y * kFN, r.dst + (size_t)y * kFN, v, lane);
    if (P == 5 || P == 7) {  // the streamfunction stencil field
        __syncthreads();
        stage_rows(buf, r.G, r.psi_plane, -1, y0);
        __syncthreads();
        row_pair(v, mine0, nullptr, lane);
        fft1024<1>(v, tb, tw2, lane);
        const float2* __restrict__ ps = r.psi_src + (size_t)y * kFN;
        float2* __restrict__ pd = r.psi_dst + (size_t)y * kFN;
#pragma unroll
        for (int i = 0; i < 32; i++) pd[lane + 32 * i] = make_float2(ps[lane + 32 * i].y, v[i].x);
    }
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = make_float2(nl[i], 0.f);
    fft1024<-1>(v, tb, tw2, lane);
    __syncthreads();  // every warp is done reading the staging buffer
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int kx = lane + 32 * i;
        if (kx < kFKC) buf[warp * kRowPitch + kx] = v[i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kFKC * kRowWarps; e += blockDim.x) {
        const int kx = e / kRowWarps, yy = e - kx * kRowWarps;
        r.H[(size_t)kx * kFN + y0 + yy] = buf[yy * kRowPitch + kx];
    }
}

// KD: N-hat of the kept modes of columns kx0 .. kx0 + kNhatWarps - 1 (one per
// warp) from H (forward transform along y), written to the row-major N-hat
// in 32-byte runs through a shared-memory staging buffer.  blockIdx.y: the flow.
template <class Src>
__global__ void __launch_bounds__(kNhatWarps * 32) k_fused_nhat(const __grid_constant__ Src src,
                                                               const float2* __restrict__ tw) {
    const float2* __restrict__ H = src.h(blockIdx.y);
    float2* __restrict__ nhat = src.nhat_out(blockIdx.y);
    constexpr int nh = kFN / 2 + 1;
    extern __shared__ float2 sm[];
    float2* tw2 = sm;
    float2* out = sm + 1024;  // [kFKR][kNhatWarps]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* tb = out + kFKR * kNhatWarps + warp * kTB;
    load_twiddles<kNhatWarps * 32>(tw2, tw);
    __syncthreads();
    const int kx0 = blockIdx.x * kNhatWarps, kx = kx0 + warp;
    float2 v[32];
    if (kx < kFKC) {  // whole warps
        const float2* __restrict__ col = H + (size_t)kx * kFN;
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = col[lane + 32 * i];
        fft1024<-1>(v, tb, tw2, lane);
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int j = lane + 32 * i;
            if (row_is_kept(j)) out[(j < kFKC ? j : j - (kFN - kFKR)) * kNhatWarps + warp] = v[i];
        }
    }
    __syncthreads();
    const int ncols = min(kNhatWarps, kFKC - kx0);
    for (int e = threadIdx.x; e < kFKR * kNhatWarps; e += blockDim.x) {
        const int rr = e / kNhatWarps, c = e - rr * kNhatWarps;
        if (c < ncols) nhat[(size_t)kept_row(rr) * nh + kx0 + c] = out[e];
    }
}

// ---- the 2048^2 step: the same four stages, each 2048-point transform on a warp pair ----

using G2 = Geo<2048>;
constexpr int k2N = 2048;
constexpr int k2Rows = 4;  // rows per block of KC2 (a warp pair each): 32-byte runs of G

// KB2: the inverse transform along y of column kx, the P planes one after
// another (S[p][kx][j] for the kept rows into G[p][kx][y]).  Block: one warp
// pair; blockIdx.y: the flow.
template <int P, class Src>
__global__ void __launch_bounds__(64) k_fused_columns2k(const __grid_constant__ Src src,
                                                        const float2* __restrict__ tw) {
    const float2* __restrict__ S = src.planes_s(blockIdx.y);
    float2* __restrict__ G = src.planes_g(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* tw2 = sm;
    float2* comb = sm + 1024;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = warp;
    float2* tb = sm + 2048 + warp * kTB;
    const float2* tb_other = sm + 2048 + (warp ^ 1) * kTB;
    load_twiddles2k<64>(tw2, comb, tw);
    __syncthreads();
    const int kx = blockIdx.x;
#pragma unroll 1
    for (int p = 0; p < P; p++) {
        const size_t col = ((size_t)p * G2::KCP + kx) * k2N;
        float2 v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int j = 2 * (lane + 32 * i) + half;  // this warp's parity of the rows
            v[i] = row_kept_n<k2N>(j) ? S[col + j] : make_float2(0.f, 0.f);
        }
        fft2048_dit<1>(v, tb, tb_other, tw2, comb, lane, half, 0);
#pragma unroll
        for (int i = 0; i < 32; i++) G[col + 1024 * half + lane + 32 * i] = v[i];
    }
}

// KC2's staging of one plane's x-spectrum (kept columns) of the block's
// k2Rows rows: buf[yy][kx] = G[p][kx][y0 + yy] (8 columns x 4 rows per warp
// request, 32-byte runs; every load of a thread issued before its stores).
constexpr int k2StageElems = G2::KC * k2Rows;
constexpr int k2Threads = 2 * k2Rows * 32;
constexpr int k2StagePasses = (k2StageElems + k2Threads - 1) / k2Threads;
__device__ __forceinline__ void stage_plane2k(float2* __restrict__ buf, const float2* __restrict__ G, int p,
                                              int y0) {
    static_assert(k2Rows == 4, "kx = e / 4, yy = e % 4");
    float2 t[k2StagePasses];
#pragma unroll
    for (int k = 0; k < k2StagePasses; k++) {
        const int e = threadIdx.x + k * k2Threads;
        if (e < k2StageElems) t[k] = G[((size_t)p * G2::KCP + (e >> 2)) * k2N + y0 + (e & 3)];
    }
#pragma unroll
    for (int k = 0; k < k2StagePasses; k++) {
        const int e = threadIdx.x + k * k2Threads;
        if (e < k2StageElems) buf[(e & 3) * G2::KCP + (e >> 2)] = t[k];
    }
}

// This warp's parity (k = 2m + half, m = lane + 32 i) of the full complex
// spectrum of two real planes packed as a + i b (bufB = nullptr: b = 0),
// from their staged kept columns (as row_pair).
__device__ __forceinline__ void row_pair2k(float2 (&v)[32], const float2* __restrict__ bufA,
                                           const float2* __restrict__ bufB, int lane, int half) {
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int k = 2 * (lane + 32 * i) + half;
        float2 z = make_float2(0.f, 0.f);
        if (k < G2::KC || k > k2N - G2::KC) {
            const int kk = k < G2::KC ? k : k2N - k;
            float2 A = bufA[kk];
            float2 B = bufB ? bufB[kk] : make_float2(0.f, 0.f);
            if (kk == 0) {
                A.y = 0.f;
                B.y = 0.f;
            }
            z = k < G2::KC ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
        }
        v[i] = z;
    }
}

// KC2: rows y0 .. y0 + 3, a warp pair each (as KC; each warp holds the half
// x in [1024 half, 1024 half + 1024) of its row between the transforms).
// Measured (2048^2, 4 planes): keeping (wx, wy) in shared memory instead of
// registers and loading planes 0 and 1 during the first transform, as KC
// does, took 71 us against 68 us.
template <int P, class Src>
__global__ void __launch_bounds__(k2Threads, 1) k_fused_rows2k(const __grid_constant__ Src src) {
    const auto& r = src.rows(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* tw2 = sm;
    float2* comb = sm + 1024;
    float2* buf = sm + 2048;  // 2 planes x k2Rows rows x KCP
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = warp >> 1, half = warp & 1;
    float2* tb = buf + 2 * k2Rows * G2::KCP + warp * kTB;
    const float2* tb_other = buf + 2 * k2Rows * G2::KCP + (warp ^ 1) * kTB;
    const float2* mine0 = buf + row * G2::KCP;
    const float2* mine1 = buf + (k2Rows + row) * G2::KCP;
    const int y0 = blockIdx.x * k2Rows, y = y0 + row;
    load_twiddles2k<k2Threads>(tw2, comb, r.tw);
    stage_plane2k(buf, r.G, 2, y0);
    stage_plane2k(buf + k2Rows * G2::KCP, r.G, 3, y0);
    __syncthreads();
    float2 v[32], hold[32];
    row_pair2k(v, mine0, mine1, lane, half);  // wx + i wy
    fft2048_dit<1>(v, tb, tb_other, tw2, comb, lane, half, row);
#pragma unroll
    for (int i = 0; i < 32; i++) hold[i] = v[i];
    __syncthreads();  // every warp has read the staging buffer
    stage_plane2k(buf, r.G, 0, y0);
    stage_plane2k(buf + k2Rows * G2::KCP, r.G, 1, y0);
    __syncthreads();
    row_pair2k(v, mine0, mine1, lane, half);  // u + i v
    fft2048_dit<1>(v, tb, tb_other, tw2, comb, lane, half, row);
    float nl[32];  // N at this warp's x
#pragma unroll
    for (int i = 0; i < 32; i++) nl[i] = fmaf(v[i].x, hold[i].x, v[i].y * hold[i].y);  // Eq. 7
    if (P == 6 || P == 7) {  // the level pair holds the spline coefficients
        __syncthreads();
        stage_plane2k(buf, r.G, 4, y0);
        stage_plane2k(buf + k2Rows * G2::KCP, r.G, 5, y0);
        __syncthreads();
        row_pair2k(v, mine0, mine1, lane, half);
        fft2048_dit<1>(v, tb, tb_other, tw2, comb, lane, half, row);
    }
    const size_t x0 = (size_t)y * k2N + 1024 * half;
    write_pair_row(r.src + x0, r.dst + x0, v, lane);
    if (P == 5 || P == 7) {  // the streamfunction stencil field
        __syncthreads();
        stage_plane2k(buf, r.G, r.psi_plane, y0);
        __syncthreads();
        row_pair2k(v, mine0, nullptr, lane, half);
        fft2048_dit<1>(v, tb, tb_other, tw2, comb, lane, half, row);
        const float2* __restrict__ ps = r.psi_src + x0;
        float2* __restrict__ pd = r.psi_dst + x0;
#pragma unroll
        for (int i = 0; i < 32; i++) pd[lane + 32 * i] = make_float2(ps[lane + 32 * i].y, v[i].x);
    }
    // the forward transform of N along x by decimation in frequency: each
    // warp needs the other warp's half (N real: lo + hi, (lo - hi) W^n)
    float* tbf = reinterpret_cast<float*>(tb);
    const float* tbf_other = reinterpret_cast<const float*>(tb_other);
#pragma unroll
    for (int i = 0; i < 32; i++) tbf[lane + 32 * i] = nl[i];
    pair_sync(row);
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const float o = tbf_other[lane + 32 * i];  // A: x[n + 1024], B: x[n]
        v[i] = half ? cmul(make_float2(o - nl[i], 0.f), comb_w<-1>(comb, lane + 32 * i))
                    : make_float2(nl[i] + o, 0.f);
    }
    pair_sync(row);  // both halves read before fft1024 reuses the buffers
    fft1024<-1>(v, tb, tw2, lane);  // X[2k + half]
    __syncthreads();  // every warp is done with the staging buffer
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int kx = 2 * (lane + 32 * i) + half;
        if (kx < G2::KC) buf[row * G2::KCP + kx] = v[i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < G2::KC * k2Rows; e += blockDim.x) {
        const int kx = e / k2Rows, yy = e - kx * k2Rows;
        r.H[(size_t)kx * k2N + y0 + yy] = buf[yy * G2::KCP + kx];
    }
}

// KD2: N-hat of the kept modes of columns kx0, kx0 + 1 (a warp pair each)
// from H (forward transform along y, by decimation in frequency: each warp
// reads both halves of its column), written to the row-major N-hat in
// 16-byte runs through a staging buffer (two columns a block: three blocks
// fit an SM, so the 342 blocks run in one wave).
constexpr int k2NhatCols = 2;
template <class Src>
__global__ void __launch_bounds__(2 * k2NhatCols * 32) k_fused_nhat2k(const __grid_constant__ Src src,
                                                                      const float2* __restrict__ tw) {
    const float2* __restrict__ H = src.h(blockIdx.y);
    float2* __restrict__ nhat = src.nhat_out(blockIdx.y);
    constexpr int nh = k2N / 2 + 1;
    extern __shared__ float2 sm[];
    float2* tw2 = sm;
    float2* comb = sm + 1024;
    float2* out = sm + 2048;  // [KR][k2NhatCols]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = warp >> 1, half = warp & 1;
    float2* tb = out + G2::KR * k2NhatCols + warp * kTB;
    load_twiddles2k<2 * k2NhatCols * 32>(tw2, comb, tw);
    __syncthreads();
    const int kx0 = blockIdx.x * k2NhatCols, kx = kx0 + c;
    if (kx < G2::KC) {  // whole warp pairs
        const float2* __restrict__ col = H + (size_t)kx * k2N;
        float2 lo[32], hi[32], v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) {
            lo[i] = col[lane + 32 * i];
            hi[i] = col[1024 + lane + 32 * i];
        }
        fft2048_dif<-1>(v, lo, hi, tb, tw2, comb, lane, half);
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int j = 2 * (lane + 32 * i) + half;
            if (row_kept_n<k2N>(j)) out[(j < G2::KC ? j : j - (k2N - G2::KR)) * k2NhatCols + c] = v[i];
        }
    }
    __syncthreads();
    const int ncols = min(k2NhatCols, G2::KC - kx0);
    for (int e = threadIdx.x; e < G2::KR * k2NhatCols; e += blockDim.x) {
        const int rr = e / k2NhatCols, cc = e - rr * k2NhatCols;
        if (cc < ncols) nhat[(size_t)kept_row_n<k2N>(rr) * nh + kx0 + cc] = out[e];
    }
}

constexpr size_t k2ColSmem = (size_t)(2048 + 2 * kTB) * sizeof(float2);
constexpr size_t k2RowSmem = (size_t)(2048 + 2 * k2Rows * G2::KCP + 2 * k2Rows * kTB) * sizeof(float2);
constexpr size_t k2NhatSmem = (size_t)(2048 + G2::KR * k2NhatCols + 2 * k2NhatCols * kTB) * sizeof(float2);

// ---- 256^2, 512^2 (any N = 32 M with M = 4, 8, 16): the same four stages on lane groups ----
// Each N = 32 M-point transform is held by a group of M lanes (fft_group), a
// warp holds 32 / M of them, a block four warps.

constexpr int kGWarps = 4;
template <int N>
struct GroupGeo {
    static constexpr int M = N / 32, GW = 32 / M, GB = kGWarps * GW;  // lanes a transform; transforms a warp, a block
    static constexpr int TB = 32 * (M + 1);                              // float2 in a group's transpose buffer
};

// KBg: the inverse transform along y of item t = (plane t / KC, column t % KC),
// one group each.  blockIdx.y: the flow.
template <int N, int P, class Src>
__global__ void __launch_bounds__(kGWarps * 32) k_fusedg_columns(const __grid_constant__ Src src,
                                                                 const float2* __restrict__ tw) {
    using Gm = Geo<N>;
    using Gg = GroupGeo<N>;
    constexpr int M = Gg::M;
    const float2* __restrict__ S = src.planes_s(blockIdx.y);
    float2* __restrict__ G = src.planes_g(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* twg = sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane / M, gl = lane % M;
    float2* tbg = sm + N + (warp * Gg::GW + gi) * Gg::TB;
    load_twiddles_group<M, kGWarps * 32>(twg, tw);
    __syncthreads();
    const int t = (blockIdx.x * kGWarps + warp) * Gg::GW + gi;
    const bool ok = t < P * Gm::KC;  // groups past the last item transform zeros
    const int p = ok ? t / Gm::KC : 0, kx = ok ? t - p * Gm::KC : 0;
    const size_t col = ((size_t)p * Gm::KCP + kx) * N;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int j = gl + M * i;
        v[i] = ok && row_kept_n<N>(j) ? S[col + j] : make_float2(0.f, 0.f);
    }
    fft_group<1, M>(v, tbg, twg, gl);
    if (ok) {
#pragma unroll
        for (int i = 0; i < 32; i++) G[col + gl + M * i] = v[i];
    }
}

// KCg's staging of one plane's x-spectrum (kept columns) of the block's R
// rows: buf[yy][kx] = G[p][kx][y0 + yy] (runs of R consecutive rows).
template <int N, int R>
__device__ __forceinline__ void stage_plane_g(float2* __restrict__ buf, const float2* __restrict__ G, int p,
                                              int y0) {
    using Gm = Geo<N>;
    constexpr int E = Gm::KC * R, NT = kGWarps * 32, passes = (E + NT - 1) / NT;
    float2 t[passes];
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < E) t[k] = G[((size_t)p * Gm::KCP + e / R) * N + y0 + e % R];
    }
#pragma unroll
    for (int k = 0; k < passes; k++) {
        const int e = threadIdx.x + k * NT;
        if (e < E) buf[(e % R) * Gm::KCP + e / R] = t[k];
    }
}

// This lane's elements k = gl + M i of the full complex spectrum of two real
// planes packed as a + i b (bufB = nullptr: b = 0), as row_pair.
template <int N>
__device__ __forceinline__ void row_pair_g(float2 (&v)[32], const float2* __restrict__ bufA,
                                           const float2* __restrict__ bufB, int gl) {
    using Gm = Geo<N>;
    constexpr int M = N / 32;
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int k = gl + M * i;
        float2 z = make_float2(0.f, 0.f);
        if (k < Gm::KC || k > N - Gm::KC) {
            const int kk = k < Gm::KC ? k : N - k;
            float2 A = bufA[kk];
            float2 B = bufB ? bufB[kk] : make_float2(0.f, 0.f);
            if (kk == 0) {
                A.y = 0.f;
                B.y = 0.f;
            }
            z = k < Gm::KC ? make_float2(A.x - B.y, A.y + B.x) : make_float2(A.x + B.y, B.x - A.y);
        }
        v[i] = z;
    }
}

// dst[x] = (src[x].z, src[x].w, new[x]) for this lane's nodes x = gl + M i
// of a row, in batches of 8 loads (as write_pair_row).
template <int M>
__device__ __forceinline__ void write_pair_group(const float4* __restrict__ src, float4* __restrict__ dst,
                                                 const float2 (&v)[32], int gl) {
#pragma unroll
    for (int b = 0; b < 4; b++) {
        float4 cur[8];
#pragma unroll
        for (int k = 0; k < 8; k++) cur[k] = src[gl + M * (8 * b + k)];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int i = 8 * b + k;
            dst[gl + M * i] = make_float4(cur[k].z, cur[k].w, v[i].x, v[i].y);
        }
    }
}

// KCg: the block's R rows, one group each (as KC).  blockIdx.y: the flow.
template <int N, int P, class Src>
__global__ void __launch_bounds__(kGWarps * 32) k_fusedg_rows(const __grid_constant__ Src src) {
    using Gm = Geo<N>;
    using Gg = GroupGeo<N>;
    constexpr int M = Gg::M, R = Gg::GB;
    const auto& r = src.rows(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* twg = sm;
    float2* buf = sm + N;  // 2 planes x R rows x KCP
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane / M, gl = lane % M;
    const int row = warp * Gg::GW + gi;
    float2* tbg = buf + 2 * R * Gm::KCP + row * Gg::TB;
    const float2* mine0 = buf + row * Gm::KCP;
    const float2* mine1 = buf + (R + row) * Gm::KCP;
    const int y0 = blockIdx.x * R, y = y0 + row;
    load_twiddles_group<M, kGWarps * 32>(twg, r.tw);
    stage_plane_g<N, R>(buf, r.G, 2, y0);
    stage_plane_g<N, R>(buf + R * Gm::KCP, r.G, 3, y0);
    __syncthreads();
    float2 v[32], hold[32];
    row_pair_g<N>(v, mine0, mine1, gl);  // wx + i wy
    fft_group<1, M>(v, tbg, twg, gl);
#pragma unroll
    for (int i = 0; i < 32; i++) hold[i] = v[i];
    __syncthreads();  // every group has read the staging buffer
    stage_plane_g<N, R>(buf, r.G, 0, y0);
    stage_plane_g<N, R>(buf + R * Gm::KCP, r.G, 1, y0);
    __syncthreads();
    row_pair_g<N>(v, mine0, mine1, gl);  // u + i v
    fft_group<1, M>(v, tbg, twg, gl);
    float nl[32];
#pragma unroll
    for (int i = 0; i < 32; i++) nl[i] = fmaf(v[i].x, hold[i].x, v[i].y * hold[i].y);  // Eq. 7
    if (P == 6 || P == 7) {  // the level pair holds the spline coefficients
        __syncthreads();
        stage_plane_g<N, R>(buf, r.G, 4, y0);
        stage_plane_g<N, R>(buf + R * Gm::KCP, r.G, 5, y0);
        __syncthreads();
        row_pair_g<N>(v, mine0, mine1, gl);
        fft_group<1, M>(v, tbg, twg, gl);
    }
    write_pair_group<M>(r.src + (size_t)y * N, r.dst + (size_t)y * N, v, gl);
    if (P == 5 || P == 7) {  // the streamfunction stencil field
        __syncthreads();
        stage_plane_g<N, R>(buf, r.G, r.psi_plane, y0);
        __syncthreads();
        row_pair_g<N>(v, mine0, nullptr, gl);
        fft_group<1, M>(v, tbg, twg, gl);
        const float2* __restrict__ ps = r.psi_src + (size_t)y * N;
        float2* __restrict__ pd = r.psi_dst + (size_t)y * N;
#pragma unroll
        for (int i = 0; i < 32; i++) pd[gl + M * i] = make_float2(ps[gl + M * i].y, v[i].x);
    }
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = make_float2(nl[i], 0.f);
    fft_group<-1, M>(v, tbg, twg, gl);
    __syncthreads();  // every group is done reading the staging buffer
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const int kx = gl + M * i;
        if (kx < Gm::KC) buf[row * Gm::KCP + kx] = v[i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Gm::KC * R; e += blockDim.x) {
        const int kx = e / R, yy = e - kx * R;
        r.H[(size_t)kx * N + y0 + yy] = buf[yy * Gm::KCP + kx];
    }
}

// KDg: N-hat of the kept modes of the block's columns (one group each) from
// H, written to the row-major N-hat in runs of the block's columns through a
// staging buffer.  blockIdx.y: the flow.
template <int N, class Src>
__global__ void __launch_bounds__(kGWarps * 32) k_fusedg_nhat(const __grid_constant__ Src src,
                                                              const float2* __restrict__ tw) {
    using Gm = Geo<N>;
    using Gg = GroupGeo<N>;
    constexpr int M = Gg::M, C = Gg::GB, nh = N / 2 + 1;
    const float2* __restrict__ H = src.h(blockIdx.y);
    float2* __restrict__ nhat = src.nhat_out(blockIdx.y);
    extern __shared__ float2 sm[];
    float2* twg = sm;
    float2* out = sm + N;  // [KR][C]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane / M, gl = lane % M;
    const int c = warp * Gg::GW + gi;
    float2* tbg = out + Gm::KR * C + c * Gg::TB;
    load_twiddles_group<M, kGWarps * 32>(twg, tw);
    __syncthreads();
    const int kx0 = blockIdx.x * C, kx = kx0 + c;
    const bool ok = kx < Gm::KC;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = ok ? H[(size_t)kx * N + gl + M * i] : make_float2(0.f, 0.f);
    fft_group<-1, M>(v, tbg, twg, gl);
    if (ok) {
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const int j = gl + M * i;
            if (row_kept_n<N>(j)) out[(j < Gm::KC ? j : j - (N - Gm::KR)) * C + c] = v[i];
        }
    }
    __syncthreads();
    const int ncols = min(C, Gm::KC - kx0);
    for (int e = threadIdx.x; e < Gm::KR * C; e += blockDim.x) {
        const int rr = e / C, cc = e - rr * C;
        if (cc < ncols) nhat[(size_t)kept_row_n<N>(rr) * nh + kx0 + cc] = out[e];
    }
}

template <int N>
constexpr size_t kgColSmem() { return (size_t)(N + GroupGeo<N>::GB * GroupGeo<N>::TB) * sizeof(float2); }
template <int N>
constexpr size_t kgRowSmem() {
    return (size_t)(N + 2 * GroupGeo<N>::GB * Geo<N>::KCP + GroupGeo<N>::GB * GroupGeo<N>::TB) * sizeof(float2);
}
template <int N>
constexpr size_t kgNhatSmem() {
    return (size_t)(N + Geo<N>::KR * GroupGeo<N>::GB + GroupGeo<N>::GB * GroupGeo<N>::TB) * sizeof(float2);
}

constexpr size_t kColSmem(int P) { return (size_t)(1024 + P * kTB) * sizeof(float2); }
constexpr size_t kRowSmem =
    (size_t)(1024 + 2 * kRowWarps * kRowPitch + kRowWarps * (kTB + 1024)) * sizeof(float2);
constexpr size_t kNhatSmem = (size_t)(1024 + kFKR * kNhatWarps + kNhatWarps * kTB) * sizeof(float2);

template <int N, int P, class Src>
cudaError_t allow_smem() {
    cudaError_t e;
    if constexpr (N <= 512) {
        e = cudaFuncSetAttribute(k_fusedg_columns<N, P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kgColSmem<N>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fusedg_rows<N, P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kgRowSmem<N>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fusedg_nhat<N, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kgNhatSmem<N>());
    } else if constexpr (N == 1024) {
        e = cudaFuncSetAttribute(k_fused_columns<P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kColSmem(P));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_rows<P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRowSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_nhat<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kNhatSmem);
    } else {
        e = cudaFuncSetAttribute(k_fused_columns2k<P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)k2ColSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_rows2k<P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)k2RowSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused_nhat2k<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)k2NhatSmem);
    }
    constexpr int cv = EL_SMEM_CARVEOUT_FLUID;
    if (e == cudaSuccess) e = set_carveout(k_fused_advance<N, P, Src>, cv);
    if constexpr (N <= 512) {
        if (e == cudaSuccess) e = set_carveout(k_fusedg_columns<N, P, Src>, cv);
        if (e == cudaSuccess) e = set_carveout(k_fusedg_rows<N, P, Src>, cv);
        if (e == cudaSuccess) e = set_carveout(k_fusedg_nhat<N, Src>, cv);
    } else if constexpr (N == 1024) {
        if (e == cudaSuccess) e = set_carveout(k_fused_columns<P, Src>, cv);
        if (e == cudaSuccess) e = set_carveout(k_fused_rows<P, Src>, cv);
        if (e == cudaSuccess) e = set_carveout(k_fused_nhat<Src>, cv);
    } else {
        if (e == cudaSuccess) e = set_carveout(k_fused_columns2k<P, Src>, cv);
        if (e == cudaSuccess) e = set_carveout(k_fused_rows2k<P, Src>, cv);
        if (e == cudaSuccess) e = set_carveout(k_fused_nhat2k<Src>, cv);
    }
    return e;
}

template <int N, class Src>
cudaError_t allow_smem_n(int planes) {
    switch (planes) {
        case 4: return allow_smem<N, 4, Src>();
        case 5: return allow_smem<N, 5, Src>();
        case 6: return allow_smem<N, 6, Src>();
        default: return allow_smem<N, 7, Src>();
    }
}

template <class Src>
cudaError_t allow_smem(int n, int planes) {
    switch (n) {
        case 256: return allow_smem_n<256, Src>(planes);
        case 512: return allow_smem_n<512, Src>(planes);
        case 1024: return allow_smem_n<1024, Src>(planes);
        default: return allow_smem_n<2048, Src>(planes);
    }
}

// The four kernels for `count` flows of N^2 and P planes (the grid's member slice).
template <int N, int P, class Src>
void launch(const Src& src, int count, const float2* tw, cudaStream_t st) {
    using Gm = Geo<N>;
    const dim3 tiles((Gm::KC + kTile - 1) / kTile, (Gm::KR + kTile - 1) / kTile, count);
    k_fused_advance<N, P, Src><<<tiles, 256, 0, st>>>(src);
    if constexpr (N <= 512) {
        using Gg = GroupGeo<N>;
        k_fusedg_columns<N, P, Src><<<dim3((P * Gm::KC + Gg::GB - 1) / Gg::GB, count), kGWarps * 32,
                                      kgColSmem<N>(), st>>>(src, tw);
        k_fusedg_rows<N, P, Src><<<dim3(N / Gg::GB, count), kGWarps * 32, kgRowSmem<N>(), st>>>(src);
        k_fusedg_nhat<N, Src><<<dim3((Gm::KC + Gg::GB - 1) / Gg::GB, count), kGWarps * 32, kgNhatSmem<N>(),
                                st>>>(src, tw);
    } else if constexpr (N == 1024) {
        k_fused_columns<P, Src><<<dim3(kFKC, count), P * 32, kColSmem(P), st>>>(src, tw);
        k_fused_rows<P, Src><<<dim3(kFN / kRowWarps, count), kRowWarps * 32, kRowSmem, st>>>(src);
        k_fused_nhat<Src><<<dim3((kFKC + kNhatWarps - 1) / kNhatWarps, count), kNhatWarps * 32, kNhatSmem,
                            st>>>(src, tw);
    } else {
        k_fused_columns2k<P, Src><<<dim3(G2::KC, count), 64, k2ColSmem, st>>>(src, tw);
        k_fused_rows2k<P, Src><<<dim3(k2N / k2Rows, count), k2Threads, k2RowSmem, st>>>(src);
        k_fused_nhat2k<Src><<<dim3((G2::KC + k2NhatCols - 1) / k2NhatCols, count), 2 * k2NhatCols * 32,
                              k2NhatSmem, st>>>(src, tw);
    }
}

template <int N, class Src>
void launch_n(int planes, const Src& src, int count, const float2* tw, cudaStream_t st) {
    switch (planes) {
        case 4: launch<N, 4>(src, count, tw, st); break;
        case 5: launch<N, 5>(src, count, tw, st); break;
        case 6: launch<N, 6>(src, count, tw, st); break;
        default: launch<N, 7>(src, count, tw, st); break;
    }
}

template <class Src>
void launch(int n, int planes, const Src& src, int count, const float2* tw, cudaStream_t st) {
    switch (n) {
        case 256: launch_n<256>(planes, src, count, tw, st); break;
        case 512: launch_n<512>(planes, src, count, tw, st); break;
        case 1024: launch_n<1024>(planes, src, count, tw, st); break;
        default: launch_n<2048>(planes, src, count, tw, st); break;
    }
}

}  // namespace

// Whether the flow's fluid step runs the kernels of this file: the 1024^2 and
// 2048^2 solvers (not the prescribed kinematic field; at 2048^2 without the
// streamfunction plane).  ELPATH_FLUID_CUFFT set
// in the environment keeps the cuFFT path (for comparing the two).
bool fused_fluid_supported(const el_flow* f) {
    static const bool off = std::getenv("ELPATH_FLUID_CUFFT") != nullptr;
    if (f->kinematic || off) return false;
    // Measured one flow at a time (fluid step, direct launches, ms, fused
    // against cuFFT): 128^2 0.034 / 0.028, 256^2 0.030 / 0.031, 512^2
    // 0.030 / 0.036, 2048^2 0.130 / 0.171; with the streamfunction plane (5
    // or 7 planes) the row kernels' extra sequential transform was slower
    // at 256^2 (0.042 / 0.033) and 2048^2 (0.223 / 0.203), even at 512^2.
    // Batched, 256^2 and 512^2 members gain too (64-member ensemble step
    // 0.895 against 0.990 ms).
    const bool plain = f->nplanes == 4 || f->nplanes == 6;
    return f->n == 1024 || ((f->n == 256 || f->n == 512 || f->n == 2048) && plain);
}

// Launch attributes (dynamic shared memory above 48 KiB), at flow creation,
// outside any stream capture.
el_status fused_fluid_prepare(el_flow* f) {
    const cudaError_t e = allow_smem<OneFlow>(f->n, f->nplanes);
    if (e != cudaSuccess) return fail(f, EL_ECUDA, "fused fluid step attributes: %s", cudaGetErrorString(e));
    return EL_OK;
}

// Fluid n -> n+1 for step number n = `step` (the new level m = step + 1).
el_status fluid_step_fused(el_flow* f, const SpecArgs& a, int64_t step) {
    const int64_t m = step + 1;
    // S (the planes before the column transforms) in the spectral planes'
    // buffer, G (after them) in the physical planes' buffer, H in the
    // nonlinear term's: none of them holds state between steps
    OneFlow o{};
    o.a = a;
    o.S = f->spec;
    o.G = reinterpret_cast<float2*>(f->phys);
    o.nhat = f->nhat;
    RowArgs& r = o.r;
    r.G = o.G;
    r.H = reinterpret_cast<float2*>(f->nl);
    r.tw = f->twiddle;
    r.src = f->snap[m % 2];        // pair (m-2, m-1): level m-1 in its second half
    r.dst = f->snap[(m + 1) % 2];  // pair (m-1, m)
    r.psi_src = f->psi_plane >= 0 ? f->psi[m % 2] : nullptr;
    r.psi_dst = f->psi_plane >= 0 ? f->psi[(m + 1) % 2] : nullptr;
    r.psi_plane = f->psi_plane;
    launch(f->n, f->nplanes, o, 1, f->twiddle, f->stream);
    f->launches += 4;
    EL_CUDA_OK(f, cudaGetLastError());
    return EL_OK;
}

// Launch attributes of the batched kernels for (n, planes), outside any capture.
cudaError_t fused_fluid_batch_prepare(int n, int planes) { return allow_smem<Members>(n, planes); }

cudaError_t fused_fluid_batch(cudaStream_t s, const FusedMember* d_members, int count, int n, int planes,
                              int ahead, const float2* twiddle) {
    if (count <= 0) return cudaSuccess;
    Members src{d_members, twiddle, ahead};
    launch(n, planes, src, count, twiddle, s);
    return cudaGetLastError();
}

}  // namespace el
