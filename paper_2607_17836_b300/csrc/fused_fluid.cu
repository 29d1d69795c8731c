// The pseudospectral step (Sec. 3.1, Eqs. 4-10) on a 1024^2 grid as four
// kernels of our own instead of the pointwise kernels around cuFFT's 2-D
// transforms, for one flow or for every 1024^2 member of a batch at once
// (the member in the grid's last dimension; OneFlow / Members below).  Only the modes the 2/3 rule keeps are ever nonzero (the
// initial field is projected, N-hat is masked every step), so every
// transform is pruned to them: 342 of the 513 columns kx, 683 of the 1024
// rows ky.
//
//   k_fused_advance<P> : the AB2 update of the kept modes (advance_mode) in
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
template <int P, class Src>
__global__ void __launch_bounds__(256) k_fused_advance(const __grid_constant__ Src src) {
    const auto& a = src.spec(blockIdx.z);
    float2* __restrict__ S = src.planes_s(blockIdx.z);
    __shared__ float2 tile[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int kx0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
    const int kx = kx0 + tx;
    ModeIn in[kTile / 8];
#pragma unroll
    for (int m = 0; m < kTile / 8; m++) {  // every load first
        const int r = r0 + ty + 8 * m, j = kept_row(r);
        if (r < kFKR && kx < kFKC) in[m] = load_mode(a, kx, j, (size_t)j * a.nh + kx);
    }
#pragma unroll
    for (int m = 0; m < kTile / 8; m++) {
        const int r = r0 + ty + 8 * m, j = kept_row(r);
        float2 w = make_float2(0.f, 0.f);
        if (r < kFKR && kx < kFKC) w = advance_loaded(a, kx, j, (size_t)j * a.nh + kx, in[m]);
        tile[ty + 8 * m][tx] = w;
    }
    __syncthreads();
    const int r = r0 + tx;
    if (r >= kFKR) return;  // no barrier follows
    const int j = kept_row(r);
#pragma unroll
    for (int m = 0; m < kTile / 8; m++) {
        const int kx = kx0 + ty + 8 * m;
        if (kx >= kFKC) break;
        const float2 w = tile[tx][ty + 8 * m];
#pragma unroll
        for (int p = 0; p < P; p++) S[((size_t)p * kFKCP + kx) * kFN + j] = plane_value(a, p, kx, j, w);
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

constexpr size_t kColSmem(int P) { return (size_t)(1024 + P * kTB) * sizeof(float2); }
constexpr size_t kRowSmem =
    (size_t)(1024 + 2 * kRowWarps * kRowPitch + kRowWarps * (kTB + 1024)) * sizeof(float2);
constexpr size_t kNhatSmem = (size_t)(1024 + kFKR * kNhatWarps + kNhatWarps * kTB) * sizeof(float2);

template <int P, class Src>
cudaError_t allow_smem() {
    cudaError_t e = cudaFuncSetAttribute(k_fused_columns<P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kColSmem(P));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused_rows<P, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRowSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused_nhat<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kNhatSmem);
    return e;
}

template <class Src>
cudaError_t allow_smem(int planes) {
    switch (planes) {
        case 4: return allow_smem<4, Src>();
        case 5: return allow_smem<5, Src>();
        case 6: return allow_smem<6, Src>();
        default: return allow_smem<7, Src>();
    }
}

// The four kernels for `count` flows of P planes (the grid's member slice).
template <int P, class Src>
void launch(const Src& src, int count, const float2* tw, cudaStream_t st) {
    const dim3 tiles((kFKC + kTile - 1) / kTile, (kFKR + kTile - 1) / kTile, count);
    k_fused_advance<P, Src><<<tiles, 256, 0, st>>>(src);
    k_fused_columns<P, Src><<<dim3(kFKC, count), P * 32, kColSmem(P), st>>>(src, tw);
    k_fused_rows<P, Src><<<dim3(kFN / kRowWarps, count), kRowWarps * 32, kRowSmem, st>>>(src);
    k_fused_nhat<Src><<<dim3((kFKC + kNhatWarps - 1) / kNhatWarps, count), kNhatWarps * 32, kNhatSmem, st>>>(
        src, tw);
}

template <class Src>
void launch(int planes, const Src& src, int count, const float2* tw, cudaStream_t st) {
    switch (planes) {
        case 4: launch<4>(src, count, tw, st); break;
        case 5: launch<5>(src, count, tw, st); break;
        case 6: launch<6>(src, count, tw, st); break;
        default: launch<7>(src, count, tw, st); break;
    }
}

}  // namespace

// Whether the flow's fluid step runs the kernels of this file: the 1024^2
// solver (not the prescribed kinematic field).  ELPATH_FLUID_CUFFT set in the
// environment keeps the cuFFT path (for comparing the two).
bool fused_fluid_supported(const el_flow* f) {
    static const bool off = std::getenv("ELPATH_FLUID_CUFFT") != nullptr;
    return f->n == kFN && !f->kinematic && !off;
}

// Launch attributes (dynamic shared memory above 48 KiB), at flow creation,
// outside any stream capture.
el_status fused_fluid_prepare(el_flow* f) {
    const cudaError_t e = allow_smem<OneFlow>(f->nplanes);
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
    launch(f->nplanes, o, 1, f->twiddle, f->stream);
    f->launches += 4;
    EL_CUDA_OK(f, cudaGetLastError());
    return EL_OK;
}

// Launch attributes of the batched kernels for `planes`, outside any capture.
cudaError_t fused_fluid_batch_prepare(int planes) { return allow_smem<Members>(planes); }

cudaError_t fused_fluid_batch(cudaStream_t s, const FusedMember* d_members, int count, int planes,
                              int ahead, const float2* twiddle) {
    if (count <= 0) return cudaSuccess;
    Members src{d_members, twiddle, ahead};
    launch(planes, src, count, twiddle, s);
    return cudaGetLastError();
}

}  // namespace el
