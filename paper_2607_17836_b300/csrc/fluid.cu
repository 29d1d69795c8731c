// Pseudospectral vorticity solver (Sec. 3.1).  One step is two launches of
// the fused passes in fft.cuh:
//
//   k_column : forward FFT along y of the x-transformed N -> N-hat (Eq. 8),
//              2/3 rule + AB2 update of omega-hat (Eqs. 9, 10), the velocity,
//              gradient, spline and streamfunction planes (Eqs. 4-6) and
//              their inverse FFT along y
//   k_row    : inverse real FFT along x of the planes, N = u wx + v wy
//              (Eq. 7), the level pair the particle step reads, forward real
//              FFT along x of N
//
// omega-hat, its low part and the AB2 history are stored column-major,
// [kx][j] with kx = 0..n/2 and ky = j for j < n/2, j - n otherwise, so the
// column pass reads and writes them in whole columns.  The planes and the
// x-transformed N live in row space, [y][kx] with a row pitch that is a
// multiple of 4 (one 32-byte sector per row of a 4-column tile).
//
// cuFFT serves only the set-up (the initial field into Fourier space) and
// the on-demand readback of physical fields (el_get_field).
#include "common.cuh"
#include "fft.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace el {
namespace {

constexpr int kProjThreads = 128;

template <int REM>
__global__ void __launch_bounds__(256) k_column(const __grid_constant__ ColArgs a, int first,
                                                int advance) {
    extern __shared__ float2 sm[];
    column_tile<REM>(a, first, advance, blockIdx.x, sm);
}

template <int REM>
__global__ void __launch_bounds__(512) k_row(const __grid_constant__ RowArgs a, const RowLevel lv) {
    extern __shared__ float2 sm[];
    row_pass<REM>(a, lv, blockIdx.x, sm);
}

using ColumnKernel = void (*)(ColArgs, int, int);
using RowKernel = void (*)(RowArgs, RowLevel);
const ColumnKernel kColumn[4] = {k_column<0>, k_column<1>, k_column<2>, k_column<3>};
const RowKernel kRow[4] = {k_row<0>, k_row<1>, k_row<2>, k_row<3>};

// Initial projection: mean removed, 2/3 rule (Sec. 3.1); row-major cuFFT
// output [j][kx] -> column-major omega-hat [kx][j].
__global__ void k_project(const float2* __restrict__ src, float2* __restrict__ what, int n, int nh) {
    const int i = blockIdx.x * kProjThreads + threadIdx.x, j = blockIdx.y;
    if (i >= nh) return;
    const int ky = wavenumber_row(j, n), kx = i;
    const bool keep = kept(kx, ky, n) && !(kx == 0 && ky == 0);
    what[(size_t)kx * n + j] = keep ? src[(size_t)j * nh + i] : make_float2(0.f, 0.f);
}

// One plane (or, for p < 0, omega-hat / n^2) of the current level as a
// row-major half spectrum for cuFFT's C2R.
__global__ void k_plane_rowmajor(const __grid_constant__ ColArgs a, int p, float2* __restrict__ dst) {
    const int i = blockIdx.x * kProjThreads + threadIdx.x, j = blockIdx.y;
    const int n = a.n, nh = n / 2 + 1;
    if (i >= nh) return;
    float2 v = make_float2(0.f, 0.f);
    if (i < n / 2) {
        const float2 w = a.what[(size_t)i * n + j];
        const float2 ws = make_float2(w.x * a.scale, w.y * a.scale);
        v = p < 0 ? ws : plane_value(a, p, ws, i, j);
    }
    dst[(size_t)j * nh + i] = v;
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

// FP64 partial sums over the half spectrum for E, Z, P (Parseval).  Modes
// with 0 < kx < n/2 stand for themselves and their conjugates (weight 2).
__global__ void __launch_bounds__(kRedThreads) k_spec_diag(const float2* __restrict__ what, int n,
                                                           size_t nmodes, double* __restrict__ partial) {
    double se = 0.0, sz = 0.0, sp = 0.0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nmodes;
         q += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(q / n), j = (int)(q - (size_t)kx * n);
        const int ky = wavenumber_row(j, n);
        double k2 = (double)kx * kx + (double)ky * ky;
        double wgt = (kx == 0 || kx == n / 2) ? 1.0 : 2.0;
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

ColArgs column_args(const el_flow* f) {
    ColArgs a{};
    a.what = f->what;
    a.what_lo = f->what_lo;
    a.hist = f->hist;
    a.nrow = f->nrow;
    a.planes = f->planes;
    a.ex = f->ex;
    a.ey = f->ey;
    a.pre_x = f->pre_x;
    a.pre_y = f->pre_y;
    a.tw = f->tw_col;
    a.pstride = (size_t)f->n * f->pitch;
    a.n = f->n;
    a.log2n = f->log2n;
    a.pitch = f->pitch;
    a.nplanes = f->nplanes;
    a.log2tc = f->log2tc;
    a.mode = f->d.ab2_mode;
    a.spline = f->stencil_plane != 0;
    a.psi_plane = f->psi_plane;
    a.scale = 1.0f / (float)f->n2;
    a.dt = (float)f->d.dt;
    a.nu = (float)f->d.nu;
    return a;
}

RowArgs row_args(const el_flow* f) {
    RowArgs r{};
    r.planes = f->planes;
    r.nrow = f->nrow;
    r.tw = f->tw_row;
    r.wn = f->wn;
    r.pstride = (size_t)f->n * f->pitch;
    r.n = f->n;
    r.log2n = f->log2n;
    r.pitch = f->pitch;
    r.nplanes = f->nplanes;
    r.stencil_plane = f->stencil_plane;
    r.psi_plane = f->psi_plane;
    return r;
}

// Level m is written into pair (m-1, m) = snap[(m + 1) % 2].
RowLevel row_level(const el_flow* f, int64_t m, bool setup) {
    RowLevel l{};
    l.snap_dst = f->snap[(m + 1) % 2];
    l.snap_src = setup ? nullptr : f->snap[m % 2];
    l.snap_other = setup ? f->snap[m % 2] : nullptr;
    l.psi_dst = f->psi[(m + 1) % 2];
    l.psi_src = setup ? nullptr : f->psi[m % 2];
    l.psi_other = setup ? f->psi[m % 2] : nullptr;
    l.setup = setup ? 1 : 0;
    return l;
}

size_t max_col_smem_bytes() {
    size_t m = 0;
    for (int l = 4; l <= 12; l++) m = std::max(m, col_smem_bytes(l, col_log2tc(1 << l)));
    return m;
}

size_t max_row_smem_bytes() { return row_smem_bytes(12, kMaxPlanes); }

el_status fluid_kernel_setup(el_flow* f) {
    for (int r = 0; r < 4; r++) {
        EL_CUDA_OK(f, cudaFuncSetAttribute(kRow[r], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)max_row_smem_bytes()));
        EL_CUDA_OK(f, cudaFuncSetAttribute(kColumn[r], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)max_col_smem_bytes()));
    }
    return EL_OK;
}

// Column pass then row pass producing level m.
static el_status launch_passes(el_flow* f, int first, int advance, int64_t m, bool setup) {
    kColumn[f->log2n & 3]<<<col_tiles(f->n, f->log2tc), col_threads(f->n, f->log2tc),
                            col_smem_bytes(f->log2n, f->log2tc), f->stream>>>(column_args(f), first,
                                                                               advance);
    EL_LAUNCHED(f);
    kRow[(f->log2n - 1) & 3]<<<f->n, row_threads(f->n, f->nplanes),
                               row_smem_bytes(f->log2n, f->nplanes), f->stream>>>(
        row_args(f), row_level(f, m, setup));
    EL_LAUNCHED(f);
    return EL_OK;
}

static el_status fft_exec_c2r(el_flow* f, float2* in, float* out) {
    cufftResult r = cufftExecC2R(f->plan_c2r1, reinterpret_cast<cufftComplex*>(in), out);
    if (r != CUFFT_SUCCESS) return fail(f, EL_ECUFFT, "cufftExecC2R failed (%d)", (int)r);
    return EL_OK;
}

el_status fluid_init(el_flow* f, const double* omega0_host) {
    const int T = 256;
    EL_CUDA_OK(f, cudaMemcpyAsync(f->stage64, omega0_host, f->n2 * sizeof(double),
                                  cudaMemcpyHostToDevice, f->stream));
    k_d2f<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(f->stage64, f->aux_phys, f->n2);
    EL_LAUNCHED(f);
    cufftResult cr = cufftExecR2C(f->plan_r2c, f->aux_phys, reinterpret_cast<cufftComplex*>(f->aux_spec));
    if (cr != CUFFT_SUCCESS) return fail(f, EL_ECUFFT, "cufftExecR2C failed (%d)", (int)cr);
    k_project<<<dim3((unsigned)((f->nh + kProjThreads - 1) / kProjThreads), (unsigned)f->n),
                kProjThreads, 0, f->stream>>>(f->aux_spec, f->what, f->n, f->nh);
    EL_LAUNCHED(f);
    EL_CUDA_OK(f, cudaMemsetAsync(f->hist, 0, f->nmodes * sizeof(float2), f->stream));
    EL_CUDA_OK(f, cudaMemsetAsync(f->what_lo, 0, f->nmodes * sizeof(float2), f->stream));
    // the planes' Nyquist column (and the row padding) stays zero from here on
    EL_CUDA_OK(f, cudaMemsetAsync(f->planes, 0,
                                  (size_t)f->nplanes * f->n * f->pitch * sizeof(float2), f->stream));
    EL_TRY(fluid_kernel_setup(f));
    return launch_passes(f, 0, 0, 0, true);
}

// Fluid n -> n+1 for step number n = `step`.
el_status fluid_step(el_flow* f, int64_t step) {
    return launch_passes(f, step == 0, 1, step + 1, false);
}

el_status fluid_diagnostics(el_flow* f) {
    k_spec_diag<<<kRedBlocks, kRedThreads, 0, f->stream>>>(f->what, f->n, f->nmodes, f->red);
    EL_LAUNCHED(f);
    double nn = (double)f->n2;
    k_spec_diag_final<<<1, kRedThreads, 0, f->stream>>>(f->red, kRedBlocks, 0.5 / (nn * nn),
                                                        f->red_out);
    EL_LAUNCHED(f);
    return EL_OK;
}

el_status fluid_get_field(el_flow* f, int which, double* host_nn) {
    const int T = 256;
    double* out = f->stage64;
    if (which <= 2) {
        // 0: omega, 1: u, 2: v of the current level, from omega-hat
        k_plane_rowmajor<<<dim3((unsigned)((f->nh + kProjThreads - 1) / kProjThreads), (unsigned)f->n),
                           kProjThreads, 0, f->stream>>>(column_args(f), which - 1, f->aux_spec);
        EL_LAUNCHED(f);
        EL_TRY(fft_exec_c2r(f, f->aux_spec, f->aux_phys));
        k_f2d<<<blocks_for((int64_t)f->n2, T), T, 0, f->stream>>>(f->aux_phys, out, f->n2, 1, 0);
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

void fft_twiddles(int log2l, std::vector<float2>& out) {
    out.clear();
    const FftSchedule s = fft_schedule(log2l);
    int64_t ns = 1;
    for (int p = 0; p < s.npass; p++) {
        const int64_t R = (int64_t)1 << s.log2r[p];
        if (p > 0)
            for (int64_t r = 1; r < R; r++)
                for (int64_t q = 0; q < ns; q++) {
                    const double ang = -kTwoPi * (double)(q * r) / (double)(ns * R);
                    out.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
                }
        ns *= R;
    }
}

// Host-side FP64 tables: the 1-D integrating factors exp(-nu k^2 dt) as
// float pairs (hi, lo), the spline prefilter factors 3 / (2 + cos k dx), the
// FFT twiddles of the column (length n) and row (length n/2) transforms and
// exp(-2 pi i k / n), k = 0..n/2, of the real-transform split.
void fluid_tables(const el_flow_desc& d, FluidTables& t) {
    int n = d.n, nh = n / 2 + 1, log2n = 0;
    while ((1 << log2n) < n) log2n++;
    t.ex.resize(nh);
    t.px.resize(nh);
    t.ey.resize(n);
    t.py.resize(n);
    double dxg = kTwoPi / n;
    auto pair = [](double v) {
        float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    for (int i = 0; i < nh; i++) {
        double k = i;
        t.ex[i] = pair(std::exp(-d.nu * k * k * d.dt));
        t.px[i] = (float)(3.0 / (2.0 + std::cos(k * dxg)));
    }
    for (int j = 0; j < n; j++) {
        double k = j < n / 2 ? j : j - n;
        t.ey[j] = pair(std::exp(-d.nu * k * k * d.dt));
        t.py[j] = (float)(3.0 / (2.0 + std::cos(k * dxg)));
    }
    fft_twiddles(log2n, t.tw_col);
    fft_twiddles(log2n - 1, t.tw_row);
    t.wn.resize(nh);
    for (int k = 0; k < nh; k++) {
        const double ang = -kTwoPi * k / n;
        t.wn[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
}

}  // namespace el
