// Allocation-free dispersion statistics.
//
// Some callers cannot allocate device memory when they need these numbers:
// a serving or simulation loop that must not stall (cudaMalloc and cudaFree
// can synchronise the whole device, so every stream in flight waits), or a
// host application whose device memory is all reserved up front by another
// allocator, where a fresh cudaMalloc fails.  el_dispersion_noalloc computes
// the same mean-square displacement and clustering index as the statistics of
// a flow, from positions the caller already holds on the device, with all of
// its scratch in one fixed device array of this library.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds its kNoAllocScratchBytes (about 4 MiB) until the process
// exits.  In host code the array's name is only a host-side handle, not a
// device address; the device address is looked up on every call with
// cudaGetSymbolAddress (in the current device's context, so a context made
// again after a cudaDeviceReset gets its own array's address; the lookup
// allocates nothing) and passed to the kernels.
// All calls share the array and it keeps the last call's contents: the box
// counters are cleared at the start of every call, the other parts are fully
// overwritten before they are read.  Calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on the array.
#include "common.cuh"

namespace el {

cudaError_t launch_reduce_double2(cudaStream_t stream, const double2* in, int64_t count,
                                  double* partial, double* out2);
cudaError_t launch_cluster_final(cudaStream_t stream, const unsigned long long* boxes,
                                 double* out);

namespace {

constexpr int64_t kNoAllocMaxParticles = EL_NOALLOC_MAX_PARTICLES;
constexpr size_t kTermsBytes = (size_t)kNoAllocMaxParticles * sizeof(double2);
constexpr size_t kPartialBytes = (size_t)kRedBlocks * 2 * sizeof(double);
constexpr size_t kBoxBytes = (size_t)kBoxes * kBoxes * sizeof(unsigned long long);
constexpr size_t kNoAllocScratchBytes = kTermsBytes + kPartialBytes + kBoxBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array in the current device's context.
cudaError_t scratch_address(void** out) {
    *out = nullptr;
    return cudaGetSymbolAddress(out, g_noalloc_scratch);
}

// Squared displacement per particle, unwrapped FP64 positions.
__global__ void k_disp_terms(const double2* __restrict__ xy, const double2* __restrict__ xy0,
                             int64_t np, double2* __restrict__ terms) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double dx = xy[p].x - xy0[p].x, dy = xy[p].y - xy0[p].y;
    terms[p] = make_double2(dx * dx, dy * dy);
}

// Box counts of the positions mapped periodically onto [0, 2 pi)^2.
__global__ void k_disp_boxes(const double2* __restrict__ xy, int64_t np,
                             unsigned long long* __restrict__ boxes) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double inv = 1.0 / kTwoPi;
    double x = xy[p].x, y = xy[p].y;
    double xw = x - kTwoPi * floor(x * inv), yw = y - kTwoPi * floor(y * inv);
    int bx = (int)(xw * (kBoxes * inv)), by = (int)(yw * (kBoxes * inv));
    bx = bx < 0 ? 0 : (bx > kBoxes - 1 ? kBoxes - 1 : bx);
    by = by < 0 ? 0 : (by > kBoxes - 1 ? kBoxes - 1 : by);
    atomicAdd(boxes + by * kBoxes + bx, 1ull);
}

el_status noalloc_fail(el_status s, const char* what, cudaError_t e) {
    return fail(nullptr, s, "el_dispersion_noalloc: %s: %s", what, cudaGetErrorString(e));
}

}  // namespace
}  // namespace el

using namespace el;

extern "C" el_status el_dispersion_noalloc(const double* d_xy, const double* d_xy0, int64_t np,
                                           double* d_out3, void* cuda_stream) {
    if (np < 0 || np > kNoAllocMaxParticles)
        return fail(nullptr, EL_EINVAL,
                    "el_dispersion_noalloc: np = %lld outside [0, %lld] (the fixed scratch holds "
                    "%lld particles)",
                    (long long)np, (long long)kNoAllocMaxParticles, (long long)kNoAllocMaxParticles);
    if (!d_out3 || (np > 0 && (!d_xy || !d_xy0)))
        return fail(nullptr, EL_EINVAL, "el_dispersion_noalloc: NULL array");
    // the kernels read positions as (x, y) pairs of 16 bytes and store doubles
    if (np > 0 && (((uintptr_t)d_xy | (uintptr_t)d_xy0) & 15u))
        return fail(nullptr, EL_EINVAL, "el_dispersion_noalloc: d_xy and d_xy0 must be 16-byte aligned");
    if ((uintptr_t)d_out3 & 7u)
        return fail(nullptr, EL_EINVAL, "el_dispersion_noalloc: d_out3 must be 8-byte aligned");
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return noalloc_fail(EL_ECUDA, "scratch address", e);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    char* b = (char*)base;
    double2* terms = (double2*)b;
    double* partial = (double*)(b + kTermsBytes);
    unsigned long long* boxes = (unsigned long long*)(b + kTermsBytes + kPartialBytes);
    e = cudaMemsetAsync(boxes, 0, kBoxBytes, s);
    if (e != cudaSuccess) return noalloc_fail(EL_ECUDA, "clear box counters", e);
    const int T = 256;
    if (np > 0) {
        k_disp_terms<<<blocks_for(np, T), T, 0, s>>>((const double2*)d_xy, (const double2*)d_xy0,
                                                     np, terms);
        k_disp_boxes<<<blocks_for(np, T), T, 0, s>>>((const double2*)d_xy, np, boxes);
        e = cudaGetLastError();
        if (e != cudaSuccess) return noalloc_fail(EL_ECUDA, "launch", e);
    }
    e = launch_reduce_double2(s, terms, np, partial, d_out3);
    if (e != cudaSuccess) return noalloc_fail(EL_ECUDA, "reduction", e);
    e = launch_cluster_final(s, boxes, d_out3 + 2);
    if (e != cudaSuccess) return noalloc_fail(EL_ECUDA, "clustering index", e);
    return EL_OK;
}
