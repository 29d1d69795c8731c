// K8: FP64 sums in a fixed order.  A fixed grid of kRedBlocks x kRedThreads
// threads each sum a fixed strided subset, warps and blocks combine in a
// fixed tree, and one thread adds the block partials in index order: the
// same input always gives the same bits, whatever the device or the timing.
#include "common.cuh"

namespace el {
namespace {

__global__ void __launch_bounds__(kRedThreads) k_reduce2(const double2* __restrict__ in,
                                                         int64_t count,
                                                         double* __restrict__ partial) {
    double a = 0.0, b = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        double2 v = in[q];
        a += v.x;
        b += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    __shared__ double sa[kRedThreads / 32], sb[kRedThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kRedThreads / 32; w++) {
            ta += sa[w];
            tb += sb[w];
        }
        partial[2 * blockIdx.x] = ta;
        partial[2 * blockIdx.x + 1] = tb;
    }
}

// out = sums / count (means); one block of kRedThreads, fixed tree.
__global__ void __launch_bounds__(kRedThreads) k_reduce2_final(const double* __restrict__ partial,
                                                               int nblocks, int64_t count,
                                                               double* __restrict__ out) {
    __shared__ double sh[2][kRedThreads / 32];
    for (int c = 0; c < 2; c++) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) x += partial[2 * b + c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double x = 0.0;
        for (int w = 0; w < kRedThreads / 32; w++) x += sh[threadIdx.x][w];
        out[threadIdx.x] = count > 0 ? x / (double)count : 0.0;
    }
}

}  // namespace

el_status reduce_double2(el_flow* f, const double2* in, int64_t count, double* out2) {
    k_reduce2<<<kRedBlocks, kRedThreads, 0, f->stream>>>(in, count, f->red);
    EL_LAUNCHED(f);
    k_reduce2_final<<<1, kRedThreads, 0, f->stream>>>(f->red, kRedBlocks, count, out2);
    EL_LAUNCHED(f);
    return EL_OK;
}

}  // namespace el

namespace el {

// The same fixed-order reduction on a caller-chosen stream and partials
// buffer (kRedBlocks * 2 doubles); used where no flow exists.
cudaError_t launch_reduce_double2(cudaStream_t stream, const double2* in, int64_t count,
                                  double* partial, double* out2) {
    k_reduce2<<<kRedBlocks, kRedThreads, 0, stream>>>(in, count, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce2_final<<<1, kRedThreads, 0, stream>>>(partial, kRedBlocks, count, out2);
    return cudaGetLastError();
}

}  // namespace el
