// Level-1/2 kernels of the GMRES on the Schur system (FP64, face vectors).
//
// Reductions are deterministic: every block writes one partial per column in
// a fixed order (warp shuffles, then shared memory), and a second kernel sums
// the partials of each column in block order.
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

constexpr int kDotThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial[b * ncols + c] = sum_{i in block b's rows} V[c * ld + i] * w[i]
__global__ void __launch_bounds__(kDotThreads) k_mdot(const double* __restrict__ V, int64_t ld, int ncols,
                                                      const double* __restrict__ w, int64_t n,
                                                      double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int c = 0; c < ncols; ++c) {
    const double* v = V + (int64_t)c * ld;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc = fma(v[i], w[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = threadIdx.x < (kDotThreads / 32) ? red[threadIdx.x] : 0.0;
      s = warp_sum(s);
      if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * ncols + c] = s;
    }
    __syncthreads();
  }
}

__global__ void k_reduce_cols(const double* __restrict__ partial, int nblocks, int ncols, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * ncols + c];
  out[c] = s;
}

__global__ void k_gemv_sub(const double* __restrict__ V, int64_t ld, int ncols, const double* __restrict__ h,
                           double* __restrict__ w, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = w[i];
  for (int c = 0; c < ncols; ++c) acc = fma(-V[(int64_t)c * ld + i], h[c], acc);
  w[i] = acc;
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

cudaError_t launch_mdot(const double* V, int64_t ld, int ncols, const double* w, int64_t n, double* partial,
                        int nblocks, cudaStream_t st) {
  k_mdot<<<nblocks, kDotThreads, 0, st>>>(V, ld, ncols, w, n, partial);
  return cudaGetLastError();
}
cudaError_t launch_reduce_cols(const double* partial, int nblocks, int ncols, double* out, cudaStream_t st) {
  k_reduce_cols<<<(ncols + 127) / 128, 128, 0, st>>>(partial, nblocks, ncols, out);
  return cudaGetLastError();
}
cudaError_t launch_gemv_sub(const double* V, int64_t ld, int ncols, const double* h, double* w, int64_t n,
                            cudaStream_t st) {
  k_gemv_sub<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, ld, ncols, h, w, n);
  return cudaGetLastError();
}
cudaError_t launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st) {
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, x, a, b, n);
  return cudaGetLastError();
}

}  // namespace ahoc
