// Level-1/2 kernels of the GMRES on the Schur system (FP64, face vectors).
//
// Reductions are deterministic: every block writes one partial per column in
// a fixed order (warp shuffles, then shared memory), and a second kernel sums
// the partials of each column in block order.  A batch of problems runs in
// one launch (the problem on the last grid dimension, each problem's vectors
// at its own stride); the block split depends on the vector length only, so
// a problem's sums are the same bits alone and in a batch.
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

constexpr int kDotThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial[b * ncols + c] = sum over block-row b's rows of V[c * ld + i] * w[i];
// blockIdx.y selects a group of kCols columns, so one pass over the rows
// serves kCols dot products with one shared-memory reduction.
constexpr int kCols = 4;

__global__ void __launch_bounds__(kDotThreads) k_mdot(const double* __restrict__ V, int64_t ld, int ncols,
                                                      const double* __restrict__ w, int64_t n,
                                                      double* __restrict__ partial, BatchDot bd) {
  const int bi = blockIdx.z;
  if (bd.act && !bd.act[bi]) return;
  V += (int64_t)bi * bd.vstride;
  w += (int64_t)bi * bd.wstride;
  partial += (int64_t)bi * bd.pstride;
  __shared__ double red[kCols][kDotThreads / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  const int c0 = blockIdx.y * kCols;
  const int nc = (ncols - c0) < kCols ? (ncols - c0) : kCols;
  double acc[kCols] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int q = 0; q < kCols; ++q)
      if (q < nc) acc[q] = fma(V[(int64_t)(c0 + q) * ld + i], wi, acc[q]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kCols; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < kCols; ++q) {
      double v = threadIdx.x < (kDotThreads / 32) ? red[q][threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0 && q < nc) partial[(int64_t)blockIdx.x * ncols + c0 + q] = v;
    }
  }
}

// out[c] = sum_b partial[b * ncols + c]: one warp per column, fixed order
__global__ void k_reduce_cols(const double* __restrict__ partial, int nblocks, int ncols, double* __restrict__ out,
                              int64_t pstride, int64_t ostride, const int* act) {
  if (act && !act[blockIdx.y]) return;
  partial += (int64_t)blockIdx.y * pstride;
  out += (int64_t)blockIdx.y * ostride;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(int64_t)b * ncols + c];
  s = warp_sum(s);
  if (lane == 0) out[c] = s;
}

// Fused CGS pass: dst = src - V h (h: nh columns; no update when h is NULL,
// dst then unused), then the partial dots of the updated vector with V's
// columns c (self: with itself), and the last block of each column group
// sums the partials in block order into out -- the same arithmetic and
// order as k_gemv_sub, k_mdot and k_reduce_cols, so the bits are theirs.
// Every block of a column group computes the update of its rows (reading
// src only); the blocks of group 0 write it.  cnt: one zeroed counter per
// (problem, column group); the last block resets it.
__global__ void __launch_bounds__(kDotThreads) k_cgs(const double* __restrict__ V, int64_t ld, int ncols,
                                                     const double* __restrict__ h, int nh,
                                                     const double* __restrict__ src, double* __restrict__ dst,
                                                     int64_t n, double* __restrict__ partial,
                                                     double* __restrict__ out, BatchDot bd, int64_t hstride,
                                                     int64_t ostride, int* __restrict__ cnt, int self) {
  const int bi = blockIdx.z;
  if (bd.act && !bd.act[bi]) return;
  V += (int64_t)bi * bd.vstride;
  src += (int64_t)bi * bd.wstride;
  if (dst) dst += (int64_t)bi * bd.wstride;
  partial += (int64_t)bi * bd.pstride;
  out += (int64_t)bi * ostride;
  if (h) h += (int64_t)bi * hstride;
  cnt += (int64_t)bi * gridDim.y + blockIdx.y;
  __shared__ double red[kCols][kDotThreads / 32];
  __shared__ int last;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  const int c0 = blockIdx.y * kCols;
  const int nc = (ncols - c0) < kCols ? (ncols - c0) : kCols;
  double acc[kCols] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double wi = src[i];
    if (h) {
      for (int c = 0; c < nh; ++c) wi = fma(-V[(int64_t)c * ld + i], h[c], wi);
      if (blockIdx.y == 0) dst[i] = wi;
    }
#pragma unroll
    for (int q = 0; q < kCols; ++q)
      if (q < nc) acc[q] = fma(self ? wi : V[(int64_t)(c0 + q) * ld + i], wi, acc[q]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kCols; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < kCols; ++q) {
      double v = threadIdx.x < (kDotThreads / 32) ? red[q][threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0 && q < nc) partial[(int64_t)blockIdx.x * ncols + c0 + q] = v;
    }
  }
  // the last block of this column group reduces its columns
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(cnt, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (warp < nc) {
    const int c = c0 + warp;
    double sacc = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) sacc += __ldcg(partial + (int64_t)b * ncols + c);
    sacc = warp_sum(sacc);
    if (lane == 0) out[c] = sacc;
  }
  if (threadIdx.x == 0) *cnt = 0;
}

__global__ void k_gemv_sub(const double* __restrict__ V, int64_t ld, int ncols, const double* __restrict__ h,
                           double* __restrict__ w, int64_t n, BatchDot bd, int64_t hstride, const int* ncols_b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (i >= n || (bd.act && !bd.act[bi])) return;
  if (ncols_b) ncols = ncols_b[bi];
  V += (int64_t)bi * bd.vstride;
  w += (int64_t)bi * bd.wstride;
  h += (int64_t)bi * hstride;
  double acc = w[i];
  for (int c = 0; c < ncols; ++c) acc = fma(-V[(int64_t)c * ld + i], h[c], acc);
  w[i] = acc;
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, int64_t n,
                        const double* __restrict__ a_b, const int* act, int64_t ystride, int64_t xstride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (i >= n || (act && !act[bi])) return;
  if (a_b) a = a_b[bi];
  y += (int64_t)bi * ystride;
  x += (int64_t)bi * xstride;
  y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

// out[c] = <V_c, w> for c < ncols: block partials into `partial` (capacity
// nblocks * ncols), then a fixed-order reduction per column into out
cudaError_t launch_mdot(const double* V, int64_t ld, int ncols, const double* w, int64_t n, double* partial,
                        int nblocks, double* out, cudaStream_t st, int nbat, const BatchDot& bd, int64_t ostride) {
  const int64_t want = (n + 4095) / 4096;
  const int nb = (int)(want < 1 ? 1 : (want > nblocks ? nblocks : want));
  dim3 grid(nb, (ncols + kCols - 1) / kCols, nbat);
  k_mdot<<<grid, kDotThreads, 0, st>>>(V, ld, ncols, w, n, partial, bd);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_cols<<<dim3((ncols + 7) / 8, nbat), 256, 0, st>>>(partial, nb, ncols, out, bd.pstride, ostride, bd.act);
  return cudaGetLastError();
}
cudaError_t launch_cgs(const double* V, int64_t ld, int ncols, const double* h, int nh, const double* src,
                       double* dst, int64_t n, double* partial, int nblocks, double* out, cudaStream_t st, int nbat,
                       const BatchDot& bd, int64_t hstride, int64_t ostride, int* cnt, bool self) {
  const int64_t want = (n + 4095) / 4096;
  const int nb = (int)(want < 1 ? 1 : (want > nblocks ? nblocks : want));
  dim3 grid(nb, self ? 1 : (ncols + kCols - 1) / kCols, nbat);
  k_cgs<<<grid, kDotThreads, 0, st>>>(V, ld, self ? 1 : ncols, h, nh, src, dst, n, partial, out, bd, hstride, ostride,
                                     cnt, self ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_reduce_cols(const double* partial, int nblocks, int ncols, double* out, cudaStream_t st) {
  k_reduce_cols<<<(ncols + 7) / 8, 256, 0, st>>>(partial, nblocks, ncols, out, 0, 0, nullptr);
  return cudaGetLastError();
}
cudaError_t launch_gemv_sub(const double* V, int64_t ld, int ncols, const double* h, double* w, int64_t n,
                            cudaStream_t st, int nbat, const BatchDot& bd, int64_t hstride, const int* ncols_b) {
  k_gemv_sub<<<dim3((unsigned)((n + 255) / 256), nbat), 256, 0, st>>>(V, ld, ncols, h, w, n, bd, hstride, ncols_b);
  return cudaGetLastError();
}
cudaError_t launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st, int nbat,
                         const double* a_b, const int* act, int64_t ystride, int64_t xstride) {
  if (ystride < 0) ystride = n;
  if (xstride < 0) xstride = n;
  k_axpby<<<dim3((unsigned)((n + 255) / 256), nbat), 256, 0, st>>>(y, x, a, b, n, a_b, act, ystride, xstride);
  return cudaGetLastError();
}

}  // namespace ahoc
