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

// ---------------------------------------------------------------------------
// GMRES's Hessenberg QR on the device (one thread per problem).  Per-problem
// state (GivensLayout): the rotated columns R (column j at j * (m + 1)), the
// rotations cs, sn, the rotated right-hand side g, and the scalars beta0
// (||b||), tol and rel (the residual estimate); ints iters, maxit, status,
// jend (columns of this cycle) and cyc (taking part in this cycle).
// ---------------------------------------------------------------------------
struct GivensView {
  double *R, *cs, *sn, *g, *sc;
  int* st;
};
__device__ __forceinline__ GivensView givens_view(double* gs, int* gi, int b, int m) {
  GivensView v;
  v.R = gs + (int64_t)b * givens_doubles(m);
  v.cs = v.R + (int64_t)(m + 1) * m;
  v.sn = v.cs + m;
  v.g = v.sn + m;
  v.sc = v.g + (m + 1);
  v.st = gi + kGivensInts * b;
  return v;
}

// start of a cycle: ini[3 b .. 3 b + 2] = (beta, beta0, tol), ii[2 b .. 2 b + 1] = (iters, maxit)
__global__ void k_givens_init(int nb, int m, const int* __restrict__ act, const double* __restrict__ ini,
                              const int* __restrict__ ii, double* __restrict__ gs, int* __restrict__ gi,
                              double* __restrict__ rel) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  GivensView v = givens_view(gs, gi, b, m);
  v.g[0] = ini[3 * b];
  v.sc[0] = ini[3 * b + 1];
  v.sc[1] = ini[3 * b + 2];
  v.sc[2] = ini[3 * b + 1] > 0 ? ini[3 * b] / ini[3 * b + 1] : 0.0;
  rel[b] = v.sc[2];
  v.st[0] = ii[2 * b];
  v.st[1] = ii[2 * b + 1];
  v.st[2] = 0;
  v.st[3] = 0;
  v.st[4] = act[b];
}

// step j: column j of the Hessenberg matrix from the CGS2 coefficients of
// both passes (h[k] + h[j + 1 + k]) and ||w|| (h[2 (j + 1)] holds ||w||^2),
// the earlier rotations, a new rotation zeroing the subdiagonal, and the
// residual estimate |g[j + 1]| / beta0.  A problem that converges, reaches
// maxit or meets a NaN / Inf leaves the mask; the others get 1 / ||w|| for
// the normalisation of the next Krylov vector.
__global__ void k_givens_step(int j, int nb, int m, const double* __restrict__ hdev, int hs, int* __restrict__ act,
                              double* __restrict__ scal, double* __restrict__ gs, int* __restrict__ gi,
                              double* __restrict__ relo) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !act[b]) return;
  GivensView v = givens_view(gs, gi, b, m);
  const double* hh = hdev + (int64_t)b * hs;
  double* Hc = v.R + (int64_t)j * (m + 1);
  bool bad = false;
  for (int k = 0; k <= j; ++k) {
    Hc[k] = hh[k] + hh[j + 1 + k];
    bad = bad || !isfinite(Hc[k]);
  }
  const double hn = sqrt(hh[2 * (j + 1)]);
  bad = bad || !isfinite(hn);
  v.st[0] += 1;
  if (bad) {  // this problem leaves the batch; its iterate stays as at the cycle start
    v.st[2] = kGivensNumeric;
    v.st[3] = 0;
    act[b] = 0;
    return;
  }
  Hc[j + 1] = hn;
  for (int k = 0; k < j; ++k) {
    const double a = Hc[k], c = Hc[k + 1];
    Hc[k] = v.cs[k] * a + v.sn[k] * c;
    Hc[k + 1] = -v.sn[k] * a + v.cs[k] * c;
  }
  const double den = hypot(Hc[j], Hc[j + 1]);
  v.cs[j] = (den > 0) ? Hc[j] / den : 1.0;
  v.sn[j] = (den > 0) ? Hc[j + 1] / den : 0.0;
  Hc[j] = den;
  Hc[j + 1] = 0.0;
  v.g[j + 1] = -v.sn[j] * v.g[j];
  v.g[j] = v.cs[j] * v.g[j];
  v.st[3] = j + 1;
  const double rel = fabs(v.g[j + 1]) / v.sc[0];
  v.sc[2] = rel;
  relo[b] = rel;
  if (rel <= v.sc[1] || hn == 0.0) {
    act[b] = 0;  // converged
  } else if (v.st[0] >= v.st[1]) {
    act[b] = 0;
    v.st[2] = kGivensNoConv;
  } else {
    scal[b] = 1.0 / hn;
  }
}

// end of a cycle: y = R^-1 g over the cycle's columns (back substitution),
// hy[b * hs + k] = -y_k for the update X -= Z hy, ncols[b] = the columns used
// (0 for problems outside the cycle); summary[b] = (iters, status, jend) and
// rel[b] for the host.
__global__ void k_givens_solve(int nb, int m, const double* __restrict__ gs, const int* __restrict__ gi,
                               double* __restrict__ hy, int hs, int* __restrict__ ncols) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  GivensView v = givens_view(const_cast<double*>(gs), const_cast<int*>(gi), b, m);
  const int je = v.st[4] ? v.st[3] : 0;
  ncols[b] = je;
  double* y = hy + (int64_t)b * hs;
  for (int k = je - 1; k >= 0; --k) {
    double acc = v.g[k];
    for (int l = k + 1; l < je; ++l) acc -= v.R[(int64_t)l * (m + 1) + k] * (-y[l]);
    y[k] = -(acc / v.R[(int64_t)k * (m + 1) + k]);
  }
}

cudaError_t launch_givens_init(int nb, int m, const int* act, const double* ini, const int* ii, double* gs, int* gi,
                               double* rel, cudaStream_t st) {
  k_givens_init<<<(nb + 31) / 32, 32, 0, st>>>(nb, m, act, ini, ii, gs, gi, rel);
  return cudaGetLastError();
}
cudaError_t launch_givens_step(int j, int nb, int m, const double* hdev, int hs, int* act, double* scal, double* gs,
                               int* gi, double* rel, cudaStream_t st) {
  k_givens_step<<<(nb + 31) / 32, 32, 0, st>>>(j, nb, m, hdev, hs, act, scal, gs, gi, rel);
  return cudaGetLastError();
}
cudaError_t launch_givens_solve(int nb, int m, const double* gs, const int* gi, double* hy, int hs, int* ncols,
                                cudaStream_t st) {
  k_givens_solve<<<(nb + 31) / 32, 32, 0, st>>>(nb, m, gs, gi, hy, hs, ncols);
  return cudaGetLastError();
}

}  // namespace ahoc
