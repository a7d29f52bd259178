// Solve along the last axis of a Dirichlet HOC Poisson problem in the
// spectral domain of the other axes.
//
// After the DST-I along x (and y in 3D), L_h acts on each transverse mode as
// a symmetric Toeplitz tridiagonal T = tridiag(b, a, b) along the last axis
// with zero Dirichlet ends (the three-term recurrence of Lemma 4's proof).
// With r the root of modulus < 1 of b r^2 + a r + b = 0 and sigma = a/(1+r^2),
//     T = sigma (1 - r E^-1)(1 - r E)        (E: shift j -> j+1),
// so T u = d is two first-order recurrences plus one boundary correction:
//     w_j = r w_{j-1} + s d_j,  w_0 = 0             (s = scale / sigma)
//     P   = sum_j r^{j-1} w_j                       (= the uncorrected u_1)
//     u_j = r u_{j+1} + w_j + K r^j,  u_N = 0,   K = kap * P,
// where kap = -r (1 - r^2) / (1 - r^{2N}) makes u_0 = 0 exactly.  No
// division is done on the device.  K r^j is run downward from j0 (the last
// index where |r|^j is representable) by multiplying with 1/r.  scale folds in
// the (2/N)^(d-1) of the inverse DST-I.
//
// One thread owns one mode column; a warp covers 32 adjacent x-modes, so
// every row access is a coalesced 32-element segment.
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

template <typename T>
__global__ void __launch_bounds__(128) k_tri(Geom g, T* __restrict__ a, const Mode<T>* __restrict__ modes) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ncols) return;
  const int ix = 1 + (int)(m % nx);
  const int iy = (g.dim == 3) ? 1 + (int)(m / nx) : 0;
  const int Nt = (g.dim == 3) ? g.N[2] : g.N[1];
  const int64_t stride = (g.dim == 3) ? g.n0 * g.n1 : g.n0;
  T* col = a + ix + g.n0 * (int64_t)iy;
  const Mode<T> md = modes[m];
  const int nt = Nt - 1;
  constexpr int B = 8;

  // forward recurrence and the accumulated first value P
  T w = 0, P = 0, rp = 1;
  int j = 1;
  for (; j + B - 1 <= nt; j += B) {
    T d[B];
#pragma unroll
    for (int q = 0; q < B; ++q) d[q] = col[(int64_t)(j + q) * stride];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      w = md.r * w + md.s * d[q];
      P += rp * w;
      rp *= md.r;
      d[q] = w;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) col[(int64_t)(j + q) * stride] = d[q];
  }
  for (; j <= nt; ++j) {
    T d = col[(int64_t)j * stride];
    w = md.r * w + md.s * d;
    P += rp * w;
    rp *= md.r;
    col[(int64_t)j * stride] = w;
  }

  // backward recurrence with the boundary correction K r^j
  const T K = md.kap * P;
  T u = 0, e = 0;
  j = nt;
  for (; j - B + 1 >= 1; j -= B) {
    T d[B];
#pragma unroll
    for (int q = 0; q < B; ++q) d[q] = col[(int64_t)(j - q) * stride];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      if (j - q == md.j0) e = K * md.rj0;
      u = md.r * u + (d[q] + e);
      e *= md.rinv;
      d[q] = u;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) col[(int64_t)(j - q) * stride] = d[q];
  }
  for (; j >= 1; --j) {
    T d = col[(int64_t)j * stride];
    if (j == md.j0) e = K * md.rj0;
    u = md.r * u + (d + e);
    e *= md.rinv;
    col[(int64_t)j * stride] = u;
  }
}

template <typename T>
cudaError_t launch_tri(const Geom& g, T* a, const Mode<T>* modes, cudaStream_t st) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int threads = 128;
  const int64_t blocks = (ncols + threads - 1) / threads;
  k_tri<T><<<(unsigned)blocks, threads, 0, st>>>(g, a, modes);
  return cudaGetLastError();
}

template cudaError_t launch_tri<double>(const Geom&, double*, const Mode<double>*, cudaStream_t);
template cudaError_t launch_tri<float>(const Geom&, float*, const Mode<float>*, cudaStream_t);

}  // namespace ahoc
