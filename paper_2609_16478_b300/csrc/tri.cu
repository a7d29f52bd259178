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

// r x formed as x - (1 - r) x with 1 - r stored on its own (see Mode::q1)
__device__ __forceinline__ double rmul(double q1, double x) { return fma(-q1, x, x); }
__device__ __forceinline__ float rmul(float q1, float x) { return fmaf(-q1, x, x); }

template <typename T>
__global__ void __launch_bounds__(128) k_tri(Geom g, T* __restrict__ a, const Mode<T>* __restrict__ modes) {
  if (g.skip(blockIdx.y)) return;
  a += (int64_t)blockIdx.y * g.npad;
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
      w = rmul(md.q1, w) + md.s * d[q];
      P += rp * w;
      rp = rmul(md.q1, rp);
      d[q] = w;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) col[(int64_t)(j + q) * stride] = d[q];
  }
  for (; j <= nt; ++j) {
    T d = col[(int64_t)j * stride];
    w = rmul(md.q1, w) + md.s * d;
    P += rp * w;
    rp = rmul(md.q1, rp);
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
      u = rmul(md.q1, u) + (d[q] + e);
      e *= md.rinv;
      d[q] = u;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) col[(int64_t)(j - q) * stride] = d[q];
  }
  for (; j >= 1; --j) {
    T d = col[(int64_t)j * stride];
    if (j == md.j0) e = K * md.rj0;
    u = rmul(md.q1, u) + (d + e);
    e *= md.rinv;
    col[(int64_t)j * stride] = u;
  }
}

// ---------------------------------------------------------------------------
// Chunked form for few columns (2D): each column is cut into chunks of L rows
// so that (columns x chunks) threads share the work.  With u = p + C phi,
// phi_j = r^j - r^(2N-j) and C = kapC * p_1:
//   T1  forward recurrence per chunk from a zero carry: chunk end value E_c
//   T1b per column: carries  w_{s_c - 1} = E_{c-1} + r^len carry_{c-1}
//   T2  forward recurrence with the true carry, then the backward recurrence
//       from a zero carry at the chunk end: local p stored, chunk start B_c
//   T2b per column: backward carries p_{e_c + 1} and p_1, hence C
//   T3  u_j = p_local_j + r^(e_c + 1 - j) p_{e_c + 1} + C (r^j - r^(2N - j))
// Powers are run in the direction in which they shrink (no underflow is ever
// scaled back up); r^n at a chunk boundary comes from binary powering.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ipow(T r, int n) {
  T out = 1, b = r;
  while (n > 0) {
    if (n & 1) out *= b;
    b *= b;
    n >>= 1;
  }
  return out;
}

struct TriShape {
  int64_t ncols;
  int nt, Nt, C, L;
  int64_t stride;
};

__device__ __forceinline__ TriShape tri_shape(const Geom& g, int L) {
  TriShape s;
  const int nx = g.N[0] - 1;
  s.ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  s.Nt = (g.dim == 3) ? g.N[2] : g.N[1];
  s.nt = s.Nt - 1;
  s.L = L;
  s.C = (s.nt + L - 1) / L;
  s.stride = (g.dim == 3) ? g.n0 * g.n1 : g.n0;
  return s;
}

__device__ __forceinline__ int64_t col_base(const Geom& g, int64_t m) {
  const int nx = g.N[0] - 1;
  const int ix = 1 + (int)(m % nx);
  const int iy = (g.dim == 3) ? 1 + (int)(m / nx) : 0;
  return ix + g.n0 * (int64_t)iy;
}

// per-problem scratch of the chunked solve: (4C + 1) ncols doubles
__device__ __forceinline__ int64_t tri_sstride(const TriShape& sh) { return (4 * (int64_t)sh.C + 1) * sh.ncols; }

// the generator arrays of problem b (rx: N1 + 1 apart, qy: 2 N0 apart)
template <typename T>
__device__ __forceinline__ void vgen_at(VGen2D<T>& G, const Geom& g, int b) {
  if (!G.rxm) return;
  const int64_t rs = (int64_t)b * (g.N[1] + 1), qs = (int64_t)b * 2 * g.N[0];
  G.rxm += rs;
  G.rxp += rs;
  G.qhm += qs;
  G.qhp += qs;
}

// generated right-hand side of the homogeneous v-equation (2D), see VGen2D
template <typename T>
__device__ __forceinline__ T vgen(const VGen2D<T>& G, int k, int j, int Nt) {
  T v = G.sk[k] * (G.rxm[j] + ((k & 1) ? G.rxp[j] : -G.rxp[j]));
  if (j == 1 || j == Nt - 1) {
    const T bk = G.Ly + (T)2 * G.ck[k] * G.Lxy;
    if (j == 1) v -= bk * G.qhm[k - 1];
    if (j == Nt - 1) v -= bk * G.qhp[k - 1];
  }
  return v;
}

// right-hand side element: GEN 0 loaded, 1 generated, 2 loaded + generated
template <typename T, int GEN>
__device__ __forceinline__ T rhs_elem(const T* col, const VGen2D<T>& G, int k, int j, const TriShape& sh) {
  if (GEN == 0) return col[(int64_t)j * sh.stride];
  if (GEN == 1) return vgen(G, k, j, sh.Nt);
  return col[(int64_t)j * sh.stride] + vgen(G, k, j, sh.Nt);
}

template <typename T, int L, int GEN>
__global__ void __launch_bounds__(128) k_tri_t1(Geom g, const T* __restrict__ a, const Mode<T>* __restrict__ modes,
                                                double* __restrict__ E, VGen2D<T> G) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  E += (int64_t)blockIdx.y * tri_sstride(sh);
  vgen_at(G, g, blockIdx.y);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  const T* col = a + col_base(g, m);
  const T q1 = modes[m].q1, s = modes[m].s;
  T d[L];
#pragma unroll
  for (int q = 0; q < L; ++q)
    d[q] = (q < len) ? rhs_elem<T, GEN>(col, G, (int)m + 1, s0 + q, sh) : (T)0;
  T w = 0;
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) w = rmul(q1, w) + s * d[q];
  E[(int64_t)c * sh.ncols + m] = (double)w;
}

__global__ void k_tri_t1b(Geom g, const Mode<double>* __restrict__ modes, const double* __restrict__ E,
                          double* __restrict__ carry, int L) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  E += (int64_t)blockIdx.y * tri_sstride(sh);
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sh.ncols) return;
  const double r = modes[m].r;
  const double rL = ipow(r, L);
  double cy = 0;
  // only the last chunk may be shorter; its carry-out is unused
  constexpr int B = 8;
  int c = 0;
  for (; c + B <= sh.C; c += B) {
    double e[B];
#pragma unroll
    for (int q = 0; q < B; ++q) e[q] = E[(int64_t)(c + q) * sh.ncols + m];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      carry[(int64_t)(c + q) * sh.ncols + m] = cy;
      cy = e[q] + rL * cy;
    }
  }
  for (; c < sh.C; ++c) {
    carry[(int64_t)c * sh.ncols + m] = cy;
    cy = E[(int64_t)c * sh.ncols + m] + rL * cy;
  }
}

template <typename T, int L, int GEN>
__global__ void __launch_bounds__(128) k_tri_t2(Geom g, T* __restrict__ a, const Mode<T>* __restrict__ modes,
                                                const double* __restrict__ carry, double* __restrict__ B, VGen2D<T> G) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  B += (int64_t)blockIdx.y * tri_sstride(sh);
  vgen_at(G, g, blockIdx.y);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  T* col = a + col_base(g, m);
  const T q1 = modes[m].q1, s = modes[m].s;
  T d[L];
#pragma unroll
  for (int q = 0; q < L; ++q)
    d[q] = (q < len) ? rhs_elem<T, GEN>(col, G, (int)m + 1, s0 + q, sh) : (T)0;
  T w = (T)carry[(int64_t)c * sh.ncols + m];
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) {
      w = rmul(q1, w) + s * d[q];
      d[q] = w;
    }
  T p = 0;
#pragma unroll
  for (int q = L - 1; q >= 0; --q)
    if (q < len) {
      p = rmul(q1, p) + d[q];
      d[q] = p;
    }
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) col[(int64_t)(s0 + q) * sh.stride] = d[q];
  B[(int64_t)c * sh.ncols + m] = (double)p;
}

__global__ void k_tri_t2b(Geom g, const Mode<double>* __restrict__ modes, const double* __restrict__ B,
                          double* __restrict__ bcarry, double* __restrict__ Cc, int L) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  B += (int64_t)blockIdx.y * tri_sstride(sh);
  bcarry += (int64_t)blockIdx.y * tri_sstride(sh);
  Cc += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= sh.ncols) return;
  const double r = modes[m].r;
  const double rL = ipow(r, L);
  const int lastlen = sh.nt - (sh.C - 1) * L;
  // last (possibly shorter) chunk first, then the full ones in batches
  double bc = 0;
  int c = sh.C - 1;
  bcarry[(int64_t)c * sh.ncols + m] = bc;
  bc = B[(int64_t)c * sh.ncols + m] + ipow(r, lastlen) * bc;  // p at the chunk start
  --c;
  constexpr int NB = 8;
  for (; c - NB + 1 >= 0; c -= NB) {
    double bv[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) bv[q] = B[(int64_t)(c - q) * sh.ncols + m];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      bcarry[(int64_t)(c - q) * sh.ncols + m] = bc;
      bc = bv[q] + rL * bc;
    }
  }
  for (; c >= 0; --c) {
    bcarry[(int64_t)c * sh.ncols + m] = bc;
    bc = B[(int64_t)c * sh.ncols + m] + rL * bc;
  }
  Cc[m] = modes[m].kapC * bc;  // bc = p_1
}

template <typename T, int L>
__global__ void __launch_bounds__(128) k_tri_t3(Geom g, T* __restrict__ a, const Mode<T>* __restrict__ modes,
                                                const Mode<double>* __restrict__ md64,
                                                const double* __restrict__ rpow,
                                                const double* __restrict__ bcarry, const double* __restrict__ Cc) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  bcarry += (int64_t)blockIdx.y * tri_sstride(sh);
  Cc += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  const int e0 = s0 + len - 1;
  T* col = a + col_base(g, m);
  const T q1 = modes[m].q1;
  const double r = md64[m].r;
  const double bc = bcarry[(int64_t)c * sh.ncols + m];
  const double Cm = Cc[m];
  T d[L];
#pragma unroll
  for (int q = 0; q < L; ++q) d[q] = (q < len) ? col[(int64_t)(s0 + q) * sh.stride] : (T)0;
  // descending: r^(e0 + 1 - j) bc - C r^(2N - j) = X_j, one geometric term
  // (X_{j-1} = r X_j) that shrinks as j decreases
  T X = (T)(r * bc - Cm * rpow[(int64_t)(sh.C + c) * sh.ncols + m]);  // r^(2N - e0) tabulated
#pragma unroll
  for (int q = L - 1; q >= 0; --q)
    if (q < len) {
      d[q] += X;
      X = rmul(q1, X);
    }
  // ascending: + C r^j, shrinking as j increases
  T Aj = (T)(Cm * rpow[(int64_t)c * sh.ncols + m]);  // r^(s0) tabulated
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) {
      d[q] += Aj;
      Aj = rmul(q1, Aj);
    }
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) col[(int64_t)(s0 + q) * sh.stride] = d[q];
}

size_t tri_chunked_scratch(const Geom& g, int L) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int nt = ((g.dim == 3) ? g.N[2] : g.N[1]) - 1;
  const int C = (nt + L - 1) / L;
  return (size_t)(4 * C + 1) * ncols;  // doubles (the carries are FP64 for every T)
}

template <typename T, int L, int GEN>
static cudaError_t tri_chunked_L(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                                 const double* rpow, double* scratch, const VGen2D<T>& G, cudaStream_t st) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int nt = ((g.dim == 3) ? g.N[2] : g.N[1]) - 1;
  const int C = (nt + L - 1) / L;
  double* E = scratch;
  double* carry = E + (int64_t)C * ncols;
  double* B = carry + (int64_t)C * ncols;
  double* bcarry = B + (int64_t)C * ncols;
  double* Cc = bcarry + (int64_t)C * ncols;
  const int64_t work = ncols * C;
  const dim3 gb((unsigned)((work + 127) / 128), (unsigned)g.nb);
  const dim3 cb((unsigned)((ncols + 127) / 128), (unsigned)g.nb);
  k_tri_t1<T, L, GEN><<<gb, 128, 0, st>>>(g, a, modes, E, G);
  k_tri_t1b<<<cb, 128, 0, st>>>(g, md64, E, carry, L);
  k_tri_t2<T, L, GEN><<<gb, 128, 0, st>>>(g, a, modes, carry, B, G);
  k_tri_t2b<<<cb, 128, 0, st>>>(g, md64, B, bcarry, Cc, L);
  k_tri_t3<T, L><<<gb, 128, 0, st>>>(g, a, modes, md64, rpow, bcarry, Cc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tri_chunked(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                               const double* rpow, double* scratch, int L, cudaStream_t st) {
  VGen2D<T> G{};
  if (L == 32) return tri_chunked_L<T, 32, 0>(g, a, modes, md64, rpow, scratch, G, st);
  if (L == 16) return tri_chunked_L<T, 16, 0>(g, a, modes, md64, rpow, scratch, G, st);
  if (L == 8) return tri_chunked_L<T, 8, 0>(g, a, modes, md64, rpow, scratch, G, st);
  return cudaErrorInvalidValue;
}

// rpow[c][m] = r_m^(1 + cL) and rpow[C + c][m] = r_m^(2N - e_c), by binary powering in FP64
__global__ void k_tri_powers(Geom g, const Mode<double>* __restrict__ md64, double* __restrict__ rpow, int L) {
  const TriShape sh = tri_shape(g, L);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int e0 = min(s0 + L - 1, sh.nt);
  const double r = md64[m].r;
  rpow[(int64_t)c * sh.ncols + m] = ipow(r, s0);
  rpow[(int64_t)(sh.C + c) * sh.ncols + m] = ipow(r, 2 * sh.Nt - e0);
}

size_t tri_powers_size(const Geom& g, int L) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int nt = ((g.dim == 3) ? g.N[2] : g.N[1]) - 1;
  const int C = (nt + L - 1) / L;
  return (size_t)2 * C * ncols;  // doubles
}

cudaError_t launch_tri_powers(const Geom& g, const Mode<double>* md64, double* rpow, int L, cudaStream_t st) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int nt = ((g.dim == 3) ? g.N[2] : g.N[1]) - 1;
  const int C = (nt + L - 1) / L;
  const int64_t work = ncols * C;
  k_tri_powers<<<(unsigned)((work + 127) / 128), 128, 0, st>>>(g, md64, rpow, L);
  return cudaGetLastError();
}

// the same solve with the v-equation right-hand side generated on the fly (2D)
template <typename T>
cudaError_t launch_tri_chunked_gen(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                                   const double* rpow, double* scratch, int L, const VGen2D<T>& G, cudaStream_t st,
                                   bool add) {
  if (g.dim != 2) return cudaErrorInvalidValue;
  if (L == 32) return add ? tri_chunked_L<T, 32, 2>(g, a, modes, md64, rpow, scratch, G, st)
                          : tri_chunked_L<T, 32, 1>(g, a, modes, md64, rpow, scratch, G, st);
  if (L == 16) return add ? tri_chunked_L<T, 16, 2>(g, a, modes, md64, rpow, scratch, G, st)
                          : tri_chunked_L<T, 16, 1>(g, a, modes, md64, rpow, scratch, G, st);
  if (L == 8) return add ? tri_chunked_L<T, 8, 2>(g, a, modes, md64, rpow, scratch, G, st)
                         : tri_chunked_L<T, 8, 1>(g, a, modes, md64, rpow, scratch, G, st);
  return cudaErrorInvalidValue;
}
template cudaError_t launch_tri_chunked_gen<double>(const Geom&, double*, const Mode<double>*, const Mode<double>*,
                                                    const double*, double*, int, const VGen2D<double>&, cudaStream_t,
                                                    bool);
template cudaError_t launch_tri_chunked_gen<float>(const Geom&, float*, const Mode<float>*, const Mode<double>*,
                                                   const double*, double*, int, const VGen2D<float>&, cudaStream_t,
                                                   bool);

template cudaError_t launch_tri_chunked<double>(const Geom&, double*, const Mode<double>*, const Mode<double>*,
                                                const double*, double*, int, cudaStream_t);
template cudaError_t launch_tri_chunked<float>(const Geom&, float*, const Mode<float>*, const Mode<double>*,
                                               const double*, double*, int, cudaStream_t);

template <typename T>
cudaError_t launch_tri(const Geom& g, T* a, const Mode<T>* modes, cudaStream_t st) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int threads = 128;
  const int64_t blocks = (ncols + threads - 1) / threads;
  k_tri<T><<<dim3((unsigned)blocks, (unsigned)g.nb), threads, 0, st>>>(g, a, modes);
  return cudaGetLastError();
}

template cudaError_t launch_tri<double>(const Geom&, double*, const Mode<double>*, cudaStream_t);
template cudaError_t launch_tri<float>(const Geom&, float*, const Mode<float>*, cudaStream_t);

}  // namespace ahoc
