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
// index where |r|^j is above 1e-18 in FP64, 1e-9 in FP32) by multiplying
// with 1/r.  scale folds in
// the (2/N)^(d-1) of the inverse DST-I.
//
// One thread owns one mode column; a warp covers 32 adjacent x-modes, so
// every row access is a coalesced 32-element segment.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

// r x formed as x - (1 - r) x with 1 - r stored on its own (see Mode::q1)
__device__ __forceinline__ double rmul(double q1, double x) { return fma(-q1, x, x); }
__device__ __forceinline__ float rmul(float q1, float x) { return fmaf(-q1, x, x); }

// The terms that carry the boundary correction -- r^(j-1) w_j in P and K r^j --
// fall below the rounding of the solution beyond j0 (Mode::j0: |r|^j0 ~ 1e-18
// in FP64), so each recurrence runs in two phases: rows up to the warp's
// largest j0 with the correction terms (4 operations per row), the rest
// without them (2 per row).  The split is uniform across the warp.
// GEN: the right-hand side of the forward recurrence is generated from G
// (VGen3D: the v-equation's face terms in (x, y)-modes) instead of read.
template <typename T, bool GEN>
__global__ void __launch_bounds__(128) k_tri(Geom g, T* __restrict__ a, const Mode<T>* __restrict__ modes,
                                             VGen3D<T> G) {
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
  const int jw = __reduce_max_sync(__activemask(), md.j0);  // uniform phase boundary
  constexpr int B = 8;

  // the generator: row j's value is ax A[j - 1] + ay Bv[j - 1] (+ the z-face
  // terms on the first and last rows), A and Bv strided by ny and nx
  T ax = 0, ay = 0;
  const T *A = nullptr, *Bv = nullptr;
  const int ny = g.N[1] - 1;
  if (GEN) {
    const T* gen = G.gen + (int64_t)blockIdx.y * g.ngamma;
    ax = G.sx[ix];
    ay = G.sy[iy];
    A = gen + g.face_off[(ix & 1) ? 0 : 1] + (iy - 1);
    Bv = gen + g.face_off[(iy & 1) ? 2 : 3] + (ix - 1);
  }
  auto rhs = [&](int jj) -> T {
    if (!GEN) return col[(int64_t)jj * stride];
    T v = ax * A[(int64_t)(jj - 1) * ny] + ay * Bv[(int64_t)(jj - 1) * nx];
    if (jj == 1) v += G.gen[(int64_t)blockIdx.y * g.ngamma + g.face_off[4] + m];
    if (jj == nt) v += G.gen[(int64_t)blockIdx.y * g.ngamma + g.face_off[5] + m];
    return v;
  };
  // forward recurrence and the accumulated first value P = sum r^(j-1) w_j
  T w = 0, P = 0, rp = 1;
  int j = 1;
  for (; j + B - 1 <= nt; j += B) {
    T d[B];
#pragma unroll
    for (int q = 0; q < B; ++q) d[q] = rhs(j + q);
    if (j <= jw) {
#pragma unroll
      for (int q = 0; q < B; ++q) {
        w = rmul(md.q1, w) + md.s * d[q];
        P += rp * w;
        rp = rmul(md.q1, rp);
        d[q] = w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < B; ++q) {
        w = rmul(md.q1, w) + md.s * d[q];
        d[q] = w;
      }
    }
#pragma unroll
    for (int q = 0; q < B; ++q) col[(int64_t)(j + q) * stride] = d[q];
  }
  for (; j <= nt; ++j) {
    T d = rhs(j);
    w = rmul(md.q1, w) + md.s * d;
    if (j <= jw) {
      P += rp * w;
      rp = rmul(md.q1, rp);
    }
    col[(int64_t)j * stride] = w;
  }

  // backward recurrence with the boundary correction K r^j, started at j0
  const T K = md.kap * P;
  T u = 0, e = 0;
  j = nt;
  for (; j - B + 1 >= 1; j -= B) {
    T d[B];
#pragma unroll
    for (int q = 0; q < B; ++q) d[q] = col[(int64_t)(j - q) * stride];
    if (j - B + 1 <= jw) {
#pragma unroll
      for (int q = 0; q < B; ++q) {
        if (j - q == md.j0) e = K * md.rj0;
        u = rmul(md.q1, u) + (d[q] + e);
        e *= md.rinv;
        d[q] = u;
      }
    } else {
#pragma unroll
      for (int q = 0; q < B; ++q) {
        u = rmul(md.q1, u) + d[q];
        d[q] = u;
      }
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

// The generated right-hand side of one mode column m, as a function of the
// row j: 2D from VGen2D (x-mode k = m + 1), 3D from VGen3D (x- and y-modes).
template <typename T>
struct ColGen2 {
  VGen2D<T> G;
  int k, Nt;
  __device__ __forceinline__ T operator()(int j) const { return vgen(G, k, j, Nt); }
};
template <typename T>
struct ColGen3 {
  T ax, ay;
  const T *A, *B, *Zm, *Zp;
  int nx, ny, nt;
  __device__ __forceinline__ T operator()(int j) const {
    T v = ax * A[(int64_t)(j - 1) * ny] + ay * B[(int64_t)(j - 1) * nx];
    if (j == 1) v += *Zm;
    if (j == nt) v += *Zp;
    return v;
  }
};
template <typename T>
__device__ __forceinline__ ColGen2<T> col_gen(VGen2D<T> G, const Geom& g, int b, int64_t m, const TriShape& sh) {
  vgen_at(G, g, b);
  return ColGen2<T>{G, (int)m + 1, sh.Nt};
}
template <typename T>
__device__ __forceinline__ ColGen3<T> col_gen(const VGen3D<T>& G, const Geom& g, int b, int64_t m,
                                              const TriShape& sh) {
  ColGen3<T> c;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1;
  const int ix = 1 + (int)(m % nx), iy = 1 + (int)(m / nx);
  const T* gen = G.gen ? G.gen + (int64_t)b * g.ngamma : nullptr;
  c.ax = G.sx ? G.sx[ix] : (T)0;
  c.ay = G.sy ? G.sy[iy] : (T)0;
  c.A = gen ? gen + g.face_off[(ix & 1) ? 0 : 1] + (iy - 1) : nullptr;
  c.B = gen ? gen + g.face_off[(iy & 1) ? 2 : 3] + (ix - 1) : nullptr;
  c.Zm = gen ? gen + g.face_off[4] + m : nullptr;
  c.Zp = gen ? gen + g.face_off[5] + m : nullptr;
  c.nx = nx;
  c.ny = ny;
  c.nt = sh.nt;
  return c;
}

// right-hand side element: GEN 0 loaded, 1 generated, 2 loaded + generated
template <typename T, int GEN, class CG>
__device__ __forceinline__ T rhs_elem(const T* col, const CG& cg, int j, const TriShape& sh) {
  if (GEN == 0) return col[(int64_t)j * sh.stride];
  if (GEN == 1) return cg(j);
  return col[(int64_t)j * sh.stride] + cg(j);
}

template <typename T, int L, int GEN, class GT>
__global__ void __launch_bounds__(128) k_tri_t1(Geom g, const T* __restrict__ a, const Mode<T>* __restrict__ modes,
                                                double* __restrict__ E, GT G) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  E += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  const T* col = a + col_base(g, m);
  const T q1 = modes[m].q1, s = modes[m].s;
  const auto cg = col_gen(G, g, blockIdx.y, m, sh);
  T d[L];
#pragma unroll
  for (int q = 0; q < L; ++q)
    d[q] = (q < len) ? rhs_elem<T, GEN>(col, cg, s0 + q, sh) : (T)0;
  T w = 0;
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) w = rmul(q1, w) + s * d[q];
  E[(int64_t)c * sh.ncols + m] = (double)w;
}

// Carries of the chunked tridiagonal solves.  Along a column the chunk values
// v_c combine as s_{c+1} = v_c + rL s_c (forward, c = 0 .. C-1) or
// s_c = v_c + rL s_{c+1} (backward, c = C-1 .. 0), from s = 0; out_c is the
// value that enters chunk c (an exclusive scan) and the return value the
// total.  A CTA takes kScanCols columns (one per lane, so every load and
// store is coalesced across the columns) and cuts the C chunks into
// kScanSegs segments, one per warp: each warp composes its segment's affine
// map s -> rL^n s + b, the maps of the earlier segments are applied in
// order from shared memory, and each warp writes its segment's outputs.  The
// serial chain per column is C / kScanSegs chunks instead of C.
constexpr int kScanCols = 32, kScanSegs = 8;
template <bool FWD, class VF>
__device__ __forceinline__ double carry_scan(int C, double rL, const VF& v, double* out, int64_t ostride,
                                             bool in_range) {
  __shared__ double mA[kScanSegs][kScanCols], mB[kScanSegs][kScanCols];
  const int lane = threadIdx.x & (kScanCols - 1), seg = threadIdx.x / kScanCols;
  const int per = (C + kScanSegs - 1) / kScanSegs;
  const int c0 = seg * per, c1 = min(C, c0 + per);
  // this segment's map, in the scan's direction
  double a = 1.0, b = 0.0;
  if (in_range) {
    for (int q = 0; q < c1 - c0; ++q) {
      const int c = FWD ? c0 + q : c1 - 1 - q;
      b = fma(rL, b, v(c));
      a *= rL;
    }
  }
  mA[seg][lane] = a;
  mB[seg][lane] = b;
  __syncthreads();
  // the value entering this segment: the earlier segments' maps in order
  double sv = 0.0;
  for (int t = 0; t < kScanSegs; ++t) {
    const int u = FWD ? t : kScanSegs - 1 - t;
    if (FWD ? (u >= seg) : (u <= seg)) break;
    sv = fma(mA[u][lane], sv, mB[u][lane]);
  }
  double total = 0.0;
  if (in_range) {
    for (int q = 0; q < c1 - c0; ++q) {
      const int c = FWD ? c0 + q : c1 - 1 - q;
      out[(int64_t)c * ostride] = sv;
      sv = fma(rL, sv, v(c));
    }
    total = sv;  // after the last segment in the scan's direction: the whole column's value
  }
  return total;
}

__global__ void __launch_bounds__(kScanCols * kScanSegs) k_tri_t1b(Geom g, const Mode<double>* __restrict__ modes,
                                                                   const double* __restrict__ E,
                                                                   double* __restrict__ carry, int L) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  E += (int64_t)blockIdx.y * tri_sstride(sh);
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t m = (int64_t)blockIdx.x * kScanCols + (threadIdx.x & (kScanCols - 1));
  const bool in = m < sh.ncols;
  const double rL = in ? ipow(modes[m].r, L) : 0.0;
  // only the last chunk may be shorter; its carry-out is unused
  carry_scan<true>(sh.C, rL, [&](int c) { return E[(int64_t)c * sh.ncols + m]; }, carry + (in ? m : 0), sh.ncols,
                   in);
}

template <typename T, int L, int GEN, class GT>
__global__ void __launch_bounds__(128) k_tri_t2(Geom g, T* __restrict__ a, const Mode<T>* __restrict__ modes,
                                                const double* __restrict__ carry, double* __restrict__ B, GT G) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  B += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  T* col = a + col_base(g, m);
  const T q1 = modes[m].q1, s = modes[m].s;
  const auto cg = col_gen(G, g, blockIdx.y, m, sh);
  T d[L];
#pragma unroll
  for (int q = 0; q < L; ++q)
    d[q] = (q < len) ? rhs_elem<T, GEN>(col, cg, s0 + q, sh) : (T)0;
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

__global__ void __launch_bounds__(kScanCols * kScanSegs) k_tri_t2b(Geom g, const Mode<double>* __restrict__ modes,
                                                                   const double* __restrict__ B,
                                                                   double* __restrict__ bcarry, double* __restrict__ Cc,
                                                                   int L) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  B += (int64_t)blockIdx.y * tri_sstride(sh);
  bcarry += (int64_t)blockIdx.y * tri_sstride(sh);
  Cc += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t m = (int64_t)blockIdx.x * kScanCols + (threadIdx.x & (kScanCols - 1));
  const bool in = m < sh.ncols;
  const double rL = in ? ipow(modes[m].r, L) : 0.0;
  // the last (possibly shorter) chunk enters first, from zero: its own power of r never multiplies
  const double p1 = carry_scan<false>(sh.C, rL, [&](int c) { return B[(int64_t)c * sh.ncols + m]; },
                                      bcarry + (in ? m : 0), sh.ncols, in);
  if (in && threadIdx.x < kScanCols) Cc[m] = modes[m].kapC * p1;  // segment 0 ends at chunk 0: p_1
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

// ---------------------------------------------------------------------------
// FP64 chunked form in two passes over the field.  Per chunk of len rows from
// zero carries: the forward recurrence wl and the backward recurrence pl of
// wl (pl stored in place).  With the forward carry cf = w_{s0-1} and the
// backward carry cb = p_{e0+1},
//   w_{s0+q} = wl_q + cf r^(q+1),
//   p_{s0+q} = pl_q + cf G_q + cb r^(len-q),   G_q = sum_{q'=q}^{len-1} r^(2q'-q+1),
//   u_{s0+q} = p_{s0+q} + C (r^(s0+q) - r^(2N-s0-q)).
// With R_q = r^(len-1-q), P_q = r^q and G_q = (r P_q - r^(len+2) R_q)/(1 - r^2),
//   u_{s0+q} = pl_q + X R_q + Y P_q,
//   X = cb r - C r^(2N-e0) - cf r^(len+2)/(1-r^2),   Y = C r^(s0) + cf r/(1-r^2),
// two FMAs per row.  (For r near 1 the two cf terms are each about
// 1/(1 - r^2) times cf G_q and cancel: at most ~log10(1/((len+1)(1-r)))
// digits of that term, about 1.3 at N = 4096.)  R, P, the per-mode factors
// and the chunk powers come from a table built from the exact root in long
// double (tri2_table_size).  Within a chunk the recurrences multiply by the
// rounded r directly: over len <= 32 rows its representation error stays
// below 32 ulp.  The carry passes run one thread per column with their loads
// issued in batches of 8 chunks.
// ---------------------------------------------------------------------------
struct Tri2Off {
  int64_t Rf, Rl, P, rL, rlast, G0f, G0l, K1, K2f, K2l, rp1, rp2, total;
};
__host__ __device__ inline Tri2Off tri2_offsets(int64_t ncols, int C, int L) {
  Tri2Off o;
  const int64_t blk = (int64_t)L * ncols;
  o.Rf = 0;
  o.Rl = blk;
  o.P = 2 * blk;
  o.rL = 3 * blk;
  o.rlast = o.rL + ncols;
  o.G0f = o.rlast + ncols;
  o.G0l = o.G0f + ncols;
  o.K1 = o.G0l + ncols;
  o.K2f = o.K1 + ncols;
  o.K2l = o.K2f + ncols;
  o.rp1 = o.K2l + ncols;
  o.rp2 = o.rp1 + (int64_t)C * ncols;
  o.total = o.rp2 + (int64_t)C * ncols;
  return o;
}

size_t tri2_table_size(const Geom& g, int L) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int nt = ((g.dim == 3) ? g.N[2] : g.N[1]) - 1;
  const int C = (nt + L - 1) / L;
  return (size_t)tri2_offsets(ncols, C, L).total;  // doubles
}

void tri2_table_fill(const Geom& g, int L, const long double* r, double* out) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int Nt = (g.dim == 3) ? g.N[2] : g.N[1];
  const int nt = Nt - 1;
  const int C = (nt + L - 1) / L;
  const int lastlen = nt - (C - 1) * L;
  const Tri2Off o = tri2_offsets(ncols, C, L);
  std::vector<long double> pw(2 * L + 3);
  for (int64_t m = 0; m < ncols; ++m) {
    const long double rm = r[m];
    pw[0] = 1.0L;
    for (int k = 1; k < (int)pw.size(); ++k) pw[k] = pw[k - 1] * rm;
    for (int q = 0; q < L; ++q) {
      out[o.Rf + (int64_t)q * ncols + m] = (double)pw[L - 1 - q];
      out[o.Rl + (int64_t)q * ncols + m] = q < lastlen ? (double)pw[lastlen - 1 - q] : 0.0;
      out[o.P + (int64_t)q * ncols + m] = (double)pw[q];
    }
    long double g0 = 0.0L, g0l = 0.0L;  // G_0 = sum_{q'<len} r^(2q'+1)
    for (int qq = 0; qq < L; ++qq) g0 += pw[2 * qq + 1];
    for (int qq = 0; qq < lastlen; ++qq) g0l += pw[2 * qq + 1];
    const long double inv = 1.0L / (1.0L - rm * rm);
    out[o.rL + m] = (double)pw[L];
    out[o.rlast + m] = (double)pw[lastlen];
    out[o.G0f + m] = (double)g0;
    out[o.G0l + m] = (double)g0l;
    out[o.K1 + m] = (double)(rm * inv);
    out[o.K2f + m] = (double)(pw[L + 2] * inv);
    out[o.K2l + m] = (double)(pw[lastlen + 2] * inv);
    // r^(s0) = r^(1 + cL), ascending (shrinking); r^(2 Nt - e0), descending in c (shrinking)
    long double a = rm;
    for (int c = 0; c < C; ++c) {
      out[o.rp1 + (int64_t)c * ncols + m] = (double)a;
      a *= pw[L];
    }
    long double b = powl(rm, (long double)(2 * Nt - nt));  // chunk C-1 ends at e0 = nt
    for (int c = C - 1; c >= 0; --c) {
      out[o.rp2 + (int64_t)c * ncols + m] = (double)b;
      b *= (c == C - 1) ? pw[lastlen] : pw[L];
    }
  }
}

// Pass 1: local recurrences of a chunk.  GEN 1/2: the generated v-equation
// right-hand side s sk (rxm_j +- rxp_j) (VGen2D) replaces / is added to the
// field; its face rows (j = 1, N1 - 1) are corrected once outside the row loop.
template <int L, int GEN>
__global__ void __launch_bounds__(128) k_tri2_t1(Geom g, double* __restrict__ a,
                                                 const Mode<double>* __restrict__ modes, double* __restrict__ E,
                                                 double* __restrict__ B, VGen2D<double> G) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  E += (int64_t)blockIdx.y * tri_sstride(sh);
  B += (int64_t)blockIdx.y * tri_sstride(sh);
  vgen_at(G, g, blockIdx.y);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  double* col = a + col_base(g, m);
  const double r = modes[m].r, s = modes[m].s;
  double a1 = 0.0, a2 = 0.0;
  if (GEN) {
    const int k = (int)m + 1;
    a1 = s * G.sk[k];
    a2 = (k & 1) ? a1 : -a1;
  }
  double d[L];  // s times the right-hand side
#pragma unroll
  for (int q = 0; q < L; ++q) {
    double v = 0.0;
    if (q < len) {
      const int j = s0 + q;
      if (GEN) v = fma(a1, G.rxm[j], a2 * G.rxp[j]);
      if (GEN != 1) v = GEN ? fma(s, col[(int64_t)j * sh.stride], v) : s * col[(int64_t)j * sh.stride];
    }
    d[q] = v;
  }
  if (GEN && (s0 == 1 || s0 + len - 1 == sh.Nt - 1)) {
    const int k = (int)m + 1;
    const double bk = s * (G.Ly + 2.0 * G.ck[k] * G.Lxy);
    if (s0 == 1) d[0] -= bk * G.qhm[k - 1];
#pragma unroll
    for (int q = 0; q < L; ++q)
      if (q == len - 1 && s0 + q == sh.Nt - 1) d[q] -= bk * G.qhp[k - 1];
  }
  double w = 0.0;
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) {
      w = fma(r, w, d[q]);
      d[q] = w;
    }
  E[(int64_t)c * sh.ncols + m] = w;
  double pl = 0.0;
#pragma unroll
  for (int q = L - 1; q >= 0; --q)
    if (q < len) {
      pl = fma(r, pl, d[q]);
      d[q] = pl;
    }
  B[(int64_t)c * sh.ncols + m] = pl;
#pragma unroll
  for (int q = 0; q < L; ++q)
    if (q < len) col[(int64_t)(s0 + q) * sh.stride] = d[q];
}

// forward carries cf_c = w_{s0(c)-1}
__global__ void __launch_bounds__(kScanCols * kScanSegs) k_tri2_t1b(Geom g, const double* __restrict__ tab,
                                                                    const double* __restrict__ E,
                                                                    double* __restrict__ carry, int L) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  E += (int64_t)blockIdx.y * tri_sstride(sh);
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t m = (int64_t)blockIdx.x * kScanCols + (threadIdx.x & (kScanCols - 1));
  const bool in = m < sh.ncols;
  const Tri2Off o = tri2_offsets(sh.ncols, sh.C, L);
  const double rL = in ? tab[o.rL + m] : 0.0;
  carry_scan<true>(sh.C, rL, [&](int c) { return E[(int64_t)c * sh.ncols + m]; }, carry + (in ? m : 0), sh.ncols,
                   in);
}

// backward carries cb_c = p_{e0(c)+1} and C = kapC p_1; a chunk's value is
// its local p plus the forward carry's share cf G_0 (G_0 of the shorter last
// chunk for c = C - 1)
__global__ void __launch_bounds__(kScanCols * kScanSegs) k_tri2_t2b(Geom g, const Mode<double>* __restrict__ modes,
                                                                    const double* __restrict__ tab,
                                                                    const double* __restrict__ B,
                                                                    const double* __restrict__ carry,
                                                                    double* __restrict__ bcarry,
                                                                    double* __restrict__ Cc, int L) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  B += (int64_t)blockIdx.y * tri_sstride(sh);
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  bcarry += (int64_t)blockIdx.y * tri_sstride(sh);
  Cc += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t m = (int64_t)blockIdx.x * kScanCols + (threadIdx.x & (kScanCols - 1));
  const bool in = m < sh.ncols;
  const Tri2Off o = tri2_offsets(sh.ncols, sh.C, L);
  const double rL = in ? tab[o.rL + m] : 0.0;
  const double G0 = in ? tab[o.G0f + m] : 0.0, G0l = in ? tab[o.G0l + m] : 0.0;
  const int last = sh.C - 1;
  const double p1 = carry_scan<false>(
      sh.C, rL,
      [&](int c) {
        const int64_t i = (int64_t)c * sh.ncols + m;
        return fma(carry[i], c == last ? G0l : G0, B[i]);
      },
      bcarry + (in ? m : 0), sh.ncols, in);
  if (in && threadIdx.x < kScanCols) Cc[m] = modes[m].kapC * p1;  // segment 0 ends at chunk 0: p_1
}

template <int L>
__global__ void __launch_bounds__(128) k_tri2_t3(Geom g, double* __restrict__ a,
                                                 const Mode<double>* __restrict__ modes,
                                                 const double* __restrict__ tab, const double* __restrict__ carry,
                                                 const double* __restrict__ bcarry, const double* __restrict__ Cc) {
  if (g.skip(blockIdx.y)) return;
  const TriShape sh = tri_shape(g, L);
  a += (int64_t)blockIdx.y * g.npad;
  carry += (int64_t)blockIdx.y * tri_sstride(sh);
  bcarry += (int64_t)blockIdx.y * tri_sstride(sh);
  Cc += (int64_t)blockIdx.y * tri_sstride(sh);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= sh.ncols * sh.C) return;
  const int64_t m = t % sh.ncols;
  const int c = (int)(t / sh.ncols);
  const int s0 = 1 + c * L;
  const int len = min(L, sh.nt - s0 + 1);
  double* col = a + col_base(g, m);
  const Tri2Off o = tri2_offsets(sh.ncols, sh.C, L);
  const bool last = (c == sh.C - 1);
  const double* Rt = tab + (last ? o.Rl : o.Rf) + m;
  const double* Pt = tab + o.P + m;
  const int64_t i = (int64_t)c * sh.ncols + m;
  const double cf = carry[i], Cm = Cc[m];
  const double X = fma(-cf, tab[(last ? o.K2l : o.K2f) + m], fma(bcarry[i], modes[m].r, -Cm * tab[o.rp2 + i]));
  const double Y = fma(cf, tab[o.K1 + m], Cm * tab[o.rp1 + i]);
  // rows are independent here: batches of 8 keep the register count (and so
  // the occupancy that hides the loads) at that of an 8-row chunk
  constexpr int Q = L < 8 ? L : 8;
#pragma unroll 1
  for (int q0 = 0; q0 < L; q0 += Q) {
    double d[Q], rr[Q], pp[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const bool in = q0 + q < len;
      const int64_t k = (int64_t)(q0 + q) * sh.ncols;
      d[q] = in ? col[(int64_t)(s0 + q0 + q) * sh.stride] : 0.0;
      rr[q] = in ? Rt[k] : 0.0;
      pp[q] = in ? Pt[k] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (q0 + q < len) col[(int64_t)(s0 + q0 + q) * sh.stride] = fma(Y, pp[q], fma(X, rr[q], d[q]));
  }
}

template <int L, int GEN>
static cudaError_t tri2_L(const Geom& g, double* a, const Mode<double>* modes, const double* tab, double* scratch,
                          const VGen2D<double>& G, cudaStream_t st) {
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
  const dim3 cb((unsigned)((ncols + kScanCols - 1) / kScanCols), (unsigned)g.nb);
  k_tri2_t1<L, GEN><<<gb, 128, 0, st>>>(g, a, modes, E, B, G);
  k_tri2_t1b<<<cb, kScanCols * kScanSegs, 0, st>>>(g, tab, E, carry, L);
  k_tri2_t2b<<<cb, kScanCols * kScanSegs, 0, st>>>(g, modes, tab, B, carry, bcarry, Cc, L);
  k_tri2_t3<L><<<gb, 128, 0, st>>>(g, a, modes, tab, carry, bcarry, Cc);
  return cudaGetLastError();
}

cudaError_t launch_tri2(const Geom& g, double* a, const Mode<double>* modes, const double* tab, double* scratch,
                        int L, cudaStream_t st, const VGen2D<double>* G, bool add) {
  if (G && g.dim != 2) return cudaErrorInvalidValue;
  const VGen2D<double> Gz{};
  const VGen2D<double>& Gv = G ? *G : Gz;
  const int gen = G ? (add ? 2 : 1) : 0;
#define AHOC_TRI2(LL)                                                  \
  if (L == LL) {                                                       \
    if (gen == 0) return tri2_L<LL, 0>(g, a, modes, tab, scratch, Gv, st); \
    if (gen == 1) return tri2_L<LL, 1>(g, a, modes, tab, scratch, Gv, st); \
    return tri2_L<LL, 2>(g, a, modes, tab, scratch, Gv, st);           \
  }
  AHOC_TRI2(32)
  AHOC_TRI2(16)
  AHOC_TRI2(8)
#undef AHOC_TRI2
  return cudaErrorInvalidValue;
}

size_t tri_chunked_scratch(const Geom& g, int L) {
  const int nx = g.N[0] - 1;
  const int64_t ncols = (g.dim == 3) ? (int64_t)nx * (g.N[1] - 1) : nx;
  const int nt = ((g.dim == 3) ? g.N[2] : g.N[1]) - 1;
  const int C = (nt + L - 1) / L;
  return (size_t)(4 * C + 1) * ncols;  // doubles (the carries are FP64 for every T)
}

template <typename T, int L, int GEN, class GT>
static cudaError_t tri_chunked_L(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                                 const double* rpow, double* scratch, const GT& G, cudaStream_t st) {
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
  const dim3 cb((unsigned)((ncols + kScanCols - 1) / kScanCols), (unsigned)g.nb);
  k_tri_t1<T, L, GEN, GT><<<gb, 128, 0, st>>>(g, a, modes, E, G);
  k_tri_t1b<<<cb, kScanCols * kScanSegs, 0, st>>>(g, md64, E, carry, L);
  k_tri_t2<T, L, GEN, GT><<<gb, 128, 0, st>>>(g, a, modes, carry, B, G);
  k_tri_t2b<<<cb, kScanCols * kScanSegs, 0, st>>>(g, md64, B, bcarry, Cc, L);
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
// the same solve with the 3D v-equation right-hand side generated from VGen3D
template <typename T>
cudaError_t launch_tri_chunked_gen3(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                                    const double* rpow, double* scratch, int L, const VGen3D<T>& G,
                                    cudaStream_t st) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  if (L == 32) return tri_chunked_L<T, 32, 1>(g, a, modes, md64, rpow, scratch, G, st);
  if (L == 16) return tri_chunked_L<T, 16, 1>(g, a, modes, md64, rpow, scratch, G, st);
  if (L == 8) return tri_chunked_L<T, 8, 1>(g, a, modes, md64, rpow, scratch, G, st);
  return cudaErrorInvalidValue;
}
template cudaError_t launch_tri_chunked_gen3<float>(const Geom&, float*, const Mode<float>*, const Mode<double>*,
                                                    const double*, double*, int, const VGen3D<float>&, cudaStream_t);

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
  k_tri<T, false><<<dim3((unsigned)blocks, (unsigned)g.nb), threads, 0, st>>>(g, a, modes, VGen3D<T>{});
  return cudaGetLastError();
}

template cudaError_t launch_tri<double>(const Geom&, double*, const Mode<double>*, cudaStream_t);
template cudaError_t launch_tri<float>(const Geom&, float*, const Mode<float>*, cudaStream_t);

template <typename T>
cudaError_t launch_tri_gen3(const Geom& g, T* a, const Mode<T>* modes, const VGen3D<T>& G, cudaStream_t st) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  const int64_t ncols = (int64_t)(g.N[0] - 1) * (g.N[1] - 1);
  const int threads = 128;
  const int64_t blocks = (ncols + threads - 1) / threads;
  k_tri<T, true><<<dim3((unsigned)blocks, (unsigned)g.nb), threads, 0, st>>>(g, a, modes, G);
  return cudaGetLastError();
}
template cudaError_t launch_tri_gen3<double>(const Geom&, double*, const Mode<double>*, const VGen3D<double>&,
                                             cudaStream_t);

}  // namespace ahoc
