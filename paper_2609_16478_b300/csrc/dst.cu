// DST-I along the x axis (contiguous lines) and the y axis (strided lines).
//
// The transform is X_k = sum_{j=1}^{N-1} x_j sin(pi j k / N), k = 1..N-1,
// the sine expansion that diagonalises the compact operators (Lemma 4 and its
// appendix proof).  It is computed through one complex FFT of length M = N/2:
//   z_j = sin(pi j/N)(x_j + x_{N-j}) + (x_j - x_{N-j})/2        (z_0 = 0)
//   C   = FFT_M(z_0 + i z_1, z_2 + i z_3, ...)
//   F_k = E_k + e^{-2 pi i k/N} O_k,  E_k = (C_k + conj C_{M-k})/2,
//         O_k = -i (C_k - conj C_{M-k})/2                       (real FFT of z)
//   X_{2k} = -Im F_k,   X_{2k+1} = Re F_0 / 2 + sum_{m=1}^{k} Re F_m,
// i.e. the odd outputs are a prefix sum.  The 1/2 factors are folded into the
// pre-processing table (sn[j] = sin(pi j/N)/2, and 1/4 on the difference).
//
// The FFT is a self-sorting (Stockham) radix-4 transform in shared memory,
// with one radix-2 stage first when log2 M is odd.  A line of N elements is
// handled by TPL = N/8 threads (one radix-4 butterfly each per stage); a CTA
// holds LPC lines.  All twiddles come from per-plan tables computed on the
// host in long double: tw[t] = exp(-2 pi i t/N), t < N, followed by the same
// values per FFT stage in the order its threads read them (dst_tw_len).
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

template <typename T> struct Cplx;
template <> struct Cplx<double> { using t = double2; };
template <> struct Cplx<float> { using t = float2; };

__device__ __forceinline__ double fmaT(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return ::fmaf(a, b, c); }

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = fmaT(a.x, b.x, -a.y * b.y);
  r.y = fmaT(a.x, b.y, a.y * b.x);
  return r;
}

// A factor zeta held as (c, t) (table layout at dst_tw_len): zeta q is c R,
// R = rot(q + i t q), rot the identity or (when `swap`) multiplication by i.
// The products c R enter the butterflies as FMAs: with
//   Rx = swap ? T.y : T.x,  Ry = swap ? T.x : T.y,  cx = swap ? -c : c,
// (c R).x = cx Rx and (c R).y = c Ry.  The selects and the sign flip are
// integer operations, off the FP64 pipe.
template <typename C>
__device__ __forceinline__ C lf_rot(C q, decltype(C{}.x) t, bool swap) {
  const auto tx = fmaT(-t, q.y, q.x), ty = fmaT(t, q.x, q.y);
  C r;
  r.x = swap ? ty : tx;
  r.y = swap ? tx : ty;
  return r;
}
__device__ __forceinline__ double negif(double x, bool f) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)f << 63));
}
__device__ __forceinline__ float negif(float x, bool f) {
  return __int_as_float(__float_as_int(x) ^ ((int)f << 31));
}

// Barrier of the threads of one line (see dst_lines): bar > 0 a named
// barrier of TPL threads, bar == 0 the CTA, bar < 0 the warp.
__device__ __forceinline__ void line_sync(int bar, int TPL) {
  if (bar > 0) asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(TPL) : "memory");
  else if (bar == 0) __syncthreads();
  else __syncwarp();
}

// In-place DST-I of the LPC lines of this CTA.  Line l occupies s[l*LS .. l*LS+N)
// with s[l*LS] == 0.  Every thread of the CTA must call this.  wsum: >= 32
// elements of scratch for the cross-warp scan.
template <typename T>
__device__ void dst_lines(T* s, int LS, int N, int logN, int TPL, const typename Cplx<T>::t* __restrict__ tw,
                          const T* __restrict__ sn, T* wsum) {
  using C = typename Cplx<T>::t;
  const int tid = threadIdx.x;
  const int l = tid / TPL;
  const int lt = tid - l * TPL;
  // the threads of one line synchronise among themselves: a named barrier per
  // line (ids 1..15) when a line spans several warps, the warp itself when it
  // fits in one, the whole CTA only when it holds more than 15 multi-warp lines
  const int bar = (TPL <= 32) ? -1 : ((int)blockDim.x / TPL <= 15 ? l + 1 : 0);
  T* y = s + (int64_t)l * LS;
  C* c = reinterpret_cast<C*>(y);
  const int M = N >> 1;
  const int logM = logN - 1;

  // 1. pre-processing, pairs (j, N-j): z_j = (s_j + 1/4) x_j + (s_j - 1/4) x_{N-j}
  //    and z_{N-j} the other way round, s_j = sin(pi j/N)/2 (tabulated sums)
  const C* pm = tw + N;
  for (int j = lt + 1; j <= (N >> 1); j += TPL) {
    const T a = y[j], b = y[N - j];
    const C f = pm[j];
    y[j] = fmaT(f.x, a, f.y * b);
    if (j != (N >> 1)) y[N - j] = fmaT(f.y, a, f.x * b);
  }
  line_sync(bar, TPL);

  // 2. complex FFT of length M (Stockham, natural order in and out)
  int Ns = 1;
  if (logM & 1) {
    C x[4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int j = lt + q * TPL;
      x[2 * q] = c[j];
      x[2 * q + 1] = c[j + (M >> 1)];
    }
    line_sync(bar, TPL);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int j = lt + q * TPL;
      C a = x[2 * q], b = x[2 * q + 1];
      C u, v;
      u.x = a.x + b.x; u.y = a.y + b.y;
      v.x = a.x - b.x; v.y = a.y - b.y;
      c[2 * j] = u;
      c[2 * j + 1] = v;
    }
    line_sync(bar, TPL);
    Ns = 2;
  }
  const int M4 = M >> 2;
  // stage factors w = W^kk and w^2, W = exp(-2 pi i/(4 Ns)), contiguous in kk
  const C* tws = tw + N + (N >> 1) + 1;
  for (; Ns < M; Ns <<= 2) {
    const int j = lt;
    const int kk = j & (Ns - 1);
    const C x0 = c[j], x1 = c[j + M4], x2 = c[j + 2 * M4], x3 = c[j + 3 * M4];
    C y0, y1, y2, y3;
    if (Ns > 1) {
      // y_r = sum_m (-i)^{rm} w^m x_m, factored as a = x0 +- w^2 x2,
      // b = x1 +- w^2 x3, y = a +- w b (and a -+ i w b): every product with a
      // factor becomes FMAs (24 FP64 operations instead of 28)
      const C f1 = tws[kk], f2 = tws[Ns + kk];
      const bool s1 = dst_swap_w1(kk, Ns), s2 = dst_swap_w2(kk, Ns);
      const T c1 = f1.x, c1x = negif(f1.x, s1), c2 = f2.x, c2x = negif(f2.x, s2);
      tws += 2 * Ns;
      line_sync(bar, TPL);
      C r = lf_rot(x2, f2.y, s2);
      C a0, a1, b0, b1;
      a0.x = fmaT(c2x, r.x, x0.x); a0.y = fmaT(c2, r.y, x0.y);
      a1.x = fmaT(-c2x, r.x, x0.x); a1.y = fmaT(-c2, r.y, x0.y);
      r = lf_rot(x3, f2.y, s2);
      b0.x = fmaT(c2x, r.x, x1.x); b0.y = fmaT(c2, r.y, x1.y);
      b1.x = fmaT(-c2x, r.x, x1.x); b1.y = fmaT(-c2, r.y, x1.y);
      r = lf_rot(b0, f1.y, s1);
      y0.x = fmaT(c1x, r.x, a0.x); y0.y = fmaT(c1, r.y, a0.y);
      y2.x = fmaT(-c1x, r.x, a0.x); y2.y = fmaT(-c1, r.y, a0.y);
      // y1 = a1 - i w b1, y3 = a1 + i w b1; -i (c R) = (c R.y, -(cx R.x))
      r = lf_rot(b1, f1.y, s1);
      y1.x = fmaT(c1, r.y, a1.x); y1.y = fmaT(-c1x, r.x, a1.y);
      y3.x = fmaT(-c1, r.y, a1.x); y3.y = fmaT(c1x, r.x, a1.y);
    } else {
      line_sync(bar, TPL);
      C a0, a1, b0, b1;
      a0.x = x0.x + x2.x; a0.y = x0.y + x2.y;
      a1.x = x0.x - x2.x; a1.y = x0.y - x2.y;
      b0.x = x1.x + x3.x; b0.y = x1.y + x3.y;
      b1.x = x1.x - x3.x; b1.y = x1.y - x3.y;
      y0.x = a0.x + b0.x; y0.y = a0.y + b0.y;
      y2.x = a0.x - b0.x; y2.y = a0.y - b0.y;
      // -i * b1 = (b1.y, -b1.x)
      y1.x = a1.x + b1.y; y1.y = a1.y - b1.x;
      y3.x = a1.x - b1.y; y3.y = a1.y + b1.x;
    }
    const int o = ((j - kk) << 2) + kk;
    c[o] = y0;
    c[o + Ns] = y1;
    c[o + 2 * Ns] = y2;
    c[o + 3 * Ns] = y3;
    line_sync(bar, TPL);
  }

  // 3. post-processing: F_k and F_{M-k} from C_k, C_{M-k}; even outputs in
  //    place, prefix-sum inputs Re F_k into the odd slots
  for (int k = lt; k <= (M >> 1); k += TPL) {
    if (k == 0) {
      C a = c[0];
      y[0] = (T)0;
      y[1] = a.x + a.y;
    } else if (k == (M >> 1)) {
      C a = c[k];
      y[2 * k] = (T)2 * a.y;
      y[2 * k + 1] = (T)2 * a.x;
    } else {
      C A = c[k], B = c[M - k];
      C E, D, O;
      E.x = A.x + B.x; E.y = A.y - B.y;
      D.x = A.x - B.x; D.y = A.y + B.y;
      O.x = D.y; O.y = -D.x;
      // Tt = exp(-2 pi i k/N) O = c R (factor table after the stages)
      const C f = tws[k];
      const bool sw = dst_swap_post(k, N);
      const C r = lf_rot(O, f.y, sw);
      const T cx = negif(f.x, sw);
      y[2 * k] = fmaT(-f.x, r.y, -E.y);
      y[2 * k + 1] = fmaT(cx, r.x, E.x);
      y[2 * (M - k)] = fmaT(-f.x, r.y, E.y);
      y[2 * (M - k) + 1] = fmaT(-cx, r.x, E.x);
    }
  }
  line_sync(bar, TPL);

  // 4. inclusive prefix sum over the odd slots: each thread owns 4 consecutive values
  T v0 = y[8 * lt + 1], v1 = y[8 * lt + 3], v2 = y[8 * lt + 5], v3 = y[8 * lt + 7];
  v1 += v0;
  v2 += v1;
  v3 += v2;
  const int lane = tid & 31;
  const int W = TPL < 32 ? TPL : 32;
  T x = v3;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    if (off < W) {
      T n = __shfl_up_sync(0xffffffffu, x, off, W);
      if ((lane & (W - 1)) >= off) x += n;
    }
  }
  T ex = __shfl_up_sync(0xffffffffu, x, 1, W);
  if ((lane & (W - 1)) == 0) ex = (T)0;
  if (TPL > 32) {
    // cross-warp: warp totals of this line, scanned by the line's first warp
    const int warp = tid >> 5;
    const int wpl = TPL >> 5;  // warps per line (<= 32)
    if (lane == 31) wsum[warp] = x;
    line_sync(bar, TPL);
    const int wl = warp - l * wpl;  // warp index within the line
    if (wl == 0) {
      T t = (lane < wpl) ? wsum[warp + lane] : (T)0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, t, off);
        if (lane >= off) t += n;
      }
      T te = __shfl_up_sync(0xffffffffu, t, 1);
      if (lane == 0) te = (T)0;
      if (lane < wpl) wsum[warp + lane] = te;
    }
    line_sync(bar, TPL);
    ex += wsum[warp];
  }
  y[8 * lt + 1] = v0 + ex;
  y[8 * lt + 3] = v1 + ex;
  y[8 * lt + 5] = v2 + ex;
  y[8 * lt + 7] = v3 + ex;
  __syncthreads();  // the callers' stores map threads across lines
}

// ---------------------------------------------------------------------------
// x axis: lines are rows (j, k) of the padded layout, contiguous in memory.
// LOAD 0: plain load of src.  LOAD 1 (2D): the u-equation right-hand side
// M(W) with W = V/alpha in src (W = 0 in the pad slots) plus the face
// values Q/alpha where M reaches the boundary; src must not alias dst.
// STORE 0: out = scale * X.  STORE 1: out = X * (1/alpha) at the point.
// ---------------------------------------------------------------------------
template <typename T>
struct DstIO {
  const T* src;
  const T* qa;          // LOAD 1: Q / alpha at the face points (precision T; may be NULL)
  const T* ainv;        // STORE 1: 1/alpha on the full grid; LOAD 1: if set, src holds V, not V/alpha
  T Mc, Mn;             // LOAD 1: weighting M
  const T* src2;        // LOAD 1: a source field added to M(W) (may be NULL)
  T lscale;             // LOAD 0: factor applied on load
};

// All arithmetic of the fused loads and stores is in T: on this GPU a single
// FP64 operation per element would bound an FP32 pass by the FP64 pipe.
template <typename T>
__device__ __forceinline__ T wval(const Geom& g, const DstIO<T>& io, int i, int j) {
  const T v = io.src[g.pad(i, j, 0)];
  return io.ainv ? v * io.ainv[g.full(i, j, 0)] : v;
}
template <typename T>
__device__ __forceinline__ T qval(const DstIO<T>& io, int64_t q) {
  return io.qa ? io.qa[q] : (T)0;
}

template <typename T>
__device__ __forceinline__ T mstencil2d(const Geom& g, const DstIO<T>& io, int i, int j) {
  const T acc = io.Mc * wval(g, io, i, j);
  T nb = 0;
  // x neighbours (i-1 = 0 and i+1 = N0 are faces x-/x+, holding Q)
  nb += (i > 1) ? wval(g, io, i - 1, j) : qval(io, g.face(0, 0, 0, j, 0));
  nb += (i < g.N[0] - 1) ? wval(g, io, i + 1, j) : qval(io, g.face(0, 1, g.N[0], j, 0));
  // y neighbours (faces y-/y+)
  nb += (j > 1) ? wval(g, io, i, j - 1) : qval(io, g.face(1, 0, i, 0, 0));
  nb += (j < g.N[1] - 1) ? wval(g, io, i, j + 1) : qval(io, g.face(1, 1, i, g.N[1], 0));
  T v = acc + io.Mn * nb;
  if (io.src2) v += io.src2[g.pad(i, j, 0)];
  return v;
}

// LOAD 2 (3D): M(W) with the seven-point weighting M; W = V/alpha in src
template <typename T>
__device__ __forceinline__ T mstencil3d(const Geom& g, const DstIO<T>& io, int i, int j, int k) {
  auto W = [&](int ii, int jj, int kk) { return io.src[g.pad(ii, jj, kk)]; };
  const T acc = io.Mc * W(i, j, k);
  T nb = 0;
  nb += (i > 1) ? W(i - 1, j, k) : qval(io, g.face(0, 0, 0, j, k));
  nb += (i < g.N[0] - 1) ? W(i + 1, j, k) : qval(io, g.face(0, 1, g.N[0], j, k));
  nb += (j > 1) ? W(i, j - 1, k) : qval(io, g.face(1, 0, i, 0, k));
  nb += (j < g.N[1] - 1) ? W(i, j + 1, k) : qval(io, g.face(1, 1, i, g.N[1], k));
  nb += (k > 1) ? W(i, j, k - 1) : qval(io, g.face(2, 0, i, j, 0));
  nb += (k < g.N[2] - 1) ? W(i, j, k + 1) : qval(io, g.face(2, 1, i, j, g.N[2]));
  T v = acc + io.Mn * nb;
  if (io.src2) v += io.src2[g.pad(i, j, k)];
  return v;
}

template <typename T, int LOAD, int STORE>
__global__ void __launch_bounds__(1024) k_dst_x(Geom g, T* __restrict__ a, DstIO<T> io,
                                               const typename Cplx<T>::t* __restrict__ tw,
                                               const T* __restrict__ sn, T scale, int logN, int TPL, int LPC) {
  const int bi = blockIdx.y;  // problem of the batch
  if (g.skip(bi)) return;
  a += (int64_t)bi * g.npad;
  if (io.src) io.src += (int64_t)bi * g.npad;
  if (io.src2) io.src2 += (int64_t)bi * g.npad;
  if (io.qa) io.qa += (int64_t)bi * g.ngamma;
  if (io.ainv) io.ainv += (int64_t)bi * g.nfull;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* wsum = s + (int64_t)LPC * g.n0;
  // per-line row data, computed once (no per-element division)
  int64_t* rbase = reinterpret_cast<int64_t*>(wsum + 32);
  int64_t* fbase = rbase + LPC;
  int* rj = reinterpret_cast<int*>(fbase + LPC);
  int* rk = rj + LPC;
  const int N = (int)g.n0;
  const int nj = g.N[1] - 1;
  const int nrows = nj * (g.kmax - g.kmin);
  const int r0 = blockIdx.x * LPC;
  for (int l = threadIdx.x; l < LPC; l += blockDim.x) {
    const int r = r0 + l;
    if (r < nrows) {
      const int j = 1 + r % nj, k = g.kmin + r / nj;
      rbase[l] = g.pad(0, j, k);
      fbase[l] = g.full(0, j, k);
      rj[l] = j;
      rk[l] = k;
    } else {
      rbase[l] = -1;
    }
  }
  __syncthreads();
  using C = typename Cplx<T>::t;
  const int tot2 = (LPC * N) >> 1;
  for (int e = threadIdx.x; e < tot2; e += blockDim.x) {
    const int l = (2 * e) >> logN;
    const int pos = (2 * e) & (N - 1);
    const int64_t rb = rbase[l];
    C v;
    v.x = 0;
    v.y = 0;
    if (rb >= 0) {
      if (LOAD == 0) {
        v = *reinterpret_cast<const C*>(io.src + rb + pos);
        if (io.lscale != (T)1) {  // uniform branch: no FP64 work for the common factor 1
          v.x *= io.lscale;
          v.y *= io.lscale;
        }
        if (pos == 0) v.x = 0;
      } else if (LOAD == 1) {
        const int j = rj[l];
        if (pos > 0) v.x = mstencil2d<T>(g, io, pos, j);
        v.y = mstencil2d<T>(g, io, pos + 1, j);
      } else {
        const int j = rj[l], k = rk[l];
        if (pos > 0) v.x = mstencil3d<T>(g, io, pos, j, k);
        v.y = mstencil3d<T>(g, io, pos + 1, j, k);
      }
    }
    *reinterpret_cast<C*>(s + l * N + pos) = v;
  }
  __syncthreads();
  dst_lines<T>(s, N, N, logN, TPL, tw, sn, wsum);
  for (int e = threadIdx.x; e < tot2; e += blockDim.x) {
    const int l = (2 * e) >> logN;
    const int pos = (2 * e) & (N - 1);
    const int64_t rb = rbase[l];
    if (rb >= 0) {
      C v = *reinterpret_cast<const C*>(s + l * N + pos);
      if (STORE == 0) {
        if (scale != (T)1) {
          v.x *= scale;
          v.y *= scale;
        }
      } else {
        const int64_t f = fbase[l] + pos;
        v.x *= io.ainv[f];
        v.y *= io.ainv[f + 1];
      }
      if (pos == 0) v.x = 0;
      *reinterpret_cast<C*>(a + rb + pos) = v;
    }
  }
}

// ---------------------------------------------------------------------------
// y axis (3D only): a CTA takes LPC adjacent x-columns of one z-plane; the
// columns are staged through shared memory so global accesses stay row-wise.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) k_dst_y(Geom g, T* __restrict__ a, const typename Cplx<T>::t* __restrict__ tw,
                                               const T* __restrict__ sn, T scale, int logN, int TPL, int LPC, int LS) {
  const int bi = blockIdx.z;
  if (g.skip(bi)) return;
  a += (int64_t)bi * g.npad;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* wsum = s + (int64_t)LPC * LS;
  const int N = g.N[1];
  const int i0 = blockIdx.x * LPC;
  const int k = g.kmin + blockIdx.y;
  const int tot = LPC * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int c = e % LPC;
    const int j = e / LPC;
    const int i = i0 + c;
    T v = 0;
    if (i < g.n0 && j > 0) v = a[g.pad(i, j, k)];
    s[c * LS + j] = v;
  }
  __syncthreads();
  dst_lines<T>(s, LS, N, logN, TPL, tw, sn, wsum);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int c = e % LPC;
    const int j = e / LPC;
    const int i = i0 + c;
    if (i < g.n0) a[g.pad(i, j, k)] = (j > 0) ? (scale != (T)1 ? s[c * LS + j] * scale : s[c * LS + j]) : (T)0;
  }
}

// ---------------------------------------------------------------------------
// Generic lines (face arrays): line l has N-1 elements at
//   base + (l / lpg) * gstride + (l % lpg) * lstride + (j - 1) * estride,  j = 1..N-1
// (the zero x_0 is implicit).  Used for the transverse DSTs of the boundary
// preconditioner on the face arrays.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_dst_gen(T* __restrict__ base, int nlines, int lpg, int64_t gstride,
                                                 int64_t lstride, int64_t estride, int N,
                                                 const typename Cplx<T>::t* __restrict__ tw, const T* __restrict__ sn,
                                                 int logN, int TPL, int LPC, int64_t bstride, const int* act) {
  if (act && !act[blockIdx.y]) return;
  base += (int64_t)blockIdx.y * bstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* wsum = s + (int64_t)LPC * N;
  const int l0 = blockIdx.x * LPC;
  const int tot = LPC * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN;
    const int j = e & (N - 1);
    const int line = l0 + l;
    T v = 0;
    if (j > 0 && line < nlines)
      v = base[(int64_t)(line / lpg) * gstride + (int64_t)(line % lpg) * lstride + (int64_t)(j - 1) * estride];
    s[e] = v;
  }
  __syncthreads();
  dst_lines<T>(s, N, N, logN, TPL, tw, sn, wsum);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN;
    const int j = e & (N - 1);
    const int line = l0 + l;
    if (j > 0 && line < nlines)
      base[(int64_t)(line / lpg) * gstride + (int64_t)(line % lpg) * lstride + (int64_t)(j - 1) * estride] = s[e];
  }
}

// ---------------------------------------------------------------------------
// Boundary preconditioner on 2D face lines in one pass: out = alpha *
// DST(pre * DST(in / alpha)) per line, the line kept in shared memory in
// precision T (FP32 is enough: GMRES is flexible, and stores P^-1 v).
// Line l holds N-1 contiguous face values at l * lstride; in and out may alias.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) k_precond_lines(double* out, const double* in, const double* __restrict__ afac,
                                                       const double* __restrict__ pre, int nlines, int64_t lstride,
                                                       int N, const typename Cplx<T>::t* __restrict__ tw,
                                                       const T* __restrict__ sn, int logN, int TPL, int LPC,
                                                       int64_t bstride, const int* act) {
  if (act && !act[blockIdx.y]) return;
  out += (int64_t)blockIdx.y * bstride;
  in += (int64_t)blockIdx.y * bstride;
  afac += (int64_t)blockIdx.y * bstride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* wsum = s + (int64_t)LPC * N;
  const int l0 = blockIdx.x * LPC;
  const int tot = LPC * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN, j = e & (N - 1), line = l0 + l;
    T v = 0;
    if (j > 0 && line < nlines) {
      const int64_t q = (int64_t)line * lstride + (j - 1);
      v = (T)(in[q] / afac[q]);
    }
    s[e] = v;
  }
  __syncthreads();
  dst_lines<T>(s, N, N, logN, TPL, tw, sn, wsum);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN, j = e & (N - 1), line = l0 + l;
    if (j > 0 && line < nlines) s[e] = (T)((double)s[e] * pre[(int64_t)line * lstride + (j - 1)]);
  }
  __syncthreads();
  dst_lines<T>(s, N, N, logN, TPL, tw, sn, wsum);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN, j = e & (N - 1), line = l0 + l;
    if (j > 0 && line < nlines) {
      const int64_t q = (int64_t)line * lstride + (j - 1);
      out[q] = (double)s[e] * afac[q];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// CTA size of the line DSTs when the tuner has not set one (measured on
// B300 with per-line barriers: 256 threads for the FP64 3D transforms, which
// are bound by the FP64 pipe, 512 otherwise)
template <typename T>
static inline int default_cta(const Geom& g) {
  return (sizeof(T) == 8 && g.dim == 3) ? 256 : 512;
}
static inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <typename T, int LOAD, int STORE>
static cudaError_t dst_x_impl(const Geom& g, T* dst, const DstIO<T>& io, const void* tw, const T* sn, T scale,
                              cudaStream_t st) {
  const int N = (int)g.n0;
  const int logN = ilog2(N);
  const int TPL = N / 8;
  const int cta = g.dst_cta ? g.dst_cta : default_cta<T>(g);
  const int LPC = TPL >= cta ? 1 : cta / TPL;
  const int threads = TPL * LPC;
  const int64_t nrows = (int64_t)(g.N[1] - 1) * (g.kmax - g.kmin);
  const int64_t blocks = (nrows + LPC - 1) / LPC;
  const size_t smem = ((size_t)LPC * N + 32) * sizeof(T) + (size_t)LPC * (2 * sizeof(int64_t) + 2 * sizeof(int));
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_dst_x<T, LOAD, STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_dst_x<T, LOAD, STORE><<<dim3((unsigned)blocks, (unsigned)g.nb), threads, smem, st>>>(
      g, dst, io, reinterpret_cast<const typename Cplx<T>::t*>(tw), sn, scale, logN, TPL, LPC);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dst_x(const Geom& g, T* a, const void* tw, const T* sn, T scale, cudaStream_t st) {
  DstIO<T> io{a, nullptr, nullptr, (T)0, (T)0, nullptr, (T)1};
  return dst_x_impl<T, 0, 0>(g, a, io, tw, sn, scale, st);
}

// dst = DST_x(lscale * src) (src may alias dst)
template <typename T>
cudaError_t launch_dst_x_from(const Geom& g, T* dst, const T* src, double lscale, const void* tw, const T* sn,
                              cudaStream_t st) {
  DstIO<T> io{src, nullptr, nullptr, (T)0, (T)0, nullptr, (T)lscale};
  return dst_x_impl<T, 0, 0>(g, dst, io, tw, sn, (T)1, st);
}
template cudaError_t launch_dst_x_from<float>(const Geom&, float*, const float*, double, const void*, const float*,
                                              cudaStream_t);
template cudaError_t launch_dst_x_from<double>(const Geom&, double*, const double*, double, const void*,
                                               const double*, cudaStream_t);

// in place, storing X / alpha (the inverse transform of V, giving W = V/alpha);
// ainv: 1/alpha on the full grid in precision T
template <typename T>
cudaError_t launch_dst_x_store_ainv(const Geom& g, T* a, const T* ainv, const void* tw, const T* sn,
                                    cudaStream_t st) {
  DstIO<T> io{a, nullptr, ainv, (T)0, (T)0, nullptr, (T)1};
  return dst_x_impl<T, 0, 1>(g, a, io, tw, sn, (T)1, st);
}

// dst = DST_x( M(W) + qa terms at the faces + src2 ), 2D, src = W must not alias dst
template <typename T>
cudaError_t launch_dst_x_mload(const Geom& g, T* dst, const T* W, const T* qa, T Mc, T Mn, const void* tw,
                               const T* sn, cudaStream_t st, const T* src2, const T* ainv_load) {
  DstIO<T> io{W, qa, ainv_load, Mc, Mn, src2, (T)1};
  return dst_x_impl<T, 1, 0>(g, dst, io, tw, sn, (T)1, st);
}

// dst = DST_x( M(W) + qa terms at the faces + src2 ), 3D, src = W must not alias dst
template <typename T>
cudaError_t launch_dst_x_mload3d(const Geom& g, T* dst, const T* W, const T* qa, T Mc, T Mn, const void* tw,
                                 const T* sn, cudaStream_t st, const T* src2) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  DstIO<T> io{W, qa, nullptr, Mc, Mn, src2, (T)1};
  return dst_x_impl<T, 2, 0>(g, dst, io, tw, sn, (T)1, st);
}
template cudaError_t launch_dst_x_mload3d<double>(const Geom&, double*, const double*, const double*, double, double,
                                                  const void*, const double*, cudaStream_t, const double*);
template cudaError_t launch_dst_x_mload3d<float>(const Geom&, float*, const float*, const float*, float, float,
                                                 const void*, const float*, cudaStream_t, const float*);

template cudaError_t launch_dst_x_store_ainv<double>(const Geom&, double*, const double*, const void*, const double*,
                                                     cudaStream_t);
template cudaError_t launch_dst_x_store_ainv<float>(const Geom&, float*, const float*, const void*, const float*,
                                                    cudaStream_t);
template cudaError_t launch_dst_x_mload<double>(const Geom&, double*, const double*, const double*, double, double,
                                                const void*, const double*, cudaStream_t, const double*,
                                                const double*);
template cudaError_t launch_dst_x_mload<float>(const Geom&, float*, const float*, const float*, float, float,
                                               const void*, const float*, cudaStream_t, const float*, const float*);

template <typename T>
cudaError_t launch_dst_y(const Geom& g, T* a, const void* tw, const T* sn, T scale, cudaStream_t st) {
  const int N = g.N[1];
  const int logN = ilog2(N);
  const int TPL = N / 8;
  const int cta = g.dst_cta ? g.dst_cta : default_cta<T>(g);
  int LPC = TPL >= cta ? 1 : cta / TPL;
  if (LPC > g.n0) LPC = (int)g.n0;
  const int threads = TPL * LPC;
  const int LS = N + (int)(16 / sizeof(T));
  dim3 grid((unsigned)((g.n0 + LPC - 1) / LPC), (unsigned)(g.kmax - g.kmin), (unsigned)g.nb);
  const size_t smem = ((size_t)LPC * LS + 32) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_dst_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_dst_y<T><<<grid, threads, smem, st>>>(g, a, reinterpret_cast<const typename Cplx<T>::t*>(tw), sn, scale, logN,
                                          TPL, LPC, LS);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dst_gen(T* base, int nlines, int lpg, int64_t gstride, int64_t lstride, int64_t estride, int N,
                           const void* tw, const T* sn, cudaStream_t st, int nb, int64_t bstride, const int* act) {
  const int logN = ilog2(N);
  const int TPL = N / 8;
  const int LPC = TPL >= 512 ? 1 : 512 / TPL;
  const int threads = TPL * LPC;
  const int blocks = (nlines + LPC - 1) / LPC;
  const size_t smem = ((size_t)LPC * N + 32) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_dst_gen<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_dst_gen<T><<<dim3(blocks, nb), threads, smem, st>>>(base, nlines, lpg, gstride, lstride, estride, N,
                                                         reinterpret_cast<const typename Cplx<T>::t*>(tw), sn, logN,
                                                         TPL, LPC, bstride, act);
  return cudaGetLastError();
}
template cudaError_t launch_dst_gen<double>(double*, int, int, int64_t, int64_t, int64_t, int, const void*,
                                            const double*, cudaStream_t, int, int64_t, const int*);
template cudaError_t launch_dst_gen<float>(float*, int, int, int64_t, int64_t, int64_t, int, const void*, const float*,
                                           cudaStream_t, int, int64_t, const int*);

template <typename T>
cudaError_t launch_precond_lines(double* out, const double* in, const double* afac, const double* pre, int nlines,
                                 int64_t lstride, int N, const void* tw, const T* sn, cudaStream_t st, int nb,
                                 int64_t bstride, const int* act) {
  const int logN = ilog2(N);
  const int TPL = N / 8;
  const int LPC = TPL >= 512 ? 1 : 512 / TPL;
  const int threads = TPL * LPC;
  const int blocks = (nlines + LPC - 1) / LPC;
  const size_t smem = ((size_t)LPC * N + 32) * sizeof(T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_precond_lines<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_precond_lines<T><<<dim3(blocks, nb), threads, smem, st>>>(out, in, afac, pre, nlines, lstride, N,
                                                               reinterpret_cast<const typename Cplx<T>::t*>(tw), sn,
                                                               logN, TPL, LPC, bstride, act);
  return cudaGetLastError();
}
template cudaError_t launch_precond_lines<float>(double*, const double*, const double*, const double*, int, int64_t,
                                                 int, const void*, const float*, cudaStream_t, int, int64_t,
                                                 const int*);
template cudaError_t launch_precond_lines<double>(double*, const double*, const double*, const double*, int, int64_t,
                                                  int, const void*, const double*, cudaStream_t, int, int64_t,
                                                  const int*);

template cudaError_t launch_dst_x<double>(const Geom&, double*, const void*, const double*, double, cudaStream_t);
template cudaError_t launch_dst_y<double>(const Geom&, double*, const void*, const double*, double, cudaStream_t);
template cudaError_t launch_dst_x<float>(const Geom&, float*, const void*, const float*, float, cudaStream_t);
template cudaError_t launch_dst_y<float>(const Geom&, float*, const void*, const float*, float, cudaStream_t);

}  // namespace ahoc
