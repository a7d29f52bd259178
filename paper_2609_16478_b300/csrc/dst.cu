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
//
// Shared-memory banks.  A stage reads its four inputs at stride M/4
// (consecutive threads, consecutive words) and writes its outputs in groups
// of Ns consecutive complex values, 4 Ns apart.  While a group is narrower
// than one wavefront (16 complex values in FP32, 8 in FP64) the four stores
// of a thread are issued in a rotated order, y_{(r+t)&3} in store r with t
// taken from the thread's group index, so that the groups of one wavefront
// land in distinct banks.  The post-processing leaves the even outputs in
// place and writes the odd outputs' summands to a contiguous buffer after
// the line, so that the prefix sum reads four consecutive values per thread
// as one vector.
#include <map>
#include <mutex>
#include <tuple>

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

// (a + zeta q, a - zeta q) and (a - i zeta q, a + i zeta q) for a factor
// zeta = (c, t, swap) as above: six FP operations per pair
template <typename C, typename T>
__device__ __forceinline__ void bfly(C a, C q, T c, T t, bool sw, C& u, C& v) {
  const C r = lf_rot(q, t, sw);
  const T cx = negif(c, sw);
  u.x = fmaT(cx, r.x, a.x);
  u.y = fmaT(c, r.y, a.y);
  v.x = fmaT(-cx, r.x, a.x);
  v.y = fmaT(-c, r.y, a.y);
}
template <typename C, typename T>
__device__ __forceinline__ void bfly_i(C a, C q, T c, T t, bool sw, C& u, C& v) {
  const C r = lf_rot(q, t, sw);
  const T cx = negif(c, sw);
  // -i (c R) = (c R.y, -(cx R.x))
  u.x = fmaT(c, r.y, a.x);
  u.y = fmaT(-cx, r.x, a.y);
  v.x = fmaT(-c, r.y, a.x);
  v.y = fmaT(cx, r.x, a.y);
}

// Rotation of the eight stores of a radix-8 stage with groups of Ns (as
// store_rot for radix 4): the group index bits that separate the groups of
// one wavefront (16 complex FP32 values, 8 FP64 values); 0 beyond.
template <typename T>
__device__ __forceinline__ int store_rot8(int j, int Ns) {
  if (sizeof(T) == 4) return Ns >= 16 ? 0 : ((j >> (Ns <= 2 ? 1 : (Ns == 4 ? 2 : 3))) & 7);
  return Ns >= 8 ? 0 : ((j >> (Ns == 1 ? 0 : (Ns == 2 ? 1 : 2))) & 7);
}

// Barrier of the threads of one line (see dst_lines): bar > 0 a named
// barrier of TPL threads, bar == 0 the CTA, bar < 0 the warp.
__device__ __forceinline__ void line_sync(int bar, int TPL) {
  if (bar > 0) asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(TPL) : "memory");
  else if (bar == 0) __syncthreads();
  else __syncwarp();
}

// Rotation of the four stores of a radix-4 stage with groups of Ns (see the
// file header): 0 where a group fills a wavefront (16 complex FP32 values
// or 8 FP64 values), else the group index bits that separate the groups of
// one wavefront.
template <typename T>
__device__ __forceinline__ int store_rot(int j, int Ns) {
  if (sizeof(T) == 4) return Ns >= 16 ? 0 : ((j >> (Ns == 8 ? 3 : 2)) & 3);
  return Ns >= 8 ? 0 : ((j >> (Ns == 4 ? 2 : 1)) & 3);
}

// four consecutive values at p (16-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 v = *reinterpret_cast<const double2*>(p), w = *reinterpret_cast<const double2*>(p + 2);
  a = v.x; b = v.y; c = w.x; d = w.y;
}
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}
// the two consecutive complex values (u, v) at p (radix-2 stage): one 16-byte
// store in FP32; two in FP64 (a 2-way conflict, hidden behind the FP64 pipe)
__device__ __forceinline__ void st_pair(float2* p, float2 u, float2 v, int) {
  *reinterpret_cast<float4*>(p) = make_float4(u.x, u.y, v.x, v.y);
}
__device__ __forceinline__ void st_pair(double2* p, double2 u, double2 v, int) {
  p[0] = u;
  p[1] = v;
}

// The pre-processing of one pair (j, N-j) (step 1 of dst_lines), for callers
// that fold it into their loads: z_j = (s_j + 1/4) x_j + (s_j - 1/4) x_{N-j}
// and z_{N-j} the other way round; the middle pair (j = N/2) also clears the
// slot y[0] (x_0 = 0).
template <typename T>
__device__ __forceinline__ void dst_pre_pair(T* y, int N, int j, T xa, T xb, const typename Cplx<T>::t* __restrict__ tw) {
  const typename Cplx<T>::t f = tw[N + j];
  y[j] = fmaT(f.x, xa, f.y * xb);
  if (j != (N >> 1)) y[N - j] = fmaT(f.y, xa, f.x * xb);
  else y[0] = (T)0;
}

// In-place DST-I of the LPC lines of this CTA.  Line l occupies s[l*LS .. l*LS+N)
// with s[l*LS] == 0, followed by N/2 elements of scratch (LS >= 3N/2); s and
// LS * sizeof(T) are multiples of 16 bytes.  With `pre_done` the lines hold
// the pre-processed z (dst_pre_pair) instead of x.  The output is in natural
// order when `natural`; otherwise X_j is at y[j] for even j and X_{2m+1} at
// y[N + m].  Every thread of the CTA must call this.  wsum: >= 32 elements
// of scratch for the cross-warp scan.
template <typename T, bool R8 = false>
__device__ void dst_lines(T* s, int LS, int N, int logN, int TPL, const typename Cplx<T>::t* __restrict__ tw,
                          const T* __restrict__ sn, T* wsum, bool natural = false, bool pre_done = false) {
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
  if (!pre_done) {
    const C* pm = tw + N;
    for (int j = lt + 1; j <= (N >> 1); j += TPL) {
      const T a = y[j], b = y[N - j];
      const C f = pm[j];
      y[j] = fmaT(f.x, a, f.y * b);
      if (j != (N >> 1)) y[N - j] = fmaT(f.y, a, f.x * b);
    }
    line_sync(bar, TPL);
  }

  // 2. complex FFT of length M (Stockham, natural order in and out): radix-4
  //    stages (one radix-2 stage first when log2 M is odd), or radix-8 stages
  //    after one radix-2 or radix-4 stage when log2 M is not a multiple of 3
  constexpr bool r8 = R8;
  int Ns = 1;
  if (r8 ? (logM % 3 == 1) : (logM & 1)) {
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
      st_pair(c + 2 * j, u, v, j);
    }
    line_sync(bar, TPL);
    Ns = 2;
  }
  const int M4 = M >> 2;
  // stage factors w = W^kk and w^2, W = exp(-2 pi i/(4 Ns)), contiguous in kk
  const C* tws = tw + N + (N >> 1) + 1;
  // radix-4 stages: all of them, or the one without twiddles before radix 8
  const int r4end = r8 ? ((logM % 3 == 2) ? 4 : Ns) : M;
  for (; Ns < r4end; Ns <<= 2) {
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
    const int t = store_rot<T>(j, Ns);
    if ((sizeof(T) == 4 && Ns < 16) || (sizeof(T) == 8 && Ns < 8)) {  // uniform over the CTA
      // z_r = y_{(r+t)&3}: rotate by 2 when t & 2, then by 1 when t & 1
      const bool h = t & 2, q1 = t & 1;
      const C a0 = h ? y2 : y0, a1 = h ? y3 : y1, a2 = h ? y0 : y2, a3 = h ? y1 : y3;
      const C z0 = q1 ? a1 : a0, z1 = q1 ? a2 : a1, z2 = q1 ? a3 : a2, z3 = q1 ? a0 : a3;
      c[o + (t & 3) * Ns] = z0;
      c[o + ((t + 1) & 3) * Ns] = z1;
      c[o + ((t + 2) & 3) * Ns] = z2;
      c[o + ((t + 3) & 3) * Ns] = z3;
    } else {
      c[o] = y0;
      c[o + Ns] = y1;
      c[o + 2 * Ns] = y2;
      c[o + 3 * Ns] = y3;
    }
    line_sync(bar, TPL);
  }

  if constexpr (R8) {
    // radix-8 stages: M/8 butterflies, on the first half of the line's threads
    const C* t8 = tw + dst_tw_len_r4(N);
    const int M8 = M >> 3;
    for (; Ns < M; Ns <<= 3) {
      const int j = lt;
      const bool on = j < M8;
      const int kk = j & (Ns - 1);
      C x0, x1, x2, x3, x4, x5, x6, x7;
      if (on) {
        x0 = c[j]; x1 = c[j + M8]; x2 = c[j + 2 * M8]; x3 = c[j + 3 * M8];
        x4 = c[j + 4 * M8]; x5 = c[j + 5 * M8]; x6 = c[j + 6 * M8]; x7 = c[j + 7 * M8];
      }
      line_sync(bar, TPL);
      if (on) {
        // y_r = sum_m W8^{rm} w^m x_m, r = r0 + 2 r1 + 4 r2, in three radix-2 layers:
        // over m's high bit with w^4, its middle bit with (-i)^r0 w^2, its low bit
        // with (-i)^r1 w (r0 = 0) or (-i)^r1 w e^{-i pi/4} (r0 = 1)
        const C f1 = t8[kk], f2 = t8[Ns + kk], f4 = t8[2 * Ns + kk], f5 = t8[3 * Ns + kk];
        const bool s2 = dst_swap_w1(kk, Ns), s4 = dst_swap_w2(kk, Ns), s5 = kk > 0;
        C a00, a01, a02, a03, a10, a11, a12, a13;
        bfly(x0, x4, f4.x, f4.y, s4, a00, a10);
        bfly(x1, x5, f4.x, f4.y, s4, a01, a11);
        bfly(x2, x6, f4.x, f4.y, s4, a02, a12);
        bfly(x3, x7, f4.x, f4.y, s4, a03, a13);
        C b000, b001, b010, b011, b100, b101, b110, b111;
        bfly(a00, a02, f2.x, f2.y, s2, b000, b010);
        bfly(a01, a03, f2.x, f2.y, s2, b001, b011);
        bfly_i(a10, a12, f2.x, f2.y, s2, b100, b110);
        bfly_i(a11, a13, f2.x, f2.y, s2, b101, b111);
        C y0, y1, y2, y3, y4, y5, y6, y7;
        bfly(b000, b001, f1.x, f1.y, false, y0, y4);
        bfly_i(b010, b011, f1.x, f1.y, false, y2, y6);
        bfly(b100, b101, f5.x, f5.y, s5, y1, y5);
        bfly_i(b110, b111, f5.x, f5.y, s5, y3, y7);
        const int o = ((j - kk) << 3) + kk;
        const int t = store_rot8<T>(j, Ns);
        if (t == 0 && ((sizeof(T) == 4 && Ns >= 16) || (sizeof(T) == 8 && Ns >= 8))) {
          c[o] = y0; c[o + Ns] = y1; c[o + 2 * Ns] = y2; c[o + 3 * Ns] = y3;
          c[o + 4 * Ns] = y4; c[o + 5 * Ns] = y5; c[o + 6 * Ns] = y6; c[o + 7 * Ns] = y7;
        } else {
          // z_r = y_{(r+t)&7}: rotate by 4, 2, 1 as the bits of t say
          const bool h4 = t & 4, h2 = t & 2, h1 = t & 1;
          C z0 = h4 ? y4 : y0, z1 = h4 ? y5 : y1, z2 = h4 ? y6 : y2, z3 = h4 ? y7 : y3;
          C z4 = h4 ? y0 : y4, z5 = h4 ? y1 : y5, z6 = h4 ? y2 : y6, z7 = h4 ? y3 : y7;
          C w0 = h2 ? z2 : z0, w1 = h2 ? z3 : z1, w2 = h2 ? z4 : z2, w3 = h2 ? z5 : z3;
          C w4 = h2 ? z6 : z4, w5 = h2 ? z7 : z5, w6 = h2 ? z0 : z6, w7 = h2 ? z1 : z7;
          z0 = h1 ? w1 : w0; z1 = h1 ? w2 : w1; z2 = h1 ? w3 : w2; z3 = h1 ? w4 : w3;
          z4 = h1 ? w5 : w4; z5 = h1 ? w6 : w5; z6 = h1 ? w7 : w6; z7 = h1 ? w0 : w7;
          c[o + (t & 7) * Ns] = z0;
          c[o + ((t + 1) & 7) * Ns] = z1;
          c[o + ((t + 2) & 7) * Ns] = z2;
          c[o + ((t + 3) & 7) * Ns] = z3;
          c[o + ((t + 4) & 7) * Ns] = z4;
          c[o + ((t + 5) & 7) * Ns] = z5;
          c[o + ((t + 6) & 7) * Ns] = z6;
          c[o + ((t + 7) & 7) * Ns] = z7;
        }
      }
      t8 += 4 * Ns;
      line_sync(bar, TPL);
    }
    // the post-processing factors follow the whole radix-4 stage layout
    tws = tw + dst_tw_len_r4(N) - ((M >> 1) + 1);
  }

  // 3. post-processing: F_k and F_{M-k} from C_k, C_{M-k}; the even outputs
  //    in place, the prefix-sum summands Re F_k to Pb[k] = y[N + k]
  T* Pb = y + N;
  for (int k = lt; k <= (M >> 1); k += TPL) {
    if (k == 0) {
      C a = c[0];
      y[0] = (T)0;
      Pb[0] = a.x + a.y;
    } else if (k == (M >> 1)) {
      C a = c[k];
      y[2 * k] = (T)2 * a.y;
      Pb[k] = (T)2 * a.x;
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
      Pb[k] = fmaT(cx, r.x, E.x);
      y[2 * (M - k)] = fmaT(-f.x, r.y, E.y);
      Pb[M - k] = fmaT(-cx, r.x, E.x);
    }
  }
  line_sync(bar, TPL);

  // 4. inclusive prefix sum of the summands Pb[0 .. M): each thread owns 4
  //    consecutive values, read and written as one vector
  T* P = Pb + 4 * lt;
  T v0, v1, v2, v3;
  ld4(P, v0, v1, v2, v3);
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
  st4(P, v0 + ex, v1 + ex, v2 + ex, v3 + ex);
  if (natural) {  // uniform: the odd outputs to their slots
    line_sync(bar, TPL);
#pragma unroll
    for (int q = 0; q < 4; ++q) y[2 * (lt + q * TPL) + 1] = Pb[lt + q * TPL];
  }
  __syncthreads();  // the callers' stores map threads across lines
}

// ---------------------------------------------------------------------------
// x axis: lines are rows (j, k) of the padded layout, contiguous in memory.
// LOAD 0: plain load of src.  LOAD 1 (2D): the u-equation right-hand side
// M(W) with W = V/alpha in src (W = 0 in the pad slots) plus the face
// values Q/alpha where M reaches the boundary; src must not alias dst.
// STORE 0: out = X.  STORE 1: out = X * (1/alpha) at the point.  STORE 2:
// out = scale * X (a separate instantiation: a branch on the factor costs
// predicated FP64 multiplies even when it is 1).
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

// A CTA transforms LPC rows.  Each thread loads the pairs (x_j, x_{N-j}) of
// its slots and stores their pre-processed values (dst_pre_pair), so the
// transform starts at the FFT.
// radix-8 CTAs take at most 512 threads (the registers of an eight-point butterfly)
template <typename T, int LOAD, int STORE, bool R8>
__global__ void __launch_bounds__(R8 ? 512 : 1024) k_dst_x(Geom g, T* __restrict__ a, DstIO<T> io,
                                                          const typename Cplx<T>::t* __restrict__ tw,
                                                          const T* __restrict__ sn, T scale, int logN, int TPL,
                                                          int LPC) {
  const int bi = blockIdx.y;  // problem of the batch
  if (g.skip(bi)) return;
  a += (int64_t)bi * g.npad;
  if (io.src) io.src += (int64_t)bi * g.npad;
  if (io.src2) io.src2 += (int64_t)bi * g.npad;
  if (io.qa) io.qa += (int64_t)bi * g.ngamma;
  if (io.ainv) io.ainv += (int64_t)bi * g.nfull;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int N = (int)g.n0;
  const int LS = N + (N >> 1);  // the line and its scan buffer
  T* wsum = s + (int64_t)LPC * LS;
  // per-line row data, computed once (no per-element division)
  int64_t* rbase = reinterpret_cast<int64_t*>(wsum + 32);
  int64_t* fbase = rbase + LPC;
  int* rj = reinterpret_cast<int*>(fbase + LPC);
  int* rk = rj + LPC;
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
  const int half = N >> 1;
  if (LOAD == 0) {
    // plain rows: the pairs (x_j, x_{N-j}), pre-processed on the way in
    for (int e = threadIdx.x; e < LPC * half; e += blockDim.x) {
      const int l = e >> (logN - 1), j = (e & (half - 1)) + 1;
      const int64_t rb = rbase[l];
      T xa = 0, xb = 0;
      if (rb >= 0) {
        xa = io.src[rb + j];
        xb = io.src[rb + N - j];
        if (io.lscale != (T)1) {  // uniform branch: no FP64 work for the common factor 1
          xa *= io.lscale;
          xb *= io.lscale;
        }
      }
      dst_pre_pair<T>(s + l * LS, N, j, xa, xb, tw);
    }
  } else {
    // stencil loads (the weighting M at two neighbouring points per thread;
    // pairs (j, N-j) would hold two stencils' operands in registers)
    for (int e = threadIdx.x; e < LPC * half; e += blockDim.x) {
      const int l = (2 * e) >> logN;
      const int pos = (2 * e) & (N - 1);
      C v;
      v.x = 0;
      v.y = 0;
      if (rbase[l] >= 0) {
        if (LOAD == 1) {
          const int j = rj[l];
          if (pos > 0) v.x = mstencil2d<T>(g, io, pos, j);
          v.y = mstencil2d<T>(g, io, pos + 1, j);
        } else {
          const int j = rj[l], k = rk[l];
          if (pos > 0) v.x = mstencil3d<T>(g, io, pos, j, k);
          v.y = mstencil3d<T>(g, io, pos + 1, j, k);
        }
      }
      *reinterpret_cast<C*>(s + l * LS + pos) = v;
    }
  }
  __syncthreads();
  dst_lines<T, R8>(s, LS, N, logN, TPL, tw, sn, wsum, false, LOAD == 0);
  const int tot2 = LPC * half;
  for (int e = threadIdx.x; e < tot2; e += blockDim.x) {
    const int l = (2 * e) >> logN;
    const int pos = (2 * e) & (N - 1);
    const int64_t rb = rbase[l];
    if (rb >= 0) {
      const T* yl = s + l * LS;  // X_pos at yl[pos], X_{pos+1} at yl[N + pos/2]
      C v;
      v.x = yl[pos];
      v.y = yl[N + (pos >> 1)];
      if (STORE == 2) {
        v.x *= scale;
        v.y *= scale;
      } else if (STORE == 1) {
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
__device__ __forceinline__ void dsty_fetch(const Geom& g, const T* __restrict__ a, int grp, int ncb, int LPC, int N,
                                           T (&pa)[4], T (&pb)[4]) {
  const int i0 = (grp % ncb) * LPC, k = g.kmin + grp / ncb;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    const int c = e % LPC, j = e / LPC + 1;
    const int i = i0 + c;
    pa[q] = (T)0;
    pb[q] = (T)0;
    if (i < g.n0) {
      pa[q] = a[g.pad(i, j, k)];
      pb[q] = a[g.pad(i, N - j, k)];
    }
  }
}

// A group is LPC adjacent columns of one plane (ncb column blocks per
// plane); each thread owns four (column, pair) slots, as in k_dst_x, and the
// next group's loads are in flight during the current transform.
template <typename T, bool R8, bool SC>
__global__ void __launch_bounds__(R8 ? 512 : 1024) k_dst_y(Geom g, T* __restrict__ a,
                                                          const typename Cplx<T>::t* __restrict__ tw,
                                                          const T* __restrict__ sn, T scale, int logN, int TPL,
                                                          int LPC, int LS) {
  const int bi = blockIdx.y;
  if (g.skip(bi)) return;
  a += (int64_t)bi * g.npad;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* wsum = s + (int64_t)LPC * LS;
  const int N = g.N[1];
  const int ncb = (int)((g.n0 + LPC - 1) / LPC);
  const int ngroups = ncb * (g.kmax - g.kmin);
  constexpr bool PREF = sizeof(T) == 4;  // register prefetch of the next group (FP32; FP64 is pipe-bound)
  T pa[4], pb[4];
  if constexpr (PREF) {
    if ((int)blockIdx.x < ngroups) dsty_fetch<T>(g, a, blockIdx.x, ncb, LPC, N, pa, pb);
  }
  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int i0 = (grp % ncb) * LPC, k = g.kmin + grp / ncb;
    __syncthreads();  // the previous group's stores have read s
    if constexpr (PREF) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        const int c = e % LPC, j = e / LPC + 1;
        dst_pre_pair<T>(s + c * LS, N, j, pa[q], pb[q], tw);
      }
      if (grp + (int)gridDim.x < ngroups) dsty_fetch<T>(g, a, grp + gridDim.x, ncb, LPC, N, pa, pb);
    } else {
      // FP64: plain loads, the pre-processing inside the transform
      for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
        const int c = e % LPC, j = e / LPC;
        const int i = i0 + c;
        s[c * LS + j] = (i < g.n0 && j > 0) ? a[g.pad(i, j, k)] : (T)0;
      }
    }
    __syncthreads();
    dst_lines<T, R8>(s, LS, N, logN, TPL, tw, sn, wsum, false, PREF);
    // X_{2m} at 2m, X_{2m+1} at N + m of each column
#pragma unroll(PREF ? 4 : 1)
    for (int e = threadIdx.x; e < LPC * (N >> 1); e += blockDim.x) {
      const int c = e % LPC, m = e / LPC;
      const int i = i0 + c;
      if (i < g.n0) {
        T xe = s[c * LS + 2 * m], xo = s[c * LS + N + m];
        if (SC) {  // a separate instantiation: no FP64 work per element for the common factor 1
          xe *= scale;
          xo *= scale;
        }
        a[g.pad(i, 2 * m, k)] = (m > 0) ? xe : (T)0;
        a[g.pad(i, 2 * m + 1, k)] = xo;
      }
    }
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
  const int LS = N + N / 2;
  T* wsum = s + (int64_t)LPC * LS;
  const int l0 = blockIdx.x * LPC;
  const int tot = LPC * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN;
    const int j = e & (N - 1);
    const int line = l0 + l;
    T v = 0;
    if (j > 0 && line < nlines)
      v = base[(int64_t)(line / lpg) * gstride + (int64_t)(line % lpg) * lstride + (int64_t)(j - 1) * estride];
    s[l * LS + j] = v;
  }
  __syncthreads();
  dst_lines<T>(s, LS, N, logN, TPL, tw, sn, wsum, true);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN;
    const int j = e & (N - 1);
    const int line = l0 + l;
    if (j > 0 && line < nlines)
      base[(int64_t)(line / lpg) * gstride + (int64_t)(line % lpg) * lstride + (int64_t)(j - 1) * estride] =
          s[l * LS + j];
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
  const int LS = N + N / 2;
  T* wsum = s + (int64_t)LPC * LS;
  const int l0 = blockIdx.x * LPC;
  const int tot = LPC * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN, j = e & (N - 1), line = l0 + l;
    T v = 0;
    if (j > 0 && line < nlines) {
      const int64_t q = (int64_t)line * lstride + (j - 1);
      v = (T)(in[q] / afac[q]);
    }
    s[l * LS + j] = v;
  }
  __syncthreads();
  dst_lines<T>(s, LS, N, logN, TPL, tw, sn, wsum, true);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN, j = e & (N - 1), line = l0 + l;
    if (j > 0 && line < nlines) s[l * LS + j] = (T)((double)s[l * LS + j] * pre[(int64_t)line * lstride + (j - 1)]);
  }
  __syncthreads();
  dst_lines<T>(s, LS, N, logN, TPL, tw, sn, wsum, true);
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int l = e >> logN, j = e & (N - 1), line = l0 + l;
    if (j > 0 && line < nlines) {
      const int64_t q = (int64_t)line * lstride + (j - 1);
      out[q] = (double)s[l * LS + j] * afac[q];
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
// FFT radix of the line DSTs when the tuner has not set one
template <typename T>
static inline int dst_radix(const Geom& g) {
  return g.dst_radix ? g.dst_radix : 4;
}
static inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Dynamic shared memory above the 48 KB default: the kernel's limit is raised
// once, to the device's opt-in maximum, not to each launch's size.  A launch
// captured in a CUDA graph keeps its size; a later launch of the same kernel
// with a smaller size must not lower the limit under it.  Cached per device
// and kernel.
static cudaError_t allow_smem(const void* kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({dev, kernel});
  if (it != done.end()) return (size_t)it->second >= smem ? cudaSuccess : cudaErrorInvalidValue;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if ((size_t)optin < smem) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e != cudaSuccess) return e;
  done[{dev, kernel}] = optin;
  return cudaSuccess;
}

// CTAs of one launch of a grid-stride line kernel (k_dst_y in FP32): its
// groups of lines, but no more than the device holds resident at once
// (occupancy x SMs, shared by the nb problems of a batch), so that every CTA
// loops and prefetches.
// Cached per device, kernel and launch shape.
static int stride_ctas(const void* kernel, int threads, size_t smem, int64_t groups, int nb) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const auto key = std::make_tuple(dev, kernel, threads, smem);
  int resident = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) resident = it->second;
  }
  if (!resident) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) per_sm = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
    resident = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = resident;
  }
  int64_t b = resident / (nb > 0 ? nb : 1);
  if (b < 1) b = 1;
  return (int)(b < groups ? b : groups);
}

template <typename T, int LOAD, int STORE, bool R8>
static cudaError_t dst_x_launch(const Geom& g, T* dst, const DstIO<T>& io, const void* tw, const T* sn, T scale,
                                cudaStream_t st) {
  const int N = (int)g.n0;
  const int logN = ilog2(N);
  const int TPL = N / 8;
  int cta = g.dst_cta ? g.dst_cta : default_cta<T>(g);
  if (R8 && cta > 512) cta = 512;
  const int LPC = TPL >= cta ? 1 : cta / TPL;
  const int threads = TPL * LPC;
  if (R8 && threads > 512) return cudaErrorInvalidConfiguration;  // N = 8192 lines are not offered
  const int64_t nrows = (int64_t)(g.N[1] - 1) * (g.kmax - g.kmin);
  const int64_t blocks = (nrows + LPC - 1) / LPC;
  const size_t smem =
      ((size_t)LPC * (N + N / 2) + 32) * sizeof(T) + (size_t)LPC * (2 * sizeof(int64_t) + 2 * sizeof(int));
  {
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_dst_x<T, LOAD, STORE, R8>), smem);
    if (e != cudaSuccess) return e;
  }
  k_dst_x<T, LOAD, STORE, R8><<<dim3((unsigned)blocks, (unsigned)g.nb), threads, smem, st>>>(
      g, dst, io, reinterpret_cast<const typename Cplx<T>::t*>(tw), sn, scale, logN, TPL, LPC);
  return cudaGetLastError();
}
template <typename T, int LOAD, int STORE>
static cudaError_t dst_x_impl(const Geom& g, T* dst, const DstIO<T>& io, const void* tw, const T* sn, T scale,
                              cudaStream_t st) {
  if constexpr (LOAD == 0 && STORE == 0) {
    if (scale != (T)1)
      return dst_radix<T>(g) == 8 ? dst_x_launch<T, 0, 2, true>(g, dst, io, tw, sn, scale, st)
                                  : dst_x_launch<T, 0, 2, false>(g, dst, io, tw, sn, scale, st);
  }
  return dst_radix<T>(g) == 8 ? dst_x_launch<T, LOAD, STORE, true>(g, dst, io, tw, sn, scale, st)
                              : dst_x_launch<T, LOAD, STORE, false>(g, dst, io, tw, sn, scale, st);
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

template <typename T, bool R8, bool SC>
static cudaError_t dst_y_launch(const Geom& g, T* a, const void* tw, const T* sn, T scale, cudaStream_t st) {
  const int N = g.N[1];
  const int logN = ilog2(N);
  const int TPL = N / 8;
  int cta = g.dst_cta ? g.dst_cta : default_cta<T>(g);
  if (R8 && cta > 512) cta = 512;
  int LPC = TPL >= cta ? 1 : cta / TPL;
  if (LPC > g.n0) LPC = (int)g.n0;
  const int threads = TPL * LPC;
  if (R8 && threads > 512) return cudaErrorInvalidConfiguration;
  // line, scan buffer and a bank offset: the LPC columns of one wavefront
  // (128 / sizeof(T) words) start in distinct banks; LS * sizeof(T) stays a
  // multiple of 16 bytes
  int off = (int)(128 / sizeof(T)) / LPC;
  if (off < (int)(16 / sizeof(T))) off = (int)(16 / sizeof(T));
  const int LS = N + N / 2 + off;
  const size_t smem = ((size_t)LPC * LS + 32) * sizeof(T);
  {
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_dst_y<T, R8, SC>), smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t groups = ((g.n0 + LPC - 1) / LPC) * (int64_t)(g.kmax - g.kmin);
  // FP32: grid-stride CTAs with the next group's loads in flight; FP64 (bound
  // by the FP64 pipe): one CTA per group
  const int nx = sizeof(T) == 4 ? stride_ctas(reinterpret_cast<const void*>(k_dst_y<T, R8, SC>), threads, smem, groups,
                                              g.nb)
                                : (int)groups;
  k_dst_y<T, R8, SC><<<dim3((unsigned)nx, (unsigned)g.nb), threads, smem, st>>>(
      g, a, reinterpret_cast<const typename Cplx<T>::t*>(tw), sn, scale, logN, TPL, LPC, LS);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dst_y(const Geom& g, T* a, const void* tw, const T* sn, T scale, cudaStream_t st) {
  const bool sc = scale != (T)1;
  if (dst_radix<T>(g) == 8)
    return sc ? dst_y_launch<T, true, true>(g, a, tw, sn, scale, st) : dst_y_launch<T, true, false>(g, a, tw, sn, scale, st);
  return sc ? dst_y_launch<T, false, true>(g, a, tw, sn, scale, st) : dst_y_launch<T, false, false>(g, a, tw, sn, scale, st);
}

template <typename T>
cudaError_t launch_dst_gen(T* base, int nlines, int lpg, int64_t gstride, int64_t lstride, int64_t estride, int N,
                           const void* tw, const T* sn, cudaStream_t st, int nb, int64_t bstride, const int* act) {
  const int logN = ilog2(N);
  const int TPL = N / 8;
  const int LPC = TPL >= 512 ? 1 : 512 / TPL;
  const int threads = TPL * LPC;
  const int blocks = (nlines + LPC - 1) / LPC;
  const size_t smem = ((size_t)LPC * (N + N / 2) + 32) * sizeof(T);
  {
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_dst_gen<T>), smem);
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
  const size_t smem = ((size_t)LPC * (N + N / 2) + 32) * sizeof(T);
  {
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_precond_lines<T>), smem);
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
