// Shared definitions of the augmented HOC library (device + host).
//
// Internal field layout ("padded interior"): an array of N0 x N1 (x N2)
// elements, x fastest, holding grid point (i, j, k) with 1 <= i <= N_a - 1 at
// offset i + N0 * (j + N1 * k).  The slots with an index 0 are padding and
// stay zero; along a line they are the zero x_0 of the DST-I input, so every
// line is N elements long and 16-byte aligned.  In 2D there is one layer
// k = 0 (no z padding).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ahoc {

constexpr int kMaxN = 4096;

struct Geom {
  int dim;
  int N[3];           // intervals per axis (N[2] = 1 in 2D)
  double h[3];
  int64_t n0, n1, n2; // padded extents (N0, N1, N2 or 1)
  int64_t npad;       // n0 * n1 * n2
  int64_t f0, f1, f2; // full-grid extents N + 1 (f2 = 1 in 2D)
  int64_t nfull;
  int64_t face_off[7];
  int64_t ngamma;
  int kmin, kmax;     // layers holding interior points: 3D [1, N2), 2D [0, 1)
  int64_t nint;       // interior points
  // Batch of nb problems of this shape: every per-problem array holds nb
  // copies back to back (fields npad apart, full-grid arrays nfull apart,
  // face arrays ngamma apart); kernels take the problem from a grid
  // dimension.  act (device, nb flags; NULL = all) masks problems out of a
  // launch: their blocks return at once.
  int nb;
  const int* act;
  int navier;  // bit 2a + side: Navier face (v = alpha g_L is data); other faces clamped
  int triL;     // rows per chunk of the chunked tridiagonal solve (0: default)
  int dst_cta;  // threads per CTA of the line DSTs along x and y (0: default 512)
  int dst_radix;  // FFT radix of the line DSTs along x and y: 4 or 8 (0: default)

  __host__ __device__ inline bool is_navier(int face_id) const { return (navier >> face_id) & 1; }

  __host__ __device__ inline bool skip(int b) const { return act != nullptr && act[b] == 0; }

  __host__ __device__ inline int64_t pad(int i, int j, int k) const { return i + n0 * (j + n1 * (int64_t)k); }
  __host__ __device__ inline int64_t full(int i, int j, int k) const { return i + f0 * (j + f1 * (int64_t)k); }
  // index of a face point within the face arrays (axis a on the boundary)
  __host__ __device__ inline int64_t face(int a, int side, int i, int j, int k) const {
    int64_t o = face_off[2 * a + side];
    if (a == 0) return o + (j - 1) + (int64_t)(N[1] - 1) * (dim == 3 ? (k - 1) : 0);
    if (a == 1) return o + (i - 1) + (int64_t)(N[0] - 1) * (dim == 3 ? (k - 1) : 0);
    return o + (i - 1) + (int64_t)(N[0] - 1) * (j - 1);
  }
};

// Stencil coefficients for one plan (anisotropic h).  L is indexed
// (dz+1)*9 + (dy+1)*3 + (dx+1); in 2D only the dz = 0 plane is used.
struct Coefs {
  double L[27];
  double Mc, Mn;          // weighting M: centre and each axis neighbour
  double w[3][4];         // one-sided u_nn weights on U0..U3 per normal axis (1/h^2 scaled)
  double wg[3];           // weight on g_N per normal axis (11/(3h))
  double gam;             // constant beta / alpha: the v-equation is -L_h V + gam M V = M f
  double fsign;           // sign of M f in the right-hand side of the equation solved first:
                          // -1 for the v-equation (-L_h V = M f), +1 for the triharmonic w-equation
  // triharmonic class: one-sided fourth normal derivative at a clamped face,
  // u_ssss ~ sum_m w4[a][m] U_m + w4s[a] u_s + w4ss[a] u_ss (s the inward normal)
  double w4[3][5], w4s[3], w4ss[3];
};

// Per-mode factors of the tridiagonal solve along the last axis (see tri.cu).
template <typename T>
struct alignas(16) Mode {
  T r, rinv, s, kap, rj0;
  T kapC;  // -r / (1 - r^(2N)): coefficient of the boundary correction r^j - r^(2N-j)
  T q1;    // 1 - r, rounded on its own: r x is formed as x - q1 x, so the effective r
           // of the slowest modes (r close to 1) keeps full relative accuracy
  int j0;
};

// DST twiddle table for lines of N points, in entries of two reals:
//   [0, N)           tw[t] = exp(-2 pi i t/N)
//   [N, N + N/2 + 1) pre-processing factors (sin(pi j/N)/2 + 1/4, sin(pi j/N)/2 - 1/4)
//   then per radix-4 stage with Ns > 1 of the N/2-point FFT (Ns = 2 or 4,
//   then x4 up to N/8): Ns entries (c, t) of w = W^kk, then Ns of w^2
//   (W = exp(-2 pi i/(4 Ns))), contiguous in kk so a warp reads consecutive
//   entries; then N/4 + 1 entries (c, t) of exp(-2 pi i k/N), k <= N/4, for the
//   post-processing.
// A factor zeta = exp(i theta) is held as (c, t) with zeta = c (1 + i t), or,
// where the swap rule of dst_swap_* holds, zeta = i c (1 + i t); either way
// |t| <= 1, and zeta q costs two FMAs plus a scaling that the butterfly's
// additions absorb into FMAs.
__host__ __device__ inline bool dst_swap_w1(int kk, int Ns) { return 2 * kk > Ns; }
__host__ __device__ inline bool dst_swap_w2(int kk, int Ns) { return 4 * kk > Ns && 4 * kk < 3 * Ns; }
__host__ __device__ inline bool dst_swap_post(int k, int N) { return 8 * k > N; }

// Entries up to the end of the post-processing factors (the radix-4 layout).
__host__ __device__ inline int64_t dst_tw_len_r4(int N) {
  const int M = N >> 1;
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  int64_t len = N + N / 2 + 1;
  for (int Ns = (logM & 1) ? 2 : 1; Ns < M; Ns <<= 2)
    if (Ns > 1) len += 2 * (int64_t)Ns;
  return len + M / 2 + 1;
}
// Radix-8 plan of the M-point FFT (M = N/2): a stage without twiddles first
// when log2 M is not a multiple of 3 (radix 2 for 1 mod 3, radix 4 with
// Ns = 1 for 2 mod 3), then radix-8 stages from this Ns on.
__host__ __device__ inline int dst_r8_first_ns(int logM) {
  const int r = logM % 3;
  return r == 0 ? 1 : (r == 1 ? 2 : 4);
}
// After the radix-4 layout, per radix-8 stage Ns entries (c, t) of each of
// w = W^kk (W = exp(-2 pi i/(8 Ns))), w^2, w^4 and w e^{-i pi/4}, contiguous
// in kk.  Swap rules: none for w, dst_swap_w1 for w^2, dst_swap_w2 for w^4,
// kk > 0 for w e^{-i pi/4}.
__host__ __device__ inline int64_t dst_tw_len(int N) {
  const int M = N >> 1;
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  int64_t len = dst_tw_len_r4(N);
  for (int Ns = dst_r8_first_ns(logM); Ns < M; Ns <<= 3) len += 4 * (int64_t)Ns;
  return len;
}

}  // namespace ahoc
