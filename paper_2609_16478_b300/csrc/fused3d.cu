// Helpers of the fused 3D Schur matvec (Algorithm 1, SchurMatVec, homogeneous
// part).  The same algebra as the plain form, with two passes over the field
// fewer at each end:
//
//   v3d_prep       the v-equation right-hand side is nonzero only on the
//                  interior layers next to the faces, and each face's part is
//                  a five-point stencil of that face's Q on its own layer.
//                  After the DST-I along x and y (Lemma 4's sine basis) a
//                  layer next to an x-face becomes sin(kx pi/N0) times the
//                  face part transformed along y, and the x+ layer adds
//                  (-1)^(kx+1) times its own: so the x-faces enter through
//                  their sum (odd kx) and difference (even kx), transformed
//                  along y; the y-faces likewise along x; the z-faces are the
//                  first and last rows of the z-solve, transformed along x and
//                  y.  These six face-sized arrays ("gen", face layout: x- =
//                  x sum, x+ = x difference, y- = y sum, y+ = y difference,
//                  z-, z+) generate the right-hand side inside the
//                  tridiagonal solve (tri.cu, VGen3D).  Also Q/alpha on the
//                  faces for the u-equation's M stencil.
//   trace3d_x/y    the one-sided combination w1 U1 + w2 U2 + w3 U3 of an
//                  x-face from U-hat(kx, ky, k) (the z-solve's output):
//                  sum_kx tau_x(kx) U-hat, tau_x(kx) = sum_m w_m sin(m kx pi/N0),
//                  odd and even kx apart (the x+ face takes (-1)^(kx+1));
//                  likewise the y-faces over ky (a second read of U-hat).
//                  Written in face layout, still in the in-face modes.
//   trace3d_z      the z-faces' combinations of the planes k = 1, 2, 3 and
//                  N2-1, N2-2, N2-3 in (kx, ky) modes.
//   trace3d_fin    after the in-face inverse DSTs: R = alpha (.) - Q.
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

// in-face coordinates (u, v) of face f's point q-local: remaining axes, lowest fastest
__device__ __forceinline__ void face_uv(const Geom& g, int a, int64_t loc, int& u, int& v, int& nu, int& nv) {
  const int b0 = (a == 0) ? 1 : 0;
  const int b1 = (a == 2) ? 1 : 2;
  nu = g.N[b0] - 1;
  nv = g.N[b1] - 1;
  u = 1 + (int)(loc % nu);
  v = 1 + (int)(loc / nu);
}

// the face part of -(L - gam M)_bdry Q on the interior layer next to face
// (a, side), at in-face point (u, v): the stencil entries whose offset crosses
// the face, applied to Q of that face (zero on the face edges, which carry no
// unknown in the homogeneous part)
__device__ __forceinline__ double face_part(const Geom& g, const Coefs& cf, const double* __restrict__ Qf, int a,
                                            int side, int u, int v, int nu, int nv) {
  const int b0 = (a == 0) ? 1 : 0;
  const int b1 = (a == 2) ? 1 : 2;
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int du = (t == 1) ? -1 : (t == 2) ? 1 : 0;
    const int dv = (t == 3) ? -1 : (t == 4) ? 1 : 0;
    const int uu = u + du, vv = v + dv;
    if (uu < 1 || uu > nu || vv < 1 || vv > nv) continue;
    int d[3] = {0, 0, 0};
    d[a] = side ? 1 : -1;
    d[b0] = du;
    d[b1] = dv;
    double c = cf.L[(d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1)];
    if (t == 0) c -= cf.gam * cf.Mn;  // the shift reaches the axis neighbour
    acc -= c * Qf[(uu - 1) + (int64_t)nu * (vv - 1)];
  }
  return acc;
}

template <typename T>
__global__ void k_v3d_prep(Geom g, Coefs cf, const double* __restrict__ Q, const double* __restrict__ afinv,
                           T* __restrict__ gen, T* __restrict__ qa) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (q >= g.ngamma || g.skip(bi)) return;
  const int64_t fo = (int64_t)bi * g.ngamma;
  Q += fo;
  gen += fo;
  qa += fo;
  qa[q] = (T)(Q[q] * afinv[fo + q]);
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  const int a = f >> 1;
  const int64_t loc = q - g.face_off[f];
  int u, v, nu, nv;
  face_uv(g, a, loc, u, v, nu, nv);
  if (a < 2) {
    // x- and y-faces: the slot of side 0 takes the sum of the two faces' parts,
    // the slot of side 1 their difference
    const double pm = face_part(g, cf, Q + g.face_off[2 * a], a, 0, u, v, nu, nv);
    const double pp = face_part(g, cf, Q + g.face_off[2 * a + 1], a, 1, u, v, nu, nv);
    gen[q] = (T)((f & 1) ? pm - pp : pm + pp);
  } else {
    gen[q] = (T)face_part(g, cf, Q + g.face_off[f], a, f & 1, u, v, nu, nv);
  }
}

// x-faces: one warp per row (ky, k) of U-hat sums tau_x(kx) U-hat over kx;
// lane l takes kx = 1 + l + 32 t, so a lane sees one kx parity and the
// xor-shuffles over lanes of equal parity leave the odd-kx sum in lane 0 and
// the even-kx sum in lane 1.  Sums in T (an FP32 pass takes no FP64 operation
// per element), the two results in FP64.
constexpr int kRedThreads = 256;
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_trace3d_x(Geom g, const T* __restrict__ Uh,
                                                           const T* __restrict__ taux, double* __restrict__ out) {
  const int bi = blockIdx.y;
  if (g.skip(bi)) return;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1;
  const int64_t row = (int64_t)blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);  // (ky - 1) + ny (k - 1)
  if (row >= (int64_t)ny * (g.N[2] - 1)) return;
  const int lane = threadIdx.x & 31;
  const int ky = 1 + (int)(row % ny), k = 1 + (int)(row / ny);
  const T* r = Uh + (int64_t)bi * g.npad + g.pad(0, ky, k);
  T acc = 0;
  int kx = 1 + lane;
  for (; kx + 96 <= nx; kx += 128)  // four loads in flight per lane
    acc += taux[kx] * r[kx] + taux[kx + 32] * r[kx + 32] + taux[kx + 64] * r[kx + 64] + taux[kx + 96] * r[kx + 96];
  for (; kx <= nx; kx += 32) acc += taux[kx] * r[kx];
  double a = (double)acc;
#pragma unroll
  for (int o = 16; o >= 2; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  const double other = __shfl_down_sync(0xffffffffu, a, 1);  // lane 0 gets lane 1's even-kx sum
  if (lane == 0) {
    out += (int64_t)bi * g.ngamma;
    out[g.face_off[0] + row] = a + other;  // x-: U(m) = sum U-hat sin(m kx pi/N0)
    out[g.face_off[1] + row] = a - other;  // x+: U(N0 - m) picks up (-1)^(kx+1)
  }
}

// y-faces: a CTA takes a strip of 32 x-modes of one plane k; warp w sums
// tau_y(ky) U-hat over the rows ky = 1 + w + W t (W warps, even: one ky parity
// per warp), lane l over its column; the warps' sums are combined in shared
// memory in warp order.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_trace3d_y(Geom g, const T* __restrict__ Uh,
                                                           const T* __restrict__ tauy, double* __restrict__ out) {
  __shared__ double part[kRedThreads / 32][32];
  const int bi = blockIdx.z;
  if (g.skip(bi)) return;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1;
  const int k = 1 + blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int W = kRedThreads / 32;
  const int kx = 1 + blockIdx.x * 32 + lane;
  const T* base = Uh + (int64_t)bi * g.npad + g.pad(0, 0, k);
  T acc = 0;
  if (kx <= nx) {
    int ky = 1 + w;
    for (; ky + 3 * W <= ny; ky += 4 * W)
      acc += tauy[ky] * base[g.n0 * (int64_t)ky + kx] + tauy[ky + W] * base[g.n0 * (int64_t)(ky + W) + kx] +
             tauy[ky + 2 * W] * base[g.n0 * (int64_t)(ky + 2 * W) + kx] +
             tauy[ky + 3 * W] * base[g.n0 * (int64_t)(ky + 3 * W) + kx];
    for (; ky <= ny; ky += W) acc += tauy[ky] * base[g.n0 * (int64_t)ky + kx];
  }
  part[w][lane] = (double)acc;
  __syncthreads();
  if (w == 0 && kx <= nx) {
    double O = 0.0, E = 0.0;  // warps of even w take odd ky
    for (int v = 0; v < W; v += 2) {
      O += part[v][lane];
      E += part[v + 1][lane];
    }
    out += (int64_t)bi * g.ngamma;
    const int64_t loc = (kx - 1) + (int64_t)nx * (k - 1);
    out[g.face_off[2] + loc] = O + E;
    out[g.face_off[3] + loc] = O - E;
  }
}

// z-faces: w1 U-hat(., ., 1) + w2 U-hat(., ., 2) + w3 U-hat(., ., 3) and the same from the top
template <typename T>
__global__ void k_trace3d_z(Geom g, Coefs cf, const T* __restrict__ Uh, double* __restrict__ out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1;
  if (m >= (int64_t)nx * ny || g.skip(bi)) return;
  Uh += (int64_t)bi * g.npad;
  out += (int64_t)bi * g.ngamma;
  const int kx = 1 + (int)(m % nx), ky = 1 + (int)(m / nx);
  const int N2 = g.N[2];
  const double w1 = cf.w[2][1], w2 = cf.w[2][2], w3 = cf.w[2][3];
  auto U = [&](int k) { return (double)Uh[g.pad(kx, ky, k)]; };
  out[g.face_off[4] + m] = w1 * U(1) + w2 * U(2) + w3 * U(3);
  out[g.face_off[5] + m] = w1 * U(N2 - 1) + w2 * U(N2 - 2) + w3 * U(N2 - 3);
}

// y = alpha T - Q - srcq on clamped faces, -Q - srcq on Navier faces
__global__ void k_trace3d_fin(Geom g, double* __restrict__ y, const double* __restrict__ Tr,
                              const double* __restrict__ Q, const double* __restrict__ afac,
                              const double* __restrict__ srcq) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (q >= g.ngamma || g.skip(bi)) return;
  const int64_t fo = (int64_t)bi * g.ngamma;
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  double r = g.is_navier(f) ? 0.0 : afac[fo + q] * Tr[fo + q];
  if (Q) r -= Q[fo + q];
  if (srcq) r -= srcq[fo + q];
  y[fo + q] = r;
}

static inline unsigned nblk3(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

template <typename T>
cudaError_t launch_v3d_prep(const Geom& g, const Coefs& cf, const double* Q, const double* afinv, T* gen, T* qa,
                            cudaStream_t st) {
  k_v3d_prep<T><<<dim3(nblk3(g.ngamma, 256), g.nb), 256, 0, st>>>(g, cf, Q, afinv, gen, qa);
  return cudaGetLastError();
}

bool trace3d_red_ok(const Geom& g) { return g.dim == 3; }

// three kernels: the x-face sums, the y-face sums, the z-face planes
template <typename T>
cudaError_t launch_trace3d(const Geom& g, const Coefs& cf, const T* Uh, const T* taux, const T* tauy,
                           double* Tr, cudaStream_t st) {
  const int nx = g.N[0] - 1, ny = g.N[1] - 1, nz = g.N[2] - 1;
  const int64_t rows = (int64_t)ny * nz;
  k_trace3d_x<T><<<dim3(nblk3(rows, kRedThreads / 32), g.nb), kRedThreads, 0, st>>>(g, Uh, taux, Tr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_trace3d_y<T><<<dim3((unsigned)((nx + 31) / 32), (unsigned)nz, g.nb), kRedThreads, 0, st>>>(g, Uh, tauy, Tr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nzf = (int64_t)nx * ny;
  k_trace3d_z<T><<<dim3(nblk3(nzf, 256), g.nb), 256, 0, st>>>(g, cf, Uh, Tr);
  return cudaGetLastError();
}

cudaError_t launch_trace3d_fin(const Geom& g, double* y, const double* Tr, const double* Q, const double* afac,
                               const double* srcq, cudaStream_t st) {
  k_trace3d_fin<<<dim3(nblk3(g.ngamma, 256), g.nb), 256, 0, st>>>(g, y, Tr, Q, afac, srcq);
  return cudaGetLastError();
}

template cudaError_t launch_v3d_prep<double>(const Geom&, const Coefs&, const double*, const double*, double*,
                                             double*, cudaStream_t);
template cudaError_t launch_v3d_prep<float>(const Geom&, const Coefs&, const double*, const double*, float*, float*,
                                            cudaStream_t);
template cudaError_t launch_trace3d<double>(const Geom&, const Coefs&, const double*, const double*, const double*,
                                            double*, cudaStream_t);
template cudaError_t launch_trace3d<float>(const Geom&, const Coefs&, const float*, const float*, const float*,
                                           double*, cudaStream_t);

}  // namespace ahoc
