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
//   trace3d_red    the one-sided combination w1 U1 + w2 U2 + w3 U3 of an
//                  x-face from U-hat(kx, ky, k) (the z-solve's output):
//                  sum_kx tau_x(kx) U-hat, tau_x(kx) = sum_m w_m sin(m kx pi/N0),
//                  odd and even kx apart (the x+ face takes (-1)^(kx+1));
//                  likewise the y-faces over ky; one read of U-hat.  Written
//                  in face layout, still in the in-face transverse modes.
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

// One CTA per (k plane, problem).  Thread t owns the x-mode columns
// kx = 1 + t + c * blockDim.x; per row ky it adds tau_y(ky) U-hat into its
// column sums (odd / even ky apart), and the warps reduce tau_x(kx) U-hat over
// their lanes (odd / even kx apart) into shared memory, summed in warp order
// once per batch of rows.
constexpr int kRedThreads = 512;
constexpr int kRedRows = 8;
constexpr int kRedCols = 8;  // columns per thread: N0 <= kRedThreads * kRedCols

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_trace3d_red(Geom g, const T* __restrict__ Uh,
                                                             const T* __restrict__ taux,
                                                             const T* __restrict__ tauy, double* __restrict__ out) {
  __shared__ double red[kRedRows][2][kRedThreads / 32];
  const int k = 1 + blockIdx.x;
  const int bi = blockIdx.y;
  if (g.skip(bi)) return;
  Uh += (int64_t)bi * g.npad + g.pad(0, 0, k);
  out += (int64_t)bi * g.ngamma;
  const int N0 = g.N[0], N1 = g.N[1];
  const int nx = N0 - 1, ny = N1 - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int ncol = (nx + blockDim.x - 1) / blockDim.x;
  // sums in T: an FP32 pass must not take FP64 operations per element
  T ys[kRedCols][2];
  T tx[kRedCols];
#pragma unroll
  for (int c = 0; c < kRedCols; ++c) {
    ys[c][0] = ys[c][1] = (T)0;
    const int kx = 1 + threadIdx.x + c * blockDim.x;
    tx[c] = (c < ncol && kx <= nx) ? taux[kx] : (T)0;
  }
  for (int r0 = 1; r0 <= ny; r0 += kRedRows) {
#pragma unroll
    for (int rr = 0; rr < kRedRows; ++rr) {
      const int ky = r0 + rr;
      T xs = 0;
      if (ky <= ny) {
        const T* row = Uh + g.n0 * (int64_t)ky;
        const T wy = tauy[ky];
#pragma unroll
        for (int c = 0; c < kRedCols; ++c) {
          const int kx = 1 + threadIdx.x + c * blockDim.x;
          if (c < ncol && kx <= nx) {
            const T val = row[kx];
            ys[c][ky & 1] += wy * val;
            xs += tx[c] * val;
          }
        }
      }
      // lanes of equal kx parity: lane 0 ends with the sum over its warp's odd kx
      // (kx = 1 + t + c * blockDim.x has the parity of 1 + lane), lane 1 with the even
#pragma unroll
      for (int o = 16; o >= 2; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o);
      if (lane < 2) red[rr][lane][warp] = (double)xs;
    }
    __syncthreads();
    if (threadIdx.x < 2 * kRedRows) {
      const int rr = threadIdx.x >> 1, par = threadIdx.x & 1;  // par 0: odd kx, 1: even kx
      const int ky = r0 + rr;
      if (ky <= ny) {
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += red[rr][par][w];
        red[rr][par][0] = s;
      }
    }
    __syncthreads();
    if (threadIdx.x < kRedRows) {
      const int ky = r0 + threadIdx.x;
      if (ky <= ny) {
        const double O = red[threadIdx.x][0][0], E = red[threadIdx.x][1][0];
        const int64_t loc = (ky - 1) + (int64_t)ny * (k - 1);
        out[g.face_off[0] + loc] = O + E;  // x-: U(m) = sum U-hat sin(m kx pi/N0)
        out[g.face_off[1] + loc] = O - E;  // x+: U(N0 - m) picks up (-1)^(kx+1)
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < kRedCols; ++c) {
    const int kx = 1 + threadIdx.x + c * blockDim.x;
    if (c < ncol && kx <= nx) {
      const double O = (double)ys[c][1], E = (double)ys[c][0];  // ky odd, ky even
      const int64_t loc = (kx - 1) + (int64_t)nx * (k - 1);
      out[g.face_off[2] + loc] = O + E;
      out[g.face_off[3] + loc] = O - E;
    }
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

bool trace3d_red_ok(const Geom& g) { return g.dim == 3 && g.N[0] - 1 <= kRedThreads * kRedCols; }

template <typename T>
cudaError_t launch_trace3d(const Geom& g, const Coefs& cf, const T* Uh, const T* taux, const T* tauy,
                           double* Tr, cudaStream_t st) {
  const int nx = g.N[0] - 1;
  int th = nx < kRedThreads ? ((nx + 31) / 32) * 32 : kRedThreads;
  if (th < 64) th = 64;
  k_trace3d_red<T><<<dim3((unsigned)(g.N[2] - 1), g.nb), th, 0, st>>>(g, Uh, taux, tauy, Tr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nz = (int64_t)nx * (g.N[1] - 1);
  k_trace3d_z<T><<<dim3(nblk3(nz, 256), g.nb), 256, 0, st>>>(g, cf, Uh, Tr);
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
