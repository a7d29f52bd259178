// Helpers of the fused 2D Schur matvec (Algorithm 1, SchurMatVec, homogeneous
// part), which never forms the v-equation right-hand side in physical space
// and never transforms U back to physical space in full:
//
//   v2d_prep     boundary stencil of Q on the first interior columns
//                (r_x-(j), r_x+(j)) and a copy of the y-face data, whose DST
//                gives the y-face part of the right-hand side in x-modes;
//   trace2d_x    x-face traces from U-hat(k, j) (x-spectral, y-physical):
//                sum_m w_m U(m, j) = sum_k U-hat(k, j) tau_k with
//                tau_k = sum_m w_m sin(m k pi/N0), and U(N0 - m, j) picks up
//                (-1)^(k+1): odd and even k are summed separately;
//   trace2d_y*   y-face traces: the one-sided combination of rows 1..3 (and
//                N1-1..N1-3) in x-modes, an inverse DST of those two lines,
//                then R = alpha (.) - Q.
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

template <typename T>
__global__ void k_v2d_prep(Geom g, Coefs cf, const double* __restrict__ Q, const double* __restrict__ afinv,
                           T* __restrict__ rxm, T* __restrict__ rxp, T* __restrict__ qy, T* __restrict__ qa) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int N0 = g.N[0], N1 = g.N[1];
  const int bi = blockIdx.y;
  if (g.skip(bi)) return;
  Q += (int64_t)bi * g.ngamma;
  afinv += (int64_t)bi * g.ngamma;
  qa += (int64_t)bi * g.ngamma;
  rxm += (int64_t)bi * (N1 + 1);
  rxp += (int64_t)bi * (N1 + 1);
  qy += (int64_t)bi * 2 * N0;
  if (t < g.ngamma) qa[t] = (T)(Q[t] * afinv[t]);
  if (t <= N1) {
    const int j = t;
    double am = 0.0, ap = 0.0;
    if (j >= 1 && j <= N1 - 1) {
      const double* Qm = Q + g.face_off[0];  // x- face, index j - 1
      const double* Qp = Q + g.face_off[1];
      for (int dy = -1; dy <= 1; ++dy) {
        const int jj = j + dy;
        if (jj < 1 || jj > N1 - 1) continue;  // corners carry no unknown (zero in the homogeneous part)
        // (L - gam M)_bdry: the shift reaches the face point of the same row only
        const double sm = dy == 0 ? cf.gam * cf.Mn : 0.0;
        am -= (cf.L[9 + (dy + 1) * 3 + 0] - sm) * Qm[jj - 1];
        ap -= (cf.L[9 + (dy + 1) * 3 + 2] - sm) * Qp[jj - 1];
      }
    }
    if (j < N1) {
      rxm[j] = (T)am;
      rxp[j] = (T)ap;
    }
  }
  if (t < 2 * (N0 - 1)) qy[t] = (T)Q[g.face_off[2] + t];
}

constexpr int kRowThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_trace2d_x(Geom g, double* __restrict__ y,
                                                           const T* __restrict__ Uh,
                                                           const double* __restrict__ Q,
                                                           const double* __restrict__ afac,
                                                           const T* __restrict__ tau,
                                                           const double* __restrict__ srcq) {
  __shared__ double red[2][kRowThreads / 32];
  const int j = blockIdx.x + 1;
  const int N0 = g.N[0];
  const int bi = blockIdx.y;
  if (g.skip(bi)) return;
  {
    const int64_t fo = (int64_t)bi * g.ngamma;
    y += fo;
    Uh += (int64_t)bi * g.npad;
    if (Q) Q += fo;
    afac += fo;
    if (srcq) srcq += fo;
  }
  const T* row = Uh + g.pad(0, j, 0);
  T part = 0;  // k = 1 + tid + 256 m has the parity of 1 + tid; at most N0/256 terms in T
  for (int k = 1 + threadIdx.x; k < N0; k += kRowThreads) part += row[k] * tau[k];
  double acc = (double)part;
  // sum lanes of equal parity: lane 0 gets the odd-k sum, lane 1 the even-k sum
#pragma unroll
  for (int o = 16; o >= 2; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < 2) red[lane][warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double E = 0.0, O = 0.0;
    for (int w = 0; w < kRowThreads / 32; ++w) {
      E += red[0][w];
      O += red[1][w];
    }
    const int64_t qm = g.face(0, 0, 0, j, 0), qp = g.face(0, 1, N0, j, 0);
    // Navier faces carry v as data: the homogeneous R_p there is -Q_p
    double ym = g.is_navier(0) ? 0.0 : afac[qm] * (E + O), yp = g.is_navier(1) ? 0.0 : afac[qp] * (E - O);
    if (Q) {
      ym -= Q[qm];
      yp -= Q[qp];
    }
    if (srcq) {
      ym -= srcq[qm];
      yp -= srcq[qp];
    }
    y[qm] = ym;
    y[qp] = yp;
  }
}

template <typename T>
__global__ void k_trace2d_ylines(Geom g, Coefs cf, T* __restrict__ R, const T* __restrict__ Uh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int N0 = g.N[0], N1 = g.N[1];
  const int bi = blockIdx.y;
  if (k >= N0 || g.skip(bi)) return;
  R += (int64_t)bi * 2 * N0;
  Uh += (int64_t)bi * g.npad;
  const T w1 = (T)cf.w[1][1], w2 = (T)cf.w[1][2], w3 = (T)cf.w[1][3];
  R[k - 1] = w1 * Uh[g.pad(k, 1, 0)] + w2 * Uh[g.pad(k, 2, 0)] + w3 * Uh[g.pad(k, 3, 0)];
  R[(N0 - 1) + k - 1] = w1 * Uh[g.pad(k, N1 - 1, 0)] + w2 * Uh[g.pad(k, N1 - 2, 0)] + w3 * Uh[g.pad(k, N1 - 3, 0)];
}

template <typename T>
__global__ void k_trace2d_y(Geom g, double* __restrict__ y, const T* __restrict__ R,
                            const double* __restrict__ Q, const double* __restrict__ afac,
                            const double* __restrict__ srcq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int N0 = g.N[0];
  const int bi = blockIdx.y;
  if (i >= N0 || g.skip(bi)) return;
  {
    const int64_t fo = (int64_t)bi * g.ngamma;
    y += fo;
    R += (int64_t)bi * 2 * N0;
    if (Q) Q += fo;
    afac += fo;
    if (srcq) srcq += fo;
  }
  const int64_t qm = g.face(1, 0, i, 0, 0), qp = g.face(1, 1, i, g.N[1], 0);
  double ym = g.is_navier(2) ? 0.0 : afac[qm] * (double)R[i - 1];
  double yp = g.is_navier(3) ? 0.0 : afac[qp] * (double)R[(N0 - 1) + i - 1];
  if (Q) {
    ym -= Q[qm];
    yp -= Q[qp];
  }
  if (srcq) {
    ym -= srcq[qm];
    yp -= srcq[qp];
  }
  y[qm] = ym;
  y[qp] = yp;
}

template <typename T>
cudaError_t launch_v2d_prep(const Geom& g, const Coefs& cf, const double* Q, const double* afinv, T* rxm, T* rxp,
                            T* qy, T* qa, cudaStream_t st) {
  int64_t n = (g.N[1] + 1 > 2 * (g.N[0] - 1)) ? g.N[1] + 1 : 2 * (g.N[0] - 1);
  if (g.ngamma > n) n = g.ngamma;
  k_v2d_prep<T><<<dim3((unsigned)((n + 255) / 256), g.nb), 256, 0, st>>>(g, cf, Q, afinv, rxm, rxp, qy, qa);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_trace2d_x(const Geom& g, double* y, const T* Uh, const double* Q, const double* afac,
                             const T* tau, cudaStream_t st, const double* srcq) {
  k_trace2d_x<T><<<dim3(g.N[1] - 1, g.nb), kRowThreads, 0, st>>>(g, y, Uh, Q, afac, tau, srcq);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_trace2d_ylines(const Geom& g, const Coefs& cf, T* R, const T* Uh, cudaStream_t st) {
  k_trace2d_ylines<T><<<dim3((g.N[0] + 255) / 256, g.nb), 256, 0, st>>>(g, cf, R, Uh);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_trace2d_y(const Geom& g, double* y, const T* R, const double* Q, const double* afac,
                             cudaStream_t st, const double* srcq) {
  k_trace2d_y<T><<<dim3((g.N[0] + 255) / 256, g.nb), 256, 0, st>>>(g, y, R, Q, afac, srcq);
  return cudaGetLastError();
}

__global__ void k_to_float(float* __restrict__ out, const double* __restrict__ in, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}
cudaError_t launch_to_float(float* out, const double* in, int64_t n, cudaStream_t st) {
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, in, n);
  return cudaGetLastError();
}

#define AHOC_FUSED2D_INST(T)                                                                                    \
  template cudaError_t launch_v2d_prep<T>(const Geom&, const Coefs&, const double*, const double*, T*, T*, T*, \
                                          T*, cudaStream_t);                                                   \
  template cudaError_t launch_trace2d_x<T>(const Geom&, double*, const T*, const double*, const double*,       \
                                           const T*, cudaStream_t, const double*);                             \
  template cudaError_t launch_trace2d_ylines<T>(const Geom&, const Coefs&, T*, const T*, cudaStream_t);        \
  template cudaError_t launch_trace2d_y<T>(const Geom&, double*, const T*, const double*, const double*,       \
                                           cudaStream_t, const double*);
AHOC_FUSED2D_INST(double)
AHOC_FUSED2D_INST(float)
#undef AHOC_FUSED2D_INST

}  // namespace ahoc
