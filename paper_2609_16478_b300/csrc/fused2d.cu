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

__global__ void k_v2d_prep(Geom g, Coefs cf, const double* __restrict__ Q, double* __restrict__ rxm,
                           double* __restrict__ rxp, double* __restrict__ qy) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int N0 = g.N[0], N1 = g.N[1];
  if (t <= N1) {
    const int j = t;
    double am = 0.0, ap = 0.0;
    if (j >= 1 && j <= N1 - 1) {
      const double* Qm = Q + g.face_off[0];  // x- face, index j - 1
      const double* Qp = Q + g.face_off[1];
      for (int dy = -1; dy <= 1; ++dy) {
        const int jj = j + dy;
        if (jj < 1 || jj > N1 - 1) continue;  // corners carry no unknown (zero in the homogeneous part)
        am -= cf.L[9 + (dy + 1) * 3 + 0] * Qm[jj - 1];
        ap -= cf.L[9 + (dy + 1) * 3 + 2] * Qp[jj - 1];
      }
    }
    if (j < N1) {
      rxm[j] = am;
      rxp[j] = ap;
    }
  }
  if (t < 2 * (N0 - 1)) qy[t] = Q[g.face_off[2] + t];
}

constexpr int kRowThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_trace2d_x(Geom g, double* __restrict__ y,
                                                           const T* __restrict__ Uh,
                                                           const double* __restrict__ Q,
                                                           const double* __restrict__ afac,
                                                           const double* __restrict__ tau,
                                                           const double* __restrict__ srcq) {
  __shared__ double red[2][kRowThreads / 32];
  const int j = blockIdx.x + 1;
  const int N0 = g.N[0];
  const T* row = Uh + g.pad(0, j, 0);
  double acc = 0.0;  // k = 1 + tid + 256 m has the parity of 1 + tid
  for (int k = 1 + threadIdx.x; k < N0; k += kRowThreads) acc = fma((double)row[k], tau[k], acc);
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
    double ym = afac[qm] * (E + O), yp = afac[qp] * (E - O);
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
__global__ void k_trace2d_ylines(Geom g, Coefs cf, double* __restrict__ R, const T* __restrict__ Uh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int N0 = g.N[0], N1 = g.N[1];
  if (k >= N0) return;
  const double w1 = cf.w[1][1], w2 = cf.w[1][2], w3 = cf.w[1][3];
  R[k - 1] = w1 * (double)Uh[g.pad(k, 1, 0)] + w2 * (double)Uh[g.pad(k, 2, 0)] + w3 * (double)Uh[g.pad(k, 3, 0)];
  R[(N0 - 1) + k - 1] = w1 * (double)Uh[g.pad(k, N1 - 1, 0)] + w2 * (double)Uh[g.pad(k, N1 - 2, 0)] +
                        w3 * (double)Uh[g.pad(k, N1 - 3, 0)];
}

__global__ void k_trace2d_y(Geom g, double* __restrict__ y, const double* __restrict__ R,
                            const double* __restrict__ Q, const double* __restrict__ afac,
                            const double* __restrict__ srcq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int N0 = g.N[0];
  if (i >= N0) return;
  const int64_t qm = g.face(1, 0, i, 0, 0), qp = g.face(1, 1, i, g.N[1], 0);
  double ym = afac[qm] * R[i - 1], yp = afac[qp] * R[(N0 - 1) + i - 1];
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

cudaError_t launch_v2d_prep(const Geom& g, const Coefs& cf, const double* Q, double* rxm, double* rxp, double* qy,
                            cudaStream_t st) {
  const int n = (g.N[1] + 1 > 2 * (g.N[0] - 1)) ? g.N[1] + 1 : 2 * (g.N[0] - 1);
  k_v2d_prep<<<(n + 255) / 256, 256, 0, st>>>(g, cf, Q, rxm, rxp, qy);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_trace2d_x(const Geom& g, double* y, const T* Uh, const double* Q, const double* afac,
                             const double* tau, cudaStream_t st, const double* srcq) {
  k_trace2d_x<T><<<g.N[1] - 1, kRowThreads, 0, st>>>(g, y, Uh, Q, afac, tau, srcq);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_trace2d_ylines(const Geom& g, const Coefs& cf, double* R, const T* Uh, cudaStream_t st) {
  k_trace2d_ylines<T><<<(g.N[0] + 255) / 256, 256, 0, st>>>(g, cf, R, Uh);
  return cudaGetLastError();
}
cudaError_t launch_trace2d_y(const Geom& g, double* y, const double* R, const double* Q, const double* afac,
                             cudaStream_t st, const double* srcq) {
  k_trace2d_y<<<(g.N[0] + 255) / 256, 256, 0, st>>>(g, y, R, Q, afac, srcq);
  return cudaGetLastError();
}
template cudaError_t launch_trace2d_x<double>(const Geom&, double*, const double*, const double*, const double*,
                                              const double*, cudaStream_t, const double*);
template cudaError_t launch_trace2d_x<float>(const Geom&, double*, const float*, const double*, const double*,
                                             const double*, cudaStream_t, const double*);
template cudaError_t launch_trace2d_ylines<double>(const Geom&, const Coefs&, double*, const double*, cudaStream_t);
template cudaError_t launch_trace2d_ylines<float>(const Geom&, const Coefs&, double*, const float*, cudaStream_t);

}  // namespace ahoc
