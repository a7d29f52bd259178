// Compact-stencil kernels of the augmented HOC scheme (Sec. 2.2):
// right-hand sides of the v- and u-equations, the boundary residual R of
// Lemma 1, and layout conversions.
//
// Stencils (coefficients per plan, anisotropic h): the 9-point (2D) /
// 19-point (3D) fourth-order Laplacian L_h with prefactor 1/12, the
// weighting M (centre 8/12 in 2D, 6/12 in 3D, 1/12 per axis neighbour) and
// the one-sided second normal derivative
//   u_nn ~ h^-2 (-85/18 U0 + 6 U1 - 3/2 U2 + 2/9 U3) + 11/(3h) g_N.
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

__device__ __forceinline__ void decompose(const Geom& g, int64_t t, int& i, int& j, int& k) {
  i = (int)(t % g.n0);
  int64_t r = t / g.n0;
  j = (int)(r % g.n1);
  k = (int)(r / g.n1);
}

__device__ __forceinline__ bool is_pad(const Geom& g, int i, int j, int k) {
  return i == 0 || j == 0 || (g.dim == 3 && k == 0);
}

// number of coordinates of (i, j, k) on the boundary, and the first such axis/side
__device__ __forceinline__ int bclass(const Geom& g, int i, int j, int k, int& axis, int& side) {
  int nb = 0;
  axis = -1;
  side = 0;
  if (i == 0 || i == g.N[0]) { ++nb; axis = 0; side = (i != 0); }
  if (j == 0 || j == g.N[1]) { if (!nb) { axis = 1; side = (j != 0); } ++nb; }
  if (g.dim == 3 && (k == 0 || k == g.N[2])) { if (!nb) { axis = 2; side = (k != 0); } ++nb; }
  return nb;
}

__device__ __forceinline__ bool near_bdry(const Geom& g, int i, int j, int k) {
  return i == 1 || i == g.N[0] - 1 || j == 1 || j == g.N[1] - 1 ||
         (g.dim == 3 && (k == 1 || k == g.N[2] - 1));
}

// The right-hand-side kernels run on a (ceil(n0/256), n1, n2) grid: thread
// (i, j, k) of the padded interior, no 64-bit index division.  Arithmetic is
// in T; the FP64 face data (Q, v on the edges) is rounded to T on the
// boundary-adjacent points that read it.
template <typename T>
__global__ void k_vrhs(Geom g, Coefs cf, T* __restrict__ out, const double* __restrict__ Q,
                       const double* __restrict__ f, const double* __restrict__ vedge,
                       const T* __restrict__ srcv, const double* __restrict__ gam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.z / (int)g.n2;
  if (i >= g.n0 || g.skip(bi)) return;
  const int j = blockIdx.y, k = blockIdx.z - bi * (int)g.n2;
  out += (int64_t)bi * g.npad;
  if (srcv) srcv += (int64_t)bi * g.npad;
  if (Q) Q += (int64_t)bi * g.ngamma;
  if (f) f += (int64_t)bi * g.nfull;
  if (vedge) vedge += (int64_t)bi * g.nfull;
  if (gam) gam += (int64_t)bi * g.nfull;
  const int64_t t = g.pad(i, j, k);
  if (is_pad(g, i, j, k)) { out[t] = (T)0; return; }
  T acc = 0;
  if ((Q || vedge) && near_bdry(g, i, j, k)) {
    const int dzlo = (g.dim == 3) ? -1 : 0, dzhi = (g.dim == 3) ? 1 : 0;
    for (int dz = dzlo; dz <= dzhi; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const double c = cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
          if (c == 0.0) continue;
          const int ii = i + dx, jj = j + dy, kk = k + dz;
          int ax, sd;
          const int nb = bclass(g, ii, jj, kk, ax, sd);
          if (nb == 0) continue;
          double vb = 0.0;
          if (nb == 1) {
            if (Q) vb = Q[g.face(ax, sd, ii, jj, kk)];
          } else if (vedge) {
            vb = vedge[g.full(ii, jj, kk)];
          }
          // the shift gam M V reaches the axis neighbours (weight Mn): (L - gam M) V = ...
          const double gn = gam ? gam[g.full(ii, jj, kk)] : cf.gam;
          const double ce = (dx * dx + dy * dy + dz * dz == 1) ? c - gn * cf.Mn : c;
          acc -= (T)ce * (T)vb;
        }
  }
  if (f) {
    T m = (T)cf.Mc * (T)f[g.full(i, j, k)];
    m += (T)cf.Mn * (T)(f[g.full(i - 1, j, k)] + f[g.full(i + 1, j, k)] + f[g.full(i, j - 1, k)] + f[g.full(i, j + 1, k)]);
    if (g.dim == 3) m += (T)cf.Mn * (T)(f[g.full(i, j, k - 1)] + f[g.full(i, j, k + 1)]);
    acc += (T)cf.fsign * m;
  }
  if (srcv) acc -= srcv[t];
  out[t] = acc;
}

// ainv: 1/alpha on the full grid, in T
template <typename T>
__global__ void k_urhs(Geom g, Coefs cf, T* __restrict__ out, const T* __restrict__ V,
                       const T* __restrict__ ainv, const double* __restrict__ Q,
                       const double* __restrict__ gD, const T* __restrict__ srcu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.z / (int)g.n2;
  if (i >= g.n0 || g.skip(bi)) return;
  const int j = blockIdx.y, k = blockIdx.z - bi * (int)g.n2;
  out += (int64_t)bi * g.npad;
  V += (int64_t)bi * g.npad;
  if (srcu) srcu += (int64_t)bi * g.npad;
  ainv += (int64_t)bi * g.nfull;
  if (Q) Q += (int64_t)bi * g.ngamma;
  if (gD) gD += (int64_t)bi * g.nfull;
  const int64_t t = g.pad(i, j, k);
  if (is_pad(g, i, j, k)) { out[t] = (T)0; return; }
  // M(V / alpha): centre and the axis neighbours; a neighbour on a face holds Q
  const int64_t fc = g.full(i, j, k);
  const T Mn = (T)cf.Mn;
  T acc = (T)cf.Mc * V[t] * ainv[fc];
  const int64_t pst[3] = {1, g.n0, g.n0 * g.n1}, fst[3] = {1, g.f0, g.f0 * g.f1};
  const int idx[3] = {i, j, k};
  for (int a = 0; a < g.dim; ++a) {
    for (int s = -1; s <= 1; s += 2) {
      const int ia = idx[a] + s;
      T v;
      if (ia == 0 || ia == g.N[a]) {
        const int ii = i + (a == 0 ? s : 0), jj = j + (a == 1 ? s : 0), kk = k + (a == 2 ? s : 0);
        v = Q ? (T)Q[g.face(a, ia != 0, ii, jj, kk)] : (T)0;
      } else {
        v = V[t + s * pst[a]];
      }
      acc += Mn * v * ainv[fc + s * fst[a]];
    }
  }
  if (gD && near_bdry(g, i, j, k)) {
    const int dzlo = (g.dim == 3) ? -1 : 0, dzhi = (g.dim == 3) ? 1 : 0;
    for (int dz = dzlo; dz <= dzhi; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const double c = cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
          if (c == 0.0) continue;
          const int ii = i + dx, jj = j + dy, kk = k + dz;
          int ax, sd;
          if (bclass(g, ii, jj, kk, ax, sd) == 0) continue;
          acc -= (T)c * (T)gD[g.full(ii, jj, kk)];
        }
  }
  if (srcu) acc += srcu[t];
  out[t] = acc;
}

template <typename T>
__global__ void k_trace(Geom g, Coefs cf, double* __restrict__ y, const T* __restrict__ U,
                        const double* __restrict__ Q, const double* __restrict__ afac,
                        const double* __restrict__ gD, const double* __restrict__ gN,
                        const double* __restrict__ lapt, const double* __restrict__ srcq,
                        const double* __restrict__ gL) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (q >= g.ngamma || g.skip(bi)) return;
  {
    const int64_t fo = (int64_t)bi * g.ngamma;
    y += fo;
    U += (int64_t)bi * g.npad;
    if (Q) Q += fo;
    afac += fo;
    if (gD) gD += (int64_t)bi * g.nfull;
    if (gN) gN += fo;
    if (lapt) lapt += fo;
    if (srcq) srcq += fo;
    if (gL) gL += fo;
  }
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  if (g.is_navier(f)) {  // R_p = alpha_p g_L,p - Q_p: v is data on a Navier face
    double res = gL ? afac[q] * gL[q] : 0.0;
    if (Q) res -= Q[q];
    if (srcq) res -= srcq[q];
    y[q] = res;
    return;
  }
  const int a = f >> 1, side = f & 1;
  const int64_t loc = q - g.face_off[f];
  int c[3] = {0, 0, 0};
  // remaining axes, lowest fastest
  int64_t r = loc;
  for (int b = 0; b < g.dim; ++b) {
    if (b == a) continue;
    const int nb = g.N[b] - 1;
    c[b] = 1 + (int)(r % nb);
    r /= nb;
  }
  c[a] = side ? g.N[a] : 0;
  const int step = side ? -1 : 1;
  double U1, U2, U3;
  {
    int p[3] = {c[0], c[1], c[2]};
    p[a] = c[a] + step;
    U1 = (double)U[g.pad(p[0], p[1], p[2])];
    p[a] = c[a] + 2 * step;
    U2 = (double)U[g.pad(p[0], p[1], p[2])];
    p[a] = c[a] + 3 * step;
    U3 = (double)U[g.pad(p[0], p[1], p[2])];
  }
  double unn = cf.w[a][1] * U1 + cf.w[a][2] * U2 + cf.w[a][3] * U3;
  if (gD) unn += cf.w[a][0] * gD[g.full(c[0], c[1], c[2])];
  if (gN) unn += cf.wg[a] * gN[q];
  if (lapt) unn += lapt[q];
  double res = afac[q] * unn;
  if (Q) res -= Q[q];
  if (srcq) res -= srcq[q];
  y[q] = res;
}

// Triharmonic class: R_p = u_ssss(U)_p + lapt_w_p - Q_p at a clamped face point
// (Lap^2 u there, with u_ssss one-sided from U_0 = g_D, U_1..U_4 and the data
// u_s = -g_N, u_ss = g_NN), R_p = bilap_p - Q_p on the other faces (Lap^2 u is
// data there).  Data arrays may be NULL (zero).
__global__ void k_trace_tri(Geom g, Coefs cf, double* __restrict__ y, const double* __restrict__ U,
                            const double* __restrict__ Q, const double* __restrict__ gD,
                            const double* __restrict__ gN, const double* __restrict__ gNN,
                            const double* __restrict__ laptw, const double* __restrict__ bilap) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (q >= g.ngamma || g.skip(bi)) return;
  const int64_t fo = (int64_t)bi * g.ngamma, ff = (int64_t)bi * g.nfull;
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  const int a = f >> 1, side = f & 1;
  const int64_t loc = q - g.face_off[f];
  int c[3] = {0, 0, 0};
  int64_t r = loc;
  for (int b = 0; b < g.dim; ++b) {
    if (b == a) continue;
    const int nb = g.N[b] - 1;
    c[b] = 1 + (int)(r % nb);
    r /= nb;
  }
  c[a] = side ? g.N[a] : 0;
  double res;
  if (g.is_navier(f)) {
    res = bilap ? bilap[ff + g.full(c[0], c[1], c[2])] : 0.0;
  } else {
    U += (int64_t)bi * g.npad;
    const int step = side ? -1 : 1;
    res = 0.0;
    for (int m = 1; m <= 4; ++m) {
      int p[3] = {c[0], c[1], c[2]};
      p[a] = c[a] + m * step;
      res += cf.w4[a][m] * U[g.pad(p[0], p[1], p[2])];
    }
    if (gD) res += cf.w4[a][0] * gD[ff + g.full(c[0], c[1], c[2])];
    if (gN) res -= cf.w4s[a] * gN[fo + q];
    if (gNN) res += cf.w4ss[a] * gNN[fo + q];
    if (laptw) res += laptw[fo + q];
  }
  if (Q) res -= Q[fo + q];
  y[fo + q] = res;
}

// full-grid output: interior from the padded field, boundary from bnd (or 0)
__global__ void k_write_full(Geom g, double* __restrict__ out, const double* __restrict__ Uin,
                             const double* __restrict__ bnd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (t >= g.nfull || g.skip(bi)) return;
  out += (int64_t)bi * g.nfull;
  Uin += (int64_t)bi * g.npad;
  if (bnd) bnd += (int64_t)bi * g.nfull;
  const int i = (int)(t % g.f0);
  const int64_t r = t / g.f0;
  const int j = (int)(r % g.f1);
  const int k = (int)(r / g.f1);
  int ax, sd;
  if (bclass(g, i, j, k, ax, sd) == 0) out[t] = Uin[g.pad(i, j, k)];
  else out[t] = bnd ? bnd[t] : 0.0;
}

// full-grid V: interior from the padded field, faces = Q, edges/corners = vedge
__global__ void k_v_full(Geom g, double* __restrict__ out, const double* __restrict__ Vin,
                         const double* __restrict__ Q, const double* __restrict__ vedge) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (t >= g.nfull || g.skip(bi)) return;
  out += (int64_t)bi * g.nfull;
  Vin += (int64_t)bi * g.npad;
  if (Q) Q += (int64_t)bi * g.ngamma;
  if (vedge) vedge += (int64_t)bi * g.nfull;
  const int i = (int)(t % g.f0);
  const int64_t r = t / g.f0;
  const int j = (int)(r % g.f1);
  const int k = (int)(r / g.f1);
  int ax, sd;
  const int nb = bclass(g, i, j, k, ax, sd);
  if (nb == 0) out[t] = Vin[g.pad(i, j, k)];
  else if (nb == 1) out[t] = Q ? Q[g.face(ax, sd, i, j, k)] : 0.0;
  else out[t] = vedge ? vedge[t] : 0.0;
}

__global__ void k_pack(Geom g, double* __restrict__ dense, const double* __restrict__ padded) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nint) return;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1;
  const int i = 1 + (int)(t % nx);
  const int64_t r = t / nx;
  const int j = 1 + (int)(r % ny);
  const int k = g.kmin + (int)(r / ny);
  dense[t] = padded[g.pad(i, j, k)];
}

__global__ void k_unpack(Geom g, double* __restrict__ padded, const double* __restrict__ dense) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nint) return;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1;
  const int i = 1 + (int)(t % nx);
  const int64_t r = t / nx;
  const int j = 1 + (int)(r % ny);
  const int k = g.kmin + (int)(r / ny);
  padded[g.pad(i, j, k)] = dense[t];
}

__global__ void k_face_gather(Geom g, double* __restrict__ face, const double* __restrict__ full) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.ngamma) return;
  face += (int64_t)blockIdx.y * g.ngamma;
  full += (int64_t)blockIdx.y * g.nfull;
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  const int a = f >> 1, side = f & 1;
  int64_t r = q - g.face_off[f];
  int c[3] = {0, 0, 0};
  for (int b = 0; b < g.dim; ++b) {
    if (b == a) continue;
    const int nb = g.N[b] - 1;
    c[b] = 1 + (int)(r % nb);
    r /= nb;
  }
  c[a] = side ? g.N[a] : 0;
  face[q] = full[g.full(c[0], c[1], c[2])];
}

__global__ void k_recip(double* __restrict__ out, const double* __restrict__ in, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = in ? 1.0 / in[t] : 1.0;  // in == NULL: a unit coefficient
}

static inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

// min, max and sum of beta / alpha over n points, one triple per block
// (out[3 b .. 3 b + 2]), summed by the host in block order
constexpr int kStatThreads = 256;
__global__ void __launch_bounds__(kStatThreads) k_ratio_stats(const double* __restrict__ beta,
                                                              const double* __restrict__ alpha, int64_t n,
                                                              double* __restrict__ out) {
  __shared__ double smin[kStatThreads], smax[kStatThreads], ssum[kStatThreads];
  double mn = INFINITY, mx = -INFINITY, sm = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double r = beta[t] / alpha[t];
    mn = fmin(mn, r);
    mx = fmax(mx, r);
    sm += r;
  }
  smin[threadIdx.x] = mn;
  smax[threadIdx.x] = mx;
  ssum[threadIdx.x] = sm;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[3 * blockIdx.x] = smin[0];
    out[3 * blockIdx.x + 1] = smax[0];
    out[3 * blockIdx.x + 2] = ssum[0];
  }
}
cudaError_t launch_ratio_stats(const double* beta, const double* alpha, int64_t n, double* out, int blocks,
                               cudaStream_t st) {
  k_ratio_stats<<<blocks, kStatThreads, 0, st>>>(beta, alpha, n, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vrhs(const Geom& g, const Coefs& cf, T* out, const double* Q, const double* f,
                        const double* vedge, cudaStream_t st, const T* srcv, const double* gam) {
  const dim3 grid((unsigned)((g.n0 + 255) / 256), (unsigned)g.n1, (unsigned)(g.n2 * g.nb));
  k_vrhs<T><<<grid, 256, 0, st>>>(g, cf, out, Q, f, vedge, srcv, gam);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_urhs(const Geom& g, const Coefs& cf, T* out, const T* V, const T* ainv, const double* Q,
                        const double* gD, cudaStream_t st, const T* srcu) {
  const dim3 grid((unsigned)((g.n0 + 255) / 256), (unsigned)g.n1, (unsigned)(g.n2 * g.nb));
  k_urhs<T><<<grid, 256, 0, st>>>(g, cf, out, V, ainv, Q, gD, srcu);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_trace(const Geom& g, const Coefs& cf, double* y, const T* U, const double* Q,
                         const double* afac, const double* gD, const double* gN, const double* lapt,
                         cudaStream_t st, const double* srcq, const double* gL) {
  k_trace<T><<<dim3(nblk(g.ngamma, 256), g.nb), 256, 0, st>>>(g, cf, y, U, Q, afac, gD, gN, lapt, srcq, gL);
  return cudaGetLastError();
}
cudaError_t launch_trace_tri(const Geom& g, const Coefs& cf, double* y, const double* U, const double* Q,
                             const double* gD, const double* gN, const double* gNN, const double* laptw,
                             const double* bilap, cudaStream_t st) {
  k_trace_tri<<<dim3(nblk(g.ngamma, 256), g.nb), 256, 0, st>>>(g, cf, y, U, Q, gD, gN, gNN, laptw, bilap);
  return cudaGetLastError();
}
cudaError_t launch_write_full(const Geom& g, double* out, const double* Uin, const double* bnd, cudaStream_t st) {
  k_write_full<<<dim3(nblk(g.nfull, 256), g.nb), 256, 0, st>>>(g, out, Uin, bnd);
  return cudaGetLastError();
}
cudaError_t launch_v_full(const Geom& g, double* vfull, const double* Vpad, const double* Q, const double* vedge,
                          cudaStream_t st) {
  k_v_full<<<dim3(nblk(g.nfull, 256), g.nb), 256, 0, st>>>(g, vfull, Vpad, Q, vedge);
  return cudaGetLastError();
}
cudaError_t launch_pack(const Geom& g, double* dense, const double* padded, cudaStream_t st) {
  k_pack<<<nblk(g.nint, 256), 256, 0, st>>>(g, dense, padded);
  return cudaGetLastError();
}
cudaError_t launch_unpack(const Geom& g, double* padded, const double* dense, cudaStream_t st) {
  k_unpack<<<nblk(g.nint, 256), 256, 0, st>>>(g, padded, dense);
  return cudaGetLastError();
}
cudaError_t launch_face_gather(const Geom& g, double* face, const double* full, cudaStream_t st) {
  k_face_gather<<<dim3(nblk(g.ngamma, 256), g.nb), 256, 0, st>>>(g, face, full);
  return cudaGetLastError();
}
__global__ void k_fill_scaled_recip(double* __restrict__ out, const double* __restrict__ in, double a, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = in ? a / in[t] : a;
}
cudaError_t launch_scaled_recip(double* out, const double* in, double a, int64_t n, cudaStream_t st) {
  k_fill_scaled_recip<<<nblk(n, 256), 256, 0, st>>>(out, in, a, n);
  return cudaGetLastError();
}
cudaError_t launch_recip(double* out, const double* in, int64_t n, cudaStream_t st) {
  k_recip<<<nblk(n, 256), 256, 0, st>>>(out, in, n);
  return cudaGetLastError();
}

template cudaError_t launch_vrhs<double>(const Geom&, const Coefs&, double*, const double*, const double*,
                                         const double*, cudaStream_t, const double*, const double*);
template cudaError_t launch_urhs<double>(const Geom&, const Coefs&, double*, const double*, const double*,
                                         const double*, const double*, cudaStream_t, const double*);
template cudaError_t launch_trace<double>(const Geom&, const Coefs&, double*, const double*, const double*,
                                          const double*, const double*, const double*, const double*, cudaStream_t,
                                          const double*, const double*);
template cudaError_t launch_vrhs<float>(const Geom&, const Coefs&, float*, const double*, const double*,
                                        const double*, cudaStream_t, const float*, const double*);
template cudaError_t launch_urhs<float>(const Geom&, const Coefs&, float*, const float*, const float*,
                                        const double*, const double*, cudaStream_t, const float*);
template cudaError_t launch_trace<float>(const Geom&, const Coefs&, double*, const float*, const double*,
                                         const double*, const double*, const double*, const double*, cudaStream_t,
                                         const double*, const double*);

}  // namespace ahoc

namespace ahoc {

// ---------------------------------------------------------------------------
// Grid transfer for the nested (coarse-to-fine) initial guess: coarse data
// by injection (the coarse grid points are every other fine point), and the
// coarse Q prolonged to the fine face points by cubic Lagrange interpolation
// along each in-face axis (one-sided near the face edges).
// ---------------------------------------------------------------------------
__global__ void k_inject_full(Geom gc, Geom gf, double* __restrict__ out, const double* __restrict__ in) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.nfull || gc.skip(blockIdx.y)) return;
  out += (int64_t)blockIdx.y * gc.nfull;
  in += (int64_t)blockIdx.y * gf.nfull;
  const int i = (int)(t % gc.f0);
  const int64_t r = t / gc.f0;
  const int j = (int)(r % gc.f1);
  const int k = (int)(r / gc.f1);
  out[t] = in[gf.full(2 * i, 2 * j, 2 * k)];
}

__device__ __forceinline__ void face_coords(const Geom& g, int64_t q, int& a, int& side, int c[3]) {
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  a = f >> 1;
  side = f & 1;
  int64_t r = q - g.face_off[f];
  c[0] = c[1] = c[2] = 0;
  for (int b = 0; b < g.dim; ++b) {
    if (b == a) continue;
    const int nb = g.N[b] - 1;
    c[b] = 1 + (int)(r % nb);
    r /= nb;
  }
  c[a] = side ? g.N[a] : 0;
}

__global__ void k_inject_face(Geom gc, Geom gf, double* __restrict__ out, const double* __restrict__ in) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= gc.ngamma || gc.skip(blockIdx.y)) return;
  out += (int64_t)blockIdx.y * gc.ngamma;
  in += (int64_t)blockIdx.y * gf.ngamma;
  int a, side, c[3];
  face_coords(gc, q, a, side, c);
  out[q] = in[gf.face(a, side, 2 * c[0], 2 * c[1], 2 * c[2])];
}

// nodes and weights of the fine coordinate cf on the coarse line 1..Nc-1
__device__ __forceinline__ int prolong_weights(int cf, int Nc, int* node, double* w) {
  if ((cf & 1) == 0) {
    node[0] = cf >> 1;
    w[0] = 1.0;
    return 1;
  }
  const double t = 0.5 * cf;
  int lo = (cf >> 1) - 1;  // floor(t) - 1
  if (lo < 1) lo = 1;
  if (lo > Nc - 4) lo = Nc - 4;
  for (int m = 0; m < 4; ++m) {
    double l = 1.0;
    for (int n = 0; n < 4; ++n)
      if (n != m) l *= (t - (lo + n)) / (double)(m - n);
    node[m] = lo + m;
    w[m] = l;
  }
  return 4;
}

__global__ void k_face_prolong(Geom gf, Geom gc, double* __restrict__ out, const double* __restrict__ in) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= gf.ngamma || gf.skip(blockIdx.y)) return;
  out += (int64_t)blockIdx.y * gf.ngamma;
  in += (int64_t)blockIdx.y * gc.ngamma;
  int a, side, c[3];
  face_coords(gf, q, a, side, c);
  int rem[2] = {-1, -1}, nr = 0;
  for (int b = 0; b < gf.dim; ++b)
    if (b != a) rem[nr++] = b;
  int n0[4], n1[4] = {0, 0, 0, 0};
  double w0[4], w1[4] = {1.0, 0, 0, 0};
  const int k0 = prolong_weights(c[rem[0]], gc.N[rem[0]], n0, w0);
  int k1 = 1;
  if (nr == 2) k1 = prolong_weights(c[rem[1]], gc.N[rem[1]], n1, w1);
  double acc = 0.0;
  for (int u = 0; u < k0; ++u)
    for (int v = 0; v < k1; ++v) {
      int cc[3] = {0, 0, 0};
      cc[a] = side ? gc.N[a] : 0;
      cc[rem[0]] = n0[u];
      if (nr == 2) cc[rem[1]] = n1[v];
      acc += w0[u] * w1[v] * in[gc.face(a, side, cc[0], cc[1], cc[2])];
    }
  out[q] = acc;
}

cudaError_t launch_inject_full(const Geom& gc, const Geom& gf, double* out, const double* in, cudaStream_t st) {
  k_inject_full<<<dim3(nblk(gc.nfull, 256), gc.nb), 256, 0, st>>>(gc, gf, out, in);
  return cudaGetLastError();
}
cudaError_t launch_inject_face(const Geom& gc, const Geom& gf, double* out, const double* in, cudaStream_t st) {
  k_inject_face<<<dim3(nblk(gc.ngamma, 256), gc.nb), 256, 0, st>>>(gc, gf, out, in);
  return cudaGetLastError();
}
cudaError_t launch_face_prolong(const Geom& gf, const Geom& gc, double* out, const double* in, cudaStream_t st) {
  k_face_prolong<<<dim3(nblk(gf.ngamma, 256), gf.nb), 256, 0, st>>>(gf, gc, out, in);
  return cudaGetLastError();
}

}  // namespace ahoc

namespace ahoc {

// ---------------------------------------------------------------------------
// Iterative refinement of the coupled system (mixed precision): the FP64
// residual r = F - A x of the three block rows of Sec. 2.2 at the current
// iterate x = (U, V, Q), U and V padded FP64 fields, boundary values from the
// data (U = g_D, V = Q on faces, v_edge on edges and corners):
//   r_u = -(L_h U - M(V/alpha))            (u-equation, right-hand side 0)
//   r_v = M f - (-L_h V + gam M V)          (v-equation, gam = beta / alpha constant)
//   r_q = -(alpha (delta_nn U + lapt) - Q)  (augmented equation, Lemma 1's R; on a
//                                            Navier face -(alpha g_L - Q))
// r_u and r_v are stored in FP32 (they are the sources of an FP32 correction
// solve), r_q in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ufull(const Geom& g, const double* U, const double* gD, int i, int j, int k) {
  int ax, sd;
  if (bclass(g, i, j, k, ax, sd) == 0) return U[g.pad(i, j, k)];
  return gD ? gD[g.full(i, j, k)] : 0.0;
}
__device__ __forceinline__ double vfull(const Geom& g, const double* V, const double* Q, const double* vedge, int i,
                                        int j, int k) {
  int ax, sd;
  const int nb = bclass(g, i, j, k, ax, sd);
  if (nb == 0) return V[g.pad(i, j, k)];
  if (nb == 1) return Q[g.face(ax, sd, i, j, k)];
  return vedge ? vedge[g.full(i, j, k)] : 0.0;
}

// DIM: 2 or 3 (the stencil loops unroll: the 3D corners, which carry no
// weight, cost nothing).  SH: the shift term of the v-row, 0 none, 1 the
// constant cf.gam, 2 the field gam (separate instantiations: this kernel is
// bound by the FP64 pipe, and a runtime branch becomes predicated FP64
// operations)
template <int DIM, int SH>
__global__ void k_residual(Geom g, Coefs cf, const double* __restrict__ gam, float* __restrict__ ru,
                           float* __restrict__ rv, const double* __restrict__ U, const double* __restrict__ V, const double* __restrict__ Q,
                           const double* __restrict__ f, const double* __restrict__ gD,
                           const double* __restrict__ vedge, const double* __restrict__ ainv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (t >= g.npad || g.skip(bi)) return;
  {
    const int64_t po = (int64_t)bi * g.npad, fo = (int64_t)bi * g.nfull;
    ru += po;
    rv += po;
    U += po;
    V += po;
    Q += (int64_t)bi * g.ngamma;
    if (f) f += fo;
    if (gD) gD += fo;
    if (vedge) vedge += fo;
    ainv += fo;
    if (gam) gam += fo;
  }
  int i, j, k;
  decompose(g, t, i, j, k);
  if (is_pad(g, i, j, k)) {
    ru[t] = 0.f;
    rv[t] = 0.f;
    return;
  }
  const bool near = near_bdry(g, i, j, k);
  double lu = 0.0, lv = 0.0;
  constexpr int dzlo = (DIM == 3) ? -1 : 0, dzhi = (DIM == 3) ? 1 : 0;
#pragma unroll
  for (int dz = dzlo; dz <= dzhi; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (DIM == 3 && dx != 0 && dy != 0 && dz != 0) continue;  // the 19-point stencil has no corners
        const double c = cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        const int ii = i + dx, jj = j + dy, kk = k + dz;
        if (near) {
          lu += c * ufull(g, U, gD, ii, jj, kk);
          lv += c * vfull(g, V, Q, vedge, ii, jj, kk);
        } else {
          const int64_t o = g.pad(ii, jj, kk);
          lu += c * U[o];
          lv += c * V[o];
        }
      }
  // M(V/alpha), M(gam V) (the shift term) and M f: centre and the axis
  // neighbours; the neighbour sums are formed first and weighted once (this
  // kernel is bound by the FP64 pipe)
  const int64_t fc = g.full(i, j, k);
  const double vc = V[t];
  double swn = 0.0, svn = 0.0, sgn = 0.0, sfn = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int s = -1; s <= 1; s += 2) {
      const int ii = i + (a == 0 ? s : 0), jj = j + (a == 1 ? s : 0), kk = k + (a == 2 ? s : 0);
      const int64_t fn = g.full(ii, jj, kk);
      const double vn = near ? vfull(g, V, Q, vedge, ii, jj, kk) : V[g.pad(ii, jj, kk)];
      swn = fma(vn, ainv[fn], swn);
      if (SH == 2) sgn = fma(vn, gam[fn], sgn);
      if (SH == 1) svn += vn;
      if (f) sfn += f[fn];
    }
  const double mv = fma(cf.Mn, swn, cf.Mc * (vc * ainv[fc]));
  double mgv = 0.0;
  if (SH == 2) mgv = fma(cf.Mn, sgn, cf.Mc * (vc * gam[fc]));
  if (SH == 1) mgv = cf.gam * fma(cf.Mn, svn, cf.Mc * vc);
  const double mf = f ? fma(cf.Mn, sfn, cf.Mc * f[fc]) : 0.0;
  ru[t] = (float)(mv - lu);
  rv[t] = (float)(SH ? (mf + lv - mgv) : (mf + lv));
}

// r_q at every face point (FP64)
__global__ void k_residual_q(Geom g, Coefs cf, double* __restrict__ rq, const double* __restrict__ U,
                             const double* __restrict__ Q, const double* __restrict__ afac,
                             const double* __restrict__ gD, const double* __restrict__ gN,
                             const double* __restrict__ lapt, const double* __restrict__ gL) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (q >= g.ngamma || g.skip(bi)) return;
  {
    const int64_t fo = (int64_t)bi * g.ngamma;
    rq += fo;
    U += (int64_t)bi * g.npad;
    Q += fo;
    afac += fo;
    if (gD) gD += (int64_t)bi * g.nfull;
    if (gN) gN += fo;
    if (lapt) lapt += fo;
    if (gL) gL += fo;
  }
  int a, side, c[3];
  face_coords(g, q, a, side, c);
  if (g.is_navier(2 * a + side)) {
    rq[q] = -((gL ? afac[q] * gL[q] : 0.0) - Q[q]);
    return;
  }
  const int step = side ? -1 : 1;
  int p[3] = {c[0], c[1], c[2]};
  double unn = gD ? cf.w[a][0] * gD[g.full(c[0], c[1], c[2])] : 0.0;
  for (int m = 1; m <= 3; ++m) {
    p[a] = c[a] + m * step;
    unn += cf.w[a][m] * U[g.pad(p[0], p[1], p[2])];
  }
  if (gN) unn += cf.wg[a] * gN[q];
  if (lapt) unn += lapt[q];
  rq[q] = -(afac[q] * unn - Q[q]);
}

// x += correction: U += dU, V += dV (FP32 padded fields), with the block
// partial sums of dU^2 and of the updated U^2 (the size of the correction
// relative to the iterate, for the refinement's stopping test)
constexpr int kAccThreads = 512;
__global__ void __launch_bounds__(kAccThreads) k_accumulate(Geom g, double* __restrict__ U, const float* __restrict__ dU,
                                                            double* __restrict__ V, const float* __restrict__ dV,
                                                            double* __restrict__ partial) {
  __shared__ double red[2][kAccThreads / 32];
  double sdu = 0.0, su = 0.0;
  const int bi = blockIdx.y;
  const int64_t n = g.skip(bi) ? 0 : g.npad;  // a masked problem contributes zero partials
  {
    const int64_t po = (int64_t)bi * g.npad;
    U += po;
    dU += po;
    V += po;
    dV += po;
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double du = (double)dU[t];
    const double u = U[t] + du;
    U[t] = u;
    V[t] += (double)dV[t];
    sdu = fma(du, du, sdu);
    su = fma(u, u, su);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sdu += __shfl_down_sync(0xffffffffu, sdu, o);
    su += __shfl_down_sync(0xffffffffu, su, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = sdu;
    red[1][warp] = su;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kAccThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    // partial[block][problem][2]: column 2 bi + c of a (2 nb)-column reduction
    const int64_t o = 2 * ((int64_t)blockIdx.x * g.nb + bi);
    partial[o] = a;
    partial[o + 1] = b;
  }
}

cudaError_t launch_residual(const Geom& g, const Coefs& cf, float* ru, float* rv, double* rq, const double* U,
                            const double* V, const double* Q, const double* f, const double* gD, const double* vedge,
                            const double* gN, const double* lapt, const double* ainv, const double* afac,
                            cudaStream_t st, const double* gL, const double* gam) {
  const dim3 grid(nblk(g.npad, 256), g.nb);
  const int sh = gam ? 2 : (cf.gam != 0.0 ? 1 : 0);
#define AHOC_RESID(D, S) k_residual<D, S><<<grid, 256, 0, st>>>(g, cf, gam, ru, rv, U, V, Q, f, gD, vedge, ainv)
  if (g.dim == 3) {
    if (sh == 2) AHOC_RESID(3, 2);
    else if (sh == 1) AHOC_RESID(3, 1);
    else AHOC_RESID(3, 0);
  } else {
    if (sh == 2) AHOC_RESID(2, 2);
    else if (sh == 1) AHOC_RESID(2, 1);
    else AHOC_RESID(2, 0);
  }
#undef AHOC_RESID
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_residual_q<<<dim3(nblk(g.ngamma, 256), g.nb), 256, 0, st>>>(g, cf, rq, U, Q, afac, gD, gN, lapt, gL);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const Geom& g, double* U, const float* dU, double* V, const float* dV,
                              double* partial, int nblocks, double* out, cudaStream_t st) {
  k_accumulate<<<dim3(nblocks, g.nb), kAccThreads, 0, st>>>(g, U, dU, V, dV, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_cols(partial, nblocks, 2 * g.nb, out, st);
}

}  // namespace ahoc

namespace ahoc {

// ---------------------------------------------------------------------------
// Variable beta / alpha (Sec. 2.2 v-equation, beta/alpha not constant): the
// interior operator B V = L_h V - M(gam V) with V = 0 on the boundary
// (gam = beta/alpha on the full grid), for the preconditioned BiCGSTAB
// v-solve (Sec. 4, solver settings), and the linear combinations it needs.
// ---------------------------------------------------------------------------
__global__ void k_vop(Geom g, Coefs cf, double* __restrict__ y, const double* __restrict__ x,
                      const double* __restrict__ gam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.z / (int)g.n2;
  if (i >= g.n0 || g.skip(bi)) return;
  const int j = blockIdx.y, k = blockIdx.z - bi * (int)g.n2;
  y += (int64_t)bi * g.npad;
  x += (int64_t)bi * g.npad;
  gam += (int64_t)bi * g.nfull;
  const int64_t t = g.pad(i, j, k);
  if (is_pad(g, i, j, k)) {
    y[t] = 0.0;
    return;
  }
  auto xv = [&](int ii, int jj, int kk) -> double {
    int ax, sd;
    return bclass(g, ii, jj, kk, ax, sd) ? 0.0 : x[g.pad(ii, jj, kk)];
  };
  double acc = 0.0;
  const int dzlo = (g.dim == 3) ? -1 : 0, dzhi = (g.dim == 3) ? 1 : 0;
  for (int dz = dzlo; dz <= dzhi; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const double c = cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        if (c != 0.0) acc += c * xv(i + dx, j + dy, k + dz);
      }
  double m = cf.Mc * gam[g.full(i, j, k)] * x[t];
  for (int a = 0; a < g.dim; ++a)
    for (int s = -1; s <= 1; s += 2) {
      const int ii = i + (a == 0 ? s : 0), jj = j + (a == 1 ? s : 0), kk = k + (a == 2 ? s : 0);
      m += cf.Mn * gam[g.full(ii, jj, kk)] * xv(ii, jj, kk);
    }
  y[t] = acc - m;
}

// y = c[3b] x0 + c[3b + 1] x1 + c[3b + 2] x2 per problem b (x1, x2 may be NULL;
// any x may alias y), over n entries per problem
__global__ void k_comb(int64_t n, const int* act, double* __restrict__ y, const double* x0, const double* x1,
                       const double* x2, const double* __restrict__ c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (i >= n || (act && !act[bi])) return;
  const int64_t o = (int64_t)bi * n + i;
  double v = c[3 * bi] * x0[o];
  if (x1) v += c[3 * bi + 1] * x1[o];
  if (x2) v += c[3 * bi + 2] * x2[o];
  y[o] = v;
}

__global__ void k_mul(double* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b,
                      int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = a[t] * b[t];
}

cudaError_t launch_vop(const Geom& g, const Coefs& cf, double* y, const double* x, const double* gam,
                       cudaStream_t st) {
  const dim3 grid((unsigned)((g.n0 + 255) / 256), (unsigned)g.n1, (unsigned)(g.n2 * g.nb));
  k_vop<<<grid, 256, 0, st>>>(g, cf, y, x, gam);
  return cudaGetLastError();
}
cudaError_t launch_comb(const Geom& g, int64_t n, double* y, const double* x0, const double* x1, const double* x2,
                        const double* c, cudaStream_t st) {
  k_comb<<<dim3(nblk(n, 256), g.nb), 256, 0, st>>>(n, g.act, y, x0, x1, x2, c);
  return cudaGetLastError();
}
cudaError_t launch_mul(double* out, const double* a, const double* b, int64_t n, cudaStream_t st) {
  k_mul<<<nblk(n, 256), 256, 0, st>>>(out, a, b, n);
  return cudaGetLastError();
}

}  // namespace ahoc
