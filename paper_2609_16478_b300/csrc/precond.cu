// Boundary-symbol preconditioner for the Schur system S_h Q = b.
//
// The paper drives GMRES with a "boundary-symbol preconditioner" (Sec. 4,
// solver settings) without defining it.  This is our construction: for a
// single clamped face with alpha = 1 and zero data on the other faces, the
// Schur action is diagonal in the face's transverse sine basis (the
// representation of Lemma 4): a face mode l excites V = q_l * (discrete
// harmonic profile along the normal), U = L_h^-1 M V, and the trace
// alpha * delta_nn U - q returns s_l * q_l with
//
//   s_l = (2/N_a) sum_k sin(k pi/N_a) (m_o a_l - b_l m_d) / lam_k^2
//                        * sum_{m=1..3} w_m sin(m k pi/N_a)  - 1,
//   lam_k = a_l + 2 b_l cos(k pi/N_a),
//
// where (a_l, b_l) are the centre and normal-neighbour weights of L_h and
// (m_d, m_o) those of M in the transverse mode l, and w_m the one-sided
// weights along the normal a.  With the shift gam = beta/alpha of the
// v-equation the V extension solves with L_h - gam M, whose weights are
// aV_l = a_l - gam m_d, bV_l = b_l - gam m_o, and the summand becomes
//   (m_o lamV_k - bV_l Mhat_k) / (lamV_k lam_k),  Mhat_k = m_d + 2 m_o cos(k pi/N_a),
// lamV_k = aV_l + 2 bV_l cos(k pi/N_a) (the form above at gam = 0).  A Navier
// face has the symbol -1: its augmented rows are -I.  The preconditioner
// applies, face by face,
//   P^-1 q = D_alpha  DST^-1 [ DST(D_alpha^-1 q) / s ],
// i.e. the inverse of that single-face symbol with the coefficient frozen
// pointwise on the face (for constant alpha the scaling cancels exactly).
#include "common.cuh"
#include "kernels.cuh"

namespace ahoc {

// pre[q] = prod_{b != a} (2 / N_b) / s_l(q): the normalisation of the inverse
// transverse DSTs is folded in.
__global__ void k_face_symbols(Geom g, Coefs cf, double* __restrict__ pre, const double* __restrict__ st0,
                               const double* __restrict__ st1, const double* __restrict__ st2,
                               const double* __restrict__ ct0, const double* __restrict__ ct1,
                               const double* __restrict__ ct2) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.ngamma) return;
  int f = 0;
  while (q >= g.face_off[f + 1]) ++f;
  const int a = f >> 1;
  int64_t r = q - g.face_off[f];
  int l[3] = {0, 0, 0};
  for (int b = 0; b < g.dim; ++b) {
    if (b == a) continue;
    const int nb = g.N[b] - 1;
    l[b] = 1 + (int)(r % nb);
    r /= nb;
  }
  const double* ct[3] = {ct0, ct1, ct2};
  const double* stab = (a == 0) ? st0 : (a == 1) ? st1 : st2;
  double c[3] = {1.0, 1.0, 1.0};
  for (int b = 0; b < g.dim; ++b)
    if (b != a) c[b] = ct[b][l[b]];
  // transverse-mode weights of L_h (centre plane and one normal neighbour plane) and of M
  double al = 0.0, bl = 0.0;
  const int dzlo = (g.dim == 3) ? -1 : 0, dzhi = (g.dim == 3) ? 1 : 0;
  for (int dz = dzlo; dz <= dzhi; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const double w = cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        if (w == 0.0) continue;
        const int o[3] = {dx, dy, dz};
        if (o[a] < 0) continue;
        double t = w;
        for (int b = 0; b < g.dim; ++b)
          if (b != a && o[b] != 0) t *= c[b];
        if (o[a] == 0) al += t;
        else bl += t;
      }
  double md = cf.Mc;
  for (int b = 0; b < g.dim; ++b)
    if (b != a) md += 2.0 * cf.Mn * c[b];
  const double mo = cf.Mn;
  double norm = 1.0;
  for (int b = 0; b < g.dim; ++b)
    if (b != a) norm *= 2.0 / g.N[b];
  if (g.is_navier(f)) {
    pre[q] = -norm;
    return;
  }
  const double av = al - cf.gam * md, bv = bl - cf.gam * mo;
  const int Na = g.N[a];
  const double* ca = ct[a];
  double kap = 0.0;
  for (int k = 1; k < Na; ++k) {
    const double s1 = stab[k];
    const double s2 = stab[(2 * k) % (2 * Na)];
    const double s3 = stab[(3 * k) % (2 * Na)];
    const double lam = al + 2.0 * bl * ca[k];
    const double lamv = av + 2.0 * bv * ca[k];
    const double mhat = md + 2.0 * mo * ca[k];
    const double tr = cf.w[a][1] * s1 + cf.w[a][2] * s2 + cf.w[a][3] * s3;
    kap += s1 * (mo * lamv - bv * mhat) / (lamv * lam) * tr;
  }
  kap *= 2.0 / Na;
  pre[q] = norm / (kap - 1.0);
}

__global__ void k_face_muldiv(double* __restrict__ out, const double* __restrict__ in, const double* __restrict__ mul,
                              const double* __restrict__ div, int64_t n, int64_t mstride, int64_t dstride,
                              const int* act) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bi = blockIdx.y;
  if (i >= n || (act && !act[bi])) return;
  out += (int64_t)bi * n;
  in += (int64_t)bi * n;
  if (mul) mul += (int64_t)bi * mstride;
  if (div) div += (int64_t)bi * dstride;
  double v = in[i];
  if (mul) v *= mul[i];
  if (div) v /= div[i];
  out[i] = v;
}

cudaError_t launch_face_symbols(const Geom& g, const Coefs& cf, double* pre, const double* const* stab,
                                const double* const* ctab, cudaStream_t st) {
  const unsigned blocks = (unsigned)((g.ngamma + 127) / 128);
  k_face_symbols<<<blocks, 128, 0, st>>>(g, cf, pre, stab[0], stab[1], stab[2], ctab[0], ctab[1], ctab[2]);
  return cudaGetLastError();
}

cudaError_t launch_face_muldiv(double* out, const double* in, const double* mul, const double* div, int64_t n,
                               cudaStream_t st, int nb, int64_t mstride, int64_t dstride, const int* act) {
  k_face_muldiv<<<dim3((unsigned)((n + 255) / 256), nb), 256, 0, st>>>(out, in, mul, div, n, mstride, dstride, act);
  return cudaGetLastError();
}

}  // namespace ahoc
