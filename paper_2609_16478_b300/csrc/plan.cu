// Plan, solver engine and C ABI of the augmented HOC method (Sec. 2.3,
// Algorithm 1): ConstructSchurRHS, SchurMatVec, GMRES on S_h Q = b, recovery.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ahoc.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace ahoc;

namespace {

thread_local std::string g_err;

// NVTX range over one phase of a solve, for profilers (ncu --nvtx
// --nvtx-include, nsys); with no tool attached a push or pop returns at once
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
};

ahoc_status fail(ahoc_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

// Device arrays of doubles must be 8-byte aligned: a kernel's 8-byte load
// from a misaligned address would fault the context, so such a pointer is
// refused on the host before any launch (NULL passes).
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) != 0; }

bool bdata_misaligned(const ahoc_bdata* bd) {
  if (!bd) return false;
  const void* ps[] = {bd->g_D, bd->g_N, bd->lapt_gD, bd->v_edge, bd->g_L,
                      bd->beta, bd->lap_gD, bd->bilap, bd->g_NN, bd->lapt_w};
  for (const void* q : ps)
    if (misaligned(q)) return true;
  return false;
}

constexpr const char* kAlignMsg = "device arrays of doubles must be 8-byte aligned";

// beta / alpha < 0 (the high-wavenumber problem of Sec. 4.2, beta = -k^2)
// makes the v-equation a Helmholtz equation with an indefinite shift, whose
// per-mode factors along the last axis are not diagonally dominant
constexpr const char* kIndefiniteMsg =
    "beta / alpha < 0 (an indefinite Helmholtz v-equation) is outside the exact last-axis factorisation";

// Serialises CUDA graph captures with the library's own synchronising entry
// points (plan creation, loading, destruction: pinned allocations, frees,
// stream synchronisations), which would otherwise invalidate a capture open
// in another thread.
std::recursive_mutex& capture_mutex() {
  static std::recursive_mutex m;
  return m;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(AHOC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

#define CKS(expr)                  \
  do {                             \
    ahoc_status s_ = (expr);       \
    if (s_ != AHOC_OK) return s_;  \
  } while (0)

bool pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

struct Opts {
  ahoc_precision prec = AHOC_FP64;
  int max_iters = 500;
  int restart = 100;
  int precond = 1;
  int timing = 0;
  int levels = -1;  // coarse levels of the nested initial guess (-1: automatic)
  double refine_tol = 3e-6;  // mixed precision: relative residual of each FP32 correction solve
  double coarse_tol = AHOC_COARSE_TOL_AUTO;  // relative Schur residual of the coarse levels
  int batch = 1;  // problems of this shape solved together
  int graphs = 1;  // replay GMRES iterations as CUDA graphs
  int navier = 0;        // Navier faces (bit 2a + side)
  double shift = 0.0;    // constant beta / alpha of the v-equation (reference value if variable)
  int varb = 0;          // variable beta / alpha (problems bring beta)
  int uhat = 0;          // U-hat slots of the recovery (0 automatic, < 0 none)
  int unfused = 0;       // 3D: the plain Schur matvec (eight DST passes) instead of the fused one
  int tri = 0;           // the triharmonic class: Lap^3 u = f, navier = the simply supported faces
  int first64 = 1;       // mixed: right-hand side and recovery of the first correction in FP64
  int nest_auto = 0;     // automatic nested guess: a coarse level is used only where it resolves the data
  void* workspace = nullptr;
  size_t workspace_bytes = 0;
};

ahoc_status read_opts(const ahoc_opts* o, Opts* out) {
  Opts d;
  if (o) {
    d.prec = o->prec;
    if (o->max_iters > 0) d.max_iters = o->max_iters;
    if (o->restart > 0) d.restart = o->restart;
    d.precond = o->precond < 0 ? 1 : o->precond;
    d.timing = o->timing;
    d.levels = o->levels;
    d.nest_auto = o->levels < 0 ? 1 : 0;
    if (o->refine_tol > 0) d.refine_tol = o->refine_tol;
    if (o->coarse_tol > 0) d.coarse_tol = o->coarse_tol;
    else if (o->prec == AHOC_MIXED) d.coarse_tol = AHOC_COARSE_TOL_AUTO_MIXED;
    if (o->batch > 0) d.batch = o->batch;
    d.graphs = o->no_graphs ? 0 : 1;
    d.navier = o->navier;
    d.shift = o->shift;
    d.varb = o->variable_beta ? 1 : 0;
    d.uhat = o->uhat_slots;
    d.unfused = o->unfused ? 1 : 0;
    d.tri = o->triharmonic ? 1 : 0;
    d.first64 = o->first32 ? 0 : 1;
    d.workspace = o->workspace;
    d.workspace_bytes = o->workspace_bytes;
  }
  if (d.prec != AHOC_FP64 && d.prec != AHOC_MIXED) return fail(AHOC_EUNSUPPORTED, "prec must be AHOC_FP64 or AHOC_MIXED");
  if (d.tri) {
    if (d.prec != AHOC_FP64) return fail(AHOC_EUNSUPPORTED, "the triharmonic class runs in FP64 only");
    if (d.varb || d.shift != 0.0) return fail(AHOC_EINVAL, "the triharmonic class takes no beta");
    d.levels = 0;
    d.uhat = -1;
  }
  // automatic depth: the nested guess of a mixed plan only shortens its first
  // correction solve (the later ones start from zero), which did not repay
  // the coarse solves on B300 (2D 4096^2: 55 against 47 ms; 3D 512^3: 2 %
  // faster); an explicit depth is honoured
  if (d.prec == AHOC_MIXED && d.levels < 0) d.levels = 0;
  if (d.precond != 0 && d.precond != 1) return fail(AHOC_EINVAL, "precond must be 0 (none) or 1 (boundary symbol)");
  if (d.restart > 1000) return fail(AHOC_EINVAL, "restart > 1000");
  if (d.batch > 4096) return fail(AHOC_EINVAL, "batch > 4096");
  if (d.navier < 0 || d.navier > 63) return fail(AHOC_EINVAL, "navier must be a mask of faces 0..5");
  if (!std::isfinite(d.shift)) return fail(AHOC_EINVAL, "shift must be finite");
  if (d.shift < 0) return fail(AHOC_EUNSUPPORTED, kIndefiniteMsg);
  if (d.levels < -1 || d.levels > 8) return fail(AHOC_EINVAL, "levels must be -1 (automatic) or 0..8");
  if (d.workspace && (reinterpret_cast<uintptr_t>(d.workspace) & 255))
    return fail(AHOC_EINVAL, "workspace must be 256-byte aligned");
  *out = d;
  return AHOC_OK;
}

ahoc_status make_geom(int dim, const int64_t* N, const double* lo, const double* hi, Geom* g) {
  if (dim != 2 && dim != 3) return fail(AHOC_EINVAL, "dim must be 2 or 3");
  if (!N) return fail(AHOC_EINVAL, "N is NULL");
  for (int a = 0; a < dim; ++a) {
    if (N[a] < 8 || N[a] > kMaxN || !pow2(N[a]))
      return fail(AHOC_EUNSUPPORTED, "N[a] must be a power of two in [8, 4096]");
  }
  std::memset(g, 0, sizeof(*g));
  g->dim = dim;
  for (int a = 0; a < 3; ++a) g->N[a] = (a < dim) ? (int)N[a] : 1;
  for (int a = 0; a < dim; ++a) {
    const double l = lo ? lo[a] : 0.0, r = hi ? hi[a] : 1.0;
    if (!(r > l) || !std::isfinite(l) || !std::isfinite(r)) return fail(AHOC_EINVAL, "need lo[a] < hi[a], finite");
    g->h[a] = (r - l) / (double)N[a];
  }
  g->n0 = g->N[0];
  g->n1 = g->N[1];
  g->n2 = (dim == 3) ? g->N[2] : 1;
  g->npad = g->n0 * g->n1 * g->n2;
  g->f0 = g->N[0] + 1;
  g->f1 = g->N[1] + 1;
  g->f2 = (dim == 3) ? g->N[2] + 1 : 1;
  g->nfull = g->f0 * g->f1 * g->f2;
  g->kmin = (dim == 3) ? 1 : 0;
  g->kmax = (dim == 3) ? g->N[2] : 1;
  g->nint = 1;
  for (int a = 0; a < dim; ++a) g->nint *= (N[a] - 1);
  g->face_off[0] = 0;
  for (int a = 0; a < 3; ++a) {
    int64_t s = 0;
    if (a < dim) {
      s = 1;
      for (int b = 0; b < dim; ++b)
        if (b != a) s *= (N[b] - 1);
    }
    g->face_off[2 * a + 1] = g->face_off[2 * a] + s;
    g->face_off[2 * a + 2] = g->face_off[2 * a + 1] + s;
  }
  g->ngamma = g->face_off[6];
  g->nb = 1;
  g->act = nullptr;
  return AHOC_OK;
}

// Weights of the one-sided fourth normal derivative at a clamped face of the
// triharmonic class: with U_m = u(m h) along the inward normal s,
//   sum_{m=0}^{4} c_m U_m + c_s h u_s + c_ss h^2 u_ss = h^4 u_ssss + O(h^7).
// Expanding U_m = sum_k (m h)^k / k! u_k, the coefficients of u_3..u_6 give
// four equations in c_1..c_4 (right-hand side 1 for u_4, 0 otherwise); those
// of u_0, u_1, u_2 then give c_0, c_s, c_ss.  Solved here in long double.
void fourth_weights(long double c[5], long double& cs, long double& css) {
  long double A[4][5];
  for (int k = 3; k <= 6; ++k) {
    long double fact = 1;
    for (int t = 2; t <= k; ++t) fact *= t;
    for (int m = 1; m <= 4; ++m) A[k - 3][m - 1] = powl((long double)m, (long double)k) / fact;
    A[k - 3][4] = (k == 4) ? 1.0L : 0.0L;
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabsl(A[r][col]) > fabsl(A[piv][col])) piv = r;
    for (int t = 0; t < 5; ++t) std::swap(A[col][t], A[piv][t]);
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const long double f = A[r][col] / A[col][col];
      for (int t = col; t < 5; ++t) A[r][t] -= f * A[col][t];
    }
  }
  c[0] = 0;
  cs = 0;
  css = 0;
  for (int m = 1; m <= 4; ++m) {
    c[m] = A[m - 1][4] / A[m - 1][m - 1];
    c[0] -= c[m];
    cs -= c[m] * m;
    css -= c[m] * m * m / 2.0L;
  }
}

// Stencil coefficients (Sec. 2.2; prefactor 1/12; 2D nine-point operator).
Coefs make_coefs(const Geom& g) {
  Coefs c;
  std::memset(&c, 0, sizeof(c));
  double inv[3] = {0, 0, 0};
  for (int a = 0; a < g.dim; ++a) inv[a] = 1.0 / (g.h[a] * g.h[a]);
  if (g.dim == 2) {
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        double v;
        if (dx && dy) v = inv[0] + inv[1];
        else if (dx) v = 10 * inv[0] - 2 * inv[1];
        else if (dy) v = 10 * inv[1] - 2 * inv[0];
        else v = -20 * (inv[0] + inv[1]);
        c.L[9 + (dy + 1) * 3 + (dx + 1)] = v / 12.0;
      }
    c.Mc = 8.0 / 12.0;
  } else {
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int o[3] = {dx, dy, dz};
          int nz[3], cnt = 0;
          for (int a = 0; a < 3; ++a)
            if (o[a]) nz[cnt++] = a;
          double v = 0;
          if (cnt == 3) continue;
          if (cnt == 2) v = inv[nz[0]] + inv[nz[1]];
          else if (cnt == 1) {
            const int a = nz[0];
            v = 8 * inv[a];
            for (int b = 0; b < 3; ++b)
              if (b != a) v -= 2 * inv[b];
          } else v = -16 * (inv[0] + inv[1] + inv[2]);
          c.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = v / 12.0;
        }
    c.Mc = 6.0 / 12.0;
  }
  c.Mn = 1.0 / 12.0;
  const double os[4] = {-85.0 / 18.0, 6.0, -1.5, 2.0 / 9.0};
  for (int a = 0; a < g.dim; ++a) {
    for (int m = 0; m < 4; ++m) c.w[a][m] = os[m] * inv[a];
    c.wg[a] = (11.0 / 3.0) / g.h[a];
  }
  c.fsign = -1.0;
  long double c4[5], cs, css;
  fourth_weights(c4, cs, css);
  for (int a = 0; a < g.dim; ++a) {
    const long double h = g.h[a];
    for (int m = 0; m < 5; ++m) c.w4[a][m] = (double)(c4[m] / (h * h * h * h));
    c.w4s[a] = (double)(cs / (h * h * h));
    c.w4ss[a] = (double)(css / (h * h));
  }
  return c;
}

int ilog2i(int64_t n);

// (c, t) with exp(i theta) = c (1 + i t), or = i c (1 + i t) when swap
void dst_factor(long double theta, bool swap, double* out) {
  const long double c = cosl(theta), sn = sinl(theta);
  out[0] = (double)(swap ? sn : c);
  out[1] = (double)(swap ? -c / sn : sn / c);
}

// DST tables for one axis (layout at dst_tw_len); sn[j] = sin(pi j/N)/2 (j <= N/2)
void dst_tables(int N, std::vector<double>& tw, std::vector<double>& sn) {
  tw.assign(2 * (size_t)dst_tw_len(N), 0.0);
  sn.resize((size_t)N / 2 + 1);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int t = 0; t < N; ++t) {
    const long double ang = -2.0L * pi * (long double)t / (long double)N;
    tw[2 * t] = (double)cosl(ang);
    tw[2 * t + 1] = (double)sinl(ang);
  }
  size_t off = (size_t)N;
  for (int j = 0; j <= N / 2; ++j) {
    const long double h = 0.5L * sinl(pi * (long double)j / (long double)N);
    tw[2 * (off + j)] = (double)(h + 0.25L);
    tw[2 * (off + j) + 1] = (double)(h - 0.25L);
  }
  off += (size_t)N / 2 + 1;
  const int M = N / 2;
  const int logM = ilog2i(M > 0 ? M : 1);
  for (int Ns = (logM & 1) ? 2 : 1; Ns < M; Ns <<= 2) {
    if (Ns == 1) continue;
    for (int kk = 0; kk < Ns; ++kk) {
      const long double th = -pi * (long double)kk / (2.0L * Ns);  // W^kk, W = exp(-2 pi i/(4 Ns))
      dst_factor(th, dst_swap_w1(kk, Ns), &tw[2 * (off + kk)]);
      dst_factor(2 * th, dst_swap_w2(kk, Ns), &tw[2 * (off + Ns + kk)]);
    }
    off += 2 * (size_t)Ns;
  }
  for (int k = 0; k <= M / 2; ++k)
    dst_factor(-2.0L * pi * (long double)k / (long double)N, dst_swap_post(k, N), &tw[2 * (off + k)]);
  off += (size_t)M / 2 + 1;
  // radix-8 stages
  for (int Ns = dst_r8_first_ns(logM); Ns < M; Ns <<= 3) {
    for (int kk = 0; kk < Ns; ++kk) {
      const long double th = -pi * (long double)kk / (4.0L * Ns);  // W^kk, W = exp(-2 pi i/(8 Ns))
      dst_factor(th, false, &tw[2 * (off + kk)]);
      dst_factor(2 * th, dst_swap_w1(kk, Ns), &tw[2 * (off + Ns + kk)]);
      dst_factor(4 * th, dst_swap_w2(kk, Ns), &tw[2 * (off + 2 * Ns + kk)]);
      dst_factor(th - pi / 4, kk > 0, &tw[2 * (off + 3 * Ns + kk)]);
    }
    off += 4 * (size_t)Ns;
  }
  for (int j = 0; j <= N / 2; ++j) sn[j] = (double)(0.5L * sinl(pi * (long double)j / (long double)N));
}

// Per-mode factors of the tridiagonal solve along the last axis (tri.cu).
// log10 of the smallest power of r that the one-thread-per-column kernel keeps
// in the boundary-correction terms (K r^j and r^(j-1) w_j in P): below it they
// are under the rounding of the solution (K is at most a few times |w|)
template <typename T> constexpr long double pow_floor() { return -18.0L; }
template <> constexpr long double pow_floor<float>() { return -9.0L; }

// gam: shift of the operator, L_h - gam M (0: L_h itself)
template <typename T>
ahoc_status mode_table(const Geom& g, const Coefs& cf, std::vector<Mode<T>>& out, double gam = 0.0,
                       std::vector<long double>* roots = nullptr) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const int nx = g.N[0] - 1;
  const int ny = (g.dim == 3) ? g.N[1] - 1 : 1;
  const int Nt = (g.dim == 3) ? g.N[2] : g.N[1];
  const int nt = Nt - 1;
  long double scale = 2.0L / g.N[0];
  if (g.dim == 3) scale *= 2.0L / g.N[1];
  auto L = [&](int dx, int dy, int dz) { return (long double)cf.L[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; };
  out.resize((size_t)nx * ny);
  if (roots) roots->assign((size_t)nx * ny, 0.0L);
  for (int ky = 1; ky <= ny; ++ky) {
    const long double cy = (g.dim == 3) ? cosl(pi * ky / g.N[1]) : 0.0L;
    for (int kx = 1; kx <= nx; ++kx) {
      const long double cx = cosl(pi * kx / g.N[0]);
      long double a, b;
      const long double gm = gam, mc = cf.Mc, mn = cf.Mn;
      if (g.dim == 2) {
        a = L(0, 0, 0) + 2 * cx * L(1, 0, 0) - gm * (mc + 2 * cx * mn);
        b = L(0, 1, 0) + 2 * cx * L(1, 1, 0) - gm * mn;
      } else {
        a = L(0, 0, 0) + 2 * cx * L(1, 0, 0) + 2 * cy * L(0, 1, 0) + 4 * cx * cy * L(1, 1, 0) -
            gm * (mc + 2 * (cx + cy) * mn);
        b = L(0, 0, 1) + 2 * cx * L(1, 0, 1) + 2 * cy * L(0, 1, 1) - gm * mn;
      }
      const long double gam = -b / a;
      if (!(fabsl(gam) < 0.5L)) return fail(AHOC_EUNSUPPORTED, "tridiagonal factor not diagonally dominant (mesh aspect ratio)");
      const long double r = 2 * gam / (1 + sqrtl(1 - 4 * gam * gam));
      if (roots) (*roots)[(size_t)(ky - 1) * nx + (kx - 1)] = r;
      const long double sigma = a / (1 + r * r);
      Mode<T> m;
      m.r = (T)r;
      m.s = (T)(scale / sigma);
      const long double r2N = powl(r, 2.0L * Nt);
      m.kap = (T)(-r * (1 - r * r) / (1 - r2N));
      m.kapC = (T)(-r / (1 - r2N));
      m.q1 = (T)(1.0L - r);
      if (r == 0.0L) {
        m.rinv = 0;
        m.rj0 = 0;
        m.j0 = 0;
      } else {
        long double lim = pow_floor<T>() * logl(10.0L) / logl(fabsl(r));
        int j0 = (lim >= nt) ? nt : (int)lim;
        if (j0 < 0) j0 = 0;
        m.rinv = (T)(1.0L / r);
        m.rj0 = (T)powl(r, (long double)j0);
        m.j0 = j0;
      }
      out[(size_t)(ky - 1) * nx + (kx - 1)] = m;
    }
  }
  return AHOC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t W1, W2, ainv, afac, gD, vedge, gN, lapt, twx, snx, twy, sny, twz, snz, modes, b, Q, r, Kry, partial, hdev,
      tmp, pre, stab[3], ctab[3], tri, rxm, rxp, qy, R2, tau, act, scal, ncolsb, modes_v, modesf_v, rpow_v, gL,
      gam, bcg, bcoef, bank, Ud, Vd, cgscnt,
      // mixed precision (AHOC_MIXED only)
      F1, F2, Ru, Rv, U64, V64, twf[3], snf[3], modesf, trif, Rq, dQ, b2, Zb,
      // per-precision side arrays of the fused 2D path
      afinv, qa, rpow, ainvf, rxmf, rxpf, qyf, qaf, R2f, tauf, skf, ckf, tri2, tri2_v,
      // fused 3D matvec: generator and trace arrays (face layout), y-face trace weights
      gen3, tr3, tauy,
      // triharmonic class: Lap u and Lap^2 u on the boundary, u_nn and the tangential
      // part of Lap^2 u on the faces, Lap u gathered on the faces
      lapgD, bilap, gNN, laptw, vface,
      // fused 3D matvec of the mixed path: FP32 generator, y sine table and y trace weights
      gen3f, skyf, tauyf,
      // GMRES's Hessenberg QR on the device: per-problem state, residual estimates, cycle start values
      gs, gi, grel, gini, gii, total;
};

// The chunked tridiagonal form is used when the transverse modes alone give
// too few threads (2D, small 3D grids).
constexpr int64_t kChunkedBelow = 65536;
// FP32 solves always take the chunked form: its carries are FP64, and the
// one-thread-per-column form accumulates the whole column in FP32, which
// loses the near-boundary cancellation u = p + C phi on large grids.
int tri_chunk_len(const Geom& g) {
  if (g.triL) return g.triL;
  return ((g.dim == 3 ? g.N[2] : g.N[1]) >= 1024) ? 32 : 16;
}

// Tuned launch shapes (ahoc_tune_set), per kind, dim, precision and log2 N
// (N of the last axis for the chunk length, of x for the DST CTA); 0 = default.
std::atomic<int> g_tune[AHOC_TUNE_NKINDS][2][2][13];

int ilog2i(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

// a plan's tuned shapes, fixed at its creation
void apply_tuning(Geom& g, const Opts& o) {
  const int pi = o.prec == AHOC_MIXED ? 1 : 0, di = g.dim - 2;
  const int nt = g.dim == 3 ? g.N[2] : g.N[1];
  g.triL = g_tune[AHOC_TUNE_TRI_CHUNK][di][pi][ilog2i(nt)].load();
  g.dst_cta = g_tune[AHOC_TUNE_DST_THREADS][di][pi][ilog2i(g.N[0])].load();
  g.dst_radix = g_tune[AHOC_TUNE_DST_RADIX][di][pi][ilog2i(g.N[0])].load();
}
int64_t tri_ncols(const Geom& g) { return (int64_t)(g.N[0] - 1) * (g.dim == 3 ? (g.N[1] - 1) : 1); }
bool chunked_for(const Geom& g, ahoc_precision prec) {
  return prec == AHOC_MIXED || tri_ncols(g) < kChunkedBelow;
}
// FP64 solves take the chunked form (two passes, tables of tri2_table_fill)
// below kChunkedBelow columns, in either precision of the plan
bool tri2_for(const Geom& g) { return tri_ncols(g) < kChunkedBelow; }

constexpr int kDotBlocks = 296;  // 2 x 148 SMs
// Arnoldi steps per CUDA graph: the host reads the per-problem convergence
// state once per block (the steps of a block run back to back on the device)
constexpr int kArnoldiBlock = 4;

// per-problem sizes of the GMRES scratch: dot partials and the device side
// of the Hessenberg column exchange
int64_t pstride(const Opts& o) { return (int64_t)kDotBlocks * (2 * (o.restart + 1) + 2); }
int hstride(const Opts& o) { return 2 * (o.restart + 1) + 4; }
// counters of the fused CGS passes: one per problem and group of 4 Krylov columns
int cgs_groups(const Opts& o) { return (o.restart + 1 + 3) / 4 + 1; }

bool fused_ok(const Geom& g);

// U-hat slots of the recovery (2D FP64 fused Schur matvec, constant beta/alpha):
// the matvecs of GMRES's first cycle leave U in x-modes in a slot each, so the
// recovery of U is a combination of those fields and one inverse DST.
constexpr int kAutoUhatSlots = 16;
int bank_slots(const Geom& g, const Opts& o) {
  if (o.uhat < 0 || o.prec != AHOC_FP64 || o.varb || o.tri || !fused_ok(g)) return 0;
  const int want = o.uhat > 0 ? o.uhat : kAutoUhatSlots;
  return want < o.restart ? want : o.restart;
}

// Workspace layout.  Per-problem arrays hold g.nb copies back to back at the
// element strides the kernels assume (fields npad, full-grid arrays nfull,
// face arrays ngamma, the 2D generator lines N1 + 1 and 2 N0, the chunked
// tridiagonal scratch (4C + 1) ncols); the Krylov bases are laid out
// [column][problem][face point], so column j of every problem is one batched
// face array.  Tables that depend on the shape alone are held once.
Layout make_layout(const Geom& g, const Opts& o) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t p = off;
    off += align256(bytes);
    return p;
  };
  const size_t B = (size_t)g.nb;
  const size_t fld = (size_t)g.npad * sizeof(double);
  const size_t full = (size_t)g.nfull * sizeof(double);
  const size_t face = (size_t)g.ngamma * sizeof(double);
  const size_t rxn = (size_t)g.N[1] + 1, qyn = 2 * (size_t)g.N[0];
  L.W1 = take(B * fld);
  L.W2 = take(B * fld);
  L.ainv = take(B * full);
  L.afac = take(B * face);
  L.gD = take(B * full);
  L.vedge = take(B * full);
  L.gN = take(B * face);
  L.lapt = take(B * face);
  L.twx = take(2 * (size_t)dst_tw_len(g.N[0]) * sizeof(double));
  L.snx = take(((size_t)g.N[0] / 2 + 1) * sizeof(double));
  L.twy = take(2 * (size_t)dst_tw_len(g.N[1]) * sizeof(double));
  L.sny = take(((size_t)g.N[1] / 2 + 1) * sizeof(double));
  L.twz = take(2 * (size_t)dst_tw_len(g.N[2]) * sizeof(double));
  L.snz = take(((size_t)g.N[2] / 2 + 1) * sizeof(double));
  for (int a = 0; a < 3; ++a) {
    L.stab[a] = take(2 * (size_t)g.N[a] * sizeof(double));
    L.ctab[a] = take(((size_t)g.N[a] + 1) * sizeof(double));
  }
  L.pre = take(face);
  L.tri = take(chunked_for(g, o.prec) ? B * tri_chunked_scratch(g, tri_chunk_len(g)) * sizeof(double) : 0);
  // fused 2D matvec scratch
  L.rxm = take(B * rxn * sizeof(double));
  L.rxp = take(B * rxn * sizeof(double));
  L.qy = take(B * qyn * sizeof(double));
  L.R2 = take(B * qyn * sizeof(double));
  L.tau = take(((size_t)g.N[0] + 1) * sizeof(double));
  L.tauy = take(((size_t)g.N[1] + 1) * sizeof(double));
  L.gen3 = take(g.dim == 3 ? B * face : 0);
  L.tr3 = take(g.dim == 3 ? B * face : 0);
  const size_t nmodes = (size_t)(g.N[0] - 1) * (g.dim == 3 ? (g.N[1] - 1) : 1);
  L.modes = take(nmodes * sizeof(Mode<double>));
  const bool shifted = o.shift != 0.0;  // the V solves take their own (shifted) mode tables
  L.modes_v = take(shifted ? nmodes * sizeof(Mode<double>) : 0);
  L.b = take(B * face);
  L.Q = take(B * face);
  L.r = take(B * face);
  L.tmp = take(B * face);
  L.Kry = take(B * face * (size_t)(o.restart + 1));
  L.Zb = take(B * face * (size_t)o.restart);
  L.afinv = take(B * face);
  L.qa = take(B * face);
  L.rpow = take(chunked_for(g, o.prec) ? tri_powers_size(g, tri_chunk_len(g)) * sizeof(double) : 0);
  L.rpow_v = take(shifted && chunked_for(g, o.prec) ? tri_powers_size(g, tri_chunk_len(g)) * sizeof(double) : 0);
  L.tri2 = take(tri2_for(g) ? tri2_table_size(g, tri_chunk_len(g)) * sizeof(double) : 0);
  L.tri2_v = take(shifted && tri2_for(g) ? tri2_table_size(g, tri_chunk_len(g)) * sizeof(double) : 0);
  // variable beta/alpha: gam = beta/alpha per problem; the BiCGSTAB v-solve's 9 fields (FP64 path)
  L.gam = take(o.varb ? B * full : 0);
  L.bcg = take(o.varb && o.prec == AHOC_FP64 ? 9 * B * fld : 0);
  L.bcoef = take(o.varb ? 3 * B * sizeof(double) : 0);
  L.gL = take(B * face);
  L.lapgD = take(o.tri ? B * full : 0);
  L.bilap = take(o.tri ? B * full : 0);
  L.gNN = take(o.tri ? B * face : 0);
  L.laptw = take(o.tri ? B * face : 0);
  L.vface = take(o.tri ? B * face : 0);
  // the recovery's U-hat slots (one more: the guess's U-hat and the sum) and the data's U and V
  const int nbank = bank_slots(g, o);
  L.bank = take(nbank ? (size_t)(nbank + 1) * B * fld : 0);
  L.Ud = take(nbank ? B * fld : 0);
  L.Vd = take(nbank ? B * fld : 0);
  L.partial = take(B * (size_t)pstride(o) * sizeof(double));
  L.hdev = take(B * (size_t)hstride(o) * sizeof(double));
  L.cgscnt = take(B * (size_t)cgs_groups(o) * sizeof(int));
  L.gs = take(B * (size_t)givens_doubles(o.restart) * sizeof(double));
  L.gi = take(B * (size_t)kGivensInts * sizeof(int));
  L.grel = take(B * sizeof(double));
  L.gini = take(3 * B * sizeof(double));
  L.gii = take(2 * B * sizeof(int));
  L.act = take(B * sizeof(int));
  L.scal = take(B * sizeof(double));
  L.ncolsb = take(B * sizeof(int));
  const bool mixed = (o.prec == AHOC_MIXED);
  const size_t ffl = mixed ? B * (size_t)g.npad * sizeof(float) : 0;
  L.F1 = take(ffl);
  L.F2 = take(ffl);
  L.Ru = take(ffl);
  L.Rv = take(ffl);
  L.U64 = take(mixed ? B * fld : 0);
  L.V64 = take(mixed ? B * fld : 0);
  for (int a = 0; a < 3; ++a) {  // FP32 DST tables: mixed inner solves and the preconditioner
    L.twf[a] = take(2 * (size_t)dst_tw_len(g.N[a]) * sizeof(float));
    L.snf[a] = take(((size_t)g.N[a] / 2 + 1) * sizeof(float));
  }
  L.modesf = take(mixed ? nmodes * sizeof(Mode<float>) : 0);
  L.modesf_v = take(mixed && shifted ? nmodes * sizeof(Mode<float>) : 0);
  L.trif = take(0);  // the chunked solve's carries are FP64 in both precisions (shared scratch L.tri)
  L.Rq = take(mixed ? B * face : 0);
  L.dQ = take(mixed ? B * face : 0);
  L.b2 = take(mixed ? B * face : 0);
  const size_t fface = (size_t)g.ngamma * sizeof(float);
  L.ainvf = take(mixed ? B * (size_t)g.nfull * sizeof(float) : 0);
  L.rxmf = take(mixed ? B * rxn * sizeof(float) : 0);
  L.rxpf = take(mixed ? B * rxn * sizeof(float) : 0);
  L.qyf = take(mixed ? B * qyn * sizeof(float) : 0);
  L.qaf = take(mixed ? B * fface : 0);
  L.R2f = take(mixed ? B * qyn * sizeof(float) : 0);
  L.tauf = take(mixed ? ((size_t)g.N[0] + 1) * sizeof(float) : 0);
  L.skf = take(mixed ? 2 * (size_t)g.N[0] * sizeof(float) : 0);
  L.ckf = take(mixed ? ((size_t)g.N[0] + 1) * sizeof(float) : 0);
  L.gen3f = take(mixed && g.dim == 3 ? B * fface : 0);
  L.skyf = take(mixed ? 2 * (size_t)g.N[1] * sizeof(float) : 0);
  L.tauyf = take(mixed ? ((size_t)g.N[1] + 1) * sizeof(float) : 0);
  L.total = off;
  return L;
}

// Nested initial guess: coarse grids halve every axis.  Automatic depth:
// coarsen while every axis keeps at least kMinCoarse intervals (2D 512, 3D
// 128), at most kAutoLevels times: deeper levels cost more in fixed latency
// than they save.  Measured on B300 (FP64, ms per solve, levels 0/1/2/3):
// 2D 512^2 6.1/7.5/9.6/11.6, 1024^2 9.5/8.9/10.3/12.3, 2048^2
// 22.0/15.1/14.1/15.5, 4096^2 70.6/37.5/32.6/29.6; 3D 128^3 26.0/31.4/38.9,
// 256^3 101/84/89/97, 512^3 698/440/423/429.
constexpr int kMinCoarse2 = 512, kMinCoarse3 = 128;
constexpr int kAutoLevels = 3;
int coarse_levels(const Geom& g, int requested) {
  int maxl = 0;
  int n = 1 << 30;
  for (int a = 0; a < g.dim; ++a) n = (g.N[a] < n) ? g.N[a] : n;
  const int kMinCoarse = g.dim == 2 ? kMinCoarse2 : kMinCoarse3;
  while ((n >> (maxl + 1)) >= kMinCoarse && (n >> (maxl + 1)) >= 8) ++maxl;
  if (requested < 0) return maxl < kAutoLevels ? maxl : kAutoLevels;
  // an explicit request may go down to 8 intervals per axis
  int lim = 0;
  while ((n >> (lim + 1)) >= 8) ++lim;
  return requested < lim ? requested : lim;
}

// total workspace of a plan and its coarse levels
size_t total_bytes(const Geom& g, const Opts& o) {
  size_t b = make_layout(g, o).total;
  const int lv = coarse_levels(g, o.levels);
  if (lv > 0) {
    int64_t Nc[3];
    for (int a = 0; a < g.dim; ++a) Nc[a] = g.N[a] / 2;
    Geom gc;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    make_geom(g.dim, Nc, lo, hi, &gc);
    gc.nb = g.nb;
    Opts oc = o;
    oc.levels = lv - 1;
    oc.uhat = -1;  // coarse levels only solve for Q
    apply_tuning(gc, oc);
    b += total_bytes(gc, oc);
  }
  return b;
}

}  // namespace

// Per-problem outcome of a solve.
struct ProbStat {
  int iters = 0, restarts = 0, coarse_iters = 0, refine_steps = 0, levels = 0;
  double rel = 0.0, ms_mv = 0.0;
  ahoc_status status = AHOC_OK;
  double hist[16] = {0}, du[16] = {0};
  int inner[16] = {0};
};

struct ahoc_plan {
  Geom g;
  Coefs cf;
  Opts o;
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  bool own_ws = false;
  Layout L;
  double *W1, *W2, *ainv, *afac, *gD = nullptr, *vedge = nullptr, *gN = nullptr, *lapt = nullptr;
  double *twx, *snx, *twy, *sny, *twz, *snz, *b, *Q, *r, *tmp, *Kry, *partial, *hdev, *pre, *tri;
  double *stab[3], *ctab[3];
  double *rxm, *rxp, *qy, *R2, *tau;
  double *tauy = nullptr, *gen3 = nullptr, *tr3 = nullptr;  // fused 3D matvec
  Mode<double>* modes;
  // the V solves' tables: the shifted operator L_h - gam M (aliases of the
  // U tables when gam = 0)
  Mode<double>* modes_v = nullptr;
  Mode<float>* modesf_v = nullptr;
  double* rpow_v = nullptr;
  double* gL = nullptr;
  bool has_gL = false;
  // variable beta/alpha: gam = beta/alpha per problem (full grid) and the
  // BiCGSTAB fields (rhs, x is W1, r, r-hat, p, v, s, t, p-hat, s-hat)
  double* gam = nullptr;
  double* bcg = nullptr;
  double* bcoef = nullptr;
  int bicg_iters = 0;  // BiCGSTAB iterations of the last solve (summed over v-solves)
  // recovery from the U-hat slots: bank holds nbank + 1 batched fields (slot
  // j: U-hat of z_j; slot nbank: U-hat of the initial guess, then the sum);
  // Ud, Vd: U and V of the data alone (Q = 0).  bank_valid: the last GMRES
  // ended in its first cycle within nbank steps.  v_lazy: V was not
  // recovered by the last solve (ahoc_last_qv forms it on request).
  double *bank = nullptr, *Ud = nullptr, *Vd = nullptr;
  int nbank = 0;
  bool bank_valid = false, v_lazy = false;
  bool rhs_ready = false;  // a coarse level's b was computed by the finer level's resolution check
  const double* q0 = nullptr;  // the caller's initial Q for the current ahoc_solve_from call
  // mixed precision
  float *F1 = nullptr, *F2 = nullptr, *Ru = nullptr, *Rv = nullptr, *twf[3] = {nullptr, nullptr, nullptr},
        *snf[3] = {nullptr, nullptr, nullptr}, *trif = nullptr;
  double *U64 = nullptr, *V64 = nullptr, *Rq = nullptr, *dQ = nullptr, *b2 = nullptr;
  double* Zb = nullptr;  // flexible GMRES: the preconditioned directions z_j = P^-1 v_j
  double *afinv = nullptr, *qa = nullptr, *rpow = nullptr;
  double *tri2 = nullptr, *tri2_v = nullptr;  // tables of the FP64 chunked solve (U and shifted V operators)
  float *ainvf = nullptr, *rxmf = nullptr, *rxpf = nullptr, *qyf = nullptr, *qaf = nullptr, *R2f = nullptr,
        *tauf = nullptr, *skf = nullptr, *ckf = nullptr, *gen3f = nullptr, *skyf = nullptr, *tauyf = nullptr;
  Mode<float>* modesf = nullptr;
  // batch state: the device mask g.act points to `act`; act_now mirrors it
  int* act = nullptr;
  double* scal = nullptr;  // per-problem scalars of the batched axpy
  int* ncolsb = nullptr;   // per-problem column counts of the batched update
  int* cgscnt = nullptr;   // zeroed counters of the fused CGS passes (launch_cgs)
  // device Hessenberg QR (blas.cu, k_givens_*): state, residual estimates,
  // cycle start values; pinned host copies of the start values and of the
  // state read back after each block of Arnoldi steps
  double *gs = nullptr, *grel = nullptr, *gini = nullptr;
  int *gi = nullptr, *gii = nullptr;
  double *gini_h = nullptr, *rb_rel = nullptr;
  int *gii_h = nullptr, *rb_act = nullptr, *rb_gi = nullptr;
  std::vector<int> act_now, part;  // current mask; problems taking part in solves
  std::vector<ProbStat> ps;
  bool has_gD = false, has_vedge = false, has_gN = false, has_lapt = false;
  // triharmonic class data (Lap u, Lap^2 u on the boundary; u_nn, tangential part of Lap^2 u; Lap u on the faces)
  double *lapgD = nullptr, *bilap = nullptr, *gNN = nullptr, *laptw = nullptr, *vface = nullptr;
  bool has_lapgD = false, has_bilap = false, has_gNN = false, has_laptw = false;
  double* hhost = nullptr;  // pinned
  // CUDA graphs of the GMRES iterations, one per iteration index, captured on
  // first use; the per-problem scalars and the mask reach them through
  // pinned host arrays copied inside the graph
  struct GCount {
    int64_t launches = 0;
    int64_t kn[AHOC_NK] = {0};
  };
  bool use_graphs = false;
  std::vector<cudaGraphExec_t> gexec;
  std::vector<GCount> gcount;
  double* scal_h = nullptr;  // pinned
  int* act_h = nullptr;      // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // the graphs are captured and replayed on a stream of the plan's own, so
  // that no other work can land on a stream while it is capturing; two
  // events order it with the caller's stream
  cudaStream_t gst = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  bool have_last = false;
  // launch accounting (and, with opts.timing, per-launch CUDA events)
  struct EvPair {
    cudaEvent_t a, b;
    int kid;
  };
  std::vector<EvPair> pool, pending;
  int64_t launches = 0;
  double kms[AHOC_NK] = {0};
  int64_t kn[AHOC_NK] = {0};
  ahoc_plan* coarse = nullptr;  // next coarser level of the nested initial guess
  int levels = 0;
  // device staging grids of ahoc_solve_host (f in, u out), allocated on its first call
  double *hf = nullptr, *hu = nullptr;
  double kms_top[AHOC_NK] = {0};  // this level only (no coarse levels)
  int64_t kn_top[AHOC_NK] = {0};
};

namespace {

template <typename P>
P* at(ahoc_plan* p, size_t off) {
  return reinterpret_cast<P*>(p->ws + off);
}

// Launch one kernel through `f`, counting it and, when timing is on,
// bracketing it with CUDA events on the plan's stream.
template <class F>
ahoc_status run(ahoc_plan* p, int kid, const char* what, F&& f, int nkernels = 1) {
  ahoc_plan::EvPair ev{nullptr, nullptr, kid};
  if (p->o.timing) {
    if (!p->pool.empty()) {
      ev = p->pool.back();
      p->pool.pop_back();
      ev.kid = kid;
    } else {
      CK(cudaEventCreate(&ev.a));
      CK(cudaEventCreate(&ev.b));
    }
    CK(cudaEventRecord(ev.a, p->st));
  }
  cudaError_t e = f();
  if (e != cudaSuccess) return fail(AHOC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  if (p->o.timing) {
    CK(cudaEventRecord(ev.b, p->st));
    p->pending.push_back(ev);
  }
  p->launches += nkernels;
  p->kn[kid] += nkernels;
  return AHOC_OK;
}

// Collect the event timings of completed launches (call after a stream sync).
ahoc_status harvest(ahoc_plan* p) {
  for (auto& ev : p->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev.a, ev.b));
    p->kms[ev.kid] += ms;
    p->pool.push_back(ev);
  }
  p->pending.clear();
  return AHOC_OK;
}

#define RUN(kid, call) CKS(run(p, kid, #call, [&]() { return (call); }))
// a launcher that issues n kernels
#define RUNN(kid, n, call) CKS(run(p, kid, #call, [&]() { return (call); }, n))

// vsolve: the operator of the v-equation, L_h - gam M (the shifted tables)
ahoc_status poisson_inplace(ahoc_plan* p, double* W, bool vsolve = false) {
  const Geom& g = p->g;
  const Mode<double>* md = vsolve ? p->modes_v : p->modes;
  RUN(AHOC_K_DST_X, launch_dst_x<double>(g, W, p->twx, p->snx, 1.0, p->st));
  if (g.dim == 3) RUN(AHOC_K_DST_Y, launch_dst_y<double>(g, W, p->twy, p->sny, 1.0, p->st));
  if (tri2_for(g))
    RUNN(AHOC_K_TRI, 4, launch_tri2(g, W, md, vsolve ? p->tri2_v : p->tri2, p->tri, tri_chunk_len(g), p->st));
  else
    RUN(AHOC_K_TRI, launch_tri<double>(g, W, md, p->st));
  if (g.dim == 3) RUN(AHOC_K_DST_Y, launch_dst_y<double>(g, W, p->twy, p->sny, 1.0, p->st));
  RUN(AHOC_K_DST_X, launch_dst_x<double>(g, W, p->twx, p->snx, 1.0, p->st));
  return AHOC_OK;
}

// V-solve then U-solve (Algorithm 1, two FFT-based solves); leaves V in W1, U in W2.
ahoc_status bicgstab_v(ahoc_plan* p);

ahoc_status solve_VU(ahoc_plan* p, const double* Q, const double* f, bool data) {
  const Geom& g = p->g;
  RUN(AHOC_K_VRHS, launch_vrhs<double>(g, p->cf, p->W1, Q, f, data && p->has_vedge ? p->vedge : nullptr, p->st,
                                       nullptr, p->gam));
  if (p->o.varb)
    CKS(bicgstab_v(p));  // variable beta/alpha: (L_h - M(gam .)) V = rhs iteratively
  else
    CKS(poisson_inplace(p, p->W1, true));
  RUN(AHOC_K_URHS,
      launch_urhs<double>(g, p->cf, p->W2, p->W1, p->ainv, Q, data && p->has_gD ? p->gD : nullptr, p->st));
  CKS(poisson_inplace(p, p->W2));
  return AHOC_OK;
}

// Triharmonic class (Sec. 4.2, triharmonic equation): the three sequential
// Dirichlet solves of the mixed form Lap w = f, Lap v = w, Lap u = v with the
// w boundary values Q on the faces.  Leaves U in W1 and V in W2.  data: with f
// and the boundary data (edges and corners of w, v on the boundary, g_D);
// otherwise the homogeneous part (Q alone).
ahoc_status solve_tri(ahoc_plan* p, const double* Q, const double* f, bool data) {
  const Geom& g = p->g;
  // L_h W = M f - L_bdry(W_b): W_b = Q on the faces, Lap^2 u on edges and corners
  RUN(AHOC_K_VRHS, launch_vrhs<double>(g, p->cf, p->W1, Q, f, data && p->has_bilap ? p->bilap : nullptr, p->st,
                                       nullptr, nullptr));
  CKS(poisson_inplace(p, p->W1));
  // L_h V = M W - L_bdry(V_b): M reaches W = Q on the faces, V_b = Lap u (data)
  RUN(AHOC_K_URHS, launch_urhs<double>(g, p->cf, p->W2, p->W1, p->ainv, Q,
                                       data && p->has_lapgD ? p->lapgD : nullptr, p->st));
  CKS(poisson_inplace(p, p->W2));
  // L_h U = M V - L_bdry(g_D): M reaches V = Lap u on the faces
  RUN(AHOC_K_URHS, launch_urhs<double>(g, p->cf, p->W1, p->W2, p->ainv, data && p->has_lapgD ? p->vface : nullptr,
                                       data && p->has_gD ? p->gD : nullptr, p->st));
  CKS(poisson_inplace(p, p->W1));
  return AHOC_OK;
}

// FP32 Dirichlet Poisson solve in place (mixed precision inner solves)
ahoc_status poisson_inplace_f(ahoc_plan* p, float* W, bool vsolve = false) {
  const Geom& g = p->g;
  const Mode<float>* mf = vsolve ? p->modesf_v : p->modesf;
  const Mode<double>* md = vsolve ? p->modes_v : p->modes;
  const double* rp = vsolve ? p->rpow_v : p->rpow;
  RUN(AHOC_K_DST_X, launch_dst_x<float>(g, W, p->twf[0], p->snf[0], 1.0f, p->st));
  if (g.dim == 3) RUN(AHOC_K_DST_Y, launch_dst_y<float>(g, W, p->twf[1], p->snf[1], 1.0f, p->st));
  RUNN(AHOC_K_TRI, 5, launch_tri_chunked<float>(g, W, mf, md, rp, p->tri, tri_chunk_len(g), p->st));
  if (g.dim == 3) RUN(AHOC_K_DST_Y, launch_dst_y<float>(g, W, p->twf[1], p->snf[1], 1.0f, p->st));
  RUN(AHOC_K_DST_X, launch_dst_x<float>(g, W, p->twf[0], p->snf[0], 1.0f, p->st));
  return AHOC_OK;
}

// FP32 correction solves of the coupled system with residual sources:
// L_h dV = -r_v - L_bdry(dQ)  ->  F1;   L_h dU = r_u + M(dV/alpha)  ->  F2
ahoc_status solve_VU_f(ahoc_plan* p, const double* Q, const float* srcv, const float* srcu) {
  const Geom& g = p->g;
  RUN(AHOC_K_VRHS, launch_vrhs<float>(g, p->cf, p->F1, Q, nullptr, nullptr, p->st, srcv));
  CKS(poisson_inplace_f(p, p->F1, true));
  RUN(AHOC_K_URHS, launch_urhs<float>(g, p->cf, p->F2, p->F1, p->ainvf, Q, nullptr, p->st, srcu));
  CKS(poisson_inplace_f(p, p->F2));
  return AHOC_OK;
}

// The fused 2D solves (DST-I along x, exact tridiagonal solve along y) in
// precision T, with the v-equation right-hand side generated in x-modes from
// q and the traces taken from U-hat without a full inverse transform:
//   q      face values: the v-equation boundary data and M's face terms (may be NULL)
//   srcv   r_v field (FP32 correction solves; NULL in the Schur action)
//   srcu   r_u field added to the u-equation right-hand side (may be NULL)
//   srcq   r_q face array subtracted from the trace (may be NULL)
//   recover == false: y = alpha delta_nn U - q - srcq (SchurMatVec, Algorithm 1)
//   recover == true:  W1 <- V, W2 <- U, both physical (the recovery step)
template <typename T>
struct F2Arrays {
  T *W1, *W2;
  const Mode<T>* modes;
  const Mode<T>* modes_v;  // the V solve's (shifted) tables
  const void* tw;
  const T *sn, *ainv, *tau, *sk, *ck;
  T *rxm, *rxp, *qy, *qa, *R2;
};
F2Arrays<double> f2arrays_d(ahoc_plan* p) {
  return F2Arrays<double>{p->W1, p->W2, p->modes, p->modes_v, p->twx, p->snx, p->ainv, p->tau, p->stab[0], p->ctab[0],
                          p->rxm, p->rxp, p->qy, p->qa, p->R2};
}
F2Arrays<float> f2arrays_f(ahoc_plan* p) {
  return F2Arrays<float>{p->F1, p->F2, p->modesf, p->modesf_v, p->twf[0], p->snf[0], p->ainvf, p->tauf, p->skf, p->ckf,
                         p->rxmf, p->rxpf, p->qyf, p->qaf, p->R2f};
}

// The chunked tridiagonal solve of a fused 2D pass in precision T: FP64 in two
// passes with the plan's tables (4 kernels), FP32 in three with FP64 carries
// (5 kernels); vsolve selects the (shifted) V operator, G a generated
// right-hand side (added to the field when `add`).
cudaError_t tri_fused(ahoc_plan* p, double* W, const Mode<double>* mT, bool vsolve, const VGen2D<double>* G,
                      bool add, int L) {
  return launch_tri2(p->g, W, mT, vsolve ? p->tri2_v : p->tri2, p->tri, L, p->st, G, add);
}
cudaError_t tri_fused(ahoc_plan* p, float* W, const Mode<float>* mT, bool vsolve, const VGen2D<float>* G, bool add,
                      int L) {
  const Mode<double>* md = vsolve ? p->modes_v : p->modes;
  const double* rp = vsolve ? p->rpow_v : p->rpow;
  if (G) return launch_tri_chunked_gen<float>(p->g, W, mT, md, rp, p->tri, L, *G, p->st, add);
  return launch_tri_chunked<float>(p->g, W, mT, md, rp, p->tri, L, p->st);
}
template <typename T> constexpr int tri_kernels() { return sizeof(T) == 8 ? 4 : 5; }

template <typename T>
ahoc_status fused2d(ahoc_plan* p, const F2Arrays<T>& A, const double* q, const T* srcv, const T* srcu,
                    const double* srcq, double* y, bool recover) {
  const Geom& g = p->g;
  const Coefs& cf = p->cf;
  const int N0 = g.N[0];
  const int L = tri_chunk_len(g);
  // y-face terms of (L - gam M)_bdry: the shift reaches the face point of the same column
  VGen2D<T> G{A.rxm, A.rxp, A.qy, A.qy + (N0 - 1), A.sk, A.ck, (T)(cf.L[16] - cf.gam * cf.Mn), (T)cf.L[17]};
  if (q) {
    RUN(AHOC_K_VRHS, launch_v2d_prep<T>(g, cf, q, p->afinv, A.rxm, A.rxp, A.qy, A.qa, p->st));
    RUN(AHOC_K_VRHS, launch_dst_gen<T>(A.qy, 2, 1, N0 - 1, 0, 1, N0, A.tw, A.sn, p->st, g.nb, 2 * N0, g.act));
  }
  const T* qa = q ? A.qa : nullptr;
  // V-hat: L_h V = -r_v - L_bdry(q) in x-modes
  if (srcv) {
    RUN(AHOC_K_DST_X, launch_dst_x_from<T>(g, A.W1, srcv, -1.0, A.tw, A.sn, p->st));
    RUNN(AHOC_K_TRI, tri_kernels<T>(), tri_fused(p, A.W1, A.modes_v, true, q ? &G : nullptr, true, L));
  } else {
    RUNN(AHOC_K_TRI, tri_kernels<T>(), tri_fused(p, A.W1, A.modes_v, true, &G, false, L));
  }
  // U-hat: L_h U = M(V/alpha) + face terms + r_u, by one forward DST of the fused right-hand side
  if (!recover) {
    RUN(AHOC_K_DST_X, launch_dst_x_store_ainv<T>(g, A.W1, A.ainv, A.tw, A.sn, p->st));
    RUN(AHOC_K_DST_X, launch_dst_x_mload<T>(g, A.W2, A.W1, qa, (T)cf.Mc, (T)cf.Mn, A.tw, A.sn, p->st, srcu, nullptr));
  } else {
    RUN(AHOC_K_DST_X, launch_dst_x<T>(g, A.W1, A.tw, A.sn, (T)1, p->st));
    RUN(AHOC_K_DST_X, launch_dst_x_mload<T>(g, A.W2, A.W1, qa, (T)cf.Mc, (T)cf.Mn, A.tw, A.sn, p->st, srcu, A.ainv));
  }
  RUNN(AHOC_K_TRI, tri_kernels<T>(), tri_fused(p, A.W2, A.modes, false, nullptr, false, L));
  if (recover) {
    RUN(AHOC_K_DST_X, launch_dst_x<T>(g, A.W2, A.tw, A.sn, (T)1, p->st));
    return AHOC_OK;
  }
  RUN(AHOC_K_TRACE, launch_trace2d_x<T>(g, y, A.W2, q, p->afac, A.tau, p->st, srcq));
  RUN(AHOC_K_TRACE, launch_trace2d_ylines<T>(g, cf, A.R2, A.W2, p->st));
  RUN(AHOC_K_TRACE, launch_dst_gen<T>(A.R2, 2, 1, N0 - 1, 0, 1, N0, A.tw, A.sn, p->st, g.nb, 2 * N0, g.act));
  RUN(AHOC_K_TRACE, launch_trace2d_y<T>(g, y, A.R2, q, p->afac, p->st, srcq));
  return AHOC_OK;
}

bool fused_ok(const Geom& g) { return g.dim == 2 && tri_ncols(g) < kChunkedBelow; }

// The fused 3D form (FP64, constant beta/alpha; both z-solves one thread per
// mode column, whatever the number of columns): fused3d.cu's header gives
// the algebra.
bool fused3d_ok(const ahoc_plan* p) {
  const Geom& g = p->g;
  return g.dim == 3 && !p->o.varb && !p->o.tri && !p->o.unfused && trace3d_red_ok(g);
}

// DST-I of face-layout arrays along the in-face axes other than z for the x-
// and y-faces, along both for the z-faces (the generator and the traces)
template <typename T>
ahoc_status face_dsts3(ahoc_plan* p, T* v, const void* twx, const T* snx, const void* twy, const T* sny, int kid) {
  const Geom& g = p->g;
  const int nx = g.N[0] - 1, ny = g.N[1] - 1, nz = g.N[2] - 1;
  RUN(kid, launch_dst_gen<T>(v + g.face_off[0], 2 * nz, 1, ny, 0, 1, g.N[1], twy, sny, p->st, g.nb, g.ngamma,
                             g.act));
  RUN(kid, launch_dst_gen<T>(v + g.face_off[2], 2 * nz, 1, nx, 0, 1, g.N[0], twx, snx, p->st, g.nb, g.ngamma,
                             g.act));
  RUN(kid, launch_dst_gen<T>(v + g.face_off[4], 2 * ny, 1, nx, 0, 1, g.N[0], twx, snx, p->st, g.nb, g.ngamma,
                             g.act));
  RUN(kid, launch_dst_gen<T>(v + g.face_off[4], 2 * nx, nx, (int64_t)nx * ny, 1, nx, g.N[1], twy, sny, p->st,
                             g.nb, g.ngamma, g.act));
  return AHOC_OK;
}
ahoc_status face_dsts3(ahoc_plan* p, double* v, int kid) {
  return face_dsts3<double>(p, v, p->twx, p->snx, p->twy, p->sny, kid);
}

// y = S q (Algorithm 1, SchurMatVec) in 4 full DST passes: the V solve's
// right-hand side generated in (x, y)-modes inside the z-solve, V back to
// physical space with V/alpha stored, M(V/alpha) fused into the U solve's
// first DST, and the traces from U-hat without transforming U back
ahoc_status fused3d(ahoc_plan* p, const double* q, double* y) {
  const Geom& g = p->g;
  const Coefs& cf = p->cf;
  RUN(AHOC_K_VRHS, launch_v3d_prep<double>(g, cf, q, p->afinv, p->gen3, p->qa, p->st));
  CKS(face_dsts3(p, p->gen3, AHOC_K_VRHS));
  const VGen3D<double> G{p->gen3, p->stab[0], p->stab[1]};
  RUN(AHOC_K_TRI, launch_tri_gen3<double>(g, p->W1, p->modes_v, G, p->st));
  RUN(AHOC_K_DST_Y, launch_dst_y<double>(g, p->W1, p->twy, p->sny, 1.0, p->st));
  RUN(AHOC_K_DST_X, launch_dst_x_store_ainv<double>(g, p->W1, p->ainv, p->twx, p->snx, p->st));
  RUN(AHOC_K_DST_X, launch_dst_x_mload3d<double>(g, p->W2, p->W1, p->qa, cf.Mc, cf.Mn, p->twx, p->snx, p->st));
  RUN(AHOC_K_DST_Y, launch_dst_y<double>(g, p->W2, p->twy, p->sny, 1.0, p->st));
  RUN(AHOC_K_TRI, launch_tri<double>(g, p->W2, p->modes, p->st));
  RUNN(AHOC_K_TRACE, 3, launch_trace3d<double>(g, cf, p->W2, p->tau, p->tauy, p->tr3, p->st));
  CKS(face_dsts3(p, p->tr3, AHOC_K_TRACE));
  RUN(AHOC_K_TRACE, launch_trace3d_fin(g, y, p->tr3, q, p->afac, nullptr, p->st));
  return AHOC_OK;
}

// The same in FP32 (the mixed path's Schur action): the z-solves take the
// chunked form with FP64 carries; the generator arrays, the fields and the
// stencil in FP32, the traces summed in FP32 and finished in FP64.
ahoc_status fused3d_f(ahoc_plan* p, const double* q, double* y) {
  const Geom& g = p->g;
  const Coefs& cf = p->cf;
  const int L = tri_chunk_len(g);
  RUN(AHOC_K_VRHS, launch_v3d_prep<float>(g, cf, q, p->afinv, p->gen3f, p->qaf, p->st));
  CKS(face_dsts3<float>(p, p->gen3f, p->twf[0], p->snf[0], p->twf[1], p->snf[1], AHOC_K_VRHS));
  const VGen3D<float> G{p->gen3f, p->skf, p->skyf};
  RUNN(AHOC_K_TRI, 5, launch_tri_chunked_gen3<float>(g, p->F1, p->modesf_v, p->modes_v, p->rpow_v, p->tri, L, G,
                                                      p->st));
  RUN(AHOC_K_DST_Y, launch_dst_y<float>(g, p->F1, p->twf[1], p->snf[1], 1.0f, p->st));
  RUN(AHOC_K_DST_X, launch_dst_x_store_ainv<float>(g, p->F1, p->ainvf, p->twf[0], p->snf[0], p->st));
  RUN(AHOC_K_DST_X, launch_dst_x_mload3d<float>(g, p->F2, p->F1, p->qaf, (float)cf.Mc, (float)cf.Mn, p->twf[0],
                                                p->snf[0], p->st));
  RUN(AHOC_K_DST_Y, launch_dst_y<float>(g, p->F2, p->twf[1], p->snf[1], 1.0f, p->st));
  RUNN(AHOC_K_TRI, 5, launch_tri_chunked<float>(g, p->F2, p->modesf, p->modes, p->rpow, p->tri, L, p->st));
  RUNN(AHOC_K_TRACE, 3, launch_trace3d<float>(g, cf, p->F2, p->tauf, p->tauyf, p->tr3, p->st));
  CKS(face_dsts3(p, p->tr3, AHOC_K_TRACE));
  RUN(AHOC_K_TRACE, launch_trace3d_fin(g, y, p->tr3, q, p->afac, nullptr, p->st));
  return AHOC_OK;
}

// uhat: where the FP64 fused 2D matvec leaves U in x-modes (NULL: W2)
ahoc_status matvec_dev(ahoc_plan* p, const double* q, double* y, double* uhat = nullptr) {
  if (p->o.tri) {
    CKS(solve_tri(p, q, nullptr, false));
    RUN(AHOC_K_TRACE, launch_trace_tri(p->g, p->cf, y, p->W1, q, nullptr, nullptr, nullptr, nullptr, nullptr, p->st));
    return AHOC_OK;
  }
  if (p->o.prec == AHOC_MIXED) {
    if (fused_ok(p->g)) return fused2d<float>(p, f2arrays_f(p), q, nullptr, nullptr, nullptr, y, false);
    if (fused3d_ok(p)) return fused3d_f(p, q, y);
    CKS(solve_VU_f(p, q, nullptr, nullptr));
    RUN(AHOC_K_TRACE, launch_trace<float>(p->g, p->cf, y, p->F2, q, p->afac, nullptr, nullptr, nullptr, p->st));
    return AHOC_OK;
  }
  if (fused_ok(p->g) && !p->o.varb) {
    F2Arrays<double> A = f2arrays_d(p);
    if (uhat) A.W2 = uhat;
    return fused2d<double>(p, A, q, nullptr, nullptr, nullptr, y, false);
  }
  if (fused3d_ok(p)) return fused3d(p, q, y);
  CKS(solve_VU(p, q, nullptr, false));
  RUN(AHOC_K_TRACE, launch_trace<double>(p->g, p->cf, y, p->W2, q, p->afac, nullptr, nullptr, nullptr, p->st));
  return AHOC_OK;
}

// Transverse DST-I of every face with normal `a`, along each in-face axis.
ahoc_status face_dsts(ahoc_plan* p, double* v, int a) {
  const Geom& g = p->g;
  double* base = v + g.face_off[2 * a];
  const int64_t fs = g.face_off[2 * a + 1] - g.face_off[2 * a];
  int rem[2], nr = 0;
  for (int b = 0; b < g.dim; ++b)
    if (b != a) rem[nr++] = b;
  const double* tw[3] = {p->twx, p->twy, p->twz};
  const double* sn[3] = {p->snx, p->sny, p->snz};
  if (nr == 1) {
    const int b = rem[0];
    RUN(AHOC_K_KRYLOV,
        launch_dst_gen<double>(base, 2, 1, fs, 0, 1, g.N[b], tw[b], sn[b], p->st, g.nb, g.ngamma, g.act));
  } else {
    const int b0 = rem[0], b1 = rem[1];
    const int n0 = g.N[b0] - 1, n1 = g.N[b1] - 1;
    RUN(AHOC_K_KRYLOV, launch_dst_gen<double>(base, 2 * n1, n1, fs, n0, 1, g.N[b0], tw[b0], sn[b0], p->st, g.nb,
                                              g.ngamma, g.act));
    RUN(AHOC_K_KRYLOV, launch_dst_gen<double>(base, 2 * n0, n0, fs, 1, n0, g.N[b1], tw[b1], sn[b1], p->st, g.nb,
                                              g.ngamma, g.act));
  }
  return AHOC_OK;
}

// out = P^-1 in: the boundary-symbol preconditioner (precond.cu); in, out may alias.
ahoc_status precond_apply(ahoc_plan* p, const double* in, double* out) {
  const Geom& g = p->g;
  const int64_t n = g.ngamma;
  if (!p->o.precond) {
    if (in != out) RUN(AHOC_K_KRYLOV, launch_axpby(out, in, 1.0, 0.0, n, p->st, g.nb, nullptr, g.act));
    return AHOC_OK;
  }
  if (g.dim == 2) {
    // x-faces are lines of N1 - 1 points (DST length N1), y-faces of N0 - 1
    const int64_t ox = g.face_off[0], oy = g.face_off[2];
    if (g.N[0] == g.N[1]) {  // the four faces are four consecutive lines of equal length
      RUN(AHOC_K_KRYLOV, launch_precond_lines<float>(out, in, p->afac, p->pre, 4, g.N[0] - 1, g.N[0], p->twf[0],
                                                     p->snf[0], p->st, g.nb, n, g.act));
      return AHOC_OK;
    }
    RUN(AHOC_K_KRYLOV, launch_precond_lines<float>(out + ox, in + ox, p->afac + ox, p->pre + ox, 2, g.N[1] - 1,
                                                   g.N[1], p->twf[1], p->snf[1], p->st, g.nb, n, g.act));
    RUN(AHOC_K_KRYLOV, launch_precond_lines<float>(out + oy, in + oy, p->afac + oy, p->pre + oy, 2, g.N[0] - 1,
                                                   g.N[0], p->twf[0], p->snf[0], p->st, g.nb, n, g.act));
    return AHOC_OK;
  }
  RUN(AHOC_K_KRYLOV, launch_face_muldiv(out, in, nullptr, p->afac, n, p->st, g.nb, 0, n, g.act));
  for (int a = 0; a < g.dim; ++a) CKS(face_dsts(p, out, a));
  RUN(AHOC_K_KRYLOV, launch_face_muldiv(out, out, p->pre, nullptr, n, p->st, g.nb, 0, 0, g.act));
  for (int a = 0; a < g.dim; ++a) CKS(face_dsts(p, out, a));
  RUN(AHOC_K_KRYLOV, launch_face_muldiv(out, out, p->afac, nullptr, n, p->st, g.nb, n, 0, g.act));
  return AHOC_OK;
}

ahoc_status schur_rhs_dev(ahoc_plan* p, const double* f, double* b) {
  Phase ph("ahoc schur rhs");
  const Geom& g = p->g;
  if (p->o.tri) {
    CKS(solve_tri(p, nullptr, f, true));
    RUN(AHOC_K_TRACE, launch_trace_tri(g, p->cf, b, p->W1, nullptr, p->has_gD ? p->gD : nullptr,
                                       p->has_gN ? p->gN : nullptr, p->has_gNN ? p->gNN : nullptr,
                                       p->has_laptw ? p->laptw : nullptr, p->has_bilap ? p->bilap : nullptr, p->st));
    RUN(AHOC_K_KRYLOV, launch_axpby(b, b, -1.0, 0.0, g.ngamma, p->st, g.nb, nullptr, g.act));
    return AHOC_OK;
  }
  CKS(solve_VU(p, nullptr, f, true));
  RUN(AHOC_K_TRACE, launch_trace<double>(g, p->cf, b, p->W2, nullptr, p->afac, p->has_gD ? p->gD : nullptr,
                                         p->has_gN ? p->gN : nullptr, p->has_lapt ? p->lapt : nullptr, p->st,
                                         nullptr, p->has_gL ? p->gL : nullptr));
  RUN(AHOC_K_KRYLOV, launch_axpby(b, b, -1.0, 0.0, g.ngamma, p->st, g.nb, nullptr, g.act));
  return AHOC_OK;
}

// dots of every active problem: out[b * hstride + c] = <V_c, w> (problem b's
// V_c at V + b * ngamma + c * ld, its w at w + b * ngamma), c < ncols
ahoc_status mdot(ahoc_plan* p, const double* V, int64_t ld, int ncols, const double* w, double* out) {
  const Geom& g = p->g;
  BatchDot bd;
  bd.vstride = g.ngamma;
  bd.wstride = g.ngamma;
  bd.pstride = pstride(p->o);
  bd.act = g.act;
  RUNN(AHOC_K_KRYLOV, 2,
       launch_mdot(V, ld, ncols, w, g.ngamma, p->partial, kDotBlocks, out, p->st, g.nb, bd, hstride(p->o)));
  return AHOC_OK;
}

// w -= V h per active problem (h at hdev + b * hstride; ncols_b: per-problem counts or NULL)
ahoc_status gemv_sub(ahoc_plan* p, const double* V, int64_t ld, int ncols, const double* h, double* w,
                     const int* ncols_b) {
  const Geom& g = p->g;
  BatchDot bd;
  bd.vstride = g.ngamma;
  bd.wstride = g.ngamma;
  bd.act = g.act;
  RUN(AHOC_K_KRYLOV, launch_gemv_sub(V, ld, ncols, h, w, g.ngamma, p->st, g.nb, bd, hstride(p->o), ncols_b));
  return AHOC_OK;
}

// the Hessenberg exchange area of every problem, device to host (synchronises)
ahoc_status fetch(ahoc_plan* p) {
  CK(cudaMemcpyAsync(p->hhost, p->hdev, (size_t)p->g.nb * hstride(p->o) * sizeof(double), cudaMemcpyDeviceToHost,
                     p->st));
  CK(cudaStreamSynchronize(p->st));
  return harvest(p);
}

// Set the problem mask of the next launches (uploaded only when it changes;
// the host array is pageable, so the copy has consumed it on return).
ahoc_status set_act(ahoc_plan* p, const std::vector<int>& m) {
  if (m == p->act_now) return AHOC_OK;
  CK(cudaMemcpyAsync(p->act, m.data(), m.size() * sizeof(int), cudaMemcpyHostToDevice, p->st));
  p->act_now = m;
  return AHOC_OK;
}

bool any(const std::vector<int>& m) {
  for (int v : m)
    if (v) return true;
  return false;
}

// The v-solve with variable beta/alpha (Sec. 2.2 v-equation; Sec. 4 solver
// settings: BiCGSTAB preconditioned by an FFT solver): B V = rhs with
// B = L_h - M(gam .) and V = 0 on the boundary, rhs in W1 on entry, V in W1 on
// exit.  Right-preconditioned BiCGSTAB; the preconditioner and the initial
// guess are the FFT solve with the constant shift gam0 = opts.shift, so
// B P^-1 = I - M((gam - gam0) .) P^-1, a lower-order perturbation of the
// identity.  Every problem of the batch in lockstep, each stopping on its own
// at ||r|| <= 1e-14 ||rhs|| (or on stagnation); the caller's mask is restored.
constexpr double kBicgTol = 1e-14;
constexpr int kBicgMaxIters = 200;
ahoc_status bicgstab_v(ahoc_plan* p) {
  const Geom& g = p->g;
  const int nb = g.nb, hs = hstride(p->o);
  const int64_t n = g.npad;
  double* b = p->bcg;
  double* r = b + (int64_t)nb * n;
  double* rh = r + (int64_t)nb * n;
  double* pv = rh + (int64_t)nb * n;
  double* v = pv + (int64_t)nb * n;
  double* s = v + (int64_t)nb * n;
  double* t = s + (int64_t)nb * n;
  double* ph = t + (int64_t)nb * n;
  double* sh = ph + (int64_t)nb * n;
  double* x = p->W1;
  const std::vector<int> caller = p->act_now;
  std::vector<int> live = caller;
  std::vector<double> c(3 * (size_t)nb, 0.0);
  auto comb = [&](double* y, const double* x0, const double* x1, const double* x2) -> ahoc_status {
    CK(cudaMemcpyAsync(p->bcoef, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
    RUN(AHOC_K_OTHER, launch_comb(g, n, y, x0, x1, x2, p->bcoef, p->st));
    return AHOC_OK;
  };
  auto set3 = [&](double a0, const std::vector<double>* a1, double s1, const std::vector<double>* a2, double s2) {
    for (int i = 0; i < nb; ++i) {
      c[3 * i] = a0;
      c[3 * i + 1] = a1 ? s1 * (*a1)[i] : s1;
      c[3 * i + 2] = a2 ? s2 * (*a2)[i] : s2;
    }
  };
  // <a_b, x_b> of every problem in the mask into the exchange area at off
  auto fdot = [&](const double* a, const double* w, int off) -> ahoc_status {
    BatchDot bd;
    bd.vstride = n;
    bd.wstride = n;
    bd.pstride = pstride(p->o);
    bd.act = g.act;
    RUNN(AHOC_K_KRYLOV, 2, launch_mdot(a, n, 1, w, n, p->partial, kDotBlocks, p->hdev + off, p->st, nb, bd, hs));
    return AHOC_OK;
  };
  auto h = [&](int i, int off) { return p->hhost[(size_t)i * hs + off]; };
  std::vector<double> bn(nb), rho(nb, 1.0), rho1(nb), alpha(nb, 1.0), omega(nb, 1.0), beta(nb), best(nb);
  std::vector<int> stall(nb, 0);
  set3(1.0, nullptr, 0.0, nullptr, 0.0);
  CKS(comb(b, x, nullptr, nullptr));  // b = rhs
  CKS(poisson_inplace(p, x, true));    // x0 = P^-1 rhs
  RUN(AHOC_K_OTHER, launch_vop(g, p->cf, v, x, p->gam, p->st));
  set3(1.0, nullptr, -1.0, nullptr, 0.0);
  CKS(comb(r, b, v, nullptr));  // r = rhs - B x0
  set3(1.0, nullptr, 0.0, nullptr, 0.0);
  CKS(comb(rh, r, nullptr, nullptr));
  CK(cudaMemsetAsync(pv, 0, (size_t)nb * n * sizeof(double), p->st));
  CK(cudaMemsetAsync(v, 0, (size_t)nb * n * sizeof(double), p->st));
  CKS(fdot(b, b, 0));
  CKS(fdot(rh, r, 1));
  CKS(fetch(p));
  for (int i = 0; i < nb; ++i) {
    if (!live[i]) continue;
    bn[i] = std::sqrt(h(i, 0));
    rho1[i] = h(i, 1);
    best[i] = std::sqrt(std::fabs(rho1[i]));
    if (!(bn[i] > 0) || best[i] <= kBicgTol * bn[i]) live[i] = 0;
  }
  for (int it = 0; it < kBicgMaxIters && any(live); ++it) {
    CKS(set_act(p, live));
    for (int i = 0; i < nb; ++i)
      if (live[i]) {
        beta[i] = (rho1[i] / rho[i]) * (alpha[i] / omega[i]);
        rho[i] = rho1[i];
      }
    // p = r + beta (p - omega v)
    for (int i = 0; i < nb; ++i) {
      c[3 * i] = 1.0;
      c[3 * i + 1] = beta[i];
      c[3 * i + 2] = -beta[i] * omega[i];
    }
    CKS(comb(pv, r, pv, v));
    set3(1.0, nullptr, 0.0, nullptr, 0.0);
    CKS(comb(ph, pv, nullptr, nullptr));
    CKS(poisson_inplace(p, ph, true));
    RUN(AHOC_K_OTHER, launch_vop(g, p->cf, v, ph, p->gam, p->st));
    CKS(fdot(rh, v, 0));
    CKS(fetch(p));
    for (int i = 0; i < nb; ++i)
      if (live[i]) {
        const double d = h(i, 0);
        alpha[i] = d != 0.0 ? rho[i] / d : 0.0;
        if (!std::isfinite(alpha[i])) return fail(AHOC_ENUMERIC, "BiCGSTAB breakdown in the v-solve");
      }
    // s = r - alpha v
    set3(1.0, &alpha, -1.0, nullptr, 0.0);
    CKS(comb(s, r, v, nullptr));
    set3(1.0, nullptr, 0.0, nullptr, 0.0);
    CKS(comb(sh, s, nullptr, nullptr));
    CKS(poisson_inplace(p, sh, true));
    RUN(AHOC_K_OTHER, launch_vop(g, p->cf, t, sh, p->gam, p->st));
    CKS(fdot(t, s, 0));
    CKS(fdot(t, t, 1));
    CKS(fetch(p));
    for (int i = 0; i < nb; ++i)
      if (live[i]) omega[i] = h(i, 1) > 0 ? h(i, 0) / h(i, 1) : 0.0;
    // x += alpha p-hat + omega s-hat;  r = s - omega t
    set3(1.0, &alpha, 1.0, &omega, 1.0);
    CKS(comb(x, x, ph, sh));
    set3(1.0, &omega, -1.0, nullptr, 0.0);
    CKS(comb(r, s, t, nullptr));
    CKS(fdot(r, r, 0));
    CKS(fdot(rh, r, 1));
    CKS(fetch(p));
    ++p->bicg_iters;
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      const double rn = std::sqrt(h(i, 0));
      rho1[i] = h(i, 1);
      if (!std::isfinite(rn)) return fail(AHOC_ENUMERIC, "non-finite residual in the v-solve");
      if (rn <= kBicgTol * bn[i] || omega[i] == 0.0 || rho1[i] == 0.0) {
        live[i] = 0;
        continue;
      }
      // stagnation at the rounding floor: three steps without a new best
      if (rn < 0.5 * best[i]) {
        best[i] = rn;
        stall[i] = 0;
      } else if (++stall[i] >= 3) {
        live[i] = 0;
      }
    }
  }
  return set_act(p, caller);
}

bool is_fin(double x) { return std::isfinite(x); }

}  // namespace

// host helpers shared with other translation units of the library
namespace ahoc {
ahoc_status host_make_geom(int dim, const int64_t* N, const double* lo, const double* hi, Geom* g) {
  return make_geom(dim, N, lo, hi, g);
}
Coefs host_make_coefs(const Geom& g) { return make_coefs(g); }
ahoc_status host_fail(ahoc_status s, const char* msg) { return fail(s, msg); }
bool host_tri_chunked(const Geom& g) { return tri_ncols(g) < kChunkedBelow; }
int host_tri_chunk_len(const Geom& g) { return tri_chunk_len(g); }
}  // namespace ahoc

extern "C" {

const char* ahoc_status_string(ahoc_status s) {
  switch (s) {
    case AHOC_OK: return "AHOC_OK";
    case AHOC_EINVAL: return "AHOC_EINVAL: invalid argument";
    case AHOC_ENOMEM: return "AHOC_ENOMEM: out of device memory or workspace too small";
    case AHOC_ECUDA: return "AHOC_ECUDA: CUDA runtime error";
    case AHOC_ENOCONV: return "AHOC_ENOCONV: GMRES did not reach the tolerance";
    case AHOC_ENUMERIC: return "AHOC_ENUMERIC: NaN or Inf in a residual";
    case AHOC_ETIMEOUT: return "AHOC_ETIMEOUT: device wait timed out";
    case AHOC_EUNSUPPORTED: return "AHOC_EUNSUPPORTED: not supported by the library";
    case AHOC_EINTERNAL: return "AHOC_EINTERNAL: internal error";
  }
  return "unknown ahoc_status";
}

const char* ahoc_last_error(void) { return g_err.c_str(); }

ahoc_status ahoc_workspace_bytes(int dim, const int64_t* N, const ahoc_opts* opts, size_t* bytes) {
  if (!bytes) return fail(AHOC_EINVAL, "bytes is NULL");
  Geom g;
  CKS(make_geom(dim, N, nullptr, nullptr, &g));
  Opts o;
  CKS(read_opts(opts, &o));
  g.nb = o.batch;
  apply_tuning(g, o);
  if (opts && opts->auto_shift && !o.tri) {
    // the data decide the beta class: size for the larger of the two
    // (variable beta: BiCGSTAB fields; constant shift: shifted tables, U-hat slots)
    Opts a = o, b = o;
    a.varb = 1;
    a.shift = 1.0;
    b.varb = 0;
    b.shift = 1.0;
    *bytes = std::max(total_bytes(g, a), total_bytes(g, b));
    return AHOC_OK;
  }
  *bytes = total_bytes(g, o);
  return AHOC_OK;
}

int64_t ahoc_n_gamma(const ahoc_plan* p) { return p ? p->g.ngamma : -1; }

}  // extern "C"

namespace {

#define CKC(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(AHOC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Shape-only part of a plan: workspace, shared tables (DST twiddles, per-mode
// tridiagonal factors, preconditioner symbols, trace weights) and the coarse
// levels of the nested guess; the per-problem arrays are filled by
// plan_load.  On failure *out may hold a partial plan for the caller to destroy.
ahoc_status plan_alloc(ahoc_plan** out, int dim, const int64_t* N, const double* lo, const double* hi, const Opts& o,
                       cudaStream_t stream) {
  Geom g;
  CKS(make_geom(dim, N, lo, hi, &g));
  g.nb = o.batch;
  apply_tuning(g, o);
  if (g.n2 * g.nb > 65535) return fail(AHOC_EUNSUPPORTED, "batch too large for this grid (N2 * batch > 65535)");
  if (o.navier >> (2 * dim)) return fail(AHOC_EINVAL, "navier names a face beyond 2 * dim");
  g.navier = o.navier;
  Coefs cf = make_coefs(g);
  cf.gam = o.shift;
  if (o.tri) cf.fsign = 1.0;  // the w-equation L_h W = M f
  const bool shifted = o.shift != 0.0;
  std::vector<Mode<double>> modes, modes_v;
  std::vector<long double> roots, roots_v;
  CKS(mode_table<double>(g, cf, modes, 0.0, &roots));
  if (shifted) CKS(mode_table<double>(g, cf, modes_v, o.shift, &roots_v));
  std::vector<Mode<float>> modesf, modesf_v;
  if (o.prec == AHOC_MIXED) CKS(mode_table<float>(g, cf, modesf));
  if (o.prec == AHOC_MIXED && shifted) CKS(mode_table<float>(g, cf, modesf_v, o.shift));
  Layout L = make_layout(g, o);
  const size_t need = total_bytes(g, o);
  if (o.workspace && o.workspace_bytes < need) return fail(AHOC_ENOMEM, "caller workspace too small");

  ahoc_plan* p = new (std::nothrow) ahoc_plan();
  if (!p) return fail(AHOC_ENOMEM, "host allocation failed");
  *out = p;
  p->g = g;
  p->cf = cf;
  p->o = o;
  p->L = L;
  p->st = stream;
  if (o.workspace) {
    p->ws = reinterpret_cast<char*>(o.workspace);
  } else {
    cudaError_t e = cudaMalloc(&p->ws, L.total);
    if (e != cudaSuccess) {
      p->ws = nullptr;
      cudaGetLastError();
      return fail(AHOC_ENOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
    }
    p->own_ws = true;
  }
  p->W1 = at<double>(p, L.W1);
  p->W2 = at<double>(p, L.W2);
  p->nbank = bank_slots(g, o);
  if (p->nbank) {
    p->bank = at<double>(p, L.bank);
    p->Ud = at<double>(p, L.Ud);
    p->Vd = at<double>(p, L.Vd);
  }
  p->ainv = at<double>(p, L.ainv);
  p->afac = at<double>(p, L.afac);
  p->gD = at<double>(p, L.gD);
  p->vedge = at<double>(p, L.vedge);
  p->gN = at<double>(p, L.gN);
  p->lapt = at<double>(p, L.lapt);
  p->twx = at<double>(p, L.twx);
  p->snx = at<double>(p, L.snx);
  p->twy = at<double>(p, L.twy);
  p->sny = at<double>(p, L.sny);
  p->twz = at<double>(p, L.twz);
  p->snz = at<double>(p, L.snz);
  for (int a = 0; a < 3; ++a) {
    p->stab[a] = at<double>(p, L.stab[a]);
    p->ctab[a] = at<double>(p, L.ctab[a]);
    p->twf[a] = at<float>(p, L.twf[a]);
    p->snf[a] = at<float>(p, L.snf[a]);
  }
  p->pre = at<double>(p, L.pre);
  p->tri = at<double>(p, L.tri);
  p->rxm = at<double>(p, L.rxm);
  p->rxp = at<double>(p, L.rxp);
  p->qy = at<double>(p, L.qy);
  p->R2 = at<double>(p, L.R2);
  p->tau = at<double>(p, L.tau);
  p->tauy = at<double>(p, L.tauy);
  p->gen3 = at<double>(p, L.gen3);
  p->tr3 = at<double>(p, L.tr3);
  p->modes = at<Mode<double>>(p, L.modes);
  p->modes_v = shifted ? at<Mode<double>>(p, L.modes_v) : p->modes;
  p->gL = at<double>(p, L.gL);
  if (o.tri) {
    p->lapgD = at<double>(p, L.lapgD);
    p->bilap = at<double>(p, L.bilap);
    p->gNN = at<double>(p, L.gNN);
    p->laptw = at<double>(p, L.laptw);
    p->vface = at<double>(p, L.vface);
  }
  if (o.varb) {
    p->gam = at<double>(p, L.gam);
    p->bcoef = at<double>(p, L.bcoef);
    if (o.prec == AHOC_FP64) p->bcg = at<double>(p, L.bcg);
  }
  p->b = at<double>(p, L.b);
  p->Q = at<double>(p, L.Q);
  p->r = at<double>(p, L.r);
  p->tmp = at<double>(p, L.tmp);
  p->Kry = at<double>(p, L.Kry);
  p->Zb = at<double>(p, L.Zb);
  p->afinv = at<double>(p, L.afinv);
  p->qa = at<double>(p, L.qa);
  p->rpow = at<double>(p, L.rpow);
  p->rpow_v = shifted ? at<double>(p, L.rpow_v) : p->rpow;
  if (tri2_for(g)) {
    p->tri2 = at<double>(p, L.tri2);
    p->tri2_v = shifted ? at<double>(p, L.tri2_v) : p->tri2;
  }
  p->partial = at<double>(p, L.partial);
  p->hdev = at<double>(p, L.hdev);
  p->act = at<int>(p, L.act);
  p->scal = at<double>(p, L.scal);
  p->ncolsb = at<int>(p, L.ncolsb);
  p->cgscnt = at<int>(p, L.cgscnt);
  p->gs = at<double>(p, L.gs);
  p->gi = at<int>(p, L.gi);
  p->grel = at<double>(p, L.grel);
  p->gini = at<double>(p, L.gini);
  p->gii = at<int>(p, L.gii);
  p->g.act = p->act;
  if (o.prec == AHOC_MIXED) {
    p->F1 = at<float>(p, L.F1);
    p->F2 = at<float>(p, L.F2);
    p->Ru = at<float>(p, L.Ru);
    p->Rv = at<float>(p, L.Rv);
    p->U64 = at<double>(p, L.U64);
    p->V64 = at<double>(p, L.V64);
    p->modesf = at<Mode<float>>(p, L.modesf);
    p->modesf_v = shifted ? at<Mode<float>>(p, L.modesf_v) : p->modesf;
    p->trif = at<float>(p, L.trif);
    p->Rq = at<double>(p, L.Rq);
    p->dQ = at<double>(p, L.dQ);
    p->b2 = at<double>(p, L.b2);
    p->ainvf = at<float>(p, L.ainvf);
    p->rxmf = at<float>(p, L.rxmf);
    p->rxpf = at<float>(p, L.rxpf);
    p->qyf = at<float>(p, L.qyf);
    p->qaf = at<float>(p, L.qaf);
    p->R2f = at<float>(p, L.R2f);
    p->tauf = at<float>(p, L.tauf);
    p->skf = at<float>(p, L.skf);
    p->ckf = at<float>(p, L.ckf);
    p->gen3f = at<float>(p, L.gen3f);
    p->skyf = at<float>(p, L.skyf);
    p->tauyf = at<float>(p, L.tauyf);
  }
  const size_t B = (size_t)g.nb;
  const size_t fld = (size_t)g.npad * sizeof(double);
  const size_t full = (size_t)g.nfull * sizeof(double);
  const size_t face = (size_t)g.ngamma * sizeof(double);
  p->part.assign(g.nb, 1);
  p->ps.assign(g.nb, ProbStat{});
  CKC(cudaMallocHost(&p->hhost, B * (size_t)hstride(o) * sizeof(double)));
  CKC(cudaMallocHost(&p->scal_h, B * sizeof(double)));
  CKC(cudaMallocHost(&p->act_h, B * sizeof(int)));
  CKC(cudaMallocHost(&p->gini_h, 3 * B * sizeof(double)));
  CKC(cudaMallocHost(&p->gii_h, 2 * B * sizeof(int)));
  CKC(cudaMallocHost(&p->rb_rel, B * sizeof(double)));
  CKC(cudaMallocHost(&p->rb_act, B * sizeof(int)));
  CKC(cudaMallocHost(&p->rb_gi, B * (size_t)kGivensInts * sizeof(int)));
  // the BiCGSTAB v-solves read residual norms on the host inside the matvec
  p->use_graphs = o.graphs && !o.timing && !(o.varb && o.prec == AHOC_FP64);
  p->gexec.assign((o.restart + kArnoldiBlock - 1) / kArnoldiBlock, nullptr);
  p->gcount.assign((o.restart + kArnoldiBlock - 1) / kArnoldiBlock, ahoc_plan::GCount{});
  CKC(cudaEventCreate(&p->ev0));
  CKC(cudaEventCreate(&p->ev1));
  if (p->use_graphs) {
    // the graph stream takes the caller's stream priority, so that a plan on a
    // high-priority stream keeps it for its GMRES steps
    int prio = 0;
    if (stream == nullptr || cudaStreamGetPriority(stream, &prio) != cudaSuccess) {
      cudaGetLastError();
      prio = 0;
    }
    CKC(cudaStreamCreateWithPriority(&p->gst, cudaStreamNonBlocking, prio));
    CKC(cudaEventCreateWithFlags(&p->gev_in, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&p->gev_out, cudaEventDisableTiming));
  }
  // zero padding of the fields and zero boundary data until a problem brings its own
  CKC(cudaMemsetAsync(p->W1, 0, B * fld, p->st));
  CKC(cudaMemsetAsync(p->W2, 0, B * fld, p->st));
  if (p->nbank) CKC(cudaMemsetAsync(p->bank, 0, (size_t)(p->nbank + 1) * B * fld, p->st));
  CKC(cudaMemsetAsync(p->gD, 0, B * full, p->st));
  CKC(cudaMemsetAsync(p->vedge, 0, B * full, p->st));
  CKC(cudaMemsetAsync(p->gN, 0, B * face, p->st));
  CKC(cudaMemsetAsync(p->lapt, 0, B * face, p->st));
  CKC(cudaMemsetAsync(p->gL, 0, B * face, p->st));
  CKC(cudaMemsetAsync(p->cgscnt, 0, B * (size_t)cgs_groups(o) * sizeof(int), p->st));
  CKS(set_act(p, p->part));
  std::vector<double> tw, sn;
  dst_tables(g.N[0], tw, sn);
  CKC(cudaMemcpyAsync(p->twx, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
  CKC(cudaMemcpyAsync(p->snx, sn.data(), sn.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
  CKC(cudaStreamSynchronize(p->st));
  dst_tables(g.N[1], tw, sn);
  CKC(cudaMemcpyAsync(p->twy, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
  CKC(cudaMemcpyAsync(p->sny, sn.data(), sn.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
  CKC(cudaMemcpyAsync(p->modes, modes.data(), modes.size() * sizeof(Mode<double>), cudaMemcpyHostToDevice, p->st));
  if (shifted)
    CKC(cudaMemcpyAsync(p->modes_v, modes_v.data(), modes_v.size() * sizeof(Mode<double>), cudaMemcpyHostToDevice,
                        p->st));
  CKC(cudaStreamSynchronize(p->st));
  if (o.prec == AHOC_MIXED) {
    const size_t ffl = (size_t)g.npad * sizeof(float);
    CKC(cudaMemsetAsync(p->F1, 0, B * ffl, p->st));
    CKC(cudaMemsetAsync(p->F2, 0, B * ffl, p->st));
    CKC(cudaMemcpyAsync(p->modesf, modesf.data(), modesf.size() * sizeof(Mode<float>), cudaMemcpyHostToDevice,
                        p->st));
    if (shifted)
      CKC(cudaMemcpyAsync(p->modesf_v, modesf_v.data(), modesf_v.size() * sizeof(Mode<float>),
                          cudaMemcpyHostToDevice, p->st));
  }
  for (int a = 0; a < g.dim; ++a) {
    dst_tables(g.N[a], tw, sn);
    std::vector<float> twf(tw.begin(), tw.end()), snf(sn.begin(), sn.end());
    CKC(cudaMemcpyAsync(p->twf[a], twf.data(), twf.size() * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CKC(cudaMemcpyAsync(p->snf[a], snf.data(), snf.size() * sizeof(float), cudaMemcpyHostToDevice, p->st));
    CKC(cudaStreamSynchronize(p->st));
  }
  if (g.dim == 3) {
    dst_tables(g.N[2], tw, sn);
    CKC(cudaMemcpyAsync(p->twz, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
    CKC(cudaMemcpyAsync(p->snz, sn.data(), sn.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
    CKC(cudaStreamSynchronize(p->st));
  }
  {
    // sin(j pi / N_a), j < 2 N_a and cos(k pi / N_a), k <= N_a, for the preconditioner symbols
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<double> st, ct;
    for (int a = 0; a < g.dim; ++a) {
      const int Na = g.N[a];
      st.resize(2 * (size_t)Na);
      ct.resize((size_t)Na + 1);
      for (int j = 0; j < 2 * Na; ++j) st[j] = (double)sinl(pi * j / Na);
      for (int k = 0; k <= Na; ++k) ct[k] = (double)cosl(pi * k / Na);
      CKC(cudaMemcpyAsync(p->stab[a], st.data(), st.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
      CKC(cudaMemcpyAsync(p->ctab[a], ct.data(), ct.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
      CKC(cudaStreamSynchronize(p->st));
    }
    // tau_k = sum_m w_m sin(m k pi / N_a): one-sided weights of the a-faces in
    // a-modes (fused traces; x and, for 3D, y)
    for (int a = 0; a < 2; ++a) {
      std::vector<double> tau((size_t)g.N[a] + 1, 0.0);
      for (int k = 1; k < g.N[a]; ++k) {
        long double t = 0;
        for (int m = 1; m <= 3; ++m) t += (long double)cf.w[a][m] * sinl(pi * (long double)(m * k) / g.N[a]);
        tau[k] = (double)t;
      }
      CKC(cudaMemcpyAsync(a == 0 ? p->tau : p->tauy, tau.data(), tau.size() * sizeof(double),
                          cudaMemcpyHostToDevice, p->st));
      CKC(cudaStreamSynchronize(p->st));
    }
  }
  if (tri2_for(g)) {
    const int L2 = tri_chunk_len(g);
    std::vector<double> t2(tri2_table_size(g, L2));
    tri2_table_fill(g, L2, roots.data(), t2.data());
    CKC(cudaMemcpyAsync(p->tri2, t2.data(), t2.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
    CKC(cudaStreamSynchronize(p->st));
    if (shifted) {
      tri2_table_fill(g, L2, roots_v.data(), t2.data());
      CKC(cudaMemcpyAsync(p->tri2_v, t2.data(), t2.size() * sizeof(double), cudaMemcpyHostToDevice, p->st));
      CKC(cudaStreamSynchronize(p->st));
    }
  }
  if (chunked_for(g, o.prec)) CKC(launch_tri_powers(g, p->modes, p->rpow, tri_chunk_len(g), p->st));
  if (chunked_for(g, o.prec) && shifted)
    CKC(launch_tri_powers(g, p->modes_v, p->rpow_v, tri_chunk_len(g), p->st));
  if (o.prec == AHOC_MIXED) {
    CKC(launch_to_float(p->tauf, p->tau, g.N[0] + 1, p->st));
    CKC(launch_to_float(p->skf, p->stab[0], 2 * (int64_t)g.N[0], p->st));
    CKC(launch_to_float(p->ckf, p->ctab[0], g.N[0] + 1, p->st));
    CKC(launch_to_float(p->skyf, p->stab[1], 2 * (int64_t)g.N[1], p->st));
    CKC(launch_to_float(p->tauyf, p->tauy, g.N[1] + 1, p->st));
  }
  if (o.precond && !o.tri) {  // the triharmonic class measures its symbols (tri_symbols)
    const double* stp[3] = {p->stab[0], p->stab[1], g.dim == 3 ? p->stab[2] : nullptr};
    const double* ctp[3] = {p->ctab[0], p->ctab[1], g.dim == 3 ? p->ctab[2] : nullptr};
    CKC(launch_face_symbols(g, cf, p->pre, stp, ctp, p->st));
  }
  CKC(cudaStreamSynchronize(p->st));
  const int lv = coarse_levels(g, o.levels);
  if (lv > 0) {
    int64_t Nc[3];
    double lo_[3], hi_[3];
    for (int a = 0; a < dim; ++a) {
      Nc[a] = g.N[a] / 2;
      lo_[a] = lo ? lo[a] : 0.0;
      hi_[a] = hi ? hi[a] : 1.0;
    }
    Opts oc = o;
    oc.levels = lv - 1;
    oc.uhat = -1;  // coarse levels only solve for Q
    oc.workspace = o.workspace ? (void*)(p->ws + L.total) : nullptr;
    oc.workspace_bytes = o.workspace ? o.workspace_bytes - L.total : 0;
    CKS(plan_alloc(&p->coarse, dim, Nc, lo_, hi_, oc, stream));
    p->levels = lv;
  }
  return AHOC_OK;
}

// Problem b's coefficient and boundary data (device, single-problem sizes):
// 1/alpha, the face alpha and its inverse, the FP32 copies of the mixed
// path, the data arrays (zero where bd gives none) and, recursively, the
// injected data of the coarse levels.
ahoc_status plan_load(ahoc_plan* p, int b, const double* alpha, const ahoc_bdata* bd) {
  Geom g = p->g;
  g.nb = 1;
  g.act = nullptr;
  const size_t full = (size_t)g.nfull * sizeof(double);
  const size_t face = (size_t)g.ngamma * sizeof(double);
  const int64_t pf = (int64_t)b * g.nfull, pg = (int64_t)b * g.ngamma, pp = (int64_t)b * g.npad;
  CKC(launch_recip(p->ainv + pf, alpha, g.nfull, p->st));
  if (alpha) CKC(launch_face_gather(g, p->afac + pg, alpha, p->st));
  else CKC(launch_recip(p->afac + pg, nullptr, g.ngamma, p->st));  // unit coefficient (triharmonic class)
  CKC(launch_recip(p->afinv + pg, p->afac + pg, g.ngamma, p->st));
  if (p->o.prec == AHOC_MIXED) CKC(launch_to_float(p->ainvf + pf, p->ainv + pf, g.nfull, p->st));
  auto put = [&](double* dst, const double* src, size_t bytes, bool& flag) -> ahoc_status {
    if (src) {
      CKC(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, p->st));
      flag = true;
    } else {
      CKC(cudaMemsetAsync(dst, 0, bytes, p->st));
    }
    return AHOC_OK;
  };
  CKS(put(p->gD + pf, bd ? bd->g_D : nullptr, full, p->has_gD));
  CKS(put(p->vedge + pf, bd ? bd->v_edge : nullptr, full, p->has_vedge));
  CKS(put(p->gN + pg, bd ? bd->g_N : nullptr, face, p->has_gN));
  CKS(put(p->lapt + pg, bd ? bd->lapt_gD : nullptr, face, p->has_lapt));
  CKS(put(p->gL + pg, bd ? bd->g_L : nullptr, face, p->has_gL));
  if (p->o.tri) {
    CKS(put(p->lapgD + pf, bd ? bd->lap_gD : nullptr, full, p->has_lapgD));
    CKS(put(p->bilap + pf, bd ? bd->bilap : nullptr, full, p->has_bilap));
    CKS(put(p->gNN + pg, bd ? bd->g_NN : nullptr, face, p->has_gNN));
    CKS(put(p->laptw + pg, bd ? bd->lapt_w : nullptr, face, p->has_laptw));
    if (bd && bd->lap_gD) CKC(launch_face_gather(g, p->vface + pg, bd->lap_gD, p->st));
    else CKC(cudaMemsetAsync(p->vface + pg, 0, face, p->st));
  }
  if (p->o.varb) {
    if (!bd || !bd->beta) return fail(AHOC_EINVAL, "variable_beta needs beta for every problem");
    CKC(launch_mul(p->gam + pf, bd->beta, p->ainv + pf, g.nfull, p->st));
  }
  if (p->coarse) {
    // coarse data by injection, staged in this problem's field and face buffers
    Geom gc = p->coarse->g;
    gc.nb = 1;
    gc.act = nullptr;
    double* a_c = p->W1 + pp;
    double* gD_c = bd && bd->g_D ? p->W2 + pp : nullptr;
    double* vE_c = bd && bd->v_edge ? p->W2 + pp + gc.nfull : nullptr;
    double* gN_c = bd && bd->g_N ? p->b + pg : nullptr;
    double* lt_c = bd && bd->lapt_gD ? p->r + pg : nullptr;
    double* gL_c = bd && bd->g_L ? p->tmp + pg : nullptr;
    double* be_c = bd && bd->beta ? p->W2 + pp + 2 * gc.nfull : nullptr;
    CKC(launch_inject_full(gc, g, a_c, alpha, p->st));
    if (gD_c) CKC(launch_inject_full(gc, g, gD_c, bd->g_D, p->st));
    if (vE_c) CKC(launch_inject_full(gc, g, vE_c, bd->v_edge, p->st));
    if (gN_c) CKC(launch_inject_face(gc, g, gN_c, bd->g_N, p->st));
    if (lt_c) CKC(launch_inject_face(gc, g, lt_c, bd->lapt_gD, p->st));
    if (gL_c) CKC(launch_inject_face(gc, g, gL_c, bd->g_L, p->st));
    if (be_c) CKC(launch_inject_full(gc, g, be_c, bd->beta, p->st));
    ahoc_bdata bc{gD_c, gN_c, lt_c, vE_c, gL_c, be_c};
    CKS(plan_load(p->coarse, b, a_c, &bc));
    CKC(cudaStreamSynchronize(p->st));
    CKC(cudaMemsetAsync(p->W1 + pp, 0, (size_t)g.npad * sizeof(double), p->st));
    CKC(cudaMemsetAsync(p->W2 + pp, 0, (size_t)g.npad * sizeof(double), p->st));
  }
  return AHOC_OK;
}
#undef CKC

// Preconditioner of the triharmonic class.  With one clamped face and the
// others simply supported, the Schur operator of that face is diagonal in the
// face's sine basis (every Poisson solve of the mixed form then separates in
// the transverse sine modes, as in Lemma 4), so one Schur action gives every
// mode's symbol s: with T the face's DST-I (T^2 = c I, c the product of N_b/2
// over the in-face axes) and Phi = T / sqrt(c), S Phi 1 = Phi s.  The
// preconditioner (out = T(pre T(in))) then has pre = 1 / (c s) on a clamped
// face, the exact inverse in that setting and the per-face inverse symbol
// otherwise, and pre = -1 / c on a simply supported face (its rows are -I).
// Measured on problem 0 (the symbol depends on the shape alone).
ahoc_status tri_symbols(ahoc_plan* p) {
  const Geom& g = p->g;
  std::vector<int> m0(g.nb, 0);
  m0[0] = 1;
  CKS(set_act(p, m0));
  for (int f = 0; f < 2 * g.dim; ++f) {
    const int a = f >> 1;
    double c = 1.0;
    for (int b = 0; b < g.dim; ++b)
      if (b != a) c *= g.N[b] / 2.0;
    const int64_t off = g.face_off[f], len = g.face_off[f + 1] - g.face_off[f];
    if (g.is_navier(f)) {
      CK(launch_scaled_recip(p->pre + off, nullptr, -1.0 / c, len, p->st));
      continue;
    }
    CK(cudaMemsetAsync(p->tmp, 0, (size_t)g.ngamma * sizeof(double), p->st));
    CK(launch_scaled_recip(p->tmp + off, nullptr, 1.0 / std::sqrt(c), len, p->st));
    CKS(face_dsts(p, p->tmp, a));  // Phi 1 on face f, zero elsewhere
    CKS(matvec_dev(p, p->tmp, p->r));
    CKS(face_dsts(p, p->r, a));    // T S Phi 1 = sqrt(c) s on face f
    CK(launch_scaled_recip(p->pre + off, p->r + off, 1.0 / std::sqrt(c), len, p->st));
  }
  CK(cudaStreamSynchronize(p->st));
  CKS(set_act(p, p->part));
  return AHOC_OK;
}

// opts.auto_shift: the beta class from the data.  gamma = beta / alpha over
// every point of every problem: one value everywhere -> the constant shift;
// otherwise variable beta with the mean of gamma as the reference shift of the
// v-solves' FFT preconditioner.  A few KB of device scratch, freed on return.
ahoc_status derive_shift(const Geom& g, Opts& o, const double* alpha, const ahoc_bdata* bd, cudaStream_t st) {
  o.varb = 0;
  o.shift = 0.0;
  if (!bd || !bd->beta) return AHOC_OK;
  constexpr int kBlocks = 296;
  const int64_t n = g.nfull * (int64_t)o.batch;
  double* dev = nullptr;
  if (cudaMalloc(&dev, 3 * kBlocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(AHOC_ENOMEM, "cudaMalloc of the beta/alpha statistics failed");
  }
  std::vector<double> h(3 * kBlocks);
  cudaError_t e = launch_ratio_stats(bd->beta, alpha, n, dev, kBlocks, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dev, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dev);
  if (e != cudaSuccess) return fail(AHOC_ECUDA, std::string("beta/alpha statistics: ") + cudaGetErrorString(e));
  double mn = INFINITY, mx = -INFINITY, sum = 0.0;
  for (int b = 0; b < kBlocks; ++b) {
    mn = std::fmin(mn, h[3 * b]);
    mx = std::fmax(mx, h[3 * b + 1]);
    sum += h[3 * b + 2];
  }
  if (!std::isfinite(mn) || !std::isfinite(mx) || !std::isfinite(sum)) return fail(AHOC_EINVAL, "beta/alpha not finite");
  if (mn < 0) return fail(AHOC_EUNSUPPORTED, kIndefiniteMsg);
  if (mn == mx) {
    o.shift = mn;
  } else {
    o.varb = 1;
    o.shift = sum / (double)n;
  }
  return AHOC_OK;
}

}  // namespace

extern "C" {

ahoc_status ahoc_plan_create(ahoc_plan** out, int dim, const int64_t* N, const double* lo, const double* hi,
                             const double* alpha, const ahoc_bdata* bd, const ahoc_opts* opts, void* stream) {
  std::lock_guard<std::recursive_mutex> lk(capture_mutex());
  Phase ph("ahoc plan create");
  if (!out) return fail(AHOC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!alpha && !(opts && opts->triharmonic)) return fail(AHOC_EINVAL, "alpha is NULL");
  if (misaligned(alpha) || bdata_misaligned(bd)) return fail(AHOC_EINVAL, kAlignMsg);
  Geom g;
  CKS(make_geom(dim, N, lo, hi, &g));
  Opts o;
  CKS(read_opts(opts, &o));
  if (opts && opts->auto_shift && !o.tri) CKS(derive_shift(g, o, alpha, bd, reinterpret_cast<cudaStream_t>(stream)));
  ahoc_plan* p = nullptr;
  ahoc_status s = plan_alloc(&p, dim, N, lo, hi, o, reinterpret_cast<cudaStream_t>(stream));
  for (int b = 0; s == AHOC_OK && b < o.batch; ++b) {
    ahoc_bdata bb{};
    if (bd) {
      bb.g_D = bd->g_D ? bd->g_D + (int64_t)b * g.nfull : nullptr;
      bb.g_N = bd->g_N ? bd->g_N + (int64_t)b * g.ngamma : nullptr;
      bb.lapt_gD = bd->lapt_gD ? bd->lapt_gD + (int64_t)b * g.ngamma : nullptr;
      bb.v_edge = bd->v_edge ? bd->v_edge + (int64_t)b * g.nfull : nullptr;
      bb.g_L = bd->g_L ? bd->g_L + (int64_t)b * g.ngamma : nullptr;
      bb.beta = bd->beta ? bd->beta + (int64_t)b * g.nfull : nullptr;
      bb.lap_gD = bd->lap_gD ? bd->lap_gD + (int64_t)b * g.nfull : nullptr;
      bb.bilap = bd->bilap ? bd->bilap + (int64_t)b * g.nfull : nullptr;
      bb.g_NN = bd->g_NN ? bd->g_NN + (int64_t)b * g.ngamma : nullptr;
      bb.lapt_w = bd->lapt_w ? bd->lapt_w + (int64_t)b * g.ngamma : nullptr;
    }
    s = plan_load(p, b, alpha ? alpha + (int64_t)b * g.nfull : nullptr, &bb);
  }
  if (s == AHOC_OK && cudaStreamSynchronize(p->st) != cudaSuccess) s = fail(AHOC_ECUDA, "plan setup failed");
  if (s == AHOC_OK && o.tri && o.precond) s = tri_symbols(p);
  if (s != AHOC_OK) {
    if (p) ahoc_plan_destroy(p);
    return s;
  }
  *out = p;
  return AHOC_OK;
}

ahoc_status ahoc_plan_load(ahoc_plan* p, int b, const double* alpha, const ahoc_bdata* bd) {
  std::lock_guard<std::recursive_mutex> lk(capture_mutex());
  Phase ph("ahoc plan load");
  if (!p || (!alpha && !p->o.tri)) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(alpha) || bdata_misaligned(bd)) return fail(AHOC_EINVAL, kAlignMsg);
  if (b < 0 || b >= p->g.nb) return fail(AHOC_EINVAL, "problem index out of range");
  p->have_last = false;
  CKS(plan_load(p, b, alpha, bd));
  CK(cudaStreamSynchronize(p->st));
  return AHOC_OK;
}

ahoc_status ahoc_set_active(ahoc_plan* p, const int* mask) {
  if (!p) return fail(AHOC_EINVAL, "NULL argument");
  for (int b = 0; b < p->g.nb; ++b) p->part[b] = mask ? (mask[b] != 0) : 1;
  return AHOC_OK;
}

int ahoc_batch(const ahoc_plan* p) { return p ? p->g.nb : -1; }

ahoc_status ahoc_tune_set(int kind, int dim, int64_t N, int prec, int value) {
  if (kind < 0 || kind >= AHOC_TUNE_NKINDS) return fail(AHOC_EINVAL, "unknown tuning kind");
  if (dim != 2 && dim != 3) return fail(AHOC_EINVAL, "dim must be 2 or 3");
  if (N < 8 || N > kMaxN || !pow2(N)) return fail(AHOC_EINVAL, "N must be a power of two in [8, 4096]");
  if (prec != AHOC_FP64 && prec != AHOC_MIXED) return fail(AHOC_EINVAL, "prec must be AHOC_FP64 or AHOC_MIXED");
  const bool ok = value == 0 || (kind == AHOC_TUNE_TRI_CHUNK    ? (value == 8 || value == 16 || value == 32)
                                 : kind == AHOC_TUNE_DST_RADIX ? (value == 4 || value == 8)
                                                               : (value == 128 || value == 256 || value == 512 ||
                                                                  value == 1024));
  if (!ok) return fail(AHOC_EINVAL, "value not offered for this kind");
  g_tune[kind][dim - 2][prec][ilog2i(N)].store(value);
  return AHOC_OK;
}

int ahoc_tune_get(int kind, int dim, int64_t N, int prec) {
  if (kind < 0 || kind >= AHOC_TUNE_NKINDS || (dim != 2 && dim != 3) || N < 8 || N > kMaxN || !pow2(N) ||
      (prec != AHOC_FP64 && prec != AHOC_MIXED))
    return -1;
  return g_tune[kind][dim - 2][prec][ilog2i(N)].load();
}

ahoc_status ahoc_plan_destroy(ahoc_plan* p) {
  if (!p) return AHOC_OK;
  std::lock_guard<std::recursive_mutex> lk(capture_mutex());
  ahoc_status s = AHOC_OK;
  if (p->st) {
    if (cudaStreamSynchronize(p->st) != cudaSuccess) s = fail(AHOC_ECUDA, "stream sync at destroy failed");
  }
  if (p->coarse) {
    if (ahoc_plan_destroy(p->coarse) != AHOC_OK) s = AHOC_ECUDA;
    p->coarse = nullptr;
  }
  if (p->own_ws && p->ws) cudaFree(p->ws);
  if (p->hf) cudaFree(p->hf);
  if (p->hu) cudaFree(p->hu);
  if (p->hhost) cudaFreeHost(p->hhost);
  if (p->scal_h) cudaFreeHost(p->scal_h);
  if (p->act_h) cudaFreeHost(p->act_h);
  if (p->gini_h) cudaFreeHost(p->gini_h);
  if (p->gii_h) cudaFreeHost(p->gii_h);
  if (p->rb_rel) cudaFreeHost(p->rb_rel);
  if (p->rb_act) cudaFreeHost(p->rb_act);
  if (p->rb_gi) cudaFreeHost(p->rb_gi);
  for (auto& ge : p->gexec)
    if (ge) cudaGraphExecDestroy(ge);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->gev_in) cudaEventDestroy(p->gev_in);
  if (p->gev_out) cudaEventDestroy(p->gev_out);
  if (p->gst) cudaStreamDestroy(p->gst);
  for (auto& ev : p->pool) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (auto& ev : p->pending) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  delete p;
  return s;
}

ahoc_status ahoc_matvec(ahoc_plan* p, const double* q, double* y) {
  if (!p || !q || !y) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(q) || misaligned(y)) return fail(AHOC_EINVAL, kAlignMsg);
  if (q == y) return fail(AHOC_EINVAL, "q and y may not alias");
  CKS(set_act(p, p->part));
  return matvec_dev(p, q, y);
}

ahoc_status ahoc_schur_rhs(ahoc_plan* p, const double* f, double* b) {
  if (!p || !f || !b) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(f) || misaligned(b)) return fail(AHOC_EINVAL, kAlignMsg);
  CKS(set_act(p, p->part));
  return schur_rhs_dev(p, f, b);
}

ahoc_status ahoc_dst1(ahoc_plan* p, int axis, const double* in, double* out, double scale) {
  if (!p || !in || !out) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(in) || misaligned(out)) return fail(AHOC_EINVAL, kAlignMsg);
  if (p->g.nb != 1) return fail(AHOC_EINVAL, "ahoc_dst1 takes a single-problem plan");
  if (axis < 0 || axis >= p->g.dim - 1) return fail(AHOC_EINVAL, "axis must be < dim - 1");
  CKS(set_act(p, p->part));
  RUN(AHOC_K_OTHER, launch_unpack(p->g, p->W1, in, p->st));
  if (axis == 0) RUN(AHOC_K_DST_X, launch_dst_x<double>(p->g, p->W1, p->twx, p->snx, scale, p->st));
  else RUN(AHOC_K_DST_Y, launch_dst_y<double>(p->g, p->W1, p->twy, p->sny, scale, p->st));
  RUN(AHOC_K_OTHER, launch_pack(p->g, out, p->W1, p->st));
  return AHOC_OK;
}

ahoc_status ahoc_poisson(ahoc_plan* p, const double* rhs, double* w) {
  if (!p || !rhs || !w) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(rhs) || misaligned(w)) return fail(AHOC_EINVAL, kAlignMsg);
  if (p->g.nb != 1) return fail(AHOC_EINVAL, "ahoc_poisson takes a single-problem plan");
  CKS(set_act(p, p->part));
  RUN(AHOC_K_OTHER, launch_unpack(p->g, p->W1, rhs, p->st));
  CKS(poisson_inplace(p, p->W1));
  RUN(AHOC_K_OTHER, launch_pack(p->g, w, p->W1, p->st));
  return AHOC_OK;
}

ahoc_status ahoc_last_qv(ahoc_plan* p, double* q, double* v) {
  if (!p || !q) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(q) || misaligned(v)) return fail(AHOC_EINVAL, kAlignMsg);
  if (!p->have_last) return fail(AHOC_EINVAL, "no solve has completed on this plan");
  if (v && p->o.tri) return fail(AHOC_EUNSUPPORTED, "a triharmonic plan returns Q only (v must be NULL)");
  CK(cudaMemcpyAsync(q, p->Q, (size_t)p->g.nb * p->g.ngamma * sizeof(double), cudaMemcpyDeviceToDevice, p->st));
  CKS(set_act(p, p->part));
  if (v && p->v_lazy) {
    // V = V(data) + V(Q): the v-equation with the converged Q alone, plus the stored data part
    const Geom& g = p->g;
    RUN(AHOC_K_VRHS, launch_vrhs<double>(g, p->cf, p->W1, p->Q, nullptr, nullptr, p->st, nullptr, p->gam));
    CKS(poisson_inplace(p, p->W1, true));
    RUN(AHOC_K_OTHER, launch_axpby(p->W1, p->Vd, 1.0, 1.0, g.npad, p->st, g.nb, nullptr, g.act));
    p->v_lazy = false;
  }
  if (v)
    RUN(AHOC_K_OTHER, launch_v_full(p->g, v, p->o.prec == AHOC_MIXED ? p->V64 : p->W1, p->Q,
                                    p->has_vedge ? p->vedge : nullptr, p->st));
  return AHOC_OK;
}

}  // extern "C"

namespace {

// One Arnoldi step j for every problem in the mask: v_j = src * scal[b]
// (src = r at j = 0, v_j itself after), z_j = P^-1 v_j, w = v_{j+1} = S z_j,
// CGS2 of w against v_0..v_j (the coefficients of both passes and ||w||^2 in
// the Hessenberg exchange area), then that area to the pinned host copy.
ahoc_status arnoldi_step(ahoc_plan* p, int j, int64_t ld, const double* src) {
  const Geom& g = p->g;
  const int64_t n = g.ngamma;
  double* vj = p->Kry + (int64_t)j * ld;
  double* w = p->Kry + (int64_t)(j + 1) * ld;
  double* zj = p->Zb + (int64_t)j * ld;
  double* uh = j < p->nbank ? p->bank + (int64_t)j * g.nb * g.npad : nullptr;
  RUN(AHOC_K_KRYLOV, launch_axpby(vj, src, 0.0, 0.0, n, p->st, g.nb, p->scal, g.act));
  CKS(precond_apply(p, vj, zj));
  CKS(matvec_dev(p, zj, w, uh));
  // CGS2 in three fused passes (the bits of separate dot, update and
  // reduction kernels): h1 = V^T w; w' = w - V h1 (in tmp), h2 = V^T w';
  // w = w' - V h2, ||w||^2
  BatchDot bd;
  bd.vstride = n;
  bd.wstride = n;
  bd.pstride = pstride(p->o);
  bd.act = g.act;
  const int hs = hstride(p->o);
  RUN(AHOC_K_KRYLOV, launch_cgs(p->Kry, ld, j + 1, nullptr, 0, w, nullptr, n, p->partial, kDotBlocks, p->hdev, p->st,
                                g.nb, bd, hs, hs, p->cgscnt, false));
  RUN(AHOC_K_KRYLOV, launch_cgs(p->Kry, ld, j + 1, p->hdev, j + 1, w, p->tmp, n, p->partial, kDotBlocks,
                                p->hdev + (j + 1), p->st, g.nb, bd, hs, hs, p->cgscnt, false));
  RUN(AHOC_K_KRYLOV, launch_cgs(p->Kry, ld, 1, p->hdev + (j + 1), j + 1, p->tmp, w, n, p->partial, kDotBlocks,
                                p->hdev + 2 * (j + 1), p->st, g.nb, bd, hs, hs, p->cgscnt, true));
  // column j of the Hessenberg QR, the convergence test and the next 1 / ||w||, on the device
  RUN(AHOC_K_KRYLOV, launch_givens_step(j, g.nb, p->o.restart, p->hdev, hs, p->act, p->scal, p->gs, p->gi, p->grel,
                                        p->st));
  return AHOC_OK;
}

// Arnoldi steps j0 .. j0 + K - 1 for the problems in the device mask (the
// mask and the scalars pass from step to step on the device: a problem that
// converges leaves the mask at once), then the per-problem state (mask,
// counters, residual estimates) to pinned host memory: one CUDA graph per
// block start, captured on first use and replayed, or plain launches.
// Returns after the host copy is complete.
ahoc_status arnoldi_block(ahoc_plan* p, int j0, int K, int64_t ld) {
  Phase ph("ahoc arnoldi block");
  const int nb = p->g.nb;
  const int slot = j0 / kArnoldiBlock;
  cudaStream_t user = p->st;
  auto body = [&]() -> ahoc_status {
    for (int j = j0; j < j0 + K; ++j) CKS(arnoldi_step(p, j, ld, j == 0 ? p->r : p->Kry + (int64_t)j * ld));
    CK(cudaMemcpyAsync(p->rb_act, p->act, nb * sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CK(cudaMemcpyAsync(p->rb_gi, p->gi, nb * (size_t)kGivensInts * sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CK(cudaMemcpyAsync(p->rb_rel, p->grel, nb * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    return AHOC_OK;
  };
  if (p->use_graphs) {
    // the caller's stream hands over to the plan's graph stream
    CK(cudaEventRecord(p->gev_in, user));
    CK(cudaStreamWaitEvent(p->gst, p->gev_in, 0));
    p->st = p->gst;
  }
  if (p->use_graphs && !p->gexec[slot]) {
    const int64_t l0 = p->launches;
    int64_t k0[AHOC_NK];
    for (int k = 0; k < AHOC_NK; ++k) k0[k] = p->kn[k];
    bool captured = false;
    {
      // no plan of this process allocates or frees (synchronising calls)
      // while a capture is open
      std::lock_guard<std::recursive_mutex> lk(capture_mutex());
      if (cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const ahoc_status s = body();
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->st, &graph);
        if (s == AHOC_OK && e == cudaSuccess && graph &&
            cudaGraphInstantiate(&p->gexec[slot], graph, 0) == cudaSuccess)
          captured = true;
        if (graph) cudaGraphDestroy(graph);
      }
    }
    // the capture issued nothing: count the graph's launches per replay instead
    ahoc_plan::GCount& gc = p->gcount[slot];
    gc.launches = p->launches - l0;
    p->launches = l0;
    for (int k = 0; k < AHOC_NK; ++k) {
      gc.kn[k] = p->kn[k] - k0[k];
      p->kn[k] = k0[k];
    }
    if (!captured) {
      // a capture can be invalidated by another thread's synchronising CUDA
      // call (outside this library); drop the error it left and run this
      // plan with plain launches from now on
      cudaGetLastError();
      p->gexec[slot] = nullptr;
      p->use_graphs = false;
      g_err.clear();
    }
  }
  if (p->use_graphs) {
    const cudaError_t e = cudaGraphLaunch(p->gexec[slot], p->st);
    p->st = user;
    CK(e);
    CK(cudaEventRecord(p->gev_out, p->gst));
    CK(cudaStreamWaitEvent(user, p->gev_out, 0));
    const ahoc_plan::GCount& gc = p->gcount[slot];
    p->launches += gc.launches;
    for (int k = 0; k < AHOC_NK; ++k) p->kn[k] += gc.kn[k];
  } else {
    if (p->st != user) {  // the capture failed: hand back to the caller's stream
      CK(cudaEventRecord(p->gev_out, p->st));
      p->st = user;
      CK(cudaStreamWaitEvent(user, p->gev_out, 0));
    }
    CKS(body());
  }
  CK(cudaStreamSynchronize(p->st));
  p->act_now.assign(p->rb_act, p->rb_act + nb);
  return harvest(p);
}

// Flexible GMRES on S X = b for every problem of the batch in lockstep
// (right-preconditioned with the boundary-symbol operator, whose inexact
// FP32 application is absorbed by storing the directions z_j = P^-1 v_j;
// CGS2 Arnoldi on the device, Givens rotations and the least-squares solve
// on the host in FP64, per problem).  live: the problems to solve; a problem
// that converges (relative residual <= tol[b]) or exhausts maxit[b] is
// masked out of every later launch, so its arithmetic -- and its result --
// is the same as in a solve of its own.  X holds the initial guess on entry
// when `guess` (else it is zeroed) and the iterate on exit; tolerances are
// relative to beta0[b] = ||b_b||.  Restarts (an explicit residual) only when
// the basis is full.
ahoc_status gmres(ahoc_plan* p, const double* b, const std::vector<double>& beta0, double* X, bool guess,
                  const std::vector<double>& tol, const std::vector<int>& maxit, std::vector<int> live,
                  std::vector<ProbStat>& go) {
  Phase ph("ahoc gmres");
  const Geom& g = p->g;
  const int nb = g.nb;
  const int64_t n = g.ngamma;
  const int64_t ld = (int64_t)nb * n;  // Krylov column stride: [column][problem][point]
  const int m = p->o.restart;
  const int hs = hstride(p->o);
  for (int i = 0; i < nb; ++i) {
    go[i].status = AHOC_OK;
    if (live[i] && !(beta0[i] > 0)) live[i] = 0;
  }
  std::vector<double> beta(beta0);
  // U-hat slot of the guess (then of the recovery's sum)
  double* ux0 = p->nbank ? p->bank + (int64_t)p->nbank * nb * g.npad : nullptr;
  p->bank_valid = p->nbank > 0;
  if (guess) {
    // the U-hat slot of a problem GMRES leaves alone (b = 0: Q = 0) must hold
    // zero for the recovery, as after a cold start
    if (ux0) CK(cudaMemsetAsync(ux0, 0, (size_t)nb * g.npad * sizeof(double), p->st));
    CKS(set_act(p, live));
    CKS(matvec_dev(p, X, p->tmp, ux0));
    RUN(AHOC_K_KRYLOV, launch_axpby(p->r, b, 1.0, 0.0, n, p->st, nb, nullptr, g.act));
    RUN(AHOC_K_KRYLOV, launch_axpby(p->r, p->tmp, -1.0, 1.0, n, p->st, nb, nullptr, g.act));
    CKS(mdot(p, p->r, n, 1, p->r, p->hdev));
    CKS(fetch(p));
    for (int i = 0; i < nb; ++i)
      if (live[i]) {
        beta[i] = std::sqrt(p->hhost[(size_t)i * hs]);
        if (!is_fin(beta[i])) {  // this problem fails alone: masked out, the others go on
          go[i].status = AHOC_ENUMERIC;
          live[i] = 0;
        }
      }
  } else {
    CK(cudaMemsetAsync(X, 0, (size_t)nb * n * sizeof(double), p->st));
    if (ux0) CK(cudaMemsetAsync(ux0, 0, (size_t)nb * g.npad * sizeof(double), p->st));
    CKS(set_act(p, live));
    RUN(AHOC_K_KRYLOV, launch_axpby(p->r, b, 1.0, 0.0, n, p->st, nb, nullptr, g.act));
  }
  for (int i = 0; i < nb; ++i)
    if (live[i]) {
      go[i].rel = beta[i] / beta0[i];
      if (go[i].rel <= tol[i]) live[i] = 0;
    }
  if (!any(live)) return AHOC_OK;
  std::vector<int> cyc(nb, 0), nc(nb, 0);
  while (any(live)) {
    for (int i = 0; i < nb; ++i)
      if (live[i] && go[i].iters >= maxit[i]) {
        go[i].status = AHOC_ENOCONV;
        live[i] = 0;
      }
    if (!any(live)) break;
    cyc = live;
    // the cycle's start on the device: mask, 1 / beta, and the QR state
    for (int i = 0; i < nb; ++i) {
      p->scal_h[i] = live[i] ? 1.0 / beta[i] : 0.0;
      p->gini_h[3 * i] = live[i] ? beta[i] : 0.0;
      p->gini_h[3 * i + 1] = beta0[i];
      p->gini_h[3 * i + 2] = tol[i];
      p->gii_h[2 * i] = go[i].iters;
      p->gii_h[2 * i + 1] = maxit[i];
    }
    CKS(set_act(p, live));
    CK(cudaMemcpyAsync(p->scal, p->scal_h, nb * sizeof(double), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemcpyAsync(p->gini, p->gini_h, 3 * nb * sizeof(double), cudaMemcpyHostToDevice, p->st));
    CK(cudaMemcpyAsync(p->gii, p->gii_h, 2 * nb * sizeof(int), cudaMemcpyHostToDevice, p->st));
    RUN(AHOC_K_KRYLOV, launch_givens_init(nb, m, p->act, p->gini, p->gii, p->gs, p->gi, p->grel, p->st));
    for (int j0 = 0; j0 < m && any(live); j0 += kArnoldiBlock) {
      const int K = std::min(kArnoldiBlock, m - j0);
      CK(cudaEventRecord(p->ev0, p->st));
      CKS(arnoldi_block(p, j0, K, ld));
      CK(cudaEventRecord(p->ev1, p->st));
      CK(cudaEventSynchronize(p->ev1));
      float evms = 0.f;
      cudaEventElapsedTime(&evms, p->ev0, p->ev1);
      for (int i = 0; i < nb; ++i) {
        if (!live[i]) continue;
        ProbStat& gi = go[i];
        gi.ms_mv += evms;
        const int* st = p->rb_gi + (size_t)kGivensInts * i;
        gi.iters = st[0];
        gi.rel = p->rb_rel[i];
        if (st[2] == kGivensNumeric) gi.status = AHOC_ENUMERIC;
        if (st[2] == kGivensNoConv) gi.status = AHOC_ENOCONV;
        live[i] = p->rb_act[i];
      }
    }
    // y = R^-1 g and X += Z y per problem of this cycle, on the device
    RUN(AHOC_K_KRYLOV, launch_givens_solve(nb, m, p->gs, p->gi, p->hdev, hs, p->ncolsb, p->st));
    for (int i = 0; i < nb; ++i) nc[i] = cyc[i] ? p->rb_gi[(size_t)kGivensInts * i + 3] : 0;
    CKS(set_act(p, cyc));
    CKS(gemv_sub(p, p->Zb, ld, 0, p->hdev, X, p->ncolsb));
    if (p->bank_valid) {
      // the same combination of the slots' U-hat fields: U-hat of X
      int jmax = 0;
      for (int i = 0; i < nb; ++i) jmax = nc[i] > jmax ? nc[i] : jmax;
      if (jmax <= p->nbank) {
        BatchDot bd;
        bd.vstride = g.npad;
        bd.wstride = g.npad;
        bd.act = g.act;
        RUN(AHOC_K_KRYLOV, launch_gemv_sub(p->bank, (int64_t)nb * g.npad, 0, p->hdev, ux0, g.npad, p->st, nb, bd,
                                           hstride(p->o), p->ncolsb));
      } else {
        p->bank_valid = false;
      }
    }
    CK(cudaStreamSynchronize(p->st));
    CKS(harvest(p));
    if (!any(live)) break;
    // restart the problems whose basis filled: explicit residual r = b - S X
    p->bank_valid = false;
    for (int i = 0; i < nb; ++i)
      if (live[i]) ++go[i].restarts;
    CKS(set_act(p, live));
    CKS(matvec_dev(p, X, p->tmp));
    RUN(AHOC_K_KRYLOV, launch_axpby(p->r, b, 1.0, 0.0, n, p->st, nb, nullptr, g.act));
    RUN(AHOC_K_KRYLOV, launch_axpby(p->r, p->tmp, -1.0, 1.0, n, p->st, nb, nullptr, g.act));
    CKS(mdot(p, p->r, n, 1, p->r, p->hdev));
    CKS(fetch(p));
    for (int i = 0; i < nb; ++i)
      if (live[i]) {
        beta[i] = std::sqrt(p->hhost[(size_t)i * hs]);
        if (!is_fin(beta[i])) {
          go[i].status = AHOC_ENUMERIC;
          live[i] = 0;
          continue;
        }
        go[i].rel = beta[i] / beta0[i];
        if (go[i].rel <= tol[i]) live[i] = 0;
      }
  }
  return AHOC_OK;
}

// ||v_b|| of every problem in the current mask (others: 0); a problem whose
// vector holds a NaN or Inf gets a non-finite norm (the caller masks it out)
ahoc_status norms(ahoc_plan* p, const double* v, std::vector<double>& out) {
  CKS(mdot(p, v, p->g.ngamma, 1, v, p->hdev));
  CKS(fetch(p));
  out.assign(p->g.nb, 0.0);
  for (int i = 0; i < p->g.nb; ++i)
    if (p->act_now[i]) out[i] = std::sqrt(p->hhost[(size_t)i * hstride(p->o)]);
  return AHOC_OK;
}

ahoc_status solve_internal(ahoc_plan* p, const double* f, double* u, double tol);

// A coarse level is used by the automatic nested guess only where it
// resolves the data: its Schur right-hand side, prolonged to this grid's
// faces, within this fraction of this grid's (relative 2-norm).  Smooth data
// agree to the discretisation error; data the coarse grid does not resolve
// (a sin(32 pi x) factor on 512^3 and coarser grids) differ by order one, and
// their coarse solution is a guess no better than zero (measured on B300: the
// 1024^3 high-wavenumber solve took 22 fine iterations after three coarse
// levels, 19 without them, 6.3 against 4.8 s).
constexpr double kNestAgree = 0.1;

// Nested initial guess: solve on the coarser grid (recursively, in the
// plan's precision scheme), then prolong its Q to this grid's faces (the
// coarse-grid interpolated initial guess of Sec. 4.1) into X0.  bfine: this
// grid's Schur right-hand side.  Returns in `used` whether any problem took a
// guess (X0 = 0 for those that did not).
ahoc_status coarse_guess(ahoc_plan* p, const double* f, const std::vector<int>& live, double tol, double* X0,
                         const double* bfine, bool& used) {
  Phase ph("ahoc nested guess");
  const Geom& g = p->g;
  const int nb = g.nb;
  ahoc_plan* c = p->coarse;
  double* f_c = p->W2;  // W2 is free at this point of both solve paths
  CKS(set_act(c, live));
  RUN(AHOC_K_OTHER, launch_inject_full(c->g, g, f_c, f, p->st));
  CK(cudaStreamSynchronize(p->st));
  std::vector<int> use = live;
  if (p->o.nest_auto) {
    // the resolution check; the coarse solve then starts from this b_c.  On
    // a clamped face b carries the one-sided delta_nn's (u_n - g_N) / h term
    // of the data-only solution, so it scales as 1/h: the coarse b, doubled
    // there (every axis halves), is compared with this grid's.  A Navier
    // face's rows (alpha g_L - Q) do not scale.
    CKS(schur_rhs_dev(c, f_c, c->b));
    CKS(set_act(p, live));
    RUN(AHOC_K_KRYLOV, launch_face_prolong(g, c->g, p->tmp, c->b, p->st));
    for (int fc = 0; fc < 2 * g.dim; ++fc) {
      if (g.is_navier(fc)) continue;
      const int64_t off = g.face_off[fc], len = g.face_off[fc + 1] - off;
      RUN(AHOC_K_KRYLOV, launch_axpby(p->tmp + off, p->tmp + off, 2.0, 0.0, len, p->st, nb, nullptr, g.act,
                                      g.ngamma, g.ngamma));
    }
    RUN(AHOC_K_KRYLOV, launch_axpby(p->tmp, bfine, 1.0, -1.0, g.ngamma, p->st, nb, nullptr, g.act));
    std::vector<double> dn, bn;
    CKS(norms(p, p->tmp, dn));
    CKS(norms(p, bfine, bn));
    for (int i = 0; i < nb; ++i)
      if (use[i] && !(dn[i] <= kNestAgree * bn[i])) use[i] = 0;
    c->rhs_ready = true;
  }
  used = any(use);
  if (!used) {
    c->rhs_ready = false;
    CK(cudaMemsetAsync(p->W2, 0, (size_t)nb * g.npad * sizeof(double), p->st));
    return AHOC_OK;
  }
  CKS(set_act(c, use));
  c->part = use;
  const double ctol = p->o.coarse_tol > tol ? p->o.coarse_tol : tol;
  // only the coarse Q is used: the coarse level skips its recovery of V and U
  ahoc_status cs_ = solve_internal(c, f_c, nullptr, ctol);
  c->rhs_ready = false;
  if (cs_ != AHOC_OK) return cs_;  // a coarse level's ENOCONV or ENUMERIC is kept in its stats
  CKS(harvest(p));
  for (int k = 0; k < AHOC_NK; ++k) {
    // kms_top collects minus the coarse share, so kms + kms_top is this level's own time
    const double cms = c->kms[k];
    const int64_t cn = c->kn[k];
    p->kms_top[k] -= cms;
    p->kn_top[k] -= cn;
    p->kms[k] += cms;
    p->kn[k] += cn;
  }
  p->launches += c->launches;
  for (int i = 0; i < nb; ++i) {
    if (!use[i]) continue;
    p->ps[i].coarse_iters = c->ps[i].iters + c->ps[i].coarse_iters;
    p->ps[i].ms_mv += c->ps[i].ms_mv;
    p->ps[i].levels = 1 + c->ps[i].levels;
  }
  CKS(set_act(p, live));
  RUN(AHOC_K_KRYLOV, launch_face_prolong(g, c->g, X0, c->Q, p->st));
  for (int i = 0; i < nb; ++i)  // problems whose data the coarse grid does not resolve start from zero
    if (live[i] && !use[i]) CK(cudaMemsetAsync(X0 + (int64_t)i * g.ngamma, 0, g.ngamma * sizeof(double), p->st));
  // f_c borrowed W2 as a temporary: restore its zero padding
  CK(cudaMemsetAsync(p->W2, 0, (size_t)nb * g.npad * sizeof(double), p->st));
  return AHOC_OK;
}

// Algorithm 1 in FP64: b = -R(0), GMRES on S_h Q = b (from the nested
// coarse-grid guess when the plan has coarse levels), recovery of V and U.
ahoc_status solve_fp64(ahoc_plan* p, const double* f, double* u, double tol) {
  const Geom& g = p->g;
  const int nb = g.nb;
  std::vector<int> live = p->part;
  CKS(set_act(p, live));
  if (!p->rhs_ready) CKS(schur_rhs_dev(p, f, p->b));  // (a coarse level's b may come from the finer level)
  if (p->nbank && u) {  // U and V of the data alone, for the recovery from the slots
    CK(cudaMemcpyAsync(p->Ud, p->W2, (size_t)nb * g.npad * sizeof(double), cudaMemcpyDeviceToDevice, p->st));
    CK(cudaMemcpyAsync(p->Vd, p->W1, (size_t)nb * g.npad * sizeof(double), cudaMemcpyDeviceToDevice, p->st));
  }
  std::vector<double> beta0;
  CKS(norms(p, p->b, beta0));
  for (int i = 0; i < nb; ++i)
    if (live[i] && !is_fin(beta0[i])) {  // NaN or Inf in this problem's data: it fails alone
      p->ps[i].status = AHOC_ENUMERIC;
      live[i] = 0;
      beta0[i] = 0.0;
    }
  bool guess = false;
  bool any_rhs = false;
  for (int i = 0; i < nb; ++i) any_rhs = any_rhs || (live[i] && beta0[i] > 0);
  if (p->q0) {  // the caller's initial Q (ahoc_solve_from) in place of the nested guess
    CK(cudaMemcpyAsync(p->Q, p->q0, (size_t)nb * g.ngamma * sizeof(double), cudaMemcpyDeviceToDevice, p->st));
    for (int i = 0; i < nb; ++i)  // b = 0: Q = 0 exactly (GMRES leaves such a problem's iterate alone)
      if (!(live[i] && beta0[i] > 0))
        CK(cudaMemsetAsync(p->Q + (int64_t)i * g.ngamma, 0, g.ngamma * sizeof(double), p->st));
    guess = true;
  } else if (any_rhs && p->coarse) {
    CKS(coarse_guess(p, f, live, tol, p->Q, p->b, guess));
  }
  std::vector<ProbStat> go(nb);
  CKS(gmres(p, p->b, beta0, p->Q, guess, std::vector<double>(nb, tol), std::vector<int>(nb, p->o.max_iters), live,
            go));
  for (int i = 0; i < nb; ++i) {
    ProbStat& s = p->ps[i];
    s.iters = go[i].iters;
    s.restarts = go[i].restarts;
    s.rel = live[i] && beta0[i] > 0 ? go[i].rel : 0.0;
    if (s.status == AHOC_OK) s.status = go[i].status;
    s.ms_mv += go[i].ms_mv;
  }
  if (!u) return AHOC_OK;  // a coarse level of the nested guess: Q only
  Phase ph("ahoc recovery");
  CKS(set_act(p, p->part));
  if (p->bank_valid) {
    // U = U(data) + U(Q), U(Q) the inverse DST of the combined U-hat (linear
    // in Q: Q = X0 + Z y, so its U-hat is the guess's plus Z's combination);
    // V is formed only if ahoc_last_qv asks for it
    double* ux = p->bank + (int64_t)p->nbank * nb * g.npad;
    RUN(AHOC_K_DST_X, launch_dst_x<double>(g, ux, p->twx, p->snx, 1.0, p->st));
    RUN(AHOC_K_OTHER, launch_axpby(ux, p->Ud, 1.0, 1.0, g.npad, p->st, nb, nullptr, g.act));
    RUN(AHOC_K_OTHER, launch_write_full(g, u, ux, p->has_gD ? p->gD : nullptr, p->st));
    p->v_lazy = true;
    return AHOC_OK;
  }
  p->v_lazy = false;
  if (p->o.tri) {  // W, V and U with the converged Q
    CKS(solve_tri(p, p->Q, f, true));
    RUN(AHOC_K_OTHER, launch_write_full(g, u, p->W1, p->has_gD ? p->gD : nullptr, p->st));
    return AHOC_OK;
  }
  // recovery: V and U with the converged Q (and the data)
  CKS(solve_VU(p, p->Q, f, true));
  RUN(AHOC_K_OTHER, launch_write_full(g, u, p->W2, p->has_gD ? p->gD : nullptr, p->st));
  return AHOC_OK;
}

// Mixed precision: iterative refinement of the coupled system, every problem
// of the batch in lockstep.  Each step takes the FP64 residual of all three
// block rows at x = (U, V, Q), solves the coupled correction system with FP32
// Poisson solves (the same Schur method: b = -R_d(0), GMRES on S dQ = b to
// refine_tol, recovery of dV, dU) and adds the correction in FP64 (the first
// correction, the whole solution, takes its right-hand side and its recovery
// from FP64 solves unless opts.first32).  The
// relative size of the correction right-hand side -- the Schur residual of
// the current iterate, evaluated from the FP64 residual -- is the stopping
// test, so tol has the meaning it has on the FP64 path.
constexpr int kMaxRefine = 8;
ahoc_status solve_mixed(ahoc_plan* p, const double* f, double* u, double tol) {
  const Geom& g = p->g;
  const int nb = g.nb;
  const int64_t n = g.ngamma;
  CK(cudaMemsetAsync(p->U64, 0, (size_t)nb * g.npad * sizeof(double), p->st));
  CK(cudaMemsetAsync(p->V64, 0, (size_t)nb * g.npad * sizeof(double), p->st));
  CK(cudaMemsetAsync(p->Q, 0, (size_t)nb * n * sizeof(double), p->st));
  std::vector<int> live = p->part;
  std::vector<double> bref(nb, 0.0), bn;
  const bool first64 = p->o.first64 && !p->o.varb;
  for (int step = 0; step <= kMaxRefine && any(live); ++step) {
    Phase ph("ahoc refinement step");
    CKS(set_act(p, live));
    if (step == 0 && first64) {
      // x = 0: the correction system is the whole system; its Schur
      // right-hand side -R(0) from the data by FP64 solves
      CKS(schur_rhs_dev(p, f, p->b2));
    } else {
      RUNN(AHOC_K_OTHER, 2,
           launch_residual(g, p->cf, p->Ru, p->Rv, p->Rq, p->U64, p->V64, p->Q, f, p->has_gD ? p->gD : nullptr,
                           p->has_vedge ? p->vedge : nullptr, p->has_gN ? p->gN : nullptr,
                           p->has_lapt ? p->lapt : nullptr, p->ainv, p->afac, p->st, p->has_gL ? p->gL : nullptr,
                           p->gam));
      // correction right-hand side b = -R_d(0)
      if (fused_ok(g)) {
        CKS(fused2d<float>(p, f2arrays_f(p), nullptr, p->Rv, p->Ru, p->Rq, p->b2, false));
      } else {
        CKS(solve_VU_f(p, nullptr, p->Rv, p->Ru));
        RUN(AHOC_K_TRACE, launch_trace<float>(g, p->cf, p->b2, p->F2, nullptr, p->afac, nullptr, nullptr, nullptr,
                                              p->st, p->Rq));
      }
      RUN(AHOC_K_KRYLOV, launch_axpby(p->b2, p->b2, -1.0, 0.0, n, p->st, nb, nullptr, g.act));
    }
    CKS(norms(p, p->b2, bn));
    std::vector<double> itol(nb, 0.0);
    std::vector<int> maxit(nb, 0);
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      ProbStat& s = p->ps[i];
      if (!is_fin(bn[i])) {  // NaN or Inf in this problem: it leaves the batch, the others refine on
        s.status = AHOC_ENUMERIC;
        live[i] = 0;
        continue;
      }
      if (step == 0) bref[i] = bn[i];
      s.rel = (bref[i] > 0) ? bn[i] / bref[i] : 0.0;
      s.hist[step] = s.rel;
      if (bn[i] == 0.0 || s.rel <= tol) {
        live[i] = 0;
        continue;
      }
      // Slow steps: the residual has reached the floor of its evaluation
      // (the FP32 recovery's rounding, amplified by L_h, or data whose Schur
      // right-hand side is tiny next to the solution, or a tol at that
      // floor).  A step that removed less than half of the residual while
      // the last correction changed U by at most tol (relative 2-norm): the
      // iterate is settled to the accuracy asked for, the solve has
      // converged.  A step that removed less than a tenth: if the
      // corrections still shrink (at least halve), the next step settles it
      // further; otherwise the FP32 solves are too inaccurate for this grid
      // and the solve has not converged.
      if (step >= 2 && s.rel > 0.5 * s.hist[step - 1] && s.du[step - 1] <= tol) {
        live[i] = 0;
        continue;
      }
      if (step >= 2 && s.rel > 0.9 * s.hist[step - 1]) {
        if (!(s.du[step - 1] < 0.5 * s.du[step - 2])) {
          s.status = AHOC_ENOCONV;
          live[i] = 0;
          continue;
        }
      }
      if (step == kMaxRefine) {
        s.status = AHOC_ENOCONV;
        live[i] = 0;
        continue;
      }
      // inner tolerance: refine_tol, but no tighter than the outer goal needs
      itol[i] = p->o.refine_tol;
      const double need = 0.5 * tol * bref[i] / bn[i];
      if (need > itol[i]) itol[i] = need;
      maxit[i] = p->o.max_iters - s.iters;
    }
    if (!any(live)) break;
    // the first correction is the whole solution: it starts from the nested
    // coarse-grid guess when the plan has coarse levels
    bool guess = false;
    if (step == 0 && p->coarse) CKS(coarse_guess(p, f, live, tol, p->dQ, p->b2, guess));
    std::vector<ProbStat> gi(nb);
    CKS(gmres(p, p->b2, bn, p->dQ, guess, itol, maxit, live, gi));
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      ProbStat& s = p->ps[i];
      s.iters += gi[i].iters;
      s.restarts += gi[i].restarts;
      s.ms_mv += gi[i].ms_mv;
      s.inner[step] = gi[i].iters;
      if (gi[i].status == AHOC_ENUMERIC) {
        s.status = AHOC_ENUMERIC;
        live[i] = 0;
      }
    }
    // recovery of the correction and the FP64 update
    CKS(set_act(p, live));
    const bool rec64 = (step == 0 && first64);
    if (rec64) {
      // the first correction is the whole solution (x = 0): V and U from it
      // by the FP64 solves.  An FP32 recovery here leaves rounding noise of
      // the size of U itself, which L_h amplifies in the next FP64 residual
      // and which then floors the next correction at about eps32 / h^2
      // (relative); the later corrections are small, so is their noise.
      CKS(solve_VU(p, p->dQ, f, true));
      RUN(AHOC_K_OTHER, launch_axpby(p->U64, p->W2, 1.0, 0.0, g.npad, p->st, nb, nullptr, g.act));
      RUN(AHOC_K_OTHER, launch_axpby(p->V64, p->W1, 1.0, 0.0, g.npad, p->st, nb, nullptr, g.act));
    } else {
      if (fused_ok(g))
        CKS(fused2d<float>(p, f2arrays_f(p), p->dQ, p->Rv, p->Ru, nullptr, nullptr, true));
      else
        CKS(solve_VU_f(p, p->dQ, p->Rv, p->Ru));
      RUNN(AHOC_K_OTHER, 2,
           launch_accumulate(g, p->U64, p->F2, p->V64, p->F1, p->partial, kDotBlocks, p->hdev, p->st));
    }
    RUN(AHOC_K_KRYLOV, launch_axpby(p->Q, p->dQ, 1.0, 1.0, n, p->st, nb, nullptr, g.act));
    if (!rec64) CKS(fetch(p));
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      ProbStat& s = p->ps[i];
      const double su = p->hhost[2 * i + 1], sdu = p->hhost[2 * i];
      s.du[step] = rec64 ? 1.0 : (su > 0 ? std::sqrt(sdu / su) : 0.0);
      ++s.refine_steps;
      if (s.iters >= p->o.max_iters) {
        s.status = AHOC_ENOCONV;
        live[i] = 0;
      }
    }
  }
  if (!u) return AHOC_OK;
  CKS(set_act(p, p->part));
  RUN(AHOC_K_OTHER, launch_write_full(g, u, p->U64, p->has_gD ? p->gD : nullptr, p->st));
  return AHOC_OK;
}

// One solve of the problems in p->part (statistics in p->ps); u == NULL: Q
// only (the nested guess's coarse levels), V and U are not recovered.
ahoc_status solve_internal(ahoc_plan* p, const double* f, double* u, double tol) {
  Phase ph(p->o.prec == AHOC_MIXED ? "ahoc solve (mixed)" : "ahoc solve (fp64)");
  p->have_last = false;
  CK(cudaStreamSynchronize(p->st));
  CKS(harvest(p));
  p->launches = 0;
  for (int k = 0; k < AHOC_NK; ++k) {
    p->kms[k] = 0;
    p->kn[k] = 0;
    p->kms_top[k] = 0;
    p->kn_top[k] = 0;
  }
  p->ps.assign(p->g.nb, ProbStat{});
  p->bicg_iters = 0;
  if (p->o.prec == AHOC_MIXED) CKS(solve_mixed(p, f, u, tol));
  else CKS(solve_fp64(p, f, u, tol));
  CK(cudaStreamSynchronize(p->st));
  CKS(harvest(p));
  p->have_last = true;
  return AHOC_OK;
}

}  // namespace

extern "C" {

// Algorithm 1, Main procedure (FP64, or FP32 inner solves with FP64 refinement).
ahoc_status ahoc_solve(ahoc_plan* p, const double* f, double* u, double tol, ahoc_info* info) {
  if (!p || !f || !u) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(f) || misaligned(u)) return fail(AHOC_EINVAL, kAlignMsg);
  if (!(tol > 0) || !std::isfinite(tol)) return fail(AHOC_EINVAL, "tol must be positive");
  const auto t0 = std::chrono::steady_clock::now();
  CKS(solve_internal(p, f, u, tol));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  ahoc_status st = AHOC_OK;
  for (int i = 0; i < p->g.nb; ++i) {
    if (!p->part[i]) continue;
    const ProbStat& s = p->ps[i];
    if (s.status != AHOC_OK && st != AHOC_ENUMERIC) st = s.status;
    if (!info) continue;
    ahoc_info* in = info + i;
    in->status = s.status;
    in->vsolve_iters = p->bicg_iters;
    in->iters = s.iters;
    in->restarts = s.restarts;
    in->rel_resid = s.rel;
    in->ms_total = ms;
    in->ms_matvec = s.ms_mv;
    in->launches = p->launches;
    in->levels = s.levels;
    in->coarse_iters = s.coarse_iters;
    in->refine_steps = s.refine_steps;
    for (int k = 0; k < 16; ++k) {
      in->refine_hist[k] = s.hist[k];
      in->refine_du[k] = s.du[k];
      in->inner_iters[k] = s.inner[k];
    }
    for (int k = 0; k < AHOC_NK; ++k) {
      in->kernel_ms[k] = p->kms[k];
      in->kernel_launches[k] = p->kn[k];
      in->kernel_ms_top[k] = p->kms[k] + p->kms_top[k];
      in->kernel_launches_top[k] = p->kn[k] + p->kn_top[k];
    }
  }
  if (st == AHOC_ENUMERIC)
    return fail(st, "NaN or Inf in a problem's data or iterates: that problem was masked out of the batch "
                    "(info[b].status), the others were solved");
  if (st != AHOC_OK) return fail(st, "GMRES reached max_iters (or refinement did not converge)");
  return AHOC_OK;
}

// ahoc_solve with the caller's initial Q: GMRES starts from q0 (FP64 plans).
ahoc_status ahoc_solve_from(ahoc_plan* p, const double* f, const double* q0, double* u, double tol,
                            ahoc_info* info) {
  if (!p || !f || !q0 || !u) return fail(AHOC_EINVAL, "NULL argument");
  if (misaligned(q0)) return fail(AHOC_EINVAL, kAlignMsg);
  if (p->o.prec != AHOC_FP64)
    return fail(AHOC_EUNSUPPORTED,
                "an initial Q is taken by FP64 plans (a mixed plan's first step solves for all of u)");
  p->q0 = q0;
  const ahoc_status s = ahoc_solve(p, f, u, tol, info);
  p->q0 = nullptr;
  return s;
}

// ahoc_solve with host arrays: f of every problem taking part is copied to a
// device staging grid, the solve runs as ahoc_solve, and u comes back, all on
// the plan's stream (one cudaMemcpyAsync per problem and direction).
ahoc_status ahoc_solve_host(ahoc_plan* p, const double* f, double* u, double tol, ahoc_info* info) {
  if (!p || !f || !u) return fail(AHOC_EINVAL, "NULL argument");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(AHOC_EINVAL, "tol must be positive");
  const size_t one = (size_t)p->g.nfull * sizeof(double);
  const size_t bytes = (size_t)p->g.nb * one;
  if (!p->hf || !p->hu) {
    std::lock_guard<std::recursive_mutex> lk(capture_mutex());
    if (!p->hf && cudaMalloc(&p->hf, bytes) != cudaSuccess) {
      cudaGetLastError();
      p->hf = nullptr;
      return fail(AHOC_ENOMEM, "cudaMalloc of the staging grid for f failed");
    }
    if (!p->hu && cudaMalloc(&p->hu, bytes) != cudaSuccess) {
      cudaGetLastError();
      p->hu = nullptr;
      return fail(AHOC_ENOMEM, "cudaMalloc of the staging grid for u failed");
    }
  }
  for (int b = 0; b < p->g.nb; ++b)
    if (p->part[b])
      CK(cudaMemcpyAsync((char*)p->hf + b * one, (const char*)f + b * one, one, cudaMemcpyHostToDevice, p->st));
  const ahoc_status s = ahoc_solve(p, p->hf, p->hu, tol, info);
  if (s != AHOC_OK && s != AHOC_ENOCONV) return s;
  for (int b = 0; b < p->g.nb; ++b)
    if (p->part[b])
      CK(cudaMemcpyAsync((char*)u + b * one, (const char*)p->hu + b * one, one, cudaMemcpyDeviceToHost, p->st));
  CK(cudaStreamSynchronize(p->st));
  return s;
}

}  // extern "C"
