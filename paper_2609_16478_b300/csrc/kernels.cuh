// Launchers of the device kernels (internal).
#pragma once

#include "common.cuh"

namespace ahoc {

template <typename T>
cudaError_t launch_dst_x(const Geom& g, T* a, const void* tw, const T* sn, T scale, cudaStream_t st);
template <typename T>
cudaError_t launch_dst_y(const Geom& g, T* a, const void* tw, const T* sn, T scale, cudaStream_t st);
template <typename T>
cudaError_t launch_dst_x_store_ainv(const Geom& g, T* a, const T* ainv, const void* tw, const T* sn,
                                    cudaStream_t st);
// dst = DST_x( M(W) + face terms qa = Q/alpha + src2 ), 2D; W = V/alpha, or V
// when ainv_load is given (then W = V * ainv on load); W must not alias dst;
// every array in precision T
template <typename T>
cudaError_t launch_dst_x_mload(const Geom& g, T* dst, const T* W, const T* qa, T Mc, T Mn, const void* tw,
                               const T* sn, cudaStream_t st, const T* src2 = nullptr, const T* ainv_load = nullptr);
// dst = DST_x(lscale * src)
template <typename T>
cudaError_t launch_dst_x_from(const Geom& g, T* dst, const T* src, double lscale, const void* tw, const T* sn,
                              cudaStream_t st);

// Generated right-hand side of the homogeneous v-equation in the x-spectral
// domain (2D): d(k, j) = sin(k pi/N0) (rxm_j + (-1)^(k+1) rxp_j)
//                        - b_k (Qh-_k [j = 1] + Qh+_k [j = N1-1]),  b_k = L_y + 2 cos(k pi/N0) L_xy
template <typename T>
struct VGen2D {
  const T* rxm;  // index j (1..N1-1)
  const T* rxp;
  const T* qhm;  // index k - 1
  const T* qhp;
  const T* sk;   // sin(k pi / N0), index k
  const T* ck;   // cos(k pi / N0), index k
  T Ly, Lxy;
};
// generated right-hand side; with `add` the generated terms are added to the
// right-hand side already in a (x-spectral), otherwise they replace it
// rpow: per chunk c and mode m, r^(1 + cL) at [c][m] and r^(2N - e_c) at [C + c][m]
template <typename T>
cudaError_t launch_tri_chunked_gen(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                                   const double* rpow, double* scratch, int L, const VGen2D<T>& G, cudaStream_t st,
                                   bool add = false);

// fused 2D matvec helpers (fused2d.cu)
// from the face values Q (FP64): rxm, rxp (boundary stencil on the first
// interior columns), qy (y-face data) and qa = Q/alpha (all faces), in T
template <typename T>
cudaError_t launch_v2d_prep(const Geom& g, const Coefs& cf, const double* Q, const double* afinv, T* rxm, T* rxp,
                            T* qy, T* qa, cudaStream_t st);
template <typename T>
cudaError_t launch_trace2d_x(const Geom& g, double* y, const T* Uh, const double* Q, const double* afac,
                             const T* tau, cudaStream_t st, const double* srcq = nullptr);
template <typename T>
cudaError_t launch_trace2d_ylines(const Geom& g, const Coefs& cf, T* R, const T* Uh, cudaStream_t st);
template <typename T>
cudaError_t launch_trace2d_y(const Geom& g, double* y, const T* R, const double* Q, const double* afac,
                             cudaStream_t st, const double* srcq = nullptr);
// chunk-start powers of r for the chunked tridiagonal solve (tri.cu)
cudaError_t launch_tri_powers(const Geom& g, const Mode<double>* md64, double* rpow, int L, cudaStream_t st);
size_t tri_powers_size(const Geom& g, int L);
cudaError_t launch_to_float(float* out, const double* in, int64_t n, cudaStream_t st);

// DST-I of generic strided lines (see dst.cu, k_dst_gen)
template <typename T>
// (nb problems: base + b * bstride for problem b; act masks problems out, may be NULL)
cudaError_t launch_dst_gen(T* base, int nlines, int lpg, int64_t gstride, int64_t lstride, int64_t estride, int N,
                           const void* tw, const T* sn, cudaStream_t st, int nb = 1, int64_t bstride = 0,
                           const int* act = nullptr);

// Boundary preconditioner on 2D face lines, one pass (dst.cu)
template <typename T>
// (out, in, afac of problem b at + b * bstride; pre is shared)
cudaError_t launch_precond_lines(double* out, const double* in, const double* afac, const double* pre, int nlines,
                                 int64_t lstride, int N, const void* tw, const T* sn, cudaStream_t st, int nb = 1,
                                 int64_t bstride = 0, const int* act = nullptr);

// Boundary preconditioner (precond.cu)
struct SymAxis {
  const double* stab;  // sin(j pi / N_a), j < 2 N_a
  const double* ctab;  // cos(k pi / N_b) per transverse axis b (indexed by axis)
};
cudaError_t launch_face_symbols(const Geom& g, const Coefs& cf, double* pre, const double* const* stab,
                                const double* const* ctab, cudaStream_t st);
// out[q] = in[q] * (mul ? mul[q] : 1) / (div ? div[q] : 1); nb problems of n
// entries each, mul and div advancing by mstride / dstride per problem (0: shared)
cudaError_t launch_face_muldiv(double* out, const double* in, const double* mul, const double* div, int64_t n,
                               cudaStream_t st, int nb = 1, int64_t mstride = 0, int64_t dstride = 0,
                               const int* act = nullptr);

// chunked tridiagonal solve (2D: few columns, many chunks per column)
// modes: the element-wise factors (precision T); md64: the FP64 factors used
// for the chunk carries; scratch: tri_chunked_scratch() doubles
template <typename T>
cudaError_t launch_tri_chunked(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                               const double* rpow, double* scratch, int L, cudaStream_t st);
size_t tri_chunked_scratch(const Geom& g, int L);
// FP64 chunked solve in two passes over the field with exact tables (tri.cu):
// tab holds tri2_table_size() doubles from tri2_table_fill (roots r[m] in
// long double, mode order of the Mode tables); G (2D) generates the
// v-equation right-hand side, added to the field when `add`
size_t tri2_table_size(const Geom& g, int L);
void tri2_table_fill(const Geom& g, int L, const long double* r, double* out);
cudaError_t launch_tri2(const Geom& g, double* a, const Mode<double>* modes, const double* tab, double* scratch,
                        int L, cudaStream_t st, const VGen2D<double>* G = nullptr, bool add = false);

template <typename T>
cudaError_t launch_tri(const Geom& g, T* a, const Mode<T>* modes, cudaStream_t st);

// Generated right-hand side of the homogeneous v-equation in the (x, y)-mode
// domain (3D), for mode column (kx, ky) and row k of the solve along z:
//   d = sx[kx] Ax(ky, k) + sy[ky] By(kx, k) + [k = 1] Zm(kx, ky) + [k = N2-1] Zp(kx, ky)
// Ax: the x-face sum (odd kx) or difference (even kx) slot of `gen`, By the
// same for y, Zm / Zp the z-face slots (face layout; fused3d.cu, v3d_prep).
template <typename T>
struct VGen3D {
  const T* gen;  // face layout, problems ngamma apart
  const T* sx;   // sin(k pi / N0), index k
  const T* sy;   // sin(k pi / N1), index k
};
// the one-thread-per-column solve with the right-hand side generated from G
template <typename T>
cudaError_t launch_tri_gen3(const Geom& g, T* a, const Mode<T>* modes, const VGen3D<T>& G, cudaStream_t st);
// the chunked solve (FP64 carries) with the right-hand side generated from G
template <typename T>
cudaError_t launch_tri_chunked_gen3(const Geom& g, T* a, const Mode<T>* modes, const Mode<double>* md64,
                                    const double* rpow, double* scratch, int L, const VGen3D<T>& G,
                                    cudaStream_t st);

// fused 3D matvec helpers (fused3d.cu)
template <typename T>
cudaError_t launch_v3d_prep(const Geom& g, const Coefs& cf, const double* Q, const double* afinv, T* gen, T* qa,
                            cudaStream_t st);
// Tr (face layout, in-face modes) from U-hat; the in-face inverse DSTs follow
template <typename T>
cudaError_t launch_trace3d(const Geom& g, const Coefs& cf, const T* Uh, const T* taux, const T* tauy, double* Tr,
                           cudaStream_t st);
cudaError_t launch_trace3d_fin(const Geom& g, double* y, const double* Tr, const double* Q, const double* afac,
                               const double* srcq, cudaStream_t st);
bool trace3d_red_ok(const Geom& g);
// dst = DST_x( M(W) + face terms qa + src2 ), 3D (seven-point M); W must not alias dst
template <typename T>
cudaError_t launch_dst_x_mload3d(const Geom& g, T* dst, const T* W, const T* qa, T Mc, T Mn, const void* tw,
                                 const T* sn, cudaStream_t st, const T* src2 = nullptr);

// V-equation right-hand side for (L_h - gam M) V_int = rhs:
//   rhs = -M f - (L - gam M)_bdry(V_b),  V_b = Q on face points, v_edge on edges/corners.
template <typename T>
cudaError_t launch_vrhs(const Geom& g, const Coefs& cf, T* out, const double* Q, const double* f,
                        const double* vedge, cudaStream_t st, const T* srcv = nullptr,
                        const double* gam = nullptr);
// u-equation right-hand side for L_h U_int = rhs:
//   rhs = M(V / alpha) - L_bdry(g_D),  V = Q on face points (M reaches no edges);
//   ainv = 1/alpha on the full grid, in T.
template <typename T>
cudaError_t launch_urhs(const Geom& g, const Coefs& cf, T* out, const T* V, const T* ainv, const double* Q,
                        const double* gD, cudaStream_t st, const T* srcu = nullptr);
// Boundary residual R_p = alpha_p [u_nn(U)_p + lapt_p] - Q_p at every point of a
// clamped face, R_p = alpha_p g_L,p - Q_p on a Navier face (minus srcq if given).
template <typename T>
cudaError_t launch_trace(const Geom& g, const Coefs& cf, double* y, const T* U, const double* Q,
                         const double* afac, const double* gD, const double* gN, const double* lapt,
                         cudaStream_t st, const double* srcq = nullptr, const double* gL = nullptr);

// Triharmonic class (Lap^3 u = f): R_p = u_ssss(U)_p + lapt_w_p - Q_p on clamped
// faces (one-sided u_ssss with g_D, g_N, g_NN), bilap_p - Q_p on the others
cudaError_t launch_trace_tri(const Geom& g, const Coefs& cf, double* y, const double* U, const double* Q,
                             const double* gD, const double* gN, const double* gNN, const double* laptw,
                             const double* bilap, cudaStream_t st);
// mixed precision: FP64 residual of the coupled system (r_u, r_v in FP32, r_q in FP64)
cudaError_t launch_residual(const Geom& g, const Coefs& cf, float* ru, float* rv, double* rq, const double* U,
                            const double* V, const double* Q, const double* f, const double* gD, const double* vedge,
                            const double* gN, const double* lapt, const double* ainv, const double* afac,
                            cudaStream_t st, const double* gL = nullptr, const double* gam = nullptr);
// variable beta/alpha (gam on the full grid): y = L_h x - M(gam x) on interior
// points, x = 0 on the boundary (stencil.cu)
cudaError_t launch_vop(const Geom& g, const Coefs& cf, double* y, const double* x, const double* gam,
                       cudaStream_t st);
// y = c[3b] x0 + c[3b+1] x1 + c[3b+2] x2 per problem b of g.nb (n entries each;
// x1, x2 may be NULL; c on the device, 3 g.nb entries); masked by g.act
cudaError_t launch_comb(const Geom& g, int64_t n, double* y, const double* x0, const double* x1, const double* x2,
                        const double* c, cudaStream_t st);
// out = a * b elementwise
cudaError_t launch_mul(double* out, const double* a, const double* b, int64_t n, cudaStream_t st);
// U += dU, V += dV; for problem b, out[2b] = sum dU^2 and out[2b + 1] = sum U^2
// after the update (deterministic: nblocks fixed partials per problem in
// `partial`, 2 * nb * nblocks doubles)
cudaError_t launch_accumulate(const Geom& g, double* U, const float* dU, double* V, const float* dV,
                              double* partial, int nblocks, double* out, cudaStream_t st);

cudaError_t launch_write_full(const Geom& g, double* out, const double* Uin, const double* bnd, cudaStream_t st);
cudaError_t launch_pack(const Geom& g, double* dense, const double* padded, cudaStream_t st);
cudaError_t launch_unpack(const Geom& g, double* padded, const double* dense, cudaStream_t st);
cudaError_t launch_face_gather(const Geom& g, double* face, const double* full, cudaStream_t st);
// per block b: out[3b] = min, out[3b+1] = max, out[3b+2] = sum of beta/alpha over n points
cudaError_t launch_ratio_stats(const double* beta, const double* alpha, int64_t n, double* out, int blocks,
                               cudaStream_t st);
// out = a / in (in == NULL: out = a)
cudaError_t launch_scaled_recip(double* out, const double* in, double a, int64_t n, cudaStream_t st);
// out = 1 / in (in == NULL: out = 1)
cudaError_t launch_recip(double* out, const double* in, int64_t n, cudaStream_t st);
cudaError_t launch_v_full(const Geom& g, double* vfull, const double* Vpad, const double* Q, const double* vedge,
                          cudaStream_t st);

// grid transfer for the nested initial guess (stencil.cu)
cudaError_t launch_inject_full(const Geom& gc, const Geom& gf, double* out, const double* in, cudaStream_t st);
cudaError_t launch_inject_face(const Geom& gc, const Geom& gf, double* out, const double* in, cudaStream_t st);
cudaError_t launch_face_prolong(const Geom& gf, const Geom& gc, double* out, const double* in, cudaStream_t st);

// GMRES level-1/2 kernels on face vectors (FP64), over a batch of nbat
// problems: problem b's V, w and partials start at b * vstride, wstride,
// pstride; act masks problems out (NULL: all).
struct BatchDot {
  int64_t vstride = 0, wstride = 0, pstride = 0;
  const int* act = nullptr;
};
// out[c] = <V_c, w>, c < ncols (deterministic two-stage reduction through
// `partial`, which holds nblocks * ncols doubles per problem); problem b's
// results at out + b * ostride
// One fused CGS pass (blas.cu, k_cgs): dst = src - V h over nh columns when
// h is set (dst must not alias src), then out[c] = <V_c, dst> for c < ncols
// (self: out[0] = <dst, dst>; without h the dots take src) in one launch,
// with the block split, order and bits of launch_gemv_sub + launch_mdot.
// cnt: zeroed ints, one per (problem, group of 4 columns), left zeroed.
cudaError_t launch_cgs(const double* V, int64_t ld, int ncols, const double* h, int nh, const double* src,
                       double* dst, int64_t n, double* partial, int nblocks, double* out, cudaStream_t st, int nbat,
                       const BatchDot& bd, int64_t hstride, int64_t ostride, int* cnt, bool self);
cudaError_t launch_mdot(const double* V, int64_t ld, int ncols, const double* w, int64_t n, double* partial,
                        int nblocks, double* out, cudaStream_t st, int nbat = 1, const BatchDot& bd = BatchDot{},
                        int64_t ostride = 0);
// out[c] = sum_b partial[b * ncols + c] in block order
cudaError_t launch_reduce_cols(const double* partial, int nblocks, int ncols, double* out, cudaStream_t st);
// w -= V h (h on device, ncols entries; problem b's h at + b * hstride and,
// when ncols_b is set, ncols_b[b] columns)
cudaError_t launch_gemv_sub(const double* V, int64_t ld, int ncols, const double* h, double* w, int64_t n,
                            cudaStream_t st, int nbat = 1, const BatchDot& bd = BatchDot{}, int64_t hstride = 0,
                            const int* ncols_b = nullptr);
// y = a * x + b * y (b == 0: y = a * x); nbat problems of n entries, problem
// b's y and x at + b * ystride, xstride (-1: n), a taken from a_b[b] when set
cudaError_t launch_axpby(double* y, const double* x, double a, double b, int64_t n, cudaStream_t st, int nbat = 1,
                         const double* a_b = nullptr, const int* act = nullptr, int64_t ystride = -1,
                         int64_t xstride = -1);

// GMRES's Hessenberg QR on the device (blas.cu): per-problem state of
// givens_doubles(m) doubles and kGivensInts ints (iters, maxit, status, jend,
// cyc); status codes as ahoc_status (0 ok, kGivensNoConv, kGivensNumeric)
constexpr int kGivensInts = 5;
constexpr int kGivensNoConv = 4;   // AHOC_ENOCONV
constexpr int kGivensNumeric = 5;  // AHOC_ENUMERIC
__host__ __device__ inline int64_t givens_doubles(int m) { return (int64_t)(m + 1) * m + 2 * m + (m + 1) + 3; }
cudaError_t launch_givens_init(int nb, int m, const int* act, const double* ini, const int* ii, double* gs, int* gi,
                               double* rel, cudaStream_t st);
cudaError_t launch_givens_step(int j, int nb, int m, const double* hdev, int hs, int* act, double* scal, double* gs,
                               int* gi, double* rel, cudaStream_t st);
cudaError_t launch_givens_solve(int nb, int m, const double* gs, const int* gi, double* hy, int hs, int* ncols,
                                cudaStream_t st);

}  // namespace ahoc
