/*
 * ahoc.h -- C ABI of the matrix-free augmented high-order compact (HOC)
 * solver for clamped, variable-coefficient biharmonic problems
 *
 *     -Laplace(alpha * Laplace u) = f        in a box (d = 2, 3)       (Sec. 2, Eq. 1, beta = 0)
 *     u = g_D on the boundary,  u_n = g_N on every face                 (Eq. 2, fully clamped)
 *
 * discretised by the compact fourth-order scheme of Sec. 2.2 (mixed form
 * v = alpha Laplace u, 9-point / 19-point L_h, weighting M, one-sided second
 * normal derivative with the augmented unknowns Q = v on the face interiors),
 * and solved by the Schur-complement method of Sec. 2.3: GMRES on S_h Q = b
 * with the matrix-free action S_h Q = R(Q) - R(0), b = -R(0) of Lemma 1, each
 * action running two Dirichlet HOC Poisson solves (Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      N[a] intervals along axis a (x = 0, y = 1, z = 2), N[a] a power of
 *           two with 8 <= N[a] <= 4096, spacing h_a = (hi[a] - lo[a]) / N[a].
 * Full grid arrays hold (N[0]+1) x ... x (N[d-1]+1) doubles, x fastest.
 * Interior arrays hold (N[0]-1) x ... x (N[d-1]-1) doubles, x fastest.
 * Face arrays (g_N, lapt_gD, Q, y) hold the relative-interior points of the
 *           faces in the order x-, x+, y-, y+, z-, z+; within a face the
 *           remaining axes keep their order, lowest axis fastest.  Their
 *           length is n_gamma = sum over faces of prod_{b != a} (N[b] - 1).
 * Memory    every array pointer is DEVICE memory owned by the caller unless
 *           stated otherwise; the library never frees caller memory.  A
 *           device array of doubles must be 8-byte aligned (AHOC_EINVAL
 *           otherwise, before any launch).
 * Streams   all work is enqueued on the plan's CUDA stream; calls return
 *           once the work is enqueued, except where stated.
 * Errors    every call returns an ahoc_status; no call aborts, throws or
 *           prints.  ahoc_last_error() gives a one-line description of the
 *           most recent failure on the calling thread.
 */
#ifndef AHOC_H
#define AHOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AHOC_OK = 0,
  AHOC_EINVAL = 1,        /* bad argument (checked before any allocation or launch) */
  AHOC_ENOMEM = 2,        /* device allocation failed, or caller workspace too small */
  AHOC_ECUDA = 3,         /* a CUDA runtime call failed */
  AHOC_ENOCONV = 4,       /* GMRES reached max_iters; outputs hold the best iterate */
  AHOC_ENUMERIC = 5,      /* NaN or Inf met in a residual norm */
  AHOC_ETIMEOUT = 6,      /* reserved: a bounded device wait ran out */
  AHOC_EUNSUPPORTED = 7,  /* valid request outside what the library supports */
  AHOC_EINTERNAL = 8
} ahoc_status;

typedef enum { AHOC_FP64 = 0, AHOC_MIXED = 1 } ahoc_precision;

/* Kernel classes reported by ahoc_info when opts.timing is set. */
enum {
  AHOC_K_DST_X = 0,   /* DST-I along x (Sec. 2.3 fast solver)            */
  AHOC_K_DST_Y = 1,   /* DST-I along y (3D)                              */
  AHOC_K_TRI = 2,     /* tridiagonal solve along the last axis           */
  AHOC_K_VRHS = 3,    /* v-equation right-hand side                      */
  AHOC_K_URHS = 4,    /* u-equation right-hand side M(V/alpha)           */
  AHOC_K_TRACE = 5,   /* boundary residual R (Lemma 1)                   */
  AHOC_K_KRYLOV = 6,  /* GMRES dot products, updates                     */
  AHOC_K_OTHER = 7,   /* layout conversion, output                       */
  AHOC_NK = 8
};

typedef struct ahoc_plan ahoc_plan;  /* opaque; created and owned by the library */

/* Boundary data (Sec. 2, Eq. 2; Lemma 1).  Device pointers, NULL = zero.
 * They are copied into the plan at creation; the caller may free them after. */
typedef struct {
  const double* g_D;     /* full grid; only boundary entries are read: u on the boundary        */
  const double* g_N;     /* face array: outward normal derivative of u on the face interiors     */
  const double* lapt_gD; /* face array: sum of the tangential second derivatives of g_D          */
  const double* v_edge;  /* full grid; only edge and corner entries are read: alpha * Laplace u,
                            known there from g_D by tangential differentiation (Remark, Sec. 2.2) */
  const double* g_L;     /* face array: Laplace u on the face interiors; read on Navier faces
                            only (opts.navier), where v = alpha g_L is data (Eq. 2)              */
  const double* beta;    /* full grid: beta of Eq. 1, read when opts.variable_beta is set        */
  /* triharmonic class only (opts.triharmonic; the paper's triharmonic extension, Sec. 4.2): */
  const double* lap_gD;  /* full grid; boundary entries read: Laplace u on the whole boundary    */
  const double* bilap;   /* full grid; boundary entries read: Laplace^2 u on the simply
                            supported faces and on every edge and corner                        */
  const double* g_NN;    /* face array: second normal derivative of u on the clamped faces      */
  const double* lapt_w;  /* face array: 2 Lap_t u_nn + Lap_t^2 u on the clamped faces, Lap_t the
                            sum of the tangential second derivatives                            */
} ahoc_bdata;

/* Options; a NULL pointer selects the defaults given in brackets. */
typedef struct {
  ahoc_precision prec;    /* [AHOC_FP64] arithmetic of the Poisson solves.  AHOC_MIXED: FP32
                             inner solves (DST, tridiagonal, stencils) inside FP64 iterative
                             refinement of the coupled system (FP64 residual of all three
                             block rows, FP64 GMRES vectors, Hessenberg and updates); the
                             stopping test is the same relative Schur residual, evaluated
                             from the FP64 residual of the iterate.  When a step removes
                             less than a tenth of it (limiting accuracy), the solve has
                             converged if the last correction changed U by at most tol
                             (relative 2-norm; rel_resid may then exceed tol), refines on
                             while the corrections at least halve, and returns AHOC_ENOCONV
                             otherwise.  In a MIXED plan ahoc_matvec runs the FP32 inner
                             solves.                                                           */
  int max_iters;          /* [500] total GMRES iterations allowed                               */
  int restart;            /* [100] Krylov basis size before a restart (the paper's GMRES is not
                             restarted; the cap only bounds memory)                            */
  int precond;            /* [1] 1: right-precondition GMRES with the boundary-symbol operator
                             (inverse single-face Schur symbol per face, coefficient frozen
                             pointwise on the face); 0: no preconditioner                    */
  double refine_tol;      /* [3e-6] AHOC_MIXED: relative residual each FP32 correction GMRES
                             aims for (<= 0 selects the default)                               */
  int timing;             /* [0] nonzero: time every kernel launch of ahoc_solve with CUDA
                             events on the plan's stream (ahoc_info.kernel_ms)               */
  void* workspace;        /* [NULL] caller-owned device workspace of at least
                             ahoc_workspace_bytes() bytes, 256-byte aligned; NULL lets the
                             plan allocate its own with cudaMalloc                             */
  size_t workspace_bytes; /* size of the caller workspace                                      */
  int levels;             /* [-1] coarse levels of the nested initial guess: the problem is
                             solved on grids with N/2, N/4, ... (data injected), each
                             solution's Q interpolated (cubic, along the faces) to the next
                             finer grid as GMRES's initial guess (the coarse-grid
                             interpolated guess of Sec. 4.1).  -1: automatic (halve while
                             every axis keeps >= 512 intervals in 2D, >= 128 in 3D, at most
                             3 levels, and use a
                             coarse level for a problem only where it resolves the data: its
                             Schur right-hand side, interpolated to the finer faces, within
                             10% of the finer one's, which costs nothing more as the coarse
                             solve starts from it; off in an AHOC_MIXED plan, where it only
                             starts the first correction solve); 0: off.  In an AHOC_MIXED
                             plan the coarse levels are mixed-precision solves too           */
  double coarse_tol;      /* [0] relative Schur residual the coarse levels of the nested guess
                             solve to (never tighter than the solve's tol).  The prolonged
                             guess is only as good as the coarse grid's discretisation and
                             the interpolation, so a coarse solve past that is wasted.
                             <= 0: automatic (AHOC_COARSE_TOL_AUTO, or
                             AHOC_COARSE_TOL_AUTO_MIXED in an AHOC_MIXED plan, whose first
                             FP32 correction only needs the guess to refine_tol)             */
  int batch;              /* [1] problems of this shape held by the plan and solved together:
                             every launch covers all of them (one grid dimension per problem),
                             GMRES runs in lockstep and a problem that has converged is masked
                             out of later launches, so each result is the one a single-problem
                             plan gives.  Per-problem arguments (alpha, data, f, u, q, y, b)
                             hold `batch` arrays of their single-problem size back to back.  */
  int navier;             /* [0] problem class: bit 2a + side set makes face (axis a, side) a
                             Navier face (Eq. 2, Laplace u = g_L, so v = alpha g_L is data and
                             the face carries no augmented unknown: its rows of the Schur
                             system are -I, right-hand side -alpha g_L); other faces clamped */
  double shift;           /* [0] problem class: the constant ratio gamma = beta / alpha of the
                             beta term of Eq. 1.  The v-equation is -L_h V + gamma M V = M f
                             (Sec. 2.2 with beta / alpha constant, e.g. constant alpha and
                             beta): its Poisson solves take the shifted eigenvalues
                             -lambda_L + gamma lambda_M.  gamma >= 0 (a negative gamma, the
                             indefinite Helmholtz v-equation of the high-wavenumber problem
                             of Sec. 4.2, gives AHOC_EUNSUPPORTED); with variable_beta set,
                             the reference shift of the iterative v-solve                      */
  int no_graphs;          /* [0] 0: each GMRES iteration (mask and scalar uploads, the
                             normalisation of v_j, the preconditioner, the Schur matvec, CGS2
                             and the read-back of the Hessenberg column) is captured once as a
                             CUDA graph per iteration index and replayed on a stream the plan
                             owns, ordered after and before the caller's stream by events (no
                             graphs with timing != 0; a capture that another thread's CUDA
                             call invalidates leaves the plan on plain launches).  nonzero:
                             plain launches.                                                   */
  int variable_beta;      /* [0] problem class: nonzero makes beta / alpha variable, with beta
                             from each problem's bd->beta.  FP64: every v-solve is a
                             right-preconditioned BiCGSTAB on (L_h - M(beta/alpha .)) V = rhs,
                             preconditioned by (and started from) the FFT solve with the
                             constant shift opts.shift (a representative beta/alpha), as in the
                             paper's solver settings (Sec. 4); no CUDA graphs.  MIXED: the FP32
                             corrections use the constant shift and the FP64 residual the
                             exact beta/alpha, so the refinement converges to the same
                             discrete solution                                                 */
  int uhat_slots;         /* [0] 2D FP64 with constant beta / alpha: the Schur matvecs of
                             GMRES's first cycle leave U in x-modes (U-hat, the transform
                             along x of the u-solve) in a field each, and U and V of the data
                             alone are kept, so that the recovery of U is one combination of
                             those fields (Q = Q0 + Z y is linear) and one inverse DST instead
                             of two Poisson solves; V is then formed only when
                             ahoc_last_qv asks for it.  Falls back to the two solves when
                             GMRES restarts or takes more steps than slots.  0: automatic
                             (min(restart, 16) slots); > 0: that many (at most restart);
                             < 0: none.  Each slot holds one field per problem (workspace).  */
  int unfused;            /* [0] 3D FP64 with constant beta / alpha: 0 runs the Schur matvec in
                             four full DST passes (the v-equation's right-hand side generated
                             in the transverse modes inside the solve along z, V/alpha stored
                             by the last inverse DST, M(V/alpha) fused into the u-solve's first
                             DST, the traces taken from U-hat); nonzero: the plain form, two
                             full Poisson solves (eight DST passes) and the trace of physical
                             U.  Both give the same discrete action.                           */
  int triharmonic;        /* [0] problem class: nonzero solves Laplace^3 u = f (the paper's
                             triharmonic extension, Sec. 4.2, Table 5) in the mixed form
                             Laplace u = v, Laplace v = w, Laplace w = f, each discretised
                             with the compact scheme (L_h X = M(Laplace x)); the augmented
                             unknowns Q are w = Laplace^2 u on the faces.  The faces in
                             opts.navier are simply supported (u, Laplace u, Laplace^2 u
                             given: their Schur rows are -I, right-hand side -bilap), the
                             others clamped (u, u_n, u_nn given; the augmented equation is
                             Laplace^2 u = u_ssss + 2 Lap_t u_nn + Lap_t^2 u with u_ssss
                             one-sided from U_0 = g_D, U_1..U_4, u_s = -g_N and u_nn = g_NN,
                             exact for polynomials of degree 6 in s).  Each Schur action
                             runs three Poisson solves.  FP64 only, alpha = 1 (alpha may be
                             NULL), no beta, no preconditioner, no nested guess; f is the
                             right-hand side of Laplace^3 u = f; ahoc_last_qv returns Q
                             only.                                                             */
  int auto_shift;         /* [0] nonzero: ahoc_plan_create derives the beta class of Eq. 1 from
                             the data instead of opts.shift / opts.variable_beta: with
                             gamma = beta / alpha over every point of every problem
                             (bd->beta; none: beta = 0), one value everywhere gives the
                             constant shift gamma, several give variable beta with the mean
                             of gamma as the reference shift (gamma < 0 anywhere:
                             AHOC_EUNSUPPORTED, as for opts.shift).  Uses a few KB of temporary
                             device memory (cudaMalloc) and synchronises the stream; with it,
                             ahoc_workspace_bytes sizes for the variable-beta class.          */
  int first32;            /* [0] AHOC_MIXED: 0 takes the first correction (the whole solution)
                             with its Schur right-hand side from the data and its recovery of
                             V and U by FP64 solves (four FP64 Poisson solves), only its GMRES
                             in FP32: an FP32 right-hand side or recovery of the whole
                             solution carries rounding amplified by L_h (about eps32 / h^2
                             relative), which stalls the first steps on high-wavenumber data
                             and fine grids.  Nonzero keeps them in FP32 like the later
                             corrections.  Variable-beta plans always do                      */
} ahoc_opts;

/* automatic coarse-level tolerance of the nested initial guess (FP64 and
   mixed-precision plans) */
#define AHOC_COARSE_TOL_AUTO 3e-11
#define AHOC_COARSE_TOL_AUTO_MIXED 1e-8

typedef struct {
  int iters;              /* GMRES iterations (matrix-vector products) of the last solve        */
  int restarts;
  double rel_resid;       /* ||b - S_h Q|| / ||b|| estimated by GMRES at exit                   */
  double ms_total;        /* wall time of the last ahoc_solve, host clock                       */
  double ms_matvec;       /* device time of the Arnoldi steps (preconditioner, matvec, CGS2)   */
  int64_t launches;       /* kernels this library launched during the last solve                */
  double kernel_ms[AHOC_NK];      /* with opts.timing: summed device time per kernel class      */
  int64_t kernel_launches[AHOC_NK];
  int levels;             /* coarse levels this problem's initial guess used                    */
  int coarse_iters;       /* GMRES iterations summed over the coarse levels                     */
  double kernel_ms_top[AHOC_NK];      /* as kernel_ms, this grid's launches only (no coarse)  */
  int64_t kernel_launches_top[AHOC_NK];
  int refine_steps;       /* AHOC_MIXED: FP32 correction solves taken                           */
  double refine_hist[16]; /* AHOC_MIXED: relative Schur residual before each correction, then at exit */
  int inner_iters[16];    /* AHOC_MIXED: GMRES iterations of each correction solve              */
  double refine_du[16];   /* AHOC_MIXED: ||dU||_2 / ||U||_2 of each correction (U after it)    */
  ahoc_status status;     /* this problem's outcome (AHOC_OK, AHOC_ENOCONV or AHOC_ENUMERIC)    */
  int vsolve_iters;       /* opts.variable_beta, FP64: BiCGSTAB iterations over all v-solves   */
} ahoc_info;

/* Bytes of device workspace a plan of this shape needs (Sec. 2.3, Algorithm 1:
 * two interior fields, coefficient and boundary copies, the Krylov basis;
 * plus the coarse levels of the nested initial guess).
 * Returns AHOC_EINVAL on a bad shape.  Allocates nothing. */
ahoc_status ahoc_workspace_bytes(int dim, const int64_t* N, const ahoc_opts* opts, size_t* bytes);

/* Create a plan (Sec. 2.2 discretisation on the box [lo, hi]).
 *   dim      2 or 3;  N, lo, hi: host arrays of length dim, lo[a] < hi[a]
 *   alpha    device, full grid, alpha > 0 (not checked on the device);
 *            opts->batch grids back to back for a batched plan
 *   bd       host struct of device pointers (NULL = homogeneous data); each
 *            array holds opts->batch copies back to back
 *   opts     host struct (NULL = defaults)
 *   stream   a cudaStream_t (NULL = the legacy default stream)
 * Precomputes the DST twiddle tables, the per-mode tridiagonal factors of
 * L_h along the last axis, 1/alpha and the boundary data copies.  Arguments
 * are checked before any allocation.  On success *out owns the plan. */
ahoc_status ahoc_plan_create(ahoc_plan** out, int dim, const int64_t* N, const double* lo,
                             const double* hi, const double* alpha, const ahoc_bdata* bd,
                             const ahoc_opts* opts, void* stream);

/* Solve the discrete problem (Algorithm 1, Main procedure):
 *   b = -R(0) (ConstructSchurRHS), GMRES on S_h Q = b to relative residual
 *   tol, then V and U by two Poisson solves with the converged Q.
 *   f     device, full grid (boundary entries are used by M near the boundary)
 *   u     device, full grid output; boundary entries = g_D
 *   tol   relative residual of the Schur system, > 0
 *   info  host, may be NULL; a batched plan fills info[b] for every problem b
 *         taking part (see ahoc_set_active)
 * A batched plan solves the problems taking part; f and u hold one grid per
 * problem of the plan (the others are neither read nor written).
 * Synchronises the plan's stream (it reads residual norms) and returns when
 * u is written.  AHOC_ENOCONV: u holds the solution for the best iterate.
 * A problem whose data or iterates turn NaN or Inf is masked out of the
 * batch with info[b].status = AHOC_ENUMERIC (its u is not meaningful); the
 * other problems are solved as if it were absent, and the call returns
 * AHOC_ENUMERIC. */
ahoc_status ahoc_solve(ahoc_plan* p, const double* f, double* u, double tol, ahoc_info* info);

/* ahoc_solve with HOST arrays (Algorithm 1, Main procedure, as ahoc_solve):
 * f of every problem taking part is copied to the device, the problem is
 * solved, and u is copied back, all on the plan's stream.
 *   f_host  host, opts.batch full grids back to back (read for the problems
 *           taking part); page-locked memory gives the fastest copies,
 *           pageable memory works
 *   u_host  host, same size, output (boundary entries = g_D)
 * The first call allocates two device staging arrays of opts.batch full
 * grids each with cudaMalloc (freed by ahoc_plan_destroy; AHOC_ENOMEM if that
 * fails).  Returns when u_host is written; otherwise as ahoc_solve. */
ahoc_status ahoc_solve_host(ahoc_plan* p, const double* f_host, double* u_host, double tol, ahoc_info* info);

/* ahoc_solve with the caller's initial Q (the boundary values of v on the
 * face interiors, the unknowns of S_h Q = b, Lemma 1): GMRES starts from q0
 * instead of zero or the nested coarse-grid guess (Algorithm 1 with a warm
 * start, as Sec. 4.1 starts from an interpolated coarse solution); the
 * converged Q of an earlier solve of nearby data (ahoc_last_qv) is the
 * typical q0.  The result is the same discrete solution to within tol.
 *   q0  device, one face array (n_gamma doubles, the face order of ahoc_bdata)
 *       per problem of the plan, back to back (all of it is read; the
 *       entries of problems not taking part are not used).  A problem whose
 *       Schur right-hand side is zero ignores it
 *       (its Q is 0).  A NaN or Inf in a problem's q0 fails that problem alone
 *       (AHOC_ENUMERIC, as ahoc_solve).
 * FP64 plans only (a mixed plan's first refinement step solves for the whole
 * solution: AHOC_EUNSUPPORTED).  Otherwise as ahoc_solve. */
ahoc_status ahoc_solve_from(ahoc_plan* p, const double* f, const double* q0, double* u, double tol,
                            ahoc_info* info);

/* y = S_h q = R(q) - R(0) (Lemma 1; Algorithm 1, SchurMatVec), the
 * homogeneous part of the boundary residual: V(q) by the v-equation with
 * zero f and edge data, U(V) by the u-equation with zero g_D, then
 * y_p = alpha_p * delta_nn U_p - q_p with the one-sided formula of Sec. 2.2.
 * q, y: device face arrays (n_gamma); may not alias. */
ahoc_status ahoc_matvec(ahoc_plan* p, const double* q, double* y);

/* b = -R(0) (Lemma 1; Algorithm 1, ConstructSchurRHS) for right-hand side f
 * (device, full grid); b: device face array. */
ahoc_status ahoc_schur_rhs(ahoc_plan* p, const double* f, double* b);

/* Copy the augmented unknowns Q (v = alpha Laplace u on the face interiors,
 * Sec. 2.2; the solution of S_h Q = b, Lemma 1) of the last successful
 * ahoc_solve into q (device face array), and, if v is not NULL, V on the
 * full grid (faces = Q, edges and corners = v_edge) into v.  Caller-owned
 * outputs, one per problem of the plan.  AHOC_EINVAL before any solve. */
ahoc_status ahoc_last_qv(ahoc_plan* p, double* q, double* v);

/* Component entry points (the building blocks of SchurMatVec) ------------- */

/* DST-I along axis (0 <= axis < dim - 1) of an interior array:
 * out_k = scale * sum_{j=1}^{N-1} in_j sin(pi j k / N), all other indices
 * fixed (the sine expansion of Lemma 4).  in, out: device interior arrays;
 * they may alias. */
ahoc_status ahoc_dst1(ahoc_plan* p, int axis, const double* in, double* out, double scale);

/* Dirichlet HOC Poisson solve (the FFT-based solver of Algorithm 1):
 * L_h w = rhs at interior points, w = 0 on the boundary.  rhs, w: device
 * interior arrays; they may alias. */
ahoc_status ahoc_poisson(ahoc_plan* p, const double* rhs, double* w);

/* Dirichlet HOC Poisson solve without a plan and without any device
 * allocation (the paper has no counterpart: this is a deployment aid).
 * It computes the same result as ahoc_poisson on a plan of this grid,
 * L_h w = rhs at interior points with w = 0 on the boundary, for callers
 * that cannot call cudaMalloc: code running under another component's
 * memory pool, latency-critical loops where an allocation would
 * synchronise the device, or hosts that forbid allocation after start-up.
 *   dim, N, lo, hi  as for ahoc_plan_create (host arrays)
 *   rhs, w          device interior arrays (caller-owned); may alias
 *   stream          a cudaStream_t of the current device (NULL = legacy default)
 * All scratch (the padded field, the DST and per-mode tables, the carries
 * of the chunked tridiagonal solve) lives in one static device array of
 * 16 MiB that every GPU loading this library holds until the process exits;
 * grids needing more (e.g. beyond 1024 x 1024 in 2D or 64^3 in 3D) return
 * AHOC_EUNSUPPORTED before any launch.  The first call on a device looks up
 * the array's device address with that device current; make that first call
 * before any stream capture.  Under CUDA's lazy module loading (the default)
 * that first call is also what creates the 16 MiB array on the device, so a
 * caller that hands the device's memory to a pool should make it first.
 * The looked-up address is kept for the life of the process: do not call
 * this entry point on a device after a cudaDeviceReset of it.  Every call
 * shares the array: calls that overlap on the GPU (other streams or threads)
 * race.  Calls no cudaMalloc, cudaFree or allocating library routine. */
ahoc_status ahoc_poisson_noalloc(int dim, const int64_t* N, const double* lo, const double* hi,
                                 const double* rhs, double* w, void* stream);

/* Free a plan and everything it allocated (workspace unless caller-owned,
 * coarse levels, staging grids, streams and graphs); NULL is accepted.
 * Synchronises the plan's stream first.  No counterpart in the paper. */
ahoc_status ahoc_plan_destroy(ahoc_plan* p);

/* Batched plans (serving; no counterpart in the paper, which solves one
 * problem at a time: a plan of opts.batch same-shape problems runs every
 * step of Algorithm 1 for all of them in each launch) ---------------------- */

/* Replace problem b's coefficient and boundary data (single-problem sizes,
 * device) in an existing plan, coarse levels included; the shape tables and
 * the workspace are kept.  Synchronises the plan's stream. */
ahoc_status ahoc_plan_load(ahoc_plan* p, int b, const double* alpha, const ahoc_bdata* bd);

/* Problems taking part in the next solves, matvecs and Schur right-hand
 * sides: mask[b] != 0 (host array of ahoc_batch(p) flags; NULL = all).
 * The others are skipped by every launch and their outputs are untouched. */
ahoc_status ahoc_set_active(ahoc_plan* p, const int* mask);

/* Number of problems a plan holds (opts.batch). */
int ahoc_batch(const ahoc_plan* p);

/* Launch-shape tuning (no paper counterpart) ------------------------------ */

/* Tunable launch shapes, kept in a process-wide table per (kind, dim, N,
 * precision) and fixed into a plan when it is created (and read by
 * ahoc_workspace_bytes, so set them before both):
 *   AHOC_TUNE_TRI_CHUNK    rows per thread of the chunked tridiagonal solve
 *                          along the last axis: 8, 16 or 32 (key N: that axis)
 *   AHOC_TUNE_DST_THREADS  threads per CTA of the line DSTs along x and y:
 *                          128, 256, 512 or 1024 (key N: the x axis)
 *   AHOC_TUNE_DST_RADIX    radix of the FFT stages of the line DSTs along x
 *                          and y: 4 (one radix-2 stage first when log2(N/2) is
 *                          odd) or 8 (one radix-2 or radix-4 stage first when
 *                          log2(N/2) is not a multiple of 3) (key N: the x axis)
 * value 0 restores the built-in choice.  The shapes change rounding, not the
 * discrete problem: results stay within the solver's tolerance. */
enum { AHOC_TUNE_TRI_CHUNK = 0, AHOC_TUNE_DST_THREADS = 1, AHOC_TUNE_DST_RADIX = 2, AHOC_TUNE_NKINDS = 3 };
ahoc_status ahoc_tune_set(int kind, int dim, int64_t N, int prec, int value);
/* the table entry (0: built-in), or -1 for arguments out of range */
int ahoc_tune_get(int kind, int dim, int64_t N, int prec);

/* Error reporting (no counterpart in the paper): the name of a status, and
 * a one-line description of the calling thread's most recent failure.
 * Static or thread-local strings owned by the library; never NULL. */
const char* ahoc_status_string(ahoc_status s);
const char* ahoc_last_error(void);

/* n_gamma, the number of augmented unknowns Q of one problem (the face
 * relative interiors, Sec. 2.2): the length of a face array.  -1 for NULL. */
int64_t ahoc_n_gamma(const ahoc_plan* p);

#ifdef __cplusplus
}
#endif
#endif /* AHOC_H */
