/*
 * sc4dvar.h -- C ABI of the GB300 SC-4DVAR Gauss-Newton library.
 *
 * The library implements the hot path of the strong-constraint 4D-Var
 * Gauss-Newton solve of Cheng, Rao, Sandu and Saibaba, "Randomized
 * preconditioned solvers for strong constraint 4D-Var data assimilation"
 * (arXiv 2401.15758): block Gauss-Newton Hessian products through tangent-linear
 * (TLM) and adjoint (ADJ) sweeps of a discretized model, the randomized low-rank
 * preconditioners built from them (RandSVD, Nystrom, SingleView; fixed or
 * adaptive size; reuse or recompute), and the preconditioned CG that uses them.
 *
 * Conventions (every entry point):
 *  - Return value: SC4DVAR_OK (0) or a negative SC4DVAR_ERR_* code. Nothing
 *    throws across the ABI. sc4dvar_last_error() returns a message for the last
 *    failing call on the calling thread.
 *  - Pointers named *_dev are device pointers owned by the caller; the library
 *    never frees them. Pointers named *_host are host pointers.
 *  - Dense blocks are column-major with an explicit leading dimension (ld >= rows).
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls are asynchronous on that stream unless the description says
 *    that they return a host value; those synchronize the stream.
 *  - prec selects the arithmetic of the TLM/ADJ sweeps and the element type of
 *    the block buffers: SC4DVAR_FP64 -> double*, SC4DVAR_FP32 -> float*.
 *    Vectors of the outer iteration (v, g, d, PCG vectors) are always double.
 *  - Opaque handles own device workspaces (the stored trajectory, sketches) and
 *    are released with the matching *_destroy call.
 *
 * The control variable: x0 = xb + Gamma^{1/2} v. In v the GN system of
 * Eq. (gniterf1)/(pcgsystem) reads (I + H) dv = -g_v with H = A^T A and
 *   A = [ R_i^{-1/2} O_i M_i Gamma^{1/2} ]_{i=1..n_t}    (Eq. Rhalf, m x n),
 * rows ordered time-major (row i*n_o + o).
 */
#ifndef SC4DVAR_H
#define SC4DVAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SC4DVAR_OK                 0
#define SC4DVAR_ERR_INVALID_ARG   -1
#define SC4DVAR_ERR_CUDA          -2
#define SC4DVAR_ERR_NOT_SPD       -3   /* a Cholesky factorization failed        */
#define SC4DVAR_ERR_BREAKDOWN     -4   /* PCG: p^T (I+H) p <= 0 or not finite     */
#define SC4DVAR_ERR_NOT_CONVERGED -5   /* PCG: maxit reached above tolerance      */
#define SC4DVAR_ERR_TIMEOUT       -6   /* a bounded device wait gave up (the tensor-
                                           core tall products wait on their MMAs)    */
#define SC4DVAR_ERR_OOM           -7
#define SC4DVAR_ERR_STATE         -8   /* e.g. no forward trajectory stored yet   */

/* ---- enumerations ------------------------------------------------------- */
#define SC4DVAR_MODEL_BURGERS1D 1      /* periodic 1D viscous Burgers, Sec. 5.1  */
#define SC4DVAR_MODEL_BVE2D     2      /* doubly periodic barotropic vorticity   */
#define SC4DVAR_MODEL_BURGERS1D_DIRICHLET 3 /* 1D viscous Burgers on (0, 1) with
                                          u(0) = u(1) = 0 (the paper's set-up, Sec.
                                          5.1): nx = n interior points x_j = j/(n+1),
                                          3..1024, ny = 1                        */
#define SC4DVAR_MODEL_BVE_GYRE  4      /* wind-driven barotropic vorticity in the
                                          closed basin (0, 1) x (-1, 1) with psi =
                                          omega = 0 on the boundary (the double-gyre
                                          set-up of Sec. 5.2): omega_t = -J(psi,
                                          omega) + Ro^{-1} psi_x + Re^{-1} Lap omega +
                                          Ro^{-1} sin(pi y), Lap psi = -omega, central
                                          differences on nx x ny interior points,
                                          h = 1/(nx+1), ny = 2 nx + 1, nx a power of two
                                          in [8, 128]; nu = 1/Re, forcing_amp = 1/Ro;
                                          prior SC4DVAR_PRIOR_DIRICHLET_INV_HELMHOLTZ
                                          with the five-point Delta*                */

/* Time integrators (sc4dvar_problem_desc.integrator). The TLM and ADJ are the
   discrete tangent-linear and adjoint models of the chosen scheme. */
#define SC4DVAR_RK4     0              /* classic RK4 (all models)                */
#define SC4DVAR_RK3_TVD 1              /* third-order TVD Runge-Kutta (Dirichlet
                                          Burgers and the double gyre; the paper's
                                          experiments)                          */

#define SC4DVAR_FP64 0
#define SC4DVAR_FP32 1
#define SC4DVAR_DF64 2   /* FP64-class accuracy (~1e-14 per operation) from double-float
                            arithmetic on the FP32 pipe: blocks are double in and out,
                            the sweeps run on (hi, lo) float pairs. Periodic Burgers
                            only, sc4dvar_gn_hessian_apply_block only; PCG uses it for
                            the defect-correction residual of periodic Burgers problems. */

#define SC4DVAR_PRIOR_SYMBOL    0      /* caller gives the Fourier symbol of Gamma^{1/2} */
#define SC4DVAR_PRIOR_SE        1      /* sigma_b^2 exp(-d^2/(2 L^2)), periodic distance */
#define SC4DVAR_PRIOR_DIRICHLET_INV_HELMHOLTZ 3 /* Gamma^{1/2} = (a I - b Delta*)^{-1},
                                          Delta* the unscaled Laplacian stencil with
                                          zero boundary values (tridiag(1, -2, 1) for
                                          Dirichlet Burgers, five-point for the
                                          double gyre): a = prior_sigma, b =
                                          prior_length (the paper's Gamma = (0.5 I -
                                          500 Delta*)^{-2} and (-0.06 Delta*)^{-2}) */
#define SC4DVAR_PRIOR_INV_HELMHOLTZ 2  /* Gamma^{1/2} = c (I - ell^2 Lap)^{-1} on the 2D grid:
                                          c = prior_sigma, ell = prior_length (BVE)         */

#define SC4DVAR_SKETCH_NONE       0    /* Prec_Gamma: plain CG on (I + H)           */
#define SC4DVAR_SKETCH_RANDSVD    1    /* Alg. 1 (adaptive: Alg. 4)                 */
#define SC4DVAR_SKETCH_NYSTROM    2    /* Alg. 2 (adaptive: grown sketch, Alg. 2)   */
#define SC4DVAR_SKETCH_SINGLEVIEW 3    /* Alg. 3 (adaptive: Alg. 5)                 */

/* Philox stream ids of the method's own random draws at GN iteration k
 * (seed = sc4dvar_sketch_opts.seed / sc4dvar_gn_opts.seed):
 *   Omega  <- stream SC4DVAR_STREAM_SKETCH + k
 *   Psi    <- stream SC4DVAR_STREAM_SKETCH + k + SC4DVAR_STREAM_PSI
 *   kappa  <- stream SC4DVAR_STREAM_KAPPA + k (column 0: kappa_re, 1.. kappa_sk)
 * Element (i, j) of a rows x cols draw is the Box-Muller normal number
 * e = i + rows * j of that stream (Philox4x32-10, counter (e/2, stream), key seed). */
#define SC4DVAR_STREAM_SKETCH 100
#define SC4DVAR_STREAM_KAPPA  200
#define SC4DVAR_STREAM_PSI    1000

typedef struct sc4dvar_problem_s* sc4dvar_problem_t;
typedef struct sc4dvar_precond_s* sc4dvar_precond_t;

/* Problem description (all pointers are host pointers, copied at creation). */
typedef struct {
    int model;             /* SC4DVAR_MODEL_*                                        */
    int nx, ny;            /* grid; Burgers: n = nx (power of two, 8..8192), ny = 1;
                              BVE: nx = ny = N (power of two, 16..1024), n = N^2,
                              fields row-major (y slow, x fast) on [0, 2 pi)^2     */
    double nu;             /* viscosity                                              */
    double dt;             /* RK4 step                                               */
    int n_steps;           /* RK4 steps in the window (N)                            */
    int n_obs_times;       /* n_t                                                    */
    const int* obs_steps;  /* [n_t] RK step of each observation time, 1..N, increasing */
    int n_obs;             /* n_o sites per observation time                         */
    const int* obs_idx;    /* [n_t * n_o] grid indices (time-major)                  */
    double sigma_obs;      /* R_i = sigma_obs^2 I                                    */
    int prior_kind;        /* SC4DVAR_PRIOR_*                                        */
    double prior_sigma;    /* SE: sigma_b                                            */
    double prior_length;   /* SE: correlation length L                               */
    const double* prior_symbol; /* SYMBOL: [n] real even Fourier symbol of Gamma^{1/2} */
    double forcing_amp;    /* BVE forcing amplitude (F = amp sin(k y))                */
    int forcing_k;         /* BVE forcing wavenumber                                 */
    int n_checkpoints;     /* BVE: 0 = keep every RK stage state of the FWD (the sweeps
                              read them); c in [1, n_steps] = keep only the FP64 state
                              at c evenly spaced steps (every L = ceil(n_steps / c)
                              steps) and recompute one segment of L steps at a time
                              inside each TLM / ADJ sweep and the gradient: device
                              memory for states falls from 4 N n (12 B + 12 B) to
                              c n 8 B + 4 L n 12 B at the cost of one extra FWD per
                              sweep (sqrt-N checkpointing, c ~ sqrt(N)). Results are
                              identical to c = 0. Burgers: must be 0.              */
    /* BVE (Sec. 5.2, doubly periodic form): q_t = -J_A(psi, q) + nu Lap_h q + F,
       psi = Lap^{-1} q (spectral), J_A Arakawa's Jacobian, Lap_h five-point. */
    int integrator;        /* SC4DVAR_RK4 (default) or SC4DVAR_RK3_TVD               */
} sc4dvar_problem_desc;

/* Sketch options (Sec. 3.1). */
typedef struct {
    int method;            /* SC4DVAR_SKETCH_*                                   */
    int l;                 /* l (RandSVD, Nystrom) or l_1 (SingleView); initial size when adaptive */
    int l2;                /* SingleView l_2; <= 0 selects 2 l_1 + 1             */
    int adaptive;          /* 1: grow by l_hat until kappa_sk <= eps_sk          */
    int l_hat;             /* adaptive increment; <= 0 selects l / 2             */
    int l_max;             /* adaptive cap; <= 0 selects min(8 l, n)             */
    double eps_sk;         /* adaptive tolerance (Eq. condtext), e.g. 1.01        */
    uint64_t seed;         /* Philox key                                          */
    int gn_iter;           /* GN iteration index k (selects the Philox streams)   */
    int prec;              /* SC4DVAR_FP64 / SC4DVAR_FP32 sweeps and sketch storage */
    int gemm;              /* FP32 sketches: arithmetic of the tall products with an
                              l x l factor (Q = Y R^{-1}, V = W^T U S^{-1}, W = L^{-1} Y^T,
                              Gram-Schmidt updates): SC4DVAR_GEMM_*. Gram matrices
                              stay FP64-accurate in every mode.                        */
} sc4dvar_sketch_opts;

/* Tall-product arithmetic of FP32 sketches (sc4dvar_sketch_opts.gemm). */
#define SC4DVAR_GEMM_3XTF32 0   /* tensor cores, three TF32 products per term (hi*hi +
                                   hi*lo + lo*hi): FP32 accuracy (default)          */
#define SC4DVAR_GEMM_SIMT   1   /* CUDA cores, FP32 fused multiply-adds             */
#define SC4DVAR_GEMM_TF32   2   /* tensor cores, one TF32 product (~1e-4 relative)   */
#define SC4DVAR_GEMM_BF16   3   /* tensor cores, BF16 inputs (~1e-3 relative)        */

typedef struct {
    double tol;            /* relative residual |r|/|b| of the recurrence residual  */
    int maxit;             /* <= 0 selects n                                        */
    int prec;              /* operator precision of the inner iteration             */
    int refine;            /* FP32 operator only: max FP64 defect-correction restarts */
} sc4dvar_pcg_opts;

typedef struct {
    int iterations;        /* PCG iterations (all restarts)                        */
    int restarts;          /* defect-correction restarts performed                 */
    double relres;         /* final |b - (I+H) x| / |b| with the FP64 operator     */
    int status;            /* SC4DVAR_OK / _BREAKDOWN / _NOT_CONVERGED             */
} sc4dvar_pcg_info;

typedef struct {
    int iters;             /* GN iterations                                       */
    double gtol;           /* stop when |g_k|_inf / |g_0|_inf < gtol (0: never)   */
    sc4dvar_sketch_opts sketch;   /* method NONE = Prec_Gamma                      */
    double eps_re;         /* reuse tolerance (Eq. condtext2); adaptive only       */
    sc4dvar_pcg_opts pcg;
    int line_search;       /* 0: full steps (alpha = 1); 1: strong-Wolfe step length
                              (bracketing + zoom with cubic interpolation, Nocedal &
                              Wright Algs. 3.5 / 3.6; the paper uses a Moré-Thuente
                              search, Sec. 5). Each trial step costs one FWD and one
                              gradient (ADJ); the last trial's state is reused.      */
    double ls_c1, ls_c2;   /* sufficient decrease / curvature constants, 0<c1<c2<1 */
    double ls_alpha1;      /* first trial step (> 0)                               */
    int solve;             /* 0: PCG on (I + H) (SketchPrec / Prec_Gamma);
                              1: SketchSolv, dv = -(I + H_hat)^{-1} g (Eq. dxsol; needs
                              a sketch method, no PCG)                             */
} sc4dvar_gn_opts;

#define SC4DVAR_GN_MAX_ITERS 64
typedef struct {
    int iters_done;
    double J[SC4DVAR_GN_MAX_ITERS];        /* cost at each iterate                 */
    double g_inf[SC4DVAR_GN_MAX_ITERS];    /* |g_v|_inf at each iterate            */
    int pcg_its[SC4DVAR_GN_MAX_ITERS];
    double relres[SC4DVAR_GN_MAX_ITERS];
    int sketched[SC4DVAR_GN_MAX_ITERS];    /* 1 if a new sketch was built          */
    int rank[SC4DVAR_GN_MAX_ITERS];        /* sketch size in use                   */
    double kappa_re[SC4DVAR_GN_MAX_ITERS]; /* reuse estimate (0 when not computed) */
    double alpha[SC4DVAR_GN_MAX_ITERS];    /* step length taken                    */
    int ls_evals[SC4DVAR_GN_MAX_ITERS];    /* line-search trial steps              */
    int ls_status[SC4DVAR_GN_MAX_ITERS];   /* 0 ok, 1 not a descent direction (full
                                              step taken), 2 trial budget spent   */
} sc4dvar_gn_info;

/* Counters in the paper's accounting (Sec. 5, Tables 3-5): a Hessian product
 * counts one TLM and one ADJ per column; a sketch counts its TLM/ADJ columns as
 * offline; kappa estimates are counted apart. */
typedef struct {
    int64_t fwd;
    int64_t tlm_online, adj_online;
    int64_t tlm_offline, adj_offline;
    int64_t tlm_kappa, adj_kappa;
    int64_t qr_shifted;    /* CholeskyQR passes that failed and were redone with a
                              diagonal shift (shifted CholeskyQR3, no counterpart in
                              the paper, which takes Householder QR)               */
} sc4dvar_counters_t;

/* ---- library --------------------------------------------------------------- */
const char* sc4dvar_last_error(void);
int sc4dvar_version(void);
/* Number of CUDA kernels this library has launched since it was loaded (all
 * threads, all devices). A diagnostic with no counterpart in the paper, used to
 * count the kernels inside a timed region. */
long long sc4dvar_launch_count(void);

/* ---- problem ---------------------------------------------------------------
 * sc4dvar_problem_create: validates the description, copies the observation
 * pattern to the device, computes the prior symbol and allocates the trajectory
 * store ((N+1) x n doubles and (N+1) x n floats). Returns ERR_INVALID_ARG for
 * an unsupported grid, ERR_OOM if allocation fails. Runs on the default stream
 * and synchronizes it. */
int sc4dvar_problem_create(const sc4dvar_problem_desc* desc, sc4dvar_problem_t* out);
int sc4dvar_problem_destroy(sc4dvar_problem_t p);
/* n (state size) and m (= n_t * n_o) of a problem. */
int sc4dvar_problem_dims(sc4dvar_problem_t p, int* n, int* m);

/* Background xb [n] and observations y [m] (time-major), device doubles. */
int sc4dvar_set_background(sc4dvar_problem_t p, const double* xb_dev, void* stream);
int sc4dvar_set_observations(sc4dvar_problem_t p, const double* y_dev, void* stream);

/* Y = Gamma^{1/2} X for k columns (FP64). The prior square root used by A. */
int sc4dvar_prior_sqrt_apply(sc4dvar_problem_t p, const double* X_dev, int ldx, int k,
                             double* Y_dev, int ldy, void* stream);
/* The prior symbol actually in use (n doubles, host), for inspection. */
int sc4dvar_prior_symbol(sc4dvar_problem_t p, double* symbol_host);

/* Model run from an arbitrary initial state x0 [n] (FP64): writes O x_{t_i} for
 * every observation time to obs_dev [m] (time-major) and, if xN_dev is not
 * NULL, the final state. Does not touch the stored trajectory. */
int sc4dvar_forecast(sc4dvar_problem_t p, const double* x0_dev, double* obs_dev,
                     double* xN_dev, void* stream);

/* FWD at the iterate v [n]: x0 = xb + Gamma^{1/2} v, the FP64 trajectory (and
 * its FP32 copy) is stored in the handle, d = R^{-1/2}(O x_i - y_i) is formed.
 * Eq. 4dvar_cf: J(v) = 1/2 |v|^2 + 1/2 |d|^2. If J_host is not NULL the call
 * synchronizes and returns J. d_dev [m] is optional. */
int sc4dvar_fwd(sc4dvar_problem_t p, const double* v_dev, double* J_host, double* d_dev,
                void* stream);

/* g_v = v + A^T d at the stored iterate (Eq. 4dvar_gradient, in v); one FP64
 * ADJ sweep. ERR_STATE if sc4dvar_fwd was not called. */
int sc4dvar_gradient(sc4dvar_problem_t p, double* g_dev, void* stream);

/* A X (Eq. Rhalf): Gamma^{1/2}, then the TLM sweep of k columns; W is m x k. */
int sc4dvar_tlm_block(sc4dvar_problem_t p, const void* X_dev, int ldx, int k,
                      void* W_dev, int ldw, int prec, void* stream);
/* A^T W (Eq. Rhalf): the ADJ sweep of k columns, then Gamma^{1/2}; X is n x k. */
int sc4dvar_adj_block(sc4dvar_problem_t p, const void* W_dev, int ldw, int k,
                      void* X_dev, int ldx, int prec, void* stream);
/* Y = (I + A^T A) X, or A^T A X when misfit_only != 0 (Eq. Rhalf / gniterf1):
 * one TLM and one ADJ sweep per column, all k columns at once. Needs internal
 * scratch for A X (m x k in the problem's workspace, grown on demand). */
int sc4dvar_gn_hessian_apply_block(sc4dvar_problem_t p, const void* X_dev, int ldx, int k,
                                   void* Y_dev, int ldy, int misfit_only, int prec,
                                   void* stream);

/* The same product as sc4dvar_gn_hessian_apply_block, for callers that may not
 * allocate device memory during the call (a host that owns all device memory
 * through its own pool, a loop that must not enter the driver's allocator,
 * which can synchronize the device). This entry point has no counterpart in the
 * paper. It allocates nothing: its three work arrays (Gamma^{1/2} X, A X, the
 * adjoint state: (2 n + m) k elements of the prec type, each rounded up to 256
 * bytes) are carved from one fixed 32 MiB device array that the library holds on
 * every GPU that loads it, until the process exits. Larger k returns
 * SC4DVAR_ERR_INVALID_ARG (use sc4dvar_gn_hessian_apply_block then). The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress)
 * and keeps it for the process; make that first call before any stream capture
 * begins. A cudaDeviceReset frees the array with every other allocation on the
 * device (problems included), so the entry point is not usable after one. All
 * calls share the array, and it keeps the previous call's contents (nothing in
 * it needs clearing): calls that overlap on the GPU, on any stream or problem,
 * race and give wrong results. Burgers problems only. */
int sc4dvar_gn_hessian_apply_block_noalloc(sc4dvar_problem_t p, const void* X_dev, int ldx, int k,
                                           void* Y_dev, int ldy, int misfit_only, int prec,
                                           void* stream);

/* ---- preconditioners (Sec. 3.1) ---------------------------------------------
 * Builds H_hat = V diag(lam) V^T at the stored iterate with Alg. 1/2/3 (or their
 * adaptive forms). Omega_dev (n x l, double, ld n) may be NULL (then drawn with
 * Philox from opts->seed / gn_iter); Psi_dev likewise (m x l2). Synchronizes.
 * ERR_NOT_SPD if a Cholesky factorization fails. */
/* The sketches' tall product on its own: C (rows x c) = alpha A op(B) + beta C
 * with A (rows x kk, FP32, column-major, ld lda), B FP64 (kk x c, ld ldb; or
 * c x kk when transB != 0) and C FP32 (c_double = 0) or FP64 (c_double = 1),
 * column-major with ld ldc; mode SC4DVAR_GEMM_*. All pointers are device
 * memory owned by the caller. The products of Algs. 1-5 with an l x l factor
 * (CholeskyQR's Q = Y R^{-1}, the thin SVD's V = W^T U S^{-1}, ...) run through
 * it; in the tensor-core modes one CTA computes 128 rows x 256 columns with
 * tcgen05 MMAs accumulating in tensor memory. Synchronizes; SC4DVAR_ERR_TIMEOUT
 * if a bounded wait on the tensor cores gave up. */
int sc4dvar_tall_gemm(int mode, int rows, int kk, int c, double alpha, const float* A_dev, int lda,
                      const double* B_dev, int ldb, int transB, double beta, void* C_dev, int c_double,
                      int ldc, void* stream);

int sc4dvar_build_precond(sc4dvar_problem_t p, const sc4dvar_sketch_opts* opts,
                          const double* Omega_dev, const double* Psi_dev,
                          sc4dvar_precond_t* out, void* stream);
int sc4dvar_precond_destroy(sc4dvar_precond_t P);
/* rank l and, optionally, lam [l] (descending) and V (n x l, ld n) copied to host. */
int sc4dvar_precond_info(sc4dvar_precond_t P, int* rank, double* lam_host, double* V_host);
/* A preconditioner (I + V Lam V^T)^{-1} rebuilt from host copies of its factors
 * (as sc4dvar_precond_info returns them): 0 <= l <= n, lam [l] finite and
 * >= 0, V n x l (ld n), n the problem's size. It applies bit for bit like the
 * original. ERR_INVALID_ARG for a bad l or lam. */
int sc4dvar_precond_import(sc4dvar_problem_t p, int l, const double* lam_host, const double* V_host,
                           sc4dvar_precond_t* out);
/* Z = (I + V Lam V^T)^{-1} R (Eq. woodbury) for k columns, FP64. */
int sc4dvar_precond_apply(sc4dvar_precond_t P, const double* R_dev, int ldr, int k,
                          double* Z_dev, int ldz, void* stream);
/* kappa = |(I + H)(I + H_hat)^{-1} v|_2 with v = w/|w|, w the Philox column
 * `column` of stream (seed, stream_id) (Eqs. condtext, condtext2); one FP64
 * Hessian product. P = NULL gives |(I + H) v|. Synchronizes. */
int sc4dvar_kappa_estimate(sc4dvar_problem_t p, sc4dvar_precond_t P, uint64_t seed,
                           uint64_t stream_id, int column, double* kappa_host, void* stream);

/* ---- solvers ------------------------------------------------------------------
 * PCG on (I + H) x = b (Eq. pcgsystem), x0 = 0, preconditioned by P
 * (NULL = Prec_Gamma). FP64 vectors and reductions; the operator runs in
 * opts->prec. With FP32 and refine > 0 the iteration is restarted on the FP64
 * residual b - (I + H) x (defect correction) until that residual meets tol.
 * info->status is SC4DVAR_ERR_BREAKDOWN when p^T (I + H) p is not positive or
 * not finite, and at once (no iteration) when b has a non-finite entry.
 * Synchronizes; info may be NULL. */
int sc4dvar_pcg(sc4dvar_problem_t p, sc4dvar_precond_t P, const double* b_dev, double* x_dev,
                const sc4dvar_pcg_opts* opts, sc4dvar_pcg_info* info, void* stream);

/* SketchSolv step (Eq. dxsol, in v): dv = -(I + H_hat)^{-1} g. */
int sc4dvar_sketchsolv(sc4dvar_precond_t P, const double* g_dev, double* dv_dev, void* stream);

/* QR update of Alg. 6 (used by the adaptive SingleView sketch of Alg. 5 for the
 * QR of M = Psi^T Q_Y as Psi and Q_Y gain columns). All FP64, device,
 * column-major, caller-owned. A1 = P[:, 0:r1]^T and A2 = P[:, r1:r1+r2]^T, with
 * P m x (r1 + r2) (ld ldp); B1 = B[:, 0:k1] and B2 = B[:, k1:k1+k2] (ld ldb),
 * whose columns are orthonormal. On entry Q[0:r1, 0:k1] (ld ldq) and
 * R[0:k1, 0:k1] (ld ldr, upper triangular) hold Q1 R1 = A1 B1; on return
 * Q[0:r1+r2, 0:k1+k2] and R[0:k1+k2, 0:k1+k2] (upper triangular, zeros below the
 * diagonal) hold the thin QR of [A1; A2] [B1 B2]. Needs r1 >= k1 and
 * r1 + r2 >= k1 + k2, else ERR_INVALID_ARG; ERR_NOT_SPD if a block is rank
 * deficient. Allocates its workspace; synchronizes. */
int sc4dvar_qr_update(int m, int r1, int r2, int k1, int k2, const double* P_dev, int ldp,
                      const double* B_dev, int ldb, double* Q_dev, int ldq, double* R_dev, int ldr,
                      void* stream);

/* Gauss-Newton from v_inout (overwritten with the final iterate): per iteration
 * FWD, gradient, sketch (every iteration when fixed; when adaptive, the last
 * sketch is reused while kappa_re < eps_re, Sec. 3.2), PCG, v += alpha dv with
 * alpha = 1 or a strong-Wolfe step (opts->line_search).
 * Synchronizes. info may be NULL. */
int sc4dvar_gauss_newton(sc4dvar_problem_t p, const sc4dvar_gn_opts* opts, double* v_inout_dev,
                         sc4dvar_gn_info* info, void* stream);

/* Gauss-Newton state at an iteration boundary, for checkpoint and resume (no
 * counterpart in the paper). The sketch draws and the kappa_re probe of
 * iteration k are keyed by k (Philox streams with gn_iter = k, and
 * SC4DVAR_STREAM_KAPPA + k), so the iteration index is the whole random-number
 * state. Together with the iterate v and the preconditioner held across the
 * boundary it fixes every later iteration. */
typedef struct {
    int next_iter;         /* GN iterations completed = index of the next one     */
    double g0_inf;         /* |g_0|_inf of the first iterate (the gtol reference) */
    int sketch_iter;       /* iteration that built the held preconditioner (-1: none) */
} sc4dvar_gn_state;

/* Runs GN iterations state->next_iter .. opts->iters - 1 from v_inout with the
 * steps of sc4dvar_gauss_newton, and leaves state at the boundary where it
 * stopped: opts->iters, or the iteration at which gtol was met or an error
 * occurred (v_inout then holds the iterate at that boundary).
 *
 * *held is the preconditioner carried over the boundary. On entry it is the
 * one a previous call returned, one rebuilt by sc4dvar_precond_import, or NULL.
 * The call takes ownership of it. On return *held is the preconditioner in use
 * at the end (or NULL); whatever *held holds on return belongs to the caller,
 * also after an error (sc4dvar_precond_destroy).
 *
 * state->next_iter == 0 starts a new run; info is then cleared. Otherwise the
 * entries of info below next_iter are left as they are and those from
 * next_iter on are cleared first. info may be NULL; info->iters_done counts
 * from iteration 0. A held preconditioner needs a sketch method in opts
 * (ERR_INVALID_ARG with SC4DVAR_SKETCH_NONE).
 *
 * A resumed run repeats an uninterrupted one bit for bit, except that its
 * first iteration always runs a FWD and a gradient at v. (Across the boundary,
 * a strong-Wolfe search would otherwise reuse its last trial's J and g.) The
 * counters show that extra FWD and ADJ. Synchronizes. */
int sc4dvar_gauss_newton_resume(sc4dvar_problem_t p, const sc4dvar_gn_opts* opts, double* v_inout_dev,
                                sc4dvar_gn_state* state, sc4dvar_precond_t* held,
                                sc4dvar_gn_info* info, void* stream);

/* ---- batched serving ----------------------------------------------------------
 * A batch of independent problems (any mix of grids, windows, observations and
 * block widths). No counterpart in the paper: its experiments solve one problem
 * at a time; serving many small problems at once is how a GPU is kept busy.
 * sc4dvar_batch_hessian_apply: Y[b] = (I + A_b^T A_b) X[b] (or A_b^T A_b X[b]),
 * X[b], Y[b] device blocks n_b x k[b] (ld n_b) in prec. The first call (and any
 * call with other buffers, widths or flags) runs once eagerly to size the
 * workspaces, then records all problems' kernels into one CUDA graph (problems
 * on parallel branches); every later identical call is one graph launch.
 * Problems must have a stored trajectory (sc4dvar_fwd); the graph stays valid
 * across sc4dvar_fwd calls on the same handles. */
typedef struct sc4dvar_batch_s* sc4dvar_batch_t;
int sc4dvar_batch_create(const sc4dvar_problem_t* problems, int B, sc4dvar_batch_t* out);
int sc4dvar_batch_destroy(sc4dvar_batch_t b);
int sc4dvar_batch_hessian_apply(sc4dvar_batch_t b, const void* const* X_dev, void* const* Y_dev,
                                const int* k, int misfit_only, int prec, void* stream);
/* Batched PCG on (I + H_b) x_b = rhs_b (Eq. pcgsystem), x0 = 0, preconditioners
 * P[b] (NULL entries or NULL array = none), operator arithmetic prec. _start
 * initializes every problem and records one iteration of all problems into a
 * CUDA graph; _step launches that graph nsteps times (scalars stay on the device;
 * a problem whose |r| <= tol |rhs| or that broke down stops moving); _status
 * reads relres, iterations and status (0 or SC4DVAR_ERR_BREAKDOWN) per problem;
 * _solution copies the iterates out. */
int sc4dvar_batch_pcg_start(sc4dvar_batch_t b, const sc4dvar_precond_t* P, const double* const* rhs_dev,
                            double tol, int prec, void* stream);
int sc4dvar_batch_pcg_step(sc4dvar_batch_t b, int nsteps, void* stream);
int sc4dvar_batch_pcg_status(sc4dvar_batch_t b, double* relres_host, int* its_host, int* status_host,
                             void* stream);
int sc4dvar_batch_pcg_solution(sc4dvar_batch_t b, double* const* x_dev, void* stream);
/* Times the packed FP32 sweep of a problem (n >= 1024) for each valid number of
 * point pairs per thread with k directions and keeps the fastest for later
 * sweeps; chosen (nullable) returns it (0: nothing to tune). Synchronizes. */
int sc4dvar_autotune(sc4dvar_problem_t p, int k, int* chosen);

int sc4dvar_counters(sc4dvar_problem_t p, sc4dvar_counters_t* out);
int sc4dvar_counters_reset(sc4dvar_problem_t p);
/* Overwrites the problem's counters (to carry them across a GN checkpoint). */
int sc4dvar_counters_set(sc4dvar_problem_t p, const sc4dvar_counters_t* c);

/* Device Gaussian draw (the method's convention above): out (rows x cols, ld
 * rows, double) = columns col0.. of stream (seed, stream_id). */
int sc4dvar_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, int64_t col0,
                     double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SC4DVAR_H */
