/*
 * ceedbp -- matrix-free high-order spectral-element bake-off operators and
 * Jacobi-PCG on one GB300 (sm_103a).  C ABI.
 *
 * The library implements the bake-off problems of "Scalability of
 * High-Performance PDE Solvers" (Fischer et al.), Sec. 3 and Table 1:
 *
 *   BP1  B u = r      scalar, homogeneous Neumann,   q = N+2 Gauss (GL) points
 *   BP2  B u_i = r_i  three components, as BP1
 *   BP3  A u = r      scalar, homogeneous Dirichlet, q = N+2 GL points
 *   BP4  A u_i = r_i  three components, as BP3
 *   BP5  A u = r      scalar, homogeneous Dirichlet, q = N+1 GLL points (collocated)
 *   BP6  A u_i = r_i  three components,  as BP5
 *
 * on hexahedral meshes with an iso-parametric map (Sec. 4, Eq. (18)), with the
 * assembled operator applied matrix-free as w = Q^T A_L Q u (Eq. (21)), the
 * element operators in the factored form of Eq. (22) (stiffness) or Eq. (34)
 * (mass) with geometric factors G^e_mm' of Eq. (23), and diagonally
 * preconditioned CG around them (Sec. 3).  Around that path: the Helmholtz
 * operator A + beta B of Eq. (17) (ceedbp_set_helmholtz), a variable
 * coefficient with its adjoint gradient (ceedbp_set_kappa,
 * ceedbp_kappa_gradient), FP64 defect correction around FP32/BF16 inner
 * solves (ceedbp_prepare_mixed), batched solves (ceedbp_batch_*), the
 * unassembled element operators (ceedbp_bk_apply) and an allocation-free
 * apply (ceedbp_apply_noalloc).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Global vectors hold one value per unique node (and component): FP64,
 *   layout [nglobal][ncomp] (component fastest), in the caller's node numbering
 *   (the numbering used by the l2g map given to ceedbp_setup).  Dirichlet
 *   entries of outputs are zero.
 * - Pointers named *_dev are device pointers owned by the caller; the library
 *   never frees them.  Pointers without the suffix are host pointers, read
 *   during the call only.
 * - Every call is ordered on the CUDA stream given to ceedbp_setup.  apply
 *   and mass never synchronise the host; solve synchronises the stream at the
 *   end of every chunk of iterations to read the convergence state.
 * - Status codes are returned, never exceptions.  On any code other than
 *   CEEDBP_OK, ceedbp_last_error(ctx) describes the cause (for setup failures
 *   with ctx == NULL, and for ceedbp_apply_noalloc, ceedbp_last_error(NULL)
 *   holds the message of the calling thread's last such failure).
 * - Context objects are not thread-safe: one host thread at a time per ctx.
 */
#ifndef CEEDBP_H
#define CEEDBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CEEDBP_OK = 0,
  CEEDBP_EINVAL = 1,      /* invalid argument (sizes, order, null pointer, bad l2g) */
  CEEDBP_ENOMEM = 2,      /* device or host allocation failed */
  CEEDBP_ECUDA = 3,       /* a CUDA runtime call failed */
  CEEDBP_ENOCONV = 4,     /* solve hit maxit before the tolerance; info and x are filled */
  CEEDBP_EBREAKDOWN = 5,  /* CG breakdown: p^T A p <= 0 or a non-finite scalar */
  CEEDBP_EUNSUPPORTED = 6 /* combination of options not built */
} ceedbp_status;

/* Arithmetic of the FP64 operator and solver (ceedbp_params.arith). */
enum {
  CEEDBP_ARITH_FP64 = 0, /* native FP64 instructions */
  CEEDBP_ARITH_DF64 = 1  /* FP64-accurate pairs of FP32 numbers (hi + lo, ~2^-46 relative per
                            value) on the FP32 pipe, which the GB300 issues 63x faster than
                            FP64; BP1, BP3, BP5 and BP6 (EUNSUPPORTED for BP2 and BP4).
                            One apply matches the FP64 path to about 2e-13
                            relative and the FP64 oracle to below 1e-12. */
};

typedef struct {
  int bp;           /* bake-off problem: 1..6 (Table 1) */
  int order;        /* polynomial order N = p, 1..15; p1 = N+1 nodes per direction */
  int nquad;        /* quadrature points per direction; 0 = the BP's rule (N+2 GL or N+1 GLL) */
  int64_t nelem;    /* E, number of hexahedral elements */
  int64_t nglobal;  /* number of unique nodes */
  int arith;        /* CEEDBP_ARITH_FP64 or CEEDBP_ARITH_DF64 (apply and solve) */
  int geom;         /* CEEDBP_GEOM_STORED (0) or CEEDBP_GEOM_RECOMPUTE (see below) */
} ceedbp_params;

/*
 * Geometric factors (Eq. (23)).  STORED keeps the six factors per quadrature
 * point in device memory (48 bytes per point) and streams them every apply.
 * RECOMPUTE keeps the nodal coordinates instead (24 bytes per node, layout
 * [E][3][p1^3]) and forms J, adj(J), |J| and the factors inside the element
 * kernel each apply (about 9 p1 + 40 more FMAs per node).  RECOMPUTE is built
 * for BP5 and BP6 (collocated GLL quadrature, where the Jacobian at a node is
 * the derivative of the map of Eq. (18) with the operator's own D), with FP64
 * arithmetic, without kappa, and for BP6 up to order 12; setup returns
 * CEEDBP_EUNSUPPORTED otherwise.  The Jacobi diagonal is computed at setup
 * from temporary stored factors.  Defect correction, set_kappa and the
 * adjoint gradient need the stored factors and return CEEDBP_EUNSUPPORTED on
 * a RECOMPUTE context.
 */
#define CEEDBP_GEOM_STORED 0
#define CEEDBP_GEOM_RECOMPUTE 1

/*
 * Deformed-box mesh helper (Sec. 3: E elements in a tensor-product array;
 * element map of Eq. (18) with nodes at the GLL points).
 * Element (ex, ey, ez), id e = ex + Ex (ey + Ey ez); local node (i, j, k),
 * a = i + p1 (j + p1 k).  Undeformed node x = (ex + (xi_i + 1)/2) / Ex (same
 * for y, z); every coordinate is then shifted by
 * amp * sin(pi x) sin(pi y) sin(pi z) evaluated at the undeformed point.
 * Global id g = I + (N Ex + 1)(J + (N Ey + 1) K), I = ex N + i.
 * Outputs (host, caller-allocated, may be NULL to skip):
 *   coords    [E][p1^3][3] doubles,
 *   l2g       [E][p1^3] int64 global ids,
 *   dirichlet [nglobal] bytes, 1 on the boundary of the box.
 * nglobal_out (may be NULL) receives (N Ex + 1)(N Ey + 1)(N Ez + 1).
 */
ceedbp_status ceedbp_mesh_box(int Ex, int Ey, int Ez, int order, double amp,
                              double* coords, int64_t* l2g, uint8_t* dirichlet,
                              int64_t* nglobal_out);

typedef struct ceedbp_ctx ceedbp_ctx;

/*
 * Set up an operator context: uploads the mesh, computes the geometric
 * factors of Eq. (23) (six symmetric components per quadrature point, scaled
 * by kappa when given) or the mass factors rho_i rho_j rho_k |J| of Eq. (34),
 * the gather-scatter offsets of Q^T, and the Jacobi diagonal 1/diag(A) (0 on
 * Dirichlet nodes).
 *   params     problem description; nglobal must exceed every l2g entry.
 *   coords     host [E][p1^3][3] nodal coordinates x^e_ijk (Eq. (18)).
 *   l2g        host [E][p1^3] global ids (the Boolean map Q of Eq. (21)).
 *   dirichlet  host [nglobal] bytes (1 = homogeneous Dirichlet node) or NULL
 *              (no Dirichlet nodes; BP1 ignores it).
 *   kappa      host [E][q^3] coefficient at quadrature points (stiffness
 *              problems; Eq. (4) with mu = kappa) or NULL for kappa = 1.
 *   stream     cudaStream_t to order all work on (NULL = legacy default).
 *   out        receives the context; owns all device memory it allocates.
 * Errors: EINVAL (bad sizes, order, l2g out of range), ENOMEM, ECUDA.
 */
ceedbp_status ceedbp_setup(const ceedbp_params* params, const double* coords,
                           const int64_t* l2g, const uint8_t* dirichlet,
                           const double* kappa, void* stream, ceedbp_ctx** out);

/*
 * w = M A M u (BP3-BP6, M the 0/1 mask of non-Dirichlet nodes) or w = B u
 * (BP1, BP2): the assembled operator Q^T A_L Q of Eq. (21), applied matrix-free
 * with the element operator of Eq. (22) (or Eq. (34)) and a deterministic
 * gather-scatter sum over sorted element slots (no floating-point atomics).
 * u_dev, w_dev: device FP64 [nglobal][ncomp]; they must not overlap.
 * The call returns without synchronising; with CEEDBP_ARITH_DF64 a staging
 * copy whose bounded wait gave up (the result is then invalid) is reported by
 * the next ceedbp_check or ceedbp_solve on ctx.
 */
ceedbp_status ceedbp_apply(ceedbp_ctx* ctx, const double* u_dev, double* w_dev);

/*
 * w = B u with B the mass matrix in the BP's own quadrature (Eq. (34); for
 * BP5/BP6 the diagonal GLL mass), no mask.  Used to form right-hand sides
 * b = M B f.  Same layout and ownership as ceedbp_apply.
 */
ceedbp_status ceedbp_mass(ceedbp_ctx* ctx, const double* u_dev, double* w_dev);

/* Inner precision of FP64 defect correction (ceedbp_prepare_mixed, solve opts.mixed). */
enum {
  CEEDBP_MIXED_NONE = 0,
  CEEDBP_MIXED_FP32 = 1, /* inner operator and vectors in FP32 */
  CEEDBP_MIXED_BF16 = 2, /* inner G and direction p stored in BF16, FP32 arithmetic */
  CEEDBP_MIXED_FP32_TC = 3 /* as CEEDBP_MIXED_FP32, with the element contractions of the inner
                              operator on the tensor cores: warp-level TF32 MMAs with every
                              operand split into two TF32 parts (3xTF32, FP32-level products);
                              order 7 only (EUNSUPPORTED otherwise) */
};

/*
 * Prepare defect-correction solves (BP5/BP6): allocates the low-precision copy
 * of the geometric factors (FP32 or BF16, rounded to nearest from the FP64
 * factors of Eq. (23); CEEDBP_MIXED_FP32_TC shares the FP32 copy) and the
 * FP32 inner CG vectors.  Call once per
 * precision before ceedbp_solve with opts->mixed = precision.
 * Errors: EUNSUPPORTED (BP1/BP3), EINVAL, ENOMEM, ECUDA.
 */
ceedbp_status ceedbp_prepare_mixed(ceedbp_ctx* ctx, int precision);

/* Jacobi preconditioner: dinv_dev[nglobal] receives 1/diag (0 on Dirichlet nodes). */
ceedbp_status ceedbp_jacobi(ceedbp_ctx* ctx, double* dinv_dev);

typedef struct {
  double tol;        /* stop at the first iteration with ||r||_2 <= tol ||b||_2 (per component) */
  int maxit;         /* iteration limit (ENOCONV when reached without convergence) */
  int fixed_iters;   /* > 0: run exactly this many iterations, ignore tol */
  int chunk;         /* iterations per launched CUDA graph between host checks; 0 = 32 */
  int use_graph;     /* 1 = capture chunks in CUDA graphs (default), 0 = plain launches */
  int x0_nonzero;    /* 1 = x_dev holds an initial guess; 0 = start from x = 0 */
  int profile;       /* 1 = record CUDA events around every kernel (inside the graph) and
                        report per-kernel mean durations in info->kernel_ms */
  int mixed;         /* CEEDBP_MIXED_*: FP64 defect correction around a low-precision inner
                        PCG (outer residual r = b - A x, update x += d and all CG inner
                        products in FP64 accuracy); tol applies to the FP64 residual */
  double inner_tol;  /* inner relative tolerance (0 = 1e-4 for FP32, 3e-3 for BF16) */
  int inner_maxit;   /* inner iteration limit per outer step (0 = maxit) */
  int outer_maxit;   /* outer step limit (0 = 50) */
} ceedbp_solve_opts;

typedef struct {
  int iters[3];      /* iterations performed, per component */
  double rel_res[3]; /* final ||r||_2 / ||b||_2 (recursive residual), per component */
  double res_norm[3];
  double b_norm[3];
  double device_ms;  /* time of the iteration loop measured with CUDA events */
  double kernel_ms[3]; /* with opts->profile: mean duration of the element, update and
                          direction kernels over the iterations run (0 otherwise) */
  int status;        /* same as the return value */
  int outer_iters;   /* defect-correction steps (0 for plain solves) */
} ceedbp_solve_info;

/*
 * Jacobi-PCG (Sec. 3) on the assembled system, one independent CG per
 * component (BP6); with opts->mixed, FP64 defect correction around a
 * low-precision inner Jacobi-PCG (info->iters then counts inner iterations).  b_dev: device [nglobal][ncomp]; x_dev: device
 * [nglobal][ncomp], in: initial guess when opts->x0_nonzero, out: solution.
 * All CG scalars stay on the device; each iteration is two fused kernels plus
 * one direction update, launched from a captured CUDA graph.
 * Returns OK, ENOCONV (info filled, x holds the last iterate), EBREAKDOWN.
 */
ceedbp_status ceedbp_solve(ceedbp_ctx* ctx, const double* b_dev, double* x_dev,
                           const ceedbp_solve_opts* opts, ceedbp_solve_info* info);

/*
 * ceedbp_apply without any allocation (the paper has no counterpart; this is
 * a service for callers that cannot call cudaMalloc where they apply the
 * operator -- e.g. while another thread holds a global-mode stream capture,
 * when another allocator owns the device memory, or in time-critical loops
 * that cannot take cudaMalloc's implicit synchronisation).
 * Computes the same w as ceedbp_apply(ctx, u_dev, w_dev) with the same
 * kernels (FP64 or FP32-pair arithmetic, stored or recomputed factors, kappa
 * and the Helmholtz term as set on ctx), on `stream` (cudaStream_t, NULL =
 * legacy default), using for the element-local scratch a file-scope device
 * array of 32 MiB (2^22 doubles, or 2^22 pairs) instead of the context's
 * buffer.  The array is committed on a device when ceedbp_setup first runs
 * there (setup looks up its device address, which loads the library's device
 * image holding it, and repeats the lookup on every later setup) and is held
 * until the process exits.
 *   ctx    a context from ceedbp_setup (read only; its own scratch is untouched)
 *   u_dev  device FP64 [nglobal][ncomp] input, w_dev device FP64 output.
 * Limit: E * (N+1)^3 * ncomp <= 2^22 (N = 7: 8192 scalar elements); larger
 * problems return CEEDBP_EINVAL and launch nothing.  On any error the message
 * is in ceedbp_last_error(NULL) of the calling thread (ctx is not modified).
 * A pair-arithmetic staging wait that gives up is reported like one of
 * ceedbp_apply (ceedbp_check).  All calls share the one array: calls whose
 * kernels overlap on the GPU (other streams, other threads) race on it.  Each
 * call writes every scratch entry it later reads, so nothing needs clearing.
 */
ceedbp_status ceedbp_apply_noalloc(const ceedbp_ctx* ctx, const double* u_dev, double* w_dev,
                                   void* stream);

/*
 * Variable coefficient (Eq. (4) with mu = kappa): replace the coefficient at
 * the quadrature points, kappa_dev device FP64 [E][q^3] (q^3 points of element
 * e at kappa_dev + e q^3, point index qx + q (qy + q qz)).  The stiffness
 * factors become kappa Ghat (Ghat: Eq. (23) without coefficient) and the
 * Jacobi diagonal (and any FP32-pair or low-precision copies) are recomputed.
 * Stiffness problems only; EUNSUPPORTED for BP1.
 */
ceedbp_status ceedbp_set_kappa(ceedbp_ctx* ctx, const double* kappa_dev);

/*
 * Misfit J = 1/2 (u - u*)^T B (u - u*) with B the BP's mass (diagonal GLL mass,
 * BP5 only) and the adjoint right-hand side rhs = M B (u - u*).
 *   u_dev, ustar_dev: device FP64 [nglobal]; rhs_dev: device output [nglobal];
 *   J: host output (the call synchronises the stream).
 */
ceedbp_status ceedbp_misfit(ceedbp_ctx* ctx, const double* u_dev, const double* ustar_dev, double* rhs_dev,
                            double* J);

/*
 * Adjoint gradient of J(kappa): g_dev[e][q] = -(grad lambda)_q . Ghat_q (grad u)_q
 * = dJ/dkappa_{e,q} for the solution u of A(kappa) u = b and the adjoint
 * lambda of A(kappa) lambda = M B (u - u*) (ceedbp_misfit's rhs; one solve,
 * A is symmetric).  BP5 (collocated quadrature), orders 1..11.
 *   u_dev, lambda_dev: device FP64 [nglobal]; g_dev: device FP64 [E][q^3].
 */
ceedbp_status ceedbp_kappa_gradient(ceedbp_ctx* ctx, const double* u_dev, const double* lambda_dev, double* g_dev);

/*
 * Batched BP5 solves: nprob independent problems (own mesh, order, size) set
 * up together and solved by one batched Jacobi-PCG whose every phase is one
 * launch per polynomial order for all problems, captured in CUDA graphs.
 * Arithmetic: params[p].arith, the same for every problem (EINVAL otherwise):
 * CEEDBP_ARITH_FP64 runs the FP64 element kernels (the even-odd kernel at odd
 * orders) and FP64 vector kernels; CEEDBP_ARITH_DF64 the FP64-accurate FP32-
 * pair kernels with elements per block per order chosen by the setup
 * autotuner.  Each problem stops at its own tolerance.
 *   params[p], coords[p], l2g[p], dirichlet[p]: as for ceedbp_setup (host);
 *   params[p].bp must be 5 and params[p].geom CEEDBP_GEOM_STORED.
 * ceedbp_batch_solve: b_dev[p], x_dev[p] device FP64 [params[p].nglobal]
 * (host arrays of device pointers); opts->tol, maxit, chunk, use_graph are
 * used; infos[p] (may be NULL) receives each problem's result.
 */
typedef struct ceedbp_batch ceedbp_batch;
ceedbp_status ceedbp_batch_setup(int nprob, const ceedbp_params* params, const double* const* coords,
                                 const int64_t* const* l2g, const uint8_t* const* dirichlet, void* stream,
                                 ceedbp_batch** out);
ceedbp_status ceedbp_batch_solve(ceedbp_batch* batch, const double* const* b_dev, double* const* x_dev,
                                 const ceedbp_solve_opts* opts, ceedbp_solve_info* infos);
ceedbp_status ceedbp_batch_destroy(ceedbp_batch* batch);
const char* ceedbp_batch_last_error(const ceedbp_batch* batch);

/*
 * Helmholtz operator H = A + beta B of Eq. (17) (the equation of Eq. (4) with
 * constant mu = 1 (or kappa) and beta): after this call ceedbp_apply,
 * ceedbp_apply_noalloc, ceedbp_bk_apply and ceedbp_solve use A + beta B,
 * with B the mass matrix in the BP's own quadrature (Eq. (34)), the same
 * Dirichlet mask, and the Jacobi diagonal of A + beta B.  beta = 0 restores
 * the plain stiffness.  Built for BP3-BP6 with CEEDBP_ARITH_FP64 and stored
 * factors (CEEDBP_EUNSUPPORTED otherwise, and for contexts prepared for
 * defect correction); beta must be finite and >= 0 (CEEDBP_EINVAL).
 * Synchronises the stream and drops the context's captured graphs.
 */
ceedbp_status ceedbp_set_helmholtz(ceedbp_ctx* ctx, double beta);

/*
 * Unassembled element operator (the "BK" kernels of Table 1): for every
 * element e, w^e = A^e u^e (BP3-BP6: the stiffness of Eq. (22), or Eqs.
 * (31)-(33) with GL quadrature; no Dirichlet mask) or w^e = B^e u^e (BP1,
 * BP2: Eq. (34)), without Q or Q^T.
 *   uL, wL  device [E][p1^3][ncomp] FP64, element-local values (the layout of
 *           coords); must not overlap.
 * With CEEDBP_ARITH_DF64 the pair kernel computes w^e and an extra pass turns
 * the pairs into FP64.  The first call allocates an identity gather map of
 * E p1^3 int32 (kept until destroy); later calls allocate nothing.  Stream
 * ordered on the context's stream; returns without synchronising.
 */
ceedbp_status ceedbp_bk_apply(ceedbp_ctx* ctx, const double* uL, double* wL);

/* Shape the setup autotuner chose for the FP32-pair element kernel
 * (CEEDBP_ARITH_DF64): elements in flight per thread block, the schedule
 * (0: G fetched two slabs ahead into a ring by per-thread asynchronous copies;
 * 1: the element's G staged in shared memory by one bulk asynchronous copy;
 * 2: software-pipelined sequences, each group of p1^2 threads working through
 * `seq` consecutive elements while fetching the next one's data; 3: the
 * even-odd form of the 1D contractions (Eq. (37)) on pairs, one thread per
 * mirror octet of nodes, pipelined sequences of `seq` elements per group of
 * p1^3/8 threads -- BP5 at odd orders 3..11), and seq (1 for schedules 0 and
 * 1).  Outputs are 0 (seq 1) for contexts without the pair path; any output
 * pointer may be NULL. */
ceedbp_status ceedbp_tile_info(const ceedbp_ctx* ctx, int* elems_per_block, int* schedule, int* seq);

/* Replace the autotuner's choice by one of the shapes it times (same meaning
 * as ceedbp_tile_info; seq is ignored for schedules 0 and 1).  The shapes of
 * schedules 0..2 compute the same element results bit for bit, and so do the
 * shapes of schedule 3 among themselves; schedule 3 rounds differently from
 * 0..2 (the results agree to the pair arithmetic's accuracy, about 1e-13
 * relative).  The fused (p, A p) may differ in the last bits between shapes
 * because the summation order of the block partials changes.  Returns
 * CEEDBP_EINVAL for a shape that is not launchable at this order,
 * CEEDBP_EUNSUPPORTED on a context without the pair path.  Synchronises the
 * context's stream and drops its captured CUDA graphs. */
ceedbp_status ceedbp_set_tile(ceedbp_ctx* ctx, int elems_per_block, int schedule, int seq);

/*
 * Failure detection of the pair path (a service around the method; the paper
 * has no counterpart).  The FP32-pair element kernel with the staged schedule
 * (ceedbp_set_tile schedule 1) waits for the bulk copy of an element's G on
 * an mbarrier with a bounded number of polls; when the wait gives up, the
 * kernel sets a fault flag, waits once more (bounded) for its copy to land,
 * and returns -- its results are invalid, but the CUDA context stays usable.
 * ceedbp_check synchronises the context's stream and returns CEEDBP_ECUDA if
 * any kernel on ctx gave up a wait since the last check (or solve), clearing
 * the flag, or CEEDBP_ECUDA for a pending CUDA error; CEEDBP_OK otherwise.
 * ceedbp_solve reports and clears the flag the same way at its end.
 * ceedbp_set_wait_limit sets the number of polls of the first wait (0: give up
 * at once, which makes every staged launch report the fault -- a test of this
 * detection that involves no GPU fault; < 0: restore the default 2^22).  The
 * draining wait keeps the default.  Pair contexts only (EUNSUPPORTED
 * otherwise); synchronises the stream and drops captured graphs.
 */
ceedbp_status ceedbp_check(ceedbp_ctx* ctx);
ceedbp_status ceedbp_set_wait_limit(ceedbp_ctx* ctx, int polls);

/*
 * Measured arithmetic peak of the current device (a service for the roofline
 * of the element kernels, Sec. 8.1's empirical roofline; no counterpart in
 * the method): FMA throughput in TFLOP/s (2 flops per FMA) of a kernel that
 * runs 8 independent dependent FMA chains per thread on 8 blocks of 256
 * threads per SM, in FP64 (fp64 != 0) or FP32, best of three timed launches
 * after a warm-up (about 0.1 s each).  sm_count (may be NULL) receives the
 * device's SM count.  Allocates and frees a small buffer; synchronises.
 * Errors: EINVAL (tflops NULL), ECUDA (message in ceedbp_last_error(NULL)).
 */
ceedbp_status ceedbp_fma_peak(int fp64, double* tflops, int* sm_count);

/*
 * Measured throughput of warp-level MMA instructions (mma.sync) on the current
 * device, in TFLOP/s (2 m n k flops per instruction), for kind 0: FP64
 * m8n8k4, 1: TF32 m16n8k8 with FP32 accumulation, 2: BF16 m16n8k16 with FP32
 * accumulation; 4 independent accumulator tiles per warp, 8 blocks of 256
 * threads per SM, best of three timed launches after a warm-up.  The element
 * contractions are small dense products (Sec. 5, Eqs. (29)-(33)); these
 * rates, against ceedbp_fma_peak's, tell whether moving them to the tensor
 * cores can pay.  Errors: EINVAL (bad kind or NULL), ECUDA (message in
 * ceedbp_last_error(NULL)).
 */
ceedbp_status ceedbp_mma_peak(int kind, double* tflops);

/* Release every resource owned by ctx (NULL is accepted). */
ceedbp_status ceedbp_destroy(ceedbp_ctx* ctx);

/* Message for the last failure on ctx (or of this thread's last failed setup when ctx is NULL). */
const char* ceedbp_last_error(const ceedbp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CEEDBP_H */
