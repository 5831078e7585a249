// Internal declarations shared by the ceedbp translation units (host side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ceedbp.h"

namespace ceedbp {

constexpr int kMaxOrder = 15;
constexpr int kMaxP1 = kMaxOrder + 1;
constexpr int kMaxQ = kMaxOrder + 2;

// Operator kinds of the element kernel.
enum OpKind : int { kMass = 0, kStiff = 1 };

// 1D tables of one (order, quadrature) pair, computed on the host (setup).
struct Basis1D {
  int p1 = 0, q = 0;
  bool colloc = false;          // quadrature points are the GLL nodes (BP5/BP6)
  std::vector<double> xi, rho;  // GLL nodes and weights, p1 each
  std::vector<double> eta, w;   // quadrature points and weights, q each
  std::vector<double> J;        // [q][p1] interpolation h_j(eta_q) (identity when colloc)
  std::vector<double> Dh;       // [q][p1] derivative h_j'(eta_q)
  std::vector<double> Dq;       // [q][q] derivative of the Lagrange basis on the quadrature points
};

// Device table layout (doubles): J [q*p1] | Dh [q*p1] | Dq [q*q] | w [q]
inline size_t basis_doubles(int p1, int q) { return size_t(2) * q * p1 + size_t(q) * q + q; }

bool build_basis(int order, int q, bool gll_quad, Basis1D* out, std::string* err);

// Per-component CG scalars kept on the device.
struct CompScalars {
  double rz;     // (r, z) of the current residual
  double pAp;    // (p, A p)
  double rr;     // (r, r)
  double bb;     // (b, b)
  double alpha, beta;
  double tol2;   // tol^2 (b, b)
  int iters;     // iterations performed
  int active;    // 1 while the component is iterating
  int status;    // CEEDBP_OK or CEEDBP_EBREAKDOWN
  int pad;
};

struct SolveState {
  CompScalars c[3];
  int ncomp;
  int fixed;     // 1: fixed iteration count, never deactivate on tolerance
  int stop;      // 1: every component inactive; kernels return at once
  int fault;     // nonzero: a kernel gave up a bounded wait (its results are invalid)
  unsigned int ticket[4];  // last-block counters, one per reduction site
};

// Per-problem CG scalars of batched solves.
struct BatchScalars {
  CompScalars c;
  unsigned int ticket[4];
};
struct BatchGlobal {
  int active_count;  // problems still iterating
  int fault;
};

enum TicketSite { kTicketApply = 0, kTicketUpdate = 1, kTicketInit = 2, kTicketResidual = 3 };

struct DeviceMesh {
  int p1, q, ncomp, bp;
  bool colloc;
  int64_t nelem, nglobal;
  const int* l2g;       // [E][p1^3]; Dirichlet nodes encoded as -(g+1)
  const int* off;       // [nglobal+1]; bit 31 of off[g] = Dirichlet flag of node g
  const int* slots;     // [E p1^3] local slots sorted by node, then slot
  const double* basis;  // device 1D tables (layout above)
  int tune_eb;          // elements per block of the FP32-pair kernel (0 = default; set by the autotuner)
  int tune_stage;       // pair kernel schedule (autotuner): 0 G ring by cp.async, 1 G staged by a bulk
                        // copy, 2 software-pipelined element sequences (elem_dfp_kernel)
  int tune_ns;          // elements per slot sequence of the pipelined schedule
  const double* X;      // [E][3][p1^3] nodal coordinates when the factors are recomputed, else nullptr
};

// Message of the calling thread's last failure outside a context (ceedbp_last_error(NULL)).
void set_thread_error(const std::string& msg);
// Looks up (again) the device address of the static scratch of ceedbp_apply_noalloc on the
// current device; called by setup.
cudaError_t noalloc_scratch_refresh();

// ---- kernel launchers (one translation unit per family) ----------------------
// Geometric factors G[e][6][q^3] (kappa-scaled), mass factors M[e][q^3].
// scratch: at least geom_scratch_doubles(blocks, q) doubles.
size_t geom_scratch_doubles(int blocks, int q);
int geom_blocks(int64_t nelem);
cudaError_t launch_geom(const DeviceMesh& m, const double* coords, const double* kappa,
                        double* G, double* Mq, double* scratch, cudaStream_t s);

// Local Jacobi contributions diag(A^e) (stiffness) or diag(B^e) (mass) -> wl[E][p1^3]
cudaError_t launch_local_diag(const DeviceMesh& m, int kind, const double* G, const double* Mq,
                              double* wl, cudaStream_t s);

// Element operator: wl = A_L (Q u) or B_L (Q u) for ncomp components, optional
// per-block dot partials of (Q u, wl); mask_in = read Dirichlet nodes as zero.
struct ElemArgs {
  const double* u;       // global input [nglobal][ncomp]
  double* wl;            // local output [E p1^3][ncomp]
  const double* G;       // stiffness factors or mass factors
  double* partials;      // [ncomp][nblocks] or nullptr
  SolveState* state;     // for the fused last-block reduction (alpha) or nullptr
  int mask_in;
  int skip_dirichlet_out;
  const double* Mq;      // Helmholtz term of Eq. (17): w += beta B u with the mass factors Mq ...
  double beta;           // ... when beta != 0 (stiffness kernels in FP64 only)
  // batched solves (scalar problems, one problem per block, see BatchScalars); nullptr otherwise
  const int* blk_prob;   // [nblocks] problem of each block
  const int* blk_e0;     // [nblocks] first element of the block
  const int* blk_n;      // [nblocks] elements in the block (<= elements per block)
  const int* prob_blk0;  // [nprob] first block of each problem
  const int* prob_nblk;  // [nprob] number of blocks of each problem
  BatchScalars* bst;     // [nprob] per-problem CG scalars
  int batch_blocks;      // grid size of a batched launch
};
int elem_blocks(const DeviceMesh& m);
// Elements per block of the FP64 stiffness kernel launch_elem uses (block tables of batched solves).
int elem_stiff_per_block(const DeviceMesh& m);
cudaError_t launch_elem(const DeviceMesh& m, int kind, const ElemArgs& a, cudaStream_t s);
// Stiffness element kernel recomputing G from m.X (collocated, FP64).
cudaError_t launch_elem_rc(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
int elem_rc_blocks(const DeviceMesh& m);
bool elem_rc_supported(int p1, int ncomp);
// coords [E][p1^3][3] -> X [E][3][p1^3]
cudaError_t launch_coords_soa(const double* coords, double* X, int64_t nelem, int p3, cudaStream_t s);

// Gather-scatter sum w[g] = sum_slots wl (masked on Dirichlet nodes if mask_out).
cudaError_t launch_gs(const DeviceMesh& m, const double* wl, double* w, int mask_out, cudaStream_t s);
cudaError_t launch_scale(const double* d, const double* u, double* w, int64_t n, int ncomp, cudaStream_t s);
cudaError_t launch_dinv(const int* off, const double* diag, double* dinv, int64_t n, cudaStream_t s);

// PCG kernels.
int vec_blocks(int64_t n);
cudaError_t launch_pcg_init(const DeviceMesh& m, const double* b, const double* ax, double* x, double* r, double* p,
                            const double* dinv, double* partials, SolveState* st, double tol,
                            int fixed, cudaStream_t s);
cudaError_t launch_pcg_update(const DeviceMesh& m, const double* wl, double* x, double* r, const double* p,
                              const double* dinv, double* partials, SolveState* st, cudaStream_t s);
cudaError_t launch_pcg_dir(const DeviceMesh& m, const double* r, double* p, const double* dinv,
                           const SolveState* st, cudaStream_t s);

// FP32-pair path (df.cuh, elem_df.cuh, pcg_df.cu).
struct dfloat;
struct ElemDfArgs;
int elem_df_tile_candidates(const DeviceMesh& m, int* eb, int* stage, int* ns, int cap, bool pipelined);
cudaError_t set_df_dconst(int p1, const dfloat* host, cudaStream_t s);
cudaError_t launch_elem_df(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s);
// BK5 on FP32 pairs with the even-odd decomposition (schedule 3 of the pair kernel): one
// component, even p1 in 4..12, not for batched launches.
bool elem_dfeo_supported(const DeviceMesh& m);
int elem_dfeo_candidates(const DeviceMesh& m, int* eb, int* ns, int cap);
cudaError_t launch_elem_dfeo(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s);
// BP1/BP3 (Gauss quadrature) on FP32 pairs; a.D holds the pair tables J [q][p1] then Dq [q][q].
bool elem_dfgl_supported(const DeviceMesh& m);
int elem_dfgl_blocks(const DeviceMesh& m);
cudaError_t launch_elem_dfgl(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s);
cudaError_t launch_init_df(const DeviceMesh& m, const double* b, const double* ax, double* x, dfloat* xd, dfloat* r,
                           dfloat* p, const dfloat* dinv, int x0, double* partials, SolveState* st, double tol,
                           int fixed, cudaStream_t s);
cudaError_t launch_update_df(const DeviceMesh& m, const dfloat* wl, dfloat* x, dfloat* r, const dfloat* p,
                             const dfloat* dinv, double* partials, SolveState* st, cudaStream_t s);
cudaError_t launch_dir_df(const DeviceMesh& m, const dfloat* r, dfloat* p, const dfloat* dinv, const SolveState* st,
                          cudaStream_t s);
cudaError_t launch_df_to_f64(const dfloat* src, double* dst, int64_t n, cudaStream_t s);
cudaError_t launch_f64_to_df(const double* src, dfloat* dst, int64_t n, cudaStream_t s);
cudaError_t launch_gs_df(const DeviceMesh& m, const dfloat* wl, double* w, int mask_out, cudaStream_t s);

// Variable coefficient and adjoint gradient (adjoint.cu).
cudaError_t launch_kappa_grad(const DeviceMesh& m, const double* u, const double* lam, const double* Ghat, double* g,
                              cudaStream_t s);
cudaError_t launch_scale_factors(const double* Ghat, const double* kappa, double* G, int64_t nelem, int q3,
                                 cudaStream_t s);
cudaError_t launch_misfit(const DeviceMesh& m, const double* mdiag, const double* u, const double* us, double* rhs,
                          double* partials, unsigned* ticket, double* out, cudaStream_t s);

// Low-precision inner solve of FP64 defect correction (elem_lp.cuh, pcg_lp.cu).
struct ElemLpArgs;
int elem_lp_blocks(const DeviceMesh& m);
cudaError_t launch_elem_lp(const DeviceMesh& m, const ElemLpArgs& a, int bf16, cudaStream_t s);
// FP32 inner operator with the contractions on the tensor cores (3xTF32 mma.sync), order 7 only.
bool elem_tc_supported(const DeviceMesh& m);
cudaError_t launch_elem_tc(const DeviceMesh& m, const ElemLpArgs& a, cudaStream_t s);
cudaError_t launch_residual(const DeviceMesh& m, const double* b, const double* ax, double* r, double* partials,
                            unsigned* ticket, double* out, cudaStream_t s);
cudaError_t launch_inner_init(const DeviceMesh& m, int bf16, const double* r64, const double* scale,
                              const float* dinv, float* x, float* r, void* p, double* partials, SolveState* st,
                              double tol, cudaStream_t s);
cudaError_t launch_inner_update(const DeviceMesh& m, int bf16, const float* wl, float* x, float* r, const void* p,
                                const float* dinv, double* partials, SolveState* st, cudaStream_t s);
cudaError_t launch_inner_dir(const DeviceMesh& m, int bf16, const float* r, void* p, const float* dinv,
                             const SolveState* st, cudaStream_t s);
cudaError_t launch_correct(const DeviceMesh& m, double* x, const float* d, const double* norm, cudaStream_t s);
cudaError_t launch_narrow(const double* src, void* dst, int64_t n, int bf16, cudaStream_t s);

}  // namespace ceedbp
