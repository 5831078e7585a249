// C ABI of ceedbp: context setup, operator apply, mass, Jacobi-PCG solve.
// The entry points are declared and documented in include/ceedbp.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernel_args.h"
#include "internal.h"

namespace ceedbp {
cudaError_t launch_elem_bp1(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
cudaError_t launch_elem_bp3(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
cudaError_t launch_elem_bp5(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
cudaError_t launch_elem_bp6(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
int elem_blocks_bp1(const DeviceMesh& m);
cudaError_t launch_elem_bp2(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
cudaError_t launch_elem_bp4(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
int elem_blocks_bp4(const DeviceMesh& m);
int elem_blocks_bp3(const DeviceMesh& m);
int elem_blocks_bp5(const DeviceMesh& m);
int elem_blocks_bp6(const DeviceMesh& m);

cudaError_t launch_elem_eo(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s);
int elem_eo_blocks(const DeviceMesh& m);
bool elem_eo_available(const DeviceMesh& m);

// Collocated FP64 stiffness with even p1 (odd order) uses the even-odd kernel
// when its shape is resident on an SM (large p1 with three components is not).
static bool use_even_odd(const DeviceMesh& m) { return m.colloc && (m.p1 % 2 == 0) && elem_eo_available(m); }

cudaError_t launch_elem(const DeviceMesh& m, int kind, const ElemArgs& a, cudaStream_t s) {
  if (kind == kStiff && m.X != nullptr) return launch_elem_rc(m, a, s);
  if (kind == kStiff && use_even_odd(m)) return launch_elem_eo(m, a, s);
  if (m.colloc && kind == kStiff) return m.ncomp == 3 ? launch_elem_bp6(m, a, s) : launch_elem_bp5(m, a, s);
  if (!m.colloc && kind == kStiff) return m.ncomp == 3 ? launch_elem_bp4(m, a, s) : launch_elem_bp3(m, a, s);
  if (!m.colloc && kind == kMass) return m.ncomp == 3 ? launch_elem_bp2(m, a, s) : launch_elem_bp1(m, a, s);
  return cudaErrorInvalidValue;
}

int elem_eo_per_block_rt(const DeviceMesh& m);
int elem_per_block_bp5(const DeviceMesh& m);

int elem_stiff_per_block(const DeviceMesh& m) {
  if (m.X != nullptr) return 0;
  if (use_even_odd(m)) return elem_eo_per_block_rt(m);
  return m.colloc && m.ncomp == 1 ? elem_per_block_bp5(m) : 0;
}

int elem_blocks(const DeviceMesh& m) {
  // stiffness and mass instantiations of one (p1, q) share the block shape
  if (m.X != nullptr) return elem_rc_blocks(m);
  if (use_even_odd(m)) return std::max(elem_eo_blocks(m), m.ncomp == 3 ? elem_blocks_bp6(m) : elem_blocks_bp5(m));
  if (m.colloc) return m.ncomp == 3 ? elem_blocks_bp6(m) : elem_blocks_bp5(m);
  return m.ncomp == 3 ? elem_blocks_bp4(m) : elem_blocks_bp3(m);
}
}  // namespace ceedbp

using namespace ceedbp;

#include "ctx.h"

namespace {

thread_local std::string g_setup_error;

// Shapes of the BK5/BK6 pair kernel: the direct schedules 0..2 (elem_df_tile_candidates), then the
// even-odd kernel (schedule 3) where it is built; batched groups launch with block tables, which
// only the direct schedules take.
int pair_shape_candidates(const ceedbp_ctx* c, const DeviceMesh& m, int* eb, int* st, int* ns, int cap) {
  int n = elem_df_tile_candidates(m, eb, st, ns, cap, true);
  if (!c->pipelined_only) {
    const int k = elem_dfeo_candidates(m, eb + n, ns + n, cap - n);
    for (int q = 0; q < k; ++q) st[n + q] = 3;
    n += k;
  }
  return n;
}

ceedbp_status fail(ceedbp_ctx* c, ceedbp_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_setup_error = msg;
  return st;
}

ceedbp_status cuda_fail(ceedbp_ctx* c, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? CEEDBP_ENOMEM : CEEDBP_ECUDA, msg);
}

#define CK(ctx, call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

void release(ceedbp_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  void* ptrs[] = {c->d_l2g, c->d_off, c->d_slots, c->d_basis, c->d_G, c->d_Mq, c->d_dinv, c->d_mdiag,
                  c->d_wl, c->d_r, c->d_p, c->d_ax, c->d_part_apply, c->d_part_vec, c->d_state,
                  c->d_Gdf, c->d_Ddf, c->d_dinvdf, c->d_G32, c->d_Gbf, c->d_dinv32, c->d_xin,
                  c->d_rin, c->d_pin, c->d_outer, c->d_Ghat, c->d_scal, c->d_X, c->d_l2g_id};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_outer) cudaFreeHost(c->h_outer);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_state) cudaFreeHost(c->h_state);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (cudaEvent_t e : c->prof) cudaEventDestroy(e);
  c->prof.clear();
}

ceedbp_status setup_impl(ceedbp_ctx* c, const double* coords, const int64_t* l2g, const uint8_t* dirichlet,
                         const double* kappa) {
  const ceedbp_params& P = c->prm;
  if (P.bp < 1 || P.bp > 6) return fail(c, CEEDBP_EUNSUPPORTED, "bp must be 1..6");
  if (P.order < 1 || P.order > kMaxOrder) return fail(c, CEEDBP_EINVAL, "order must be in 1..15");
  if (P.nelem < 1 || P.nglobal < 1) return fail(c, CEEDBP_EINVAL, "nelem and nglobal must be positive");
  if (!coords || !l2g) return fail(c, CEEDBP_EINVAL, "coords and l2g are required");
  const bool gll_quad = (P.bp == 5 || P.bp == 6);
  const int p1 = P.order + 1;
  const int qdef = gll_quad ? p1 : P.order + 2;
  if (P.nquad != 0 && P.nquad != qdef) return fail(c, CEEDBP_EUNSUPPORTED, "only the BP's own quadrature is built");
  Basis1D basis;
  std::string berr;
  if (!build_basis(P.order, qdef, gll_quad, &basis, &berr)) return fail(c, CEEDBP_EINVAL, berr);
  c->p1 = p1;
  c->q = qdef;
  c->colloc = gll_quad;
  c->ncomp = (P.bp == 2 || P.bp == 4 || P.bp == 6) ? 3 : 1;
  c->op_kind = (P.bp == 1 || P.bp == 2) ? kMass : kStiff;
  const int64_t P3 = int64_t(p1) * p1 * p1, Q3 = int64_t(qdef) * qdef * qdef;
  const int64_t nloc = P.nelem * P3;
  if (nloc >= (int64_t(1) << 31) || P.nglobal >= (int64_t(1) << 31) - 1)
    return fail(c, CEEDBP_EINVAL, "problem too large for 32-bit local indices (E p1^3 and nglobal must stay below 2^31)");
  const bool masked = P.bp != 1 && P.bp != 2 && dirichlet != nullptr;
  if (P.arith != CEEDBP_ARITH_FP64 && P.arith != CEEDBP_ARITH_DF64) return fail(c, CEEDBP_EINVAL, "unknown arith");
  if (P.arith == CEEDBP_ARITH_DF64 && !gll_quad && P.bp != 1 && P.bp != 3)
    return fail(c, CEEDBP_EUNSUPPORTED, "the FP32-pair arithmetic is built for BP1, BP3, BP5 and BP6");
  c->arith = P.arith;
  if (P.geom != CEEDBP_GEOM_STORED && P.geom != CEEDBP_GEOM_RECOMPUTE) return fail(c, CEEDBP_EINVAL, "unknown geom");
  const bool recompute = P.geom == CEEDBP_GEOM_RECOMPUTE;
  if (recompute) {
    if (!gll_quad || P.arith != CEEDBP_ARITH_FP64 || kappa != nullptr)
      return fail(c, CEEDBP_EUNSUPPORTED, "recomputed factors are built for BP5/BP6, FP64, without kappa");
    if (!elem_rc_supported(p1, c->ncomp))
      return fail(c, CEEDBP_EUNSUPPORTED, "recomputed factors: the element tile does not fit at this order");
  }

  // ---- host: encoded l2g, CSR of local slots per global node (counting sort, slots ascending)
  std::vector<int> hl2g(nloc), hoff(P.nglobal + 1, 0), hslots(nloc);
  for (int64_t s = 0; s < nloc; ++s) {
    const int64_t g = l2g[s];
    if (g < 0 || g >= P.nglobal) return fail(c, CEEDBP_EINVAL, "l2g entry out of range [0, nglobal)");
    const bool dir = masked && dirichlet[g];
    hl2g[s] = dir ? -int(g) - 1 : int(g);
    hoff[g + 1] += 1;
  }
  for (int64_t g = 0; g < P.nglobal; ++g) hoff[g + 1] += hoff[g];
  {
    std::vector<int> fill(hoff.begin(), hoff.end() - 1);
    for (int64_t s = 0; s < nloc; ++s) hslots[fill[l2g[s]]++] = int(s);
  }
  if (masked)
    for (int64_t g = 0; g < P.nglobal; ++g)
      if (dirichlet[g]) hoff[g] = int(unsigned(hoff[g]) | 0x80000000u);

  std::vector<double> hb(basis_doubles(p1, qdef));
  std::copy(basis.J.begin(), basis.J.end(), hb.begin());
  std::copy(basis.Dh.begin(), basis.Dh.end(), hb.begin() + size_t(qdef) * p1);
  std::copy(basis.Dq.begin(), basis.Dq.end(), hb.begin() + 2 * size_t(qdef) * p1);
  std::copy(basis.w.begin(), basis.w.end(), hb.begin() + 2 * size_t(qdef) * p1 + size_t(qdef) * qdef);

  const int nc = c->ncomp;
  const int64_t n = P.nglobal;
  CK(c, dalloc(&c->d_l2g, nloc));
  CK(c, dalloc(&c->d_off, n + 1));
  CK(c, dalloc(&c->d_slots, nloc));
  CK(c, dalloc(&c->d_basis, hb.size()));
  if (c->op_kind == kStiff) CK(c, dalloc(&c->d_G, size_t(P.nelem) * 6 * Q3));
  CK(c, dalloc(&c->d_Mq, size_t(P.nelem) * Q3));
  CK(c, dalloc(&c->d_dinv, n));
  if (c->colloc) CK(c, dalloc(&c->d_mdiag, n));
  CK(c, dalloc(&c->d_wl, size_t(nloc) * nc));
  CK(c, dalloc(&c->d_r, size_t(n) * nc));
  CK(c, dalloc(&c->d_p, size_t(n) * nc));
  CK(c, dalloc(&c->d_ax, size_t(n) * nc));
  CK(c, dalloc(&c->d_state, 1));
  CK(c, dalloc(&c->d_scal, 4));
  CK(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_scal), 4 * sizeof(double)));
  CK(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_state), sizeof(SolveState)));
  CK(c, cudaEventCreate(&c->ev0));
  CK(c, cudaEventCreate(&c->ev1));
  cudaStream_t s = c->stream;
  CK(c, cudaMemcpyAsync(c->d_l2g, hl2g.data(), sizeof(int) * nloc, cudaMemcpyHostToDevice, s));
  CK(c, cudaMemcpyAsync(c->d_off, hoff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
  CK(c, cudaMemcpyAsync(c->d_slots, hslots.data(), sizeof(int) * nloc, cudaMemcpyHostToDevice, s));
  CK(c, cudaMemcpyAsync(c->d_basis, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, s));
  CK(c, cudaMemsetAsync(c->d_state, 0, sizeof(SolveState), s));

  DeviceMesh& m = c->mesh;
  m.p1 = p1;
  m.q = qdef;
  m.ncomp = nc;
  m.bp = P.bp;
  m.colloc = c->colloc;
  m.nelem = P.nelem;
  m.nglobal = n;
  m.l2g = c->d_l2g;
  m.off = c->d_off;
  m.slots = c->d_slots;
  m.basis = c->d_basis;

  int nb_apply = elem_blocks(m);
  if (c->colloc) nb_apply = std::max(nb_apply, std::max(int(P.nelem), elem_lp_blocks(m)));
  else if (P.arith == CEEDBP_ARITH_DF64) nb_apply = std::max(nb_apply, elem_dfgl_blocks(m));
  CK(c, dalloc(&c->d_part_apply, size_t(nb_apply) * nc));
  CK(c, dalloc(&c->d_part_vec, size_t(vec_blocks(n)) * 3 * nc));

  // ---- geometric and mass factors from the nodal coordinates
  {
    double* d_coords = nullptr;
    double* d_kappa = nullptr;
    double* d_scratch = nullptr;
    CK(c, dalloc(&d_coords, size_t(nloc) * 3));
    CK(c, dalloc(&d_scratch, geom_scratch_doubles(geom_blocks(P.nelem), qdef)));
    CK(c, cudaMemcpyAsync(d_coords, coords, sizeof(double) * nloc * 3, cudaMemcpyHostToDevice, s));
    if (kappa && c->op_kind == kStiff) {
      CK(c, dalloc(&d_kappa, size_t(P.nelem) * Q3));
      CK(c, cudaMemcpyAsync(d_kappa, kappa, sizeof(double) * P.nelem * Q3, cudaMemcpyHostToDevice, s));
    }
    cudaError_t e = cudaSuccess;
    if (d_kappa) {
      // keep the coefficient-free factors for ceedbp_set_kappa and the adjoint gradient
      e = dalloc(&c->d_Ghat, size_t(P.nelem) * 6 * Q3);
      if (e == cudaSuccess) e = launch_geom(m, d_coords, nullptr, c->d_Ghat, c->d_Mq, d_scratch, s);
      if (e == cudaSuccess) e = launch_scale_factors(c->d_Ghat, d_kappa, c->d_G, P.nelem, int(Q3), s);
    } else {
      e = launch_geom(m, d_coords, nullptr, c->d_G, c->d_Mq, d_scratch, s);
    }
    if (e == cudaSuccess && recompute) {
      e = dalloc(&c->d_X, size_t(nloc) * 3);
      if (e == cudaSuccess) e = launch_coords_soa(d_coords, c->d_X, P.nelem, int(P3), s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_coords);
    cudaFree(d_scratch);
    if (d_kappa) cudaFree(d_kappa);
    if (e != cudaSuccess) return cuda_fail(c, e, "geometric factors");
  }
  // ---- Jacobi diagonal: local diag(A^e) (or diag(B^e)), summed by Q^T, inverted
  CK(c, launch_local_diag(m, c->op_kind, c->d_G, c->d_Mq, c->d_wl, s));
  if (nc == 3) {
    // the local diagonal is per scalar node; sum it with the scalar layout
    DeviceMesh m1 = m;
    m1.ncomp = 1;
    CK(c, launch_gs(m1, c->d_wl, c->d_r, 0, s));
  } else {
    CK(c, launch_gs(m, c->d_wl, c->d_r, 0, s));
  }
  CK(c, launch_dinv(c->d_off, c->d_r, c->d_dinv, n, s));
  if (c->colloc) {
    DeviceMesh m1 = m;
    m1.ncomp = 1;
    CK(c, launch_local_diag(m1, kMass, nullptr, c->d_Mq, c->d_wl, s));
    CK(c, launch_gs(m1, c->d_wl, c->d_mdiag, 0, s));
  }
  if (recompute) {
    // from here on the element kernel forms G from the coordinates
    CK(c, cudaStreamSynchronize(s));
    cudaFree(c->d_G);
    c->d_G = nullptr;
    m.X = c->d_X;
    int nb = elem_blocks(m);
    if (nb > nb_apply) {
      cudaFree(c->d_part_apply);
      c->d_part_apply = nullptr;
      CK(c, dalloc(&c->d_part_apply, size_t(nb) * nc));
    }
  }
  // One launch of every element kernel this context uses, so that their
  // one-time attribute setup happens here and never inside a graph capture.
  {
    ElemArgs a{};
    a.u = c->d_r;
    a.wl = c->d_wl;
    a.G = c->op_kind == kStiff ? c->d_G : c->d_Mq;
    a.mask_in = 1;
    CK(c, launch_elem(m, c->op_kind, a, s));
    if (!c->colloc && c->op_kind == kStiff) {
      a.G = c->d_Mq;
      CK(c, launch_elem(m, kMass, a, s));
    }
  }
  if (c->arith == CEEDBP_ARITH_DF64 && !c->colloc) {
    // BP1 / BP3: pair copies of the factors (G, or the mass factors), of J and Dq, and of dinv;
    // the kernel sets its splitters from its own line data and the tables' row sums
    const size_t ng = c->op_kind == kStiff ? size_t(P.nelem) * 6 * Q3 : size_t(P.nelem) * Q3;
    CK(c, dalloc(&c->d_Gdf, ng));
    CK(c, dalloc(&c->d_Ddf, size_t(qdef) * p1 + size_t(qdef) * qdef));
    CK(c, dalloc(&c->d_dinvdf, n));
    CK(c, launch_f64_to_df(c->op_kind == kStiff ? c->d_G : c->d_Mq, c->d_Gdf, int64_t(ng), s));
    CK(c, launch_f64_to_df(c->d_dinv, c->d_dinvdf, n, s));
    std::vector<dfloat> hd(size_t(qdef) * p1 + size_t(qdef) * qdef);
    auto to_pair = [](double d) { const float hi = float(d); return dfloat{hi, float(d - double(hi))}; };
    for (size_t i = 0; i < basis.J.size(); ++i) hd[i] = to_pair(basis.J[i]);
    for (size_t i = 0; i < basis.Dq.size(); ++i) hd[basis.J.size() + i] = to_pair(basis.Dq[i]);
    CK(c, cudaMemcpyAsync(c->d_Ddf, hd.data(), sizeof(dfloat) * hd.size(), cudaMemcpyHostToDevice, s));
    CK(c, cudaStreamSynchronize(s));
    ElemDfArgs a = {};
    a.u_f64 = c->d_r;
    a.wl = reinterpret_cast<dfloat*>(c->d_wl);
    a.G = c->d_Gdf;
    a.D = c->d_Ddf;
    a.mask_in = 1;
    a.fault = &c->d_state->fault;
    CK(c, launch_elem_df(m, a, s));  // one launch outside any capture (attribute setup)
    CK(c, cudaStreamSynchronize(s));
  } else if (c->arith == CEEDBP_ARITH_DF64) {
    // pair copies of G, D and dinv; splitter bounds from the row and column sums of |D|
    const size_t ng = size_t(P.nelem) * 6 * Q3;
    CK(c, dalloc(&c->d_Gdf, ng));
    CK(c, dalloc(&c->d_Ddf, size_t(p1) * p1));
    CK(c, dalloc(&c->d_dinvdf, n));
    CK(c, launch_f64_to_df(c->d_G, c->d_Gdf, int64_t(ng), s));
    CK(c, launch_f64_to_df(c->d_dinv, c->d_dinvdf, n, s));
    std::vector<dfloat> hd(size_t(p1) * p1);
    double rmax = 0.0, cmax = 0.0;
    for (int a = 0; a < p1; ++a) {
      double rs = 0.0, cs = 0.0;
      for (int b = 0; b < p1; ++b) {
        const double d = basis.Dq[size_t(a) * p1 + b];
        const float hi = float(d);
        hd[size_t(a) * p1 + b] = dfloat{hi, float(d - double(hi))};
        rs += std::fabs(d);
        cs += std::fabs(basis.Dq[size_t(b) * p1 + a]);
      }
      rmax = std::max(rmax, rs);
      cmax = std::max(cmax, cs);
    }
    c->dnorm_row = float(rmax * (1.0 + 1e-6));
    c->dnorm_col = float(cmax * (1.0 + 1e-6));
    CK(c, cudaMemcpyAsync(c->d_Ddf, hd.data(), sizeof(dfloat) * hd.size(), cudaMemcpyHostToDevice, s));
    CK(c, set_df_dconst(p1, hd.data(), s));
    CK(c, cudaStreamSynchronize(s));
    ElemDfArgs a{};
    a.u_f64 = c->d_r;
    a.wl = reinterpret_cast<dfloat*>(c->d_wl);
    a.G = c->d_Gdf;
    a.D = c->d_Ddf;
    a.dnorm_row = c->dnorm_row;
    a.dnorm_col = c->dnorm_col;
    a.mask_in = 1;
    a.fault = &c->d_state->fault;
    CK(c, cudaStreamSynchronize(s));
    // autotuner: elements per block and G staging of the pair kernel, timed on this mesh
    int cand_eb[32], cand_st[32], cand_ns[32];
    int ncand = pair_shape_candidates(c, m, cand_eb, cand_st, cand_ns, 32);
    if (c->pipelined_only) {  // keep the pipelined shapes when there are any
      int np = 0;
      for (int k = 0; k < ncand; ++k)
        if (cand_st[k] == 2) {
          cand_eb[np] = cand_eb[k];
          cand_st[np] = cand_st[k];
          cand_ns[np++] = cand_ns[k];
        }
      if (np > 0) ncand = np;
    }
    if (ncand == 0) return fail(c, CEEDBP_EUNSUPPORTED, "no launchable shape for the pair kernel at this order");
    // The launches are timed as a solve makes them: with the fused (u, w) and its last-block
    // grid reduction, whose cost grows with the number of blocks (shapes with short sequences
    // have more).  The state lets every launch run to the end (fixed, active, never stopping);
    // it is zeroed again after tuning.
    {
      SolveState hs{};
      hs.ncomp = c->ncomp;
      hs.fixed = 1;
      for (int q = 0; q < c->ncomp; ++q) {
        hs.c[q].active = 1;
        hs.c[q].rz = 1.0;
      }
      CK(c, cudaMemcpyAsync(c->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
      CK(c, cudaStreamSynchronize(s));
    }
    a.partials = c->d_part_apply;
    a.state = c->d_state;
    // two passes over the candidates, each shape's best of the two (the first pass also warms
    // the clocks and caches that the first candidates would otherwise be timed without)
    std::vector<float> best_ms(size_t(ncand), 1e30f);
    for (int pass = 0; pass < 2 && ncand > 1; ++pass) {
      for (int k = 0; k < ncand; ++k) {
        m.tune_eb = cand_eb[k];
        m.tune_stage = cand_st[k];
        m.tune_ns = cand_ns[k];
        {  // warm-up of this shape
          const cudaError_t e = launch_elem_df(m, a, s);
          if (e != cudaSuccess)
            return cuda_fail(c, e, ("pair kernel shape eb=" + std::to_string(m.tune_eb) + " schedule=" +
                                    std::to_string(m.tune_stage) + " seq=" + std::to_string(m.tune_ns)).c_str());
        }
        CK(c, cudaEventRecord(c->ev0, s));
        for (int r = 0; r < 3; ++r) CK(c, launch_elem_df(m, a, s));
        CK(c, cudaEventRecord(c->ev1, s));
        CK(c, cudaEventSynchronize(c->ev1));
        float ms = 0.0f;
        CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        best_ms[size_t(k)] = std::min(best_ms[size_t(k)], ms);
      }
    }
    int best_k = 0;
    for (int k = 1; k < ncand; ++k)
      if (best_ms[size_t(k)] < best_ms[size_t(best_k)]) best_k = k;
    m.tune_eb = cand_eb[best_k];
    m.tune_stage = cand_st[best_k];
    m.tune_ns = cand_ns[best_k];
    CK(c, launch_elem_df(m, a, s));  // the chosen shape, launched once outside any capture
    CK(c, cudaStreamSynchronize(s));
    CK(c, cudaMemsetAsync(c->d_state, 0, sizeof(SolveState), s));
  }
  // the static scratch of ceedbp_apply_noalloc: its device address on this device, looked up here
  CK(c, noalloc_scratch_refresh());
  CK(c, cudaStreamSynchronize(s));
  return CEEDBP_OK;
}

}  // namespace

namespace ceedbp {
void set_thread_error(const std::string& msg) { g_setup_error = msg; }
ceedbp_status setup_context(ceedbp_ctx* c, const double* coords, const int64_t* l2g, const uint8_t* dirichlet,
                            const double* kappa) {
  return setup_impl(c, coords, l2g, dirichlet, kappa);
}
void release_context(ceedbp_ctx* c) { release(c); }
}  // namespace ceedbp

namespace {

// Helmholtz term beta B u of Eq. (17) for the stiffness kernels (beta = 0: none)
void set_helmholtz_args(const ceedbp_ctx* c, ElemArgs& a) {
  if (c->op_kind == kStiff && c->beta != 0.0) {
    a.Mq = c->d_Mq;
    a.beta = c->beta;
  }
}

ElemDfArgs df_args(ceedbp_ctx* c) {
  ElemDfArgs a{};
  a.fault = &c->d_state->fault;
  a.first_wait = c->wait_polls;
  a.G = c->d_Gdf;
  a.D = c->d_Ddf;
  a.dnorm_row = c->dnorm_row;
  a.dnorm_col = c->dnorm_col;
  a.wl = reinterpret_cast<dfloat*>(c->d_wl);
  return a;
}

// Events recorded inside a capture become event-record nodes of the graph.
void mark(ceedbp_ctx* c, int i, bool capturing) {
  if (capturing) cudaEventRecordWithFlags(c->prof[i], c->stream, cudaEventRecordExternal);
  else cudaEventRecord(c->prof[i], c->stream);
}

// inner iterations of defect correction; mode CEEDBP_MIXED_FP32, _BF16 or _FP32_TC
void run_inner_iterations(ceedbp_ctx* c, int mode, int n) {
  const DeviceMesh& m = c->mesh;
  const int bf16 = mode == CEEDBP_MIXED_BF16 ? 1 : 0;
  ElemLpArgs a{};
  a.u = c->d_pin;
  a.wl = reinterpret_cast<float*>(c->d_wl);
  a.G = bf16 ? c->d_Gbf : static_cast<const void*>(c->d_G32);
  a.partials = c->d_part_apply;
  a.state = c->d_state;
  for (int i = 0; i < n; ++i) {
    if (mode == CEEDBP_MIXED_FP32_TC) launch_elem_tc(m, a, c->stream);
    else launch_elem_lp(m, a, bf16, c->stream);
    launch_inner_update(m, bf16, a.wl, c->d_xin, c->d_rin, c->d_pin, c->d_dinv32, c->d_part_vec, c->d_state,
                        c->stream);
    launch_inner_dir(m, bf16, c->d_rin, c->d_pin, c->d_dinv32, c->d_state, c->stream);
  }
}

void run_iterations(ceedbp_ctx* c, double* x, int n, bool profile = false, bool capturing = false) {
  const DeviceMesh& m = c->mesh;
  ElemArgs a{};
  a.u = c->d_p;
  a.wl = c->d_wl;
  a.G = c->op_kind == kStiff ? c->d_G : c->d_Mq;
  set_helmholtz_args(c, a);
  a.partials = c->d_part_apply;
  a.state = c->d_state;
  a.mask_in = 0;  // p is zero on Dirichlet nodes
  a.skip_dirichlet_out = 1;
  ElemDfArgs da = df_args(c);
  da.u_df = reinterpret_cast<const dfloat*>(c->d_p);
  da.partials = c->d_part_apply;
  da.state = c->d_state;
  da.skip_dirichlet_out = 1;
  dfloat* xd = reinterpret_cast<dfloat*>(c->d_ax);
  dfloat* rd = reinterpret_cast<dfloat*>(c->d_r);
  dfloat* pd = reinterpret_cast<dfloat*>(c->d_p);
  const dfloat* wd = reinterpret_cast<const dfloat*>(c->d_wl);
  const bool df = c->arith == CEEDBP_ARITH_DF64;
  for (int i = 0; i < n; ++i) {
    if (profile) mark(c, 4 * i + 0, capturing);
    if (df) launch_elem_df(m, da, c->stream);
    else launch_elem(m, c->op_kind, a, c->stream);
    if (profile) mark(c, 4 * i + 1, capturing);
    if (df) launch_update_df(m, wd, xd, rd, pd, c->d_dinvdf, c->d_part_vec, c->d_state, c->stream);
    else launch_pcg_update(m, c->d_wl, x, c->d_r, c->d_p, c->d_dinv, c->d_part_vec, c->d_state, c->stream);
    if (profile) mark(c, 4 * i + 2, capturing);
    if (df) launch_dir_df(m, rd, pd, c->d_dinvdf, c->d_state, c->stream);
    else launch_pcg_dir(m, c->d_r, c->d_p, c->d_dinv, c->d_state, c->stream);
    if (profile) mark(c, 4 * i + 3, capturing);
  }
}

ceedbp_status ensure_prof_events(ceedbp_ctx* c, int n) {
  while (int(c->prof.size()) < 4 * n) {
    cudaEvent_t e = nullptr;
    CK(c, cudaEventCreate(&e));
    c->prof.push_back(e);
  }
  return CEEDBP_OK;
}

ceedbp_status graph_for(ceedbp_ctx* c, double* x, int n, int profile, cudaGraphExec_t* out, int mode = 0) {
  for (auto& g : c->graphs)
    if (g.x == x && g.n == n && g.profile == profile && g.mode == mode) {
      *out = g.exec;
      return CEEDBP_OK;
    }
  cudaGraph_t graph = nullptr;
  CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  if (mode == 0) run_iterations(c, x, n, profile != 0, true);
  else run_inner_iterations(c, mode, n);
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  if (c->graphs.size() >= 8) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back({x, n, profile, mode, exec});
  *out = exec;
  return CEEDBP_OK;
}

ceedbp_status solve_mixed(ceedbp_ctx* c, const double* b, double* x, const ceedbp_solve_opts& o,
                          ceedbp_solve_info* info) {
  const int bf16 = o.mixed == CEEDBP_MIXED_BF16 ? 1 : 0;
  if (o.mixed != CEEDBP_MIXED_FP32 && o.mixed != CEEDBP_MIXED_BF16 && o.mixed != CEEDBP_MIXED_FP32_TC)
    return fail(c, CEEDBP_EINVAL, "unknown mixed mode");
  if (!c->colloc) return fail(c, CEEDBP_EUNSUPPORTED, "defect correction is built for BP5 and BP6");
  if ((bf16 && !c->d_Gbf) || (!bf16 && !c->d_G32) || !c->d_xin ||
      (o.mixed == CEEDBP_MIXED_FP32_TC && !c->tc_ready))
    return fail(c, CEEDBP_EINVAL, "call ceedbp_prepare_mixed for this precision first");
  const int nc = c->ncomp;
  const int64_t n = c->prm.nglobal;
  cudaStream_t s = c->stream;
  const double inner_tol = o.inner_tol > 0.0 ? o.inner_tol : (bf16 ? 3e-3 : 1e-4);
  const int inner_maxit = o.inner_maxit > 0 ? o.inner_maxit : o.maxit;
  const int outer_maxit = o.outer_maxit > 0 ? o.outer_maxit : 50;
  const bool graphs = o.use_graph && s != nullptr;
  unsigned* ticket = &c->d_state->ticket[kTicketResidual];
  // ||b||
  CK(c, launch_residual(c->mesh, b, nullptr, c->d_r, c->d_part_vec, ticket, c->d_outer, s));
  CK(c, cudaMemcpyAsync(c->h_outer, c->d_outer, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  double bb[3] = {0, 0, 0}, rr[3] = {0, 0, 0};
  for (int k = 0; k < nc; ++k) bb[k] = rr[k] = c->h_outer[k];
  if (o.x0_nonzero) {
    ceedbp_status st = ceedbp_apply(c, x, c->d_ax);
    if (st != CEEDBP_OK) return st;
    CK(c, launch_residual(c->mesh, b, c->d_ax, c->d_r, c->d_part_vec, ticket, c->d_outer, s));
    CK(c, cudaMemcpyAsync(c->h_outer, c->d_outer, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    for (int k = 0; k < nc; ++k) rr[k] = c->h_outer[k];
  } else {
    CK(c, cudaMemsetAsync(x, 0, sizeof(double) * n * nc, s));
  }
  CK(c, cudaEventRecord(c->ev0, s));
  int outer = 0, inner_total[3] = {0, 0, 0};
  ceedbp_status result = CEEDBP_OK;
  while (true) {
    bool done = true, finite = true;
    for (int k = 0; k < nc; ++k) {
      if (!std::isfinite(rr[k]) || !std::isfinite(bb[k])) finite = false;
      if (rr[k] > o.tol * o.tol * bb[k]) done = false;
    }
    if (!finite) {
      result = CEEDBP_EBREAKDOWN;
      break;
    }
    if (done) break;
    if (outer >= outer_maxit) {
      result = CEEDBP_ENOCONV;
      break;
    }
    double scale[3] = {0, 0, 0}, norm[3] = {0, 0, 0};
    for (int k = 0; k < nc; ++k) {
      norm[k] = std::sqrt(rr[k]);
      scale[k] = norm[k] > 0.0 ? 1.0 / norm[k] : 0.0;
    }
    CK(c, launch_inner_init(c->mesh, bf16, c->d_r, scale, c->d_dinv32, c->d_xin, c->d_rin, c->d_pin, c->d_part_vec,
                            c->d_state, inner_tol, s));
    int its = 0;
    while (its < inner_maxit) {
      const int k = std::min(o.chunk, inner_maxit - its);
      if (graphs) {
        cudaGraphExec_t exec = nullptr;
        ceedbp_status st = graph_for(c, nullptr, k, 0, &exec, o.mixed);
        if (st != CEEDBP_OK) return st;
        CK(c, cudaGraphLaunch(exec, s));
      } else {
        run_inner_iterations(c, o.mixed, k);
        CK(c, cudaGetLastError());
      }
      CK(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
      CK(c, cudaStreamSynchronize(s));
      its += k;
      if (c->h_state->stop) break;
    }
    for (int k = 0; k < nc; ++k) {
      inner_total[k] += c->h_state->c[k].iters;
      if (c->h_state->c[k].status == CEEDBP_EBREAKDOWN) result = CEEDBP_EBREAKDOWN;
    }
    if (result == CEEDBP_EBREAKDOWN) break;
    CK(c, launch_correct(c->mesh, x, c->d_xin, norm, s));
    ceedbp_status st = ceedbp_apply(c, x, c->d_ax);
    if (st != CEEDBP_OK) return st;
    CK(c, launch_residual(c->mesh, b, c->d_ax, c->d_r, c->d_part_vec, ticket, c->d_outer, s));
    CK(c, cudaMemcpyAsync(c->h_outer, c->d_outer, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    for (int k = 0; k < nc; ++k) rr[k] = c->h_outer[k];
    ++outer;
  }
  CK(c, cudaEventRecord(c->ev1, s));
  CK(c, cudaEventSynchronize(c->ev1));
  float ms = 0.0f;
  CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int k = 0; k < nc; ++k) {
      info->iters[k] = inner_total[k];
      info->res_norm[k] = std::sqrt(rr[k]);
      info->b_norm[k] = std::sqrt(bb[k]);
      info->rel_res[k] = bb[k] > 0.0 ? std::sqrt(rr[k] / bb[k]) : 0.0;
    }
    info->device_ms = ms;
    info->outer_iters = outer;
    info->status = result;
  }
  if (result == CEEDBP_ENOCONV) c->err = "defect correction: outer_maxit reached before the tolerance";
  if (result == CEEDBP_EBREAKDOWN) c->err = "defect correction: inner CG breakdown";
  return result;
}

}  // namespace

extern "C" {

ceedbp_status ceedbp_prepare_mixed(ceedbp_ctx* c, int precision) {
  if (!c) return fail(c, CEEDBP_EINVAL, "null context");
  if (precision != CEEDBP_MIXED_FP32 && precision != CEEDBP_MIXED_BF16 && precision != CEEDBP_MIXED_FP32_TC)
    return fail(c, CEEDBP_EINVAL, "precision must be CEEDBP_MIXED_FP32, _BF16 or _FP32_TC");
  if (!c->colloc) return fail(c, CEEDBP_EUNSUPPORTED, "defect correction is built for BP5 and BP6");
  if (precision == CEEDBP_MIXED_FP32_TC && !elem_tc_supported(c->mesh))
    return fail(c, CEEDBP_EUNSUPPORTED, "the tensor-core inner operator is built for order 7 (p1 = 8)");
  if (c->d_X) return fail(c, CEEDBP_EUNSUPPORTED, "this call needs stored geometric factors (geom = STORED)");
  if (c->beta != 0.0) return fail(c, CEEDBP_EUNSUPPORTED, "defect correction is built for beta = 0");
  const int64_t n = c->prm.nglobal, nc = c->ncomp;
  const int64_t ng = c->prm.nelem * 6 * int64_t(c->q) * c->q * c->q;
  cudaStream_t s = c->stream;
  if (!c->d_xin) {
    CK(c, dalloc(&c->d_xin, size_t(n * nc)));
    CK(c, dalloc(&c->d_rin, size_t(n * nc)));
    CK(c, dalloc(reinterpret_cast<float**>(&c->d_pin), size_t(n * nc)));
    CK(c, dalloc(&c->d_dinv32, size_t(n)));
    CK(c, dalloc(&c->d_outer, 3));
    CK(c, cudaMallocHost(reinterpret_cast<void**>(&c->h_outer), 3 * sizeof(double)));
    CK(c, launch_narrow(c->d_dinv, c->d_dinv32, n, 0, s));
  }
  if (precision != CEEDBP_MIXED_BF16 && !c->d_G32) {
    CK(c, dalloc(&c->d_G32, size_t(ng)));
    CK(c, launch_narrow(c->d_G, c->d_G32, ng, 0, s));
  }
  if (precision == CEEDBP_MIXED_BF16 && !c->d_Gbf) {
    CK(c, cudaMalloc(&c->d_Gbf, sizeof(uint16_t) * size_t(ng)));
    CK(c, launch_narrow(c->d_G, c->d_Gbf, ng, 1, s));
  }
  // prime the inner element kernel outside any capture (one-time attribute setup)
  ElemLpArgs a{};
  a.u = c->d_pin;
  a.wl = reinterpret_cast<float*>(c->d_wl);
  a.G = precision == CEEDBP_MIXED_BF16 ? c->d_Gbf : static_cast<const void*>(c->d_G32);
  CK(c, cudaMemsetAsync(c->d_pin, 0, sizeof(float) * size_t(n * nc), s));
  if (precision == CEEDBP_MIXED_FP32_TC) {
    CK(c, launch_elem_tc(c->mesh, a, s));
    c->tc_ready = true;
  } else {
    CK(c, launch_elem_lp(c->mesh, a, precision == CEEDBP_MIXED_BF16, s));
  }
  CK(c, cudaStreamSynchronize(s));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_setup(const ceedbp_params* params, const double* coords, const int64_t* l2g,
                           const uint8_t* dirichlet, const double* kappa, void* stream, ceedbp_ctx** out) {
  if (!params || !out) return fail(nullptr, CEEDBP_EINVAL, "params and out are required");
  *out = nullptr;
  ceedbp_ctx* c = new (std::nothrow) ceedbp_ctx();
  if (!c) return fail(nullptr, CEEDBP_ENOMEM, "host allocation failed");
  c->prm = *params;
  c->stream = static_cast<cudaStream_t>(stream);
  ceedbp_status st = setup_impl(c, coords, l2g, dirichlet, kappa);
  if (st != CEEDBP_OK) {
    g_setup_error = c->err;
    release(c);
    delete c;
    return st;
  }
  *out = c;
  return CEEDBP_OK;
}

ceedbp_status ceedbp_apply(ceedbp_ctx* c, const double* u, double* w) {
  if (!c || !u || !w) return fail(c, CEEDBP_EINVAL, "null argument");
  if (c->arith == CEEDBP_ARITH_DF64) {
    ElemDfArgs da = df_args(c);
    da.u_f64 = u;
    da.mask_in = 1;
    da.skip_dirichlet_out = 1;
    CK(c, launch_elem_df(c->mesh, da, c->stream));
    CK(c, launch_gs_df(c->mesh, reinterpret_cast<const dfloat*>(c->d_wl), w, 1, c->stream));
    return CEEDBP_OK;
  }
  ElemArgs a{};
  a.u = u;
  a.wl = c->d_wl;
  a.G = c->op_kind == kStiff ? c->d_G : c->d_Mq;
  set_helmholtz_args(c, a);
  a.mask_in = c->prm.bp != 1 && c->prm.bp != 2;
  a.skip_dirichlet_out = 1;
  CK(c, launch_elem(c->mesh, c->op_kind, a, c->stream));
  CK(c, launch_gs(c->mesh, c->d_wl, w, 1, c->stream));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_mass(ceedbp_ctx* c, const double* u, double* w) {
  if (!c || !u || !w) return fail(c, CEEDBP_EINVAL, "null argument");
  if (c->colloc) {
    CK(c, launch_scale(c->d_mdiag, u, w, c->prm.nglobal, c->ncomp, c->stream));
    return CEEDBP_OK;
  }
  ElemArgs a{};
  a.u = u;
  a.wl = c->d_wl;
  a.G = c->d_Mq;
  a.mask_in = 0;
  a.skip_dirichlet_out = 0;
  CK(c, launch_elem(c->mesh, kMass, a, c->stream));
  CK(c, launch_gs(c->mesh, c->d_wl, w, 0, c->stream));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_jacobi(ceedbp_ctx* c, double* dinv) {
  if (!c || !dinv) return fail(c, CEEDBP_EINVAL, "null argument");
  CK(c, cudaMemcpyAsync(dinv, c->d_dinv, sizeof(double) * c->prm.nglobal, cudaMemcpyDeviceToDevice, c->stream));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_solve(ceedbp_ctx* c, const double* b, double* x, const ceedbp_solve_opts* opts,
                           ceedbp_solve_info* info) {
  if (!c || !b || !x) return fail(c, CEEDBP_EINVAL, "null argument");
  ceedbp_solve_opts o{1e-8, 10000, 0, 32, 1, 0, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (o.chunk <= 0) o.chunk = 32;
  if (o.maxit <= 0) o.maxit = 10000;
  if (!(o.tol >= 0.0)) return fail(c, CEEDBP_EINVAL, "tol must be >= 0");
  if (o.mixed != CEEDBP_MIXED_NONE) return solve_mixed(c, b, x, o, info);
  const int nc = c->ncomp;
  const int64_t n = c->prm.nglobal;
  cudaStream_t s = c->stream;
  const double* ax = nullptr;
  if (o.x0_nonzero) {
    ceedbp_status st = ceedbp_apply(c, x, c->d_ax);
    if (st != CEEDBP_OK) return st;
    ax = c->d_ax;
  } else {
    CK(c, cudaMemsetAsync(x, 0, sizeof(double) * n * nc, s));
  }
  const int fixed = o.fixed_iters > 0 ? 1 : 0;
  const bool df = c->arith == CEEDBP_ARITH_DF64;
  if (df)
    CK(c, launch_init_df(c->mesh, b, ax, x, reinterpret_cast<dfloat*>(c->d_ax), reinterpret_cast<dfloat*>(c->d_r),
                         reinterpret_cast<dfloat*>(c->d_p), c->d_dinvdf, o.x0_nonzero, c->d_part_vec, c->d_state,
                         o.tol, fixed, s));
  else
    CK(c, launch_pcg_init(c->mesh, b, ax, x, c->d_r, c->d_p, c->d_dinv, c->d_part_vec, c->d_state, o.tol, fixed, s));
  const int limit = fixed ? o.fixed_iters : o.maxit;
  const bool graphs = o.use_graph && s != nullptr;
  const bool profile = o.profile != 0;
  if (profile) {
    ceedbp_status st = ensure_prof_events(c, std::min(o.chunk, limit));
    if (st != CEEDBP_OK) return st;
  }
  double kms[3] = {0.0, 0.0, 0.0};
  int kcount = 0;
  CK(c, cudaEventRecord(c->ev0, s));
  int done = 0;
  while (done < limit) {
    const int k = std::min(o.chunk, limit - done);
    if (graphs) {
      cudaGraphExec_t exec = nullptr;
      ceedbp_status st = graph_for(c, x, k, profile ? 1 : 0, &exec);
      if (st != CEEDBP_OK) return st;
      CK(c, cudaGraphLaunch(exec, s));
    } else {
      run_iterations(c, x, k, profile, false);
      CK(c, cudaGetLastError());
    }
    CK(c, cudaEventRecord(c->ev1, s));
    CK(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (profile) {
      for (int i = 0; i < k; ++i) {
        float t = 0.0f;
        for (int j = 0; j < 3; ++j) {
          CK(c, cudaEventElapsedTime(&t, c->prof[4 * i + j], c->prof[4 * i + j + 1]));
          kms[j] += t;
        }
      }
      kcount += k;
    }
    done += k;
    if (c->h_state->stop) break;
  }
  if (df) {
    CK(c, launch_df_to_f64(reinterpret_cast<const dfloat*>(c->d_ax), x, n * nc, s));
    CK(c, cudaStreamSynchronize(s));
  }
  float ms = 0.0f;
  CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  ceedbp_status result = CEEDBP_OK;
  const SolveState& h = *c->h_state;
  if (h.fault) {
    c->err = "a kernel gave up a bounded wait for its staging copy (in this solve, or in an apply since the "
             "last check); results are invalid";
    CK(c, cudaMemsetAsync(&c->d_state->fault, 0, sizeof(int), s));
    CK(c, cudaStreamSynchronize(s));
    return CEEDBP_ECUDA;
  }
  for (int comp = 0; comp < nc; ++comp) {
    if (h.c[comp].status == CEEDBP_EBREAKDOWN) result = CEEDBP_EBREAKDOWN;
    else if (!fixed && h.c[comp].active && result == CEEDBP_OK) result = CEEDBP_ENOCONV;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int comp = 0; comp < nc; ++comp) {
      const CompScalars& cs = h.c[comp];
      info->iters[comp] = cs.iters;
      info->res_norm[comp] = std::sqrt(std::max(cs.rr, 0.0));
      info->b_norm[comp] = std::sqrt(std::max(cs.bb, 0.0));
      info->rel_res[comp] = cs.bb > 0.0 ? info->res_norm[comp] / info->b_norm[comp] : 0.0;
    }
    info->device_ms = ms;
    for (int j = 0; j < 3; ++j) info->kernel_ms[j] = kcount ? kms[j] / kcount : 0.0;
    info->status = result;
  }
  if (result == CEEDBP_EBREAKDOWN) c->err = "CG breakdown (p^T A p <= 0 or non-finite scalar)";
  if (result == CEEDBP_ENOCONV) c->err = "maxit reached before the tolerance";
  return result;
}

ceedbp_status ceedbp_set_kappa(ceedbp_ctx* c, const double* kappa) {
  if (!c || !kappa) return fail(c, CEEDBP_EINVAL, "null argument");
  if (c->op_kind != kStiff) return fail(c, CEEDBP_EUNSUPPORTED, "kappa applies to stiffness problems");
  if (c->d_X) return fail(c, CEEDBP_EUNSUPPORTED, "this call needs stored geometric factors (geom = STORED)");
  cudaStream_t s = c->stream;
  const int64_t q3 = int64_t(c->q) * c->q * c->q;
  const size_t ng = size_t(c->prm.nelem) * 6 * q3;
  if (!c->d_Ghat) {  // set up with kappa = 1: the current factors are coefficient-free
    CK(c, dalloc(&c->d_Ghat, ng));
    CK(c, cudaMemcpyAsync(c->d_Ghat, c->d_G, sizeof(double) * ng, cudaMemcpyDeviceToDevice, s));
  }
  CK(c, launch_scale_factors(c->d_Ghat, kappa, c->d_G, c->prm.nelem, int(q3), s));
  const DeviceMesh& m = c->mesh;
  CK(c, launch_local_diag(m, kStiff, c->d_G, c->d_Mq, c->d_wl, s));
  DeviceMesh m1 = m;
  m1.ncomp = 1;
  CK(c, launch_gs(m1, c->d_wl, c->d_r, 0, s));
  CK(c, launch_dinv(c->d_off, c->d_r, c->d_dinv, c->prm.nglobal, s));
  if (c->d_Gdf) {
    CK(c, launch_f64_to_df(c->d_G, c->d_Gdf, int64_t(ng), s));
    CK(c, launch_f64_to_df(c->d_dinv, c->d_dinvdf, c->prm.nglobal, s));
  }
  if (c->d_G32) CK(c, launch_narrow(c->d_G, c->d_G32, int64_t(ng), 0, s));
  if (c->d_Gbf) CK(c, launch_narrow(c->d_G, c->d_Gbf, int64_t(ng), 1, s));
  if (c->d_dinv32) CK(c, launch_narrow(c->d_dinv, c->d_dinv32, c->prm.nglobal, 0, s));
  if (c->beta != 0.0) return ceedbp_set_helmholtz(c, c->beta);  // Jacobi of A(kappa) + beta B
  return CEEDBP_OK;
}

ceedbp_status ceedbp_misfit(ceedbp_ctx* c, const double* u, const double* ustar, double* rhs, double* J) {
  if (!c || !u || !ustar || !rhs) return fail(c, CEEDBP_EINVAL, "null argument");
  if (!c->colloc || c->ncomp != 1) return fail(c, CEEDBP_EUNSUPPORTED, "misfit is built for BP5");
  cudaStream_t s = c->stream;
  CK(c, launch_misfit(c->mesh, c->d_mdiag, u, ustar, rhs, c->d_part_vec, &c->d_state->ticket[kTicketResidual],
                      c->d_scal, s));
  CK(c, cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  if (J) *J = c->h_scal[0];
  return CEEDBP_OK;
}

ceedbp_status ceedbp_kappa_gradient(ceedbp_ctx* c, const double* u, const double* lam, double* g) {
  if (!c || !u || !lam || !g) return fail(c, CEEDBP_EINVAL, "null argument");
  if (!c->colloc || c->ncomp != 1) return fail(c, CEEDBP_EUNSUPPORTED, "the adjoint gradient is built for BP5");
  if (c->p1 > 12) return fail(c, CEEDBP_EUNSUPPORTED, "the adjoint gradient is built for orders 1..11");
  if (c->d_X) return fail(c, CEEDBP_EUNSUPPORTED, "this call needs stored geometric factors (geom = STORED)");
  CK(c, launch_kappa_grad(c->mesh, u, lam, c->d_Ghat ? c->d_Ghat : c->d_G, g, c->stream));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_tile_info(const ceedbp_ctx* c, int* eb, int* staged, int* seq) {
  if (!c) return CEEDBP_EINVAL;
  const bool df = c->arith == CEEDBP_ARITH_DF64;
  if (eb) *eb = df ? c->mesh.tune_eb : 0;
  if (staged) *staged = df ? c->mesh.tune_stage : 0;
  if (seq) *seq = df && c->mesh.tune_stage >= 2 ? c->mesh.tune_ns : 1;
  return CEEDBP_OK;
}

namespace {
__global__ void helm_diag_kernel(const double* __restrict__ dA, const double* __restrict__ dB, double beta,
                                 double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = dA[i] + beta * dB[i];
}

__global__ void iota_kernel(int* v, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    v[i] = int(i);
}
}  // namespace

ceedbp_status ceedbp_set_helmholtz(ceedbp_ctx* c, double beta) {
  if (!c) return fail(c, CEEDBP_EINVAL, "null context");
  if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(c, CEEDBP_EINVAL, "beta must be finite and >= 0");
  if (c->op_kind != kStiff) return fail(c, CEEDBP_EUNSUPPORTED, "the Helmholtz term applies to BP3-BP6");
  if (c->arith != CEEDBP_ARITH_FP64 || c->d_G32 || c->d_Gbf)
    return fail(c, CEEDBP_EUNSUPPORTED, "the Helmholtz term is built for the FP64 arithmetic without defect correction");
  cudaStream_t s = c->stream;
  CK(c, cudaStreamSynchronize(s));
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);  // captured launches hold the old beta
  c->graphs.clear();
  c->beta = beta;
  // Jacobi diagonal of A + beta B: assembled diagonals of both, combined, inverted
  const DeviceMesh& m = c->mesh;
  DeviceMesh m1 = m;
  m1.ncomp = 1;
  const int64_t n = c->prm.nglobal;
  const double* G = c->d_G;
  if (!G && c->d_X) return fail(c, CEEDBP_EUNSUPPORTED, "the Helmholtz term needs stored geometric factors");
  CK(c, launch_local_diag(m, kStiff, G, c->d_Mq, c->d_wl, s));
  CK(c, launch_gs(m1, c->d_wl, c->d_r, 0, s));
  CK(c, launch_local_diag(m1, kMass, nullptr, c->d_Mq, c->d_wl, s));
  CK(c, launch_gs(m1, c->d_wl, c->d_ax, 0, s));
  helm_diag_kernel<<<1216, 256, 0, s>>>(c->d_r, c->d_ax, beta, c->d_r, n);
  CK(c, cudaGetLastError());
  CK(c, launch_dinv(c->d_off, c->d_r, c->d_dinv, n, s));
  // one launch of the element kernel variant now in use, outside any graph capture
  ElemArgs a{};
  a.u = c->d_r;
  a.wl = c->d_wl;
  a.G = c->d_G;
  a.mask_in = 1;
  set_helmholtz_args(c, a);
  CK(c, launch_elem(m, kStiff, a, s));
  CK(c, cudaStreamSynchronize(s));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_bk_apply(ceedbp_ctx* c, const double* uL, double* wL) {
  if (!c || !uL || !wL) return fail(c, CEEDBP_EINVAL, "null argument");
  cudaStream_t s = c->stream;
  const int64_t nloc = c->prm.nelem * int64_t(c->p1) * c->p1 * c->p1;
  if (!c->d_l2g_id) {
    // the element kernels gather through l2g; the identity map makes them read u_L directly
    CK(c, dalloc(&c->d_l2g_id, nloc));
    iota_kernel<<<1216, 256, 0, s>>>(c->d_l2g_id, nloc);
    CK(c, cudaGetLastError());
  }
  DeviceMesh mb = c->mesh;
  mb.l2g = c->d_l2g_id;
  if (c->arith == CEEDBP_ARITH_DF64) {
    ElemDfArgs a = df_args(c);
    a.u_f64 = uL;
    a.mask_in = 0;
    a.skip_dirichlet_out = 0;
    CK(c, launch_elem_df(mb, a, s));
    CK(c, launch_df_to_f64(reinterpret_cast<const dfloat*>(c->d_wl), wL, nloc * c->ncomp, s));
    return CEEDBP_OK;
  }
  ElemArgs a{};
  a.u = uL;
  a.wl = wL;
  a.G = c->op_kind == kStiff ? c->d_G : c->d_Mq;
  set_helmholtz_args(c, a);
  a.mask_in = 0;
  a.skip_dirichlet_out = 0;
  CK(c, launch_elem(mb, c->op_kind, a, s));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_set_tile(ceedbp_ctx* c, int eb, int schedule, int seq) {
  if (!c) return fail(c, CEEDBP_EINVAL, "null context");
  if (c->arith != CEEDBP_ARITH_DF64 || !c->colloc)
    return fail(c, CEEDBP_EUNSUPPORTED, "tile shapes belong to the pair path of BP5/BP6");
  int cand_eb[32], cand_st[32], cand_ns[32];
  const int ncand = pair_shape_candidates(c, c->mesh, cand_eb, cand_st, cand_ns, 32);
  int hit = -1;
  for (int k = 0; k < ncand; ++k)
    if (cand_eb[k] == eb && cand_st[k] == schedule && (schedule < 2 || cand_ns[k] == seq)) hit = k;
  if (hit < 0) return fail(c, CEEDBP_EINVAL, "not a launchable shape of the pair kernel at this order");
  cudaStream_t s = c->stream;
  CK(c, cudaStreamSynchronize(s));
  // captured iterations hold the previous shape
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  c->mesh.tune_eb = cand_eb[hit];
  c->mesh.tune_stage = cand_st[hit];
  c->mesh.tune_ns = cand_ns[hit];
  ElemDfArgs a = df_args(c);
  a.u_f64 = c->d_r;
  a.mask_in = 1;
  CK(c, launch_elem_df(c->mesh, a, s));  // one launch outside any capture (attribute setup)
  CK(c, cudaStreamSynchronize(s));
  return CEEDBP_OK;
}

ceedbp_status ceedbp_set_wait_limit(ceedbp_ctx* c, int polls) {
  if (!c) return fail(c, CEEDBP_EINVAL, "null context");
  if (c->arith != CEEDBP_ARITH_DF64) return fail(c, CEEDBP_EUNSUPPORTED, "bounded waits belong to the pair path");
  CK(c, cudaStreamSynchronize(c->stream));
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);  // captured launches hold the old limit
  c->graphs.clear();
  c->wait_polls = polls < 0 ? kDefaultWaitPolls : polls;
  return CEEDBP_OK;
}

ceedbp_status ceedbp_check(ceedbp_ctx* c) {
  if (!c) return fail(c, CEEDBP_EINVAL, "null context");
  cudaStream_t s = c->stream;
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(&c->h_state->fault, &c->d_state->fault, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  if (c->h_state->fault) {
    CK(c, cudaMemsetAsync(&c->d_state->fault, 0, sizeof(int), s));
    CK(c, cudaStreamSynchronize(s));
    return fail(c, CEEDBP_ECUDA, "a kernel gave up a bounded wait for its staging copy; results since the last "
                                 "check are invalid");
  }
  return CEEDBP_OK;
}

ceedbp_status ceedbp_destroy(ceedbp_ctx* c) {
  if (!c) return CEEDBP_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  release(c);
  delete c;
  return CEEDBP_OK;
}

const char* ceedbp_last_error(const ceedbp_ctx* c) { return c ? c->err.c_str() : g_setup_error.c_str(); }

}  // extern "C"
