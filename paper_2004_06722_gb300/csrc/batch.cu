// Batched BP5 solves: many independent problems of uneven size and order.
//
// Problems of one order are concatenated into one block-diagonal mesh (node and
// element numbers offset per problem) and set up as one context, so geometry,
// gather-scatter offsets and the Jacobi diagonal come from the single-problem
// setup.  Every CG phase is then one launch per order group for all of its
// problems: element blocks and vector blocks never straddle two problems, and
// each problem's inner products are reduced over its own contiguous range of
// blocks by the last of them to finish (fixed order, no float atomics), which
// writes that problem's alpha or beta.  Converged problems drop out (their
// blocks return at once); an iteration chunk is one captured CUDA graph.
// The arithmetic is that of the problems' params: native FP64 (the FP64
// element kernels, even-odd at odd orders, with FP64 vector kernels) or
// FP64-accurate FP32 pairs (the pipelined pair kernel, whose per-order
// elements per block come from the setup autotuner of each group).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "kernel_args.h"

namespace ceedbp {

ceedbp_status setup_context(ceedbp_ctx* c, const double* coords, const int64_t* l2g, const uint8_t* dirichlet,
                            const double* kappa);
void release_context(ceedbp_ctx* c);

namespace {

constexpr int kVecChunk = 1024;  // nodes per vector block

struct VecTable {
  const int* prob;   // [nblocks]
  const int* n0;     // [nblocks] first global node (concatenated numbering)
  const int* n1;     // [nblocks] end node
  const int* blk0;   // [nprob] first block of each problem
  const int* nblk;   // [nprob]
};

__global__ void batch_init_kernel(const int* __restrict__ off, const double* __restrict__ bcat,
                                  dfloat* __restrict__ x, dfloat* __restrict__ r, dfloat* __restrict__ p,
                                  const dfloat* __restrict__ dinv, VecTable vt, double* partials, BatchScalars* bst,
                                  BatchGlobal* glob, double tol) {
  __shared__ double red[32 * 3];
  const int pr = vt.prob[blockIdx.x];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
    const double bv = dir ? 0.0 : bcat[g];
    const dfloat rv = f64_to_df(bv);
    const dfloat zv = dw_mul(dinv[g], rv);
    x[g] = dfloat{0.0f, 0.0f};
    r[g] = rv;
    p[g] = zv;
    acc[0] += df_to_f64(dw_mul(rv, zv));
    acc[1] += bv * bv;
    acc[2] += bv * bv;
  }
  const int b0 = vt.blk0[pr];
  if (grid_sum_last<3>(acc, partials + 3 * size_t(b0), vt.nblk[pr], int(blockIdx.x) - b0,
                       &bst[pr].ticket[kTicketInit], red)) {
    if (threadIdx.x == 0) {
      CompScalars& cs = bst[pr].c;
      cs.rz = acc[0];
      cs.rr = acc[1];
      cs.bb = acc[2];
      cs.tol2 = tol * tol * cs.bb;
      cs.alpha = cs.beta = cs.pAp = 0.0;
      cs.iters = 0;
      cs.status = isfinite(cs.rz) && isfinite(cs.rr) ? CEEDBP_OK : CEEDBP_EBREAKDOWN;
      cs.active = cs.status == CEEDBP_OK && cs.rr > cs.tol2 ? 1 : 0;
      if (cs.active) atomicAdd(&glob->active_count, 1);
    }
  }
}

__global__ void batch_update_kernel(const int* __restrict__ off, const int* __restrict__ slots,
                                    const dfloat* __restrict__ wl, dfloat* __restrict__ x, dfloat* __restrict__ r,
                                    const dfloat* __restrict__ p, const dfloat* __restrict__ dinv, VecTable vt,
                                    double* partials, BatchScalars* bst, BatchGlobal* glob) {
  __shared__ double red[32 * 2];
  const int pr = vt.prob[blockIdx.x];
  if (!bst[pr].c.active) return;
  const dfloat alpha = f64_to_df(bst[pr].c.alpha);
  dfloat rz{0.0f, 0.0f}, rr{0.0f, 0.0f};
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) {
    const int o0 = __ldg(off + g);
    if (o0 < 0) continue;
    const int o1 = __ldg(off + g + 1) & 0x7fffffff;
    dfloat w{0.0f, 0.0f};
    for (int k = o0; k < o1; ++k) w = dw_add(w, wl[__ldg(slots + k)]);
    const dfloat rv = dw_add(r[g], dw_neg(dw_mul(alpha, w)));
    x[g] = dw_add(x[g], dw_mul(alpha, p[g]));
    r[g] = rv;
    rz = dw_add(rz, dw_mul(rv, dw_mul(dinv[g], rv)));
    rr = dw_add(rr, dw_mul(rv, rv));
  }
  double acc[2] = {df_to_f64(rz), df_to_f64(rr)};
  const int b0 = vt.blk0[pr];
  if (grid_sum_last<2>(acc, partials + 2 * size_t(b0), vt.nblk[pr], int(blockIdx.x) - b0,
                       &bst[pr].ticket[kTicketUpdate], red)) {
    if (threadIdx.x == 0) {
      CompScalars& cs = bst[pr].c;
      cs.beta = cs.rz != 0.0 ? acc[0] / cs.rz : 0.0;
      cs.rz = acc[0];
      cs.rr = acc[1];
      cs.iters += 1;
      if (!isfinite(acc[0])) cs.status = CEEDBP_EBREAKDOWN;
      if (cs.rr <= cs.tol2 || cs.status != CEEDBP_OK) {
        cs.active = 0;
        atomicSub(&glob->active_count, 1);
      }
    }
  }
}

__global__ void batch_dir_kernel(const int* __restrict__ off, const dfloat* __restrict__ r, dfloat* __restrict__ p,
                                 const dfloat* __restrict__ dinv, VecTable vt, const BatchScalars* bst) {
  const int pr = vt.prob[blockIdx.x];
  if (!bst[pr].c.active) return;
  const dfloat beta = f64_to_df(bst[pr].c.beta);
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) {
    if (__ldg(off + g) < 0) continue;
    p[g] = dw_add(dw_mul(dinv[g], r[g]), dw_mul(beta, p[g]));
  }
}

// ---- FP64 arithmetic: the same three phases on double vectors
__global__ void batch_init64_kernel(const int* __restrict__ off, const double* __restrict__ bcat,
                                    double* __restrict__ x, double* __restrict__ r, double* __restrict__ p,
                                    const double* __restrict__ dinv, VecTable vt, double* partials,
                                    BatchScalars* bst, BatchGlobal* glob, double tol) {
  __shared__ double red[32 * 3];
  const int pr = vt.prob[blockIdx.x];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
    const double bv = dir ? 0.0 : bcat[g];
    const double zv = dinv[g] * bv;
    x[g] = 0.0;
    r[g] = bv;
    p[g] = zv;
    acc[0] += bv * zv;
    acc[1] += bv * bv;
    acc[2] += bv * bv;
  }
  const int b0 = vt.blk0[pr];
  if (grid_sum_last<3>(acc, partials + 3 * size_t(b0), vt.nblk[pr], int(blockIdx.x) - b0,
                       &bst[pr].ticket[kTicketInit], red)) {
    if (threadIdx.x == 0) {
      CompScalars& cs = bst[pr].c;
      cs.rz = acc[0];
      cs.rr = acc[1];
      cs.bb = acc[2];
      cs.tol2 = tol * tol * cs.bb;
      cs.alpha = cs.beta = cs.pAp = 0.0;
      cs.iters = 0;
      cs.status = isfinite(cs.rz) && isfinite(cs.rr) ? CEEDBP_OK : CEEDBP_EBREAKDOWN;
      cs.active = cs.status == CEEDBP_OK && cs.rr > cs.tol2 ? 1 : 0;
      if (cs.active) atomicAdd(&glob->active_count, 1);
    }
  }
}

__global__ void batch_update64_kernel(const int* __restrict__ off, const int* __restrict__ slots,
                                      const double* __restrict__ wl, double* __restrict__ x,
                                      double* __restrict__ r, const double* __restrict__ p,
                                      const double* __restrict__ dinv, VecTable vt, double* partials,
                                      BatchScalars* bst, BatchGlobal* glob) {
  __shared__ double red[32 * 2];
  const int pr = vt.prob[blockIdx.x];
  if (!bst[pr].c.active) return;
  const double alpha = bst[pr].c.alpha;
  double acc[2] = {0.0, 0.0};
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) {
    const int o0 = __ldg(off + g);
    if (o0 < 0) continue;
    const int o1 = __ldg(off + g + 1) & 0x7fffffff;
    double w = 0.0;
    for (int k = o0; k < o1; ++k) w += wl[__ldg(slots + k)];
    const double rv = r[g] - alpha * w;
    x[g] += alpha * p[g];
    r[g] = rv;
    acc[0] += rv * dinv[g] * rv;
    acc[1] += rv * rv;
  }
  const int b0 = vt.blk0[pr];
  if (grid_sum_last<2>(acc, partials + 2 * size_t(b0), vt.nblk[pr], int(blockIdx.x) - b0,
                       &bst[pr].ticket[kTicketUpdate], red)) {
    if (threadIdx.x == 0) {
      CompScalars& cs = bst[pr].c;
      cs.beta = cs.rz != 0.0 ? acc[0] / cs.rz : 0.0;
      cs.rz = acc[0];
      cs.rr = acc[1];
      cs.iters += 1;
      if (!isfinite(acc[0])) cs.status = CEEDBP_EBREAKDOWN;
      if (cs.rr <= cs.tol2 || cs.status != CEEDBP_OK) {
        cs.active = 0;
        atomicSub(&glob->active_count, 1);
      }
    }
  }
}

__global__ void batch_dir64_kernel(const int* __restrict__ off, const double* __restrict__ r, double* __restrict__ p,
                                   const double* __restrict__ dinv, VecTable vt, const BatchScalars* bst) {
  const int pr = vt.prob[blockIdx.x];
  if (!bst[pr].c.active) return;
  const double beta = bst[pr].c.beta;
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) {
    if (__ldg(off + g) < 0) continue;
    p[g] = dinv[g] * r[g] + beta * p[g];
  }
}

__global__ void batch_scatter64_kernel(const double* __restrict__ src, double* const* __restrict__ dst, VecTable vt,
                                       const int* __restrict__ node0) {
  const int pr = vt.prob[blockIdx.x];
  double* d = dst[pr];
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) d[g - node0[pr]] = src[g];
}

// b of every problem into the concatenated vector / x back to every problem
__global__ void batch_gather_kernel(const double* const* __restrict__ src, double* __restrict__ dst, VecTable vt,
                                    const int* __restrict__ node0) {
  const int pr = vt.prob[blockIdx.x];
  const double* s = src[pr];
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x) dst[g] = s[g - node0[pr]];
}

__global__ void batch_scatter_kernel(const dfloat* __restrict__ src, double* const* __restrict__ dst, VecTable vt,
                                     const int* __restrict__ node0) {
  const int pr = vt.prob[blockIdx.x];
  double* d = dst[pr];
  for (int g = vt.n0[blockIdx.x] + threadIdx.x; g < vt.n1[blockIdx.x]; g += blockDim.x)
    d[g - node0[pr]] = df_to_f64(src[g]);
}

}  // namespace
}  // namespace ceedbp

using namespace ceedbp;

struct BatchGroup {
  ceedbp_ctx* ctx = nullptr;
  std::vector<int> members;    // problem ids
  std::vector<int64_t> node0;  // first node of each member in the concatenated numbering
  int nblk_e = 0, nblk_v = 0;
  int* d_tab = nullptr;        // all int tables in one allocation
  VecTable vt{};
  const int* blk_prob = nullptr;
  const int* blk_e0 = nullptr;
  const int* blk_n = nullptr;
  const int* prob_blk0 = nullptr;
  const int* prob_nblk = nullptr;
  const int* d_node0 = nullptr;
  BatchScalars* d_bst = nullptr;
  double* d_part = nullptr;    // [max(nblk_e, 3 nblk_v)]
  double* d_bcat = nullptr;
  const double** d_src = nullptr;
  double** d_dst = nullptr;
};

struct GraphChunk {
  int n;
  cudaGraphExec_t exec;
};

struct ceedbp_batch {
  int nprob = 0;
  int arith = CEEDBP_ARITH_DF64;
  cudaStream_t stream = nullptr;
  std::vector<BatchGroup> groups;
  std::vector<int> prob_group, prob_index;
  BatchGlobal* d_glob = nullptr;
  BatchGlobal* h_glob = nullptr;
  std::vector<BatchScalars> h_bst;
  std::vector<GraphChunk> graphs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

ceedbp_status bfail(ceedbp_batch* b, ceedbp_status st, const std::string& msg) {
  if (b) b->err = msg;
  g_batch_error = msg;
  return st;
}

#define BCK(b, call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? CEEDBP_ENOMEM : CEEDBP_ECUDA,         \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

void batch_release(ceedbp_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : b->groups) {
    void* ptrs[] = {g.d_tab, g.d_bst, g.d_part, g.d_bcat, g.d_src, g.d_dst};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    if (g.ctx) {
      release_context(g.ctx);
      delete g.ctx;
    }
  }
  if (b->d_glob) cudaFree(b->d_glob);
  if (b->h_glob) cudaFreeHost(b->h_glob);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
}

void run_batch_iterations(ceedbp_batch* b, int n) {
  for (int it = 0; it < n; ++it)
    for (auto& g : b->groups) {
      ceedbp_ctx* c = g.ctx;
      if (b->arith == CEEDBP_ARITH_FP64) {
        ElemArgs a{};
        a.u = c->d_p;
        a.wl = c->d_wl;
        a.G = c->d_G;
        a.partials = g.d_part;
        a.skip_dirichlet_out = 1;
        a.blk_prob = g.blk_prob;
        a.blk_e0 = g.blk_e0;
        a.blk_n = g.blk_n;
        a.prob_blk0 = g.prob_blk0;
        a.prob_nblk = g.prob_nblk;
        a.bst = g.d_bst;
        a.batch_blocks = g.nblk_e;
        launch_elem(c->mesh, kStiff, a, b->stream);
        batch_update64_kernel<<<g.nblk_v, 256, 0, b->stream>>>(c->mesh.off, c->mesh.slots, c->d_wl, c->d_ax,
                                                               c->d_r, c->d_p, c->d_dinv, g.vt, g.d_part, g.d_bst,
                                                               b->d_glob);
        batch_dir64_kernel<<<g.nblk_v, 256, 0, b->stream>>>(c->mesh.off, c->d_r, c->d_p, c->d_dinv, g.vt, g.d_bst);
        continue;
      }
      ElemDfArgs a{};
      a.u_df = reinterpret_cast<const dfloat*>(c->d_p);
      a.wl = reinterpret_cast<dfloat*>(c->d_wl);
      a.G = c->d_Gdf;
      a.D = c->d_Ddf;
      a.dnorm_row = c->dnorm_row;
      a.dnorm_col = c->dnorm_col;
      a.partials = g.d_part;
      a.skip_dirichlet_out = 1;
      a.fault = &b->d_glob->fault;
      a.blk_prob = g.blk_prob;
      a.blk_e0 = g.blk_e0;
      a.blk_n = g.blk_n;
      a.prob_blk0 = g.prob_blk0;
      a.prob_nblk = g.prob_nblk;
      a.bst = g.d_bst;
      a.batch_blocks = g.nblk_e;
      launch_elem_df(c->mesh, a, b->stream);
      batch_update_kernel<<<g.nblk_v, 256, 0, b->stream>>>(
          c->mesh.off, c->mesh.slots, reinterpret_cast<const dfloat*>(c->d_wl), reinterpret_cast<dfloat*>(c->d_ax),
          reinterpret_cast<dfloat*>(c->d_r), reinterpret_cast<const dfloat*>(c->d_p), c->d_dinvdf, g.vt, g.d_part,
          g.d_bst, b->d_glob);
      batch_dir_kernel<<<g.nblk_v, 256, 0, b->stream>>>(c->mesh.off, reinterpret_cast<const dfloat*>(c->d_r),
                                                        reinterpret_cast<dfloat*>(c->d_p), c->d_dinvdf, g.vt,
                                                        g.d_bst);
    }
}

}  // namespace

extern "C" {

ceedbp_status ceedbp_batch_setup(int nprob, const ceedbp_params* params, const double* const* coords,
                                 const int64_t* const* l2g, const uint8_t* const* dirichlet, void* stream,
                                 ceedbp_batch** out) {
  if (nprob < 1 || !params || !coords || !l2g || !dirichlet || !out)
    return bfail(nullptr, CEEDBP_EINVAL, "null argument or nprob < 1");
  *out = nullptr;
  ceedbp_batch* b = new (std::nothrow) ceedbp_batch();
  if (!b) return bfail(nullptr, CEEDBP_ENOMEM, "host allocation failed");
  b->nprob = nprob;
  b->stream = static_cast<cudaStream_t>(stream);
  auto fail_out = [&](ceedbp_status st) {
    batch_release(b);
    delete b;
    return st;
  };
  std::map<int, std::vector<int>> by_order;
  b->arith = params[0].arith;
  if (b->arith != CEEDBP_ARITH_FP64 && b->arith != CEEDBP_ARITH_DF64)
    return fail_out(bfail(nullptr, CEEDBP_EINVAL, "unknown arith"));
  for (int p = 0; p < nprob; ++p) {
    if (params[p].bp != 5) return fail_out(bfail(nullptr, CEEDBP_EUNSUPPORTED, "batched solves are built for BP5"));
    if (params[p].arith != b->arith)
      return fail_out(bfail(nullptr, CEEDBP_EINVAL, "all problems of a batch take the same arith"));
    if (params[p].geom != CEEDBP_GEOM_STORED)
      return fail_out(bfail(nullptr, CEEDBP_EUNSUPPORTED, "batched solves use stored geometric factors"));
    if (params[p].order < 1 || params[p].order > kMaxOrder)
      return fail_out(bfail(nullptr, CEEDBP_EINVAL, "order must be in 1..15"));
    by_order[params[p].order].push_back(p);
  }
  b->prob_group.assign(nprob, 0);
  b->prob_index.assign(nprob, 0);
  for (auto& kv : by_order) {
    const int N = kv.first, p1 = N + 1, P3 = p1 * p1 * p1;
    BatchGroup g;
    g.members = kv.second;
    int64_t E = 0, ng = 0;
    for (int p : g.members) {
      g.node0.push_back(ng);
      E += params[p].nelem;
      ng += params[p].nglobal;
    }
    std::vector<double> cc(size_t(E) * P3 * 3);
    std::vector<int64_t> ll(size_t(E) * P3);
    std::vector<uint8_t> dd(ng);
    int64_t eo = 0;
    for (size_t k = 0; k < g.members.size(); ++k) {
      const int p = g.members[k];
      const int64_t Ep = params[p].nelem, np = params[p].nglobal;
      std::memcpy(cc.data() + size_t(eo) * P3 * 3, coords[p], sizeof(double) * Ep * P3 * 3);
      for (int64_t s = 0; s < Ep * P3; ++s) {
        const int64_t gid = l2g[p][s];
        if (gid < 0 || gid >= np) return fail_out(bfail(nullptr, CEEDBP_EINVAL, "l2g entry out of range"));
        ll[size_t(eo) * P3 + s] = gid + g.node0[k];
      }
      std::memcpy(dd.data() + g.node0[k], dirichlet[p], np);
      b->prob_group[p] = int(b->groups.size());
      b->prob_index[p] = int(k);
      eo += Ep;
    }
    g.ctx = new (std::nothrow) ceedbp_ctx();
    if (!g.ctx) return fail_out(bfail(nullptr, CEEDBP_ENOMEM, "host allocation failed"));
    g.ctx->prm = ceedbp_params{5, N, 0, E, ng, b->arith, CEEDBP_GEOM_STORED};
    g.ctx->stream = b->stream;
    g.ctx->pipelined_only = true;  // pair arithmetic on large concatenated meshes: the pipelined schedule wins
    ceedbp_status st = setup_context(g.ctx, cc.data(), ll.data(), dd.data(), nullptr);
    if (st != CEEDBP_OK) {
      const std::string msg = g.ctx->err;
      b->groups.push_back(g);
      return fail_out(bfail(nullptr, st, "group setup: " + msg));
    }
    // block tables: elements per block of the FP64 kernel, or the autotuned shape of the pair
    // kernel at this order (elements per block, times the sequence length of the pipelined schedule)
    int eb = 0;
    if (b->arith == CEEDBP_ARITH_FP64) {
      eb = elem_stiff_per_block(g.ctx->mesh);
      if (eb < 1) {
        b->groups.push_back(g);
        return fail_out(bfail(nullptr, CEEDBP_EUNSUPPORTED, "no FP64 batched element kernel at this order"));
      }
    } else {
      eb = std::max(1, g.ctx->mesh.tune_eb) * (g.ctx->mesh.tune_stage == 2 ? g.ctx->mesh.tune_ns : 1);
    }
    std::vector<int> bp, be0, bn, pb0, pnb, vp, vn0, vn1, vb0, vnb, n0;
    eo = 0;
    for (size_t k = 0; k < g.members.size(); ++k) {
      const int p = g.members[k];
      pb0.push_back(int(bp.size()));
      for (int64_t e = 0; e < params[p].nelem; e += eb) {
        bp.push_back(int(k));
        be0.push_back(int(eo + e));
        bn.push_back(int(std::min<int64_t>(eb, params[p].nelem - e)));
      }
      pnb.push_back(int(bp.size()) - pb0.back());
      eo += params[p].nelem;
      vb0.push_back(int(vp.size()));
      for (int64_t v = 0; v < params[p].nglobal; v += kVecChunk) {
        vp.push_back(int(k));
        vn0.push_back(int(g.node0[k] + v));
        vn1.push_back(int(g.node0[k] + std::min<int64_t>(v + kVecChunk, params[p].nglobal)));
      }
      vnb.push_back(int(vp.size()) - vb0.back());
      n0.push_back(int(g.node0[k]));
    }
    g.nblk_e = int(bp.size());
    g.nblk_v = int(vp.size());
    std::vector<int> tab;
    auto put = [&](const std::vector<int>& v) {
      const size_t o = tab.size();
      tab.insert(tab.end(), v.begin(), v.end());
      return o;
    };
    const size_t o_bp = put(bp), o_be0 = put(be0), o_bn = put(bn), o_pb0 = put(pb0), o_pnb = put(pnb);
    const size_t o_vp = put(vp), o_vn0 = put(vn0), o_vn1 = put(vn1), o_vb0 = put(vb0), o_vnb = put(vnb);
    const size_t o_n0 = put(n0);
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&g.d_tab), sizeof(int) * tab.size()));
    BCK(b, cudaMemcpyAsync(g.d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, b->stream));
    g.blk_prob = g.d_tab + o_bp;
    g.blk_e0 = g.d_tab + o_be0;
    g.blk_n = g.d_tab + o_bn;
    g.prob_blk0 = g.d_tab + o_pb0;
    g.prob_nblk = g.d_tab + o_pnb;
    g.vt = VecTable{g.d_tab + o_vp, g.d_tab + o_vn0, g.d_tab + o_vn1, g.d_tab + o_vb0, g.d_tab + o_vnb};
    g.d_node0 = g.d_tab + o_n0;
    const size_t m = g.members.size();
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&g.d_bst), sizeof(BatchScalars) * m));
    BCK(b, cudaMemsetAsync(g.d_bst, 0, sizeof(BatchScalars) * m, b->stream));
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&g.d_part), sizeof(double) * std::max<size_t>(g.nblk_e, 3 * size_t(g.nblk_v))));
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&g.d_bcat), sizeof(double) * ng));
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&g.d_src), sizeof(double*) * m));
    BCK(b, cudaMalloc(reinterpret_cast<void**>(&g.d_dst), sizeof(double*) * m));
    b->groups.push_back(g);
  }
  BCK(b, cudaMalloc(reinterpret_cast<void**>(&b->d_glob), sizeof(BatchGlobal)));
  BCK(b, cudaMallocHost(reinterpret_cast<void**>(&b->h_glob), sizeof(BatchGlobal)));
  BCK(b, cudaEventCreate(&b->ev0));
  BCK(b, cudaEventCreate(&b->ev1));
  BCK(b, cudaStreamSynchronize(b->stream));
  *out = b;
  return CEEDBP_OK;
}

ceedbp_status ceedbp_batch_solve(ceedbp_batch* b, const double* const* b_dev, double* const* x_dev,
                                 const ceedbp_solve_opts* opts, ceedbp_solve_info* infos) {
  if (!b || !b_dev || !x_dev) return bfail(b, CEEDBP_EINVAL, "null argument");
  ceedbp_solve_opts o{1e-8, 10000, 0, 32, 1, 0, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (o.chunk <= 0) o.chunk = 32;
  if (o.maxit <= 0) o.maxit = 10000;
  cudaStream_t s = b->stream;
  BCK(b, cudaMemsetAsync(b->d_glob, 0, sizeof(BatchGlobal), s));
  for (auto& g : b->groups) {
    std::vector<const double*> src;
    std::vector<double*> dst;
    for (int p : g.members) {
      src.push_back(b_dev[p]);
      dst.push_back(x_dev[p]);
    }
    BCK(b, cudaMemcpyAsync(g.d_src, src.data(), sizeof(double*) * src.size(), cudaMemcpyHostToDevice, s));
    BCK(b, cudaMemcpyAsync(g.d_dst, dst.data(), sizeof(double*) * dst.size(), cudaMemcpyHostToDevice, s));
    batch_gather_kernel<<<g.nblk_v, 256, 0, s>>>(g.d_src, g.d_bcat, g.vt, g.d_node0);
    ceedbp_ctx* c = g.ctx;
    if (b->arith == CEEDBP_ARITH_FP64)
      batch_init64_kernel<<<g.nblk_v, 256, 0, s>>>(c->mesh.off, g.d_bcat, c->d_ax, c->d_r, c->d_p, c->d_dinv, g.vt,
                                                   g.d_part, g.d_bst, b->d_glob, o.tol);
    else
      batch_init_kernel<<<g.nblk_v, 256, 0, s>>>(c->mesh.off, g.d_bcat, reinterpret_cast<dfloat*>(c->d_ax),
                                                 reinterpret_cast<dfloat*>(c->d_r), reinterpret_cast<dfloat*>(c->d_p),
                                                 c->d_dinvdf, g.vt, g.d_part, g.d_bst, b->d_glob, o.tol);
  }
  BCK(b, cudaGetLastError());
  const bool graphs = o.use_graph && s != nullptr;
  BCK(b, cudaEventRecord(b->ev0, s));
  int done = 0;
  BCK(b, cudaMemcpyAsync(b->h_glob, b->d_glob, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, s));
  BCK(b, cudaStreamSynchronize(s));
  while (done < o.maxit && b->h_glob->active_count > 0) {
    const int k = std::min(o.chunk, o.maxit - done);
    if (graphs) {
      cudaGraphExec_t exec = nullptr;
      for (auto& gc : b->graphs)
        if (gc.n == k) exec = gc.exec;
      if (!exec) {
        cudaGraph_t graph = nullptr;
        BCK(b, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        run_batch_iterations(b, k);
        BCK(b, cudaStreamEndCapture(s, &graph));
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        BCK(b, e);
        b->graphs.push_back({k, exec});
      }
      BCK(b, cudaGraphLaunch(exec, s));
    } else {
      run_batch_iterations(b, k);
      BCK(b, cudaGetLastError());
    }
    BCK(b, cudaEventRecord(b->ev1, s));
    BCK(b, cudaMemcpyAsync(b->h_glob, b->d_glob, sizeof(BatchGlobal), cudaMemcpyDeviceToHost, s));
    BCK(b, cudaStreamSynchronize(s));
    done += k;
    if (b->h_glob->fault) return bfail(b, CEEDBP_ECUDA, "a kernel gave up a bounded wait; results are invalid");
  }
  if (done == 0) BCK(b, cudaEventRecord(b->ev1, s));
  for (auto& g : b->groups) {
    if (b->arith == CEEDBP_ARITH_FP64)
      batch_scatter64_kernel<<<g.nblk_v, 256, 0, s>>>(g.ctx->d_ax, g.d_dst, g.vt, g.d_node0);
    else
      batch_scatter_kernel<<<g.nblk_v, 256, 0, s>>>(reinterpret_cast<const dfloat*>(g.ctx->d_ax), g.d_dst, g.vt,
                                                    g.d_node0);
  }
  BCK(b, cudaGetLastError());
  BCK(b, cudaStreamSynchronize(s));
  float ms = 0.0f;
  BCK(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  ceedbp_status result = CEEDBP_OK;
  for (auto& g : b->groups) {
    std::vector<BatchScalars> h(g.members.size());
    BCK(b, cudaMemcpy(h.data(), g.d_bst, sizeof(BatchScalars) * h.size(), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < g.members.size(); ++k) {
      const CompScalars& cs = h[k].c;
      if (cs.status == CEEDBP_EBREAKDOWN) result = CEEDBP_EBREAKDOWN;
      else if (cs.active && result == CEEDBP_OK) result = CEEDBP_ENOCONV;
      if (infos) {
        ceedbp_solve_info& in = infos[g.members[k]];
        std::memset(&in, 0, sizeof(in));
        in.iters[0] = cs.iters;
        in.res_norm[0] = std::sqrt(std::max(cs.rr, 0.0));
        in.b_norm[0] = std::sqrt(std::max(cs.bb, 0.0));
        in.rel_res[0] = cs.bb > 0.0 ? in.res_norm[0] / in.b_norm[0] : 0.0;
        in.device_ms = ms;
        in.status = cs.status == CEEDBP_EBREAKDOWN ? CEEDBP_EBREAKDOWN : (cs.active ? CEEDBP_ENOCONV : CEEDBP_OK);
      }
    }
  }
  return result;
}

ceedbp_status ceedbp_batch_destroy(ceedbp_batch* b) {
  if (!b) return CEEDBP_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
  return CEEDBP_OK;
}

const char* ceedbp_batch_last_error(const ceedbp_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
