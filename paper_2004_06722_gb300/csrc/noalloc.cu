// ceedbp_apply_noalloc: the operator apply of ceedbp_apply, with the
// element-local scratch w_L taken from a fixed array that is part of the
// library's device image instead of the context's cudaMalloc'd buffer.
//
// Who needs it: callers that must not call cudaMalloc (or anything that may
// allocate) at the point where they apply the operator.  Examples are code
// that runs while another thread holds a CUDA stream capture in global mode
// (legacy allocation calls are refused then), applications whose device memory
// is entirely handed out by another allocator (a framework's memory pool), and
// time-critical loops that cannot accept cudaMalloc's implicit device
// synchronisation or a late out-of-memory failure.  This entry point performs
// no allocation of any kind: its scratch is the file-scope array below.  The
// array (32 MiB) is committed on a device when ceedbp_setup first runs there
// (its address lookup loads this file's device image) and stays held until
// the process exits.
#include <mutex>
#include <string>

#include "ctx.h"

namespace ceedbp {
namespace {

// Capacity of the static scratch in doubles: E * p1^3 * ncomp of one call
// must not exceed it (for N = 7 that is 8192 elements of a scalar problem).
constexpr size_t kNoallocScratchDoubles = size_t(1) << 22;  // 32 MiB

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

// Looks up the device address of the scratch array on the current device and
// caches it.  ceedbp_setup calls this on its device (so the lookup, and the
// loading of this file's device image that holds the array, happen at set-up,
// where allocating is allowed); a later setup on the same device repeats the
// lookup, which also renews the address after a cudaDeviceReset.
cudaError_t noalloc_scratch_refresh() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  double* p = nullptr;
  e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  g_noalloc_ptr[dev] = p;
  return cudaSuccess;
}

namespace {

// The cached address for the current device (nullptr if no setup ran on it).
double* noalloc_scratch() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  return g_noalloc_ptr[dev];
}

ceedbp_status noalloc_fail(ceedbp_status st, const std::string& msg) {
  set_thread_error("ceedbp_apply_noalloc: " + msg);
  return st;
}

}  // namespace
}  // namespace ceedbp

using namespace ceedbp;

extern "C" ceedbp_status ceedbp_apply_noalloc(const ceedbp_ctx* ctx, const double* u_dev, double* w_dev,
                                              void* stream) {
  if (!ctx || !u_dev || !w_dev) return noalloc_fail(CEEDBP_EINVAL, "null argument");
  const DeviceMesh& m = ctx->mesh;
  const size_t need = size_t(m.nelem) * m.p1 * m.p1 * m.p1 * m.ncomp;
  if (need > kNoallocScratchDoubles)
    return noalloc_fail(CEEDBP_EINVAL, "the problem needs " + std::to_string(need) +
                                           " scratch entries (E * p1^3 * ncomp) but the static scratch holds " +
                                           std::to_string(kNoallocScratchDoubles) +
                                           "; use ceedbp_apply for larger problems");
  double* scratch = noalloc_scratch();
  if (scratch == nullptr)
    return noalloc_fail(CEEDBP_ECUDA, "no scratch address for the current device (run ceedbp_setup on it first)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (ctx->arith == CEEDBP_ARITH_DF64) {
    // the pair kernels of ceedbp_apply; a pair takes the room of a double
    ElemDfArgs a{};
    a.u_f64 = u_dev;
    a.wl = reinterpret_cast<dfloat*>(scratch);
    a.G = ctx->d_Gdf;
    a.D = ctx->d_Ddf;
    a.dnorm_row = ctx->dnorm_row;
    a.dnorm_col = ctx->dnorm_col;
    a.mask_in = 1;
    a.skip_dirichlet_out = 1;
    a.fault = &ctx->d_state->fault;  // reported by ceedbp_check or the next solve, as for ceedbp_apply
    a.first_wait = ctx->wait_polls;
    e = launch_elem_df(m, a, s);
    if (e == cudaSuccess) e = launch_gs_df(m, reinterpret_cast<const dfloat*>(scratch), w_dev, 1, s);
  } else {
    ElemArgs a{};
    a.u = u_dev;
    a.wl = scratch;
    a.G = ctx->op_kind == kStiff ? ctx->d_G : ctx->d_Mq;
    a.mask_in = ctx->prm.bp != 1 && ctx->prm.bp != 2;
    if (ctx->op_kind == kStiff && ctx->beta != 0.0) {
      a.Mq = ctx->d_Mq;
      a.beta = ctx->beta;
    }
    a.skip_dirichlet_out = 1;  // the masked gather-scatter never reads the skipped slots
    e = launch_elem(m, ctx->op_kind, a, s);
    if (e == cudaSuccess) e = launch_gs(m, scratch, w_dev, 1, s);
  }
  if (e != cudaSuccess) return noalloc_fail(CEEDBP_ECUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return CEEDBP_OK;
}
