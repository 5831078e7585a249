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
// no allocation of any kind: its scratch is the file-scope array below, which
// every GPU that loads the library holds (32 MiB) until the process exits.
#include <cstdio>
#include <mutex>

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

// Device address of the scratch array on the current device, looked up once
// per device (host code may not use the array's name as a device pointer).
cudaError_t noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ceedbp

using namespace ceedbp;

extern "C" ceedbp_status ceedbp_apply_noalloc(const ceedbp_ctx* ctx, const double* u_dev, double* w_dev,
                                              void* stream) {
  if (!ctx || !u_dev || !w_dev) return CEEDBP_EINVAL;
  const DeviceMesh& m = ctx->mesh;
  const size_t need = size_t(m.nelem) * m.p1 * m.p1 * m.p1 * m.ncomp;
  if (need > kNoallocScratchDoubles) {
    std::fprintf(stderr,
                 "ceedbp_apply_noalloc: the problem needs %zu scratch doubles (E * p1^3 * ncomp) but the "
                 "static scratch holds %zu; use ceedbp_apply for larger problems\n",
                 need, kNoallocScratchDoubles);
    return CEEDBP_EINVAL;
  }
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return CEEDBP_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
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
  if (launch_elem(m, ctx->op_kind, a, s) != cudaSuccess) return CEEDBP_ECUDA;
  if (launch_gs(m, scratch, w_dev, 1, s) != cudaSuccess) return CEEDBP_ECUDA;
  return CEEDBP_OK;
}
