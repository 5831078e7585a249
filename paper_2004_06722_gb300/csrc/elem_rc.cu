// Instantiations of the recomputed-factor BK5/BK6 kernel (elem_rc.cuh) and the
// coordinate re-layout it reads.
#include "elem_rc.cuh"

namespace ceedbp {

namespace {

__global__ void coords_soa_kernel(const double* __restrict__ coords, double* __restrict__ X, int64_t nelem, int p3) {
  const int64_t total = nelem * p3 * 3;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = i / (3 * int64_t(p3));
    const int64_t r = i - e * 3 * int64_t(p3);
    const int d = int(r / p3);
    const int64_t a = r - int64_t(d) * p3;
    X[i] = coords[(e * p3 + a) * 3 + d];
  }
}

}  // namespace

cudaError_t launch_coords_soa(const double* coords, double* X, int64_t nelem, int p3, cudaStream_t s) {
  coords_soa_kernel<<<1216, 256, 0, s>>>(coords, X, nelem, p3);
  return cudaGetLastError();
}

// three-component tiles fit in shared memory up to p1 = 13
bool elem_rc_supported(int p1, int ncomp) { return p1 >= 2 && p1 <= kMaxP1 && (ncomp == 1 || p1 <= 13); }

#define CEEDBP_RC_CASE(P) \
  case P: return m.ncomp == 3 ? launch_elem_rc_t<P, 3>(m, a, s) : launch_elem_rc_t<P, 1>(m, a, s);
#define CEEDBP_RC_CASE1(P) \
  case P: return m.ncomp == 3 ? cudaErrorInvalidValue : launch_elem_rc_t<P, 1>(m, a, s);
#define CEEDBP_RC_BLOCKS(P) \
  case P: return m.ncomp == 3 ? elem_rc_blocks_t<P, 3>(m.nelem) : elem_rc_blocks_t<P, 1>(m.nelem);
#define CEEDBP_RC_BLOCKS1(P) \
  case P: return elem_rc_blocks_t<P, 1>(m.nelem);

cudaError_t launch_elem_rc(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_RC_CASE(2) CEEDBP_RC_CASE(3) CEEDBP_RC_CASE(4) CEEDBP_RC_CASE(5) CEEDBP_RC_CASE(6) CEEDBP_RC_CASE(7)
    CEEDBP_RC_CASE(8) CEEDBP_RC_CASE(9) CEEDBP_RC_CASE(10) CEEDBP_RC_CASE(11) CEEDBP_RC_CASE(12)
    CEEDBP_RC_CASE(13) CEEDBP_RC_CASE1(14) CEEDBP_RC_CASE1(15) CEEDBP_RC_CASE1(16)
    default: return cudaErrorInvalidValue;
  }
}

int elem_rc_blocks(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_RC_BLOCKS(2) CEEDBP_RC_BLOCKS(3) CEEDBP_RC_BLOCKS(4) CEEDBP_RC_BLOCKS(5) CEEDBP_RC_BLOCKS(6)
    CEEDBP_RC_BLOCKS(7) CEEDBP_RC_BLOCKS(8) CEEDBP_RC_BLOCKS(9) CEEDBP_RC_BLOCKS(10) CEEDBP_RC_BLOCKS(11)
    CEEDBP_RC_BLOCKS(12) CEEDBP_RC_BLOCKS(13) CEEDBP_RC_BLOCKS1(14) CEEDBP_RC_BLOCKS1(15)
    CEEDBP_RC_BLOCKS1(16)
    default: return 0;
  }
}

}  // namespace ceedbp
