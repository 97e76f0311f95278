// Instantiations of the SVT Jacobi kernel (float) in the wide register-blocked form:
// 16-lane groups holding blocks of 2 columns, one group per block pair of a round
// (576 threads for up to 144 columns), so that every block pair of a round is in flight
// at once.  Key: G * 10000 + B * 100 + E.
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E, int B>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<float, G, E, B, kMaxThreadsBlockedWide>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f32_blk_e(const JArgs& a, int grid, cudaStream_t st) {
  if (a.jp.threads > kMaxThreadsBlockedWide) return cudaErrorNotSupported;
  switch (a.jp.G * 10000 + a.jp.B * 100 + a.jp.E) {
    case 160207: return go<16, 7, 2>(a, grid, st);
    case 160209: return go<16, 9, 2>(a, grid, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace jac
}  // namespace lt
