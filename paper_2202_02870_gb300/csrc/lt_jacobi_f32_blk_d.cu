// Instantiations of the SVT Jacobi kernel (float), one of several translation units so
// that they compile in parallel: 8-lane groups holding two blocks of 2 columns.
// Key: G * 10000 + B * 100 + E.
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E, int B>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<float, G, E, B, kMaxThreadsBlocked>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f32_blk_d(const JArgs& a, int grid, cudaStream_t st) {
  switch (a.jp.G * 10000 + a.jp.B * 100 + a.jp.E) {
    case 80206: return go<8, 6, 2>(a, grid, st);
    case 80212: return go<8, 12, 2>(a, grid, st);
    case 80218: return go<8, 18, 2>(a, grid, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace jac
}  // namespace lt
