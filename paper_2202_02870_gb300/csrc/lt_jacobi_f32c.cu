// Instantiations of the SVT Jacobi kernel for float (split across translation units so
// that they compile in parallel).
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<float, G, E, kMaxThreadsF32>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f32_g8_large(const JArgs& a, int grid, cudaStream_t st) {
  const int key = a.jp.G * 1000 + a.jp.E;
  switch (key) {
    case 8010: return go<8, 10>(a, grid, st);
    case 8012: return go<8, 12>(a, grid, st);
    case 8014: return go<8, 14>(a, grid, st);
    case 8016: return go<8, 16>(a, grid, st);
    case 8018: return go<8, 18>(a, grid, st);
    case 8020: return go<8, 20>(a, grid, st);
    case 8024: return go<8, 24>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace jac
}  // namespace lt
