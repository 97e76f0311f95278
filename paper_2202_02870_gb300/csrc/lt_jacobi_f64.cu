// Instantiations of the SVT Jacobi kernel for double (split across translation units so
// that they compile in parallel).
#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

template <int G, int E>
static cudaError_t go(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_svt_kernel<double, G, E, kMaxThreadsF64>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, a.jp.threads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_svt_f64_g8(const JArgs& a, int grid, cudaStream_t st) {
  const int key = a.jp.G * 1000 + a.jp.E;
  switch (key) {
    case 8001: return go<8, 1>(a, grid, st);
    case 8002: return go<8, 2>(a, grid, st);
    case 8003: return go<8, 3>(a, grid, st);
    case 8004: return go<8, 4>(a, grid, st);
    case 8005: return go<8, 5>(a, grid, st);
    case 8006: return go<8, 6>(a, grid, st);
    case 8007: return go<8, 7>(a, grid, st);
    case 8008: return go<8, 8>(a, grid, st);
    case 8009: return go<8, 9>(a, grid, st);
    case 8010: return go<8, 10>(a, grid, st);
    case 8012: return go<8, 12>(a, grid, st);
    case 8014: return go<8, 14>(a, grid, st);
    case 8016: return go<8, 16>(a, grid, st);
    case 8018: return go<8, 18>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace jac
}  // namespace lt
