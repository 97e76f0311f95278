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

cudaError_t launch_svt_f64_g16_32(const JArgs& a, int grid, cudaStream_t st) {
  const int key = a.jp.G * 1000 + a.jp.E;
  switch (key) {
    case 16001: return go<16, 1>(a, grid, st);
    case 16002: return go<16, 2>(a, grid, st);
    case 16003: return go<16, 3>(a, grid, st);
    case 16004: return go<16, 4>(a, grid, st);
    case 16005: return go<16, 5>(a, grid, st);
    case 16006: return go<16, 6>(a, grid, st);
    case 16007: return go<16, 7>(a, grid, st);
    case 16008: return go<16, 8>(a, grid, st);
    case 16009: return go<16, 9>(a, grid, st);
    case 16010: return go<16, 10>(a, grid, st);
    case 16012: return go<16, 12>(a, grid, st);
    case 16014: return go<16, 14>(a, grid, st);
    case 32008: return go<32, 8>(a, grid, st);
    case 32010: return go<32, 10>(a, grid, st);
    case 32012: return go<32, 12>(a, grid, st);
    case 32014: return go<32, 14>(a, grid, st);
    case 32016: return go<32, 16>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace jac
}  // namespace lt
