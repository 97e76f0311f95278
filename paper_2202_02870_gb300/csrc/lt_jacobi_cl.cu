// Instantiations and launch of the cluster form of the SVT Jacobi kernel
// (lt_jacobi_cluster.cuh): FP64 and FP32, clusters of 3 and 4 CTAs.  Key of the
// instantiated shapes: G * 100 + E.
#include <map>
#include <mutex>
#include <tuple>

#include "lt_jacobi_cluster.cuh"

namespace lt {
namespace jac {

namespace {

template <typename T, int G, int E, int C>
cudaLaunchConfig_t config_for(const JArgs& a, int grid, cudaStream_t st,
                              cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3((unsigned)a.jp.threads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)a.jp.smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// mode 0: launch; mode 1: *ok = at least one cluster of this shape can be resident
template <typename T, int G, int E, int C>
cudaError_t go(const JArgs& a, int grid, cudaStream_t st, int mode, bool* ok) {
  constexpr int MAXT = cluster_max_threads(sizeof(T), E);
  auto k = jacobi_svt_cluster_kernel<T, G, E, C, MAXT, cluster_min_blocks(E)>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  // all of the SM's unified memory as shared memory, so that several CTAs fit
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = config_for<T, G, E, C>(a, grid, st, attr);
  if (mode == 1) {
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
    *ok = e == cudaSuccess && nclusters > 0;
    return e;
  }
  e = cudaLaunchKernelEx(&cfg, k, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T, int C>
cudaError_t dispatch(const JArgs& a, int grid, cudaStream_t st, int mode, bool* ok) {
  switch (a.jp.G * 100 + a.jp.E) {
    case 1606: return go<T, 16, 6, C>(a, grid, st, mode, ok);
    case 1609: return go<T, 16, 9, C>(a, grid, st, mode, ok);
    case 1612: return go<T, 16, 12, C>(a, grid, st, mode, ok);
    case 1618: return go<T, 16, 18, C>(a, grid, st, mode, ok);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t run(const JArgs& a, int grid, cudaStream_t st, int mode, bool* ok) {
  const bool f64 = a.jp.elem == 8;
  switch (a.jp.cluster) {
    case 3: return f64 ? dispatch<double, 3>(a, grid, st, mode, ok)
                       : dispatch<float, 3>(a, grid, st, mode, ok);
    case 4: return f64 ? dispatch<double, 4>(a, grid, st, mode, ok)
                       : dispatch<float, 4>(a, grid, st, mode, ok);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_svt_cluster(const JArgs& a, int grid, cudaStream_t st) {
  return run(a, grid, st, 0, nullptr);
}

bool svt_cluster_resident(const JArgs& a) {
  // occupancy answers per (element size, C, G, E, threads, shared memory, device)
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int, int, int>, bool> seen;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(a.jp.elem, a.jp.cluster, a.jp.G, a.jp.E, a.jp.threads,
                                   a.jp.smem, dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto it = seen.find(key);
    if (it != seen.end()) return it->second;
  }
  bool ok = false;
  ok = run(a, a.jp.cluster, nullptr, 1, &ok) == cudaSuccess && ok;
  if (!ok) cudaGetLastError();  // clear a failed query's error
  std::lock_guard<std::mutex> lk(mu);
  seen[key] = ok;
  return ok;
}

}  // namespace jac
}  // namespace lt
