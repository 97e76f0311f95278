// The rank notions and norms of Sec. 3.2 from the per-slice singular values of L(A)
// (written by the SVT kernel in its JAC_SIGMA mode): the nuclear norm of Eq. 24 (the
// transform-domain sum, without the 1/alpha factor), the spectral norm of the
// proposition on ||bdiag(L(A))||, the multirank and average rank of their definition,
// and the tubal rank of its definition and lemma (max over slices of the slice ranks,
// the singular values of a slice being descending).  One CTA, fixed summation order:
// the results are reproducible bit for bit.
#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kNThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kNThreads)
norms_finish_kernel(const T* __restrict__ sigma, int64_t P, int n, double rank_tol,
                    double* __restrict__ out, int32_t* __restrict__ multirank) {
  __shared__ double red[kNThreads / 32];
  __shared__ long long redi[kNThreads / 32];
  __shared__ double s_bcast;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t total = P * (int64_t)n;
  // largest singular value (max is order-free)
  double mx = 0.0, sum = 0.0;
  for (int64_t i = t; i < total; i += kNThreads) {
    const double v = (double)sigma[i];
    mx = v > mx ? v : mx;
    sum += v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  if (lane == 0) red[w] = mx;
  __syncthreads();
  if (t == 0) {
    double m = 0.0;
    for (int i = 0; i < kNThreads / 32; ++i) m = red[i] > m ? red[i] : m;
    s_bcast = m;
  }
  __syncthreads();
  const double smax = s_bcast;
  __syncthreads();
  // sum of all singular values, fixed order: per-thread strided sums, then a tree
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) red[w] = sum;
  __syncthreads();
  double nuclear = 0.0;
  if (t == 0)
    for (int i = 0; i < kNThreads / 32; ++i) nuclear += red[i];
  __syncthreads();
  // slice ranks against max(I1, I2) u sigma_max
  const double tol = rank_tol * smax;
  long long rsum = 0, rmax = 0;
  for (int64_t p = t; p < P; p += kNThreads) {
    int cnt = 0;
    if (smax > 0.0)
      for (int c = 0; c < n; ++c) cnt += ((double)sigma[p * n + c] > tol) ? 1 : 0;
    if (multirank) multirank[p] = cnt;
    rsum += cnt;
    rmax = cnt > rmax ? cnt : rmax;
  }
  for (int o = 16; o > 0; o >>= 1) {
    rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    const long long v = __shfl_xor_sync(0xffffffffu, rmax, o);
    rmax = v > rmax ? v : rmax;
  }
  if (lane == 0) {
    red[w] = (double)rmax;
    redi[w] = rsum;
  }
  __syncthreads();
  if (t == 0) {
    long long rs = 0;
    double rm = 0.0;
    for (int i = 0; i < kNThreads / 32; ++i) {
      rs += redi[i];
      rm = red[i] > rm ? red[i] : rm;
    }
    out[0] = nuclear;
    out[1] = smax;
    out[2] = rm;
    out[3] = P > 0 ? (double)rs / (double)P : 0.0;
  }
}

}  // namespace

cudaError_t launch_norms_finish(const void* sigma, int elem, int64_t P, int n, double rank_tol,
                                double* out, int32_t* multirank, cudaStream_t st) {
  if (elem == 8)
    norms_finish_kernel<double><<<1, kNThreads, 0, st>>>(static_cast<const double*>(sigma), P, n,
                                                         rank_tol, out, multirank);
  else
    norms_finish_kernel<float><<<1, kNThreads, 0, st>>>(static_cast<const float*>(sigma), P, n,
                                                        rank_tol, out, multirank);
  return cudaGetLastError();
}

}  // namespace lt
