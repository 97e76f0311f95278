// Warm start of the per-slice SVT across the iterations of Algorithm 5 (a context
// option, LT_OPT_WARM_START; the paper computes every SVD from scratch).
//
// The SVT of a transform-domain slice G (I1 x I2) is unitarily invariant: for an
// orthogonal n x n matrix Q (n = min(I1, I2)),
//     I1 <  I2:  D_tau(G) = Q D_tau(Q^T G),      I1 >= I2:  D_tau(G) = D_tau(G Q) Q^T.
// The Jacobi kernel orthogonalises the columns of G^T (I1 < I2) or of G, so with Q the
// previous iteration's left (resp. right) singular vectors the rotated slice starts
// close to its converged form and needs fewer sweeps: the iterates of Algorithm 5 change
// little from one iteration to the next.  The kernel returns the orthonormal basis W of
// the side it orthogonalised (rows in its QR order, with the QR permutation), and the
// next basis is Q P W.
//
// This file holds the batched products of that bookkeeping (all slices in one launch,
// general element strides, so that every transpose is free):
//   C^p(m, n) = sum_k A^p(m, kk) B^p(k, n),  kk = kperm ? kperm[p K + k] : k,
// with A^p(m, k) = A[p sap + m sam + k sak], B^p(k, n) = B[p sbp + k sbk + n sbn],
// C^p(m, n) = C[p scp + m scm + n scn]; one 48 x 48 output tile per CTA with a 3 x 3
// register tile per thread (48 divides the slice sizes of the benchmark, 144, where
// 64 x 64 tiles computed up to 44 % padding), 16-deep K steps in shared memory; and the
// scatter that turns the first basis (Q = I) into P W.  Every kernel returns at once when
// the PGA run has already met its tolerance.
#include <algorithm>

#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int WBK = 16;
constexpr int kWThreads = 256;

template <typename T, int WBM, int WTM>
__global__ void __launch_bounds__(kWThreads)
strided_gemm_kernel(const StridedGemm g, const T* __restrict__ A, const T* __restrict__ B,
                    T* __restrict__ C, const PgaScalars* scal) {
  constexpr int WBN = WBM, WTN = WTM;
  static_assert((WBM / WTM) * (WBN / WTN) == kWThreads, "one register tile per thread");
  if (scal != nullptr && scal->done) return;
  __shared__ T As[WBK][WBM];
  __shared__ T Bs[WBK][WBN + 1];
  const int tx = threadIdx.x % (WBN / WTN), ty = threadIdx.x / (WBN / WTN);
  const int64_t m0 = (int64_t)blockIdx.x * WBM, n0 = (int64_t)blockIdx.y * WBN;
  for (int64_t p = blockIdx.z; p < g.P; p += gridDim.z) {
    const T* Ap = A + p * g.sap;
    const T* Bp = B + p * g.sbp;
    const int* kp = g.kperm ? g.kperm + p * g.K : nullptr;
    T acc[WTM][WTN];
#pragma unroll
    for (int i = 0; i < WTM; ++i)
#pragma unroll
      for (int j = 0; j < WTN; ++j) acc[i][j] = T(0);
    for (int64_t k0 = 0; k0 < g.K; k0 += WBK) {
      // consecutive threads walk the unit-stride index of each operand
      for (int idx = threadIdx.x; idx < WBM * WBK; idx += kWThreads) {
        const int mm = g.sam == 1 ? idx % WBM : idx / WBK;
        const int kk = g.sam == 1 ? idx / WBM : idx % WBK;
        const int64_t gm = m0 + mm, gk = k0 + kk;
        T v = T(0);
        if (gm < g.M && gk < g.K) v = Ap[gm * g.sam + (int64_t)(kp ? kp[gk] : gk) * g.sak];
        As[kk][mm] = v;
      }
      for (int idx = threadIdx.x; idx < WBK * WBN; idx += kWThreads) {
        const int kk = g.sbk == 1 ? idx % WBK : idx / WBN;
        const int nn = g.sbk == 1 ? idx / WBK : idx % WBN;
        const int64_t gk = k0 + kk, gn = n0 + nn;
        Bs[kk][nn] = (gk < g.K && gn < g.N) ? Bp[gk * g.sbk + gn * g.sbn] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < WBK; ++kk) {
        T a[WTM], b[WTN];
#pragma unroll
        for (int i = 0; i < WTM; ++i) a[i] = As[kk][ty * WTM + i];
#pragma unroll
        for (int j = 0; j < WTN; ++j) b[j] = Bs[kk][tx * WTN + j];
#pragma unroll
        for (int i = 0; i < WTM; ++i)
#pragma unroll
          for (int j = 0; j < WTN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
    T* Cp = C + p * g.scp;
#pragma unroll
    for (int i = 0; i < WTM; ++i)
#pragma unroll
      for (int j = 0; j < WTN; ++j) {
        const int64_t gm = m0 + ty * WTM + i, gn = n0 + tx * WTN + j;
        if (gm < g.M && gn < g.N) Cp[gm * g.scm + gn * g.scn] = acc[i][j];
      }
  }
}

// Q^p(perm^p[r], c) = W^p(r, c): the basis P W of a cold iteration (previous basis I).
template <typename T>
__global__ void warm_scatter_kernel(int64_t n, int64_t P, const T* __restrict__ W,
                                    const int* __restrict__ perm, T* __restrict__ Q,
                                    const PgaScalars* scal) {
  if (scal != nullptr && scal->done) return;
  const int64_t total = n * n * P;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / (n * n), rc = i % (n * n), r = rc % n, c = rc / n;
    Q[p * n * n + perm[p * n + r] + n * c] = W[i];
  }
}

}  // namespace

cudaError_t launch_strided_gemm(const Ctx& c, const StridedGemm& g, const void* A,
                                const void* B, void* C, const PgaScalars* scal,
                                cudaStream_t st) {
  if (g.M < 1 || g.N < 1 || g.K < 1 || g.P < 1) return cudaErrorInvalidValue;
  const int64_t gz = g.P < 65535 ? g.P : 65535;
  const int64_t tile = 48;
  dim3 grid((unsigned)((g.M + tile - 1) / tile), (unsigned)((g.N + tile - 1) / tile), (unsigned)gz);
  if (c.elem == 8)
    strided_gemm_kernel<double, 48, 3><<<grid, kWThreads, 0, st>>>(
        g, static_cast<const double*>(A), static_cast<const double*>(B),
        static_cast<double*>(C), scal);
  else
    strided_gemm_kernel<float, 48, 3><<<grid, kWThreads, 0, st>>>(
        g, static_cast<const float*>(A), static_cast<const float*>(B), static_cast<float*>(C),
        scal);
  return cudaGetLastError();
}

cudaError_t launch_warm_scatter(const Ctx& c, int64_t n, int64_t P, const void* W,
                                const int* perm, void* Q, const PgaScalars* scal,
                                cudaStream_t st) {
  const int64_t total = n * n * P;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, (int64_t)c.sms * 8);
  if (c.elem == 8)
    warm_scatter_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(
        n, P, static_cast<const double*>(W), perm, static_cast<double*>(Q), scal);
  else
    warm_scatter_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
        n, P, static_cast<const float*>(W), perm, static_cast<float*>(Q), scal);
  return cudaGetLastError();
}

}  // namespace lt
