// Kernel G: the generalized face-wise product of Sec. 3.1, C^p = A^p B^p for every
// frontal slice p (the loop of Algorithm 2), all slices in one launch
// (blockIdx.z = p).  Column-major slices: A^p is M x Kd, B^p is Kd x N, C^p is M x N.
//
// SIMT path (LT_FP64, LT_FP32, and LT_MIXED slices the tensor-core kernel of
// lt_tc_gemm.cu cannot address): 64 x 64 output tile per CTA, 16-deep K steps staged in
// shared memory, 4 x 4 register tile per thread.
//
// Fourier contexts (M_3 = F, slots of lt_fourier.cu): the product of the complex slices
// sqrt(n/2) (a1 + i a2) and sqrt(n/2) (b1 + i b2), back in slots, is sqrt(n/2) times
// (a1 b1 - a2 b2) for the real-part slot and (a1 b2 + a2 b1) for the imaginary-part slot;
// a real slot (DC, Nyquist) gives sqrt(n) a0 b0.  Each output slice then runs two K
// loops (one for a real slot) and scales in the epilogue: the complex product's four
// real products, two per slot.
#include <cmath>

#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int kGThreads = (BM / TM) * (BN / TN);  // 256

template <typename T>
__global__ void __launch_bounds__(kGThreads)
facewise_gemm_simt(int64_t M, int64_t N, int64_t Kd, int64_t P, const T* __restrict__ A,
                   const T* __restrict__ B, T* __restrict__ C, int64_t fn, T scale_real,
                   T scale_pair) {
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN + 1];
  for (int64_t p = blockIdx.z; p < P; p += gridDim.z) {
  // terms t = 0, 1: C^p += sgn_t A^{pa_t} B^{pb_t}; one term for a real context
  int nt = 1;
  int64_t pa[2] = {p, p}, pb[2] = {p, p};
  T sg1 = T(1), scale = T(1);
  if (fn) {
    const int64_t s = p % fn;
    if (s == 0 || (fn % 2 == 0 && s == fn - 1)) {
      scale = scale_real;
    } else if (s & 1) {           // real part: a1 b1 - a2 b2 (slots p, p + 1)
      nt = 2; scale = scale_pair; pa[1] = pb[1] = p + 1; sg1 = T(-1);
    } else {                      // imaginary part: a1 b2 + a2 b1 (slots p - 1, p)
      nt = 2; scale = scale_pair; pa[0] = p - 1; pb[1] = p - 1;
    }
  }
  T* Cp = C + p * M * N;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int tx = threadIdx.x % (BN / TN), ty = threadIdx.x / (BN / TN);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int t = 0; t < nt; ++t) {
  const T* Ap = A + pa[t] * M * Kd;
  const T* Bp = B + pb[t] * Kd * N;
  const T sg = t ? sg1 : T(1);
  for (int64_t k0 = 0; k0 < Kd; k0 += BK) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += kGThreads) {
      const int mm = idx % BM, kk = idx / BM;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < Kd) ? sg * Ap[gm + M * gk] : T(0);
    }
    for (int idx = threadIdx.x; idx < BK * BN; idx += kGThreads) {
      const int kk = idx % BK, nn = idx / BK;
      const int64_t gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < Kd && gn < N) ? Bp[gk + Kd * gn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gm = m0 + ty * TM + i, gn = n0 + tx * TN + j;
      if (gm < M && gn < N) Cp[gm + M * gn] = fn ? scale * acc[i][j] : acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_facewise_gemm(const Ctx& c, int64_t M, int64_t N, int64_t Kd,
                                 const void* A, const void* B, void* C, cudaStream_t st) {
  if (c.prec == LT_MIXED && !c.fourier_n) {
    // tensor cores, split TF32 x 3 (lt_tc_gemm.cu); slices whose sizes or addresses
    // do not meet the TMA alignment rules take the FP32 SIMT kernel below
    TcGemm g;
    g.M = M; g.N = N; g.K = Kd; g.batch = c.P;
    g.A = static_cast<const float*>(A); g.lda = M; g.sA = M * Kd;
    g.B = static_cast<const float*>(B); g.ldb = Kd; g.sB = Kd * N;
    g.D = static_cast<float*>(C); g.ldd = M; g.sD = M * N;
    g.wait_ns = (uint64_t)(c.tc_wait_us * 1e3); g.no_loads = c.tc_no_loads;
    if (tc_gemm_supported(g, c.tc_tile_n)) {
      ++c.tc_launches;
      return launch_tc_gemm(g, c.tc_tile_n, c.d_status, st);
    }
  }
  const int64_t gz = c.P < 65535 ? c.P : 65535;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)gz);
  const double n = (double)c.fourier_n;
  const double sr = n > 0 ? std::sqrt(n) : 1.0, sp = n > 0 ? std::sqrt(n / 2.0) : 1.0;
  if (c.elem == 8)
    facewise_gemm_simt<double><<<grid, kGThreads, 0, st>>>(
        M, N, Kd, c.P, (const double*)A, (const double*)B, (double*)C, c.fourier_n, sr, sp);
  else
    facewise_gemm_simt<float><<<grid, kGThreads, 0, st>>>(
        M, N, Kd, c.P, (const float*)A, (const float*)B, (float*)C, c.fourier_n, (float)sr,
        (float)sp);
  return cudaGetLastError();
}

}  // namespace lt
