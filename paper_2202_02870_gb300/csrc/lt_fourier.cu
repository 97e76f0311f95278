// The Fourier operator of the t-product (Sec. 2: M_3 = F_{I3}, the unnormalised DFT;
// Sec. 5: the TNN-PGA-F completion) on real arithmetic.
//
// Mode 3 is stored in the orthonormal real DFT basis R_n (rows, 0-based j < n):
//   row 0        1 / sqrt(n)                                  (DC)
//   row 2k - 1   sqrt(2/n) cos(2 pi j k / n)     k = 1..(n-1)/2
//   row 2k      -sqrt(2/n) sin(2 pi j k / n)
//   row n - 1    (-1)^j / sqrt(n)                             (Nyquist, even n only)
// so that, with x_hat = F_n x, slot 0 = x_hat_0 / sqrt(n), slots (2k-1, 2k) =
// sqrt(2/n) (Re x_hat_k, Im x_hat_k), slot n-1 = x_hat_{n/2} / sqrt(n); the other half
// of F_n x is the conjugate of the first (x real).  R_n is orthogonal, so L^{-1} is its
// transpose and the real transforms of modes 3..K need nothing new.
//
// A complex transform-domain slice Z = a1 + i a2 (a pair of slots) has the singular
// values of its realification Phi(Z) = [[a1, -a2], [a2, a1]], each twice, and
// Phi(U max(S - t, 0) V^H) is the SVT of Phi(Z) at t: the SVT of the complex slices of
// Algorithm 4 runs as the real Jacobi SVT on the 2 I1 x 2 I2 realified pairs, and on
// the I1 x I2 real slots.  With the slot scaling above, the complex slice of F-domain
// data is sqrt(n/2) Z (pairs) or sqrt(n) a0 (real slots), so a threshold tau on it is
// tau sqrt(2/n) on Phi(Z) and tau / sqrt(n) on a0.
#include <cmath>

#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kThreads = 256;

int grid_for(int64_t work, int sms) {
  const int64_t g = (work + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sms * 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// Wr[(j + nr r) S + e] = G[(r n + slot_j) S + e], slot_0 = 0, slot_1 = n - 1;
// Wc[q 4S + row + col 2 I1] = Phi(a1 + i a2)(row, col), q = (k - 1) + h r.
template <typename T>
__global__ void __launch_bounds__(kThreads)
realify_kernel(const T* __restrict__ G, T* __restrict__ Wr, T* __restrict__ Wc, int64_t I1,
               int64_t I2, int64_t n, int64_t R, const PgaScalars* __restrict__ scal) {
  if (scal && scal->done) return;
  const int64_t S = I1 * I2, h = (n - 1) / 2, nr = (n % 2 == 0) ? 2 : 1;
  const int64_t totr = nr * R * S, totc = h * R * 4 * S;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < totr + totc;
       idx += stride) {
    if (idx < totr) {
      const int64_t e = idx % S, q = idx / S;
      const int64_t r = q / nr, slot = (q % nr) == 0 ? 0 : n - 1;
      Wr[idx] = G[(r * n + slot) * S + e];
    } else {
      const int64_t t = idx - totr;
      const int64_t q = t / (4 * S), w = t % (4 * S);
      const int64_t row = w % (2 * I1), col = w / (2 * I1);
      const bool rb = row >= I1, cb = col >= I2;
      const int64_t i = rb ? row - I1 : row, j = cb ? col - I2 : col;
      const int64_t r = q / h, k = q % h + 1;
      const int64_t slot = (rb == cb) ? 2 * k - 1 : 2 * k;
      const T v = G[(r * n + slot) * S + i + j * I1];
      Wc[t] = (!rb && cb) ? -v : v;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
derealify_kernel(const T* __restrict__ Wr, const T* __restrict__ Wc, T* __restrict__ G,
                 int64_t I1, int64_t I2, int64_t n, int64_t R,
                 const PgaScalars* __restrict__ scal) {
  if (scal && scal->done) return;
  const int64_t S = I1 * I2, h = (n - 1) / 2, nr = (n % 2 == 0) ? 2 : 1;
  const int64_t total = R * n * S;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += stride) {
    const int64_t e = idx % S, p = idx / S;
    const int64_t r = p / n, s = p % n;
    T v;
    if (s == 0) {
      v = Wr[(nr * r) * S + e];
    } else if (n % 2 == 0 && s == n - 1) {
      v = Wr[(1 + nr * r) * S + e];
    } else {
      const int64_t k = (s + 1) / 2, q = (k - 1) + h * r;
      const int64_t i = e % I1, j = e / I1;
      const int64_t row = (s & 1) ? i : I1 + i;  // Re: top-left block, Im: bottom-left
      v = Wc[q * 4 * S + row + j * 2 * I1];
    }
    G[idx] = v;
  }
}

}  // namespace

FourierSlots fourier_slots(const Ctx& c) {
  FourierSlots f;
  if (!c.fourier_n) return f;
  f.n = c.fourier_n;
  f.R = c.P / f.n;
  f.nreal = (f.n % 2 == 0 ? 2 : 1) * f.R;
  f.npair = (f.n - 1) / 2 * f.R;
  return f;
}

void fourier_basis(int64_t n, double* R) {
  const double pi = 3.14159265358979323846;
  const double a = 1.0 / std::sqrt((double)n), b = std::sqrt(2.0 / (double)n);
  for (int64_t j = 0; j < n; ++j) {
    R[j] = a;
    for (int64_t k = 1; 2 * k < n; ++k) {
      // the angle 2 pi j k / n reduced mod n first keeps it below 2 pi
      const double th = 2.0 * pi * (double)((j * k) % n) / (double)n;
      R[(2 * k - 1) * n + j] = b * std::cos(th);
      R[(2 * k) * n + j] = -b * std::sin(th);
    }
    if (n % 2 == 0) R[(n - 1) * n + j] = (j % 2 == 0) ? a : -a;
  }
}

cudaError_t launch_fourier_realify(const Ctx& c, int64_t I1, int64_t I2, const void* G,
                                   void* Wr, void* Wc, const PgaScalars* scal,
                                   cudaStream_t st) {
  const FourierSlots f = fourier_slots(c);
  const int64_t work = (f.nreal + 4 * f.npair) * I1 * I2;
  const int grid = grid_for(work, c.sms);
  if (c.elem == 8)
    realify_kernel<double><<<grid, kThreads, 0, st>>>((const double*)G, (double*)Wr,
                                                      (double*)Wc, I1, I2, f.n, f.R, scal);
  else
    realify_kernel<float><<<grid, kThreads, 0, st>>>((const float*)G, (float*)Wr,
                                                     (float*)Wc, I1, I2, f.n, f.R, scal);
  return cudaGetLastError();
}

cudaError_t launch_fourier_derealify(const Ctx& c, int64_t I1, int64_t I2, const void* Wr,
                                     const void* Wc, void* G, const PgaScalars* scal,
                                     cudaStream_t st) {
  const FourierSlots f = fourier_slots(c);
  const int grid = grid_for(c.P * I1 * I2, c.sms);
  if (c.elem == 8)
    derealify_kernel<double><<<grid, kThreads, 0, st>>>((const double*)Wr, (const double*)Wc,
                                                        (double*)G, I1, I2, f.n, f.R, scal);
  else
    derealify_kernel<float><<<grid, kThreads, 0, st>>>((const float*)Wr, (const float*)Wc,
                                                       (float*)G, I1, I2, f.n, f.R, scal);
  return cudaGetLastError();
}

}  // namespace lt
