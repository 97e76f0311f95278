// PGA bookkeeping on the device (Algorithm 5): the scalar sequence
// t_{k+1} = (1 + sqrt(4 t_k^2 + 1)) / 2, the momentum weight (t_{k-1} - 1) / t_k of
// Eq. 52, the stopping quantity ||Y^k - X^{k+1}||_F / ||X^{k+1}||_F of Sec. 5 and the
// objective.  Everything stays on the device so that the host only enqueues work; the
// reductions run in a fixed order (one CTA), so results are bitwise reproducible.
#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kFThreads = 256;

__global__ void pga_init_kernel(PgaScalars* s, double t_prev, double t, int64_t k0,
                                double tol) {
  s->t_prev = t_prev;
  s->t = t;
  s->beta = (t_prev - 1.0) / t;
  s->rel_residual = 0.0;
  s->objective = 0.0;
  s->tol = tol;
  s->k_done = 0;
  s->k_total = k0;
  s->done = 0;
  s->max_sweeps_used = 0;
  s->status = 0;
  s->pad = 0;
}

__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
  return t;
}

__global__ void __launch_bounds__(kFThreads)
pga_finish_kernel(PgaScalars* s, const double* __restrict__ partials, int rows,
                  const SliceInfo* __restrict__ info, int64_t P, double tau, int objective,
                  int32_t* ctx_status) {
  __shared__ double red[kFThreads / 32];
  if (s->done) return;
  double r0 = 0, r1 = 0, r2 = 0, nuc = 0;
  int sw = 0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    r0 += partials[4 * (size_t)i + 0];
    r1 += partials[4 * (size_t)i + 1];
    r2 += partials[4 * (size_t)i + 2];
  }
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) {
    nuc += info[p].nuclear;
    sw = max(sw, info[p].sweeps);
  }
  r0 = block_sum(r0, red);
  r1 = block_sum(r1, red);
  r2 = block_sum(r2, red);
  nuc = block_sum(nuc, red);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sw = max(sw, __shfl_xor_sync(0xffffffffu, sw, o));
  __shared__ int swr[kFThreads / 32];
  if (threadIdx.x % 32 == 0) swr[threadIdx.x / 32] = sw;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) sw = max(sw, swr[i]);
    const double r = (r1 > 0.0) ? sqrt(r0) / sqrt(r1) : sqrt(r0);
    s->rel_residual = r;
    s->objective = objective ? tau * nuc + 0.5 * r2 : 0.0;
    s->k_done += 1;
    s->k_total += 1;
    if (sw > s->max_sweeps_used) s->max_sweeps_used = sw;
    const double t_new = 0.5 * (1.0 + sqrt(4.0 * s->t * s->t + 1.0));
    s->t_prev = s->t;
    s->t = t_new;
    s->beta = (s->t_prev - 1.0) / s->t;
    if (s->tol > 0.0 && r <= s->tol) s->done = 1;
    s->status |= *ctx_status;
  }
}

// X (user buffer) must end up holding the newest iterate.  After k_done iterations it
// lives in buffer k_done % 2 (0 = X, 1 = alt); the previous one in the other buffer.
__global__ void select_result_kernel(const PgaScalars* __restrict__ s, uint32_t* x,
                                     const uint32_t* alt, uint32_t* prev_out, size_t words) {
  const bool odd = (s->k_done & 1) != 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t a = alt[i], b = x[i];
    if (odd) {
      if (prev_out) prev_out[i] = b;
      x[i] = a;
    } else if (prev_out) {
      prev_out[i] = a;
    }
  }
}

__global__ void copy_words_kernel(uint32_t* dst, const uint32_t* src, size_t words) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

int grid_for(size_t words) {
  size_t g = (words + 255) / 256;
  return (int)(g < 152 * 8 ? (g ? g : 1) : 152 * 8);
}

}  // namespace

cudaError_t launch_pga_init(PgaScalars* scal, double t_prev, double t, int64_t k0,
                            double tol, cudaStream_t st) {
  pga_init_kernel<<<1, 1, 0, st>>>(scal, t_prev, t, k0, tol);
  return cudaGetLastError();
}

cudaError_t launch_pga_finish(PgaScalars* scal, const double* partials, int rows,
                              const SliceInfo* info, int64_t P, double tau, int objective,
                              int32_t* ctx_status, cudaStream_t st) {
  pga_finish_kernel<<<1, kFThreads, 0, st>>>(scal, partials, rows, info, P, tau, objective,
                                             ctx_status);
  return cudaGetLastError();
}

cudaError_t launch_copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const size_t words = bytes / 4;
  copy_words_kernel<<<grid_for(words), 256, 0, st>>>((uint32_t*)dst, (const uint32_t*)src, words);
  return cudaGetLastError();
}

cudaError_t launch_select_result(const PgaScalars* scal, void* x_user, const void* x_alt,
                                 void* x_prev_out, size_t bytes, cudaStream_t st) {
  const size_t words = bytes / 4;
  select_result_kernel<<<grid_for(words), 256, 0, st>>>(scal, (uint32_t*)x_user,
                                                        (const uint32_t*)x_alt,
                                                        (uint32_t*)x_prev_out, words);
  return cudaGetLastError();
}

}  // namespace lt
