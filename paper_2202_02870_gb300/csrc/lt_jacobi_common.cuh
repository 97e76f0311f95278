// Device helpers shared by the Jacobi kernels (kernel J).
#pragma once

#include <cfloat>

#include "lt_internal.cuh"

namespace lt {
namespace jac {

constexpr int kJThreads = 512;
constexpr int kWarps = kJThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four warp-wide sums at once, every lane receiving all four: a transposed butterfly
// (the first two levels exchange halves of the vector, so each lane adds 2 + 1 + 3 = 6
// values instead of 4 x 5), then a broadcast from the lanes that hold each total.
template <typename T>
__device__ __forceinline__ void warp_allsum4(T (&w)[4]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  T k0 = h16 ? w[2] : w[0], k1 = h16 ? w[3] : w[1];
  const T s0 = h16 ? w[0] : w[2], s1 = h16 ? w[1] : w[3];
  k0 += __shfl_xor_sync(full, s0, 16);
  k1 += __shfl_xor_sync(full, s1, 16);
  T k = h8 ? k1 : k0;
  k += __shfl_xor_sync(full, h8 ? k0 : k1, 8);
  k += __shfl_xor_sync(full, k, 4);
  k += __shfl_xor_sync(full, k, 2);
  k += __shfl_xor_sync(full, k, 1);
  // the total of vector entry c = 2 h16 + h8 now sits on every lane with those bits
  w[0] = __shfl_sync(full, k, 0);
  w[1] = __shfl_sync(full, k, 8);
  w[2] = __shfl_sync(full, k, 16);
  w[3] = __shfl_sync(full, k, 24);
}

// (value, index) arg-max over the warp; ties go to the smaller index.  Every lane ends
// with the result.
template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
}

template <typename T> __device__ __forceinline__ T unit_roundoff();
template <> __device__ __forceinline__ double unit_roundoff<double>() { return DBL_EPSILON / 2; }
template <> __device__ __forceinline__ float unit_roundoff<float>() { return FLT_EPSILON / 2; }

// Rotation for the pair (alpha, beta, gamma) = (||x||^2, ||y||^2, x.y), Rutishauser's
// formulas (Golub & Van Loan, Matrix Computations, 4th ed., Sec. 8.6.3):
// zeta = (beta - alpha)/(2 gamma), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1 + t^2), s = c t.  The angle only steers convergence; what must hold to
// working precision is c^2 + s^2 = 1, so that the update is an orthogonal transform.
// FP32: the formulas directly.  FP64: the tangent is taken from the same formulas in
// FP32 (FP64 divides and square roots cost tens of FP64 pipe slots each on this GPU),
// then c = (1 + t^2)^{-1/2} is computed in FP64 by two Newton steps
// y <- y (3 - x y^2) / 2 from the FP32 reciprocal square root (2^-22 -> 2^-44 -> full
// precision), s = c t.  A tangent that is only FP32-accurate leaves |x.y| at ~1e-7 of
// its value after the rotation; later sweeps remove it.
__device__ __forceinline__ void rotation(float al, float be, float g, float& cs, float& sn,
                                         float& t) {
  const float zeta = (be - al) / (2.f * g);
  const float az = fabsf(zeta);
  t = (az > 1e15f) ? 0.5f / az : 1.f / (az + sqrtf(1.f + az * az));
  if (zeta < 0.f) t = -t;
  cs = rsqrtf(1.f + t * t);
  sn = cs * t;
}
// zeta = (beta - alpha) / (2 gamma) in FP32 when the operands are inside FP32's range,
// else by an FP64 divide (rare: slices are scaled to a maximum entry in [1, 2), so this
// takes only columns below about 1e-19 of it).
__device__ __forceinline__ float jacobi_zeta(double al, double be, double g) {
  const float df = float(be - al), gf = float(g);
  if (fabsf(gf) >= FLT_MIN && fabsf(gf) <= 1e37f && fabsf(df) <= 1e37f)
    return __fdividef(df, 2.f * gf);
  return float((be - al) / (2.0 * g));
}

__device__ __forceinline__ void rotation(double al, double be, double g, double& cs,
                                         double& sn, double& t) {
  const float zeta = jacobi_zeta(al, be, g);
  const float az = fabsf(zeta);
  float tf = (az > 1e15f) ? 0.5f / az : 1.f / (az + sqrtf(1.f + az * az));
  if (zeta < 0.f) tf = -tf;
  t = double(tf);
  const double x = fma(t, t, 1.0);
  double y = double(rsqrtf(float(x)));
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  cs = y;
  sn = y * t;
}

// Power of two s with s * maxabs in [1, 2) (in [2, 4) for maxabs in the top binade; 1 when
// maxabs is zero, subnormal, infinite or NaN).  Scaling a slice by s is exact and keeps the Jacobi arithmetic (squared norms,
// the FP32 rotation angle) inside the floating-point range whatever the data's scale.
__device__ __forceinline__ double pow2_scale(double maxabs) {
  const long long e = (__double_as_longlong(maxabs) >> 52) & 0x7ff;
  if (e == 0 || e == 0x7ff) return 1.0;
  return __longlong_as_double((long long)(e < 2046 ? 2046 - e : 1) << 52);
}
__device__ __forceinline__ float pow2_scale(float maxabs) {
  const int e = (__float_as_int(maxabs) >> 23) & 0xff;
  if (e == 0 || e == 0xff) return 1.f;
  return __int_as_float((e < 254 ? 254 - e : 1) << 23);
}

struct JArgs {
  JacobiPlan jp;
  JacobiIO io;
  double tol;
  int max_sweeps;
  int32_t* status;
};

// SVT kernel launchers by element type and group width (lt_jacobi_f32*.cu, _f64.cu).
constexpr int kMaxThreadsF32 = 768;
constexpr int kMaxThreadsF64 = 576;
constexpr int kMaxThreadsBlocked = 512;  // register-blocked FP32 sweeps: 128 registers
constexpr int kMaxThreadsBlockedWide = 576;  // wide form: 36 groups of 16, 113 registers
cudaError_t launch_svt_f32_blk_a(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f32_blk_b(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f32_blk_c(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f32_blk_d(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f32_blk_e(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f32_pw_a(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f32_pw_b(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f64_a(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f64_b(const JArgs& a, int grid, cudaStream_t st);
cudaError_t launch_svt_f64_c(const JArgs& a, int grid, cudaStream_t st);
// Instantiated (G, B, E) shapes (rows padded to G E): see svt_shape in lt_jacobi.cu.
// Cluster form (lt_jacobi_cl.cu): jp.cluster CTAs per slice; grid = jp.cluster x slices.
cudaError_t launch_svt_cluster(const JArgs& a, int grid, cudaStream_t st);
// Thread cap and minimum resident CTAs of a cluster-form instantiation (16 lanes per
// pair, E rows per lane): up to 12 rows per lane two CTAs of 384 threads share an SM
// (85 registers each); 18 rows per lane keep one CTA of up to 576 (FP64) or 768 (FP32).
constexpr int cluster_max_threads(int elem, int E) {
  return E <= 12 ? 384 : (elem == 8 ? kMaxThreadsF64 : kMaxThreadsF32);
}
constexpr int cluster_min_blocks(int E) { return E <= 12 ? 2 : 1; }
// At least one cluster of the plan's shape can be resident on the device.
bool svt_cluster_resident(const JArgs& a);

}  // namespace jac
}  // namespace lt
