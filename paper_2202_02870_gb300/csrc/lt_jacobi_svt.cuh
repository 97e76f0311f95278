// Kernel J (SVT form): the per-slice step of Algorithm 4 -- svd of A_hat^p, shrink
// max(sigma - tau, 0), reconstruct U S V^T -- one CTA per frontal slice, the slice
// resident in shared memory (or in a per-CTA region of the workspace when too large).
//
// 1. Preconditioning (QR with column pivoting, Householder).  The working matrix B
//    (m x n, m >= n; B = A^p, or (A^p)^T when I1 < I2) is factored B P = Q R.  Q is not
//    needed.  Jacobi on R^T converges in markedly fewer sweeps than on B (Drmac and
//    Veselic, "New fast and accurate Jacobi SVD algorithm", SIAM J. Matrix Anal. Appl.
//    29(4), 2008) and works on an n x n instead of an m x n matrix.
// 2. One-sided (Hestenes) Jacobi on Z = R^T: rotations from the right until every column
//    pair is orthogonal to the tolerance.  Then Z = V_r Sigma with the right singular
//    vectors V_r of R and sigma_i = ||z_i||.  Round-robin ordering.  A pair is owned by
//    a group of G lanes (G = 8 or 16, so a warp works on 32/G pairs at once): lane g of
//    the group holds rows g, g+G, ..., g+G(E-1) of both columns in registers (rows padded
//    with zeros to G E, so the loops carry no bounds tests); the dot product is reduced
//    over the group with log2(G) shuffles.
// 3. Shrink and reconstruct without Q and without the rotations: since
//    B P = (Q U_r) Sigma V_r^T and V_r = Z Sigma^{-1},
//        D_tau(B) P = (B P) Z diag(g) Z^T,   g_i = (sigma_i - tau)_+ / sigma_i^3,
//    applied row by row to the ORIGINAL slice (re-read from global memory), a warp per
//    row: y_i = g_i (b . z_i) over the k columns with sigma_i > tau, then
//    d = sum_i y_i z_i.  2 m n k multiply-adds; the result overwrites the slice.
#pragma once

#include <cfloat>

#include "lt_jacobi_common.cuh"

namespace lt {
namespace jac {

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// |v| as an unsigned integer with the same ordering (for a maximum without FP64 compares)
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ unsigned long long abs_bits(float v) {
  return (unsigned long long)(__float_as_uint(v) & 0x7fffffffu);
}
template <typename T> __device__ __forceinline__ T from_abs_bits(unsigned long long b);
template <> __device__ __forceinline__ double from_abs_bits<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}
template <> __device__ __forceinline__ float from_abs_bits<float>(unsigned long long b) {
  return __uint_as_float((unsigned)b);
}

// Fast rotation parameters.  FP32: approximate divides and square roots for the angle
// (it only steers convergence) and one Newton step on c = (1 + t^2)^{-1/2}, so that
// c^2 + s^2 = 1 to about one unit roundoff.  FP64: the FP32 angle, then two FP64 Newton
// steps on c (as in `rotation`).
__device__ __forceinline__ void rotation_fast(float al, float be, float g, float& cs,
                                              float& sn, float& t) {
  const float zeta = __fdividef(be - al, 2.f * g);
  const float az = fabsf(zeta);
  const float q = fmaf(az, az, 1.f);
  t = (az > 1e15f) ? __fdividef(0.5f, az) : __fdividef(1.f, az + q * rsqrtf(q));
  if (zeta < 0.f) t = -t;
  const float x = fmaf(t, t, 1.f);
  float y = rsqrtf(x);
  y = y * fmaf(-0.5f * x, y * y, 1.5f);
  cs = y;
  sn = y * t;
}
__device__ __forceinline__ void rotation_fast(double al, double be, double g, double& cs,
                                              double& sn, double& t) {
  const float zeta = jacobi_zeta(al, be, g);
  const float az = fabsf(zeta);
  const float q = fmaf(az, az, 1.f);
  float tf = (az > 1e15f) ? __fdividef(0.5f, az) : __fdividef(1.f, az + q * rsqrtf(q));
  if (zeta < 0.f) tf = -tf;
  t = double(tf);
  const double x = fma(t, t, 1.0);
  double y = double(rsqrtf(float(x)));
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  cs = y;
  sn = y * t;
}

// FP64 rotation for scaled columns: the tangent t as in rotation_fast, c = (1+t^2)^{-1/2}
// by two FP64 Newton steps, and 1/c = (1 + t^2) c.
__device__ __forceinline__ void rotation_scaled(double al, double be, double g, double& cs,
                                                double& ic, double& t) {
  const float zeta = jacobi_zeta(al, be, g);
  const float az = fabsf(zeta);
  const float q = fmaf(az, az, 1.f);
  float tf = (az > 1e15f) ? __fdividef(0.5f, az) : __fdividef(1.f, az + q * rsqrtf(q));
  if (zeta < 0.f) tf = -tf;
  t = double(tf);
  const double x = fma(t, t, 1.0);
  double y = double(rsqrtf(float(x)));
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  cs = y;
  ic = x * y;
}

// Packed pairs of FP32 values and the two-wide FMA of sm_100-class GPUs; each lane is
// rounded as fmaf rounds it.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float pk_sum(unsigned long long v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return lo + hi;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// A column of a block held in registers by a group of G lanes, E rows per lane: lane gl
// holds rows gl + G e.  The FP32 form holds pairs of adjacent rows instead (rows
// 2 gl + 2 G k and the next, k < E / 2, plus row 2 G (E / 2) + gl for odd E), so that one
// 8-byte load fills a register pair and the dot products and rotations run as two-wide
// FMAs; both forms cover rows 0 .. G E - 1.
template <typename T, int G, int E>
struct RegCol {
  T v[E];
  __device__ __forceinline__ void load(const T* col, int gl, bool active) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? col[gl + G * e] : T(0);
  }
  __device__ __forceinline__ void store(T* col, int gl) const {
#pragma unroll
    for (int e = 0; e < E; ++e) col[gl + G * e] = v[e];
  }
};
template <int G, int E>
struct RegCol<float, G, E> {
  static constexpr int EP = E / 2;
  static constexpr bool kTail = (E % 2) != 0;
  unsigned long long p[EP];
  float t;
  __device__ __forceinline__ void load(const float* col, int gl, bool active) {
#pragma unroll
    for (int k = 0; k < EP; ++k)
      p[k] = active ? *reinterpret_cast<const unsigned long long*>(col + 2 * gl + 2 * G * k)
                    : 0ULL;
    t = (kTail && active) ? col[2 * G * EP + gl] : 0.f;
  }
  __device__ __forceinline__ void store(float* col, int gl) const {
#pragma unroll
    for (int k = 0; k < EP; ++k)
      *reinterpret_cast<unsigned long long*>(col + 2 * gl + 2 * G * k) = p[k];
    if (kTail) col[2 * G * EP + gl] = t;
  }
};

// This lane's part of x . y
template <typename T, int G, int E>
__device__ __forceinline__ T reg_dot(const RegCol<T, G, E>& x, const RegCol<T, G, E>& y) {
  T g = T(0);
#pragma unroll
  for (int e = 0; e < E; ++e) g = fma(x.v[e], y.v[e], g);
  return g;
}
template <int G, int E>
__device__ __forceinline__ float reg_dot(const RegCol<float, G, E>& x,
                                         const RegCol<float, G, E>& y) {
  unsigned long long a = 0ULL;
#pragma unroll
  for (int k = 0; k < RegCol<float, G, E>::EP; ++k) a = fma2(x.p[k], y.p[k], a);
  float g = pk_sum(a);
  if (RegCol<float, G, E>::kTail) g = fmaf(x.t, y.t, g);
  return g;
}

// Pivot key of column c with squared norm s >= 0: the high 32 bits of s (an ordering of
// the non-negative values) above the inverted index, so that the largest key is the
// largest norm and, among equal keys, the smallest index.
__device__ __forceinline__ unsigned long long pivot_key(double s, int c) {
  return ((unsigned long long)__double_as_longlong(s) >> 32 << 32) | (0xffffffffu - (unsigned)c);
}
__device__ __forceinline__ unsigned long long pivot_key(float s, int c) {
  return ((unsigned long long)__float_as_uint(s) << 32) | (0xffffffffu - (unsigned)c);
}
__device__ __forceinline__ int pivot_index(unsigned long long key) {
  return (int)(0xffffffffu - (unsigned)(key & 0xffffffffULL));
}

// Rotate the register-held columns x, y (E rows per lane) given gamma = x.y over the
// group and the squared norms nx, ny (updated).  Returns true when a rotation was
// applied (the pair was not yet orthogonal to the tolerance).
template <typename T, int E>
__device__ __forceinline__ bool rotate_regs(T (&x)[E], T (&y)[E], T& nx, T& ny, T g, T tol2) {
  if (!(nx > T(0) && ny > T(0) && g * g > tol2 * nx * ny)) return false;
  T cs, sn, t;
  rotation_fast(nx, ny, g, cs, sn, t);
  if (sizeof(T) == 4) {
    const T h = sn / (T(1) + cs);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const T xe = x[e], ye = y[e];
      x[e] = fma(-sn, fma(h, xe, ye), xe);
      y[e] = fma(sn, fma(-h, ye, xe), ye);
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const T xe = x[e], ye = y[e];
      x[e] = fma(cs, xe, -sn * ye);
      y[e] = fma(sn, xe, cs * ye);
    }
  }
  nx = nx - t * g;
  ny = ny + t * g;
  return true;
}

// rotate_regs on register columns; the FP32 form applies the same per-row FMAs two rows
// at a time
template <typename T, int G, int E>
__device__ __forceinline__ bool reg_rotate(RegCol<T, G, E>& x, RegCol<T, G, E>& y, T& nx, T& ny,
                                           T g, T tol2) {
  return rotate_regs(x.v, y.v, nx, ny, g, tol2);
}
template <int G, int E>
__device__ __forceinline__ bool reg_rotate(RegCol<float, G, E>& x, RegCol<float, G, E>& y,
                                           float& nx, float& ny, float g, float tol2) {
  if (!(nx > 0.f && ny > 0.f && g * g > tol2 * nx * ny)) return false;
  float cs, sn, t;
  rotation_fast(nx, ny, g, cs, sn, t);
  const float h = sn / (1.f + cs);
  const unsigned long long H = pk2(h, h), NH = pk2(-h, -h), S = pk2(sn, sn), NS = pk2(-sn, -sn);
#pragma unroll
  for (int k = 0; k < RegCol<float, G, E>::EP; ++k) {
    const unsigned long long xe = x.p[k], ye = y.p[k];
    x.p[k] = fma2(NS, fma2(H, xe, ye), xe);
    y.p[k] = fma2(S, fma2(NH, ye, xe), ye);
  }
  if (RegCol<float, G, E>::kTail) {
    const float xe = x.t, ye = y.t;
    x.t = fmaf(-sn, fmaf(h, xe, ye), xe);
    y.t = fmaf(sn, fmaf(-h, ye, xe), ye);
  }
  nx = nx - t * g;
  ny = ny + t * g;
  return true;
}

// Squared column norm below which a converged column is not normalised into the basis
// of a warm start (the working matrix is scaled so that its largest entry lies in
// [1, 2), so these are far below any singular value that matters).
template <typename T> __device__ __forceinline__ T basis_min_norm2();
template <> __device__ __forceinline__ double basis_min_norm2<double>() { return 1e-280; }
template <> __device__ __forceinline__ float basis_min_norm2<float>() { return 1e-30f; }

// Warm-start output of the SVT kernels: the n x n orthonormal basis of the side the
// kernel orthogonalised, Wb(r, c) = Z(r, c) / ||z_c|| (rows in the QR order, Z the
// rotated R^T held as columns of leading dimension ld, z_c its columns 0..n-1) and the
// QR permutation.  A slice that did not converge or has a column of (near) zero norm
// gets the identity and the identity permutation, so that the caller's basis stays
// orthogonal.  Called by every thread of the CTA (contains a barrier).
template <typename T>
__device__ void write_basis(const JacobiIO& io, int64_t slice, int n, int ld, const T* Z,
                            const T* nrm2, const int* perm, bool not_converged) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = !not_converged;
    for (int c = 0; c < n && ok; ++c) {
      const T v = nrm2[c];
      ok = isfinite(v) && v > basis_min_norm2<T>();
    }
    s_ok = ok;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  T* Wo = reinterpret_cast<T*>(io.W) + (size_t)slice * n * n;
  int* Po = io.Wperm + (size_t)slice * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    Wo[idx] = ok ? Z[r + (size_t)ld * c] / sqrt(nrm2[c]) : (r == c ? T(1) : T(0));
  }
  for (int r = threadIdx.x; r < n; r += blockDim.x) Po[r] = ok ? perm[r] : r;
  __syncthreads();
}

// Round-robin pairing on n (even) items: item n-1 fixed, the others on a circle.
__host__ __device__ constexpr int rr_i(int r, int k, int n) {
  return k == 0 ? n - 1 : (r + k) % (n - 1);
}
__host__ __device__ constexpr int rr_j(int r, int k, int n) {
  return k == 0 ? r : (r - k + n - 1) % (n - 1);
}

template <typename T, int G, int E, int B, int MAXT>
__global__ void __launch_bounds__(MAXT)
jacobi_svt_kernel(const JArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const JacobiPlan& jp = a.jp;
  if (a.io.scal != nullptr && a.io.scal->done) return;  // PGA converged earlier

  constexpr int PPW = 32 / G;  // pairs (or rows) per warp
  const int m = jp.m, n = jp.n, np = jp.npad, ld = jp.ld;
  const int64_t I1 = jp.I1, I2 = jp.I2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int gl = lane % G, gw = lane / G;       // lane in group, group in warp
  const int grp = warp * PPW + gw, ngrp = nwarps * PPW;
  const T tol2 = T(a.tol) * T(a.tol);
  const T tau_in = T(a.io.tau);

  unsigned char* sp = smem_raw;
  T* Ws = nullptr;
  if (jp.w_in_smem) { Ws = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)ld * np; }
  T* nrm2 = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
  T* ref = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
  int* perm = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;
  int* list = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;
  // FP64 sweeps keep column i as d_i * (stored column); dsc = d, isc = 1/d
  constexpr bool kScaled = sizeof(T) == 8 && B == 1;
  T* dsc = nullptr;
  T* isc = nullptr;
  if constexpr (kScaled) {
    dsc = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
    isc = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
  }
  __shared__ int s_count, s_rot;
  __shared__ unsigned long long s_key[2];  // pivot keys of the QR steps, by parity
  // FP64 scaled sweeps: per-pair scalars of one batch of pairs (dot product; update
  // coefficients; rescale factors; rotate or not), so that the rotation parameters are
  // computed once per pair by one thread instead of on every lane of the pair's group
  constexpr int kPairs = kScaled ? MAXT / G : 1;
  __shared__ T s_pg[kPairs], s_pa[kPairs], s_pb[kPairs], s_sx[kPairs], s_sy[kPairs];
  __shared__ int s_pr[kPairs];
  __shared__ unsigned long long s_maxbits;

  const T* Ain = reinterpret_cast<const T*>(a.io.A);
  T* W = jp.w_in_smem ? Ws
                      : reinterpret_cast<T*>(a.io.scratch) + (size_t)blockIdx.x * ld * np;

  long long tph[7];  // phase boundaries (thread 0, profiling only)
  long long tqr[4];  // QR sub-phase totals (thread 0, profiling only)
  for (int64_t slice = blockIdx.x; slice < jp.P; slice += gridDim.x) {
    const T* A = Ain + slice * I1 * I2;
    T* D = a.io.D ? reinterpret_cast<T*>(a.io.D) + slice * I1 * I2 : nullptr;
    if (a.io.phases && threadIdx.x == 0) tph[0] = clock64();
    // ---- load B; zero the padding rows and column
    if (!jp.transposed) {
      for (int idx = threadIdx.x; idx < ld * np; idx += blockDim.x) {
        const int r = idx % ld, c = idx / ld;
        W[idx] = (r < m && c < n) ? A[r + I1 * c] : T(0);
      }
    } else {
      // consecutive threads fill consecutive rows of a column of W (the reads of the
      // slice are strided; it comes from L2 once)
      for (int idx = threadIdx.x; idx < n * m; idx += blockDim.x) {
        const int r = idx % m, c = idx / m;
        W[r + (size_t)ld * c] = A[c + I1 * r];
      }
      for (int idx = threadIdx.x; idx < ld * np; idx += blockDim.x) {
        const int r = idx % ld, c = idx / ld;
        if (r >= m || c >= n) W[idx] = T(0);
      }
    }
    if (threadIdx.x == 0) s_maxbits = 0ULL;
    __syncthreads();
    // ---- scale by a power of two (exact) so that the largest entry lies in [1, 2):
    // D_tau(B) = D_{s tau}(s B) / s, and the reconstruction below, which re-reads the
    // unscaled slice, needs no correction (Z and g scale by s and 1/s^2)
    {
      unsigned long long mb = 0ULL;
      for (int idx = threadIdx.x; idx < ld * np; idx += blockDim.x) {
        const unsigned long long v = abs_bits(W[idx]);
        mb = v > mb ? v : mb;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = v > mb ? v : mb;
      }
      if (lane == 0) atomicMax(&s_maxbits, mb);
    }
    __syncthreads();
    const T sc = pow2_scale(from_abs_bits<T>(s_maxbits));
    if (sc != T(1))
      for (int idx = threadIdx.x; idx < ld * np; idx += blockDim.x) W[idx] *= sc;
    // truncation keeps sigma unshrunk: g_i = 1 / sigma_i^2 is the SVT rule at tau = 0
    const T tau = jp.mode == JAC_SVT ? tau_in * sc : T(0);
    __syncthreads();

    if (a.io.phases && threadIdx.x == 0) tph[1] = clock64();
    // ---- 1. QR with column pivoting: B P = Q R (R in the upper triangle).  The norms of
    // the remaining columns are recomputed exactly by the trailing update of each step
    // (rows j+1.. of the updated columns; no downdating), and the next pivot is the
    // maximum of the keys (norm bits, inverted index) that the updating lanes post to
    // shared memory, so that every thread finds the pivot and the Householder vector
    // itself: two barriers per step.
    if (threadIdx.x == 0) { s_key[0] = 0ULL; s_key[1] = 0ULL; }
    __syncthreads();
    for (int c = warp; c < n; c += nwarps) {
      const T* col = W + (size_t)ld * c;
      T s = T(0);
      for (int r = lane; r < m; r += 32) s = fma(col[r], col[r], s);
      s = warp_allsum(s);
      if (lane == 0) {
        nrm2[c] = s;
        perm[c] = c;
        atomicMax(&s_key[0], pivot_key(s, c));
      }
    }
    __syncthreads();
    const bool prof = a.io.phases != nullptr && threadIdx.x == 0;
    long long tq = prof ? clock64() : 0;
    if (prof) tqr[0] = tqr[1] = tqr[2] = tqr[3] = 0;
    T alpha_prev = T(0);  // R(j-1, j-1), stored once every thread has read B(j-1, j-1)
    for (int j = 0; j < n; ++j) {
      // pivot: the remaining column of largest norm (ties: the smaller index)
      const int p = pivot_index(s_key[j & 1]);
      const T s = nrm2[p];  // ||B(j:m, p)||^2
      if (prof) { const long long t = clock64(); tqr[0] += t - tq; tq = t; }
      if (p != j) {
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
          const T t0 = W[r + (size_t)ld * j];
          W[r + (size_t)ld * j] = W[r + (size_t)ld * p];
          W[r + (size_t)ld * p] = t0;
        }
      }
      if (threadIdx.x == 0) {
        if (j > 0) W[(j - 1) + (size_t)ld * (j - 1)] = alpha_prev;
        if (p != j) { const int t2 = perm[j]; perm[j] = perm[p]; perm[p] = t2; }
        s_key[(j + 1) & 1] = 0ULL;  // read last in step j - 1, before its second barrier
      }
      __syncthreads();
      if (prof) { const long long t = clock64(); tqr[1] += t - tq; tq = t; }
      // Householder vector v = x - alpha e_1 of x = B(j:m, j), on every thread
      const T* vj = W + (size_t)ld * j;
      const T x0 = vj[j];
      const T nx = sqrt(s);
      const T alpha = (x0 >= T(0)) ? -nx : nx;
      const T v0 = x0 - alpha;
      // beta = 2 / (v.v) = 1 / (alpha (alpha - x0)) = 1 / (||x|| (||x|| + |x0|))
      const T beta = (s > T(0)) ? T(1) / (nx * (nx + fabs(x0))) : T(0);
      if (prof) { const long long t = clock64(); tqr[2] += t - tq; tq = t; }
      // B(j:m, c) -= beta v (v . B(j:m, c)) for c > j; a warp takes four columns at a
      // time so that four dot products and reductions are in flight together, and sums
      // the squares of rows j+1.. of the updated columns (the next step's norms)
      for (int c0 = j + 1 + 4 * warp; c0 < n; c0 += 4 * nwarps) {
        T* col[4];
        T w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c0 + u < n ? c0 + u : c0;  // duplicates are read-only below
          col[u] = W + (size_t)ld * c;
          w[u] = (lane == 0) ? v0 * col[u][j] : T(0);
        }
        for (int r = j + 1 + lane; r < m; r += 32) {
          const T vr = vj[r];
#pragma unroll
          for (int u = 0; u < 4; ++u) w[u] = fma(vr, col[u][r], w[u]);
        }
        warp_allsum4(w);
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] *= beta;
        __syncwarp();
        T sq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sq[u] = T(0);
          if (c0 + u >= n) continue;  // uniform over the warp
          T* cu = col[u];
          if (lane == 0) cu[j] = fma(-w[u], v0, cu[j]);
          for (int r = j + 1 + lane; r < m; r += 32) {
            const T v = fma(-w[u], vj[r], cu[r]);
            cu[r] = v;
            sq[u] = fma(v, v, sq[u]);
          }
        }
        warp_allsum4(sq);
        if (lane < 4 && c0 + lane < n) {
          const T q = lane == 0 ? sq[0] : lane == 1 ? sq[1] : lane == 2 ? sq[2] : sq[3];
          nrm2[c0 + lane] = q;
          atomicMax(&s_key[(j + 1) & 1], pivot_key(q, c0 + lane));
        }
      }
      alpha_prev = alpha;
      __syncthreads();
      if (prof) { const long long t = clock64(); tqr[3] += t - tq; tq = t; }
    }
    if (threadIdx.x == 0 && n > 0) W[(n - 1) + (size_t)ld * (n - 1)] = alpha_prev;
    __syncthreads();
    // ---- Z = R^T (lower triangular), rows n.. zeroed
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx % n, c = idx / n;
      if (r > c) {
        W[r + (size_t)ld * c] = W[c + (size_t)ld * r];
        W[c + (size_t)ld * r] = T(0);
      }
    }
    for (int idx = threadIdx.x; idx < (ld - n) * n; idx += blockDim.x) {
      const int r = n + idx % (ld - n), c = idx / (ld - n);
      W[r + (size_t)ld * c] = T(0);
    }
    if constexpr (kScaled)
      for (int c = threadIdx.x; c < np; c += blockDim.x) { dsc[c] = T(1); isc[c] = T(1); }
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    if (a.io.phases && threadIdx.x == 0) tph[2] = clock64();

    // ---- 2. one-sided Jacobi on Z (n x n), a group of G lanes per pair
    // Squared column norms, a group per column; scaled columns are first multiplied out
    // (d_i <- 1), so that the scales stay bounded and Z is in true units afterwards.
    auto column_norms = [&]() {
      for (int c0 = 0; c0 < np; c0 += ngrp) {  // trip count uniform over the warp
        const int c = c0 + grp;
        T* col = W + (size_t)ld * (c < np ? c : 0);
        T s = T(0);
        if constexpr (kScaled) {
          const T dc = c < np ? dsc[c] : T(1);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const T v = col[gl + G * e] * dc;
            if (c < np) col[gl + G * e] = v;
            s = fma(v, v, s);
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) s = fma(col[gl + G * e], col[gl + G * e], s);
        }
        s = group_sum<G>(s);
        if (gl == 0 && c < np) {
          nrm2[c] = s;
          if constexpr (kScaled) { dsc[c] = T(1); isc[c] = T(1); }
        }
      }
    };
    int sweeps = 0, nrot = 0;
    bool rotated = true;
    const int npairs = np / 2, cfix = np - 1;
    while (rotated && sweeps < a.max_sweeps) {
      column_norms();
      __syncthreads();
      int flag = 0;
      if constexpr (B > 1) {
        // Blocks of B columns; a group holds a block pair (2B columns) in registers and
        // performs all B^2 cross rotations (and, in the first block round of the sweep,
        // the intra-block ones) before writing back: B times fewer passes of the matrix
        // through shared memory per rotation, B independent rotations per step.
        const int nb = np / B, cfb = nb - 1;
        for (int br = 0; br < cfb; ++br) {
          for (int k0 = 0; k0 < nb / 2; k0 += ngrp) {
            const int k = k0 + grp;
            const bool active = k < nb / 2;
            int bx = 0, by = 0;
            if (active) {
              if (k == 0) {
                bx = cfb;
                by = br;
              } else {
                bx = br + k;
                if (bx >= cfb) bx -= cfb;
                by = br - k;
                if (by < 0) by += cfb;
              }
            }
            RegCol<T, G, E> X[B], Y[B];
            T nx[B], ny[B];
#pragma unroll
            for (int c = 0; c < B; ++c) {
              X[c].load(W + (size_t)ld * (bx * B + c), gl, active);
              Y[c].load(W + (size_t)ld * (by * B + c), gl, active);
              nx[c] = active ? nrm2[bx * B + c] : T(0);
              ny[c] = active ? nrm2[by * B + c] : T(0);
            }
            if (br == 0) {  // intra-block pairs, once per sweep
#pragma unroll
              for (int r = 0; r < B - 1; ++r) {
#pragma unroll
                for (int kk = 0; kk < B / 2; ++kk) {
                  const int i = rr_i(r, kk, B), j = rr_j(r, kk, B);
                  T g1 = reg_dot(X[i], X[j]), g2 = reg_dot(Y[i], Y[j]);
                  g1 = group_sum<G>(g1);
                  g2 = group_sum<G>(g2);
                  if (reg_rotate(X[i], X[j], nx[i], nx[j], g1, tol2)) { flag = 1; nrot += (gl == 0); }
                  if (reg_rotate(Y[i], Y[j], ny[i], ny[j], g2, tol2)) { flag = 1; nrot += (gl == 0); }
                }
              }
            }
#pragma unroll
            for (int q = 0; q < B; ++q) {  // cross pairs (X_i, Y_{(i+q) mod B})
              T g[B];
#pragma unroll
              for (int i = 0; i < B; ++i) g[i] = reg_dot(X[i], Y[(i + q) % B]);
#pragma unroll
              for (int i = 0; i < B; ++i) g[i] = group_sum<G>(g[i]);
#pragma unroll
              for (int i = 0; i < B; ++i)
                if (reg_rotate(X[i], Y[(i + q) % B], nx[i], ny[(i + q) % B], g[i], tol2)) {
                  flag = 1;
                  nrot += (gl == 0);
                }
            }
            if (active) {
#pragma unroll
              for (int c = 0; c < B; ++c) {
                X[c].store(W + (size_t)ld * (bx * B + c), gl);
                Y[c].store(W + (size_t)ld * (by * B + c), gl);
                if (gl == 0) {
                  nrm2[bx * B + c] = nx[c];
                  nrm2[by * B + c] = ny[c];
                }
              }
            }
          }
          __syncthreads();
        }
      } else
      for (int rnd = 0; rnd < cfix; ++rnd) {
        for (int k0 = 0; k0 < npairs; k0 += ngrp) {  // every group of the CTA takes a pair
          const int k = k0 + grp;
          const bool active = k < npairs;
          int i = 0, j = 0;
          if (active) {
            if (k == 0) {
              i = cfix;
              j = rnd;
            } else {
              i = rnd + k;
              if (i >= cfix) i -= cfix;
              j = rnd - k;
              if (j < 0) j += cfix;
            }
          }
          T* ci = W + (size_t)ld * i;
          T* cj = W + (size_t)ld * j;
          T x[E], y[E];
          T g = T(0);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            x[e] = active ? ci[gl + G * e] : T(0);
            y[e] = active ? cj[gl + G * e] : T(0);
            g = fma(x[e], y[e], g);
          }
          g = group_sum<G>(g);
          if constexpr (kScaled) {
            // columns d_i x~, d_j y~: the rotation x' = c (x - t y), y' = c (y + t x)
            // becomes x~' = x~ - t (d_j / d_i) y~, y~' = y~ + t (d_i / d_j) x~ with
            // d_i' = c d_i, d_j' = c d_j: two FP64 multiply-adds per row instead of four
            // (Rutishauser-style scaled rotations; the scales are multiplied out at each
            // sweep start and whenever one falls below 2^-64).  Three phases: the groups'
            // dot products, the per-pair parameters (one thread per pair), the groups'
            // column updates.
            if (gl == 0) s_pg[grp] = g;
            __syncthreads();
            const int batch = min(ngrp, npairs - k0);
            for (int q = threadIdx.x; q < batch; q += blockDim.x) {
              const int kq = k0 + q;
              int pi, pj;
              if (kq == 0) {
                pi = cfix;
                pj = rnd;
              } else {
                pi = rnd + kq;
                if (pi >= cfix) pi -= cfix;
                pj = rnd - kq;
                if (pj < 0) pj += cfix;
              }
              const T al = nrm2[pi], be = nrm2[pj];
              const T di = dsc[pi], dj = dsc[pj];
              const T gq = s_pg[q] * (di * dj);
              int rot = 0;
              if (al > T(0) && be > T(0) && gq * gq > tol2 * al * be) {
                T cs, ic, t;
                rotation_scaled(al, be, gq, cs, ic, t);
                const T ei = isc[pi], ej = isc[pj];
                T di2 = di * cs, dj2 = dj * cs, ei2 = ei * ic, ej2 = ej * ic;
                s_pa[q] = t * dj * ei;
                s_pb[q] = t * di * ej;
                T fx = T(1), fy = T(1);
                if (di2 < T(0x1p-64)) { fx = di2; di2 = ei2 = T(1); }
                if (dj2 < T(0x1p-64)) { fy = dj2; dj2 = ej2 = T(1); }
                s_sx[q] = fx;
                s_sy[q] = fy;
                nrm2[pi] = al - t * gq;
                nrm2[pj] = be + t * gq;
                dsc[pi] = di2;
                dsc[pj] = dj2;
                isc[pi] = ei2;
                isc[pj] = ej2;
                ++nrot;
                flag = 1;
                rot = 1;
              }
              s_pr[q] = rot;
            }
            __syncthreads();
            if (active && s_pr[grp]) {  // uniform over the group
              const T alpha = s_pa[grp], beta = s_pb[grp];
#pragma unroll
              for (int e = 0; e < E; ++e) {
                const T xe = x[e], ye = y[e];
                x[e] = fma(-alpha, ye, xe);
                y[e] = fma(beta, xe, ye);
              }
              const T fx = s_sx[grp], fy = s_sy[grp];
              if (fx != T(1)) {
#pragma unroll
                for (int e = 0; e < E; ++e) x[e] *= fx;
              }
              if (fy != T(1)) {
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] *= fy;
              }
#pragma unroll
              for (int e = 0; e < E; ++e) {
                ci[gl + G * e] = x[e];
                cj[gl + G * e] = y[e];
              }
            }
            continue;
          }
          const T al = active ? nrm2[i] : T(0), be = active ? nrm2[j] : T(0);
          if (al > T(0) && be > T(0) && g * g > tol2 * al * be) {
            T cs, sn, t;
            rotation_fast(al, be, g, cs, sn, t);
            if (sizeof(T) == 4) {
              // FP32: x' = x - s (y + h x), y' = y + s (x - h y), h = s / (1 + c): the
              // update is a small increment, so a small rotation adds rounding error of
              // the size of the increment and stays orthogonal to ~s^2 u.
              const T h = sn / (T(1) + cs);
#pragma unroll
              for (int e = 0; e < E; ++e) {
                ci[gl + G * e] = fma(-sn, fma(h, x[e], y[e]), x[e]);
                cj[gl + G * e] = fma(sn, fma(-h, y[e], x[e]), y[e]);
              }
            } else {
              // FP64: x' = c x - s y, y' = s x + c y (no divide; rounding at 2^-53 per
              // rotation is far below the FP64 tolerance)
#pragma unroll
              for (int e = 0; e < E; ++e) {
                ci[gl + G * e] = fma(cs, x[e], -sn * y[e]);
                cj[gl + G * e] = fma(sn, x[e], cs * y[e]);
              }
            }
            if (gl == 0) {
              nrm2[i] = al - t * g;
              nrm2[j] = be + t * g;
              ++nrot;
            }
            flag = 1;
          }
        }
        __syncthreads();
      }
      rotated = __syncthreads_or(flag) != 0;
      ++sweeps;
    }
    column_norms();
    if (nrot) atomicAdd(&s_rot, nrot);
    __syncthreads();
    if (a.io.W != nullptr) write_basis(a.io, slice, n, ld, W, nrm2, perm, rotated);
    if (a.io.phases && threadIdx.x == 0) tph[3] = clock64();

    // ---- 3. shrink (or truncate, or report sigma) and reconstruct
    if (jp.mode == JAC_TRUNC) {
      // keep column c when fewer than trunc_k columns have a larger norm (ties by
      // index) and its norm is nonzero; the flag goes to ref[], free after the QR
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const T sc2 = nrm2[c];
        int64_t rank = 0;
        for (int c2 = 0; c2 < n; ++c2) {
          const T s2 = nrm2[c2];
          rank += (s2 > sc2 || (s2 == sc2 && c2 < c)) ? 1 : 0;
        }
        ref[c] = (rank < a.io.trunc_k && sc2 > T(0)) ? T(1) : T(0);
      }
      __syncthreads();
    }
    if (a.io.sigma)
      for (int c = threadIdx.x; c < n; c += blockDim.x)
        reinterpret_cast<T*>(a.io.sigma)[slice * n + c] = sqrt(nrm2[c]) / sc;
    if (threadIdx.x == 0) {
      int st = 0, k = 0;
      T nuc = T(0);
      if (rotated) st |= LT_DEV_NOCONV;
      for (int c = 0; c < n; ++c) {
        const T s2 = nrm2[c];
        if (!isfinite(s2)) st |= LT_DEV_NONFINITE;
        const T sg = sqrt(s2);
        const bool keep = jp.mode == JAC_SVT ? sg > tau : (jp.mode == JAC_TRUNC && ref[c] != T(0));
        if (keep) {
          list[k++] = c;
          nuc += sg - tau;
        }
      }
      if (st) atomicOr(a.status, st);
      s_count = k;
      if (a.io.phases) tph[4] = clock64();
      if (a.io.info) {
        a.io.info[slice].sweeps = sweeps;
        a.io.info[slice].rank = k;
        a.io.info[slice].nuclear = double(nuc) / double(sc);
      }
      if (a.io.flops) {
        const double md = m, nd = n;
        const double f = 2.0 * md * nd * nd - 2.0 * nd * nd * nd / 3.0 +   // QR
                         sweeps * (nd * (nd - 1) * nd + 2 * nd * nd) +      // dots + norms
                         (kScaled ? 4.0 : 6.0) * nd * s_rot + 2 * nd * nd + // rotations
                         4.0 * k * md * nd;                                 // reconstruction
        atomicAdd(a.io.flops, f);
      }
    }
    __syncthreads();
    const int k = s_count;
    for (int q = threadIdx.x; q < k; q += blockDim.x) {  // nrm2[c] <- g_c for kept c
      const int c = list[q];
      const T sg = sqrt(nrm2[c]);
      nrm2[c] = ((sg - tau) / sg) / sg / sg;
    }
    __syncthreads();
    if (a.io.phases && threadIdx.x == 0) tph[5] = clock64();
    // a warp per row of B P, lane l holding columns l, l+32, ... (ER per lane)
    constexpr int ER = (G * E + 31) / 32;
    const int rows_iter = D != nullptr ? (m + nwarps - 1) / nwarps : 0;
    for (int it = 0; it < rows_iter; ++it) {
      const int r = it * nwarps + warp;
      const bool active = r < m;
      T b[ER];
#pragma unroll
      for (int e = 0; e < ER; ++e) {
        const int c = lane + 32 * e;
        b[e] = T(0);
        if (active && c < n) {
          const int pc = perm[c];
          b[e] = jp.transposed ? A[pc + I1 * r] : A[r + I1 * pc];
        }
      }
      // y_q = g_q (b . z_q), kept in registers: y_q lives on lane q % 32, slot q / 32
      T yreg[ER];
#pragma unroll
      for (int s2 = 0; s2 < ER; ++s2) {
        yreg[s2] = T(0);
        const int qn = min(32, k - s2 * 32);  // uniform over the CTA
        int gq = 0;
        if constexpr (ER <= 8)
        for (; gq + 4 <= qn; gq += 4) {  // four independent dot products in flight
          const T* z0 = W + (size_t)ld * list[s2 * 32 + gq];
          const T* z1 = W + (size_t)ld * list[s2 * 32 + gq + 1];
          const T* z2 = W + (size_t)ld * list[s2 * 32 + gq + 2];
          const T* z3 = W + (size_t)ld * list[s2 * 32 + gq + 3];
          T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
          for (int e = 0; e < ER; ++e) {
            d0 = fma(z0[lane + 32 * e], b[e], d0);
            d1 = fma(z1[lane + 32 * e], b[e], d1);
            d2 = fma(z2[lane + 32 * e], b[e], d2);
            d3 = fma(z3[lane + 32 * e], b[e], d3);
          }
          T dv[4] = {d0, d1, d2, d3};
          warp_allsum4(dv);
          d0 = dv[0]; d1 = dv[1]; d2 = dv[2]; d3 = dv[3];
          if (lane == gq) yreg[s2] = d0 * nrm2[list[s2 * 32 + gq]];
          if (lane == gq + 1) yreg[s2] = d1 * nrm2[list[s2 * 32 + gq + 1]];
          if (lane == gq + 2) yreg[s2] = d2 * nrm2[list[s2 * 32 + gq + 2]];
          if (lane == gq + 3) yreg[s2] = d3 * nrm2[list[s2 * 32 + gq + 3]];
        }
        for (; gq < qn; ++gq) {
          const T* z = W + (size_t)ld * list[s2 * 32 + gq];
          T d = T(0);
#pragma unroll
          for (int e = 0; e < ER; ++e) d = fma(z[lane + 32 * e], b[e], d);
          d = warp_allsum(d);
          if (lane == gq) yreg[s2] = d * nrm2[list[s2 * 32 + gq]];
        }
      }
      T out[ER];
#pragma unroll
      for (int e = 0; e < ER; ++e) out[e] = T(0);
#pragma unroll
      for (int s2 = 0; s2 < ER; ++s2) {
        const int qn = min(32, k - s2 * 32);
        for (int gq = 0; gq < qn; ++gq) {
          const T yq = __shfl_sync(0xffffffffu, yreg[s2], gq);
          const T* z = W + (size_t)ld * list[s2 * 32 + gq];
#pragma unroll
          for (int e = 0; e < ER; ++e) out[e] = fma(yq, z[lane + 32 * e], out[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < ER; ++e) {
        const int c = lane + 32 * e;
        if (active && c < n) {
          const int pc = perm[c];
          if (jp.transposed) D[pc + I1 * r] = out[e];
          else D[r + I1 * pc] = out[e];
        }
      }
    }
    __syncthreads();
    if (a.io.phases && threadIdx.x == 0) {
      tph[6] = clock64();
      for (int q = 0; q < 6; ++q) atomicAdd(a.io.phases + q, double(tph[q + 1] - tph[q]));
      for (int q = 0; q < 4; ++q) atomicAdd(a.io.phases + 6 + q, double(tqr[q]));
    }
  }
}

}  // namespace jac
}  // namespace lt
