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
  const float zeta = __fdividef(float(be - al), 2.f * float(g));
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

template <typename T, int G, int E, int MAXT>
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
  const T tau = T(a.io.tau);

  unsigned char* sp = smem_raw;
  T* Ws = nullptr;
  if (jp.w_in_smem) { Ws = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)ld * np; }
  T* nrm2 = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
  T* ref = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
  int* perm = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;
  int* list = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;
  __shared__ int s_piv, s_count, s_rot;
  __shared__ T s_alpha, s_beta, s_v0;

  const T* Ain = reinterpret_cast<const T*>(a.io.A);
  T* W = jp.w_in_smem ? Ws
                      : reinterpret_cast<T*>(a.io.scratch) + (size_t)blockIdx.x * ld * np;

  for (int64_t slice = blockIdx.x; slice < jp.P; slice += gridDim.x) {
    const T* A = Ain + slice * I1 * I2;
    T* D = reinterpret_cast<T*>(a.io.D) + slice * I1 * I2;
    // ---- load B; zero the padding rows and column
    if (!jp.transposed) {
      for (int idx = threadIdx.x; idx < ld * np; idx += blockDim.x) {
        const int r = idx % ld, c = idx / ld;
        W[idx] = (r < m && c < n) ? A[r + I1 * c] : T(0);
      }
    } else {
      for (int idx = threadIdx.x; idx < n * m; idx += blockDim.x) {
        const int c = idx % n, r = idx / n;
        W[r + (size_t)ld * c] = A[c + I1 * r];
      }
      for (int idx = threadIdx.x; idx < ld * np; idx += blockDim.x) {
        const int r = idx % ld, c = idx / ld;
        if (r >= m || c >= n) W[idx] = T(0);
      }
    }
    __syncthreads();

    // ---- 1. QR with column pivoting: B P = Q R (R in the upper triangle)
    for (int c = warp; c < n; c += nwarps) {
      const T* col = W + (size_t)ld * c;
      T s = T(0);
      for (int r = lane; r < m; r += 32) s = fma(col[r], col[r], s);
      s = warp_allsum(s);
      if (lane == 0) { nrm2[c] = s; ref[c] = s; perm[c] = c; }
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      if (warp == 0) {  // pivot: the remaining column of largest norm
        T best = T(-1);
        int bi = j;
        for (int c = j + lane; c < n; c += 32)
          if (nrm2[c] > best) { best = nrm2[c]; bi = c; }
        warp_argmax(best, bi);
        if (lane == 0) s_piv = bi;
      }
      __syncthreads();
      const int p = s_piv;
      if (p != j) {
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
          const T t0 = W[r + (size_t)ld * j];
          W[r + (size_t)ld * j] = W[r + (size_t)ld * p];
          W[r + (size_t)ld * p] = t0;
        }
        if (threadIdx.x == 0) {
          T t1 = nrm2[j]; nrm2[j] = nrm2[p]; nrm2[p] = t1;
          t1 = ref[j]; ref[j] = ref[p]; ref[p] = t1;
          const int t2 = perm[j]; perm[j] = perm[p]; perm[p] = t2;
        }
      }
      __syncthreads();
      if (warp == 0) {  // Householder vector v = x - alpha e_1 of x = B(j:m, j)
        const T* col = W + (size_t)ld * j;
        T s = T(0);
        for (int r = j + lane; r < m; r += 32) s = fma(col[r], col[r], s);
        s = warp_allsum(s);
        if (lane == 0) {
          const T x0 = col[j];
          const T nx = sqrt(s);
          const T alpha = (x0 >= T(0)) ? -nx : nx;
          s_alpha = alpha;
          s_v0 = x0 - alpha;
          // beta = 2 / (v.v) = 1 / (alpha (alpha - x0)) = 1 / (||x|| (||x|| + |x0|))
          s_beta = (s > T(0)) ? T(1) / (nx * (nx + fabs(x0))) : T(0);
        }
      }
      __syncthreads();
      const T alpha = s_alpha, beta = s_beta, v0 = s_v0;
      const T* vj = W + (size_t)ld * j;
      for (int c = j + 1 + warp; c < n; c += nwarps) {  // B(j:m, c) -= beta v (v . B(j:m, c))
        T* col = W + (size_t)ld * c;
        T w = (lane == 0) ? v0 * col[j] : T(0);
        for (int r = j + 1 + lane; r < m; r += 32) w = fma(vj[r], col[r], w);
        w = warp_allsum(w) * beta;
        if (lane == 0) col[j] = fma(-w, v0, col[j]);
        for (int r = j + 1 + lane; r < m; r += 32) col[r] = fma(-w, vj[r], col[r]);
        __syncwarp();
        // downdate the remaining norm; recompute it when cancellation has eaten it
        const T rjc = col[j];
        T nn = nrm2[c] - rjc * rjc;
        if (nn <= T(0.01) * ref[c]) {
          T s = T(0);
          for (int r = j + 1 + lane; r < m; r += 32) s = fma(col[r], col[r], s);
          nn = warp_allsum(s);
          if (lane == 0) ref[c] = nn;
        }
        if (lane == 0) nrm2[c] = nn > T(0) ? nn : T(0);
      }
      if (threadIdx.x == 0) W[j + (size_t)ld * j] = alpha;
      __syncthreads();
    }
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
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();

    // ---- 2. one-sided Jacobi on Z (n x n), a group of G lanes per pair
    int sweeps = 0, nrot = 0;
    bool rotated = true;
    const int npairs = np / 2, cfix = np - 1;
    while (rotated && sweeps < a.max_sweeps) {
      for (int c0 = 0; c0 < np; c0 += ngrp) {  // trip count uniform over the warp
        const int c = c0 + grp;
        const T* col = W + (size_t)ld * (c < np ? c : 0);
        T s = T(0);
#pragma unroll
        for (int e = 0; e < E; ++e) s = fma(col[gl + G * e], col[gl + G * e], s);
        s = group_sum<G>(s);
        if (gl == 0 && c < np) nrm2[c] = s;
      }
      __syncthreads();
      int flag = 0;
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
    for (int c0 = 0; c0 < np; c0 += ngrp) {
      const int c = c0 + grp;
      const T* col = W + (size_t)ld * (c < np ? c : 0);
      T s = T(0);
#pragma unroll
      for (int e = 0; e < E; ++e) s = fma(col[gl + G * e], col[gl + G * e], s);
      s = group_sum<G>(s);
      if (gl == 0 && c < np) nrm2[c] = s;
    }
    if (nrot) atomicAdd(&s_rot, nrot);
    __syncthreads();

    // ---- 3. shrink and reconstruct
    if (threadIdx.x == 0) {
      int st = 0, k = 0;
      T nuc = T(0);
      if (rotated) st |= LT_DEV_NOCONV;
      for (int c = 0; c < n; ++c) {
        const T s2 = nrm2[c];
        if (!isfinite(s2)) st |= LT_DEV_NONFINITE;
        const T sg = sqrt(s2);
        if (sg > tau) {
          list[k++] = c;
          nuc += sg - tau;
        }
      }
      if (st) atomicOr(a.status, st);
      s_count = k;
      if (a.io.info) {
        a.io.info[slice].sweeps = sweeps;
        a.io.info[slice].rank = k;
        a.io.info[slice].nuclear = double(nuc);
      }
      if (a.io.flops) {
        const double md = m, nd = n;
        const double f = 2.0 * md * nd * nd - 2.0 * nd * nd * nd / 3.0 +   // QR
                         sweeps * (nd * (nd - 1) * nd + 2 * nd * nd) +      // dots + norms
                         6.0 * nd * s_rot + 2 * nd * nd +                   // rotations
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
    // a warp per row of B P, lane l holding columns l, l+32, ... (ER per lane)
    constexpr int ER = (G * E + 31) / 32;
    const int rows_iter = (m + nwarps - 1) / nwarps;
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
        for (int gq = 0; gq < 32; ++gq) {
          const int q = s2 * 32 + gq;
          if (q < k) {  // uniform over the CTA
            const T* z = W + (size_t)ld * list[q];
            T d = T(0);
#pragma unroll
            for (int e = 0; e < ER; ++e) d = fma(z[lane + 32 * e], b[e], d);
            d = warp_allsum(d);
            if (lane == gq) yreg[s2] = d * nrm2[list[q]];
          }
        }
      }
      T out[ER];
#pragma unroll
      for (int e = 0; e < ER; ++e) out[e] = T(0);
#pragma unroll
      for (int s2 = 0; s2 < ER; ++s2) {
        for (int gq = 0; gq < 32; ++gq) {
          const int q = s2 * 32 + gq;
          if (q < k) {
            const T yq = __shfl_sync(0xffffffffu, yreg[s2], gq);
            const T* z = W + (size_t)ld * list[q];
#pragma unroll
            for (int e = 0; e < ER; ++e) out[e] = fma(yq, z[lane + 32 * e], out[e]);
          }
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
  }
}

}  // namespace jac
}  // namespace lt
