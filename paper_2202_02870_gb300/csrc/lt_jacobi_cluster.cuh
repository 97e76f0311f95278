// Kernel J, cluster form: the SVT of one frontal slice (Algorithm 4: svd, shrink,
// reconstruct) on a thread-block cluster of C CTAs instead of one CTA, so that a launch
// with fewer slices than SMs, or slices whose working matrix exceeds one CTA's shared
// memory, still spreads over the GPU.  The steps are those of jacobi_svt_kernel
// (lt_jacobi_svt.cuh): QR with column pivoting, one-sided Jacobi on R^T with the
// round-robin ordering, shrink and reconstruction without Q or V.
//
// Distribution: column c of the working matrix (and its squared norm, scales and
// permutation entry) lives in the shared memory of CTA c mod C, at local index c / C.
// Every CTA reaches the others' columns through distributed shared memory
// (shared::cluster addresses from mapa).
//   QR      step j: each CTA proposes its best pivot; the owner of column j swaps and
//           forms the Householder vector; every CTA copies the vector and updates its
//           own columns (two cluster barriers per step).
//   Jacobi  parallel block Jacobi: two half-blocks of columns per CTA, all pairs between
//           and (once per sweep) inside them rotated in the CTA's own shared memory,
//           then the half-blocks move on a round-robin tournament of the 2C half-blocks
//           (cluster barriers only around the moves).  Sweeps end when no CTA rotated.
//   Recon.  CTA r computes the rows r, r + C, ... of the result, reading the kept
//           columns of Z from their owners.
// No remote atomics: per-CTA values (pivot candidates, maxima, flags, counts) go to
// slots in CTA 0 and are read back after a barrier.  Every loop that contains a cluster
// barrier has a trip count that is uniform over the cluster.
#pragma once

#include <cooperative_groups.h>

#include "lt_jacobi_svt.cuh"

namespace lt {
namespace jac {

namespace cgx = cooperative_groups;

// Distributed shared memory by explicit shared::cluster addresses (mapa), so that remote
// accesses take the shared-memory path rather than generic loads through the LSU.
__device__ __forceinline__ uint32_t dsm_addr(const void* local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
  return r;
}
__device__ __forceinline__ double dsm_ld(uint32_t a, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float dsm_ld(uint32_t a, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ int dsm_ld(uint32_t a, int) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long dsm_ld(uint32_t a, unsigned long long) {
  unsigned long long v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void dsm_st(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" :: "r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void dsm_st(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" :: "r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void dsm_st(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_st(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" :: "r"(a), "l"(v) : "memory");
}

template <typename T, int G, int E, int C, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
jacobi_svt_cluster_kernel(const JArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgx::cluster_group cl = cgx::this_cluster();
  const JacobiPlan& jp = a.jp;
  // uniform over the cluster: every CTA reads the same flag, written by an earlier kernel
  if (a.io.scal != nullptr && a.io.scal->done) return;

  constexpr int PPW = 32 / G;
  constexpr bool kScaled = sizeof(T) == 8;
  const int m = jp.m, n = jp.n, np = jp.npad, ld = jp.ld, nl = np / C;
  const int64_t I1 = jp.I1, I2 = jp.I2;
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int gl = lane % G, gw = lane / G;
  const int grp = warp * PPW + gw, ngrp = nwarps * PPW;
  const T tol2 = T(a.tol) * T(a.tol);

  unsigned char* sp = smem_raw;
  T* Wl = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)ld * nl;
  T* nrm2 = reinterpret_cast<T*>(sp); sp += sizeof(T) * nl;
  T* ref = reinterpret_cast<T*>(sp); sp += sizeof(T) * nl;
  T* dsc = reinterpret_cast<T*>(sp); sp += sizeof(T) * nl;
  T* isc = reinterpret_cast<T*>(sp); sp += sizeof(T) * nl;
  T* vbuf = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)ld;
  T* gval = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;      // all columns (copy)
  int* perm = reinterpret_cast<int*>(sp); sp += sizeof(int) * nl;
  int* permall = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;
  int* list = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;

  constexpr int kPairs = MAXT / G;
  __shared__ T s_pg[kPairs], s_pa[kPairs], s_pb[kPairs], s_sx[kPairs], s_sy[kPairs];
  __shared__ int s_pr[kPairs];
  // slots written by every CTA into CTA 0's copy
  __shared__ unsigned long long s_maxslot[C];
  __shared__ T s_candv[C];
  __shared__ int s_candi[C];
  __shared__ int s_flagslot[2][C];
  __shared__ int s_rotslot[C];
  __shared__ T s_hh[3];  // alpha, beta, v0 of the current Householder step (owner)
  __shared__ int s_count;

  // shared::cluster addresses in the owner CTA of global column c
  auto colp = [&](int c) { return dsm_addr(Wl + (size_t)ld * (c / C), c % C); };
  auto nrmp = [&](int c) { return dsm_addr(nrm2 + c / C, c % C); };
  auto refp = [&](int c) { return dsm_addr(ref + c / C, c % C); };
  auto dscp = [&](int c) { return dsm_addr(dsc + c / C, c % C); };
  auto iscp = [&](int c) { return dsm_addr(isc + c / C, c % C); };
  auto permp = [&](int c) { return dsm_addr(perm + c / C, c % C); };
  const T tz = T(0);
  constexpr uint32_t SZ = sizeof(T);

  const T* Ain = reinterpret_cast<const T*>(a.io.A);
  const int ncl = gridDim.x / C;
  const int nvalid = n > rank ? (n - rank + C - 1) / C : 0;  // local columns with c < n

  // phase boundaries (thread 0 of CTA 0 of the cluster, profiling only): slice start,
  // QR start, sweeps start, sweeps end, selection end, coefficients end, rows end
  const bool prof = a.io.phases != nullptr && rank == 0 && threadIdx.x == 0;
  long long tph[7];
  for (int64_t slice = blockIdx.x / C; slice < jp.P; slice += ncl) {
    if (prof) tph[0] = clock64();
    const T* A = Ain + slice * I1 * I2;
    T* D = a.io.D ? reinterpret_cast<T*>(a.io.D) + slice * I1 * I2 : nullptr;
    // ---- load the local columns of B (zero padding), local maximum
    unsigned long long mb = 0ULL;
    for (int idx = threadIdx.x; idx < ld * nl; idx += blockDim.x) {
      const int r = idx % ld, q = idx / ld, c = q * C + rank;
      T v = T(0);
      if (r < m && c < n) v = jp.transposed ? A[c + I1 * r] : A[r + I1 * c];
      Wl[idx] = v;
      const unsigned long long b = abs_bits(v);
      mb = b > mb ? b : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = v > mb ? v : mb;
    }
    __shared__ unsigned long long s_mb[MAXT / 32];
    if (lane == 0) s_mb[warp] = mb;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0ULL;
      for (int w = 0; w < nwarps; ++w) t = s_mb[w] > t ? s_mb[w] : t;
      dsm_st(dsm_addr(&s_maxslot[rank], 0), t);
    }
    cl.sync();
    unsigned long long gmb = 0ULL;
    for (int r = 0; r < C; ++r) {
      const unsigned long long t = dsm_ld(dsm_addr(&s_maxslot[r], 0), 0ULL);
      gmb = t > gmb ? t : gmb;
    }
    const T sc = pow2_scale(from_abs_bits<T>(gmb));
    if (sc != T(1))
      for (int idx = threadIdx.x; idx < ld * nl; idx += blockDim.x) Wl[idx] *= sc;
    const T tau = T(a.io.tau) * sc;
    __syncthreads();

    if (prof) tph[1] = clock64();
    // ---- 1. QR with column pivoting on the distributed columns
    for (int q = warp; q < nl; q += nwarps) {
      const T* col = Wl + (size_t)ld * q;
      T s = T(0);
      for (int r = lane; r < m; r += 32) s = fma(col[r], col[r], s);
      s = warp_allsum(s);
      if (lane == 0) { nrm2[q] = s; ref[q] = s; perm[q] = q * C + rank; }
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      const int oj = j % C;
      if (warp == 0) {  // this CTA's best remaining column
        T best = T(-1);
        int bi = j;
        for (int q = lane; q < nvalid; q += 32) {
          const int c = q * C + rank;
          if (c >= j && nrm2[q] > best) { best = nrm2[q]; bi = c; }
        }
        warp_argmax(best, bi);
        if (lane == 0) {
          dsm_st(dsm_addr(&s_candv[rank], 0), best);
          dsm_st(dsm_addr(&s_candi[rank], 0), bi);
        }
      }
      cl.sync();
      if (rank == oj) {  // uniform over the CTA
        T best = T(-1);
        int p = j;
        for (int r = 0; r < C; ++r) {
          const T v = dsm_ld(dsm_addr(&s_candv[r], 0), tz);
          const int i = dsm_ld(dsm_addr(&s_candi[r], 0), 0);
          if (v > best || (v == best && i < p)) { best = v; p = i; }
        }
        if (p != j) {
          T* cj = Wl + (size_t)ld * (j / C);
          const uint32_t cp = colp(p);
          for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const T t0 = cj[r];
            cj[r] = dsm_ld(cp + SZ * r, tz);
            dsm_st(cp + SZ * r, t0);
          }
          if (threadIdx.x == 0) {
            const int qj = j / C;
            T t1 = nrm2[qj]; nrm2[qj] = dsm_ld(nrmp(p), tz); dsm_st(nrmp(p), t1);
            t1 = ref[qj]; ref[qj] = dsm_ld(refp(p), tz); dsm_st(refp(p), t1);
            const int t2 = perm[qj]; perm[qj] = dsm_ld(permp(p), 0); dsm_st(permp(p), t2);
          }
        }
        __syncthreads();
        if (warp == 0) {  // Householder vector v = x - alpha e_1 of x = B(j:m, j)
          const T* col = Wl + (size_t)ld * (j / C);
          T s = T(0);
          for (int r = j + lane; r < m; r += 32) s = fma(col[r], col[r], s);
          s = warp_allsum(s);
          if (lane == 0) {
            const T x0 = col[j];
            const T nx = sqrt(s);
            const T alpha = (x0 >= T(0)) ? -nx : nx;
            s_hh[0] = alpha;
            s_hh[1] = (s > T(0)) ? T(1) / (nx * (nx + fabs(x0))) : T(0);
            s_hh[2] = x0 - alpha;
          }
        }
      }
      cl.sync();
      {
        const uint32_t cj = colp(j);
        for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) vbuf[r] = dsm_ld(cj + SZ * r, tz);
      }
      const T alpha = dsm_ld(dsm_addr(&s_hh[0], oj), tz);
      const T beta = dsm_ld(dsm_addr(&s_hh[1], oj), tz);
      const T v0 = dsm_ld(dsm_addr(&s_hh[2], oj), tz);
      __syncthreads();
      // local columns c > j: B(j:m, c) -= beta v (v . B(j:m, c)), four per warp pass
      int qs = j + 1 - rank;
      qs = qs <= 0 ? 0 : (qs + C - 1) / C;
      for (int q0 = qs + 4 * warp; q0 < nvalid; q0 += 4 * nwarps) {
        T* col[4];
        T w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u < nvalid ? q0 + u : q0;
          col[u] = Wl + (size_t)ld * q;
          w[u] = (lane == 0) ? v0 * col[u][j] : T(0);
        }
        for (int r = j + 1 + lane; r < m; r += 32) {
          const T vr = vbuf[r];
#pragma unroll
          for (int u = 0; u < 4; ++u) w[u] = fma(vr, col[u][r], w[u]);
        }
        warp_allsum4(w);
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] *= beta;
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (q0 + u >= nvalid) continue;  // uniform over the warp
          T* cu = col[u];
          if (lane == 0) cu[j] = fma(-w[u], v0, cu[j]);
          for (int r = j + 1 + lane; r < m; r += 32) cu[r] = fma(-w[u], vbuf[r], cu[r]);
        }
        __syncwarp();
        bool redo = false;
        if (lane < 4 && q0 + lane < nvalid) {
          const int q = q0 + lane;
          const T rjc = Wl[j + (size_t)ld * q];
          const T nn = nrm2[q] - rjc * rjc;
          redo = nn <= T(0.01) * ref[q];
          if (!redo) nrm2[q] = nn > T(0) ? nn : T(0);
        }
        unsigned mask = __ballot_sync(0xffffffffu, redo);
        while (mask) {  // rare: recompute a norm that cancellation has eaten
          const int u = __ffs(mask) - 1;
          mask &= mask - 1;
          const T* cu = col[u];
          T sq = T(0);
          for (int r = j + 1 + lane; r < m; r += 32) sq = fma(cu[r], cu[r], sq);
          sq = warp_allsum(sq);
          if (lane == 0) {
            ref[q0 + u] = sq;
            nrm2[q0 + u] = sq > T(0) ? sq : T(0);
          }
        }
      }
      if (rank == oj && threadIdx.x == 0) Wl[j + (size_t)ld * (j / C)] = alpha;
      __syncthreads();
    }
    // every CTA must be past its last read of the Householder vectors and of the upper
    // triangle's owners before Z is formed
    cl.sync();
    // ---- Z = R^T: the lower part of local column c takes row c of R (upper parts of
    // the other columns, which nobody writes here); then the upper part is cleared
    for (int idx = threadIdx.x; idx < nvalid * n; idx += blockDim.x) {
      const int q = idx / n, r = idx % n, c = q * C + rank;
      if (r > c) Wl[r + (size_t)ld * q] = dsm_ld(colp(r) + SZ * c, tz);
    }
    cl.sync();
    for (int idx = threadIdx.x; idx < ld * nl; idx += blockDim.x) {
      const int r = idx % ld, q = idx / ld, c = q * C + rank;
      if (c >= n || r >= n || r < c) Wl[idx] = T(0);
    }
    for (int q = threadIdx.x; q < nl; q += blockDim.x) { dsc[q] = T(1); isc[q] = T(1); }
    __syncthreads();

    if (prof) tph[2] = clock64();
    // ---- 2. one-sided Jacobi on Z, pairs spread over the cluster
    auto column_norms = [&]() {
      for (int q0 = 0; q0 < nl; q0 += ngrp) {
        const int q = q0 + grp;
        T* col = Wl + (size_t)ld * (q < nl ? q : 0);
        T s = T(0);
        const T dc = q < nl ? dsc[q] : T(1);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const T v = col[gl + G * e] * dc;
          if (q < nl && kScaled) col[gl + G * e] = v;
          s = fma(v, v, s);
        }
        s = group_sum<G>(s);
        if (gl == 0 && q < nl) {
          nrm2[q] = s;
          dsc[q] = T(1);
          isc[q] = T(1);
        }
      }
    };
    // Parallel block Jacobi: the local columns of a CTA are two half-blocks of h columns
    // (slots 0 and 1).  A sweep is 2C - 1 block rounds of a round-robin tournament on the
    // 2C half-blocks; in block round b, CTA k holds the two half-blocks the tournament
    // pairs at position k and rotates every pair between them (h local rounds of h
    // disjoint pairs), plus, in the first block round, the pairs inside each of them
    // (h - 1 local rounds).  Local rounds touch only the CTA's own shared memory; between
    // block rounds the half-blocks move to their next holders through distributed shared
    // memory.  Every pair of columns meets once per sweep.
    int sweeps = 0, nrot = 0;
    bool rotated = true;
    const int h = nl / 2;
    constexpr int NB = 2 * C;
    auto held = [&](int b, int k, int sl) { return sl == 0 ? rr_i(b, k, NB) : rr_j(b, k, NB); };
    // local columns (i, j) of pair kq in local round lr of block round b
    auto pair_of = [&](int b, int lr, int kq, int& i, int& j) {
      if (b == 0 && lr < h - 1) {  // inside each half-block: h / 2 pairs in each slot
        const int sl = kq < h / 2 ? 0 : 1, kk = kq - sl * (h / 2);
        i = sl * h + rr_i(lr, kk, h);
        j = sl * h + rr_j(lr, kk, h);
      } else {                     // across the two half-blocks
        const int sh = b == 0 ? lr - (h - 1) : lr;
        i = kq;
        j = h + (kq + sh) % h;
      }
    };
    while (rotated && sweeps < a.max_sweeps) {
      column_norms();
      __syncthreads();
      int flag = 0;
      for (int b = 0; b < NB - 1; ++b) {
        const int nlr = (b == 0 ? h - 1 : 0) + h;
        for (int lr = 0; lr < nlr; ++lr) {
          for (int k0 = 0; k0 < h; k0 += ngrp) {
            const int kq = k0 + grp;
            const bool active = kq < h;
            int i = 0, j = 0;
            if (active) pair_of(b, lr, kq, i, j);
            T* ci = Wl + (size_t)ld * i;
            T* cj = Wl + (size_t)ld * j;
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
              // scaled rotations in three phases, as in jacobi_svt_kernel
              if (gl == 0) s_pg[grp] = g;
              __syncthreads();
              const int batch = min(ngrp, h - k0);
              for (int q = threadIdx.x; q < batch; q += blockDim.x) {
                int pi, pj;
                pair_of(b, lr, k0 + q, pi, pj);
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
              if (active && s_pr[grp]) {
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
            } else {
              const T al = active ? nrm2[i] : T(0), be = active ? nrm2[j] : T(0);
              if (al > T(0) && be > T(0) && g * g > tol2 * al * be) {
                T cs, sn, t;
                rotation_fast(al, be, g, cs, sn, t);
                const T hh = sn / (T(1) + cs);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                  ci[gl + G * e] = fma(-sn, fma(hh, x[e], y[e]), x[e]);
                  cj[gl + G * e] = fma(sn, fma(-hh, y[e], x[e]), y[e]);
                }
                if (gl == 0) {
                  nrm2[i] = al - t * g;
                  nrm2[j] = be + t * g;
                  ++nrot;
                }
                flag = 1;
              }
            }
          }
          __syncthreads();
        }
        // move the half-blocks to their holders in the next block round (cyclic, so the
        // layout at every sweep start is that of block round 0): read the two new
        // half-blocks (and their scalars) from the current holders in chunks, a cluster
        // barrier between the reads and the overwrites of each chunk
        const int nb = (b + 1) % (NB - 1);
        int srcK[2], srcS[2];
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          const int x = held(nb, rank, sl);
          srcK[sl] = 0;
          srcS[sl] = 0;
          for (int k = 0; k < C; ++k)
            for (int s2 = 0; s2 < 2; ++s2)
              if (held(b, k, s2) == x) { srcK[sl] = k; srcS[sl] = s2; }
        }
        const bool keep0 = srcK[0] == rank && srcS[0] == 0;
        const bool keep1 = srcK[1] == rank && srcS[1] == 1;
        cl.sync();  // every CTA has finished block round b
        T s0 = T(0), s1 = T(0), s2v = T(0);
        const int sq = threadIdx.x;  // scalars: thread sq < 2h moves column sq's three
        const int ssl = sq / (h > 0 ? h : 1);
        const bool smove = sq < 2 * h && !(ssl == 0 ? keep0 : keep1);
        if (smove) {
          const int src = srcS[ssl] * h + sq % h;
          s0 = dsm_ld(dsm_addr(nrm2 + src, srcK[ssl]), tz);
          s1 = dsm_ld(dsm_addr(dsc + src, srcK[ssl]), tz);
          s2v = dsm_ld(dsm_addr(isc + src, srcK[ssl]), tz);
        }
        // chunks are ranges of the offset w inside a half-block, the same for every CTA
        // and both slots, so that an offset is read (by its next holder) and overwritten
        // (by its current holder) on opposite sides of the same barrier
        constexpr int CH = 8;
        const int per = h * ld, wch = CH * (int)blockDim.x / 2;
        for (int wb = 0; wb < per; wb += wch) {
          T buf[CH];
#pragma unroll
          for (int u = 0; u < CH; ++u) {
            const int idx = u * (int)blockDim.x + (int)threadIdx.x;
            const int sl = idx & 1, w = wb + (idx >> 1);
            buf[u] = T(0);
            if (w < per && !(sl == 0 ? keep0 : keep1))
              buf[u] = dsm_ld(dsm_addr(Wl + (size_t)srcS[sl] * per + w, srcK[sl]), tz);
          }
          cl.sync();
#pragma unroll
          for (int u = 0; u < CH; ++u) {
            const int idx = u * (int)blockDim.x + (int)threadIdx.x;
            const int sl = idx & 1, w = wb + (idx >> 1);
            if (w < per && !(sl == 0 ? keep0 : keep1)) Wl[(size_t)sl * per + w] = buf[u];
          }
          if (wb == 0 && smove) {
            nrm2[sq] = s0;
            dsc[sq] = s1;
            isc[sq] = s2v;
          }
        }
        __syncthreads();
      }
      flag = __syncthreads_or(flag);
      if (threadIdx.x == 0) dsm_st(dsm_addr(&s_flagslot[sweeps & 1][rank], 0), flag);
      cl.sync();
      rotated = false;
      for (int r = 0; r < C; ++r)
        rotated |= dsm_ld(dsm_addr(&s_flagslot[sweeps & 1][r], 0), 0) != 0;
      ++sweeps;
    }
    column_norms();
    {
      __shared__ int s_nrot;
      if (threadIdx.x == 0) s_nrot = 0;
      __syncthreads();
      if (nrot) atomicAdd(&s_nrot, nrot);
      __syncthreads();
      if (threadIdx.x == 0) dsm_st(dsm_addr(&s_rotslot[rank], 0), s_nrot);
    }
    cl.sync();

    if (prof) tph[3] = clock64();
    // ---- 3. shrink and reconstruct: every CTA copies the norms and the permutation of
    // all columns, builds the same list of kept columns, then computes its rows
    // columns moved between CTAs in the sweeps: scan every padded position (a zero
    // padding column is never kept); permall indexes the rows of Z (QR order)
    for (int c = threadIdx.x; c < np; c += blockDim.x) {
      gval[c] = dsm_ld(nrmp(c), tz);
      if (c < n) permall[c] = dsm_ld(permp(c), 0);
    }
    __syncthreads();
    if (a.io.W != nullptr) {
      // warm-start basis (see write_basis): the n columns of nonzero norm in position
      // order (columns moved during the sweeps; padding columns are exactly zero), each
      // written by the CTA holding it; the identity when a column is (near) zero, not
      // finite, or the sweeps did not converge
      __shared__ int s_wok;
      if (threadIdx.x == 0) {
        int cnt = 0, ok = !rotated;
        for (int c = 0; c < np; ++c) {
          const T v = gval[c];
          if (isfinite(v) && v > basis_min_norm2<T>()) {
            if (cnt < n) list[cnt] = c;
            ++cnt;
          } else if (v != T(0)) {
            ok = 0;
          }
        }
        s_wok = ok && cnt == n;
      }
      __syncthreads();
      const bool wok = s_wok != 0;
      T* Wo = reinterpret_cast<T*>(a.io.W) + (size_t)slice * n * n;
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int r = idx % n, oc = idx / n;
        if (wok) {
          const int pos = list[oc];
          if (pos % C == rank) Wo[idx] = Wl[r + (size_t)ld * (pos / C)] / sqrt(gval[pos]);
        } else if (rank == 0) {
          Wo[idx] = r == oc ? T(1) : T(0);
        }
      }
      if (rank == 0)
        for (int r = threadIdx.x; r < n; r += blockDim.x)
          a.io.Wperm[(size_t)slice * n + r] = wok ? permall[r] : r;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      int st = 0, k = 0;
      T nuc = T(0);
      if (rotated) st |= LT_DEV_NOCONV;
      for (int c = 0; c < np; ++c) {
        const T s2 = gval[c];
        if (!isfinite(s2)) st |= LT_DEV_NONFINITE;
        const T sg = sqrt(s2);
        if (sg > tau) {
          list[k++] = c;
          nuc += sg - tau;
        }
      }
      s_count = k;
      if (prof) tph[4] = clock64();
      if (rank == 0) {
        if (st) atomicOr(a.status, st);
        if (a.io.info) {
          a.io.info[slice].sweeps = sweeps;
          a.io.info[slice].rank = k;
          a.io.info[slice].nuclear = double(nuc) / double(sc);
        }
        if (a.io.flops) {
          int rots = 0;
          for (int r = 0; r < C; ++r) rots += s_rotslot[r];
          const double md = m, nd = n;
          const double f = 2.0 * md * nd * nd - 2.0 * nd * nd * nd / 3.0 +
                           sweeps * (nd * (nd - 1) * nd + 2 * nd * nd) +
                           (kScaled ? 4.0 : 6.0) * nd * rots + 2 * nd * nd +
                           4.0 * k * md * nd;
          atomicAdd(a.io.flops, f);
        }
      }
    }
    __syncthreads();
    const int k = s_count;
    if (prof) tph[5] = clock64();
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
      const int c = list[q];
      const T sg = sqrt(gval[c]);
      gval[c] = ((sg - tau) / sg) / sg / sg;
    }
    __syncthreads();
    constexpr int ER = (G * E + 31) / 32;
    const int rows_mine = m > rank ? (m - rank + C - 1) / C : 0;
    const int rows_iter = D != nullptr ? (rows_mine + nwarps - 1) / nwarps : 0;
    for (int it = 0; it < rows_iter; ++it) {
      const int rl = it * nwarps + warp;
      const int r = rl * C + rank;
      const bool active = rl < rows_mine;
      T b[ER];
#pragma unroll
      for (int e = 0; e < ER; ++e) {
        const int c = lane + 32 * e;
        b[e] = T(0);
        if (active && c < n) {
          const int pc = permall[c];
          b[e] = jp.transposed ? A[pc + I1 * r] : A[r + I1 * pc];
        }
      }
      T yreg[ER];
#pragma unroll
      for (int s2 = 0; s2 < ER; ++s2) {
        yreg[s2] = T(0);
        const int qn = min(32, k - s2 * 32);
        for (int gq = 0; gq < qn; ++gq) {
          const uint32_t z = colp(list[s2 * 32 + gq]) + SZ * lane;
          T d = T(0);
#pragma unroll
          for (int e = 0; e < ER; ++e) d = fma(dsm_ld(z + SZ * 32 * e, tz), b[e], d);
          d = warp_allsum(d);
          if (lane == gq) yreg[s2] = d * gval[list[s2 * 32 + gq]];
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
          const uint32_t z = colp(list[s2 * 32 + gq]) + SZ * lane;
#pragma unroll
          for (int e = 0; e < ER; ++e) out[e] = fma(yq, dsm_ld(z + SZ * 32 * e, tz), out[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < ER; ++e) {
        const int c = lane + 32 * e;
        if (active && c < n) {
          const int pc = permall[c];
          if (jp.transposed) D[pc + I1 * r] = out[e];
          else D[r + I1 * pc] = out[e];
        }
      }
    }
    if (prof) {
      tph[6] = clock64();
      for (int q = 0; q < 6; ++q) atomicAdd(a.io.phases + q, double(tph[q + 1] - tph[q]));
    }
    // no CTA may reload or leave while another still reads its columns
    cl.sync();
  }
}

}  // namespace jac
}  // namespace lt
