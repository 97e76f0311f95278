// Kernel J, SVD form (Algorithm 3: svd of every slice A_hat^p, full U, S, V), plus the
// planning and dispatch of both Jacobi kernels.  The SVT form used by lt_svt and PGA
// (Algorithm 4) is in lt_jacobi_svt.cuh.
//
// Method: one-sided (Hestenes) Jacobi on the working matrix B (m x n, m >= n): B = A^p
// when I1 >= I2, B = (A^p)^T otherwise.  Plane rotations are applied from the right,
// B <- B J, until every pair of columns is orthogonal to the tolerance
// |b_i . b_j| <= tol ||b_i|| ||b_j||.  At convergence B = W = U Sigma and the accumulated
// rotations (kept in global scratch) are V.  Round-robin ordering, a warp per pair with
// both columns in registers; squared norms updated as alpha - t gamma, beta + t gamma and
// recomputed exactly at the start of each sweep.  The outputs are sorted by descending
// sigma and the W side is completed to a square orthogonal basis.
#include <algorithm>
#include <cfloat>

#include "lt_jacobi_common.cuh"

namespace lt {
namespace {

using jac::JArgs;
using jac::kJThreads;
using jac::kWarps;
using jac::rotation;
using jac::unit_roundoff;
using jac::warp_allsum;

// Round-robin pairing: column n-1 is fixed, the others rotate on a circle.
__device__ __forceinline__ void rr_pair(int r, int k, int n, int& i, int& j) {
  const int c = n - 1;
  if (k == 0) {
    i = c;
    j = r;
  } else {
    i = (r + k) % c;
    j = (r - k + c) % c;
  }
}

template <typename T, int E>
__global__ void __launch_bounds__(kJThreads)
jacobi_kernel(const JArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const JacobiPlan& jp = a.jp;
  if (a.io.scal != nullptr && a.io.scal->done) return;  // PGA converged earlier

  const int m = jp.m, n = jp.n, np = jp.npad, ld = jp.ld;
  const int64_t I1 = jp.I1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T tol2 = T(a.tol) * T(a.tol);

  // shared memory carve-up
  unsigned char* sp = smem_raw;
  T* Ws = nullptr;
  if (jp.w_in_smem) { Ws = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)ld * np; }
  T* nrm = reinterpret_cast<T*>(sp); sp += sizeof(T) * np;
  int* list = reinterpret_cast<int*>(sp); sp += sizeof(int) * np;        // SVT: kept columns / SVD: rank
  T* coef = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)kWarps * np;  // per-warp coefficients
  T* vtmp = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)(jp.mode == JAC_SVD ? 2 * m : 0);
  __shared__ int s_count, s_cand, s_rot;
  __shared__ T s_red[kWarps];

  const T* Ain = reinterpret_cast<const T*>(a.io.A);
  unsigned char* scratch = reinterpret_cast<unsigned char*>(a.io.scratch);
  T* Wg = jp.w_in_smem ? nullptr
                       : reinterpret_cast<T*>(scratch) + (size_t)blockIdx.x * ld * np;
  // Jacobi V (SVD mode only): np x np per CTA, after the global W regions
  T* Vj = nullptr;
  if (jp.mode == JAC_SVD) {
    size_t off = jp.w_in_smem ? 0 : (size_t)gridDim.x * ld * np;
    Vj = reinterpret_cast<T*>(scratch) + off + (size_t)blockIdx.x * np * np;
  }
  T* W = jp.w_in_smem ? Ws : Wg;

  for (int64_t slice = blockIdx.x; slice < jp.P; slice += gridDim.x) {
    const T* A = Ain + slice * jp.I1 * jp.I2;
    // ---- load B (transposed when I1 < I2); zero padding column(s)
    if (!jp.transposed) {
      for (int idx = threadIdx.x; idx < m * np; idx += blockDim.x) {
        const int r = idx % m, c = idx / m;
        W[r + (size_t)ld * c] = (c < n) ? A[r + I1 * c] : T(0);
      }
    } else {
      for (int idx = threadIdx.x; idx < n * m; idx += blockDim.x) {
        const int c = idx % n, r = idx / n;
        W[r + (size_t)ld * c] = A[c + I1 * r];
      }
      for (int idx = threadIdx.x; idx < m * (np - n); idx += blockDim.x)
        W[idx % m + (size_t)ld * (n + idx / m)] = T(0);
    }
    if (jp.mode == JAC_SVD) {
      for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x)
        Vj[idx] = (idx % np == idx / np) ? T(1) : T(0);
    }
    __syncthreads();

    // ---- sweeps
    int sweeps = 0;
    int nrot = 0;  // rotations applied by this warp (flop accounting)
    if (threadIdx.x == 0) s_rot = 0;
    bool rotated = true;
    while (rotated && sweeps < a.max_sweeps) {
      for (int c = warp; c < np; c += kWarps) {
        const T* col = W + (size_t)ld * c;
        T acc = T(0);
        for (int r = lane; r < m; r += 32) acc = fma(col[r], col[r], acc);
        acc = warp_allsum(acc);
        if (lane == 0) nrm[c] = acc;
      }
      __syncthreads();
      int flag = 0;
      for (int rnd = 0; rnd < np - 1; ++rnd) {
        for (int k = warp; k < np / 2; k += kWarps) {
          int i, j;
          rr_pair(rnd, k, np, i, j);
          T* ci = W + (size_t)ld * i;
          T* cj = W + (size_t)ld * j;
          T x[E], y[E];
          T g = T(0);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int r = lane + 32 * e;
            x[e] = (r < m) ? ci[r] : T(0);
            y[e] = (r < m) ? cj[r] : T(0);
            g = fma(x[e], y[e], g);
          }
          g = warp_allsum(g);
          const T al = nrm[i], be = nrm[j];
          if (al > T(0) && be > T(0) && g * g > tol2 * al * be) {
            T cs, sn, t;
            rotation(al, be, g, cs, sn, t);
            // x' = c x - s y = x - s (y + h x),  y' = s x + c y = y + s (x - h y) with
            // h = s / (1 + c) = tan(theta/2): the update is formed as a small increment,
            // so a small rotation adds rounding error of the order of the increment.
            const T h = sn / (T(1) + cs);
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int r = lane + 32 * e;
              const T xi = x[e], yi = y[e];
              if (r < m) {
                ci[r] = fma(-sn, fma(h, xi, yi), xi);
                cj[r] = fma(sn, fma(-h, yi, xi), yi);
              }
            }
            if (jp.mode == JAC_SVD) {
              T* vi = Vj + (size_t)np * i;
              T* vj = Vj + (size_t)np * j;
              for (int r = lane; r < np; r += 32) {
                const T xi = vi[r], yi = vj[r];
                vi[r] = fma(-sn, fma(h, xi, yi), xi);
                vj[r] = fma(sn, fma(-h, yi, xi), yi);
              }
            }
            if (lane == 0) {
              nrm[i] = al - t * g;
              nrm[j] = be + t * g;
            }
            flag = 1;
            ++nrot;
          }
        }
        __syncthreads();
      }
      rotated = __syncthreads_or(flag) != 0;
      ++sweeps;
    }
    // exact final norms
    for (int c = warp; c < np; c += kWarps) {
      const T* col = W + (size_t)ld * c;
      T acc = T(0);
      for (int r = lane; r < m; r += 32) acc = fma(col[r], col[r], acc);
      acc = warp_allsum(acc);
      if (lane == 0) nrm[c] = acc;
    }
    __syncthreads();
    if (lane == 0 && nrot) atomicAdd(&s_rot, nrot);
    __syncthreads();
    if (threadIdx.x == 0) {
      int st = 0;
      if (rotated) st |= LT_DEV_NOCONV;
      for (int c = 0; c < n; ++c)
        if (!isfinite(nrm[c])) { st |= LT_DEV_NONFINITE; break; }
      if (st) atomicOr(a.status, st);
      if (a.io.info) a.io.info[slice].sweeps = sweeps;
    }

    if (jp.mode == JAC_SVT) {
      // ---- shrink: keep columns with sigma > tau, g_i = (sigma_i - tau)/sigma_i^3
      const T tau = T(a.io.tau);
      if (threadIdx.x == 0) {
        int k = 0;
        T nuc = T(0);
        for (int c = 0; c < n; ++c) {
          const T sg = sqrt(nrm[c]);
          if (sg > tau) {
            list[k++] = c;
            nuc += sg - tau;
          }
        }
        s_count = k;
        if (a.io.flops) {
          // pairs visited (dot) + rotations + norm passes + reconstruction 4kmn
          const double md = m, nd = n;
          const double f = sweeps * (nd * (nd - 1) * md + 2 * md * nd) + 6.0 * md * s_rot +
                           2 * md * nd + 4.0 * k * md * nd;
          atomicAdd(a.io.flops, f);
        }
        if (a.io.info) {
          a.io.info[slice].rank = k;
          a.io.info[slice].nuclear = double(nuc);
        }
      }
      __syncthreads();
      const int k = s_count;
      T* gcoef = nrm;  // reuse: nrm[c] -> g_c for kept columns
      for (int q = threadIdx.x; q < k; q += blockDim.x) {
        const int c = list[q];
        const T sg = sqrt(nrm[c]);
        gcoef[c] = ((sg - tau) / sg) / sg / sg;
      }
      __syncthreads();
      // ---- reconstruct D_B = sum_i g_i w_i (w_i^T b_j), column by column
      T* D = reinterpret_cast<T*>(a.io.D) + slice * jp.I1 * jp.I2;
      T* cw = coef + (size_t)warp * np;
      for (int j = warp; j < n; j += kWarps) {
        T b[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int r = lane + 32 * e;
          b[e] = (r < m) ? (jp.transposed ? A[j + I1 * r] : A[r + I1 * j]) : T(0);
        }
        for (int q = 0; q < k; ++q) {
          const T* w = W + (size_t)ld * list[q];
          T d = T(0);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int r = lane + 32 * e;
            if (r < m) d = fma(w[r], b[e], d);
          }
          d = warp_allsum(d);
          if (lane == 0) cw[q] = d * gcoef[list[q]];
        }
        __syncwarp();
        T out[E];
#pragma unroll
        for (int e = 0; e < E; ++e) out[e] = T(0);
        for (int q = 0; q < k; ++q) {
          const T cq = cw[q];
          const T* w = W + (size_t)ld * list[q];
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int r = lane + 32 * e;
            if (r < m) out[e] = fma(cq, w[r], out[e]);
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int r = lane + 32 * e;
          if (r < m) {
            if (jp.transposed) D[j + I1 * r] = out[e];
            else D[r + I1 * j] = out[e];
          }
        }
        __syncwarp();
      }
    } else {
      // ---- SVD: sort descending, write Sigma, the Jacobi V side and the W side
      const int64_t I2 = jp.I2;
      if (threadIdx.x == 0 && a.io.flops) {
        const double md = m, nd = n;
        atomicAdd(a.io.flops, sweeps * (nd * (nd - 1) * md + 2 * md * nd) +
                                  (6.0 * md + 6.0 * np) * s_rot + 2 * md * nd);
      }
      T sig_max = T(0);
      for (int c = 0; c < n; ++c) sig_max = fmax(sig_max, sqrt(nrm[c]));
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const T sc = nrm[c];
        int rk = 0;
        for (int c2 = 0; c2 < n; ++c2) {
          const T s2 = nrm[c2];
          rk += (s2 > sc) || (s2 == sc && c2 < c);
        }
        list[c] = rk;
      }
      __syncthreads();
      T* S = reinterpret_cast<T*>(a.io.S) + slice * I1 * I2;
      for (int64_t idx = threadIdx.x; idx < I1 * I2; idx += blockDim.x) S[idx] = T(0);
      __syncthreads();
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const T sg = sqrt(nrm[c]);
        S[list[c] + I1 * list[c]] = sg;
        if (a.io.sigma) reinterpret_cast<T*>(a.io.sigma)[slice * n + list[c]] = sg;
      }
      // Jacobi V -> V (I1 >= I2) or U (I1 < I2); n x n
      T* Vout = jp.transposed ? reinterpret_cast<T*>(a.io.U) + slice * I1 * I1
                              : reinterpret_cast<T*>(a.io.V) + slice * I2 * I2;
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int r = idx % n, c = idx / n;
        Vout[r + (size_t)n * list[c]] = Vj[r + (size_t)np * c];
      }
      // W side: m x m, Q[:, rank] = w / sigma for sigma above the rank threshold
      T* Q = jp.transposed ? reinterpret_cast<T*>(a.io.V) + slice * I2 * I2
                           : reinterpret_cast<T*>(a.io.U) + slice * I1 * I1;
      const T thr = T(m) * unit_roundoff<T>() * sig_max;
      if (threadIdx.x == 0) {
        int nv = 0;
        for (int c = 0; c < n; ++c) nv += sqrt(nrm[c]) > thr;
        s_count = nv;
      }
      __syncthreads();
      const int nv = s_count;
      for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
        const int r = idx % m, c = idx / m;
        if (list[c] < nv) Q[r + (size_t)m * list[c]] = W[r + (size_t)ld * c] / sqrt(nrm[c]);
      }
      __syncthreads();
      // complete Q to an orthogonal m x m basis: for each missing column take the
      // canonical vector e_c farthest from span(Q) (its squared distance is
      // 1 - ||Q(c, :)||^2, at least (m - q)/m for the best c) and orthogonalise it
      // against Q twice (classical Gram-Schmidt, two passes).
      T* v = vtmp;
      T* cf = vtmp + m;
      __shared__ int s_arg[kWarps];
      __shared__ T s_val[kWarps];
      for (int q = nv; q < m; ++q) {
        // pick the candidate
        T best = T(-1);
        int bi = 0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
          T acc = T(1);
          for (int j = 0; j < q; ++j) acc -= Q[r + (size_t)m * j] * Q[r + (size_t)m * j];
          if (acc > best) { best = acc; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_val[warp] = best; s_arg[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
          T b = s_val[0];
          int ix = s_arg[0];
          for (int w = 1; w < kWarps; ++w)
            if (s_val[w] > b || (s_val[w] == b && s_arg[w] < ix)) { b = s_val[w]; ix = s_arg[w]; }
          s_cand = ix;
        }
        __syncthreads();
        const int cand = s_cand;
        // pass 1: v = e_cand - Q(:, :q) Q(cand, :q)^T
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
          T acc = (r == cand) ? T(1) : T(0);
          for (int j = 0; j < q; ++j) acc -= Q[r + (size_t)m * j] * Q[cand + (size_t)m * j];
          v[r] = acc;
        }
        __syncthreads();
        // pass 2: v -= Q (Q^T v)
        for (int j = warp; j < q; j += kWarps) {
          T acc = T(0);
          for (int r = lane; r < m; r += 32) acc = fma(Q[r + (size_t)m * j], v[r], acc);
          acc = warp_allsum(acc);
          if (lane == 0) cf[j] = acc;
        }
        __syncthreads();
        T part = T(0);
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
          T acc = v[r];
          for (int j = 0; j < q; ++j) acc -= Q[r + (size_t)m * j] * cf[j];
          v[r] = acc;
          part = fma(acc, acc, part);
        }
        part = warp_allsum(part);
        if (lane == 0) s_red[warp] = part;
        __syncthreads();
        T nv2 = T(0);
        for (int w = 0; w < kWarps; ++w) nv2 += s_red[w];
        const T inv = T(1) / sqrt(nv2);
        for (int r = threadIdx.x; r < m; r += blockDim.x) Q[r + (size_t)m * q] = v[r] * inv;
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

template <typename T>
size_t smem_need(const JacobiPlan& jp) {
  size_t b = 0;
  if (jp.w_in_smem) b += sizeof(T) * (size_t)jp.ld * jp.npad;
  b += sizeof(T) * jp.npad + sizeof(int) * jp.npad + sizeof(T) * (size_t)kWarps * jp.npad;
  if (jp.mode == JAC_SVD) b += sizeof(T) * 2 * (size_t)jp.m;
  return (b + 15) & ~size_t(15);
}

template <typename T, int E>
cudaError_t launch_e(const JArgs& a, int grid, cudaStream_t st) {
  auto k = jacobi_kernel<T, E>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.jp.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kJThreads, a.jp.smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(const JArgs& a, int grid, cudaStream_t st) {
  switch (a.jp.E) {
    case 1: return launch_e<T, 1>(a, grid, st);
    case 2: return launch_e<T, 2>(a, grid, st);
    case 4: return launch_e<T, 4>(a, grid, st);
    case 8: return launch_e<T, 8>(a, grid, st);
    case 16: return launch_e<T, 16>(a, grid, st);
    case 32: return launch_e<T, 32>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

int jacobi_grid(const Ctx& c, const JacobiPlan& jp) {
  if (jp.cluster > 1) return jp.cluster * (int)std::min<int64_t>(jp.P, 1 << 18);
  if (jp.w_in_smem && jp.mode != JAC_SVD) return (int)std::min<int64_t>(jp.P, 1 << 20);
  // global regions are per CTA: bound the grid by what can be resident (capping it
  // further so that the regions fit L2 was measured slower on 540 x 960 slices: 120
  // CTAs 279 ms, 96 CTAs 446 ms, 64 CTAs 412 ms)
  return (int)std::max<int64_t>(1, std::min<int64_t>(jp.P, (int64_t)c.sms * 2));
}

// Group width G (lanes per column pair) and rows per lane E of the SVT kernel, from the
// instantiated set (rows padded to G E >= n).  Returns false when n is too large.
// Instantiated SVT kernel shapes: (G lanes per pair, B columns per register block,
// E rows per lane), rows padded to G E >= n.  Must match the lt_jacobi_f*.cu files.
struct SvtShape { int G, B; const int* E; int nE; };
const int kBlk16x4[] = {1, 2, 3, 4, 5, 6, 7, 8, 9};
const int kBlk16x2[] = {12, 18};
const int kBlk16x2w[] = {7, 9};  // wide form (lt_jacobi_f32_blk_e.cu), n <= 144
const int kBlk32x2[] = {12, 18};
const int kBlk8x2[] = {6, 12, 18};
const int kF8[] = {2, 4, 6, 8, 12, 18, 24};
const int kF16[] = {16, 24};
const int kF32[] = {20, 24, 28, 32};
const int kD8[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 14, 16, 18};
const int kD16[] = {8, 10, 12, 14};
const int kD32[] = {8, 12, 16, 18};

int pick_E(const int* set, int cnt, int need) {
  for (int i = 0; i < cnt; ++i)
    if (set[i] >= need) return set[i];
  return -1;
}

// Choose (G, B, E) for n columns.  force_g != 0 fixes G (pairwise); pairwise != 0
// disables register blocking.  Returns false when no instantiation holds n.
bool svt_shape(int n, int elem, int force_g, int pairwise, int* G, int* B, int* E) {
  if (elem == 4 && pairwise == 3) {  // wide form: blocks of 2, a group per block pair
    if (n > 144 || (force_g && force_g != 16)) return false;
    *G = 16; *B = 2; *E = pick_E(kBlk16x2w, 2, (n + 15) / 16);
    return *E > 0;
  }
  if (elem == 4 && pairwise == 2) {  // register blocks with the forced group width
    if (force_g == 8) { *G = 8; *B = 2; *E = pick_E(kBlk8x2, 3, (n + 7) / 8); return *E > 0; }
    if (force_g == 16 && n <= 144) { *G = 16; *B = 4; *E = pick_E(kBlk16x4, 9, (n + 15) / 16); return *E > 0; }
    if (force_g == 16) { *G = 16; *B = 2; *E = pick_E(kBlk16x2, 2, (n + 15) / 16); return *E > 0; }
    if (force_g == 32) { *G = 32; *B = 2; *E = pick_E(kBlk32x2, 2, (n + 31) / 32); return *E > 0; }
    return false;
  }
  if (elem == 4 && !force_g && !pairwise && n <= 576) {
    // n <= 144: the wide form (measured on 96 slices of 144 x 176: 3.06 ms against 3.38 ms
    // for 16-lane groups with blocks of 4 columns, which keep only 18 of 32 groups busy)
    if (n <= 144) { *G = 16; *B = 2; *E = pick_E(kBlk16x2w, 2, (n + 15) / 16); }
    else if (n <= 288) { *G = 16; *B = 2; *E = pick_E(kBlk16x2, 2, (n + 15) / 16); }
    else { *G = 32; *B = 2; *E = pick_E(kBlk32x2, 2, (n + 31) / 32); }
    return *E > 0;
  }
  *B = 1;
  auto try_g = [&](int g) {
    const int need = (n + g - 1) / g;
    if (elem == 4) {
      if (g == 8) return pick_E(kF8, 7, need);
      if (g == 16) return pick_E(kF16, 2, need);
      return pick_E(kF32, 4, need);
    }
    if (g == 8) return pick_E(kD8, 12, need);
    if (g == 16) return pick_E(kD16, 4, need);
    return pick_E(kD32, 4, need);
  };
  int g = force_g ? force_g : (elem == 4 ? (n <= 192 ? 8 : (n <= 384 ? 16 : 32))
                                         : (n <= 144 ? 8 : (n <= 224 ? 16 : 32)));
  int e = try_g(g);
  if (e < 0 && force_g) return false;
  while (e < 0 && g < 32) { g *= 2; e = try_g(g); }
  if (e < 0) return false;
  *G = g;
  *E = e;
  return true;
}

template <typename T>
size_t svt_smem(const JacobiPlan& jp) {
  size_t b = 0;
  if (jp.w_in_smem) b += sizeof(T) * (size_t)jp.ld * jp.npad;
  b += sizeof(T) * 2 * (size_t)jp.npad + sizeof(int) * 2 * (size_t)jp.npad;
  if (sizeof(T) == 8) b += sizeof(T) * 2 * (size_t)jp.npad;  // column scales (FP64 sweeps)
  return (b + 15) & ~size_t(15);
}

}  // namespace

// The cluster form of the SVT kernel (lt_jacobi_cluster.cuh) with C CTAs per slice:
// columns padded to a multiple of 4C (2C half-blocks of an even number of columns), a
// C-th of them per CTA, all in shared memory.
bool cluster_plan(const Ctx& c, JacobiPlan* jp, int C) {
  // 2C half-blocks of an even number of columns
  const int np = (jp->n + 4 * C - 1) / (4 * C) * (4 * C);
  const int G = 16;
  int E;
  if (np <= 96) E = 6;
  else if (np <= 144) E = 9;
  else if (np <= 192) E = 12;
  else if (np <= 288) E = 18;
  else return false;
  JacobiPlan q = *jp;
  q.cluster = C;
  q.G = G;
  q.E = E;
  q.B = 1;
  q.npad = np;
  q.w_in_smem = true;
  const int base = std::max(q.m, 32 * ((G * E + 31) / 32));
  q.ld = base | 1;
  const int nl = np / C, ppw = 32 / G, mine = nl / 2;  // pairs per local round
  const int maxw = jac::cluster_max_threads(c.elem, E) / 32;
  q.threads = 32 * std::max(4, std::min(maxw, (mine + ppw - 1) / ppw));
  const size_t need = (size_t)c.elem * ((size_t)q.ld * nl + 4 * (size_t)nl + q.ld + np) +
                      sizeof(int) * ((size_t)nl + 2 * (size_t)np);
  // the kernel's static shared memory (per-pair scalars, slots) takes up to ~4 KB
  if (need > (size_t)kSmemOptin - 6144) return false;
  q.smem = (int)((need + 15) & ~size_t(15));
  q.ws_bytes = 0;
  jac::JArgs a;
  a.jp = q;
  if (!jac::svt_cluster_resident(a)) return false;
  *jp = q;
  return true;
}

// Relative time of the SVT launch, counted in slice-times of one CTA on an SM of its
// own: the one-CTA form runs ceil(P / SMs) rounds of slices (4x slower per slice when
// its working matrix is in global memory); the cluster form gives each SM
// ceil(P C / SMs) CTAs of 1/C of a slice each, at 1.25x the one-CTA time per column pair
// (the half-block moves, barriers and two CTAs sharing an SM; measured on 96 FP64 slices
// of 144 x 176: 16.3 ms on clusters of 3, 19.9 ms on clusters of 4, 19.8 ms on single
// CTAs).
double svt_cost(const Ctx& c, const JacobiPlan& jp) {
  const double sms = c.sms;
  if (jp.cluster > 1)
    return std::ceil((double)jp.P * jp.cluster / sms) / jp.cluster * 1.25;
  return std::ceil((double)jp.P / sms) * (jp.w_in_smem ? 1.0 : 4.0);
}

lt_status plan_jacobi(const Ctx& c, int mode, int64_t I1, int64_t I2, JacobiPlan* out,
                      int64_t count) {
  JacobiPlan jp;
  jp.mode = mode;
  jp.I1 = I1;
  jp.I2 = I2;
  jp.P = count >= 0 ? count : c.P;
  jp.transposed = I1 < I2;
  jp.m = (int)std::max(I1, I2);
  jp.n = (int)std::min(I1, I2);
  jp.npad = jp.n + (jp.n & 1);
  jp.threads = kJThreads;
  jp.w_in_smem = true;
  jp.elem = c.elem;
  if (mode == JAC_SVT && (c.jacobi_cluster == 3 || c.jacobi_cluster == 4)) {
    // forced cluster form
    if (!cluster_plan(c, &jp, c.jacobi_cluster)) return LT_ERR_SHAPE;
    *out = jp;
    return LT_OK;
  }
  size_t need;
  if (mode != JAC_SVD) {
    // QR-preconditioned kernel: Jacobi on the n x n factor R^T, G lanes per column
    // pair holding E rows each, leading dimension >= max(m, G E) and odd (conflict-free
    // transposed stores); as many warps as the pairs of a round need, within the cap.
    int G = 0, E = 0, B = 1;
    if (!svt_shape(jp.n, c.elem, c.jacobi_group, c.jacobi_pairwise, &G, &B, &E))
      return LT_ERR_SHAPE;
    jp.G = G;
    jp.B = B;
    jp.E = E;
    if (B > 1) jp.npad = (jp.n + 2 * B - 1) / (2 * B) * (2 * B);
    jp.ld = std::max(jp.m, 32 * ((G * E + 31) / 32)) | 1;
    if (c.elem == 4 && B > 1) {
      // FP32 block forms: a lane loads pairs of adjacent rows with 8-byte accesses, so
      // ld must be even; ld = 8 (mod 16) floats also puts columns two apart (the two
      // groups of a warp in the wide form) on opposite halves of the 32 banks (with an
      // odd ld and one row per access a third of the shared wavefronts were conflicts)
      const int base = std::max(jp.m, 32 * ((G * E + 31) / 32));
      jp.ld = base + ((8 - base % 16) + 16) % 16;
    }
    if (c.elem == 8 && G == 8 && B == 1) {
      // the four 8-lane groups of a warp hold consecutive columns: with ld = 8 (mod 16)
      // doubles consecutive columns start in opposite halves of the 32 banks, so a
      // warp-wide column access needs the minimum two wavefronts
      const int base = std::max(jp.m, 32 * ((G * E + 31) / 32));
      jp.ld = base + ((8 - base % 16) + 16) % 16;
    }
    if (B == 2 && G == 16 && E <= 9) {  // wide form: a group per block pair of a round
      jp.threads = 32 * std::max(1, (jp.npad / (2 * B) + (32 / G) - 1) / (32 / G));
    } else if (B > 1) {
      jp.threads = jac::kMaxThreadsBlocked;
    } else {
      const int ppw = 32 / G;
      const int maxw = (c.elem == 8 ? jac::kMaxThreadsF64 : jac::kMaxThreadsF32) / 32;
      const int want = (jp.npad / 2 + ppw - 1) / ppw;
      jp.threads = 32 * std::max(4, std::min(maxw, want));
    }
    // the kernel's static shared memory (per-pair scalars of the FP64 sweeps, counters)
    // takes up to ~4 KB beside the dynamic part
    const size_t cap = (size_t)kSmemOptin - 5120;
    need = c.elem == 8 ? svt_smem<double>(jp) : svt_smem<float>(jp);
    if (need > cap) {
      jp.w_in_smem = false;
      need = c.elem == 8 ? svt_smem<double>(jp) : svt_smem<float>(jp);
      if (need > cap) return LT_ERR_SHAPE;
    }
  } else {
    jp.ld = jp.m | 1;  // odd leading dimension: conflict-free transposed stores
    const int maxE = c.elem == 8 ? 16 : 32;
    int E = 1;
    while (32 * E < jp.m) E *= 2;
    if (E > maxE) return LT_ERR_SHAPE;  // column must fit the registers of a warp
    jp.E = E;
    need = c.elem == 8 ? smem_need<double>(jp) : smem_need<float>(jp);
    if (need > (size_t)kSmemOptin - 1024) {
      jp.w_in_smem = false;
      need = c.elem == 8 ? smem_need<double>(jp) : smem_need<float>(jp);
      if (need > (size_t)kSmemOptin - 1024) return LT_ERR_SHAPE;
    }
  }
  jp.smem = (int)need;
  const int grid = jacobi_grid(c, jp);
  size_t ws = 0;
  if (!jp.w_in_smem) ws += (size_t)c.elem * grid * jp.ld * jp.npad;
  if (mode == JAC_SVD) ws += (size_t)c.elem * grid * jp.npad * jp.npad;
  jp.ws_bytes = (ws + 255) & ~size_t(255);
  if (mode == JAC_SVT && c.jacobi_cluster == 0 && c.jacobi_group == 0 && c.jacobi_pairwise == 0 &&
      c.elem == 8) {
    // planner's choice between one CTA and a cluster per slice, FP64 only (FP32 keeps
    // the register-blocked one-CTA sweeps unless the cluster form is forced: the model
    // counts a launch as if it had the GPU to itself, which batches of FP32 problems,
    // whose other launches fill the SMs, contradicted)
    JacobiPlan best = jp;
    for (int C : {3, 4}) {
      JacobiPlan q = jp;
      if (cluster_plan(c, &q, C) && svt_cost(c, q) < svt_cost(c, best)) best = q;
    }
    jp = best;
  }
  *out = jp;
  return LT_OK;
}

cudaError_t launch_jacobi(const Ctx& c, const JacobiPlan& jp, const JacobiIO& io,
                          cudaStream_t st) {
  JArgs a;
  a.jp = jp;
  a.io = io;
  a.max_sweeps = c.max_sweeps;
  // default pair tolerance, r = rows of the orthogonalised matrix (n for the SVT kernel,
  // which works on R^T; m for the SVD kernel): r u in FP64; max(sqrt(r) / 8, 4) u in
  // FP32 -- the FP32 SVT error is proportional to the tolerance down to a floor of a
  // few 1e-7 (measured: 9.1e-6 at sqrt(r) u, 1.0e-6 at sqrt(r) u / 10 for 540 x 960
  // slices) and the momentum of PGA amplifies per-call errors about tenfold; below ~4 u
  // the rounding of the FP32 dot products keeps small slices from converging
  const double u = c.elem == 8 ? DBL_EPSILON / 2 : FLT_EPSILON / 2;
  const double rows = jp.mode != JAC_SVD ? jp.n : jp.m;
  a.tol = c.jacobi_tol > 0 ? c.jacobi_tol
                           : (c.elem == 8 ? rows * u : std::max(std::sqrt(rows) / 8.0, 4.0) * u);
  a.status = c.d_status;
  const int grid = jacobi_grid(c, jp);
  if (jp.cluster > 1) return jac::launch_svt_cluster(a, grid, st);
  if (jp.mode != JAC_SVD) {
    // try the translation units in turn; each returns cudaErrorNotSupported for shapes
    // it does not hold
    using L = cudaError_t (*)(const JArgs&, int, cudaStream_t);
    static const L f32[] = {jac::launch_svt_f32_blk_a, jac::launch_svt_f32_blk_b,
                            jac::launch_svt_f32_blk_c, jac::launch_svt_f32_blk_d,
                            jac::launch_svt_f32_blk_e, jac::launch_svt_f32_pw_a,
                            jac::launch_svt_f32_pw_b};
    static const L f64[] = {jac::launch_svt_f64_a, jac::launch_svt_f64_b, jac::launch_svt_f64_c};
    const L* tab = c.elem == 8 ? f64 : f32;
    const int cnt = c.elem == 8 ? 3 : 7;
    for (int i = 0; i < cnt; ++i) {
      const cudaError_t e = tab[i](a, grid, st);
      if (e != cudaErrorNotSupported) return e;
    }
    return cudaErrorNotSupported;
  }
  return c.elem == 8 ? launch_t<double>(a, grid, st) : launch_t<float>(a, grid, st);
}

}  // namespace lt
