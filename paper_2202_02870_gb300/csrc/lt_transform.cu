// Kernel T: the operator L of Sec. 3.2 (and its inverse), L(X) = X x_3 M_3 ... x_K M_K,
// as a sequence of n-mode products (Eq. 3) applied to tiles held in shared memory.
//
// A pass applies a group of consecutive modes to the view [outer][Pg][Sg] of the
// tensor (Sg = elements between consecutive indices of the pass's first mode).  A CTA
// owns a tile of TS consecutive Sg positions of one outer block: it loads the Pg x TS
// sub-matrix once (coalesced TS-wide rows), applies every mode of the pass in shared
// memory (ping-pong buffers; the transform matrices are staged in shared memory and
// read as warp-wide broadcasts), and writes the tile back.  With all modes in one
// pass (the common case) the tensor is read and written exactly once.
//
// Fusions for PGA (Eqs. 51-52, Sec. 5 stopping test):
//   FUSE_PGA_FORWARD  (first pass load)  Y = X + beta (X - X_old);
//                                          G = Y - step * mask * (Y - obs)
//   FUSE_PGA_INVERSE  (last pass store)  X_new -> x_out; per-CTA partial sums of
//                                          ||Y - X_new||^2, ||X_new||^2 and, if asked,
//                                          ||mask (X_new - obs)||^2 (FP64 across tiles)
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kThreads = 256;
constexpr int kU = 4;  // loads in flight per thread in the load phase

template <typename T> struct Vec;  // 16-byte vectors
template <> struct Vec<float> { using type = float4; static constexpr int width = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int width = 2; };
constexpr int kR = 4;  // FP64: outputs per work item (register blocking along the mode)

// FP32 coefficient rows are padded to a multiple of 8 (two 16-byte loads per row chunk).
__host__ __device__ constexpr int padded_rows(int I) { return (I + 7) / 8 * 8; }

template <typename T>
struct Acc;  // per-tile accumulator type of the epilogue sums
template <>
struct Acc<double> { using type = double; };
template <>
struct Acc<float> { using type = float; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct PassArgs {
  TransformPass p;
  int vec;            // 16-byte vector loads and stores are aligned for full tiles
  const void* in;
  void* out;
  const void* mats;   // base of the context's matrix array (fwd or inv)
  PgaFuse fuse;
  int fuse_mode;      // FUSE_* for this pass
};

// FP32 mode products of one tile: a work item is (fiber, R consecutive outputs
// j0..j0+R-1, C = 4 consecutive columns); per input index i one 16-byte load of x (4
// columns) and the R coefficients feed 4 R FMAs (R = 8; R = 2 spreads passes over few
// short fibres, e.g. a tile of 8 rows, over all warps).  Items are ordered output chunk
// first, so the threads of a warp mostly share j0 (uniform coefficient loads).
//
// One work item: mode size I with stride st (in rows of the tile), coefficients MT
// stored transposed with Ip padded rows, fibre start fbase, column group cg.
template <int TS, int R>
__device__ __forceinline__ void item_f32(int I, int st, int Ip, const float* MT, int fbase,
                                         int j0, int cg, const float* src, float* dst) {
  constexpr int C = 4;
  float acc[R][C];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[r][c] = 0.f;
  const float* xp = src + (size_t)fbase * TS + cg * C;
  const float* mp = MT + j0;
  for (int i = 0; i < I; ++i) {
    const float4 x = *reinterpret_cast<const float4*>(xp + (size_t)st * i * TS);
    float mv[R];
    if constexpr (R == 8) {
      const float4 m0 = *reinterpret_cast<const float4*>(mp + i * Ip);
      const float4 m1 = *reinterpret_cast<const float4*>(mp + i * Ip + 4);
      mv[0] = m0.x; mv[1] = m0.y; mv[2] = m0.z; mv[3] = m0.w;
      mv[4] = m1.x; mv[5] = m1.y; mv[6] = m1.z; mv[7] = m1.w;
    } else {
      static_assert(R == 2, "R is 8 or 2");
      const float2 m0 = *reinterpret_cast<const float2*>(mp + i * Ip);
      mv[0] = m0.x; mv[1] = m0.y;
    }
    const float xv[C] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) acc[r][c] = fmaf(mv[r], xv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (j0 + r < I)
      *reinterpret_cast<float4*>(dst + (size_t)(fbase + st * (j0 + r)) * TS + cg * C) =
          make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
}

// Geometry of work item it of a mode (size I, stride st) of a pass with Pg rows.
template <int R>
__device__ __forceinline__ void item_geometry(int it, int I, int st, int Pg, int& fbase,
                                              int& j0) {
  const int nfib = Pg / I;
  const int ch = it / nfib, fiber = it % nfib;
  fbase = fiber % st + st * I * (fiber / st);
  j0 = ch * R;
}

// One mode (index q of the pass) of the FP32 mode products of a tile, src -> dst.
template <int TS, int R = 8>
__device__ __forceinline__ void mode_f32(const TransformPass& p, int q, const float* mats_s,
                                         const int* moff_s, const float* src, float* dst) {
  constexpr int C = 4;
  const int Pg = (int)p.Pg;
  const int cg = threadIdx.x % (TS / C);
  const int rs = threadIdx.x / (TS / C);
  const int nrs = kThreads / (TS / C);  // the compute threads of either kernel
  const int I = p.msize[q], st = p.mstride[q], Ip = padded_rows(I);
  const float* MT = mats_s + moff_s[q];
  const int items = ((I + R - 1) / R) * (Pg / I);
  for (int it = rs; it < items; it += nrs) {
    int fbase, j0;
    item_geometry<R>(it, I, st, Pg, fbase, j0);
    item_f32<TS, R>(I, st, Ip, MT, fbase, j0, cg, src, dst);
  }
}

// All modes of the pass, ping-ponging between src and dst; returns the buffer holding
// the result.
template <int TS>
__device__ __forceinline__ float* modes_f32(const TransformPass& p, const float* mats_s,
                                            const int* moff_s, float* src, float* dst) {
  for (int q = 0; q < p.nm; ++q) {
    mode_f32<TS>(p, q, mats_s, moff_s, src, dst);
    __syncthreads();
    float* t = src; src = dst; dst = t;
  }
  return src;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <typename T, int TS>
__global__ void __launch_bounds__(kThreads, 3)
transform_kernel(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TransformPass& p = a.p;
  if (a.fuse.scal != nullptr && a.fuse.scal->done) return;  // PGA converged earlier

  const int Pg = (int)p.Pg;
  T* buf0 = reinterpret_cast<T*>(smem_raw);
  T* buf1 = buf0 + (size_t)Pg * TS;
  // FP32 passes keep a third tile buffer: the next tile streams in (cp.async) while the
  // current one is transformed
  T* buf2 = buf1 + (size_t)Pg * TS;
  T* mats_s = sizeof(T) == 4 ? buf2 + (size_t)Pg * TS : buf2;

  // Stage the pass's matrices in shared memory: FP64 row-major I x I; FP32 transposed
  // with rows padded to a multiple of 8 (MT[i][j] = M[j][i], zeros beyond I), so that
  // eight consecutive outputs read their coefficients with two 16-byte loads.
  int moff_s[kMaxModes];
  {
    int acc = 0;
    for (int q = 0; q < p.nm; ++q) {
      moff_s[q] = acc;
      const T* src = reinterpret_cast<const T*>(a.mats) + p.mat_off[q];
      const int I = p.msize[q];
      if constexpr (sizeof(T) == 4) {
        const int Ip = padded_rows(I);
        for (int idx = threadIdx.x; idx < I * Ip; idx += blockDim.x) {
          const int i = idx / Ip, j = idx % Ip;
          mats_s[acc + idx] = j < I ? src[j * I + i] : T(0);
        }
        acc += I * Ip;
      } else {
        for (int idx = threadIdx.x; idx < I * I; idx += blockDim.x) mats_s[acc + idx] = src[idx];
        acc += I * I;
      }
    }
  }
  __syncthreads();

  const int lane_s = threadIdx.x % TS;
  const int grp = threadIdx.x / TS;
  const int ngrp = blockDim.x / TS;
  const int64_t tiles_per_outer = (p.Sg + TS - 1) / TS;
  const int64_t ntiles = p.outer * tiles_per_outer;
  using AccT = typename Acc<T>::type;
  double sum_r = 0.0, sum_x = 0.0, sum_f = 0.0;

  const T* gin = reinterpret_cast<const T*>(a.in);
  T* gout = reinterpret_cast<T*>(a.out);
  const T* xc = reinterpret_cast<const T*>(a.fuse.x_cur);
  const T* xo = reinterpret_cast<const T*>(a.fuse.x_old);
  const T* ob = reinterpret_cast<const T*>(a.fuse.obs);
  T* xout = reinterpret_cast<T*>(a.fuse.x_out);
  const uint8_t* mk = a.fuse.mask;
  T beta = T(0), step = T(a.fuse.step);
  if (a.fuse_mode != FUSE_NONE) beta = T(a.fuse.scal->beta);

  if constexpr (sizeof(T) == 4) {
    if (a.vec && a.fuse_mode == FUSE_NONE) {
      // Plain FP32 pass: three tile buffers.  While tile t is transformed (X <-> Y) and
      // stored, tile t + gridDim.x streams into P with 16-byte cp.async copies (zero
      // filled past the end of Sg, which is a multiple of 4 here).
      float* X = buf0;
      float* Y = buf1;
      float* Pf = buf2;
      const int tv = Pg * TS / 4;
      auto issue = [&](int64_t tl, float* dst) {
        const int64_t o = tl / tiles_per_outer;
        const int64_t s0 = (tl % tiles_per_outer) * TS;
        const float* gb = gin + o * p.Pg * p.Sg + s0;
        for (int iv = threadIdx.x; iv < tv; iv += blockDim.x) {
          const int idx = iv * 4, pp = idx / TS, sc = idx % TS;
          const bool in = s0 + sc < p.Sg;
          cp_async16(dst + idx, in ? gb + (int64_t)pp * p.Sg + sc : gin, in ? 16 : 0);
        }
      };
      int64_t tile = blockIdx.x;
      if (tile < ntiles) issue(tile, X);
      cp_async_commit();
      for (; tile < ntiles; tile += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        if (tile + gridDim.x < ntiles) issue(tile + gridDim.x, Pf);
        cp_async_commit();
        const float* res = modes_f32<TS>(p, mats_s, moff_s, X, Y);
        const int64_t o = tile / tiles_per_outer;
        const int64_t s0 = (tile % tiles_per_outer) * TS;
        float* gb = gout + o * p.Pg * p.Sg + s0;
        for (int iv = threadIdx.x; iv < tv; iv += blockDim.x) {
          const int idx = iv * 4, pp = idx / TS, sc = idx % TS;
          if (s0 + sc < p.Sg)
            *reinterpret_cast<float4*>(gb + (int64_t)pp * p.Sg + sc) =
                *reinterpret_cast<const float4*>(res + idx);
        }
        __syncthreads();  // X and Y are free again
        float* t = X;
        X = Pf;
        Pf = Y;
        Y = t;
      }
      cp_async_wait_all();
      return;
    }
  }

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t o = tile / tiles_per_outer;
    const int64_t s0 = (tile % tiles_per_outer) * TS;
    const int64_t base = o * p.Pg * p.Sg + s0;
    const bool full = (s0 + TS <= p.Sg);

    // ---- load (with the PGA prologue when fusing the forward transform).  Each thread
    // issues kU loads (16-byte vectors where the tile allows) before it writes any of
    // them to shared memory, so that enough bytes are in flight to cover the latency.
    const int total = Pg * TS;
    if (a.vec && full && a.fuse_mode == FUSE_NONE) {
      using V = typename Vec<T>::type;
      constexpr int VW = Vec<T>::width;
      const int tv = total / VW;
      for (int i0 = threadIdx.x; i0 < tv; i0 += kU * blockDim.x) {
        V v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int iv = i0 + u * blockDim.x;
          if (iv < tv) {
            const int idx = iv * VW, pp = idx / TS, sc = idx % TS;
            v[u] = *reinterpret_cast<const V*>(gin + base + (int64_t)pp * p.Sg + sc);
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int iv = i0 + u * blockDim.x;
          if (iv < tv) *reinterpret_cast<V*>(buf0 + iv * VW) = v[u];
        }
      }
    } else {
      for (int i0 = threadIdx.x; i0 < total; i0 += kU * blockDim.x) {
        T v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = i0 + u * blockDim.x;
          v[u] = T(0);
          const int pp = idx / TS, sc = idx % TS;
          if (idx < total && (full || s0 + sc < p.Sg)) {
            const int64_t e = base + (int64_t)pp * p.Sg + sc;
            if (a.fuse_mode == FUSE_PGA_FORWARD) {
              const T x = xc[e], x_old = xo[e];
              const T y = x + beta * (x - x_old);
              v[u] = mk[e] ? y - step * (y - ob[e]) : y;
            } else {
              v[u] = gin[e];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = i0 + u * blockDim.x;
          if (idx < total) buf0[idx] = v[u];
        }
      }
    }
    __syncthreads();

    // ---- mode products, one mode after the other
    T* src = buf0;
    T* dst = buf1;
    if constexpr (sizeof(T) == 4) {
      src = modes_f32<TS>(p, mats_s, moff_s, src, dst);
    } else
    for (int q = 0; q < p.nm; ++q) {
      const int I = p.msize[q], st = p.mstride[q];
      const T* M = mats_s + moff_s[q];
      const int nch = (I + kR - 1) / kR;
      const int items = (Pg / I) * nch;
      for (int it = grp; it < items; it += ngrp) {
        const int fiber = it / nch, ch = it % nch;
        const int aa = fiber % st, bb = fiber / st;
        const int fbase = aa + st * I * bb;
        const int j0 = ch * kR;
        T acc[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) acc[r] = T(0);
        for (int i = 0; i < I; ++i) {
          const T x = src[(fbase + st * i) * TS + lane_s];
#pragma unroll
          for (int r = 0; r < kR; ++r)
            if (j0 + r < I) acc[r] = fma(M[(j0 + r) * I + i], x, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kR; ++r)
          if (j0 + r < I) dst[(fbase + st * (j0 + r)) * TS + lane_s] = acc[r];
      }
      __syncthreads();
      T* t = src; src = dst; dst = t;
    }

    // ---- store (with the PGA epilogue when fusing the inverse transform)
    AccT tr = AccT(0), tx = AccT(0), tf = AccT(0);
    if (a.vec && full && a.fuse_mode == FUSE_NONE) {
      using V = typename Vec<T>::type;
      constexpr int VW = Vec<T>::width;
      for (int iv = threadIdx.x; iv < total / VW; iv += blockDim.x) {
        const int idx = iv * VW, pp = idx / TS, sc = idx % TS;
        *reinterpret_cast<V*>(gout + base + (int64_t)pp * p.Sg + sc) =
            *reinterpret_cast<const V*>(src + idx);
      }
    } else
    for (int idx = threadIdx.x; idx < Pg * TS; idx += blockDim.x) {
      const int pp = idx / TS, s = idx % TS;
      if (!(full || s0 + s < p.Sg)) continue;
      const int64_t e = base + (int64_t)pp * p.Sg + s;
      const T xn = src[idx];
      if (a.fuse_mode == FUSE_PGA_INVERSE) {
        const T x = xc[e], x_old = xo[e];
        const T y = x + beta * (x - x_old);
        const T d = y - xn;
        tr = fma(AccT(d), AccT(d), tr);
        tx = fma(AccT(xn), AccT(xn), tx);
        if (a.fuse.objective && mk[e]) {
          const T f = xn - ob[e];
          tf = fma(AccT(f), AccT(f), tf);
        }
        xout[e] = xn;
      } else {
        gout[e] = xn;
      }
    }
    sum_r += double(tr);
    sum_x += double(tx);
    sum_f += double(tf);
    __syncthreads();  // buffers are reused by the next tile
  }

  if (a.fuse_mode == FUSE_PGA_INVERSE) {
    __shared__ double red[3][kThreads / 32];
    sum_r = warp_sum(sum_r);
    sum_x = warp_sum(sum_x);
    sum_f = warp_sum(sum_f);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    if (l == 0) { red[0][w] = sum_r; red[1][w] = sum_x; red[2][w] = sum_f; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double r0 = 0, r1 = 0, r2 = 0;
      for (int i = 0; i < (int)(blockDim.x / 32); ++i) { r0 += red[0][i]; r1 += red[1][i]; r2 += red[2][i]; }
      double* out = a.fuse.partials + 4 * (size_t)blockIdx.x;
      out[0] = r0; out[1] = r1; out[2] = r2; out[3] = 0.0;
    }
  }
}

template <typename T>
size_t smem_bytes(const TransformPass& p, int ts) {
  size_t mats = 0;
  for (int q = 0; q < p.nm; ++q)
    mats += (size_t)p.msize[q] * (sizeof(T) == 4 ? padded_rows(p.msize[q]) : p.msize[q]);
  return ((sizeof(T) == 4 ? 3 : 2) * (size_t)p.Pg * ts + mats) * sizeof(T);
}

// ---------------------------------------------------------------------------------
// Plain FP32 passes through the tensor memory accelerator.  The view [outer][Pg][Sg]
// is a 2-D tensor of Pg * outer rows of Sg floats, and a tile (Pg rows x TS columns of
// one outer block) is one TMA box.  A CTA is eight compute warps and one copy warp: one
// thread of the copy warp keeps up to kTmaStages tiles in flight into a ring of
// shared-memory stages (mbarrier complete_tx), writes each finished tile back with one
// TMA store and, once the store has read it, gives the buffer back (the stage to the load
// of a later tile; with an odd number of modes the result sits in one of two scratch
// tiles, which a "free" mbarrier returns to the compute warps).  The compute warps wait
// for a stage, run the mode products between the stage and scratch, synchronise among
// themselves on a named barrier and signal "done"; they never wait for a store.  Two CTAs
// share an SM.  The arithmetic is mode_f32's, so the results equal the SIMT pass bit for
// bit.  Every wait on an mbarrier is bounded (1 s, or LT_OPT_TC_WAIT_US; then
// LT_DEV_TIMEOUT, both roles stop, the loads in flight are drained with bounded waits and
// the stores completed before the copy thread exits).
// ---------------------------------------------------------------------------------
constexpr int kTmaStages = 8;
constexpr unsigned long long kTmaWaitNs = 1000000000ull;
constexpr int kTmaThreads = kThreads + 32;  // eight compute warps and one copy warp

// named barrier 1 over the compute warps; the AND form agrees on a flag
__device__ __forceinline__ void compute_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}
__device__ __forceinline__ bool compute_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kThreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool tma_mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false after kTmaWaitNs.
__device__ bool tma_mbar_wait(uint32_t a, uint32_t parity,
                              unsigned long long limit_ns = kTmaWaitNs) {
  if (tma_mbar_try(a, parity)) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 1;; ++i) {
    if (tma_mbar_try(a, parity)) return true;
    if ((i & 127u) == 0) {
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit_ns) return false;
    }
  }
}
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                              int x, int y, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tma_store_tile(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

template <int TS, int R>
__global__ void __launch_bounds__(kTmaThreads, 2)
transform_tma_kernel(const __grid_constant__ CUtensorMap map_in,
                     const __grid_constant__ CUtensorMap map_out, const PassArgs a,
                     int stages, int32_t* status, unsigned long long wait_ns, int no_loads) {
  extern __shared__ __align__(16) unsigned char tma_smem[];
  const TransformPass& p = a.p;
  const int Pg = (int)p.Pg;
  const uint32_t tile_bytes = (uint32_t)Pg * TS * 4;
  const uint32_t tile_pad = (tile_bytes + 1023u) & ~1023u;
  // [stages][T] tiles (1024-byte aligned; two T tiles when the number of modes is odd),
  // the matrices, the barriers: full[stages], done[stages], tfree[2]
  const int nt = (p.nm & 1) ? 2 : 1;
  const uint32_t raw = smem_addr(tma_smem);
  unsigned char* base = tma_smem + (((raw + 1023u) & ~1023u) - raw);
  float* stage_buf = reinterpret_cast<float*>(base);
  float* tbuf0 = reinterpret_cast<float*>(base + (size_t)stages * tile_pad);
  float* mats_s = reinterpret_cast<float*>(base + (size_t)(stages + nt) * tile_pad);
  int moff_s[kMaxModes];
  int mat_elems = 0;
  for (int q = 0; q < p.nm; ++q) {
    moff_s[q] = mat_elems;
    mat_elems += p.msize[q] * padded_rows(p.msize[q]);
  }
  uint64_t* full = reinterpret_cast<uint64_t*>(mats_s + ((mat_elems + 1) & ~1));
  uint64_t* done = full + stages;
  uint64_t* tfree = done + stages;

  // stage the matrices transposed with rows padded to a multiple of 8 (as transform_kernel)
  for (int q = 0; q < p.nm; ++q) {
    const float* src = reinterpret_cast<const float*>(a.mats) + p.mat_off[q];
    const int I = p.msize[q], Ip = padded_rows(I);
    for (int idx = threadIdx.x; idx < I * Ip; idx += blockDim.x) {
      const int i = idx / Ip, j = idx % Ip;
      mats_s[moff_s[q] + idx] = j < I ? src[j * I + i] : 0.f;
    }
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 * stages + 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(full + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the last barrier of all threads: the roles part here

  // a CTA takes a contiguous run of tiles (consecutive column ranges of the same rows),
  // so that every row of its tiles is read and written in long runs
  const int64_t tpo = (p.Sg + TS - 1) / TS;
  const int64_t ntiles = p.outer * tpo;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t first = (int64_t)blockIdx.x * per;
  const int64_t mine = first < ntiles ? std::min<int64_t>(per, ntiles - first) : 0;

  if (threadIdx.x >= kThreads) {
    // ---- copy warp: one thread issues every load and store
    if (threadIdx.x != kThreads) return;
    // tile positions advance along a row of tiles, then to the next row group (kept
    // incrementally, no 64-bit divisions per tile)
    int64_t lxt = first % tpo, lyt = first / tpo, sxt = lxt, syt = lyt;
    int64_t issued = 0;
    // (test switch: no loads at all, so that the compute warps' first waits expire)
    for (; !no_loads && issued < stages && issued < mine; ++issued) {
      tma_load_tile(smem_addr(stage_buf) + (uint32_t)issued * tile_pad, &map_in,
                    smem_addr(full + issued), (int)(lxt * TS), (int)(lyt * Pg), tile_bytes);
      if (++lxt == tpo) { lxt = 0; ++lyt; }
    }
    int64_t i = 0;
    int s = 0;
    uint32_t ph = 0;
    for (; i < mine; ++i) {
      if (!tma_mbar_wait(smem_addr(done + s), ph, wait_ns)) {
        atomicOr(status, LT_DEV_TIMEOUT);
        break;
      }
      const uint32_t res = (p.nm & 1) ? smem_addr(tbuf0) + (uint32_t)(i & 1) * tile_pad
                                      : smem_addr(stage_buf) + (uint32_t)s * tile_pad;
      tma_store_tile(&map_out, res, (int)(sxt * TS), (int)(syt * Pg));
      if (++sxt == tpo) { sxt = 0; ++syt; }
      // the stage takes tile i + stages: at once when the result is in T (the mode
      // products only read the stage), else once the store has read it
      if (!(p.nm & 1)) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      if (!no_loads && issued < mine) {
        tma_load_tile(smem_addr(stage_buf) + (uint32_t)s * tile_pad, &map_in, smem_addr(full + s),
                      (int)(lxt * TS), (int)(lyt * Pg), tile_bytes);
        if (++lxt == tpo) { lxt = 0; ++lyt; }
        ++issued;
      }
      if (p.nm & 1) {  // T(i & 1) goes back to the compute warps for tile i + 2
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        mbar_arrive(smem_addr(tfree + (i & 1)));
      }
      if (++s == stages) { s = 0; ph ^= 1u; }
    }
    // after an expired wait, the loads still in flight land before the thread exits
    for (int64_t j = i; j < issued; ++j)
      tma_mbar_wait(smem_addr(full + j % stages), (uint32_t)((j / stages) & 1), wait_ns);
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    return;
  }

  // ---- compute warps.  Each thread's work item of the first two modes is the same for
  // every tile when no row slot has more than one (true of the passes this form takes),
  // so it is computed once.
  constexpr int C = 4;
  const int cg = threadIdx.x % (TS / C), rs = threadIdx.x / (TS / C);
  const int nrs = kThreads / (TS / C);
  // (the mode sizes and strides are kernel parameters, re-read per tile; only the item's
  // fibre start and first output stay in registers, -1 when the thread has none)
  bool hoist = p.nm <= 2;
  int hfb[2] = {-1, -1}, hj0[2] = {0, 0};
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (q < p.nm) {
      const int I = p.msize[q];
      const int items = ((I + R - 1) / R) * (Pg / I);
      if (items > nrs) hoist = false;
      if (rs < items) item_geometry<R>(rs, I, p.mstride[q], Pg, hfb[q], hj0[q]);
    }
  int s = 0;
  uint32_t ph = 0;
  for (int64_t i = 0; i < mine; ++i) {
    bool ok = tma_mbar_wait(smem_addr(full + s), ph, wait_ns);
    // the scratch tile this one's result goes to was stored two tiles ago
    if ((p.nm & 1) && i >= 2)
      ok = ok && tma_mbar_wait(smem_addr(tfree + (i & 1)), (uint32_t)(((i >> 1) - 1) & 1), wait_ns);
    if (!compute_all(ok)) {
      if (threadIdx.x == 0) atomicOr(status, LT_DEV_TIMEOUT);
      break;
    }
    // modes in turn, stage -> T -> stage -> ...; the result is in T after an odd number
    float* src = stage_buf + (size_t)s * (tile_pad / 4);
    float* dst = tbuf0 + (size_t)(i & (nt - 1)) * (tile_pad / 4);
    if (hoist) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (q < p.nm) {
          const int I = p.msize[q];
          const float* MT = mats_s + (q == 0 ? 0 : p.msize[0] * padded_rows(p.msize[0]));
          if (hfb[q] >= 0)
            item_f32<TS, R>(I, p.mstride[q], padded_rows(I), MT, hfb[q], hj0[q], cg, src, dst);
          compute_sync();
          float* t = src; src = dst; dst = t;
        }
    } else {
      for (int q = 0; q < p.nm; ++q) {
        mode_f32<TS, R>(p, q, mats_s, moff_s, src, dst);
        compute_sync();
        float* t = src; src = dst; dst = t;
      }
    }
    // generic-proxy writes of the result and reads of the stage before the copy thread's
    // async-proxy store and its next load into the stage
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    compute_sync();
    if (threadIdx.x == 0) mbar_arrive(smem_addr(done + s));
    if (++s == stages) { s = 0; ph ^= 1u; }
  }
}

template <typename T, int TS>
cudaError_t launch_pass_t(const Ctx& c, const PassArgs& a, int grid, cudaStream_t st) {
  auto k = transform_kernel<T, TS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.p.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, a.p.smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass(const Ctx& c, const PassArgs& a, int grid, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {  // wide tiles for passes over few, short fibres
    if (a.p.ts == 512) return launch_pass_t<T, 512>(c, a, grid, st);
    if (a.p.ts == 128) return launch_pass_t<T, 128>(c, a, grid, st);
  }
  switch (a.p.ts) {
    case 32: return launch_pass_t<T, 32>(c, a, grid, st);
    case 16: return launch_pass_t<T, 16>(c, a, grid, st);
    case 8: return launch_pass_t<T, 8>(c, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int TS>
int occupancy(const TransformPass& p) {
  int nb = 0;
  cudaFuncSetAttribute(transform_kernel<T, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, transform_kernel<T, TS>, kThreads, p.smem) != cudaSuccess)
    nb = 1;
  return std::max(nb, 1);
}

// ---- TMA passes: host side
using TmaEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmaEncodeFn tma_encode_fn() {
  static std::once_flag once;
  static TmaEncodeFn fn = nullptr;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmaEncodeFn>(ptr);
  });
  return fn;
}

// The pass's view as a 2-D FP32 tensor: Pg * outer rows of Sg elements; box TS x Pg.
bool tma_view(CUtensorMap* map, const void* ptr, const TransformPass& p, int ts) {
  TmaEncodeFn fn = tma_encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)p.Sg, (cuuint64_t)(p.Pg * p.outer)};
  const cuuint64_t strides[1] = {(cuuint64_t)p.Sg * 4};
  const cuuint32_t box[2] = {(cuuint32_t)ts, (cuuint32_t)p.Pg};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tile width of the TMA form of a pass (a box edge is at most 256 elements), or 0 when
// the pass cannot take it.
int tma_ts(const TransformPass& p) {
  if (p.ts == 32 || p.ts == 128) return p.ts;
  if (p.ts == 512) return 256;
  return 0;
}

template <int TS, int R>
cudaError_t launch_tma_t(const Ctx& c, const PassArgs& a, const CUtensorMap& mi,
                         const CUtensorMap& mo, cudaStream_t st) {
  const TransformPass& p = a.p;
  const size_t tile_pad = ((size_t)p.Pg * TS * 4 + 1023) & ~size_t(1023);
  size_t mats = 0;
  for (int q = 0; q < p.nm; ++q) mats += (size_t)p.msize[q] * padded_rows(p.msize[q]) * 4;
  mats = (mats + 15) & ~size_t(15);
  // two CTAs per SM: half of the SM's shared memory each, less the per-CTA reservation
  const size_t fixed = 1024 + ((p.nm & 1) ? 2 : 1) * tile_pad + mats;
  const size_t limit = (size_t)kSmemOptin / 2 - 2048;
  if (fixed + 2 * tile_pad + 16 * 2 + 24 > limit) return cudaErrorNotSupported;
  int stages = (int)std::min<size_t>(kTmaStages, (limit - fixed - 24) / (tile_pad + 16));
  const size_t smem = fixed + (size_t)stages * tile_pad + 8 * (2 * (size_t)stages + 2) + 8;
  auto k = transform_tma_kernel<TS, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = p.outer * ((p.Sg + TS - 1) / TS);
  const int64_t grid = std::min<int64_t>(tiles, 2 * (int64_t)c.sms);
  const unsigned long long wait_ns =
      c.tc_wait_us > 0 ? (unsigned long long)(c.tc_wait_us * 1e3) : kTmaWaitNs;
  k<<<(unsigned)grid, kTmaThreads, smem, st>>>(mi, mo, a, stages, c.d_status, wait_ns,
                                               c.tc_no_loads);
  return cudaGetLastError();
}

// FP32 pass without a PGA fusion through TMA, or cudaErrorNotSupported when its view does
// not meet the tensor-map rules (16-byte aligned base, Sg a multiple of 4, Pg <= 256).
cudaError_t launch_pass_tma(const Ctx& c, const PassArgs& a, cudaStream_t st) {
  const TransformPass& p = a.p;
  const int ts = tma_ts(p);
  if (ts == 0 || p.Pg > 256 || p.Sg % 4 != 0 || p.Sg > (int64_t)INT32_MAX ||
      p.Pg * p.outer > (int64_t)INT32_MAX)
    return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.out)) & 15)
    return cudaErrorNotSupported;
  CUtensorMap mi, mo;
  if (!tma_view(&mi, a.in, p, ts) || !tma_view(&mo, a.out, p, ts)) return cudaErrorNotSupported;
  // work items of 8 outputs x 4 columns leave threads idle when the pass has fewer of
  // them than the CTA has threads (a single mode over a tile of few rows): 2 outputs
  int items = 1 << 30;
  for (int q = 0; q < p.nm; ++q)
    items = std::min<int>(items, (int)((p.Pg / p.msize[q]) * ((p.msize[q] + 7) / 8) * (ts / 4)));
  const bool r2 = items < kThreads && p.nm == 1;
  switch (ts) {
    case 32: return r2 ? launch_tma_t<32, 2>(c, a, mi, mo, st) : launch_tma_t<32, 8>(c, a, mi, mo, st);
    case 128: return r2 ? launch_tma_t<128, 2>(c, a, mi, mo, st) : launch_tma_t<128, 8>(c, a, mi, mo, st);
    case 256: return r2 ? launch_tma_t<256, 2>(c, a, mi, mo, st) : launch_tma_t<256, 8>(c, a, mi, mo, st);
  }
  return cudaErrorNotSupported;
}

template <typename T>
int occupancy_t(const TransformPass& p) {
  if constexpr (sizeof(T) == 4) {
    if (p.ts == 512) return occupancy<T, 512>(p);
    if (p.ts == 128) return occupancy<T, 128>(p);
  }
  switch (p.ts) {
    case 32: return occupancy<T, 32>(p);
    case 16: return occupancy<T, 16>(p);
    default: return occupancy<T, 8>(p);
  }
}

}  // namespace

int transform_grid(const Ctx& c, const TransformPass& p) {
  const int per_sm = c.elem == 8 ? occupancy_t<double>(p) : occupancy_t<float>(p);
  const int64_t tiles = p.outer * ((p.Sg + p.ts - 1) / p.ts);
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)c.sms * per_sm));
}

lt_status plan_transform(const Ctx& c, int64_t S, bool inverse, TransformPlan* plan) {
  // Application order: forward 3..K, inverse K..3 (Sec. 3.2).  The modes of a pass
  // must be consecutive in memory, so a pass is a contiguous index range [k0, k1) of
  // 0-based modes; for the inverse the ranges are visited from the last mode down and
  // each pass applies its modes from its highest to its lowest.
  const int nm = c.nmodes;
  // FP64 passes are bound by the FP64 pipe: fewest passes.  FP32 passes keep two CTAs
  // per SM (loads of one tile overlap the mode products of the other).
  const size_t budget = c.elem == 8 ? 200 * 1024 : 110 * 1024;
  TransformPlan pl;
  pl.inverse = inverse;
  // LT_MIXED: a large mode other than mode 3 gets a pass of its own on the tensor cores
  // (mode 3 stays in the SIMT passes, which carry the PGA fusions).
  auto is_tc = [&](int q) {
    return c.prec == LT_MIXED && q >= 1 && c.tc_mode_min > 0 && c.sizes[q] >= c.tc_mode_min &&
           c.sizes[q] <= 256;
  };
  int k = inverse ? nm - 1 : 0;
  while (inverse ? k >= 0 : k < nm) {
    // grow the group [lo, hi] while it fits
    int lo = k, hi = k;
    auto fits = [&](int l, int h, int ts) {
      TransformPass t;
      t.nm = h - l + 1;
      t.Pg = 1;
      for (int q = l; q <= h; ++q) { t.msize[q - l] = (int)c.sizes[q]; t.Pg *= c.sizes[q]; }
      return (c.elem == 8 ? smem_bytes<double>(t, ts) : smem_bytes<float>(t, ts)) <= budget &&
             t.Pg <= (1 << 20);
    };
    int ts = 32;
    while (ts >= 8 && !fits(lo, hi, ts)) ts /= 2;
    if (ts < 8) return LT_ERR_SHAPE;  // one mode alone too large
    for (;;) {
      if (is_tc(k)) break;
      int nlo = inverse ? lo - 1 : lo, nhi = inverse ? hi : hi + 1;
      if (nlo < 0 || nhi >= nm) break;
      if (is_tc(inverse ? nlo : nhi)) break;
      if (fits(nlo, nhi, 32)) { lo = nlo; hi = nhi; continue; }
      break;
    }
    // TS: widest that fits; FP32 passes over few rows (Pg small) take wider tiles (up to
    // 8192 elements) while that still leaves two tiles per SM
    ts = 32;
    while (ts > 8 && !fits(lo, hi, ts)) ts /= 2;
    if (c.elem == 4 && ts == 32) {
      int64_t pg = 1, before = 1;
      for (int q = lo; q <= hi; ++q) pg *= c.sizes[q];
      for (int q = 0; q < lo; ++q) before *= c.sizes[q];
      int64_t outer = 1;
      for (int q = hi + 1; q < nm; ++q) outer *= c.sizes[q];
      const int64_t sg = S * before;
      for (int w : {512, 128}) {
        if (pg * w <= 8192 && fits(lo, hi, w) && outer * ((sg + w - 1) / w) >= 2 * (int64_t)c.sms) {
          ts = w;
          break;
        }
      }
    }
    TransformPass& ps = pl.pass[pl.npass++];
    ps.nm = hi - lo + 1;
    ps.ts = ts;
    int64_t before = 1, inside = 1, after = 1;
    for (int q = 0; q < lo; ++q) before *= c.sizes[q];
    for (int q = lo; q <= hi; ++q) inside *= c.sizes[q];
    for (int q = hi + 1; q < nm; ++q) after *= c.sizes[q];
    ps.Pg = inside;
    ps.Sg = S * before;
    ps.outer = after;
    // modes in application order with their stride inside Pg
    for (int j = 0; j < ps.nm; ++j) {
      const int q = inverse ? hi - j : lo + j;
      int64_t stride = 1;
      for (int r = lo; r < q; ++r) stride *= c.sizes[r];
      ps.msize[j] = (int)c.sizes[q];
      ps.mstride[j] = (int)stride;
      ps.mat_off[j] = c.mat_off[q];
    }
    ps.smem = (int)(c.elem == 8 ? smem_bytes<double>(ps, ts) : smem_bytes<float>(ps, ts));
    if (is_tc(k)) {
      ps.tc = 1;
      ps.tc_mode = k;
    }
    k = inverse ? lo - 1 : hi + 1;
  }
  *plan = pl;
  return LT_OK;
}

cudaError_t launch_transform(const Ctx& c, const TransformPlan& plan, const void* in,
                             void* out, int fuse_mode, const PgaFuse* fuse,
                             cudaStream_t st, int* grid_out) {
  for (int i = 0; i < plan.npass; ++i) {
    PassArgs a;
    a.p = plan.pass[i];
    a.in = (i == 0) ? in : out;
    a.out = out;
    a.mats = plan.inverse ? c.d_inv : c.d_fwd;
    a.fuse_mode = FUSE_NONE;
    {
      const int vw = 16 / c.elem;
      const uintptr_t al = reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.out);
      a.vec = (a.p.Sg % vw == 0) && (a.p.ts % vw == 0) && (al % 16 == 0);
    }
    if (fuse) a.fuse = *fuse;
    if (fuse_mode == FUSE_PGA_FORWARD && i == 0) a.fuse_mode = FUSE_PGA_FORWARD;
    if (fuse_mode == FUSE_PGA_INVERSE && i == plan.npass - 1) a.fuse_mode = FUSE_PGA_INVERSE;
    if (a.p.tc && a.fuse_mode == FUSE_NONE) {
      // Y_o = X_o M_k^T for every outer block o: X_o is Sg x I column-major (Pg = I).
      const int q = a.p.tc_mode;
      const int64_t I = c.sizes[q];
      TcGemm g;
      g.M = a.p.Sg; g.N = I; g.K = I; g.batch = a.p.outer;
      g.A = static_cast<const float*>(a.in); g.lda = a.p.Sg; g.sA = a.p.Sg * I;
      g.B = (plan.inverse ? c.d_tc_inv : c.d_tc_fwd) + c.tc_off[q]; g.ldb = c.tc_ld[q]; g.sB = 0;
      g.D = static_cast<float*>(out); g.ldd = a.p.Sg; g.sD = a.p.Sg * I;
      g.wait_ns = (uint64_t)(c.tc_wait_us * 1e3); g.no_loads = c.tc_no_loads;
      if (tc_gemm_supported(g, c.tc_tile_n)) {
        const cudaError_t e = launch_tc_gemm(g, c.tc_tile_n, c.d_status, st);
        if (e != cudaSuccess) return e;
        ++c.tc_launches;
        continue;
      }
      // unaligned buffers: the SIMT kernel applies the same mode product
    }
    if (c.elem == 4 && a.fuse_mode == FUSE_NONE && !a.p.tc && c.transform_tma) {
      const cudaError_t e = launch_pass_tma(c, a, st);
      if (e == cudaSuccess) continue;
      if (e != cudaErrorNotSupported) return e;
    }
    const int grid = transform_grid(c, a.p);
    if (grid_out) *grid_out = grid;
    const cudaError_t e = (c.elem == 8) ? launch_pass<double>(c, a, grid, st)
                                        : launch_pass<float>(c, a, grid, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lt
