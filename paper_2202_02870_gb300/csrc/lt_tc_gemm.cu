// Kernel G on the fifth-generation tensor cores (LT_MIXED contexts): the batched product
//   D_b = A_b B_b,  b = 0 .. batch-1,
// in split TF32.  Every FP32 operand x is split as x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi), and the tile accumulates hi_A hi_B in one FP32 accumulator and
// hi_A lo_B + lo_A hi_B in a second one, added in the epilogue (the three-term product:
// the dropped lo_A lo_B term and the rounding of lo are below 2^-21 |a b| per product).
// The tensor cores' FP32 accumulation rounds toward zero: measured on the mode
// products (K = 32 .. 120) with one accumulator for all three terms, the relative error
// was a bias of -2.5e-7 .. -7.8e-7, growing with K; keeping the small terms apart leaves
// the large accumulator a third of the additions.
//
// It serves the two dense contractions of the method:
//  * the face-wise product of Sec. 3.1 inside Algorithm 2: A_b = L(A)^p (I1 x l),
//    B_b = L(B)^p (l x I2), D_b = L(C)^p, b = p;
//  * the n-mode products of Eq. 3 that make up L and L^{-1} (Sec. 3.2) for a large mode
//    k: with S the number of elements between consecutive indices of mode k, every
//    outer block o is an S x I_k column-major matrix X_o and Y_o = X_o M_k^T (so
//    B = M_k^T, shared by all blocks).
//
// Layouts (column-major, FP32): A_b(m, k) = A[b sA + m + k lda] (M contiguous),
// B_b(k, n) = B[b sB + k + n ldb] (K contiguous; sB = 0 when every block shares B),
// D_b(m, n) = D[b sD + m + n ldd].
//
// Persistent kernel, one CTA per SM; a CTA takes 128 x BN output tiles of the D_b in
// turn (column tiles fastest), K in chunks of 32 FP32 (one 128-byte row):
//   warp 12   TMA producer (one thread): per chunk, the raw A chunk (128 x 32, M
//             fastest, no swizzle) and the B chunk (32 x BN, K fastest, 128-byte swizzle,
//             which is the K-major canonical operand layout) into a ring of up to six
//             raw stages, completion counted on an mbarrier (complete_tx).
//   warps 4-11 converters (an accumulator row and half of K per thread): read a raw stage into
//             registers and release it at once, then write hi and lo of A transposed
//             into the K-major 128-byte-swizzled layout and hi and lo of B at the raw
//             (swizzled) positions into a ring of two converted stages.
//   warp 13   TMEM allocation (two stages of two 128 x BN accumulators; one stage when
//             BN = 256) and the MMA issuer (one thread): per 8-deep K step three
//             tcgen05.mma kind::tf32, hi hi into the stage's first accumulator, hi lo and
//             lo hi into its second; tcgen05.commit releases a converted stage and, after
//             the last chunk, hands the accumulator stage to the epilogue.
//   warps 0-3 epilogue: TMEM -> registers (tcgen05.ld of both accumulators, one row per
//             thread), their sum -> global (32 consecutive rows per warp store) while
//             the next tile accumulates in the other stage.
// Every wait on an mbarrier is bounded (1 s by default, TcGemm::wait_ns): on expiry the
// CTA raises LT_DEV_TIMEOUT, every role stops issuing work, the producer waits (bounded)
// for its copies in flight, the issuer for its MMAs, the TMEM is freed and the CTA
// returns.
#include <cuda.h>

#include <mutex>

#include "lt_internal.cuh"

namespace lt {
namespace {

constexpr int kBM = 128;                      // tile rows (TMEM lanes)
constexpr int kBK = 32;                       // K per chunk: one 128-byte row of FP32
constexpr int kThreads = 448;                 // warps 0-3 epilogue, 4-11 convert, 12 loads,
                                              // 13 allocates TMEM and issues the MMAs
constexpr int kConv = 256;                    // converter threads
constexpr int kMaxRaw = 6;                    // raw (TMA) stages at most
constexpr uint32_t kABytes = kBM * kBK * 4;   // 16 KiB per A buffer
constexpr int kSmemLimit = 232448;            // opt-in shared memory per block
constexpr unsigned long long kWaitNs = 1000000000ull;  // default wait limit (1 s)

struct TcParams {
  int64_t M, N, K, batch;
  float* D;
  int64_t ldd, sD;
  int64_t m_tiles, n_tiles;
  int raw_stages;       // TMA ring depth (<= kMaxRaw)
  int conv_stages;      // converted-operand ring depth (1 or 2)
  int b_batched;        // B has a batch coordinate (else every block uses B_0)
  int32_t* status;      // device status word (LT_DEV_TIMEOUT)
  unsigned long long wait_ns;  // limit of every mbarrier wait
  int no_loads;         // test switch: the producer issues no copies, so the first
                        // waits of the other roles expire (LT_DEV_TIMEOUT)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
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

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the completion of the mbarrier phase of the given parity.  Gives up after
// wait_ns (raising the CTA's abort flag and LT_DEV_TIMEOUT) or, when honour_abort is
// set, as soon as another role of the CTA has given up.
__device__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                          int32_t* status, bool honour_abort, unsigned long long wait_ns) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(a, parity)) return true;
    if ((i & 127u) == 0) {
      if (honour_abort && *abort_flag) return false;
      if (global_ns() - t0 > wait_ns) {
        *abort_flag = 1;
        atomicOr(status, LT_DEV_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t mbar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory operand descriptor of a K-major tile in the 128-byte swizzled canonical
// layout: rows of 128 bytes (32 FP32 along K), groups of 8 rows 1024 bytes apart,
// 1024-byte aligned groups.  Fields: start address >> 4 (bits 0-13), leading byte
// offset >> 4 (bits 16-29; unused by this layout), stride byte offset >> 4 (bits 32-45),
// descriptor version 1 (bits 46-47), base offset 0, swizzle mode 2 = 128 bytes
// (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

// 16 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_tf32x3(const __grid_constant__ CUtensorMap map_a,
               const __grid_constant__ CUtensorMap map_b, const TcParams p) {
  constexpr uint32_t kBBytes = BN * 128;                  // one B buffer: BN rows of 128 B
  constexpr uint32_t kRawBytes = kABytes + kBBytes;       // raw A [k][m] + raw B (swizzled)
  constexpr uint32_t kConvBytes = 2 * kABytes + 2 * kBBytes;  // A hi, A lo, B hi, B lo
  // An accumulator stage is a pair of 128 x BN FP32 accumulators: hi hi in the first,
  // hi lo + lo hi in the second (added in the epilogue).  Two stages (the epilogue of a
  // tile overlaps the products of the next) where they fit the 512 TMEM columns.
  constexpr uint32_t kAccCols = BN < 32 ? 32 : BN;
  constexpr int kStages = 4 * kAccCols <= 512 ? 2 : 1;
  constexpr uint32_t kTmemCols = kStages * 2 * kAccCols;  // a power of two, 128..512
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;      // swizzled tiles: 1024-aligned
  unsigned char* sbase = smem_raw + (base - raw_addr);
  const int R = p.raw_stages, C = p.conv_stages;
  const uint32_t conv0 = (uint32_t)R * kRawBytes;         // conv ring after the raw ring
  // control block: raw_full[6] raw_empty[6] conv_full[2] conv_empty[2] acc_full[2]
  // acc_empty[2] done | tmem address | abort
  uint64_t* bars = reinterpret_cast<uint64_t*>(sbase + conv0 + (size_t)C * kConvBytes);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kMaxRaw + 4 * 2 + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const uint32_t bar0 = smem_u32(bars);
  auto raw_full = [&](int i) { return bar0 + 8u * i; };
  auto raw_empty = [&](int i) { return bar0 + 8u * (kMaxRaw + i); };
  auto conv_full = [&](int i) { return bar0 + 8u * (2 * kMaxRaw + i); };
  auto conv_empty = [&](int i) { return bar0 + 8u * (2 * kMaxRaw + 2 + i); };
  auto acc_full = [&](int i) { return bar0 + 8u * (2 * kMaxRaw + 4 + i); };
  auto acc_empty = [&](int i) { return bar0 + 8u * (2 * kMaxRaw + 6 + i); };
  const uint32_t done_bar = bar0 + 8u * (2 * kMaxRaw + 8);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nchunks = (int)((p.K + kBK - 1) / kBK);
  const int64_t ntiles = p.batch * p.m_tiles * p.n_tiles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < R; ++i) {
      mbar_init(raw_full(i), 1);
      mbar_init(raw_empty(i), kConv);
    }
    for (int i = 0; i < C; ++i) {
      mbar_init(conv_full(i), kConv);
      mbar_init(conv_empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(acc_full(i), 1);
      mbar_init(acc_empty(i), 128);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 13) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  // tile t -> (batch b, row tile, column tile), column tiles fastest (neighbouring CTAs
  // share the A tile in L2)
  auto tile_coords = [&](int64_t t, int64_t& b, int& m0, int& n0) {
    const int64_t nt = t % p.n_tiles;
    const int64_t rest = t / p.n_tiles;
    m0 = (int)((rest % p.m_tiles) * kBM);
    b = rest / p.m_tiles;
    n0 = (int)(nt * BN);
  };

  if (warp == 12) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int last[kMaxRaw];
      for (int i = 0; i < kMaxRaw; ++i) last[i] = -1;
      int64_t g = 0;
      bool ok = !p.no_loads;
      for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        int64_t b;
        int m0, n0;
        tile_coords(t, b, m0, n0);
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int r = (int)(g % R);
          if (g >= R && !mbar_wait(raw_empty(r), (uint32_t)((g / R) - 1) & 1u, abort_flag,
                                   p.status, true, p.wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t st = base + (uint32_t)r * kRawBytes;
          mbar_expect_tx(raw_full(r), kRawBytes);
          tma_load_3d(st, &map_a, raw_full(r), m0, c * kBK, (int)b);
          tma_load_3d(st + kABytes, &map_b, raw_full(r), c * kBK, n0, p.b_batched ? (int)b : 0);
          last[r] = (int)(g / R);
        }
      }
      // never leave while copies into this CTA's shared memory are in flight
      for (int i = 0; i < R; ++i)
        if (last[i] >= 0) mbar_wait(raw_full(i), (uint32_t)last[i] & 1u, abort_flag, p.status, false, p.wait_ns);
    }
  } else if (warp == 13) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 =
      // 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                             ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
      int64_t g = 0, it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++it) {
        const int a = (int)(it % kStages);
        if (it >= kStages && !mbar_wait(acc_empty(a), (uint32_t)((it / kStages) - 1) & 1u, abort_flag,
                                  p.status, true, p.wait_ns))
          break;
        tc_fence_after();
        const uint32_t dmain = tmem + (uint32_t)a * 2 * kAccCols;  // hi hi
        const uint32_t dsmall = dmain + kAccCols;                   // hi lo + lo hi
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int q = (int)(g % C);
          if (!mbar_wait(conv_full(q), (uint32_t)(g / C) & 1u, abort_flag, p.status, true, p.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + conv0 + (uint32_t)q * kConvBytes;
          const uint32_t a_hi = st, a_lo = st + kABytes;
          const uint32_t b_hi = st + 2 * kABytes, b_lo = b_hi + kBBytes;
#pragma unroll
          for (int ks = 0; ks < kBK / 8; ++ks) {  // 8 TF32 = 32 bytes per MMA
            const uint32_t off = 32u * ks;
            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(dmain, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, acc);
            mma_tf32(dsmall, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, acc);
            mma_tf32(dsmall, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
          }
          mma_commit(conv_empty(q));
        }
        if (ok) mma_commit(acc_full(a));
      }
      mma_commit(done_bar);  // completes once every MMA issued above has finished
      mbar_wait(done_bar, 0u, abort_flag, p.status, false, p.wait_ns);
    }
  } else if (warp >= 4) {
    // ---------------------------------------------------------------- converters
    // thread t: accumulator row m = t % 128, K half h = t / 128 (16 of the 32 values)
    const int t = threadIdx.x - 128;
    const int mrow = t & (kBM - 1), h = t >> 7;
    const int r8 = mrow & 7;            // row within its 8-row swizzle group
    constexpr int kBVec = BN * (kBK / 4) / kConv;  // float4 of B per thread per chunk
    constexpr int kHalf = kBK / 2;
    int64_t g = 0;
    bool ok = true;
    for (int64_t tt = blockIdx.x; ok && tt < ntiles; tt += gridDim.x) {
      for (int c = 0; c < nchunks; ++c, ++g) {
        const int r = (int)(g % R), q = (int)(g % C);
        if (!mbar_wait(raw_full(r), (uint32_t)(g / R) & 1u, abort_flag, p.status, true, p.wait_ns)) {
          ok = false;
          break;
        }
        const unsigned char* raw = sbase + (size_t)r * kRawBytes;
        const float* araw = reinterpret_cast<const float*>(raw);  // [k][m], m fastest
        const float4* braw = reinterpret_cast<const float4*>(raw + kABytes);
        float v[kHalf];
#pragma unroll
        for (int k = 0; k < kHalf; ++k) v[k] = araw[(h * kHalf + k) * kBM + mrow];
        float4 bv[kBVec];
#pragma unroll
        for (int i = 0; i < kBVec; ++i) bv[i] = braw[t + kConv * i];
        mbar_arrive(raw_empty(r));  // the raw stage may be refilled
        if (g >= C && !mbar_wait(conv_empty(q), (uint32_t)((g / C) - 1) & 1u, abort_flag,
                                 p.status, true, p.wait_ns)) {
          ok = false;
          break;
        }
        unsigned char* cv = sbase + conv0 + (size_t)q * kConvBytes;
        unsigned char* row_hi = cv + (mrow >> 3) * 1024 + r8 * 128;
        unsigned char* row_lo = row_hi + kABytes;
#pragma unroll
        for (int qq = 0; qq < kHalf / 4; ++qq) {
          float4 hv, lv;
          split(v[4 * qq + 0], hv.x, lv.x);
          split(v[4 * qq + 1], hv.y, lv.y);
          split(v[4 * qq + 2], hv.z, lv.z);
          split(v[4 * qq + 3], hv.w, lv.w);
          const int kq = h * (kHalf / 4) + qq;  // 16-byte chunk of the 128-byte row
          const int off = (kq ^ r8) << 4;       // swizzled position
          *reinterpret_cast<float4*>(row_hi + off) = hv;
          *reinterpret_cast<float4*>(row_lo + off) = lv;
        }
        float4* bh = reinterpret_cast<float4*>(cv + 2 * kABytes);
        float4* bl = reinterpret_cast<float4*>(cv + 2 * kABytes + kBBytes);
#pragma unroll
        for (int i = 0; i < kBVec; ++i) {  // same (swizzled) positions as the raw stage
          float4 hv, lv;
          split(bv[i].x, hv.x, lv.x);
          split(bv[i].y, hv.y, lv.y);
          split(bv[i].z, hv.z, lv.z);
          split(bv[i].w, hv.w, lv.w);
          bh[t + kConv * i] = hv;
          bl[t + kConv * i] = lv;
        }
        fence_proxy_async();  // generic-proxy writes -> visible to the tensor cores
        mbar_arrive(conv_full(q));
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 0-3)
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int a = (int)(it % kStages);
      bool ok = mbar_wait(acc_full(a), (uint32_t)(it / kStages) & 1u, abort_flag, p.status, true,
                          p.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) break;  // warp-uniform for tcgen05.ld
      tc_fence_after();
      int64_t b;
      int m0, n0;
      tile_coords(t, b, m0, n0);
      const int64_t m = (int64_t)m0 + warp * 32 + lane;
      float* Dp = p.D + b * p.sD;
      const uint32_t lane_addr =
          tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)a * 2 * kAccCols;
#pragma unroll 1
      for (int cc = 0; cc < BN; cc += 16) {
        if (n0 + cc >= p.N) break;  // uniform across the warp
        uint32_t acc[16], sml[16];
        tmem_ld16(lane_addr + (uint32_t)cc, acc);
        tmem_ld16(lane_addr + kAccCols + (uint32_t)cc, sml);
        if (m < p.M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t n = (int64_t)n0 + cc + j;
            if (n < p.N) Dp[m + n * p.ldd] = __uint_as_float(acc[j]) + __uint_as_float(sml[j]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(acc_empty(a));  // the accumulator may be overwritten
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 13) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------- host side
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  });
  return fn;
}

uint64_t round16(uint64_t b) { return (b + 15) & ~uint64_t(15); }

// 3-D FP32 tensor map over (d0, d1, d2) with element strides (1, s1, s2).
bool make_map(CUtensorMap* map, const float* ptr, uint64_t d0, uint64_t d1, uint64_t d2,
              uint64_t s1, uint64_t s2, uint32_t box0, uint32_t box1, bool swizzle128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {s1 * 4, s2 * 4};
  const cuuint32_t box[3] = {box0, box1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
constexpr int raw_bytes() { return (int)kABytes + BN * 128; }
template <int BN>
constexpr int conv_bytes() { return 2 * (int)kABytes + 2 * BN * 128; }
constexpr int kCtlBytes = 1024 + 256;  // alignment slack + barriers

// Two converted stages where they fit (BN <= 128), then as many raw stages as fit.
template <int BN>
void ring_for(int* raw, int* conv) {
  *conv = (2 * conv_bytes<BN>() + raw_bytes<BN>() + kCtlBytes <= kSmemLimit) ? 2 : 1;
  int r = (kSmemLimit - kCtlBytes - *conv * conv_bytes<BN>()) / raw_bytes<BN>();
  *raw = r > kMaxRaw ? kMaxRaw : r;
}

template <int BN>
int smem_for(int raw, int conv) { return raw * raw_bytes<BN>() + conv * conv_bytes<BN>() + kCtlBytes; }

template <int BN>
cudaError_t launch_bn(const TcGemm& g, const CUtensorMap& ma, const CUtensorMap& mb,
                      int32_t* status, cudaStream_t st) {
  static_assert(sizeof(unsigned long long) == sizeof(uint64_t), "wait limit width");
  TcParams p;
  p.M = g.M; p.N = g.N; p.K = g.K; p.batch = g.batch;
  p.D = g.D; p.ldd = g.ldd; p.sD = g.sD;
  p.m_tiles = (g.M + kBM - 1) / kBM;
  p.n_tiles = (g.N + BN - 1) / BN;
  ring_for<BN>(&p.raw_stages, &p.conv_stages);
  p.b_batched = g.sB != 0 ? 1 : 0;
  p.status = status;
  p.wait_ns = g.wait_ns > 0 ? (unsigned long long)g.wait_ns : kWaitNs;
  p.no_loads = g.no_loads ? 1 : 0;
  const int64_t tiles = g.batch * p.m_tiles * p.n_tiles;
  if (tiles < 1 || p.raw_stages < 1) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = kNumSMs;
  const int smem = smem_for<BN>(p.raw_stages, p.conv_stages);
  auto k = tc_gemm_tf32x3<BN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = tiles < sms ? tiles : sms;  // persistent: one CTA per SM
  k<<<(unsigned)grid, kThreads, smem, st>>>(ma, mb, p);
  return cudaGetLastError();
}

}  // namespace

int tc_tile_n(const TcGemm& g, int forced) {
  if (forced) return forced;
  if (g.D == g.A || g.N > 128) {  // in place: one tile must cover every column
    if (g.N <= 32) return 32;
    if (g.N <= 64) return 64;
    if (g.N <= 128) return 128;
    return 256;
  }
  // out of place: the widest tile up to 128 columns (each A chunk is converted once per
  // 128 output columns; measured on (256x256)(256x128) slices: 0.31 ms at 128 vs 0.47 ms
  // at 64)
  if (g.N <= 32) return 32;
  if (g.N <= 64) return 64;
  return 128;
}

bool tc_gemm_supported(const TcGemm& g, int forced_bn) {
  if (!encode_fn()) return false;
  if (g.M < 1 || g.N < 1 || g.K < 1 || g.batch < 1) return false;
  const int64_t lim = INT32_MAX;
  if (g.M > lim || g.N > lim || g.K > lim || g.batch > lim) return false;
  if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(g.B) & 15))
    return false;
  if (g.lda % 4 || g.ldb % 4 || g.lda < g.M || g.ldb < g.K || g.ldd < g.M) return false;
  if (g.batch > 1 && (g.sA % 4 || (g.sB != 0 && g.sB % 4))) return false;
  if (g.D == g.A && (g.N > 256 || g.ldd != g.lda || g.sD != g.sA)) return false;
  const int bn = tc_tile_n(g, forced_bn);
  if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return false;
  if (g.D == g.A && bn < g.N) return false;
  return true;
}

cudaError_t launch_tc_gemm(const TcGemm& g, int forced_bn, int32_t* status, cudaStream_t st) {
  if (!tc_gemm_supported(g, forced_bn)) return cudaErrorInvalidValue;
  const int bn = tc_tile_n(g, forced_bn);
  CUtensorMap ma, mb;
  // A: (M, K, batch); box 128 x 32, no swizzle (converted in shared memory)
  const uint64_t sA = g.batch > 1 ? (uint64_t)g.sA : round16((uint64_t)g.lda * g.K * 4) / 4;
  if (!make_map(&ma, g.A, g.M, g.K, g.batch, g.lda, sA, kBM, kBK, false))
    return cudaErrorInvalidValue;
  // B: (K, N, batch or 1); box 32 x BN with the 128-byte swizzle
  const bool bb = g.sB != 0 && g.batch > 1;
  const uint64_t nb = bb ? (uint64_t)g.batch : 1;
  const uint64_t sB = bb ? (uint64_t)g.sB : round16((uint64_t)g.ldb * g.N * 4) / 4;
  if (!make_map(&mb, g.B, g.K, g.N, nb, g.ldb, sB, kBK, (uint32_t)bn, true))
    return cudaErrorInvalidValue;
  TcGemm h = g;
  h.sB = bb ? g.sB : 0;
  switch (bn) {
    case 32: return launch_bn<32>(h, ma, mb, status, st);
    case 64: return launch_bn<64>(h, ma, mb, status, st);
    case 128: return launch_bn<128>(h, ma, mb, status, st);
    case 256: return launch_bn<256>(h, ma, mb, status, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lt
