// Internal declarations shared by the liblt translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "lt.h"

namespace lt {

constexpr int kMaxModes = 8;          // K <= 10
constexpr int kSmemOptin = 232448;    // opt-in shared memory per block on sm_103
constexpr int kNumSMs = 152;          // grid sizing default; refined at context creation

// ----------------------------------------------------------------------------------
// Context
// ----------------------------------------------------------------------------------
struct Ctx {
  int K = 0;
  int nmodes = 0;                     // K - 2
  int64_t sizes[kMaxModes] = {};      // I3..IK
  int64_t P = 0;
  lt_precision prec = LT_FP64;
  int elem = 8;                       // bytes per element
  int sms = kNumSMs;
  int device = 0;
  // Device copies (context precision), row-major I x I each, mode order 3..K.
  void* d_fwd = nullptr;
  void* d_inv = nullptr;
  int64_t mat_off[kMaxModes] = {};    // element offset of mode k's matrix
  int32_t* d_status = nullptr;        // device status word (LT_DEV_* bits)
  // Options
  int max_sweeps = 40;
  double jacobi_tol = 0.0;            // <= 0: default
  int objective = 0;
  int jacobi_group = 0;               // 0: planner's choice
  int jacobi_pairwise = 0;            // 1: no register blocking
  int jacobi_cluster = 0;             // SVT: 0 = planner's choice, 1 = one CTA per slice,
                                      // 3 or 4 = that many CTAs per slice (a cluster)
  int tc_mode_min = 64;               // LT_MIXED: modes of at least this size (and not
                                      // mode 3) run as tensor-core passes; 0 = never
  int tc_tile_n = 0;                  // LT_MIXED: forced tensor-core tile width (0 = auto)
  double tc_wait_us = 0.0;            // LT_MIXED: tensor-core wait limit (0 = default 1 s)
  int tc_no_loads = 0;                // LT_MIXED test switch: no TMA copies are issued
  int transform_tma = 1;              // FP32 passes without PGA fusions through TMA
  int autotune = 0;                   // PGA: time the SVT kernel forms on a new slice shape
  int64_t tuned_I1 = -1, tuned_I2 = -1;  // slice shape the forms were last tuned for
  int warm_period = 0;                // PGA warm start: 0 = off; p >= 2: iterations j with
                                      // j % p == 0 (counted within a call) are cold
  double mu0 = 0.0;                   // PGA continuation: mu_0 (0 = off)
  double nu = 0.9;                    // PGA continuation: decay of mu
  mutable int64_t tc_launches = 0;    // tensor-core kernel launches (lt_ctx_get_stats)
  // Fourier operator (M_3 = F_{I3}): 0 for a real context, else I3.  Mode 3 is then
  // stored as the orthonormal real DFT basis (see lt_fourier.cu for the slot layout).
  int64_t fourier_n = 0;
  // LT_MIXED: the transform matrices as tensor-core B operands, B(k, n) = M(n, k) at
  // k + n * ld (ld = I rounded up to 4, zero padded), each at a 16-byte aligned offset.
  float* d_tc_fwd = nullptr;
  float* d_tc_inv = nullptr;
  int64_t tc_off[kMaxModes] = {};
  int tc_ld[kMaxModes] = {};
  // Pinned host staging for asynchronous reports
  void* h_pinned = nullptr;
  // Statistics (lt_ctx_get_stats)
  int profile = 0;
  lt_stats stats = {};
  double* d_counters = nullptr;       // device: [LT_K_JACOBI] executed Jacobi flops,
                                      // [4..13] Jacobi phase cycles (profiling)
  struct EventRec { cudaEvent_t a, b; int fam; };
  std::vector<EventRec> pending;
  std::vector<cudaEvent_t> pool;
  struct Retired { cudaGraphExec_t exec; cudaEvent_t done; };
  std::vector<Retired> retired;       // batched-PGA graphs awaiting destruction
};

// ----------------------------------------------------------------------------------
// Transform (kernel T): a pass applies a contiguous group of modes to a view
// [outer][Pg][Sg] of the tensor, tiled over Sg.  Element (o, p, s) sits at
// o*Pg*Sg + p*Sg + s.
// ----------------------------------------------------------------------------------
enum FuseMode { FUSE_NONE = 0, FUSE_PGA_FORWARD = 1, FUSE_PGA_INVERSE = 2 };

struct PgaScalars {        // lives in the workspace, device side
  double t_prev;           // t_{k-1}
  double t;                // t_k
  double beta;             // (t_{k-1} - 1) / t_k for the next iteration
  double rel_residual;     // of the last iteration
  double objective;        // of the last iteration (if enabled)
  double tol;
  int64_t k_done;          // iterations completed in this call
  int64_t k_total;         // global iteration counter (resume)
  int32_t done;            // tolerance reached: remaining launches return at once
  int32_t max_sweeps_used;
  int32_t status;          // LT_DEV_* bits of this call
  int32_t pad;
};

struct PgaFuse {
  const void* x_cur = nullptr;      // X^k
  const void* x_old = nullptr;      // X^{k-1}
  void* x_out = nullptr;            // X^{k+1} (may equal x_old)
  const uint8_t* mask = nullptr;
  const void* obs = nullptr;
  double step = 1.0;
  const PgaScalars* scal = nullptr;
  double* partials = nullptr;       // [grid][4]: sum (y-x)^2, sum x^2, sum mask(x-obs)^2
  int objective = 0;
};

struct TransformPass {
  int nm = 0;                         // modes in this pass (application order)
  int msize[kMaxModes] = {};
  int mstride[kMaxModes] = {};        // stride of the mode inside Pg
  int64_t mat_off[kMaxModes] = {};    // element offsets of the matrices to apply
  int64_t Pg = 1, Sg = 1, outer = 1;
  int ts = 32;                        // tile width along Sg
  int smem = 0;                       // bytes
  int tc = 0;                         // 1: single-mode pass on the tensor cores (LT_MIXED)
  int tc_mode = 0;                    // its 0-based mode index
};

struct TransformPlan {
  bool inverse = false;               // matrices from d_inv instead of d_fwd
  int npass = 0;
  TransformPass pass[kMaxModes];
};

// Build the pass plan for slices of S elements, forward (inverse = false) or inverse.
lt_status plan_transform(const Ctx& c, int64_t S, bool inverse, TransformPlan* plan);

// Enqueue the passes.  `fuse` (nullable) applies the PGA prologue on the first pass
// or the epilogue on the last pass.  `grid_out` returns the grid of the last pass
// (number of partial-sum rows written when fusing the epilogue).
cudaError_t launch_transform(const Ctx& c, const TransformPlan& plan, const void* in,
                             void* out, int fuse_mode, const PgaFuse* fuse,
                             cudaStream_t st, int* grid_out);
int transform_grid(const Ctx& c, const TransformPass& p);

// ----------------------------------------------------------------------------------
// Face-wise GEMM (kernel G): C^p = A^p B^p, column-major per slice.
// ----------------------------------------------------------------------------------
cudaError_t launch_facewise_gemm(const Ctx& c, int64_t M, int64_t N, int64_t Kd,
                                 const void* A, const void* B, void* C, cudaStream_t st);

// ----------------------------------------------------------------------------------
// Batched FP32 product on the tcgen05 tensor cores in split TF32 x 3 (lt_tc_gemm.cu):
// D_b = A_b B_b with A_b(m,k) = A[b sA + m + k lda], B_b(k,n) = B[b sB + k + n ldb]
// (sB = 0: shared by every b), D_b(m,n) = D[b sD + m + n ldd].  D may equal A (in
// place) when one tile covers all N <= 256 columns.
// ----------------------------------------------------------------------------------
struct TcGemm {
  int64_t M = 0, N = 0, K = 0, batch = 1;
  const float* A = nullptr;
  int64_t lda = 0, sA = 0;
  const float* B = nullptr;
  int64_t ldb = 0, sB = 0;
  float* D = nullptr;
  int64_t ldd = 0, sD = 0;
  uint64_t wait_ns = 0;    // limit of the kernel's bounded waits (0: the default, 1 s)
  int no_loads = 0;        // test switch: no copies are issued, the waits expire
};

int tc_tile_n(const TcGemm& g, int forced);
// Alignment and size conditions of the TMA descriptors (16-byte aligned A and B, lda,
// ldb and batch strides multiples of 4 elements, sizes below 2^31).
bool tc_gemm_supported(const TcGemm& g, int forced_bn);
cudaError_t launch_tc_gemm(const TcGemm& g, int forced_bn, int32_t* status, cudaStream_t st);

// ----------------------------------------------------------------------------------
// Jacobi SVD / SVT (kernel J), one CTA per slice.
// ----------------------------------------------------------------------------------
// JAC_SVT, JAC_TRUNC and JAC_SIGMA run the QR-preconditioned SVT kernel: shrink by tau,
// keep the trunc_k largest singular triplets, or only write the singular values.
enum JacobiMode { JAC_SVT = 0, JAC_SVD = 1, JAC_TRUNC = 2, JAC_SIGMA = 3 };

struct JacobiPlan {
  int mode = JAC_SVT;
  int64_t I1 = 0, I2 = 0, P = 0;
  int m = 0, n = 0, npad = 0, ld = 0;  // working matrix m x n (m >= n), leading dim
  bool transposed = false;              // working matrix is A^T (I1 < I2)
  bool w_in_smem = true;
  int E = 1;                            // elements per lane per column chunk
  int G = 32;                           // lanes per column pair (SVT kernel)
  int B = 1;                            // columns per register block (SVT kernel)
  int threads = 512;
  int smem = 0;
  size_t ws_bytes = 0;                  // scratch bytes (global W, Jacobi V, info)
  int cluster = 0;                      // > 1: CTAs per slice (cluster form of the SVT)
  int elem = 8;                         // bytes per element
};

struct SliceInfo {          // per slice, written by the Jacobi kernel
  int32_t sweeps;
  int32_t rank;             // singular values above the threshold
  double nuclear;           // sum of the shrunk singular values
};

// count: slices to process (default: the context's P).
lt_status plan_jacobi(const Ctx& c, int mode, int64_t I1, int64_t I2, JacobiPlan* jp,
                      int64_t count = -1);

struct JacobiIO {
  const void* A = nullptr;  // input slices (transform domain)
  void* D = nullptr;        // SVT output (may alias A)
  void* U = nullptr;        // SVD outputs (transform domain)
  void* S = nullptr;
  void* V = nullptr;
  void* sigma = nullptr;    // optional, min(I1,I2) per slice
  double tau = 0.0;         // SVT threshold (host value)
  int64_t trunc_k = 0;      // JAC_TRUNC: singular triplets kept per slice
  const PgaScalars* scal = nullptr;  // PGA: skip when done
  void* scratch = nullptr;  // jp.ws_bytes
  SliceInfo* info = nullptr;
  double* flops = nullptr;  // device counter of executed flops (atomic, per slice)
  double* phases = nullptr; // device: 10 phase cycle counters (profiling), or null
  // SVT kernels, optional (warm start): per slice the n x n orthonormal basis of the
  // orthogonalised side (n = min(I1, I2); column-major, row r in the QR order of the
  // kernel) and the QR permutation (n entries); identity where the slice is rank
  // deficient or did not converge
  void* W = nullptr;
  int* Wperm = nullptr;
};

cudaError_t launch_jacobi(const Ctx& c, const JacobiPlan& jp, const JacobiIO& io,
                          cudaStream_t st);

// ----------------------------------------------------------------------------------
// Warm start (lt_warm.cu): batched products with general element strides,
//   C^p(m, n) = sum_k A^p(m, kk) B^p(k, n),  kk = kperm ? kperm[p K + k] : k,
// A^p(m, k) = A[p sap + m sam + k sak], B^p(k, n) = B[p sbp + k sbk + n sbn],
// C^p(m, n) = C[p scp + m scm + n scn]; and Q^p(perm[r], c) = W^p(r, c).
// ----------------------------------------------------------------------------------
struct StridedGemm {
  int64_t M = 0, N = 0, K = 0, P = 0;
  int64_t sam = 1, sak = 1, sap = 0;
  int64_t sbk = 1, sbn = 1, sbp = 0;
  int64_t scm = 1, scn = 1, scp = 0;
  const int* kperm = nullptr;
};
cudaError_t launch_strided_gemm(const Ctx& c, const StridedGemm& g, const void* A,
                                const void* B, void* C, const PgaScalars* scal,
                                cudaStream_t st);
cudaError_t launch_warm_scatter(const Ctx& c, int64_t n, int64_t P, const void* W,
                                const int* perm, void* Q, const PgaScalars* scal,
                                cudaStream_t st);

// ----------------------------------------------------------------------------------
// PGA bookkeeping kernels
// ----------------------------------------------------------------------------------
cudaError_t launch_pga_init(PgaScalars* scal, double t_prev, double t, int64_t k0,
                            double tol, cudaStream_t st);
cudaError_t launch_pga_finish(PgaScalars* scal, const double* partials, int rows,
                              const SliceInfo* info, int64_t P, double tau, int objective,
                              int32_t* ctx_status, cudaStream_t st);
cudaError_t launch_copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st);
// Norms and ranks from the per-slice singular values sigma (n per slice, context
// precision): out[0] = sum of all sigma, out[1] = max sigma, out[2] = tubal rank,
// out[3] = average rank; multirank[p] (nullable) = count of sigma of slice p above
// max(I1, I2) * u * max sigma.
cudaError_t launch_norms_finish(const void* sigma, int elem, int64_t P, int n, double rank_tol,
                                double* out, int32_t* multirank, cudaStream_t st);
// ----------------------------------------------------------------------------------
// Fourier operator (lt_fourier.cu).  Slots of a mode-3 tube of length n: 0 = DC, then
// (2k-1, 2k) = the real and imaginary parts of the k-th conjugate pair (k = 1..(n-1)/2),
// and n-1 = Nyquist for even n.  Real slots and realified pairs are gathered into
// separate slice sets for the Jacobi SVT and scattered back.
// ----------------------------------------------------------------------------------
struct FourierSlots {
  int64_t n = 0, R = 0;     // tube length, tubes (P / n)
  int64_t nreal = 0;        // real slots: R (odd n) or 2R (even n)
  int64_t npair = 0;        // conjugate pairs: R (n - 1) / 2
};
FourierSlots fourier_slots(const Ctx& c);
// Wr: nreal slices I1 x I2; Wc: npair slices 2 I1 x 2 I2 holding [[a1, -a2], [a2, a1]].
cudaError_t launch_fourier_realify(const Ctx& c, int64_t I1, int64_t I2, const void* G,
                                   void* Wr, void* Wc, const PgaScalars* scal,
                                   cudaStream_t st);
// The real slots from Wr, the pairs from the left block column of Wc.
cudaError_t launch_fourier_derealify(const Ctx& c, int64_t I1, int64_t I2, const void* Wr,
                                     const void* Wc, void* G, const PgaScalars* scal,
                                     cudaStream_t st);
// Orthonormal real DFT basis of length n, row-major n x n doubles (host).
void fourier_basis(int64_t n, double* R);

cudaError_t launch_select_result(const PgaScalars* scal, void* x_user, const void* x_alt,
                                 void* x_prev_out, size_t bytes, cudaStream_t st);

}  // namespace lt
