/*
 * lt.h -- C ABI of liblt, a GB300 (sm_103a) library for the generalized *_L-product,
 * *_L-SVD, *_L-SVT and PGA tensor completion of Bentbib, Elalj, El Hachimi, Jbilou and
 * Ratnani, "Generalized L-product for high order tensors with applications using GPU
 * computations" (arXiv 2202.02870).
 *
 * Conventions shared by every call
 * --------------------------------
 * Tensors.  A K-th order tensor X in R^{I1 x I2 x I3 x ... x IK} (K >= 3) is a dense
 *   buffer in column-major order, mode 1 fastest: element (i1, ..., iK) (0-based) sits
 *   at i1 + I1*(i2 + I2*(i3 + I3*(...))).  The p-th frontal slice ("representative
 *   matrix" X^p, Eq. 3.5) is therefore the contiguous column-major I1 x I2 block at
 *   offset p*I1*I2, p = k3 + I3*k4 + I3*I4*k5 + ...  In torch this is a contiguous
 *   tensor of shape (IK, ..., I3, I2, I1).
 * Element type.  double for LT_FP64 contexts, float for LT_FP32 and LT_MIXED contexts.
 * Pointers.  Tensor arguments are DEVICE pointers owned by the caller; the library
 *   never frees or retains them after the call's work completes.  Host arguments are
 *   marked "host".
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every compute call only enqueues work on it and returns; results are valid after
 *   the stream is synchronised.
 * Workspace.  Calls that need scratch take `ws`, a caller-owned device buffer of at
 *   least `ws_bytes` >= lt_workspace_size(...) bytes, 256-byte aligned.  It must not
 *   be used by anything else until the call's work has completed on `stream`.
 * Errors.  A return value other than LT_OK means that nothing was enqueued (argument,
 *   shape, workspace and launch-configuration errors are detected on the host).
 *   Errors found while kernels run (Jacobi not converged, non-finite values, an
 *   expired bounded wait) are OR-ed into a per-context device status word, read with
 *   lt_last_device_status() after synchronisation; outputs are still written.
 * Threads.  A context may be used from one host thread at a time.
 */
#ifndef LT_H_
#define LT_H_

#include <stddef.h>
#include <stdint.h>

#if defined(_WIN32)
#define LT_API __declspec(dllexport)
#else
#define LT_API __attribute__((visibility("default")))
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LT_OK = 0,
  LT_ERR_ARG = -1,        /* null pointer, negative size, bad option, tau < 0, ... */
  LT_ERR_SHAPE = -2,      /* sizes outside what the kernels support */
  LT_ERR_SINGULAR = -3,   /* a transform matrix is singular or too ill-conditioned */
  LT_ERR_NOCONV = -4,     /* (device) Jacobi hit max_sweeps before converging */
  LT_ERR_TIMEOUT = -5,    /* (device) a bounded wait expired */
  LT_ERR_NONFINITE = -6,  /* (device) NaN or Inf met in a slice */
  LT_ERR_CUDA = -7,       /* a CUDA runtime call failed */
  LT_ERR_WORKSPACE = -8,  /* ws missing, too small or misaligned */
  LT_ERR_UNSUPPORTED = -9 /* the call is not defined for this context's operator
                             (lt_svd, lt_truncate, lt_norms and the PGA objective on a
                             Fourier context) */
} lt_status;

/* Bits of the device status word (lt_last_device_status). */
#define LT_DEV_NOCONV 0x1
#define LT_DEV_NONFINITE 0x2
#define LT_DEV_TIMEOUT 0x4

typedef enum {
  LT_FP64 = 0,  /* every step in IEEE double */
  LT_FP32 = 1,  /* every step in IEEE single (SIMT) */
  LT_MIXED = 2  /* float data; face-wise GEMMs and the mode products of large modes
                   (LT_OPT_TC_MODE_MIN) on the tcgen05 tensor cores as split TF32 x 3
                   products (x = hi + lo, hi = tf32(x), lo = tf32(x - hi);
                   hi hi + hi lo + lo hi accumulated in FP32); the other mode products,
                   the Jacobi SVT and everything else as in LT_FP32.  Operands whose
                   base address is not 16-byte aligned, or slices with I1 or l not a
                   multiple of 4 (face-wise product), take the FP32 SIMT kernels. */
} lt_precision;

typedef enum {
  LT_OP_TRANSFORM = 0,
  LT_OP_INVERSE = 1,
  LT_OP_PRODUCT = 2,
  LT_OP_SVD = 3,
  LT_OP_SVT = 4,
  LT_OP_PGA = 5,
  LT_OP_TRUNCATE = 6,
  LT_OP_NORMS = 7
} lt_op;

typedef enum {
  LT_OPT_MAX_SWEEPS = 0,     /* Jacobi sweep limit (default 40); NOCONV when hit */
  LT_OPT_JACOBI_TOL = 1,     /* pair tolerance: rotate when |a.b| > tol*sqrt(a.a b.b);
                                value <= 0 restores the default: r * unit roundoff for
                                LT_FP64, max(sqrt(r)/8, 4) * unit roundoff otherwise, r = rows of
                                the matrix being orthogonalised (min(I1,I2) for the SVT,
                                which works on the triangular factor of a pivoted QR;
                                max(I1,I2) for the SVD) */
  LT_OPT_OBJECTIVE = 2,      /* PGA: also accumulate the objective (0/1, default 0) */
  LT_OPT_PROFILE = 3,        /* 1: bracket every kernel launch with CUDA events on its
                                stream, summed per kernel family by lt_ctx_get_stats */
  LT_OPT_JACOBI_GROUP = 4,   /* SVT kernel: lanes per column pair (8, 16 or 32); 0 (the
                                default) lets the planner choose from min(I1, I2) */
  LT_OPT_JACOBI_BLOCK = 5,   /* SVT kernel: 1 = rotate column pairs straight through
                                shared memory; 0 (default) = FP32 contexts hold blocks of
                                2 columns per group in registers where they fit (for
                                n <= 144 the wide form of value 3); 2 =
                                FP32 register blocks with the group width forced by
                                LT_OPT_JACOBI_GROUP (8: blocks of 2, n <= 144; 16: blocks
                                of 4 (n <= 144) or 2; 32: blocks of 2); 3 = FP32 wide
                                form for n <= 144: 16-lane groups with blocks of 2, one
                                group per block pair of a round (up to 576 threads) */
  LT_OPT_TC_MODE_MIN = 6,    /* LT_MIXED: a mode k >= 4 with I_k >= this value (default
                                64; modes above 224 never) is applied in a pass of its own
                                on the tensor cores; mode 3 and smaller modes are applied
                                by the SIMT transform kernel (fused passes); 0 = no
                                tensor-core transform passes */
  LT_OPT_TC_TILE_N = 7,      /* LT_MIXED: output tile width of the tensor-core kernel
                                (32, 64, 128 or 256); 0 (default) = chosen per call */
  LT_OPT_MU0 = 8,            /* PGA continuation (Algorithm 5, mu_{k+1} = max(nu mu_k,
                                mu_bar)): mu_0 > 0 turns it on, with mu_bar = the tau
                                argument of lt_pga_complete; iteration k (counted from
                                the start of the run, checkpoints included) thresholds at
                                step * max(nu^k mu_0, tau).  0 (default) = off, fixed tau.
                                Not available in lt_pga_complete_batched (LT_ERR_ARG). */
  LT_OPT_NU = 9,             /* PGA continuation decay nu, 0 < nu <= 1 (default 0.9) */
  LT_OPT_JACOBI_CLUSTER = 10, /* SVT kernel form: 0 = planner's choice (default; FP64:
                                a cluster when the launch's slices leave SMs idle or do
                                not fit one CTA's shared memory, counted as if the launch
                                had the GPU to itself), 1 = one CTA per slice, 3 or 4 = a
                                thread-block cluster of that many CTAs per slice (columns
                                spread over the CTAs' shared memory; slices up to 288
                                columns after padding) */
  LT_OPT_TC_WAIT_US = 11,    /* limit of every bounded wait inside the TMA-fed kernels
                                (the LT_MIXED tensor-core kernel and the FP32 TMA
                                transform passes), in microseconds (0 = default, 1 s;
                                at most 60 s).  On expiry a kernel raises
                                LT_DEV_TIMEOUT, stops issuing work, drains the copies and
                                products it has in flight, frees its TMEM and returns;
                                its output is then undefined. */
  LT_OPT_TC_TEST_NO_LOADS = 12, /* for testing the timeout path only: 1 = the producers
                                of the TMA-fed kernels (tensor-core kernel, TMA transform
                                passes) issue no copies, so the other roles' first waits
                                expire after LT_OPT_TC_WAIT_US and every call that
                                reaches such a kernel reports LT_DEV_TIMEOUT with
                                undefined output; 0 (default) = off */
  LT_OPT_TRANSFORM_TMA = 15, /* FP32 / LT_MIXED mode-product passes outside the PGA
                                loop (lt_transform, lt_inverse, lt_product, lt_svt, ...):
                                1 (default) = tiles move through the tensor memory
                                accelerator (a ring of TMA loads, TMA stores) where the
                                view allows it (16-byte aligned buffers, I1 I2 ... a
                                multiple of 4, at most 256 slices per pass); 0 = the
                                SIMT loads and stores.  The results are identical. */
  LT_OPT_AUTOTUNE = 14,      /* lt_pga_complete and lt_pga_complete_batched (real
                                transforms): 1 = the first call on a slice shape the
                                context was not tuned for times the SVT kernel forms
                                (lt_autotune_svt) on that problem's first-iterate input
                                step * obs at the threshold step * tau and keeps the
                                fastest; the batched call tunes each slice shape once and
                                gives its other contexts of that shape the same forms.
                                Such a call synchronises the stream.  0 (default) = off */
  LT_OPT_WARM_START = 13,    /* lt_pga_complete (real transforms): 0 (default) = every
                                iteration's SVT starts from scratch; p >= 2 = warm start
                                with period p.  Iteration j of a call (j = 0, 1, ...) with
                                j % p == 0 thresholds L(G)^p from scratch and keeps the
                                orthonormal basis Q of the side the Jacobi kernel
                                orthogonalises (left singular vectors when I1 < I2, else
                                right ones); the other iterations threshold Q^T L(G)^p (or
                                L(G)^p Q), which starts near its converged form and takes
                                fewer sweeps, and map the result back (the SVT is
                                unitarily invariant), updating Q.  The cold iterations
                                bound the loss of orthogonality of the accumulated Q.
                                Needs 3 n^2 P elements + n P ints + one tensor more of
                                workspace (n = min(I1, I2); lt_workspace_size with
                                LT_OP_PGA includes them once the option is set).  The
                                batched call and Fourier contexts ignore it. */
} lt_option;

/* Kernel families counted by lt_ctx_get_stats. */
typedef enum { LT_K_TRANSFORM = 0, LT_K_JACOBI = 1, LT_K_GEMM = 2, LT_K_AUX = 3 } lt_kernel;

typedef struct {
  int64_t launches;  /* kernels of the family enqueued */
  double ms;         /* summed CUDA-event durations (LT_OPT_PROFILE on), else 0 */
  double flops;      /* algorithmic floating-point operations: transforms 2 N sum_k I_k
                        per pass set; GEMM 2 M N K P; Jacobi counted by the kernel from
                        the pairs it visited (2m), rotations it applied (6m, + 6n for V),
                        norm passes (2mn) and the SVT reconstruction (4kmn) */
  double bytes;      /* algorithmic DRAM bytes: each tensor read or written once */
} lt_kernel_stats;

typedef struct {
  lt_kernel_stats k[4];
  /* SVT Jacobi kernel, LT_OPT_PROFILE on: SM clock cycles spent per phase, summed over
     slices (measured by one thread of each CTA): [0] loading the slice, [1] pivoted
     QR (all of it), [2] Jacobi sweeps, [3] selecting the singular values above tau,
     [4] their reconstruction coefficients, [5] the reconstruction of the rows; the QR
     split into [6] pivot search, [7] column swap, [8] Householder vector, [9] update of
     the trailing columns. */
  double jacobi_phase_cycles[10];
  int64_t tc_launches;  /* launches of the tcgen05 tensor-core kernel (LT_MIXED), counted
                           among the transform and GEMM launches above */
} lt_stats;

typedef struct lt_ctx_s* lt_ctx;

/* ---------------------------------------------------------------------------------
 * Transform matrices (host helpers; no GPU needed).
 * ------------------------------------------------------------------------------- */

/* Orthonormal DCT-II matrix C_n of Sec. 2 (the matrix C under Eq. (m); "M_i = C_i" in
 * the experiments of Sec. 5), read with delta_{i,1}:
 *   C[i][j] = sqrt((2 - delta_{i,0}) / n) cos(i (2j+1) pi / (2n)),  0 <= i, j < n.
 * M: host, n*n doubles, written ROW-major (M[i*n + j] = C_{ij}).
 * Errors: LT_ERR_ARG if n < 1 or M == NULL. */
LT_API lt_status lt_make_dct(int64_t n, double* M);

/* c-product transform of Eq. (m): M = W^{-1} C (I + Z), W = diag(C(:,1)),
 * Z = superdiagonal ones.  With it on every mode the *_L-product is the generalized
 * c-product ten(btph(A) btph(B)) (Lemma of Sec. 3.1).  Same layout and errors as
 * lt_make_dct. */
LT_API lt_status lt_make_cproduct(int64_t n, double* M);

/* ---------------------------------------------------------------------------------
 * Context: the operator L of Sec. 3.2, L(A) = A x_3 M_3 x_4 ... x_K M_K.
 * ------------------------------------------------------------------------------- */

/* K: tensor order, 3 <= K <= 10.  mode_sizes: host, K-2 entries I3..IK (each >= 1,
 * product P <= 2^31 - 1).  M: host array of K-2 host pointers; M[k] is the
 * I_{k+3} x I_{k+3} matrix M_{k+3}, ROW-major doubles.  The inverses are computed on
 * the host in FP64 (LU with partial pivoting; an orthogonal matrix is inverted
 * exactly by its transpose).  The context owns device copies of M_k and M_k^{-1} (in
 * the context's precision) and a small status block; it owns no data buffers.
 * Errors: LT_ERR_ARG, LT_ERR_SINGULAR (zero pivot or estimated 1-norm condition
 * number > 1e12), LT_ERR_CUDA.  Needs a current CUDA device. */
LT_API lt_status lt_ctx_create(int K, const int64_t* mode_sizes, const double* const* M,
                        lt_precision prec, lt_ctx* out);

/* Context of the Fourier operator: M_3 = F_{I3}, the unnormalised DFT of Sec. 2
 * ((F_n)_{ij} = w^{ij}, w = exp(-2 pi i / n); the t-product for third order), and real
 * M_4..M_K as in lt_ctx_create (M_rest: host array of K-3 host pointers, ROW-major
 * doubles; NULL when K = 3).  Tensors stay real; on the transform side mode 3 holds the
 * coefficients of F_n x in the orthonormal real DFT basis ("slots"), for a tube x of
 * length n and xh = F_n x:
 *   slot 0 = xh_0 / sqrt(n);  slots 2k-1, 2k = sqrt(2/n) (Re xh_k, Im xh_k) for
 *   k = 1..(n-1)/2;  slot n-1 = xh_{n/2} / sqrt(n) for even n
 * (the other half of xh is the conjugate of the first).  On such a context
 *   lt_transform / lt_inverse  map a tensor to its slots and back (then modes 4..K);
 *   lt_product   is A *_L B with M_3 = F: each complex slice product of Algorithm 2;
 *   lt_svt       thresholds the complex slices of L(A) (n-scaled F) at tau, Algorithm 4;
 *   lt_pga_complete  is TNN-PGA-F (Sec. 5) with that SVT; continuation is available,
 *                the objective (LT_OPT_OBJECTIVE) is not (LT_ERR_UNSUPPORTED);
 *   lt_svd, lt_truncate, lt_norms return LT_ERR_UNSUPPORTED.
 * LT_MIXED Fourier contexts run the face-wise products on the FP32 SIMT kernel.
 * Errors: as lt_ctx_create. */
LT_API lt_status lt_ctx_create_fourier(int K, const int64_t* mode_sizes,
                                       const double* const* M_rest, lt_precision prec,
                                       lt_ctx* out);
LT_API lt_status lt_ctx_destroy(lt_ctx ctx);
LT_API lt_status lt_ctx_set_option(lt_ctx ctx, lt_option opt, double value);

/* Bytes of workspace that `op` needs for slices of I1 x I2 (for LT_OP_PRODUCT:
 * A is I1 x I2 and B is I2 x I2b; otherwise I2b is ignored).  out: host. */
LT_API lt_status lt_workspace_size(lt_ctx ctx, lt_op op, int64_t I1, int64_t I2, int64_t I2b,
                            size_t* out);

/* ---------------------------------------------------------------------------------
 * Operations.  Device pointers, column-major (see top of file).
 * ------------------------------------------------------------------------------- */

/* X_hat = L(X) = X x_3 M_3 ... x_K M_K (Sec. 3.2).  X, X_hat: I1*I2*P elements; may
 * alias (in place). */
LT_API lt_status lt_transform(lt_ctx ctx, int64_t I1, int64_t I2, const void* X, void* X_hat,
                       void* ws, size_t ws_bytes, void* stream);

/* X = L^{-1}(X_hat) = X_hat x_K M_K^{-1} ... x_3 M_3^{-1} (Sec. 3.2). */
LT_API lt_status lt_inverse(lt_ctx ctx, int64_t I1, int64_t I2, const void* X_hat, void* X,
                     void* ws, size_t ws_bytes, void* stream);

/* C = A *_L B = L^{-1}(L(A) tri L(B)), Algorithm 2 (Def. of Sec. 3.2): A is
 * I1 x l x I3..IK, B is l x I2 x I3..IK, C is I1 x I2 x I3..IK.  C must not alias
 * A or B. */
LT_API lt_status lt_product(lt_ctx ctx, int64_t I1, int64_t l, int64_t I2, const void* A,
                     const void* B, void* C, void* ws, size_t ws_bytes, void* stream);

/* *_L-SVD, Algorithm 3 (Theorem of Eq. tsvd1): A = U *_L S *_L V^T with U
 * (I1 x I1 x ...), S (I1 x I2 x ...), V (I2 x I2 x ...); every L(U)^p, L(V)^p is
 * orthogonal and L(S)^p = diag(sigma^p), sigma^p descending.  Singular vectors of
 * repeated or zero singular values (and the completion of U or V to a square basis)
 * are not unique.  sigma: optional device buffer of min(I1,I2)*P elements receiving
 * the per-slice singular values (slice-major), may be NULL. */
LT_API lt_status lt_svd(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, void* U, void* S,
                 void* V, void* sigma, void* ws, size_t ws_bytes, void* stream);

/* *_L-SVT D_tau(A), Algorithm 4 (Def. of D_tau, Theorem 23): per transform-domain
 * slice, singular values shrunk to max(sigma - tau, 0), threshold tau applied
 * unscaled in the transform domain.  tau >= 0.  D may alias A. */
LT_API lt_status lt_svt(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, double tau, void* D,
                 void* ws, size_t ws_bytes, void* stream);

/* Rank-k approximation of the Eckart-Young theorem (Sec. 3.2):
 *   A_k = U(:, 1:k, ...) *_L S(1:k, 1:k, ...) *_L V(:, 1:k, ...)^T,
 * i.e. per transform-domain slice the k largest singular triplets of L(A)^p (ties
 * broken by column order; zero singular values are never kept), then L^{-1}.  k >= 0;
 * k >= min(I1, I2) returns A to rounding, k = 0 zeros.  A_k may alias A.  Workspace:
 * lt_workspace_size(LT_OP_TRUNCATE). */
LT_API lt_status lt_truncate(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, int64_t k,
                             void* A_k, void* ws, size_t ws_bytes, void* stream);

/* Norms and ranks of Sec. 3.2 from the singular values sigma_i^p of every slice L(A)^p:
 *   out[0] = sum_p sum_i sigma_i^p   (nuclear norm, Eq. 24 / Theorem 21, without the
 *                                     1/alpha factor: alpha = 1 for orthonormal L)
 *   out[1] = max_p sigma_1^p         (spectral norm ||bdiag(L(A))||, proposition of
 *                                     Sec. 3.2)
 *   out[2] = tubal rank = max_p rho_p (definition of the tubal rank and its lemma)
 *   out[3] = average rank = mean_p rho_p (definition of multirank and average rank)
 *   multirank[p] = rho_p = rank(L(A)^p), nullable
 * A singular value counts as nonzero above max(I1, I2) * u * out[1] (u = 2^-53 for
 * LT_FP64, 2^-24 otherwise).  out: device, 4 doubles; multirank: device, P int32.
 * Workspace: lt_workspace_size(LT_OP_NORMS). */
LT_API lt_status lt_norms(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, double* out,
                          int32_t* multirank, void* ws, size_t ws_bytes, void* stream);

/* Checkpoint of a PGA run (Algorithm 5): X^{k-1} (caller-owned device buffer of the
 * problem's size), t_{k-1}, t_k and k.  With k == 0 the run starts from X^0 = X^1 =
 * the X argument and t_0 = t_1 = 1. */
typedef struct {
  void* X_prev;
  double t_prev;
  double t;
  int64_t k;
} lt_pga_state;

typedef struct {
  int64_t iters_done;     /* iterations performed by this call */
  double rel_residual;    /* ||Y^k - X^{k+1}||_F / ||X^{k+1}||_F of the last one */
  double objective;       /* tau*sum_p ||L(X)^p||_* + 1/2 ||P_Omega(X - M)||^2, if
                             LT_OPT_OBJECTIVE is on, else 0 */
  int32_t max_sweeps_used;
  int32_t device_status;  /* LT_DEV_* bits raised during the call */
} lt_pga_report;

/* Tensor completion by PGA, Algorithm 5 with the Eqs. 50-53 steps and a fixed
 * threshold (no mu continuation):
 *   Y = X^k + ((t_{k-1} - 1)/t_k)(X^k - X^{k-1})            (Eq. 52)
 *   G = Y - step * P_Omega(Y - M)                            (Eq. 51, l_f = 1/step)
 *   X^{k+1} = D_{step*tau}(G)                                (Eq. 53, Algorithm 4)
 *   t_{k+1} = (1 + sqrt(4 t_k^2 + 1)) / 2
 *   r_k = ||Y - X^{k+1}||_F / ||X^{k+1}||_F                  (stopping test of Sec. 5)
 * for `iters` iterations, or fewer when tol > 0 and r_k <= tol.
 * mask: device uint8, I1*I2*P, nonzero = observed (Omega).  obs: device, values of M
 * (entries outside Omega are ignored).  X: device, in = start (X^k; zeros for a cold
 * start), out = the last iterate X^{k+1}.  state: host, may be NULL (cold start and
 * no checkpoint); if given, it is read at the call and, like `report` (host, may be
 * NULL), written once the stream reaches the end of the call's work: both must stay
 * valid until then.  state->X_prev must not alias X. */
LT_API lt_status lt_pga_complete(lt_ctx ctx, int64_t I1, int64_t I2, const uint8_t* mask,
                          const void* obs, double tau, double step, int64_t iters,
                          double tol, void* X, lt_pga_state* state, lt_pga_report* report,
                          void* ws, size_t ws_bytes, void* stream);

/* Many independent completion problems (each with its own context, sizes, mask,
 * observations, tau and step; all contexts of one precision; cold starts, fixed
 * iteration count, no tolerance stop) run together: two iterations of every problem
 * are captured into one CUDA graph with an independent branch per problem, and the
 * graph is replayed iters/2 times (plus one direct iteration when iters is odd), so the
 * GPU runs the kernels of different problems concurrently while every problem keeps the
 * kernel shapes planned for its own sizes.  Results are identical to separate
 * lt_pga_complete calls.  ws: one buffer of at least lt_workspace_size_batched bytes.
 * reports: host array of nprob (may be NULL; requires a distinct context per problem),
 * written when the stream reaches the end of the work. */
LT_API lt_status lt_workspace_size_batched(int nprob, const lt_ctx* ctxs, const int64_t* I1,
                                    const int64_t* I2, size_t* out);
LT_API lt_status lt_pga_complete_batched(int nprob, const lt_ctx* ctxs, const int64_t* I1,
                                  const int64_t* I2, const uint8_t* const* mask,
                                  const void* const* obs, const double* tau,
                                  const double* step, int64_t iters, void* const* X,
                                  lt_pga_report* reports, void* ws, size_t ws_bytes,
                                  void* stream);

/* *_L-product without allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- e.g. an application that
 * reserves all GPU memory for its own pool and forbids further cudaMalloc calls, or code
 * that must not call cudaMalloc/cudaFree because they may synchronise the device --
 * and so cannot pass lt_product a workspace.  It computes exactly what lt_product
 * computes (same kernels; same arguments minus the workspace) with the transform-domain
 * operands L(A) and L(B) placed in a fixed array inside the library's device memory,
 * LT_NOALLOC_SCRATCH_BYTES (32 MiB) large, which every GPU that loads the library's
 * module holds until the process exits.
 * Limits: align256(I1*l*P*elem) + align256(l*I2*P*elem) must not exceed
 *   LT_NOALLOC_SCRATCH_BYTES (align256 rounds up to a multiple of 256), else
 *   LT_ERR_SHAPE and nothing is enqueued (the sizes are multiplied with overflow
 *   checks, so no wrapped product passes).
 * Device: the device current at the call must be the one the context was created on
 *   (LT_ERR_ARG otherwise).
 * Counters: these calls add to lt_stats.tc_launches (their tensor-core launches) but
 *   to no other counter of lt_ctx_get_stats, and LT_OPT_PROFILE does not time them.
 * Set-up: the first call made while a device is current looks up the array's device
 *   address on that device (cudaGetSymbolAddress); make that first call before any
 *   stream capture.
 * Sharing: all calls use the same array and it keeps the last call's contents (nothing
 *   in it needs to start at zero).  Calls whose work overlaps on the GPU race on it:
 *   order them, e.g. issue them on one stream.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
#define LT_NOALLOC_SCRATCH_BYTES (32u << 20)
LT_API lt_status lt_product_noalloc(lt_ctx ctx, int64_t I1, int64_t l, int64_t I2,
                                    const void* A, const void* B, void* C, void* stream);

/* Autotuning.  The kernel forms that are options of a context -- the Jacobi SVT's lanes
 * per column pair and register blocking (LT_OPT_JACOBI_GROUP / LT_OPT_JACOBI_BLOCK) and,
 * for LT_MIXED, the tensor-core tile width (LT_OPT_TC_TILE_N) -- are timed on the
 * caller's data with CUDA events (one warm-up and three timed calls each), and the
 * fastest is set on the context for the calls that follow.  Synchronises `stream`.
 * report: host, may be NULL. */
typedef struct {
  int32_t jacobi_group;     /* chosen values (0 = the planner's default) */
  int32_t jacobi_block;
  int32_t tc_tile_n;
  int32_t candidates;       /* forms timed */
  double best_ms;           /* mean time per call of the chosen form */
  double default_ms;        /* mean time per call of the planner's default form */
} lt_tune_report;

/* Times lt_svt(ctx, I1, I2, A, tau, D, ...) over the SVT kernel forms the slice shape
 * admits (planner default; 8, 16, 32 lanes per pair; register blocks of 2 or 4
 * columns for FP32).  D (not aliasing A) receives the result of the last call.
 * Workspace as lt_svt; forms that would need more workspace are skipped. */
LT_API lt_status lt_autotune_svt(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, double tau,
                                 void* D, void* ws, size_t ws_bytes, void* stream,
                                 lt_tune_report* report);

/* Times lt_product(ctx, I1, l, I2, A, B, C, ...) over the tensor-core tile widths 32,
 * 64, 128 and the default (LT_MIXED contexts; other precisions have one form and
 * report it).  C receives the result of the last call.  Workspace as lt_product. */
LT_API lt_status lt_autotune_product(lt_ctx ctx, int64_t I1, int64_t l, int64_t I2, const void* A,
                                     const void* B, void* C, void* ws, size_t ws_bytes,
                                     void* stream, lt_tune_report* report);

/* Measurement utility (the paper has no counterpart): the FMA throughput of the current
 * GPU for LT_FP64 or LT_FP32, in GFLOP/s (an FMA = 2 flops), measured by a kernel of
 * eight independent multiply-add chains per thread on four 512-thread CTAs per SM, one
 * warm-up and three timed launches on `stream`.  It is the peak against which the ALU
 * rooflines of the Jacobi and transform kernels are stated.  Synchronises `stream`;
 * takes about 0.1 s.  gflops: host.  Errors: LT_ERR_ARG (other precisions, NULL),
 * LT_ERR_CUDA. */
LT_API lt_status lt_measure_fma_peak(lt_precision prec, double* gflops, void* stream);

/* Counters of the context since creation or the last reset (reset != 0 clears them
 * after reading).  Synchronises the device when LT_OPT_PROFILE is on or when Jacobi
 * flops are pending.  out: host. */
LT_API lt_status lt_ctx_get_stats(lt_ctx ctx, lt_stats* out, int reset);

/* Device status word of the context: OR of LT_DEV_* bits raised since the previous
 * call of this function (read and cleared).  Synchronises the device. out: host. */
LT_API lt_status lt_last_device_status(lt_ctx ctx, int32_t* out);

/* Static description of a status code. */
LT_API const char* lt_status_string(lt_status s);

#ifdef __cplusplus
}
#endif
#endif /* LT_H_ */
