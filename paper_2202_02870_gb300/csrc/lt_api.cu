// Host side of the liblt C ABI: argument checks, contexts (the operator L of Sec. 3.2
// with its device-resident matrices), workspace layouts, and the orchestration of the
// kernels for every call.  Nothing here computes on tensor data: every step of
// every operation runs in the kernels of lt_transform.cu, lt_gemm.cu, lt_jacobi.cu and
// lt_pga.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lt_internal.cuh"

using lt::Ctx;

namespace {

constexpr double kPi = 3.14159265358979323846;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

lt_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LT_OK : LT_ERR_CUDA; }

// ---- dense FP64 helpers on the host (transform set-up only) ------------------------
// Inverse by Gaussian elimination with partial pivoting on [M | I]; row-major n x n.
bool invert(const double* M, int64_t n, double* out, double* pivot_min) {
  std::vector<double> a((size_t)n * 2 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < 2 * n; ++j)
      a[i * 2 * n + j] = j < n ? M[i * n + j] : (j - n == i ? 1.0 : 0.0);
  double pmin = INFINITY;
  for (int64_t col = 0; col < n; ++col) {
    int64_t piv = col;
    for (int64_t r = col + 1; r < n; ++r)
      if (std::fabs(a[r * 2 * n + col]) > std::fabs(a[piv * 2 * n + col])) piv = r;
    const double pv = a[piv * 2 * n + col];
    pmin = std::min(pmin, std::fabs(pv));
    if (pv == 0.0 || !std::isfinite(pv)) return false;
    if (piv != col)
      for (int64_t j = 0; j < 2 * n; ++j) std::swap(a[piv * 2 * n + j], a[col * 2 * n + j]);
    const double inv = 1.0 / a[col * 2 * n + col];
    for (int64_t j = 0; j < 2 * n; ++j) a[col * 2 * n + j] *= inv;
    for (int64_t r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[r * 2 * n + col];
      if (f == 0.0) continue;
      for (int64_t j = 0; j < 2 * n; ++j) a[r * 2 * n + j] -= f * a[col * 2 * n + j];
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) out[i * n + j] = a[i * 2 * n + n + j];
  *pivot_min = pmin;
  return true;
}

double norm1(const double* M, int64_t n) {  // max column sum
  double best = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += std::fabs(M[i * n + j]);
    best = std::max(best, s);
  }
  return best;
}

bool is_orthogonal(const double* M, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t k = 0; k < n; ++k) s += M[i * n + k] * M[j * n + k];
      if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 64 * 2.2e-16 * n) return false;
    }
  return true;
}

template <typename T>
void convert(const std::vector<double>& src, std::vector<unsigned char>& dst) {
  dst.resize(src.size() * sizeof(T));
  T* d = reinterpret_cast<T*>(dst.data());
  for (size_t i = 0; i < src.size(); ++i) d[i] = (T)src[i];
}

lt_status check_ctx(lt_ctx c) { return c == nullptr ? LT_ERR_ARG : LT_OK; }

lt_status check_ws(void* ws, size_t have, size_t need) {
  if (need == 0) return LT_OK;
  if (ws == nullptr || have < need) return LT_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LT_ERR_WORKSPACE;
  return LT_OK;
}

lt_status check_dims(int64_t a, int64_t b) {
  if (a < 1 || b < 1) return LT_ERR_ARG;
  if (a > (1 << 20) || b > (1 << 20)) return LT_ERR_SHAPE;
  return LT_OK;
}

// ---- launch accounting (lt_ctx_get_stats) ---------------------------------------------
cudaEvent_t take_event(Ctx& c) {
  if (!c.pool.empty()) {
    cudaEvent_t e = c.pool.back();
    c.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets a group of launches of one kernel family.  Counts launches and algorithmic
// flops/bytes on the host; with LT_OPT_PROFILE records CUDA events on the stream.
struct Scope {
  Ctx& c;
  cudaStream_t st;
  int fam;
  bool account;
  cudaEvent_t a = nullptr;
  Scope(Ctx& ctx, cudaStream_t s, int f, bool acc = true) : c(ctx), st(s), fam(f), account(acc) {
    if (c.profile && account) {
      a = take_event(c);
      cudaEventRecord(a, st);
    }
  }
  void done(int64_t launches, double flops, double bytes) {
    if (!account) return;
    c.stats.k[fam].launches += launches;
    c.stats.k[fam].flops += flops;
    c.stats.k[fam].bytes += bytes;
    if (c.profile && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, st);
      c.pending.push_back({a, b, fam});
      a = nullptr;
    }
  }
};

double transform_flops(const lt::TransformPlan& p, int64_t S, int64_t P) {
  double sum = 0;
  for (int i = 0; i < p.npass; ++i)
    for (int q = 0; q < p.pass[i].nm; ++q) sum += p.pass[i].msize[q];
  return 2.0 * (double)S * (double)P * sum;
}

// One transform call: each pass reads and writes the tensor once.
cudaError_t run_transform(Ctx& c, const lt::TransformPlan& plan, int64_t S, const void* in,
                          void* out, cudaStream_t st) {
  Scope sc(c, st, LT_K_TRANSFORM);
  cudaError_t e = lt::launch_transform(c, plan, in, out, lt::FUSE_NONE, nullptr, st, nullptr);
  sc.done(plan.npass, transform_flops(plan, S, c.P), 2.0 * plan.npass * S * c.P * c.elem);
  return e;
}

cudaError_t run_jacobi(Ctx& c, const lt::JacobiPlan& jp, lt::JacobiIO io, cudaStream_t st,
                       bool account = true) {
  Scope sc(c, st, LT_K_JACOBI, account);
  io.flops = c.d_counters + LT_K_JACOBI;
  io.phases = (c.profile && account) ? c.d_counters + 4 : nullptr;
  cudaError_t e = lt::launch_jacobi(c, jp, io, st);
  const double n = (double)jp.I1 * jp.I2 * jp.P * c.elem;
  // bytes: read the slices (SVT and truncation re-read them for the reconstruction
  // and write the result; the SVD writes its factors; the singular values alone read)
  sc.done(1, 0.0, jp.mode == lt::JAC_SVD ? 2 * n : (jp.mode == lt::JAC_SIGMA ? n : 3 * n));
  return e;
}

// Destroy executable graphs whose launches have completed.
void sweep_retired(Ctx& c) {
  for (size_t i = 0; i < c.retired.size();) {
    if (cudaEventQuery(c.retired[i].done) == cudaSuccess) {
      cudaGraphExecDestroy(c.retired[i].exec);
      cudaEventDestroy(c.retired[i].done);
      c.retired.erase(c.retired.begin() + i);
    } else {
      ++i;
    }
  }
}

// ---- SVT of a Fourier context: real slots and realified pairs (lt_fourier.cu) --------
struct FourierSvt {
  lt::FourierSlots f;
  lt::JacobiPlan jr, jc;              // real slots (I1 x I2), pairs (2 I1 x 2 I2)
  size_t wr = 0, wc = 0, scratch = 0, total = 0;  // offsets in its workspace region
};

lt_status fourier_svt_plan(const Ctx& c, int64_t I1, int64_t I2, FourierSvt* F) {
  F->f = lt::fourier_slots(c);
  lt_status s = lt::plan_jacobi(c, lt::JAC_SVT, I1, I2, &F->jr, F->f.nreal);
  if (s != LT_OK) return s;
  if (F->f.npair > 0 &&
      (s = lt::plan_jacobi(c, lt::JAC_SVT, 2 * I1, 2 * I2, &F->jc, F->f.npair)) != LT_OK)
    return s;
  size_t off = 0;
  F->wr = off; off += align256((size_t)F->f.nreal * I1 * I2 * c.elem);
  F->wc = off; off += align256((size_t)F->f.npair * 4 * I1 * I2 * c.elem);
  F->scratch = off;
  off += align256(std::max(F->jr.ws_bytes, F->f.npair > 0 ? F->jc.ws_bytes : (size_t)0));
  F->total = off;
  return LT_OK;
}

// The SVT of the complex transform-domain slices at tau (Algorithm 4 with M_3 = F), in
// place on the slot tensor G: gather, the Jacobi SVT of the real slots at tau / sqrt(n)
// and of the realified pairs at tau sqrt(2 / n), scatter.  `io` carries the PGA scalars
// and the per-slice info array (real slots first, then pairs); `region` is F.total bytes.
cudaError_t run_fourier_svt(Ctx& c, const FourierSvt& F, int64_t I1, int64_t I2, void* G,
                            double tau, lt::JacobiIO io, void* region, cudaStream_t st,
                            bool account) {
  unsigned char* w = static_cast<unsigned char*>(region);
  void* Wr = w + F.wr;
  void* Wc = w + F.wc;
  const double S = (double)I1 * I2, eb = c.elem, n = (double)F.f.n;
  const double gathered = ((double)F.f.nreal + 4.0 * F.f.npair) * S * eb;
  cudaError_t e;
  {
    Scope sc(c, st, LT_K_AUX, account);
    e = lt::launch_fourier_realify(c, I1, I2, G, Wr, Wc, io.scal, st);
    sc.done(1, 0.0, (double)c.P * S * eb + gathered);
  }
  io.scratch = w + F.scratch;
  lt::SliceInfo* info = io.info;
  if (e == cudaSuccess) {
    io.A = Wr;
    io.D = Wr;
    io.tau = tau / std::sqrt(n);
    e = run_jacobi(c, F.jr, io, st, account);
  }
  if (e == cudaSuccess && F.f.npair > 0) {
    io.A = Wc;
    io.D = Wc;
    io.tau = tau * std::sqrt(2.0 / n);
    io.info = info ? info + F.f.nreal : nullptr;
    e = run_jacobi(c, F.jc, io, st, account);
  }
  if (e == cudaSuccess) {
    Scope sc(c, st, LT_K_AUX, account);
    e = lt::launch_fourier_derealify(c, I1, I2, Wr, Wc, G, io.scal, st);
    sc.done(1, 0.0, 2.0 * (double)c.P * S * eb);
  }
  return e;
}

// ---- workspace layouts ---------------------------------------------------------------
struct PgaLayout {
  size_t x2, ghat, partials, scal, info, jac, total;
  // warm start (LT_OPT_WARM_START): two bases Q (n x n per slice), the kernel's basis W
  // and permutation, and the rotated slices C
  bool warm = false;
  int64_t wn = 0;
  size_t qa = 0, qb = 0, wb = 0, wperm = 0, cbuf = 0;
  lt::TransformPlan fwd, inv;
  lt::JacobiPlan jp;
  FourierSvt fz;                      // Fourier contexts: the SVT's plans and region
  int max_rows;
};

lt_status pga_layout(const Ctx& c, int64_t I1, int64_t I2, PgaLayout* L) {
  const int64_t N = I1 * I2 * c.P;
  lt_status s = lt::plan_transform(c, I1 * I2, false, &L->fwd);
  if (s != LT_OK) return s;
  s = lt::plan_transform(c, I1 * I2, true, &L->inv);
  if (s != LT_OK) return s;
  if (c.fourier_n) {
    if ((s = fourier_svt_plan(c, I1, I2, &L->fz)) != LT_OK) return s;
  } else if ((s = lt::plan_jacobi(c, lt::JAC_SVT, I1, I2, &L->jp)) != LT_OK) {
    return s;
  }
  L->max_rows = lt::transform_grid(c, L->inv.pass[L->inv.npass - 1]);
  size_t off = 0;
  L->x2 = off; off += align256((size_t)N * c.elem);
  L->ghat = off; off += align256((size_t)N * c.elem);
  L->partials = off; off += align256((size_t)L->max_rows * 4 * sizeof(double));
  L->scal = off; off += align256(sizeof(lt::PgaScalars));
  L->info = off; off += align256((size_t)c.P * sizeof(lt::SliceInfo));
  L->jac = off; off += align256(c.fourier_n ? L->fz.total : L->jp.ws_bytes);
  L->warm = c.warm_period >= 2 && !c.fourier_n;
  if (L->warm) {
    const int64_t n = std::min(I1, I2);
    const size_t qbytes = align256((size_t)n * n * c.P * c.elem);
    L->wn = n;
    L->qa = off; off += qbytes;
    L->qb = off; off += qbytes;
    L->wb = off; off += qbytes;
    L->wperm = off; off += align256((size_t)n * c.P * sizeof(int));
    L->cbuf = off; off += align256((size_t)N * c.elem);
  }
  L->total = off;
  return LT_OK;
}

struct ReportJob {
  const lt::PgaScalars* pinned;
  lt_pga_report* rep;
  lt_pga_state* state;
};

void CUDART_CB report_cb(void* p) {
  ReportJob* j = static_cast<ReportJob*>(p);
  const lt::PgaScalars& s = *j->pinned;
  if (j->rep) {
    j->rep->iters_done = s.k_done;
    j->rep->rel_residual = s.rel_residual;
    j->rep->objective = s.objective;
    j->rep->max_sweeps_used = s.max_sweeps_used;
    j->rep->device_status = s.status;
  }
  if (j->state) {
    j->state->t_prev = s.t_prev;
    j->state->t = s.t;
    j->state->k = s.k_total;
  }
  delete j;
}

}  // namespace

extern "C" {

const char* lt_status_string(lt_status s) {
  switch (s) {
    case LT_OK: return "ok";
    case LT_ERR_ARG: return "invalid argument";
    case LT_ERR_SHAPE: return "unsupported shape";
    case LT_ERR_SINGULAR: return "singular or ill-conditioned transform matrix";
    case LT_ERR_NOCONV: return "Jacobi SVD did not converge within max_sweeps";
    case LT_ERR_TIMEOUT: return "bounded device wait expired";
    case LT_ERR_NONFINITE: return "non-finite value";
    case LT_ERR_CUDA: return "CUDA runtime error";
    case LT_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case LT_ERR_UNSUPPORTED: return "operation not available for this context's operator";
  }
  return "unknown status";
}

lt_status lt_make_dct(int64_t n, double* M) {
  if (n < 1 || M == nullptr) return LT_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) {
    const double scale = std::sqrt((i == 0 ? 1.0 : 2.0) / (double)n);
    for (int64_t j = 0; j < n; ++j)
      M[i * n + j] = scale * std::cos((double)i * (2.0 * j + 1.0) * kPi / (2.0 * n));
  }
  return LT_OK;
}

lt_status lt_make_cproduct(int64_t n, double* M) {
  if (n < 1 || M == nullptr) return LT_ERR_ARG;
  std::vector<double> C((size_t)n * n);
  lt_make_dct(n, C.data());
  // M = W^{-1} C (I + Z): column j of C(I+Z) is C(:, j) + C(:, j-1); row i scaled by
  // 1 / C(i, 0).
  for (int64_t i = 0; i < n; ++i) {
    const double w = C[i * n + 0];
    for (int64_t j = 0; j < n; ++j) {
      const double v = C[i * n + j] + (j > 0 ? C[i * n + j - 1] : 0.0);
      M[i * n + j] = v / w;
    }
  }
  return LT_OK;
}

lt_status lt_ctx_create(int K, const int64_t* mode_sizes, const double* const* M,
                        lt_precision prec, lt_ctx* out) {
  if (out == nullptr) return LT_ERR_ARG;
  *out = nullptr;
  if (K < 3 || K - 2 > lt::kMaxModes || mode_sizes == nullptr || M == nullptr) return LT_ERR_ARG;
  if (prec != LT_FP64 && prec != LT_FP32 && prec != LT_MIXED) return LT_ERR_ARG;
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return LT_ERR_ARG;
  c->K = K;
  c->nmodes = K - 2;
  c->prec = prec;
  c->elem = prec == LT_FP64 ? 8 : 4;
  int64_t P = 1;
  std::vector<double> fwd, inv;
  for (int q = 0; q < c->nmodes; ++q) {
    const int64_t n = mode_sizes[q];
    if (n < 1 || n > 4096 || M[q] == nullptr) { delete c; return LT_ERR_ARG; }
    c->sizes[q] = n;
    P *= n;
    if (P > (int64_t)INT32_MAX) { delete c; return LT_ERR_SHAPE; }
    c->mat_off[q] = (int64_t)fwd.size();
    std::vector<double> Mi((size_t)n * n);
    for (int64_t i = 0; i < n * n; ++i) {
      if (!std::isfinite(M[q][i])) { delete c; return LT_ERR_ARG; }
    }
    if (is_orthogonal(M[q], n)) {  // inverse = transpose, exactly
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) Mi[i * n + j] = M[q][j * n + i];
    } else {
      double pmin = 0.0;
      if (!invert(M[q], n, Mi.data(), &pmin)) { delete c; return LT_ERR_SINGULAR; }
      const double cond = norm1(M[q], n) * norm1(Mi.data(), n);
      if (!(cond <= 1e12)) { delete c; return LT_ERR_SINGULAR; }
    }
    fwd.insert(fwd.end(), M[q], M[q] + n * n);
    inv.insert(inv.end(), Mi.begin(), Mi.end());
  }
  c->P = P;
  cudaGetDevice(&c->device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0)
    c->sms = sms;
  std::vector<unsigned char> bf, bi;
  if (c->elem == 8) { convert<double>(fwd, bf); convert<double>(inv, bi); }
  else { convert<float>(fwd, bf); convert<float>(inv, bi); }
  cudaError_t e = cudaMalloc(&c->d_fwd, bf.size());
  if (e == cudaSuccess) e = cudaMalloc(&c->d_inv, bi.size());
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_fwd, bf.data(), bf.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_inv, bi.data(), bi.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, sizeof(lt::PgaScalars));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counters, 14 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, 14 * sizeof(double));
  if (e == cudaSuccess && prec == LT_MIXED) {
    // tensor-core B operands: B(k, n) = M(n, k) at k + n * ld, i.e. each row-major
    // matrix with its rows padded to ld = round_up(I, 4), at 16-byte aligned offsets
    std::vector<float> tf, ti;
    for (int q = 0; q < c->nmodes; ++q) {
      const int64_t n = c->sizes[q], ld = (n + 3) / 4 * 4;
      c->tc_off[q] = (int64_t)tf.size();
      c->tc_ld[q] = (int)ld;
      tf.resize(tf.size() + (size_t)(n * ld), 0.0f);
      ti.resize(ti.size() + (size_t)(n * ld), 0.0f);
      for (int64_t r = 0; r < n; ++r)
        for (int64_t j = 0; j < n; ++j) {
          tf[c->tc_off[q] + r * ld + j] = (float)fwd[c->mat_off[q] + r * n + j];
          ti[c->tc_off[q] + r * ld + j] = (float)inv[c->mat_off[q] + r * n + j];
        }
    }
    e = cudaMalloc(&c->d_tc_fwd, tf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tc_inv, ti.size() * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_tc_fwd, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_tc_inv, ti.data(), ti.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) { lt_ctx_destroy(reinterpret_cast<lt_ctx>(c)); return LT_ERR_CUDA; }
  *out = reinterpret_cast<lt_ctx>(c);
  return LT_OK;
}

lt_status lt_ctx_create_fourier(int K, const int64_t* mode_sizes, const double* const* M_rest,
                                lt_precision prec, lt_ctx* out) {
  if (out == nullptr) return LT_ERR_ARG;
  *out = nullptr;
  if (K < 3 || K - 2 > lt::kMaxModes || mode_sizes == nullptr) return LT_ERR_ARG;
  if (K > 3 && M_rest == nullptr) return LT_ERR_ARG;
  const int64_t n = mode_sizes[0];
  if (n < 1 || n > 4096) return LT_ERR_ARG;
  // mode 3 in the orthonormal real DFT basis, modes 4..K as given
  std::vector<double> R((size_t)(n * n));
  lt::fourier_basis(n, R.data());
  std::vector<const double*> Ms((size_t)(K - 2));
  Ms[0] = R.data();
  for (int q = 1; q < K - 2; ++q) Ms[q] = M_rest[q - 1];
  const lt_status s = lt_ctx_create(K, mode_sizes, Ms.data(), prec, out);
  if (s == LT_OK) reinterpret_cast<Ctx*>(*out)->fourier_n = n;
  return s;
}

lt_status lt_ctx_destroy(lt_ctx ctx) {
  if (!ctx) return LT_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cudaDeviceSynchronize();  // pending work may still read the context's buffers
  if (c->d_fwd) cudaFree(c->d_fwd);
  if (c->d_inv) cudaFree(c->d_inv);
  if (c->d_status) cudaFree(c->d_status);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->d_counters) cudaFree(c->d_counters);
  if (c->d_tc_fwd) cudaFree(c->d_tc_fwd);
  if (c->d_tc_inv) cudaFree(c->d_tc_inv);
  for (auto& r : c->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto& r : c->retired) { cudaGraphExecDestroy(r.exec); cudaEventDestroy(r.done); }
  for (auto ev : c->pool) cudaEventDestroy(ev);
  delete c;
  return LT_OK;
}

lt_status lt_ctx_set_option(lt_ctx ctx, lt_option opt, double value) {
  if (!ctx) return LT_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  switch (opt) {
    case LT_OPT_MAX_SWEEPS:
      if (!(value >= 1 && value <= 1000)) return LT_ERR_ARG;
      c->max_sweeps = (int)value;
      return LT_OK;
    case LT_OPT_JACOBI_TOL:
      if (!(value < 1.0)) return LT_ERR_ARG;
      c->jacobi_tol = value > 0 ? value : 0.0;
      return LT_OK;
    case LT_OPT_OBJECTIVE:
      c->objective = value != 0.0;
      return LT_OK;
    case LT_OPT_PROFILE:
      c->profile = value != 0.0;
      return LT_OK;
    case LT_OPT_JACOBI_BLOCK:
      if (!(value == 0 || value == 1 || value == 2 || value == 3)) return LT_ERR_ARG;
      c->jacobi_pairwise = (int)value;
      return LT_OK;
    case LT_OPT_JACOBI_CLUSTER:
      if (!(value == 0 || value == 1 || value == 3 || value == 4)) return LT_ERR_ARG;
      c->jacobi_cluster = (int)value;
      return LT_OK;
    case LT_OPT_JACOBI_GROUP:
      if (!(value == 0 || value == 8 || value == 16 || value == 32)) return LT_ERR_ARG;
      c->jacobi_group = (int)value;
      return LT_OK;
    case LT_OPT_TC_MODE_MIN:
      if (!(value >= 0 && value <= 4096) || value != std::floor(value)) return LT_ERR_ARG;
      c->tc_mode_min = (int)value;
      return LT_OK;
    case LT_OPT_MU0:
      if (!(value >= 0.0) || !std::isfinite(value)) return LT_ERR_ARG;
      c->mu0 = value;
      return LT_OK;
    case LT_OPT_NU:
      if (!(value > 0.0 && value <= 1.0)) return LT_ERR_ARG;
      c->nu = value;
      return LT_OK;
    case LT_OPT_TRANSFORM_TMA:
      if (!(value == 0 || value == 1)) return LT_ERR_ARG;
      c->transform_tma = (int)value;
      return LT_OK;
    case LT_OPT_AUTOTUNE:
      if (!(value == 0 || value == 1)) return LT_ERR_ARG;
      c->autotune = (int)value;
      return LT_OK;
    case LT_OPT_WARM_START:
      if (!(value == 0 || (value >= 2 && value <= 1e6)) || value != std::floor(value))
        return LT_ERR_ARG;
      c->warm_period = (int)value;
      return LT_OK;
    case LT_OPT_TC_WAIT_US:
      if (!(value >= 0.0 && value <= 60e6)) return LT_ERR_ARG;
      c->tc_wait_us = value;
      return LT_OK;
    case LT_OPT_TC_TEST_NO_LOADS:
      if (!(value == 0 || value == 1)) return LT_ERR_ARG;
      c->tc_no_loads = (int)value;
      return LT_OK;
    case LT_OPT_TC_TILE_N:
      if (!(value == 0 || value == 32 || value == 64 || value == 128 || value == 256))
        return LT_ERR_ARG;
      c->tc_tile_n = (int)value;
      return LT_OK;
  }
  return LT_ERR_ARG;
}

lt_status lt_workspace_size(lt_ctx ctx, lt_op op, int64_t I1, int64_t I2, int64_t I2b,
                            size_t* out) {
  if (!ctx || !out) return LT_ERR_ARG;
  const Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  *out = 0;
  switch (op) {
    case LT_OP_TRANSFORM:
    case LT_OP_INVERSE: {
      lt::TransformPlan p;
      return lt::plan_transform(c, I1 * I2, op == LT_OP_INVERSE, &p);
    }
    case LT_OP_PRODUCT: {
      s = check_dims(I2, I2b);
      if (s != LT_OK) return s;
      *out = align256((size_t)I1 * I2 * c.P * c.elem) + align256((size_t)I2 * I2b * c.P * c.elem);
      return LT_OK;
    }
    case LT_OP_SVD: {
      if (c.fourier_n) return LT_ERR_UNSUPPORTED;
      lt::JacobiPlan jp;
      s = lt::plan_jacobi(c, lt::JAC_SVD, I1, I2, &jp);
      if (s != LT_OK) return s;
      *out = align256((size_t)I1 * I2 * c.P * c.elem) + align256(jp.ws_bytes);
      return LT_OK;
    }
    case LT_OP_SVT: {
      if (c.fourier_n) {
        FourierSvt F;
        if ((s = fourier_svt_plan(c, I1, I2, &F)) != LT_OK) return s;
        *out = F.total;
        return LT_OK;
      }
      lt::JacobiPlan jp;
      s = lt::plan_jacobi(c, lt::JAC_SVT, I1, I2, &jp);
      if (s != LT_OK) return s;
      *out = align256(jp.ws_bytes);
      return LT_OK;
    }
    case LT_OP_TRUNCATE: {
      if (c.fourier_n) return LT_ERR_UNSUPPORTED;
      lt::JacobiPlan jp;
      s = lt::plan_jacobi(c, lt::JAC_TRUNC, I1, I2, &jp);
      if (s != LT_OK) return s;
      *out = align256(jp.ws_bytes);
      return LT_OK;
    }
    case LT_OP_NORMS: {
      if (c.fourier_n) return LT_ERR_UNSUPPORTED;
      lt::JacobiPlan jp;
      s = lt::plan_jacobi(c, lt::JAC_SIGMA, I1, I2, &jp);
      if (s != LT_OK) return s;
      *out = align256((size_t)I1 * I2 * c.P * c.elem) + align256(jp.ws_bytes) +
             align256((size_t)std::min(I1, I2) * c.P * c.elem);
      return LT_OK;
    }
    case LT_OP_PGA: {
      PgaLayout L;
      s = pga_layout(c, I1, I2, &L);
      if (s != LT_OK) return s;
      *out = L.total;
      return LT_OK;
    }
  }
  return LT_ERR_ARG;
}

lt_status lt_transform(lt_ctx ctx, int64_t I1, int64_t I2, const void* X, void* X_hat,
                       void* ws, size_t ws_bytes, void* stream) {
  (void)ws; (void)ws_bytes;
  if (check_ctx(ctx) != LT_OK || !X || !X_hat) return LT_ERR_ARG;
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  lt::TransformPlan plan;
  s = lt::plan_transform(c, I1 * I2, false, &plan);
  if (s != LT_OK) return s;
  return cuda_status(run_transform(c, plan, I1 * I2, X, X_hat, (cudaStream_t)stream));
}

lt_status lt_inverse(lt_ctx ctx, int64_t I1, int64_t I2, const void* X_hat, void* X,
                     void* ws, size_t ws_bytes, void* stream) {
  (void)ws; (void)ws_bytes;
  if (check_ctx(ctx) != LT_OK || !X || !X_hat) return LT_ERR_ARG;
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  lt::TransformPlan plan;
  s = lt::plan_transform(c, I1 * I2, true, &plan);
  if (s != LT_OK) return s;
  return cuda_status(run_transform(c, plan, I1 * I2, X_hat, X, (cudaStream_t)stream));
}

lt_status lt_product(lt_ctx ctx, int64_t I1, int64_t l, int64_t I2, const void* A,
                     const void* B, void* C, void* ws, size_t ws_bytes, void* stream) {
  if (check_ctx(ctx) != LT_OK || !A || !B || !C) return LT_ERR_ARG;
  if (C == A || C == B) return LT_ERR_ARG;
  lt_status s = check_dims(I1, l);
  if (s == LT_OK) s = check_dims(l, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  size_t need = 0;
  s = lt_workspace_size(ctx, LT_OP_PRODUCT, I1, l, I2, &need);
  if (s != LT_OK) return s;
  s = check_ws(ws, ws_bytes, need);
  if (s != LT_OK) return s;
  lt::TransformPlan pa, pb, pc;
  if ((s = lt::plan_transform(c, I1 * l, false, &pa)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, l * I2, false, &pb)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, true, &pc)) != LT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  void* Ah = w;
  void* Bh = w + align256((size_t)I1 * l * c.P * c.elem);
  cudaError_t e = run_transform(c, pa, I1 * l, A, Ah, st);
  if (e == cudaSuccess) e = run_transform(c, pb, l * I2, B, Bh, st);
  if (e == cudaSuccess) {
    Scope sc(c, st, LT_K_GEMM);
    e = lt::launch_facewise_gemm(c, I1, I2, l, Ah, Bh, C, st);
    sc.done(1, 2.0 * I1 * I2 * l * c.P, (double)(I1 * l + l * I2 + I1 * I2) * c.P * c.elem);
  }
  if (e == cudaSuccess) e = run_transform(c, pc, I1 * I2, C, C, st);
  return cuda_status(e);
}

lt_status lt_svd(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, void* U, void* S,
                 void* V, void* sigma, void* ws, size_t ws_bytes, void* stream) {
  if (check_ctx(ctx) != LT_OK || !A || !U || !S || !V) return LT_ERR_ARG;
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  size_t need = 0;
  if ((s = lt_workspace_size(ctx, LT_OP_SVD, I1, I2, 0, &need)) != LT_OK) return s;
  if ((s = check_ws(ws, ws_bytes, need)) != LT_OK) return s;
  lt::JacobiPlan jp;
  lt::TransformPlan pa, pu, ps, pv;
  if ((s = lt::plan_jacobi(c, lt::JAC_SVD, I1, I2, &jp)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, false, &pa)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I1, true, &pu)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, true, &ps)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I2 * I2, true, &pv)) != LT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  void* Ah = w;
  lt::JacobiIO io;
  io.A = Ah;
  io.U = U;
  io.S = S;
  io.V = V;
  io.sigma = sigma;
  io.scratch = w + align256((size_t)I1 * I2 * c.P * c.elem);
  cudaError_t e = run_transform(c, pa, I1 * I2, A, Ah, st);
  if (e == cudaSuccess) e = run_jacobi(c, jp, io, st);
  if (e == cudaSuccess) e = run_transform(c, pu, I1 * I1, U, U, st);
  if (e == cudaSuccess) e = run_transform(c, ps, I1 * I2, S, S, st);
  if (e == cudaSuccess) e = run_transform(c, pv, I2 * I2, V, V, st);
  return cuda_status(e);
}

lt_status lt_svt(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, double tau, void* D,
                 void* ws, size_t ws_bytes, void* stream) {
  if (check_ctx(ctx) != LT_OK || !A || !D) return LT_ERR_ARG;
  if (!(tau >= 0.0) || !std::isfinite(tau)) return LT_ERR_ARG;
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  size_t need = 0;
  if ((s = lt_workspace_size(ctx, LT_OP_SVT, I1, I2, 0, &need)) != LT_OK) return s;
  if ((s = check_ws(ws, ws_bytes, need)) != LT_OK) return s;
  lt::JacobiPlan jp;
  FourierSvt F;
  lt::TransformPlan pf, pi;
  if (c.fourier_n) {
    if ((s = fourier_svt_plan(c, I1, I2, &F)) != LT_OK) return s;
  } else if ((s = lt::plan_jacobi(c, lt::JAC_SVT, I1, I2, &jp)) != LT_OK) {
    return s;
  }
  if ((s = lt::plan_transform(c, I1 * I2, false, &pf)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, true, &pi)) != LT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  lt::JacobiIO io;
  io.A = D;
  io.D = D;
  io.tau = tau;
  io.scratch = ws;
  cudaError_t e = run_transform(c, pf, I1 * I2, A, D, st);
  if (e == cudaSuccess)
    e = c.fourier_n ? run_fourier_svt(c, F, I1, I2, D, tau, io, ws, st, true)
                    : run_jacobi(c, jp, io, st);
  if (e == cudaSuccess) e = run_transform(c, pi, I1 * I2, D, D, st);
  return cuda_status(e);
}

lt_status lt_truncate(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, int64_t k, void* A_k,
                      void* ws, size_t ws_bytes, void* stream) {
  if (check_ctx(ctx) != LT_OK || !A || !A_k || k < 0) return LT_ERR_ARG;
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  size_t need = 0;
  if ((s = lt_workspace_size(ctx, LT_OP_TRUNCATE, I1, I2, 0, &need)) != LT_OK) return s;
  if ((s = check_ws(ws, ws_bytes, need)) != LT_OK) return s;
  lt::JacobiPlan jp;
  lt::TransformPlan pf, pi;
  if ((s = lt::plan_jacobi(c, lt::JAC_TRUNC, I1, I2, &jp)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, false, &pf)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, true, &pi)) != LT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  lt::JacobiIO io;
  io.A = A_k;
  io.D = A_k;
  io.trunc_k = k;
  io.scratch = ws;
  cudaError_t e = run_transform(c, pf, I1 * I2, A, A_k, st);
  if (e == cudaSuccess) e = run_jacobi(c, jp, io, st);
  if (e == cudaSuccess) e = run_transform(c, pi, I1 * I2, A_k, A_k, st);
  return cuda_status(e);
}

lt_status lt_norms(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, double* out,
                   int32_t* multirank, void* ws, size_t ws_bytes, void* stream) {
  if (check_ctx(ctx) != LT_OK || !A || !out) return LT_ERR_ARG;
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  size_t need = 0;
  if ((s = lt_workspace_size(ctx, LT_OP_NORMS, I1, I2, 0, &need)) != LT_OK) return s;
  if ((s = check_ws(ws, ws_bytes, need)) != LT_OK) return s;
  lt::JacobiPlan jp;
  lt::TransformPlan pf;
  if ((s = lt::plan_jacobi(c, lt::JAC_SIGMA, I1, I2, &jp)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, false, &pf)) != LT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* w = static_cast<unsigned char*>(ws);
  void* Ah = w;
  void* scratch = w + align256((size_t)I1 * I2 * c.P * c.elem);
  void* sigma = static_cast<unsigned char*>(scratch) + align256(jp.ws_bytes);
  lt::JacobiIO io;
  io.A = Ah;
  io.D = nullptr;
  io.sigma = sigma;
  io.scratch = scratch;
  cudaError_t e = run_transform(c, pf, I1 * I2, A, Ah, st);
  if (e == cudaSuccess) e = run_jacobi(c, jp, io, st);
  if (e == cudaSuccess) {
    Scope sc(c, st, LT_K_AUX);
    const double u = c.elem == 8 ? 0x1p-53 : 0x1p-24;
    e = lt::launch_norms_finish(sigma, c.elem, c.P, (int)std::min(I1, I2),
                                (double)std::max(I1, I2) * u, out, multirank, st);
    sc.done(1, 0.0, (double)std::min(I1, I2) * c.P * c.elem);
  }
  return cuda_status(e);
}

}  // extern "C"

namespace {

// One PGA run (Algorithm 5) split into enqueue steps, so that a batch of runs can be
// captured into one CUDA graph with a branch per problem.
struct PgaRun {
  Ctx* c;
  PgaLayout L;
  int64_t I1, I2;
  double tau, step;
  size_t bytes;
  void* X;
  void* X2;
  void* Gh;
  lt::PgaScalars* scal;
  lt::PgaFuse f;
  lt::JacobiIO io;
  double fwd_bytes, inv_bytes, fwd_flops, inv_flops;
  int rows;
  // warm start: buffers (null when off) and which basis is current
  void* Q[2] = {nullptr, nullptr};
  void* Wb = nullptr;
  int* Wperm = nullptr;
  void* Cb = nullptr;
  int qcur = 0;
};

lt_status pga_prepare(Ctx& c, int64_t I1, int64_t I2, const uint8_t* mask, const void* obs,
                      double tau, double step, void* X, void* ws, size_t ws_bytes,
                      PgaRun* r) {
  lt_status s = check_dims(I1, I2);
  if (s != LT_OK) return s;
  if (c.fourier_n && c.objective) return LT_ERR_UNSUPPORTED;
  if ((s = pga_layout(c, I1, I2, &r->L)) != LT_OK) return s;
  if ((s = check_ws(ws, ws_bytes, r->L.total)) != LT_OK) return s;
  unsigned char* w = static_cast<unsigned char*>(ws);
  r->c = &c;
  r->I1 = I1;
  r->I2 = I2;
  r->tau = tau;
  r->step = step;
  r->bytes = (size_t)I1 * I2 * c.P * c.elem;
  r->X = X;
  r->X2 = w + r->L.x2;
  r->Gh = w + r->L.ghat;
  r->scal = reinterpret_cast<lt::PgaScalars*>(w + r->L.scal);
  r->f = lt::PgaFuse();
  r->f.mask = mask;
  r->f.obs = obs;
  r->f.step = step;
  r->f.scal = r->scal;
  r->f.partials = reinterpret_cast<double*>(w + r->L.partials);
  r->f.objective = c.objective;
  r->io = lt::JacobiIO();
  r->io.A = r->Gh;
  r->io.D = r->Gh;
  r->io.tau = step * tau;
  r->io.scal = r->scal;
  r->io.scratch = w + r->L.jac;
  r->io.info = reinterpret_cast<lt::SliceInfo*>(w + r->L.info);
  // algorithmic traffic of the fused transforms: forward reads X, X_old, obs, mask and
  // writes G_hat; inverse reads D_hat, X, X_old (+ mask, obs for the objective) and
  // writes X_new; intermediate passes read and write the tensor once more each
  const double Nd = (double)I1 * I2 * c.P, eb = (double)c.elem;
  r->fwd_bytes = Nd * (4 * eb + 1) + (r->L.fwd.npass - 1) * 2 * Nd * eb;
  r->inv_bytes = Nd * (4 * eb + (c.objective ? eb + 1 : 0)) + (r->L.inv.npass - 1) * 2 * Nd * eb;
  r->fwd_flops = transform_flops(r->L.fwd, I1 * I2, c.P) + 6 * Nd;
  r->inv_flops = transform_flops(r->L.inv, I1 * I2, c.P) + 7 * Nd;
  r->rows = r->L.max_rows;
  if (r->L.warm) {
    r->Q[0] = w + r->L.qa;
    r->Q[1] = w + r->L.qb;
    r->Wb = w + r->L.wb;
    r->Wperm = reinterpret_cast<int*>(w + r->L.wperm);
    r->Cb = w + r->L.cbuf;
  }
  return LT_OK;
}

// X^0 = X^1 = X (or the checkpoint), scalars t_0, t_1.
cudaError_t pga_begin(PgaRun& r, const lt_pga_state* state, double tol, cudaStream_t st) {
  const bool resume = state && state->k > 0;
  Scope sc(*r.c, st, LT_K_AUX);
  cudaError_t e = lt::launch_copy_bytes(r.X2, resume ? state->X_prev : r.X, r.bytes, st);
  if (e == cudaSuccess)
    e = lt::launch_pga_init(r.scal, resume ? state->t_prev : 1.0, resume ? state->t : 1.0,
                            resume ? state->k : 0, tol, st);
  sc.done(2, 0.0, 2.0 * r.bytes);
  return e;
}

// The SVT step of a warm-started iteration (LT_OPT_WARM_START): with Q the basis of the
// previous iteration (n = min(I1, I2), n x n per slice) the Jacobi kernel thresholds
// C = Q^T G_hat (I1 < I2: the kernel orthogonalises the columns of the transposed slice)
// or C = G_hat Q, the result goes back as D_hat = Q D_tau(C) or D_tau(C) Q^T (the SVT is
// unitarily invariant), and the next basis is Q P W from the kernel's basis W and QR
// permutation P.  A cold iteration thresholds G_hat itself and starts the basis as P W.
cudaError_t warm_svt(PgaRun& r, bool cold, cudaStream_t st, bool account) {
  Ctx& c = *r.c;
  const int64_t I1 = r.I1, I2 = r.I2, n = r.L.wn, P = c.P;
  const bool tr = I1 < I2;
  const double eb = c.elem;
  lt::JacobiIO io = r.io;
  io.W = r.Wb;
  io.Wperm = r.Wperm;
  void* Q = r.Q[r.qcur];
  void* Qn = r.Q[1 - r.qcur];
  cudaError_t e = cudaSuccess;
  const double slice_flops = 2.0 * (double)I1 * I2 * n * P;
  const double slice_bytes = (2.0 * I1 * I2 + (double)n * n) * P * eb;
  if (!cold) {
    lt::StridedGemm g;  // C = Q^T G_hat or G_hat Q
    g.P = P; g.M = I1; g.N = I2; g.K = n;
    g.scm = 1; g.scn = I1; g.scp = I1 * I2;
    const void *A, *B;
    if (tr) {
      A = Q; g.sam = n; g.sak = 1; g.sap = n * n;
      B = r.Gh; g.sbk = 1; g.sbn = I1; g.sbp = I1 * I2;
    } else {
      A = r.Gh; g.sam = 1; g.sak = I1; g.sap = I1 * I2;
      B = Q; g.sbk = 1; g.sbn = n; g.sbp = n * n;
    }
    Scope sc(c, st, LT_K_GEMM, account);
    e = lt::launch_strided_gemm(c, g, A, B, r.Cb, r.scal, st);
    sc.done(1, slice_flops, slice_bytes);
    io.A = r.Cb;
    io.D = r.Cb;
  }
  if (e == cudaSuccess) e = run_jacobi(c, r.L.jp, io, st, account);
  if (e == cudaSuccess && !cold) {
    lt::StridedGemm g;  // D_hat = Q D_tau(C) or D_tau(C) Q^T, into G_hat
    g.P = P; g.M = I1; g.N = I2; g.K = n;
    g.scm = 1; g.scn = I1; g.scp = I1 * I2;
    const void *A, *B;
    if (tr) {
      A = Q; g.sam = 1; g.sak = n; g.sap = n * n;
      B = r.Cb; g.sbk = 1; g.sbn = I1; g.sbp = I1 * I2;
    } else {
      A = r.Cb; g.sam = 1; g.sak = I1; g.sap = I1 * I2;
      B = Q; g.sbk = n; g.sbn = 1; g.sbp = n * n;
    }
    Scope sc(c, st, LT_K_GEMM, account);
    e = lt::launch_strided_gemm(c, g, A, B, r.Gh, r.scal, st);
    sc.done(1, slice_flops, slice_bytes);
  }
  if (e == cudaSuccess) {
    if (cold) {
      Scope sc(c, st, LT_K_AUX, account);
      e = lt::launch_warm_scatter(c, n, P, r.Wb, r.Wperm, Qn, r.scal, st);
      sc.done(1, 0.0, 2.0 * (double)n * n * P * eb);
    } else {
      lt::StridedGemm g;  // next basis Q P W
      g.P = P; g.M = n; g.N = n; g.K = n;
      g.sam = 1; g.sak = n; g.sap = n * n; g.kperm = r.Wperm;
      g.sbk = 1; g.sbn = n; g.sbp = n * n;
      g.scm = 1; g.scn = n; g.scp = n * n;
      Scope sc(c, st, LT_K_GEMM, account);
      e = lt::launch_strided_gemm(c, g, Q, r.Wb, Qn, r.scal, st);
      sc.done(1, 2.0 * (double)n * n * n * P, 3.0 * (double)n * n * P * eb);
    }
    r.qcur = 1 - r.qcur;
  }
  return e;
}

// Iteration j of the run: fused forward transform, Jacobi SVT, fused inverse transform,
// scalar update.  allow_warm: the warm start may be used (not in captured batches).  `account` is false while the launches are being captured into a graph
// (they are then counted per replay).
cudaError_t pga_iteration(PgaRun& r, int64_t j, cudaStream_t st, bool account,
                          bool allow_warm = false) {
  Ctx& c = *r.c;
  const bool warm = allow_warm && r.L.warm;
  void* cur = (j % 2 == 0) ? r.X : r.X2;
  void* old = (j % 2 == 0) ? r.X2 : r.X;
  r.f.x_cur = cur;
  r.f.x_old = old;
  r.f.x_out = old;
  int rows = 0;
  cudaError_t e;
  {
    Scope sc(c, st, LT_K_TRANSFORM, account);
    e = lt::launch_transform(c, r.L.fwd, nullptr, r.Gh, lt::FUSE_PGA_FORWARD, &r.f, st, nullptr);
    sc.done(r.L.fwd.npass, r.fwd_flops, r.fwd_bytes);
  }
  if (e == cudaSuccess)
    e = c.fourier_n ? run_fourier_svt(c, r.L.fz, r.I1, r.I2, r.Gh, r.io.tau, r.io, r.io.scratch,
                                      st, account)
        : warm      ? warm_svt(r, j % c.warm_period == 0, st, account)
                    : run_jacobi(c, r.L.jp, r.io, st, account);
  if (e == cudaSuccess) {
    Scope sc(c, st, LT_K_TRANSFORM, account);
    e = lt::launch_transform(c, r.L.inv, r.Gh, r.Gh, lt::FUSE_PGA_INVERSE, &r.f, st, &rows);
    sc.done(r.L.inv.npass, r.inv_flops, r.inv_bytes);
  }
  if (e == cudaSuccess) {
    Scope sc(c, st, LT_K_AUX, account);
    const int64_t slices = c.fourier_n ? r.L.fz.f.nreal + r.L.fz.f.npair : c.P;
    e = lt::launch_pga_finish(r.scal, r.f.partials, rows, r.io.info, slices, r.tau, c.objective,
                              c.d_status, st);
    sc.done(1, 0.0, 0.0);
  }
  return e;
}

// Host-side counts of one replayed iteration (graph launches bypass Scope).
void pga_account_iteration(PgaRun& r) {
  Ctx& c = *r.c;
  c.stats.k[LT_K_TRANSFORM].launches += r.L.fwd.npass + r.L.inv.npass;
  c.stats.k[LT_K_TRANSFORM].flops += r.fwd_flops + r.inv_flops;
  c.stats.k[LT_K_TRANSFORM].bytes += r.fwd_bytes + r.inv_bytes;
  const double S = (double)r.I1 * r.I2 * c.elem;
  if (c.fourier_n) {
    const lt::FourierSlots& f = r.L.fz.f;
    c.stats.k[LT_K_JACOBI].launches += 1 + (f.npair > 0);
    c.stats.k[LT_K_JACOBI].bytes += 3.0 * ((double)f.nreal + 4.0 * f.npair) * S;
    c.stats.k[LT_K_AUX].launches += 3;
    c.stats.k[LT_K_AUX].bytes += 3.0 * (double)c.P * S + ((double)f.nreal + 4.0 * f.npair) * S;
  } else {
    c.stats.k[LT_K_JACOBI].launches += 1;
    c.stats.k[LT_K_JACOBI].bytes += 3.0 * (double)c.P * S;
    c.stats.k[LT_K_AUX].launches += 1;
  }
}

cudaError_t pga_end(PgaRun& r, lt_pga_state* state, lt_pga_report* report, cudaStream_t st) {
  cudaError_t e;
  {
    Scope sc(*r.c, st, LT_K_AUX);
    e = lt::launch_select_result(r.scal, r.X, r.X2, state ? state->X_prev : nullptr, r.bytes, st);
    sc.done(1, 0.0, 3.0 * r.bytes);
  }
  if (e == cudaSuccess && (report || state)) {
    e = cudaMemcpyAsync(r.c->h_pinned, r.scal, sizeof(lt::PgaScalars), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) {
      ReportJob* job = new ReportJob{static_cast<const lt::PgaScalars*>(r.c->h_pinned), report, state};
      e = cudaLaunchHostFunc(st, report_cb, job);
      if (e != cudaSuccess) delete job;
    }
  }
  return e;
}

// LT_OPT_AUTOTUNE: the SVT kernel forms are timed (lt_autotune_svt) on the first
// iterate's thresholding input, step * obs (X^0 = 0 makes G = step P_Omega(M)), at the
// threshold step * tau, with the run's G_hat region as output and its Jacobi region as
// workspace (forms needing more are skipped); the fastest stays set on the context, which
// remembers the slice shape.  Synchronises the stream.  The run is then re-planned (the
// chosen form needs no more workspace than the region it was timed in).
lt_status pga_autotune(lt_ctx h, PgaRun& r, const uint8_t* mask, const void* obs, double tau,
                       double step, void* X, void* ws, size_t ws_bytes, cudaStream_t st) {
  Ctx& c = *r.c;
  lt_tune_report rep;
  const lt_status s = lt_autotune_svt(h, r.I1, r.I2, obs, step * tau, r.Gh, r.io.scratch,
                                      align256(r.L.jp.ws_bytes), st, &rep);
  if (s == LT_ERR_CUDA) return s;  // otherwise (no form fitted) the options stay as they were
  c.tuned_I1 = r.I1;
  c.tuned_I2 = r.I2;
  return pga_prepare(c, r.I1, r.I2, mask, obs, tau, step, X, ws, ws_bytes, &r);
}

}  // namespace

extern "C" {

lt_status lt_pga_complete(lt_ctx ctx, int64_t I1, int64_t I2, const uint8_t* mask,
                          const void* obs, double tau, double step, int64_t iters,
                          double tol, void* X, lt_pga_state* state, lt_pga_report* report,
                          void* ws, size_t ws_bytes, void* stream) {
  if (check_ctx(ctx) != LT_OK || !mask || !obs || !X) return LT_ERR_ARG;
  if (!(tau >= 0.0) || !std::isfinite(tau) || !(step > 0.0) || !std::isfinite(step)) return LT_ERR_ARG;
  if (iters < 0 || !(tol >= 0.0)) return LT_ERR_ARG;
  if (state && (state->X_prev == nullptr || state->X_prev == X || state->k < 0)) return LT_ERR_ARG;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  PgaRun r;
  lt_status s = pga_prepare(c, I1, I2, mask, obs, tau, step, X, ws, ws_bytes, &r);
  if (s != LT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (c.autotune && !c.fourier_n && (c.tuned_I1 != I1 || c.tuned_I2 != I2) &&
      (s = pga_autotune(ctx, r, mask, obs, tau, step, X, ws, ws_bytes, st)) != LT_OK)
    return s;
  cudaError_t e = pga_begin(r, state, tol, st);
  const int64_t k0 = (state && state->k > 0) ? state->k : 0;
  for (int64_t j = 0; j < iters && e == cudaSuccess; ++j) {
    // continuation (Algorithm 5, mu_{k+1} = max(nu mu_k, mu_bar) with mu_bar = tau):
    // iteration k thresholds at step * max(nu^k mu_0, tau); off (mu_0 = 0): step * tau
    if (c.mu0 > 0.0) r.io.tau = step * std::max(std::pow(c.nu, (double)(k0 + j)) * c.mu0, tau);
    e = pga_iteration(r, j, st, true, true);
  }
  if (e == cudaSuccess) e = pga_end(r, state, report, st);
  return cuda_status(e);
}

lt_status lt_workspace_size_batched(int nprob, const lt_ctx* ctxs, const int64_t* I1,
                                    const int64_t* I2, size_t* out) {
  if (nprob < 1 || !ctxs || !I1 || !I2 || !out) return LT_ERR_ARG;
  size_t total = 0;
  for (int i = 0; i < nprob; ++i) {
    size_t b = 0;
    lt_status s = lt_workspace_size(ctxs[i], LT_OP_PGA, I1[i], I2[i], 0, &b);
    if (s != LT_OK) return s;
    total += align256(b);
  }
  *out = total;
  return LT_OK;
}

lt_status lt_pga_complete_batched(int nprob, const lt_ctx* ctxs, const int64_t* I1,
                                  const int64_t* I2, const uint8_t* const* mask,
                                  const void* const* obs, const double* tau,
                                  const double* step, int64_t iters, void* const* X,
                                  lt_pga_report* reports, void* ws, size_t ws_bytes,
                                  void* stream) {
  if (nprob < 1 || !ctxs || !I1 || !I2 || !mask || !obs || !tau || !step || !X) return LT_ERR_ARG;
  if (iters < 0) return LT_ERR_ARG;
  size_t need = 0;
  lt_status s = lt_workspace_size_batched(nprob, ctxs, I1, I2, &need);
  if (s != LT_OK) return s;
  if ((s = check_ws(ws, ws_bytes, need)) != LT_OK) return s;
  for (int i = 0; i < nprob; ++i) {
    if (!ctxs[i] || !mask[i] || !obs[i] || !X[i]) return LT_ERR_ARG;
    if (!(tau[i] >= 0.0) || !std::isfinite(tau[i]) || !(step[i] > 0.0) || !std::isfinite(step[i]))
      return LT_ERR_ARG;
    if (reinterpret_cast<Ctx*>(ctxs[i])->mu0 > 0.0) return LT_ERR_ARG;  // one graph, fixed tau
    if (reinterpret_cast<Ctx*>(ctxs[i])->prec != reinterpret_cast<Ctx*>(ctxs[0])->prec)
      return LT_ERR_ARG;
    for (int j = 0; j < i; ++j)  // one context per problem: report staging is per context
      if (ctxs[j] == ctxs[i] && reports) return LT_ERR_ARG;
  }
  std::vector<PgaRun> runs(nprob);
  unsigned char* w = static_cast<unsigned char*>(ws);
  size_t off = 0;
  for (int i = 0; i < nprob; ++i) {
    size_t b = 0;
    lt_workspace_size(ctxs[i], LT_OP_PGA, I1[i], I2[i], 0, &b);
    s = pga_prepare(*reinterpret_cast<Ctx*>(ctxs[i]), I1[i], I2[i], mask[i], obs[i], tau[i],
                    step[i], X[i], w + off, align256(b), &runs[i]);
    if (s != LT_OK) return s;
    off += align256(b);
  }
  cudaStream_t st = (cudaStream_t)stream;
  Ctx& c0 = *reinterpret_cast<Ctx*>(ctxs[0]);
  // LT_OPT_AUTOTUNE: once per slice shape in the batch; contexts of a shape tuned here
  // take the same forms
  off = 0;
  for (int i = 0; i < nprob; ++i) {
    Ctx& ci = *reinterpret_cast<Ctx*>(ctxs[i]);
    size_t b = 0;
    lt_workspace_size(ctxs[i], LT_OP_PGA, I1[i], I2[i], 0, &b);
    if (ci.autotune && !ci.fourier_n && (ci.tuned_I1 != I1[i] || ci.tuned_I2 != I2[i])) {
      int from = -1;
      for (int j = 0; j < i && from < 0; ++j) {
        const Ctx& cj = *reinterpret_cast<Ctx*>(ctxs[j]);
        if (I1[j] == I1[i] && I2[j] == I2[i] && cj.tuned_I1 == I1[i] && cj.tuned_I2 == I2[i])
          from = j;
      }
      if (from >= 0) {
        const Ctx& cj = *reinterpret_cast<Ctx*>(ctxs[from]);
        ci.jacobi_group = cj.jacobi_group;
        ci.jacobi_pairwise = cj.jacobi_pairwise;
        ci.tuned_I1 = I1[i];
        ci.tuned_I2 = I2[i];
        s = pga_prepare(ci, I1[i], I2[i], mask[i], obs[i], tau[i], step[i], X[i], w + off,
                        align256(b), &runs[i]);
      } else {
        s = pga_autotune(ctxs[i], runs[i], mask[i], obs[i], tau[i], step[i], X[i], w + off,
                         align256(b), st);
      }
      if (s != LT_OK) return s;
    }
    off += align256(b);
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nprob && e == cudaSuccess; ++i) e = pga_begin(runs[i], nullptr, 0.0, st);

  // Capture two iterations of every problem as independent branches of one graph (two,
  // so that the ping-pong buffers are back in place at the end of each replay), then
  // replay it; the GPU runs the branches of different problems concurrently.
  const int64_t pairs = iters / 2;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && pairs > 0) {
    const int ns = std::min(nprob, 32);
    std::vector<cudaStream_t> cs(ns, nullptr);
    std::vector<cudaEvent_t> ev(nprob + 1, nullptr);
    for (int i = 0; i < ns && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&cs[i], cudaStreamNonBlocking);
    for (int i = 0; i <= nprob && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t ce = cudaEventRecord(ev[nprob], cs[0]);  // fork point
      for (int i = 0; i < nprob && ce == cudaSuccess; ++i) {
        cudaStream_t si = cs[i % ns];
        if (i % ns != 0) ce = cudaStreamWaitEvent(si, ev[nprob], 0);
        for (int64_t j = 0; j < 2 && ce == cudaSuccess; ++j) ce = pga_iteration(runs[i], j, si, false);
        if (ce == cudaSuccess) ce = cudaEventRecord(ev[i], si);
      }
      for (int i = 0; i < nprob && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(cs[0], ev[i], 0);  // join
      e = cudaStreamEndCapture(cs[0], &graph);
      if (e == cudaSuccess) e = ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (auto x : cs) if (x) cudaStreamDestroy(x);
    for (auto x : ev) if (x) cudaEventDestroy(x);
    for (int64_t p = 0; p < pairs && e == cudaSuccess; ++p) {
      e = cudaGraphLaunch(exec, st);
      for (int i = 0; i < nprob; ++i) {
        pga_account_iteration(runs[i]);
        pga_account_iteration(runs[i]);
      }
    }
  }
  if (e == cudaSuccess && (iters % 2))  // an odd last iteration, directly
    for (int i = 0; i < nprob && e == cudaSuccess; ++i) e = pga_iteration(runs[i], iters - 1, st, true);
  for (int i = 0; i < nprob && e == cudaSuccess; ++i)
    e = pga_end(runs[i], nullptr, reports ? &reports[i] : nullptr, st);
  if (exec) {
    // destroy the executable graph once its launches have completed: retire it behind an
    // event and sweep the retired ones whose event has fired
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(done, st) == cudaSuccess) {
      c0.retired.push_back({exec, done});
    } else {
      cudaStreamSynchronize(st);
      cudaGraphExecDestroy(exec);
      if (done) cudaEventDestroy(done);
    }
  }
  sweep_retired(c0);
  return cuda_status(e);
}

}  // extern "C"

namespace {

// Mean CUDA-event time of `run` (one warm-up, three timed calls); +inf when a call
// fails to enqueue.
template <typename F>
double time_calls(cudaStream_t st, F run) {
  if (run() != LT_OK) return INFINITY;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return INFINITY;
  cudaEventRecord(a, st);
  lt_status s = LT_OK;
  for (int i = 0; i < 3 && s == LT_OK; ++i) s = run();
  cudaEventRecord(b, st);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (ok && s == LT_OK) ? ms / 3.0 : INFINITY;
}

}  // namespace

extern "C" {

lt_status lt_autotune_svt(lt_ctx ctx, int64_t I1, int64_t I2, const void* A, double tau,
                          void* D, void* ws, size_t ws_bytes, void* stream,
                          lt_tune_report* report) {
  if (check_ctx(ctx) != LT_OK || !A || !D || D == A) return LT_ERR_ARG;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  const int keep_g = c.jacobi_group, keep_b = c.jacobi_pairwise;
  struct Form { int g, b; };
  std::vector<Form> forms = {{0, 0}, {8, 1}, {16, 1}, {32, 1}};
  if (c.elem == 4) forms.insert(forms.end(), {{8, 2}, {16, 2}, {32, 2}, {16, 3}});
  double best = INFINITY, dflt = INFINITY;
  Form pick = {keep_g, keep_b};
  int timed = 0;
  for (const Form& f : forms) {
    c.jacobi_group = f.g;
    c.jacobi_pairwise = f.b;
    size_t need = 0;
    if (lt_workspace_size(ctx, LT_OP_SVT, I1, I2, 0, &need) != LT_OK || need > ws_bytes) continue;
    const double ms = time_calls(st, [&] { return lt_svt(ctx, I1, I2, A, tau, D, ws, ws_bytes, stream); });
    if (!std::isfinite(ms)) continue;
    ++timed;
    if (f.g == 0 && f.b == 0) dflt = ms;
    if (ms < best) { best = ms; pick = f; }
  }
  if (timed == 0) {
    c.jacobi_group = keep_g;
    c.jacobi_pairwise = keep_b;
    return cuda_status(cudaGetLastError()) == LT_OK ? LT_ERR_ARG : LT_ERR_CUDA;
  }
  c.jacobi_group = pick.g;
  c.jacobi_pairwise = pick.b;
  if (report) *report = lt_tune_report{pick.g, pick.b, c.tc_tile_n, timed, best, dflt};
  return LT_OK;
}

lt_status lt_autotune_product(lt_ctx ctx, int64_t I1, int64_t l, int64_t I2, const void* A,
                              const void* B, void* C, void* ws, size_t ws_bytes, void* stream,
                              lt_tune_report* report) {
  if (check_ctx(ctx) != LT_OK || !A || !B || !C) return LT_ERR_ARG;
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  const int keep = c.tc_tile_n;
  std::vector<int> forms = {0};
  if (c.prec == LT_MIXED) forms.insert(forms.end(), {32, 64, 128});
  double best = INFINITY, dflt = INFINITY;
  int pick = keep, timed = 0;
  for (int tn : forms) {
    c.tc_tile_n = tn;
    const double ms = time_calls(st, [&] {
      return lt_product(ctx, I1, l, I2, A, B, C, ws, ws_bytes, stream);
    });
    if (!std::isfinite(ms)) continue;
    ++timed;
    if (tn == 0) dflt = ms;
    if (ms < best) { best = ms; pick = tn; }
  }
  c.tc_tile_n = timed ? pick : keep;
  if (timed == 0) return LT_ERR_ARG;
  if (report) *report = lt_tune_report{c.jacobi_group, c.jacobi_pairwise, pick, timed, best, dflt};
  return LT_OK;
}

lt_status lt_ctx_get_stats(lt_ctx ctx, lt_stats* out, int reset) {
  if (!ctx || !out) return LT_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cudaError_t e = cudaDeviceSynchronize();
  for (auto& r : c->pending) {
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    c->stats.k[r.fam].ms += ms;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
  double dev[14] = {};
  if (e == cudaSuccess) e = cudaMemcpy(dev, c->d_counters, sizeof(dev), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, sizeof(dev));
  for (int i = 0; i < 4; ++i) c->stats.k[i].flops += dev[i];
  for (int i = 0; i < 10; ++i) c->stats.jacobi_phase_cycles[i] += dev[4 + i];
  c->stats.tc_launches += c->tc_launches;
  c->tc_launches = 0;
  *out = c->stats;
  if (reset) c->stats = lt_stats{};
  return cuda_status(e);
}

lt_status lt_last_device_status(lt_ctx ctx, int32_t* out) {
  if (!ctx || !out) return LT_ERR_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cudaError_t e = cudaDeviceSynchronize();
  int32_t v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  *out = v;
  return cuda_status(e);
}

}  // extern "C"
