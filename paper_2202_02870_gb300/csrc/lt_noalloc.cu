// lt_product_noalloc: the *_L-product for callers that cannot allocate device memory.
//
// Some callers cannot give the library a workspace: a host application that reserves
// all of the GPU's memory for its own pool up front and forbids further cudaMalloc
// calls, or code running where cudaMalloc/cudaFree are not allowed because they may
// synchronise the device.  lt_product needs scratch for the transform-domain operands
// L(A) and L(B); this entry point takes that scratch from a fixed array in the
// library's own device memory instead, and allocates nothing.
//
// The array is a file-scope __device__ object of LT_NOALLOC_SCRATCH_BYTES bytes.  Every
// GPU on which this module is loaded holds it until the process exits.  In host code
// its name is only a host-side stand-in; the device address is looked up once per
// device with cudaGetSymbolAddress (with that device current) on the first call made
// while the device is current.  That first call should therefore come before any
// stream capture.
//
// All calls share the array, and it keeps the contents of the last call.  Nothing in it
// needs to start at zero: L(A) and L(B) are written in full before they are read.
// Calls whose work overlaps on the GPU (other streams, or other host threads) race on
// the array; callers must order them, e.g. on one stream.
#include <mutex>

#include "lt_internal.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[LT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of one transform-domain operand (rows x cols x P elements of elem bytes) rounded
// up to 256, in *out; false when the product overflows or the operand alone exceeds the
// array (so that no wrapped size can pass the limit check).
bool operand_bytes(int64_t rows, int64_t cols, int64_t P, int elem, size_t* out) {
  size_t b = 0;
  if (rows < 0 || cols < 0 || P < 0 || elem < 0) return false;
  if (__builtin_mul_overflow((size_t)rows, (size_t)cols, &b) ||
      __builtin_mul_overflow(b, (size_t)P, &b) || __builtin_mul_overflow(b, (size_t)elem, &b))
    return false;
  if (b > (size_t)LT_NOALLOC_SCRATCH_BYTES) return false;
  *out = align256(b);
  return *out <= (size_t)LT_NOALLOC_SCRATCH_BYTES;
}

// Device address of g_noalloc_scratch on the current device (looked up once).
lt_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LT_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return LT_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LT_OK;
}

}  // namespace

extern "C" lt_status lt_product_noalloc(lt_ctx ctx, int64_t I1, int64_t l, int64_t I2,
                                        const void* A, const void* B, void* C,
                                        void* stream) {
  if (ctx == nullptr || !A || !B || !C || C == A || C == B) return LT_ERR_ARG;
  if (I1 < 1 || l < 1 || I2 < 1) return LT_ERR_ARG;
  if (I1 > (1 << 20) || l > (1 << 20) || I2 > (1 << 20)) return LT_ERR_SHAPE;
  const lt::Ctx& c = *reinterpret_cast<lt::Ctx*>(ctx);
  // The kernels run on the current device; the context's matrices live on c.device.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LT_ERR_CUDA;
  if (dev != c.device) return LT_ERR_ARG;
  size_t a_bytes = 0, b_bytes = 0;
  if (!operand_bytes(I1, l, c.P, c.elem, &a_bytes) || !operand_bytes(l, I2, c.P, c.elem, &b_bytes) ||
      a_bytes > (size_t)LT_NOALLOC_SCRATCH_BYTES - b_bytes)
    return LT_ERR_SHAPE;
  lt::TransformPlan pa, pb, pc;
  lt_status s;
  if ((s = lt::plan_transform(c, I1 * l, false, &pa)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, l * I2, false, &pb)) != LT_OK) return s;
  if ((s = lt::plan_transform(c, I1 * I2, true, &pc)) != LT_OK) return s;
  void* base = nullptr;
  if ((s = scratch_address(&base)) != LT_OK) return s;
  unsigned char* w = static_cast<unsigned char*>(base);
  void* Ah = w;
  void* Bh = w + a_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = lt::launch_transform(c, pa, A, Ah, lt::FUSE_NONE, nullptr, st, nullptr);
  if (e == cudaSuccess) e = lt::launch_transform(c, pb, B, Bh, lt::FUSE_NONE, nullptr, st, nullptr);
  if (e == cudaSuccess) e = lt::launch_facewise_gemm(c, I1, I2, l, Ah, Bh, C, st);
  if (e == cudaSuccess) e = lt::launch_transform(c, pc, C, C, lt::FUSE_NONE, nullptr, st, nullptr);
  return e == cudaSuccess ? LT_OK : LT_ERR_CUDA;
}
