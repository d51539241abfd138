// vie_matvec_noalloc: the FP32 Tucker matvec for callers that cannot allocate
// device memory when they need a product (a serving loop whose device memory
// belongs to another allocator under a fixed budget, or a callback that must
// not trigger the device-wide synchronisation that cudaMalloc and cudaFree can
// cause).  Its scratch (the two intermediate spectra of the staged FFT) is a
// fixed array compiled into this library instead of memory that vie_matvec
// would allocate on first use.
#include <mutex>

#include "vie_internal.cuh"

// 64 MiB of scratch on every GPU that loads the library, held until exit.
static constexpr size_t kScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d outside the supported range", dev);
    return VIE_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return VIE_OK;
}

}  // namespace

extern "C" int vie_matvec_noalloc(const vie_op* op, const void* J, void* Y, int B, void* stream) {
  clear_error();
  if (!op || !J || !Y) {
    set_error("NULL argument");
    return VIE_ERR_ARG;
  }
  if (B < 1) {
    set_error("batch %d must be >= 1", B);
    return VIE_ERR_ARG;
  }
  // T1 [B][3][P1][n2][n3] and T2 [B][3][P1][P2][n3] in complex64
  const size_t need = (size_t)B * 3 *
                      ((size_t)op->P[0] * op->n[1] * op->n[2] +
                       (size_t)op->P[0] * op->P[1] * op->n[2]) * sizeof(float2);
  if (need > kScratchBytes) {
    set_error("vie_matvec_noalloc needs %zu bytes of scratch for this grid and batch, "
              "above its fixed %zu bytes; use vie_matvec", need, kScratchBytes);
    return VIE_ERR_ARG;
  }
  void* ws = nullptr;
  VIE_TRY(scratch_address(&ws));
  return matvec_run<float>(op, ws, static_cast<const float2*>(J), static_cast<float2*>(Y), B,
                           VIE_PATH_TUCKER, 0, 0, nullptr, nullptr, nullptr,
                           static_cast<cudaStream_t>(stream));
}
