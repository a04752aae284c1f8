// noalloc.cu -- the pivoted QR of Step 2 for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: their device memory belongs to another
// allocator (a framework's caching allocator, or a fixed pool reserved at
// start-up that must not shrink behind its back), or they run on a
// latency-critical path where cudaMalloc/cudaFree may synchronize the device.
// minnorm_qr_noalloc gives them the same pivoted QR kernel the plans use, with
// its scratch (partial norms, the diagonal of R, the pivots, the words the
// CTAs exchange between steps) taken from one file-scope device array instead of a plan. The caller
// still passes the matrix and the output buffers.
//
// The array below is part of the library's module: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits. All calls
// on a device share it and it keeps the last call's contents, so each call
// clears the words that must start at zero, and calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
#include <mutex>

#include "../../include/minnorm.h"
#include "common.cuh"
#include "kernels.h"

namespace mn {

// Largest m the scratch covers; the scratch holds, for m columns:
// 2m + m + m doubles (partial norms, reference norms, diagonal of R),
// m int32 pivots, the exchange words of the QR grid and the error word.
constexpr int64_t kNoAllocMaxM = 4096;
constexpr size_t kNoAllocScratchBytes = 192 * 1024;
// exchange words of the QR kernel (flags and the posted candidates of up to 320 CTAs)
constexpr size_t kNoAllocMailBytes = 24 * 1024;

static __device__ __align__(256) unsigned char g_qr_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_qr_scratch on the current device, looked up once per
// device. (In host code the symbol's name is only a host-side handle, not a
// device address.)
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qr_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void widen_piv_kernel(const int32_t *__restrict__ a, int64_t *__restrict__ b, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) b[i] = a[i];
}

}  // namespace
}  // namespace mn

using namespace mn;

extern "C" minnorm_status minnorm_qr_noalloc(void *Y, int64_t ldy, int64_t l, int64_t m, void *R_out,
                                             void *piv_out, void *stream) {
  if (!Y || !R_out || !piv_out) return MINNORM_EINVAL;
  if (m < 1 || l < m || ldy != l || l > (int64_t)1 << 30) return MINNORM_EINVAL;
  if (m > kNoAllocMaxM) return MINNORM_ENOTSUP;  // beyond the fixed scratch
  // the kernels access Y and R as 16-byte complex128 and the pivots as int64: an offset view
  // would fault on the GPU, so it is refused here, before any device work
  if (((uintptr_t)Y & 15u) || ((uintptr_t)R_out & 15u) || ((uintptr_t)piv_out & 7u)) return MINNORM_EINVAL;
  unsigned char *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return MINNORM_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // carve the scratch: [vn1: 2m][vn2: m][beta: m] doubles, then pivots, the exchange words, the error word
  double *vn1 = reinterpret_cast<double *>(base);
  double *vn2 = vn1 + 2 * kNoAllocMaxM;
  double *beta = vn2 + kNoAllocMaxM;
  int32_t *piv = reinterpret_cast<int32_t *>(beta + kNoAllocMaxM);
  unsigned char *mail = base + 4 * kNoAllocMaxM * sizeof(double) + kNoAllocMaxM * sizeof(int32_t);
  int *err = reinterpret_cast<int *>(mail + kNoAllocMailBytes);
  static_assert(4 * kNoAllocMaxM * sizeof(double) + kNoAllocMaxM * sizeof(int32_t) + kNoAllocMailBytes +
                        sizeof(int) <= kNoAllocScratchBytes,
                "scratch too small");
  if (qr_mail_bytes() > kNoAllocMailBytes) return MINNORM_ENOTSUP;
  // the error word must start at zero (launch_qrp clears the exchange flags itself);
  // the previous call's value is still there
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return MINNORM_ECUDA;
  QrArgs q{};
  q.Y = Y;
  q.l = (int)l;
  q.m = (int)m;
  q.vn1 = vn1;
  q.vn2 = vn2;
  q.beta = beta;
  q.piv = piv;
  q.R = R_out;
  q.mail = mail;
  q.err = err;
  q.limit_ns = kBarrierLimitNs;
  if (launch_qrp(q, st) != cudaSuccess) return MINNORM_ECUDA;
  note_launch();
  widen_piv_kernel<<<(int)((m + 255) / 256), 256, 0, st>>>(piv, (int64_t *)piv_out, (int)m);
  if (cudaGetLastError() != cudaSuccess) return MINNORM_ECUDA;
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MINNORM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MINNORM_ECUDA;
  return h_err ? MINNORM_ETIMEOUT : MINNORM_OK;
}
