// Pressure recovery with no device allocation: the same kernels as the
// epilogue of tg_solve, with their scratch (inverse permeabilities, the
// row-integrated pressures and the row offsets) in one file-scope device
// array instead of handle-owned buffers.
//
// Who needs it: callers that may not call cudaMalloc -- processes whose
// device memory is owned entirely by another allocator (a framework's caching
// allocator or a fixed arena reserved at start-up, where a stray cudaMalloc
// can fail or fragment that arena), and latency-critical paths that must not
// take the implicit device synchronisation of cudaMalloc / cudaFree.
//
// The first call on a device looks up the array's device address (one-time
// set-up per device).  The call reads its status on the host and synchronises
// its stream, which a stream capture cannot record: on a capturing stream it
// returns TG_ERR_UNSUPPORTED without enqueuing anything.
#include <mutex>

#include "../../include/tgms.h"
#include "common.cuh"

namespace {

constexpr int kNoAllocMaxN = 1024;          // largest grid side served
constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kNN = (size_t)kNoAllocMaxN * kNoAllocMaxN;
// layout: kinv (FP64 n^2) | kinv32 (FP32 n^2) | status (int) | pressure work (n^2 + 2n + 2 FP64)
constexpr size_t kOffKinv = 0;
constexpr size_t kOffKinv32 = round_up(kOffKinv + sizeof(double) * kNN);
constexpr size_t kOffStatus = round_up(kOffKinv32 + sizeof(float) * kNN);
constexpr size_t kOffWork = round_up(kOffStatus + sizeof(int));
constexpr size_t kScratchBytes = round_up(kOffWork + sizeof(double) * (kNN + 2 * kNoAllocMaxN + 2));

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_pressure_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device with
// that device current.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_pressure_scratch) != cudaSuccess || !ptr) return TG_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return TG_OK;
}

}  // namespace

extern "C" int tg_pressure_noalloc(const double* kappa, const double* ux, const double* uy, double* p, int n,
                                   void* stream) {
  if (!kappa || !ux || !uy || !p || n < 2) return TG_ERR_INVALID_ARG;
  if (n > kNoAllocMaxN) return TG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // (the legacy stream answers cudaErrorStreamCaptureImplicit while a
  // blocking stream captures: work on it would join that capture)
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  const cudaError_t query = cudaStreamIsCapturing(s, &capture);
  if (query == cudaErrorStreamCaptureImplicit) return TG_ERR_UNSUPPORTED;
  if (query != cudaSuccess) return TG_ERR_CUDA;
  if (capture != cudaStreamCaptureStatusNone) return TG_ERR_UNSUPPORTED;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  unsigned char* s8 = static_cast<unsigned char*>(base);
  double* kinv = reinterpret_cast<double*>(s8 + kOffKinv);
  float* kinv32 = reinterpret_cast<float*>(s8 + kOffKinv32);
  int* status = reinterpret_cast<int*>(s8 + kOffStatus);
  double* work = reinterpret_cast<double*>(s8 + kOffWork);
  // A launch error already pending in this thread belongs to the caller's
  // earlier work: it is neither reported here nor cleared.
  const cudaError_t pending = cudaPeekAtLastError();
  // the status word keeps the previous call's value: clear it
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return TG_ERR_CUDA;
  tg::launch_kinv(kappa, kinv, kinv32, status, n, s);
  tg::launch_pressure(ux, uy, kinv, p, work, n, s);
  const cudaError_t launched = cudaPeekAtLastError();
  if (launched != cudaSuccess && launched != pending) return TG_ERR_CUDA;
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return TG_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TG_ERR_CUDA;
  return h_status ? TG_ERR_INVALID_ARG : TG_OK;
}
