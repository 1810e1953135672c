// prrp_panel_select_noalloc: the strong RRQR panel selection (the same kernel as
// prrp_panel_select) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a fixed device-memory arena
// owned by another allocator (a stray allocation there can fail or fragment it), loops
// with latency budgets that cannot absorb the implicit device synchronization that
// cudaMalloc and cudaFree may perform, and code that must not create a prrp_ctx (whose
// workspace is allocated).  This entry point therefore needs no context and allocates
// nothing: the kernel's scratch (the device state word and the cross-CTA exchange records
// of the panel tournament) lives in the file-scope array below, which every GPU that loads
// the library holds until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host that name is only a
// stand-in, not a device address.  Every call looks the device address up with
// cudaGetSymbolAddress, with the caller's current device current (cheap next to the
// launch and the synchronization), so a module reloaded after cudaDeviceReset is followed.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "prrp.h"

namespace prrp {
namespace {

constexpr int kStaticMaxCtas = kPanelMaxCtas;   // panel CTAs the static records can hold (160)
constexpr size_t kStateBytes = 256;   // DevState, padded
constexpr size_t kValBytes = 2 * kStaticMaxCtas * kXVal * sizeof(double);
constexpr size_t kKeyBytes = 2 * kStaticMaxCtas * sizeof(int2);
constexpr size_t kVecBytes = 2 * (size_t)kStaticMaxCtas * kMaxW * sizeof(double);
constexpr size_t kQKeyBytes = kQSlots * kStaticMaxCtas * kQKeyStride * sizeof(unsigned long long);
constexpr size_t kQRowBytes = kQSlots * (size_t)kStaticMaxCtas * kQStride * sizeof(double);
constexpr size_t kScratchBytes =
    kStateBytes + kValBytes + kKeyBytes + kVecBytes + kQKeyBytes + kQRowBytes;   // 2,014,976 B
static_assert(kScratchBytes == 2014976, "the documented size of the static scratch");
static_assert(sizeof(DevState) <= kStateBytes, "state word does not fit its slot");
static_assert(kScratchBytes % 256 == 0, "scratch slots keep 256-byte alignment");

static __device__ __align__(256) unsigned char g_panel_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

// With the device current: the device address of the static scratch.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_panel_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

// A caller pointer must be device memory of the current device (or managed memory):
// a kernel launched here would otherwise read another GPU's address.
bool on_device(const void* ptr, int dev) {
  if (!ptr) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace prrp

using namespace prrp;

extern "C" prrp_status prrp_panel_select_noalloc(int m, int w, const double* dP, int ldp,
                                                 double tau, int max_swaps, int* dOrder,
                                                 double* dL21, int* hSwaps, void* stream) {
  if (w < 1 || w > kMaxW || m < w || ldp < w || !dP || !dOrder || !(tau >= 1.0) || max_swaps < 0)
    return PRRP_ERR_INVALID_ARG;
  if (m > w && !dL21) return PRRP_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PRRP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return PRRP_ERR_CUDA;
  // Same grid rule as prrp_panel_select, capped by the static exchange records.
  const int G = std::max(1, std::min(std::min(sms, kStaticMaxCtas), (m + 31) / 32));
  const int rpc = (m + G - 1) / G;
  if (panel_smem_for(w, rpc) > (size_t)smem) return PRRP_ERR_UNSUPPORTED;
  if (!on_device(dP, dev) || !on_device(dOrder, dev) || !on_device(dL21, dev)) return PRRP_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PRRP_ERR_CUDA;
  DevState* st = reinterpret_cast<DevState*>(base);
  // The array keeps the previous call's contents: clear the state word (error status,
  // barrier arrivals, counters) and the QRCP step keys (a key is absent while it holds 0),
  // and fill the QRCP records with the sentinel pattern (a word is taken once it no longer
  // holds it).  The other records need no clearing: each is written before it is read
  // within a call.
  if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) return PRRP_ERR_CUDA;
  unsigned char* qbase = base + kStateBytes + kValBytes + kKeyBytes + kVecBytes;
  if (cudaMemsetAsync(qbase, 0, kQKeyBytes, s) != cudaSuccess) return PRRP_ERR_CUDA;
  if (cudaMemsetAsync(qbase + kQKeyBytes, kQSentinelByte, kQSlots * sizeof(double) * G * kQStride, s) != cudaSuccess)
    return PRRP_ERR_CUDA;
  PanelParams p{};
  p.P = dP; p.ldp = ldp; p.m = m; p.w = w; p.tau = tau; p.max_swaps = max_swaps;
  p.col_offset = 0; p.L21 = dL21; p.ldl = w; p.order = dOrder; p.pairs = nullptr;
  p.st = st;
  p.xval = reinterpret_cast<double*>(base + kStateBytes);
  p.xkey = reinterpret_cast<int2*>(base + kStateBytes + kValBytes);
  p.xvec = reinterpret_cast<double*>(base + kStateBytes + kValBytes + kKeyBytes);
  p.qkey = reinterpret_cast<unsigned long long*>(qbase);
  p.qrow = reinterpret_cast<double*>(qbase + kQKeyBytes);
  p.rows_per_cta = rpc;
  cudaError_t e = launch_panel(p, G, s);
  if (e == cudaErrorCooperativeLaunchTooLarge) return PRRP_ERR_UNSUPPORTED;
  if (e != cudaSuccess) return PRRP_ERR_CUDA;
  DevState h{};
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PRRP_ERR_CUDA;
  if (hSwaps) *hSwaps = h.panel_swaps;
  return static_cast<prrp_status>(h.status);
}
