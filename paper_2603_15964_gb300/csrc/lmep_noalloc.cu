// lmep_noalloc.cu -- the adjoint step with library-owned static scratch.
//
// lmep_adjoint_step needs a scratch buffer from the caller.  Some callers
// cannot allocate device memory at all: a plug-in hosted by an application
// whose own allocator owns every byte of the device, a latency-critical loop
// that must never enter the driver's allocator, or a sandbox whose device
// budget is fixed before the library is loaded.  lmep_adjoint_step_noalloc
// serves them: its scratch is the file-scope array below, which every GPU
// that loads this library holds until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the first call on each device (with that device current) asks
// the runtime for the array's device address with cudaGetSymbolAddress and
// caches it.  Later calls reuse the cached address after checking that the
// current context still knows it as device memory of this device (a
// cudaDeviceReset destroys the context that held it; the next call then looks
// the address up again in the new one).
#include <mutex>
#include <string>

#include "../../include/lmep.h"
#include "lmep_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_adjoint_scratch[kScratchBytes];
static __device__ __align__(256) unsigned int g_noalloc_flags[64];

struct DeviceAddresses {
  void* scratch = nullptr;
  unsigned* flags = nullptr;
  bool ready = false;
};
DeviceAddresses g_addr[kMaxDevices];
std::mutex g_mutex;

lmep_status reject(lmep_status s, const std::string& msg) {
  lmep::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" lmep_status lmep_adjoint_step_noalloc(const lmep_grid* g, const lmep_operator* op, double dt,
                                                 const void* u_dev, const void* lam_next_dev, void* lam_dev,
                                                 double* dnu_dev, int32_t precision, void* stream) {
  if (!g || !op) return reject(LMEP_ERR_INVALID, "grid/operator is NULL");
  if (g->n < 3 || g->n > 15 || (g->n % 2) == 0) return reject(LMEP_ERR_INVALID, "n must be odd, 3..15");
  if (g->N < g->n) return reject(LMEP_ERR_INVALID, "N must be >= n");
  if (g->batch > 1) return reject(LMEP_ERR_UNSUPPORTED, "lmep_adjoint_step_noalloc takes one instance (batch <= 1)");
  if (g->window_shift != 0 || g->reserved != 0)
    return reject(LMEP_ERR_UNSUPPORTED, "window_shift is for constant-coefficient linear steps");
  if (!(g->h > 0.0)) return reject(LMEP_ERR_INVALID, "h must be positive");
  if (g->bc != LMEP_BC_PERIODIC && g->bc != LMEP_BC_DIRICHLET)
    return reject(LMEP_ERR_UNSUPPORTED, "adjoint supports periodic and Dirichlet grids");
  if (g->bc == LMEP_BC_PERIODIC && g->N < 2 * g->n) return reject(LMEP_ERR_UNSUPPORTED, "periodic adjoint needs N >= 2n");
  if (precision != LMEP_PREC_FP64 && precision != LMEP_PREC_MIXED)
    return reject(LMEP_ERR_INVALID, "precision must be LMEP_PREC_FP64 or LMEP_PREC_MIXED");
  if (!u_dev || !lam_next_dev || !lam_dev || !dnu_dev) return reject(LMEP_ERR_INVALID, "NULL buffer");
  if (lam_dev == lam_next_dev) return reject(LMEP_ERR_INVALID, "lam_dev must differ from lam_next_dev");
  const bool mixed = precision == LMEP_PREC_MIXED;
  const size_t need = lmep::adjoint_scratch_bytes(g->N, g->n, mixed);
  if (need > kScratchBytes)
    return reject(LMEP_ERR_INVALID, "lmep_adjoint_step_noalloc: this grid needs " + std::to_string(need) +
                                        " bytes of scratch but the static scratch holds " +
                                        std::to_string(kScratchBytes) +
                                        " (N (n + 1) elem + 4 N + 256 bytes); use lmep_adjoint_step");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(LMEP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return reject(LMEP_ERR_UNSUPPORTED, "device index out of range");
  DeviceAddresses a;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_addr[dev].ready) {
      cudaPointerAttributes at{};
      const cudaError_t q = cudaPointerGetAttributes(&at, g_addr[dev].scratch);
      if (q != cudaSuccess) (void)cudaGetLastError();  // a stale address is not an error of this call
      if (q != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != dev ||
          at.devicePointer != g_addr[dev].scratch)
        g_addr[dev] = DeviceAddresses{};
    }
    if (!g_addr[dev].ready) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_adjoint_scratch);
      if (e != cudaSuccess)
        return reject(LMEP_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      void* f = nullptr;
      e = cudaGetSymbolAddress(&f, g_noalloc_flags);
      if (e != cudaSuccess)
        return reject(LMEP_ERR_CUDA, std::string("cudaGetSymbolAddress(flags): ") + cudaGetErrorString(e));
      g_addr[dev].scratch = p;
      g_addr[dev].flags = static_cast<unsigned*>(f);
      g_addr[dev].ready = true;
    }
    a = g_addr[dev];
  }
  const lmep::KParams p = lmep::make_params(g, op, dt, 0);
  e = lmep::launch_adjoint(p, u_dev, lam_next_dev, lam_dev, dnu_dev, a.scratch, mixed, a.flags,
                           static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return reject(LMEP_ERR_CUDA, std::string("adjoint(noalloc): ") + cudaGetErrorString(e));
  return LMEP_OK;
}
