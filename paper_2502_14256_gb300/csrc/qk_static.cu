// qk_eigs_static: the eigenvalue computation of qk_eigs with its scratch space in a
// static device array owned by this library, so that the caller passes only inputs
// and outputs and nothing is allocated.
//
// Who needs it: code that cannot obtain a device buffer at the call site, for
// instance a plug-in called back by a host application that owns every byte of GPU
// memory through its own allocator and lends none out, or a fixed-footprint service
// whose policy forbids device allocations after start-up.
//
// What it costs and how it behaves:
//   * the array below occupies QK_EIGS_STATIC_MAX_BYTES (4 MiB) on every GPU that
//     loads the library, until the process exits;
//   * in host code `g_static_scratch` only names a host-side stand-in, not device
//     memory: the device address is looked up with cudaGetSymbolAddress, once per
//     device, with that device current, on the first call made on that device (so
//     make that first call before any stream capture);
//   * all calls share the one array and it keeps whatever the last call left in it;
//     nothing in it needs to start at zero here, because every byte a call reads was
//     written earlier by the same call; calls whose kernels overlap on the GPU (two
//     streams, or two host threads on one device) race on the array, so the caller
//     must serialise them.
#include <mutex>

#include "qk_common.cuh"
#include "qk_internal.h"

namespace qk {

static __device__ __align__(256) unsigned char g_static_scratch[QK_EIGS_STATIC_MAX_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void *g_static_addr[kMaxDevices];  // device address of g_static_scratch per device

static int static_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "qk_eigs_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(QK_EINVAL, "qk_eigs_static: device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "qk_eigs_static: cudaGetSymbolAddress");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return QK_OK;
}

}  // namespace qk

using namespace qk;

extern "C" int qk_eigs_static(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form,
                              const void *col, double zeta, double eta, double *lam, uint32_t *status,
                              qk_stream stream) {
  set_error("%s", "");
  if (family != QK_DSI && family != QK_SI) return fail(QK_EINVAL, "family must be QK_DSI or QK_SI");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (batch == 0) return QK_OK;
  if (!col || !lam) return fail(QK_EINVAL, "qk_eigs_static: NULL array");
  if (!(zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  // bound the element count before any multiplication (batch << m can exceed 2^64 / 16)
  const size_t eb = elem_bytes(family, dtype);
  const size_t need = (uint64_t)batch > ((QK_EIGS_STATIC_MAX_BYTES / eb) >> m) ? SIZE_MAX : ws_eigs(family, m, batch, dtype);
  if (need > QK_EIGS_STATIC_MAX_BYTES)
    return fail(QK_EINVAL,
                "qk_eigs_static: %u column(s) of 2^%u need more scratch than the %zu-byte static array; "
                "call qk_eigs with a workspace instead",
                batch, m, (size_t)QK_EIGS_STATIC_MAX_BYTES);
  void *ws = nullptr;
  int rc = static_scratch(&ws);
  if (rc) return rc;
  return op_eigs(family, m, batch, dtype, form, col, zeta, eta, lam, ws, status, (cudaStream_t)stream);
}
