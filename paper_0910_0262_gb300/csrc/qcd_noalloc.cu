// qcd_mhat_static: the FP64 even-odd operator Mhat (or Mhat^dag) applied to one
// field without allocating any device memory.
//
// Why it exists.  qcd_dslash stages its fields in work buffers that the context
// allocates with cudaMalloc on first use (and grows later).  Some callers cannot
// accept that: a host application whose memory pool already holds the GPU's free
// memory (a cudaMalloc would fail or fragment it), or a latency-sensitive loop that
// cannot take the device-wide synchronisation cudaMalloc / cudaFree may cause.
// This entry point keeps its three work fields -- the input in the library's
// native layout, the odd-site temporary A_oo^-1 D_oe in, and the native result --
// in one file-scope device array of fixed size instead.
//
// Behaviour and limits.
//  * The array holds QCD_STATIC_SCRATCH_BYTES (24 MiB); every GPU that loads the
//    library keeps it until the process exits.  A lattice fits when
//    3 * 192 * V/2 bytes <= QCD_STATIC_SCRATCH_BYTES (for example 16^4); larger
//    lattices are rejected with QCD_ERR_ARG before anything is launched.
//  * The device address of the array is looked up once per device, by the first
//    call made on that device (cudaGetSymbolAddress, with that device current),
//    and kept for the life of the process: it assumes the device's primary
//    context is not reset (cudaDeviceReset) while the library is loaded.  Make
//    that first call before any stream capture.
//  * The call makes the context's device current while it runs and restores the
//    caller's current device before it returns.
//  * All calls share the one array and it keeps the last call's contents.  Every
//    byte a call reads from it is written earlier in the same call, so nothing
//    needs clearing; but calls whose work overlaps on the GPU (two streams, two
//    contexts on the same device) race on the array.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "qcd.h"
#include "qcd_api_scope.h"
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"


using namespace qcd;

static __device__ __align__(256) unsigned char g_static_scratch[QCD_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on `device` (current), looked up on first use.
cudaError_t scratch_on(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" qcd_status qcd_mhat_static(qcd_ctx* ctx, double* out, const double* in, int dagger) {
  CtxView v;
  const bool have_ctx = ctx_view(ctx, &v);
  // the context's device is current during the call; the caller's current device is restored on return
  ApiScope scope("qcd_mhat_static", have_ctx ? v.device : -1);
  if (scope.status() != QCD_OK) return scope.status();
  if (!out || !in) return set_error(QCD_ERR_ARG, "null field pointer");
  const size_t field = (size_t)192 * v.g.Vh;  // one FP64 even or odd field in the native layout
  if (3 * field > (size_t)QCD_STATIC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg, "lattice too large for qcd_mhat_static: needs %zu bytes of scratch, the maximum is %u",
             3 * field, (unsigned)QCD_STATIC_SCRATCH_BYTES);
    return set_error(QCD_ERR_ARG, msg);
  }
  if (v.device < 0 || v.device >= kMaxDevices) return set_error(QCD_ERR_ARG, "device index out of range");
  if (!v.have_gauge || !v.have_clover) return set_error(QCD_ERR_STATE, "qcd_mhat_static needs load_gauge and clover_build");
  if (v.slab) return set_error(QCD_ERR_STATE, "qcd_mhat_static is not available on a t-slab context");
  if ((const char*)out < (const char*)in + field && (const char*)in < (const char*)out + field)
    return set_error(QCD_ERR_ARG, "in and out overlap");
  void* base = nullptr;
  cudaError_t e = scratch_on(v.device, &base);
  if (e != cudaSuccess) return set_error(QCD_ERR_CUDA, cudaGetErrorString(e));
  unsigned char* s = static_cast<unsigned char*>(base);
  void* x_nat = s;
  void* t_nat = s + field;
  void* y_nat = s + 2 * field;
  launch_spinor_to_native(64, v.g, reinterpret_cast<const double2*>(in), x_nat, nullptr, 1, v.st);
  DslashArgs a;
  memset(&a, 0, sizeof a);
  a.g = v.g;
  a.nrhs = 1;
  a.gauge = v.g64;
  // t_o = A_oo^-1 D_oe (g5) x
  a.p = 1;
  a.in = x_nat;
  a.out = t_nat;
  a.clover = v.Ainv_odd64;
  a.in_g5 = dagger ? 1 : 0;
  launch_dslash(64, 18, EPI_CLOVER_INV, a, v.st);
  // y_e = (g5)(A_ee (g5) x - kappa^2 D_eo t_o)
  DslashArgs b;
  memset(&b, 0, sizeof b);
  b.g = v.g;
  b.nrhs = 1;
  b.gauge = v.g64;
  b.p = 0;
  b.in = t_nat;
  b.out = y_nat;
  b.x = x_nat;
  b.clover = v.A_even64;
  b.a = -v.kappa * v.kappa;
  b.x_g5 = b.out_g5 = dagger ? 1 : 0;
  launch_dslash(64, 18, EPI_XPAY, b, v.st);
  launch_spinor_to_canon(64, v.g, y_nat, nullptr, reinterpret_cast<double2*>(out), 1, v.st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(QCD_ERR_CUDA, cudaGetErrorString(e));
  return QCD_OK;
}
