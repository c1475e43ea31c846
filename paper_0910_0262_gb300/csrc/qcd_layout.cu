// Layout kernels: canonical complex128 fields <-> checkerboarded structure-of-arrays.
//
// The paper pads MILC's site structs to 128-byte multiples and odd strides so
// that the Cell's DMA engine reaches full bank bandwidth (Sec. 3).  On a GPU
// the equivalent goal -- every byte fetched is a byte used -- is met by a
// component-major, site-minor layout per parity: consecutive threads (sites)
// read consecutive 8/16-byte words, so no padding is transferred at all.
#include "qcd_kernels.h"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_layout)

std::atomic<long long> g_kernel_launches{0};

namespace {

__device__ __forceinline__ void coords_of(const Geom& g, int i, int& x, int& y, int& z, int& t) {
  int c[4];
  lattice_coords(g, i, c);
  x = c[0];
  y = c[1];
  z = c[2];
  t = c[3];
}

// canonical gauge U[i][mu][3][3] complex128 -> per-parity, per-direction SoA copies
__global__ void pack_gauge_kernel(Geom g, const double2* __restrict__ U, double2* g64, void* g32, int recon32,
                                  void* g16, int recon16) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = 2 * g.Vh;
  if (tid >= V * 4) return;
  const int i = tid >> 2, mu = tid & 3;
  int x, y, z, t;
  coords_of(g, i, x, y, z, t);
  const int p = (x + y + z + t) & 1;
  const int h = i >> 1;
  const double2* src = U + (size_t)tid * 9;
  double2 u[9];
#pragma unroll
  for (int k = 0; k < 9; k++) u[k] = src[k];
  const size_t base = (size_t)(p * 4 + mu);
#pragma unroll
  for (int k = 0; k < 9; k++) g64[(base * 9 + k) * g.Vh + h] = u[k];
  if (g32) {
    if (recon32 == 12) {
      float4* q = static_cast<float4*>(g32);
#pragma unroll
      for (int k = 0; k < 3; k++)
        q[(base * 3 + k) * g.Vh + h] = make_float4((float)u[2 * k].x, (float)u[2 * k].y, (float)u[2 * k + 1].x,
                                                   (float)u[2 * k + 1].y);
    } else {
      float2* q = static_cast<float2*>(g32);
#pragma unroll
      for (int k = 0; k < 9; k++) q[(base * 9 + k) * g.Vh + h] = make_float2((float)u[k].x, (float)u[k].y);
    }
  }
  if (g16) {
    if (recon16 == 12) {
      uint2* q = static_cast<uint2*>(g16);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        uint2 v;
        v.x = f2h((float)u[2 * k].x, (float)u[2 * k].y);
        v.y = f2h((float)u[2 * k + 1].x, (float)u[2 * k + 1].y);
        q[(base * 3 + k) * g.Vh + h] = v;
      }
    } else {
      uint32_t* q = static_cast<uint32_t*>(g16);
#pragma unroll
      for (int k = 0; k < 9; k++) q[(base * 9 + k) * g.Vh + h] = f2h((float)u[k].x, (float)u[k].y);
    }
  }
}

template <int P>
__global__ void spinor_to_native_kernel(Geom g, const double2* __restrict__ canon, void* nat, float* norm, int nrhs) {
  using R = typename Real<P>::T;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.Vh * nrhs) return;
  const int r = tid / g.Vh, h = tid - r * g.Vh;
  const double2* src = canon + (size_t)tid * 12;
  cx<R> s[12];
#pragma unroll
  for (int c = 0; c < 12; c++) {
    double2 v = src[c];
    s[c] = cmk(R(v.x), R(v.y));
  }
  SpinorIO<P>::store(nat, norm, g.Vh, r, h, s);
}

template <int P>
__global__ void spinor_to_canon_kernel(Geom g, const void* nat, const float* norm, double2* canon, int nrhs) {
  using R = typename Real<P>::T;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.Vh * nrhs) return;
  const int r = tid / g.Vh, h = tid - r * g.Vh;
  cx<R> s[12];
  SpinorIO<P>::load(nat, norm, g.Vh, r, h, s);
  double2* dst = canon + (size_t)tid * 12;
#pragma unroll
  for (int c = 0; c < 12; c++) dst[c] = make_double2(double(s[c].re), double(s[c].im));
}

__global__ void check_finite_kernel(const double* __restrict__ d, size_t n, int* flag) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (; i < n; i += stride) bad |= !isfinite(d[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

inline int nblocks(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_pack_gauge(const Geom& g, const double2* canon, void* g64, void* g32, int recon32, void* g16,
                       int recon16, cudaStream_t st) {
  g_kernel_launches += 1;
  const int B = 128;
  pack_gauge_kernel<<<nblocks(8LL * g.Vh, B), B, 0, st>>>(g, canon, static_cast<double2*>(g64), g32, recon32, g16,
                                                          recon16);
}

void launch_spinor_to_native(int prec, const Geom& g, const double2* canon, void* nat, float* norm, int nrhs,
                             cudaStream_t st) {
  g_kernel_launches += 1;
  const int B = 128;
  const int nb = nblocks((long long)g.Vh * nrhs, B);
  if (prec == 64) spinor_to_native_kernel<64><<<nb, B, 0, st>>>(g, canon, nat, norm, nrhs);
  else if (prec == 32) spinor_to_native_kernel<32><<<nb, B, 0, st>>>(g, canon, nat, norm, nrhs);
  else spinor_to_native_kernel<16><<<nb, B, 0, st>>>(g, canon, nat, norm, nrhs);
}

void launch_spinor_to_canon(int prec, const Geom& g, const void* nat, const float* norm, double2* canon, int nrhs,
                            cudaStream_t st) {
  g_kernel_launches += 1;
  const int B = 128;
  const int nb = nblocks((long long)g.Vh * nrhs, B);
  if (prec == 64) spinor_to_canon_kernel<64><<<nb, B, 0, st>>>(g, nat, norm, canon, nrhs);
  else if (prec == 32) spinor_to_canon_kernel<32><<<nb, B, 0, st>>>(g, nat, norm, canon, nrhs);
  else spinor_to_canon_kernel<16><<<nb, B, 0, st>>>(g, nat, norm, canon, nrhs);
}

void launch_check_finite(const double* data, size_t n, int* flag, cudaStream_t st) {
  if (n > 0) g_kernel_launches += 1;
  if (n == 0) return;
  const int B = 256;
  long long nb = (long long)((n + B - 1) / B);
  if (nb > 152 * 16) nb = 152 * 16;
  check_finite_kernel<<<(int)nb, B, 0, st>>>(data, n, flag);
}

void launch_zero(void* ptr, size_t bytes, cudaStream_t st) {
  if (bytes) cudaMemsetAsync(ptr, 0, bytes, st);
}

}  // namespace qcd
