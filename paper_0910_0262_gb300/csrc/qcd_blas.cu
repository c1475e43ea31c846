// BLAS-1 steps of the conjugate-gradient solve, fused with their reductions.
//
// Every kernel maps one thread to one (site, right-hand side) pair, the RHS
// index fastest, and reduces in FP64 through grid_reduce (warp shuffles ->
// shared memory -> per-block partials -> fixed-order sum in the last block), so
// the scalars of CG (alpha, beta, |r|^2) are produced on the device and the
// iteration needs no host round trip.
#include "qcd_kernels.h"

namespace qcd {

namespace {

constexpr int BB = 256;  // block size of the BLAS kernels

template <int PR, int PP>
__global__ void __launch_bounds__(BB) cg_update_kernel(Geom g, int nrhs, void* x, float* xn, void* r, float* rn,
                                                       const void* p, const float* pn, const void* Ap,
                                                       const float* Apn, ReduceArgs red, const int* halt) {
  using RR = typename Real<PR>::T;
  using RP = typename Real<PP>::T;
  if (halt && *halt) return;
  const int gid = blockIdx.x * BB + threadIdx.x;
  const int k = gid % nrhs, h = gid / nrhs;
  double v = 0.0;
  if (h < g.Vh && red.cg[k].active) {
    const double alpha = red.cg[k].alpha;
    cx<RR> xs[12], rs[12];
    cx<RP> ps[12], aps[12];
    SpinorIO<PR>::load(x, xn, g.Vh, nrhs, k, h, xs);
    SpinorIO<PR>::load(r, rn, g.Vh, nrhs, k, h, rs);
    SpinorIO<PP>::load(p, pn, g.Vh, nrhs, k, h, ps);
    SpinorIO<PP>::load(Ap, Apn, g.Vh, nrhs, k, h, aps);
    const RR a = RR(alpha);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      xs[c].re = fma(a, RR(ps[c].re), xs[c].re);
      xs[c].im = fma(a, RR(ps[c].im), xs[c].im);
      rs[c].re = fma(-a, RR(aps[c].re), rs[c].re);
      rs[c].im = fma(-a, RR(aps[c].im), rs[c].im);
      v += double(rs[c].re) * rs[c].re + double(rs[c].im) * rs[c].im;
    }
    SpinorIO<PR>::store(x, xn, g.Vh, nrhs, k, h, xs);
    SpinorIO<PR>::store(r, rn, g.Vh, nrhs, k, h, rs);
  }
  grid_reduce<BB>(v, nrhs, red);
}

template <int PR, int PP>
__global__ void __launch_bounds__(BB) p_update_kernel(Geom g, int nrhs, const void* r, const float* rn, void* p,
                                                      float* pn, const CGState* cg, const int* halt) {
  using RR = typename Real<PR>::T;
  using RP = typename Real<PP>::T;
  if (halt && *halt) return;
  const int gid = blockIdx.x * BB + threadIdx.x;
  const int k = gid % nrhs, h = gid / nrhs;
  if (h >= g.Vh || !cg[k].active) return;
  const RR beta = RR(cg[k].beta);
  cx<RR> rs[12];
  cx<RP> ps[12];
  SpinorIO<PR>::load(r, rn, g.Vh, nrhs, k, h, rs);
  SpinorIO<PP>::load(p, pn, g.Vh, nrhs, k, h, ps);
  cx<RP> out[12];
#pragma unroll
  for (int c = 0; c < 12; c++) {
    out[c].re = RP(fma(beta, RR(ps[c].re), rs[c].re));
    out[c].im = RP(fma(beta, RR(ps[c].im), rs[c].im));
  }
  SpinorIO<PP>::store(p, pn, g.Vh, nrhs, k, h, out);
}

template <int PR>
__global__ void __launch_bounds__(BB) accumulate_x_kernel(Geom g, int nrhs, double2* x_hi, void* x_lo, float* xn) {
  using RR = typename Real<PR>::T;
  const int gid = blockIdx.x * BB + threadIdx.x;
  const int k = gid % nrhs, h = gid / nrhs;
  if (h >= g.Vh) return;
  cx<RR> lo[12];
  cx<double> hi[12];
  SpinorIO<PR>::load(x_lo, xn, g.Vh, nrhs, k, h, lo);
  SpinorIO<64>::load(x_hi, nullptr, g.Vh, nrhs, k, h, hi);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    hi[c].re += double(lo[c].re);
    hi[c].im += double(lo[c].im);
    lo[c] = cmk(RR(0), RR(0));
  }
  SpinorIO<64>::store(x_hi, nullptr, g.Vh, nrhs, k, h, hi);
  SpinorIO<PR>::store(x_lo, xn, g.Vh, nrhs, k, h, lo);
}

template <int PR>
__global__ void __launch_bounds__(BB) true_residual_kernel(Geom g, int nrhs, const double2* b, const double2* Ap,
                                                           void* r_lo, float* rn, ReduceArgs red) {
  using RR = typename Real<PR>::T;
  const int gid = blockIdx.x * BB + threadIdx.x;
  const int k = gid % nrhs, h = gid / nrhs;
  double v = 0.0;
  if (h < g.Vh) {
    cx<double> bs[12], as[12];
    SpinorIO<64>::load(b, nullptr, g.Vh, nrhs, k, h, bs);
    SpinorIO<64>::load(Ap, nullptr, g.Vh, nrhs, k, h, as);
    cx<RR> rs[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
      const cx<double> d = bs[c] - as[c];
      v += norm2(d);
      rs[c] = cmk(RR(d.re), RR(d.im));
    }
    SpinorIO<PR>::store(r_lo, rn, g.Vh, nrhs, k, h, rs);
  }
  grid_reduce<BB>(v, nrhs, red);
}

__global__ void __launch_bounds__(BB) norm2_kernel(Geom g, int nrhs, const double2* a, ReduceArgs red) {
  const int gid = blockIdx.x * BB + threadIdx.x;
  const int k = gid % nrhs, h = gid / nrhs;
  double v = 0.0;
  if (h < g.Vh) {
    cx<double> s[12];
    SpinorIO<64>::load(a, nullptr, g.Vh, nrhs, k, h, s);
#pragma unroll
    for (int c = 0; c < 12; c++) v += norm2(s[c]);
  }
  grid_reduce<BB>(v, nrhs, red);
}

__global__ void __launch_bounds__(BB) redot_kernel(Geom g, int nrhs, const double2* a, const double2* b,
                                                   ReduceArgs red) {
  const int gid = blockIdx.x * BB + threadIdx.x;
  const int k = gid % nrhs, h = gid / nrhs;
  double v = 0.0;
  if (h < g.Vh) {
    cx<double> s[12], t[12];
    SpinorIO<64>::load(a, nullptr, g.Vh, nrhs, k, h, s);
    SpinorIO<64>::load(b, nullptr, g.Vh, nrhs, k, h, t);
#pragma unroll
    for (int c = 0; c < 12; c++) v += s[c].re * t[c].re + s[c].im * t[c].im;
  }
  grid_reduce<BB>(v, nrhs, red);
}

}  // namespace

int blas_block() { return BB; }
int blas_grid(const Geom& g, int nrhs) { return (g.Vh * nrhs + BB - 1) / BB; }

#define QCD_DISPATCH_RP(pr, pp, ...)                                  \
  do {                                                                \
    if (pr == 64 && pp == 64) { constexpr int PR = 64, PP = 64; __VA_ARGS__; } \
    else if (pr == 32 && pp == 32) { constexpr int PR = 32, PP = 32; __VA_ARGS__; } \
    else if (pr == 32 && pp == 16) { constexpr int PR = 32, PP = 16; __VA_ARGS__; } \
  } while (0)

void launch_cg_update(int prec_r, int prec_p, const Geom& g, int nrhs, void* x, float* xn, void* r, float* rn,
                      const void* p, const float* pn, const void* Ap, const float* Apn, const ReduceArgs& red,
                      const int* halt, cudaStream_t st) {
  g_kernel_launches += 1;
  const int nb = blas_grid(g, nrhs);
  QCD_DISPATCH_RP(prec_r, prec_p,
                  (cg_update_kernel<PR, PP><<<nb, BB, 0, st>>>(g, nrhs, x, xn, r, rn, p, pn, Ap, Apn, red, halt)));
}

void launch_p_update(int prec_r, int prec_p, const Geom& g, int nrhs, const void* r, const float* rn, void* p,
                     float* pn, const CGState* cg, const int* halt, cudaStream_t st) {
  g_kernel_launches += 1;
  const int nb = blas_grid(g, nrhs);
  QCD_DISPATCH_RP(prec_r, prec_p, (p_update_kernel<PR, PP><<<nb, BB, 0, st>>>(g, nrhs, r, rn, p, pn, cg, halt)));
}

void launch_accumulate_x(int prec_r, const Geom& g, int nrhs, double2* x_hi, void* x_lo, float* x_lon,
                         cudaStream_t st) {
  g_kernel_launches += 1;
  const int nb = blas_grid(g, nrhs);
  if (prec_r == 64) accumulate_x_kernel<64><<<nb, BB, 0, st>>>(g, nrhs, x_hi, x_lo, x_lon);
  else accumulate_x_kernel<32><<<nb, BB, 0, st>>>(g, nrhs, x_hi, x_lo, x_lon);
}

void launch_true_residual(int prec_r, const Geom& g, int nrhs, const double2* b, const double2* Ap, void* r_lo,
                          float* r_lon, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  const int nb = blas_grid(g, nrhs);
  if (prec_r == 64) true_residual_kernel<64><<<nb, BB, 0, st>>>(g, nrhs, b, Ap, r_lo, r_lon, red);
  else true_residual_kernel<32><<<nb, BB, 0, st>>>(g, nrhs, b, Ap, r_lo, r_lon, red);
}

void launch_norm2(const Geom& g, int nrhs, const double2* v, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  norm2_kernel<<<blas_grid(g, nrhs), BB, 0, st>>>(g, nrhs, v, red);
}

void launch_redot(const Geom& g, int nrhs, const double2* a, const double2* b, const ReduceArgs& red,
                  cudaStream_t st) {
  g_kernel_launches += 1;
  redot_kernel<<<blas_grid(g, nrhs), BB, 0, st>>>(g, nrhs, a, b, red);
}

}  // namespace qcd
