// BLAS-1 steps of the conjugate-gradient solve, fused with their reductions.
//
// Every kernel runs on a 2-D grid: blockIdx.y is the right-hand side, blockIdx.x * BB + threadIdx.x
// the site, so a warp reads consecutive sites of one RHS (RHS-major fields).  Sums are formed in
// FP64 by block_partial / grid_finish (warp shuffles -> shared memory -> per-block partials ->
// fixed-order sum in the last block), so the scalars of CG are produced on the device and the
// iteration needs no host round trip.
#include "qcd_kernels.h"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_blas)

namespace {

constexpr int BB = 256;  // block size of the BLAS kernels

template <int PR, int PP>
__global__ void __launch_bounds__(BB) p_update_kernel(Geom g, const void* r, const float* rn, void* p, float* pn,
                                                      const CGState* cg, const int* halt, const int* gate) {
  using RR = typename Real<PR>::T;
  using RP = typename Real<PP>::T;
  if ((halt && *halt) || (gate && !*gate)) return;
  const int k = blockIdx.y;
  const int h = blockIdx.x * BB + threadIdx.x;
  if (h >= g.Vh || !cg[k].active) return;
  const RR beta = RR(cg[k].beta);
  cx<RR> rs[12];
  cx<RP> ps[12];
  SpinorIO<PR>::load(r, rn, g.Vh, k, h, rs);
  SpinorIO<PP>::load(p, pn, g.Vh, k, h, ps);
  cx<RP> out[12];
#pragma unroll
  for (int c = 0; c < 12; c++) {
    out[c].re = RP(fma(beta, RR(ps[c].re), rs[c].re));
    out[c].im = RP(fma(beta, RR(ps[c].im), rs[c].im));
  }
  SpinorIO<PP>::store(p, pn, g.Vh, k, h, out);
}

template <int PR>
__global__ void __launch_bounds__(BB) accumulate_x_kernel(Geom g, double2* x_hi, void* x_lo, float* xn,
                                                          const int* gate) {
  using RR = typename Real<PR>::T;
  if (gate && !*gate) return;
  const int k = blockIdx.y;
  const int h = blockIdx.x * BB + threadIdx.x;
  if (h >= g.Vh) return;
  cx<RR> lo[12];
  cx<double> hi[12];
  SpinorIO<PR>::load(x_lo, xn, g.Vh, k, h, lo);
  SpinorIO<64>::load(x_hi, nullptr, g.Vh, k, h, hi);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    hi[c].re += double(lo[c].re);
    hi[c].im += double(lo[c].im);
    lo[c] = cmk(RR(0), RR(0));
  }
  SpinorIO<64>::store(x_hi, nullptr, g.Vh, k, h, hi);
  SpinorIO<PR>::store(x_lo, xn, g.Vh, k, h, lo);
}

template <int PR>
__global__ void __launch_bounds__(BB) true_residual_kernel(Geom g, int nrhs, const double2* b, const double2* Ap,
                                                           void* r_lo, float* rn, ReduceArgs red, const int* gate) {
  using RR = typename Real<PR>::T;
  if (gate && !*gate) return;  // every block: the reduction's counter is left untouched
  const int k = blockIdx.y;
  const int h = blockIdx.x * BB + threadIdx.x;
  double v = 0.0;
  if (h < g.Vh) {
    cx<double> bs[12], as[12];
    SpinorIO<64>::load(b, nullptr, g.Vh, k, h, bs);
    SpinorIO<64>::load(Ap, nullptr, g.Vh, k, h, as);
    cx<RR> rs[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
      const cx<double> d = bs[c] - as[c];
      v += norm2(d);
      rs[c] = cmk(RR(d.re), RR(d.im));
    }
    SpinorIO<PR>::store(r_lo, rn, g.Vh, k, h, rs);
  }
  block_partial<BB>(v, k, blockIdx.x, gridDim.x, red);
  grid_finish<BB>(nrhs, (long long)gridDim.x * gridDim.y, gridDim.x, red);
}

__global__ void debug_index_probe_kernel(Geom g, const double2* buf, double* out) {
  cx<double> s[12];
  SpinorIO<64>::load(buf, nullptr, g.Vh, 0, g.Vh, s);
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < 12; c++) t += s[c].re + s[c].im;
  *out = t;
}

__global__ void __launch_bounds__(BB) norm2_kernel(Geom g, int nrhs, const double2* a, ReduceArgs red) {
  const int k = blockIdx.y;
  const int h = blockIdx.x * BB + threadIdx.x;
  double v = 0.0;
  if (h < g.Vh) {
    cx<double> s[12];
    SpinorIO<64>::load(a, nullptr, g.Vh, k, h, s);
#pragma unroll
    for (int c = 0; c < 12; c++) v += norm2(s[c]);
  }
  block_partial<BB>(v, k, blockIdx.x, gridDim.x, red);
  grid_finish<BB>(nrhs, (long long)gridDim.x * gridDim.y, gridDim.x, red);
}

__global__ void __launch_bounds__(BB) redot_kernel(Geom g, int nrhs, const double2* a, const double2* b,
                                                   ReduceArgs red) {
  const int k = blockIdx.y;
  const int h = blockIdx.x * BB + threadIdx.x;
  double v = 0.0;
  if (h < g.Vh) {
    cx<double> s[12], t[12];
    SpinorIO<64>::load(a, nullptr, g.Vh, k, h, s);
    SpinorIO<64>::load(b, nullptr, g.Vh, k, h, t);
#pragma unroll
    for (int c = 0; c < 12; c++) v += s[c].re * t[c].re + s[c].im * t[c].im;
  }
  block_partial<BB>(v, k, blockIdx.x, gridDim.x, red);
  grid_finish<BB>(nrhs, (long long)gridDim.x * gridDim.y, gridDim.x, red);
}

// per parity (blockIdx.y), the sum of the 2 * Vh doubles v[p][0 .. 2 Vh) (two chiral blocks per site)
__global__ void __launch_bounds__(BB) parity_sum_kernel(Geom g, const double* v, ReduceArgs red) {
  const int p = blockIdx.y;
  const int j = blockIdx.x * BB + threadIdx.x;
  const double x = j < 2 * g.Vh ? v[(size_t)p * 2 * g.Vh + j] : 0.0;
  block_partial<BB>(x, p, blockIdx.x, gridDim.x, red);
  grid_finish<BB>(2, (long long)gridDim.x * gridDim.y, gridDim.x, red);
}

// y = a x + b y over n complex numbers
__global__ void __launch_bounds__(BB) axpby_kernel(size_t n, double a, const double2* x, double b, double2* y) {
  const size_t j = (size_t)blockIdx.x * BB + threadIdx.x;
  if (j >= n) return;
  const double2 u = x[j], w = y[j];
  y[j] = make_double2(fma(a, u.x, b * w.x), fma(a, u.y, b * w.y));
}

__global__ void gate_clear_kernel(int* gate) { *gate = 0; }

dim3 grid2(const Geom& g, int nrhs) { return dim3((g.Vh + BB - 1) / BB, nrhs); }

// x_lo += alpha p, r_lo -= alpha Ap with alpha from the CG state, |r_lo|^2 -> reduction (the update the
// fused EPI_XPAY_CG epilogue performs, as a separate pass for the t-slab solve)
template <int PR, int PP>
__global__ void __launch_bounds__(BB) xr_update_kernel(Geom g, int nrhs, void* x_lo, void* r_lo, const void* p,
                                                       const float* pn, const void* ap, const float* apn,
                                                       const CGState* cg, ReduceArgs red) {
  using RR = typename Real<PR>::T;
  using RP = typename Real<PP>::T;
  const int k = blockIdx.y;
  const int h = blockIdx.x * BB + threadIdx.x;
  double v = 0.0;
  if (h < g.Vh && cg[k].active) {
    const RR al = RR(cg[k].alpha);
    cx<RR> xs[12], rs[12];
    cx<RP> ps[12], as[12];
    SpinorIO<PR>::load(x_lo, nullptr, g.Vh, k, h, xs);
    SpinorIO<PR>::load(r_lo, nullptr, g.Vh, k, h, rs);
    SpinorIO<PP>::load(p, pn, g.Vh, k, h, ps);
    SpinorIO<PP>::load(ap, apn, g.Vh, k, h, as);
    RR n = RR(0);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      xs[c].re = fma(al, RR(ps[c].re), xs[c].re);
      xs[c].im = fma(al, RR(ps[c].im), xs[c].im);
      rs[c].re = fma(-al, RR(as[c].re), rs[c].re);
      rs[c].im = fma(-al, RR(as[c].im), rs[c].im);
      n = fma(rs[c].re, rs[c].re, n);
      n = fma(rs[c].im, rs[c].im, n);
    }
    v = double(n);
    SpinorIO<PR>::store(x_lo, nullptr, g.Vh, k, h, xs);
    SpinorIO<PR>::store(r_lo, nullptr, g.Vh, k, h, rs);
  }
  block_partial<BB>(v, k, blockIdx.x, gridDim.x, red);
  grid_finish<BB>(nrhs, (long long)gridDim.x * gridDim.y, gridDim.x, red);
}

// the finalisation a reducing kernel's last block performs, run on totals summed elsewhere (over the
// slabs of a time decomposition): finalize_total for each RHS, then, after a true residual, the halt
// word as grid_finish leaves it
__global__ void finalize_kernel(ReduceArgs red, const double* totals, int nrhs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int r = 0; r < nrhs; r++) finalize_total(red, r, totals[r]);
  if (red.mode == FIN_CG_TRUE) {
    int any = 0;
    for (int r = 0; r < nrhs; r++) any |= red.cg[r].active;
    red.ctl->halt = (any && !red.ctl->nan) ? 0 : 1;
  }
}

}  // namespace

void launch_p_update(int prec_r, int prec_p, const Geom& g, int nrhs, const void* r, const float* rn, void* p,
                     float* pn, const CGState* cg, const int* halt, cudaStream_t st, const int* gate) {
  g_kernel_launches += 1;
  if (prec_r == 64) p_update_kernel<64, 64><<<grid2(g, nrhs), BB, 0, st>>>(g, r, rn, p, pn, cg, halt, gate);
  else if (prec_p == 32) p_update_kernel<32, 32><<<grid2(g, nrhs), BB, 0, st>>>(g, r, rn, p, pn, cg, halt, gate);
  else p_update_kernel<32, 16><<<grid2(g, nrhs), BB, 0, st>>>(g, r, rn, p, pn, cg, halt, gate);
}

void launch_accumulate_x(int prec_r, const Geom& g, int nrhs, double2* x_hi, void* x_lo, float* x_lon,
                         cudaStream_t st, const int* gate) {
  g_kernel_launches += 1;
  if (prec_r == 64) accumulate_x_kernel<64><<<grid2(g, nrhs), BB, 0, st>>>(g, x_hi, x_lo, x_lon, gate);
  else accumulate_x_kernel<32><<<grid2(g, nrhs), BB, 0, st>>>(g, x_hi, x_lo, x_lon, gate);
}

void launch_debug_index_probe(const Geom& g, const double2* buf, double* out, cudaStream_t st) {
  g_kernel_launches += 1;
  debug_index_probe_kernel<<<1, 1, 0, st>>>(g, buf, out);
}

void launch_true_residual(int prec_r, const Geom& g, int nrhs, const double2* b, const double2* Ap, void* r_lo,
                          float* r_lon, const ReduceArgs& red, cudaStream_t st, const int* gate) {
  g_kernel_launches += 1;
  if (prec_r == 64) true_residual_kernel<64><<<grid2(g, nrhs), BB, 0, st>>>(g, nrhs, b, Ap, r_lo, r_lon, red, gate);
  else true_residual_kernel<32><<<grid2(g, nrhs), BB, 0, st>>>(g, nrhs, b, Ap, r_lo, r_lon, red, gate);
}

void launch_gate_clear(int* gate, cudaStream_t st) {
  g_kernel_launches += 1;
  gate_clear_kernel<<<1, 1, 0, st>>>(gate);
}

void launch_norm2(const Geom& g, int nrhs, const double2* v, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  norm2_kernel<<<grid2(g, nrhs), BB, 0, st>>>(g, nrhs, v, red);
}

void launch_parity_sum(const Geom& g, const double* v, const ReduceArgs& red, cudaStream_t st) {
  g_kernel_launches += 1;
  parity_sum_kernel<<<dim3((2 * g.Vh + BB - 1) / BB, 2), BB, 0, st>>>(g, v, red);
}

void launch_axpby(size_t n, double a, const double2* x, double b, double2* y, cudaStream_t st) {
  g_kernel_launches += 1;
  axpby_kernel<<<(unsigned)((n + BB - 1) / BB), BB, 0, st>>>(n, a, x, b, y);
}

void launch_redot(const Geom& g, int nrhs, const double2* a, const double2* b, const ReduceArgs& red,
                  cudaStream_t st) {
  g_kernel_launches += 1;
  redot_kernel<<<grid2(g, nrhs), BB, 0, st>>>(g, nrhs, a, b, red);
}

void launch_xr_update(int prec_r, int prec_p, const Geom& g, int nrhs, void* x_lo, void* r_lo, const void* p,
                      const float* pn, const void* ap, const float* apn, const CGState* cg, const ReduceArgs& red,
                      cudaStream_t st) {
  g_kernel_launches += 1;
  const dim3 grid((g.Vh + BB - 1) / BB, nrhs);
  if (prec_r == 64)
    xr_update_kernel<64, 64><<<grid, BB, 0, st>>>(g, nrhs, x_lo, r_lo, p, pn, ap, apn, cg, red);
  else if (prec_p == 32)
    xr_update_kernel<32, 32><<<grid, BB, 0, st>>>(g, nrhs, x_lo, r_lo, p, pn, ap, apn, cg, red);
  else
    xr_update_kernel<32, 16><<<grid, BB, 0, st>>>(g, nrhs, x_lo, r_lo, p, pn, ap, apn, cg, red);
}

void launch_finalize(const ReduceArgs& red, const double* totals, int nrhs, cudaStream_t st) {
  g_kernel_launches += 1;
  finalize_kernel<<<1, 32, 0, st>>>(red, totals, nrhs);
}

}  // namespace qcd
