// Wilson hopping term with spin projection, and its fused clover epilogues.
//
//   (D psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
//
// (standard Wilson-clover definition; the paper's application, Sec. 1, is MILC's
// clover_dynamical).  In the DeGrand-Rossi basis (1 -+ g_mu) has rank two: the
// lower two spin rows are fixed multiples of the upper two, so each neighbour is
// projected to a half spinor (2 spins x 3 colours), multiplied by the SU(3) link
// and expanded again.  This is the "neighbouring site" input class the paper's
// DMA engine streams (Sec. 3); here it is a coalesced structure-of-arrays gather.
#pragma once

#include <type_traits>

#include "qcd_internal.cuh"
#include "qcd_spinpair.cuh"

namespace qcd {

enum Epilogue {
  EPI_NONE = 0,        // out = D in
  EPI_CLOVER_INV = 1,  // out = C (D in)            (C = A^-1 of the output parity)
  EPI_XPAY = 2,        // out = C x + a (D in)      (C = A of the output parity)
  EPI_XPAY_CG = 3,     // Ap = C x + a (D in), not stored: x_lo += alpha p, r_lo -= alpha Ap, |r_lo|^2
};

struct DslashArgs {
  Geom g;
  int p;                   // output parity
  int nrhs;                // right-hand sides (thread index mod nrhs)
  const void* gauge;       // gauge field of this precision (both parities)
  const void* in;          // input field (parity 1-p)
  const float* in_norm;
  void* out;               // output field (parity p)
  float* out_norm;
  const void* x;           // EPI_XPAY local term (parity p)
  const float* x_norm;
  const void* clover;      // clover block field of parity p (A or A^-1)
  double a;                // EPI_XPAY coefficient on the hopping sum
  int in_g5;               // apply gamma_5 to the input before hopping
  int x_g5;                // apply gamma_5 to x before the clover multiply
  int out_g5;              // apply gamma_5 to the result
  int do_norm;             // reduce |out|^2 per RHS
  ReduceArgs red;
  const int* halt;         // non-null: return immediately when *halt != 0
  const int* gate;         // non-null: return immediately unless *gate != 0
  // EPI_XPAY_CG: the CG vectors (x_lo, r_lo in FP64 for P = 64, else FP32; p in precision P)
  void* cg_x;
  void* cg_r;
  const void* cg_p;
  const float* cg_p_norm;
  // t-slab halos (hopping kernels instantiated with HALO): the neighbouring slabs' contributions to
  // the time hops that leave this slab, one entry per site of a t-face (XYZ/2 per parity), layout of
  // HaloIO.  halo_hi: (1 - g_t) psi of the upper slab's t = 0 sites, multiplied here by U_t(x);
  // halo_lo: U_t(x - t)^dag (1 + g_t) psi of the lower slab's last time slice, already multiplied
  // and signed by the slab that sent it.
  const void* halo_lo;
  const void* halo_hi;
  // LAZY loads (the persistent FP32 iteration): the input is p' = lz_b p + lz_a r, formed where it is
  // read (p = in, r = lz_r, both FP32), so that the p update needs no pass of its own
  const void* lz_r;
  float lz_a, lz_b;
};

// Halo entries: six complex numbers (a projected half spinor) per face site and RHS, FP64 as
// [rhs][6][F] double2, FP32 and FP16 operators as [rhs][3][F] float4 (F = XYZ/2 face sites).
template <int P>
struct HaloIO {
  static constexpr int ROWS = P == 64 ? 6 : 3;
  static constexpr int BYTES = P == 64 ? 96 : 48;  // per face site and RHS
  template <typename R>
  __device__ static void load(const void* base, int F, int r, int f, cx<R> h[6]) {
    if (!dbg_check(f >= 0 && f < F && r >= 0, DBG_HALO)) {
      for (int k = 0; k < 6; k++) h[k] = {};
      return;
    }
    if (P == 64) {
      const double2* q = static_cast<const double2*>(base) + (size_t)r * 6 * F + f;
#pragma unroll
      for (int k = 0; k < 6; k++) {
        const double2 v = __ldg(q + (size_t)k * F);
        h[k] = cmk(R(v.x), R(v.y));
      }
    } else {
      const float4* q = static_cast<const float4*>(base) + (size_t)r * 3 * F + f;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const float4 v = __ldg(q + (size_t)k * F);
        h[2 * k] = cmk(R(v.x), R(v.y));
        h[2 * k + 1] = cmk(R(v.z), R(v.w));
      }
    }
  }
  template <typename R>
  __device__ static void store(void* base, int F, int r, int f, const cx<R> h[6]) {
    if (!dbg_check(f >= 0 && f < F && r >= 0, DBG_HALO)) return;
    if (P == 64) {
      double2* q = static_cast<double2*>(base) + (size_t)r * 6 * F + f;
#pragma unroll
      for (int k = 0; k < 6; k++) q[(size_t)k * F] = make_double2(double(h[k].re), double(h[k].im));
    } else {
      float4* q = static_cast<float4*>(base) + (size_t)r * 3 * F + f;
#pragma unroll
      for (int k = 0; k < 3; k++)
        q[(size_t)k * F] = make_float4(float(h[2 * k].re), float(h[2 * k].im), float(h[2 * k + 1].re),
                                       float(h[2 * k + 1].im));
    }
  }
};

// Spin projection (1 + sgn g_mu) psi -> half spinor h (spin rows 0 and 1).
// sgn = -1: forward term (1 - g_mu); sgn = +1: backward term (1 + g_mu).
template <int MU, int SGN, typename R>
__device__ __forceinline__ void project(const cx<R> s[12], cx<R> h[6]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cx<R> s0 = s[a], s1 = s[3 + a], s2 = s[6 + a], s3 = s[9 + a];
    if (MU == 0) {  // g_x: rows (i s3, i s2, -i s1, -i s0)
      h[a] = SGN < 0 ? s0 + times_mi(s3) : s0 + times_i(s3);
      h[3 + a] = SGN < 0 ? s1 + times_mi(s2) : s1 + times_i(s2);
    } else if (MU == 1) {  // g_y: rows (-s3, s2, s1, -s0)
      h[a] = SGN < 0 ? s0 + s3 : s0 - s3;
      h[3 + a] = SGN < 0 ? s1 - s2 : s1 + s2;
    } else if (MU == 2) {  // g_z: rows (i s2, -i s3, -i s0, i s1)
      h[a] = SGN < 0 ? s0 + times_mi(s2) : s0 + times_i(s2);
      h[3 + a] = SGN < 0 ? s1 + times_i(s3) : s1 + times_mi(s3);
    } else {  // g_t: rows (s2, s3, s0, s1)
      h[a] = SGN < 0 ? s0 - s2 : s0 + s2;
      h[3 + a] = SGN < 0 ? s1 - s3 : s1 + s3;
    }
  }
}

// Spin rows 2 and 3 of (1 + sgn g_mu) expanded from rows 0 and 1 (h0, h1) of one colour.
template <int MU, int SGN, typename R>
__device__ __forceinline__ void expand_rows(cx<R> h0, cx<R> h1, cx<R>& lo, cx<R>& hi) {
  if (MU == 0) {
    lo = SGN < 0 ? times_i(h1) : times_mi(h1);
    hi = SGN < 0 ? times_i(h0) : times_mi(h0);
  } else if (MU == 1) {
    lo = SGN < 0 ? -h1 : h1;
    hi = SGN < 0 ? h0 : -h0;
  } else if (MU == 2) {
    lo = SGN < 0 ? times_i(h0) : times_mi(h0);
    hi = SGN < 0 ? times_mi(h1) : times_i(h1);
  } else {
    lo = SGN < 0 ? -h0 : h0;
    hi = SGN < 0 ? -h1 : h1;
  }
}

// acc += f (expanded h) with the real factor f (the FP16 neighbour's norm, the time-boundary sign)
// folded into fused multiply-adds, one per real component, instead of a multiply and an add;
// FIRST: acc = f (expanded h).
template <int MU, int SGN, bool FIRST = false, typename R>
__device__ __forceinline__ void accumulate_scaled(const cx<R> h[6], R f, cx<R> acc[12]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (FIRST) {
      const cx<R> h0 = f * h[a], h1 = f * h[3 + a];
      cx<R> lo, hi;
      expand_rows<MU, SGN>(h0, h1, lo, hi);
      acc[a] = h0;
      acc[3 + a] = h1;
      acc[6 + a] = lo;
      acc[9 + a] = hi;
    } else {
      cx<R> lo, hi;
      expand_rows<MU, SGN>(h[a], h[3 + a], lo, hi);
      const cx<R> t[4] = {h[a], h[3 + a], lo, hi};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        acc[3 * k + a].re = fma(f, t[k].re, acc[3 * k + a].re);
        acc[3 * k + a].im = fma(f, t[k].im, acc[3 * k + a].im);
      }
    }
  }
}

// Expand the multiplied half spinor back to four spins and accumulate (FIRST: the first term of
// the sum, stored instead of added to a zero accumulator, which would cost an add per component).
template <int MU, int SGN, bool FIRST = false, typename R>
__device__ __forceinline__ void accumulate(const cx<R> h[6], cx<R> acc[12]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cx<R> h0 = h[a], h1 = h[3 + a];
    cx<R> lo, hi;  // the terms of spin rows 2 and 3
    expand_rows<MU, SGN>(h0, h1, lo, hi);
    if (FIRST) {
      acc[a] = h0;
      acc[3 + a] = h1;
      acc[6 + a] = lo;
      acc[9 + a] = hi;
    } else {
      acc[a] = acc[a] + h0;
      acc[3 + a] = acc[3 + a] + h1;
      acc[6 + a] = acc[6 + a] + lo;
      acc[9 + a] = acc[9 + a] + hi;
    }
  }
}

// out_a = sum_b U_ab v_b (both half-spinor rows)
template <typename R>
__device__ __forceinline__ void su3_mul(const cx<R> u[9], const cx<R> v[6], cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> acc = u[3 * a] * v[3 * s];
      acc = cfma(u[3 * a + 1], v[3 * s + 1], acc);
      acc = cfma(u[3 * a + 2], v[3 * s + 2], acc);
      w[3 * s + a] = acc;
    }
  }
}

// out_a = init_a + sum_b conj(U_ba) v_b (the products chained onto init)
template <typename R>
__device__ __forceinline__ void su3_adj_mul_onto(const cx<R> u[9], const cx<R> v[6], const cx<R> init[6], cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> acc = init[3 * s + a];
      acc = cfmac(u[a], v[3 * s], acc);
      acc = cfmac(u[3 + a], v[3 * s + 1], acc);
      acc = cfmac(u[6 + a], v[3 * s + 2], acc);
      w[3 * s + a] = acc;
    }
  }
}

// out_a = sum_b conj(U_ba) v_b
template <typename R>
__device__ __forceinline__ void su3_adj_mul(const cx<R> u[9], const cx<R> v[6], cx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> acc = cmk(R(0), R(0));
      acc = cfmac(u[a], v[3 * s], acc);
      acc = cfmac(u[3 + a], v[3 * s + 1], acc);
      acc = cfmac(u[6 + a], v[3 * s + 2], acc);
      w[3 * s + a] = acc;
    }
  }
}

template <typename R>
__device__ __forceinline__ void apply_g5(cx<R> s[12]) {
#pragma unroll
  for (int c = 6; c < 12; c++) s[c] = -s[c];
}

// The two links along mu used by one output site, with the neighbours' half indices and the
// time-boundary factors; loaded (and, for 12-real storage, reconstructed) once per site.
template <typename R>
struct DirLinks {
  cx<R> uf[9], ub[9];  // U_mu(x), U_mu(x - mu)
  int nbf, nbb;        // half indices of x + mu, x - mu
  R sf, sb;            // boundary factors of the two hops
  int hf, hb;          // HALO, mu = t: face index of a hop that leaves the slab forwards / backwards, else -1
};

// neighbours and boundary factors along mu (the factor t_bc belongs to the link at global time Tg-1)
template <int MU, typename R>
__device__ __forceinline__ void dir_index(const Geom& g, const Site& s, DirLinks<R>& L) {
  L.nbf = neighbor_fwd(g, s, MU) >> 1;
  L.nbb = neighbor_bwd(g, s, MU) >> 1;
  const int tg = s.t + g.t0;
  L.sf = (MU == 3 && tg == g.Tg - 1) ? R(g.t_bc) : R(1);
  L.sb = (MU == 3 && tg == 0) ? R(g.t_bc) : R(1);
  L.hf = L.hb = -1;
}

// the t-face index of a site (its half index within its time slice)
__device__ __forceinline__ int face_index(const Geom& g, const Site& s) { return (s.i - s.t * g.XYZ) >> 1; }

template <int P, int RECON, int MU>
__device__ __forceinline__ void dir_links(const DslashArgs& A, const Site& s, DirLinks<typename Real<P>::T>& L) {
  GaugeIO<P, RECON>::load(A.gauge, A.g.Vh, A.p, MU, s.i >> 1, L.uf);
  GaugeIO<P, RECON>::load(A.gauge, A.g.Vh, 1 - A.p, MU, L.nbb, L.ub);
}

template <int P, int RECON, int MU, bool HALO = false>
__device__ __forceinline__ void load_dir(const DslashArgs& A, const Site& s, DirLinks<typename Real<P>::T>& L) {
  dir_index<MU>(A.g, s, L);
  if (HALO && MU == 3) {
    // hops that leave the slab read the halos; U_t(x - t) of the backward one stays with the sender
    if (s.t == A.g.T - 1) L.hf = face_index(A.g, s);
    if (s.t == 0) L.hb = face_index(A.g, s);
    GaugeIO<P, RECON>::load(A.gauge, A.g.Vh, A.p, MU, s.i >> 1, L.uf);
    if (L.hb < 0) GaugeIO<P, RECON>::load(A.gauge, A.g.Vh, 1 - A.p, MU, L.nbb, L.ub);
  } else {
    dir_links<P, RECON, MU>(A, s, L);
  }
}

// psi_r at half index nb; returns the factor still to be applied (the FP16 per-site scale, which
// commutes with the spin projection and the link multiply, so it is applied once to the result)
template <int P, int COH, bool LAZY = false>
__device__ __forceinline__ typename Real<P>::T load_neighbor(const DslashArgs& A, int r, int nb,
                                                             cx<typename Real<P>::T> sp[12]) {
  using R = typename Real<P>::T;
  if constexpr (LAZY) {
    static_assert(P == 32, "lazy p updates serve the FP32 iteration");
    cx<float> rs[12];
    SpinorIO<32>::template load<COH>(A.in, nullptr, A.g.Vh, r, nb, sp);
    SpinorIO<32>::template load<COH>(A.lz_r, nullptr, A.g.Vh, r, nb, rs);
#pragma unroll
    for (int c = 0; c < 12; c++) {  // the p update's own expression: fma(beta, p, r)
      sp[c].re = fmaf(A.lz_b, sp[c].re, A.lz_a * rs[c].re);
      sp[c].im = fmaf(A.lz_b, sp[c].im, A.lz_a * rs[c].im);
    }
    return R(1);
  }
  if (P == 16)
    return SpinorIO<16>::template load_unscaled<COH>(A.in, A.in_norm, A.g.Vh, r, nb,
                                                     reinterpret_cast<cx<float>*>(sp));
  SpinorIO<P>::template load<COH>(A.in, A.in_norm, A.g.Vh, r, nb, sp);
  return R(1);
}

// acc += (1 - g_mu) U_mu(x) psi_r(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi_r(x-mu)  (FIRST: acc =).
// HALO (mu = t): a hop that leaves the slab takes the neighbour's projected half spinor (forward) or
// its finished contribution (backward) from the halos instead of the field.
template <int P, int MU, int COH = LD_NC, bool FIRST = false, bool HALO = false, bool FOLD = true,
          bool LAZY = false>
__device__ __forceinline__ void hop_dir(const DslashArgs& A, const DirLinks<typename Real<P>::T>& L, int r,
                                        cx<typename Real<P>::T> acc[12]) {
  using R = typename Real<P>::T;
  constexpr bool H = HALO && MU == 3;
  cx<R> sp[12], h[6], w[6];
  if constexpr (P != 16 && MU != 3 && FOLD) {
    // Unsigned, unscaled hops: the two hops along mu expand to rows 0, 1: wf + wb and rows 2, 3:
    // L(wf) - L(wb) = L(wf - wb), with L the fixed +-1 / +-i map of the forward projector.  wb is
    // chained onto wf (s = wf + wb, no separate adds) and d = 2 wf - s, which saves 12 of the 48
    // additions of two separate expansions (FP64 M^dag M pass at 16^4: 83.6 -> 81.6 us; the FP32
    // single-RHS passes 161 -> 159 us at 32^3 x 64; the staged multi-RHS kernel, where the extra live
    // registers cost a block per SM, keeps the separate expansions: FOLD = false).
    load_neighbor<P, COH, LAZY>(A, r, L.nbf, sp);
    if (A.in_g5) apply_g5(sp);
    project<MU, -1>(sp, h);
    cx<R> wf[6];
    su3_mul(L.uf, h, wf);
    load_neighbor<P, COH, LAZY>(A, r, L.nbb, sp);
    if (A.in_g5) apply_g5(sp);
    project<MU, +1>(sp, h);
    su3_adj_mul_onto(L.ub, h, wf, w);  // w = wf + wb
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cx<R> d0, d1, lo, hi;
      d0.re = fma(R(2), wf[a].re, -w[a].re);
      d0.im = fma(R(2), wf[a].im, -w[a].im);
      d1.re = fma(R(2), wf[3 + a].re, -w[3 + a].re);
      d1.im = fma(R(2), wf[3 + a].im, -w[3 + a].im);
      expand_rows<MU, -1>(d0, d1, lo, hi);
      if (FIRST) {
        acc[a] = w[a];
        acc[3 + a] = w[3 + a];
        acc[6 + a] = lo;
        acc[9 + a] = hi;
      } else {
        acc[a] = acc[a] + w[a];
        acc[3 + a] = acc[3 + a] + w[3 + a];
        acc[6 + a] = acc[6 + a] + lo;
        acc[9 + a] = acc[9 + a] + hi;
      }
    }
    return;
  }
  R f;
  if (H && L.hf >= 0) {
    HaloIO<P>::load(A.halo_hi, A.g.XYZ / 2, r, L.hf, h);
    f = R(1);
  } else {
    f = load_neighbor<P, COH, LAZY>(A, r, L.nbf, sp);
    if (A.in_g5) apply_g5(sp);
    project<MU, -1>(sp, h);
  }
  su3_mul(L.uf, h, w);
  if (MU == 3) f *= L.sf;
  if (MU == 3 || P == 16) accumulate_scaled<MU, -1, FIRST>(w, f, acc);
  else accumulate<MU, -1, FIRST>(w, acc);
  if (H && L.hb >= 0) {
    HaloIO<P>::load(A.halo_lo, A.g.XYZ / 2, r, L.hb, w);
    accumulate<MU, +1>(w, acc);
    return;
  }
  f = load_neighbor<P, COH, LAZY>(A, r, L.nbb, sp);
  if (A.in_g5) apply_g5(sp);
  project<MU, +1>(sp, h);
  su3_adj_mul(L.ub, h, w);
  if (MU == 3) f *= L.sb;
  if (MU == 3 || P == 16) accumulate_scaled<MU, +1>(w, f, acc);
  else accumulate<MU, +1>(w, acc);
}

// acc = the two hops along mu of one output site and RHS r, links loaded here.
template <int P, int RECON, int MU, int COH, bool HALO = false, bool LAZY = false>
__device__ __forceinline__ void dir_unit(const DslashArgs& A, const Site& s, int r, cx<typename Real<P>::T> acc[12]) {
  DirLinks<typename Real<P>::T> L;
  load_dir<P, RECON, MU, HALO>(A, s, L);
  hop_dir<P, MU, COH, true, HALO, true, LAZY>(A, L, r, acc);
}

template <int P>
struct CloverPrec;
template <>
struct CloverPrec<64> { static constexpr int CP = 64; };
template <>
struct CloverPrec<32> { static constexpr int CP = 32; };
template <>
struct CloverPrec<16> { static constexpr int CP = 16; };

// Staging of the epilogue's operands.  The clover blocks, the local term x and the CG vectors of a
// unit's 32 sites do not depend on the hopping sum, so the unit starts by copying them into shared
// memory with cp.async (through L2 only); they arrive while the hops are computed and the epilogue
// reads them from shared memory.  Rows of 32 consecutive 16-byte elements, in the order: clover
// pair, x (+ 32 norms for FP16), p (+ norms), x_lo, r_lo.  FP64 units (bound by the FP64 pipe)
// load their operands directly.
template <int P, int EPI>
struct Stage {
  static constexpr bool ON = P != 64 && EPI != EPI_NONE;
  static constexpr int CL = P == 32 ? 18 : 9;               // rows of the clover pair
  static constexpr int SP = P == 32 ? 6 : 3;                // rows of a spinor of precision P
  static constexpr int SPN = SP * 32 + (P == 16 ? 8 : 0);   // elements, with the norms
  static constexpr bool XR = EPI == EPI_XPAY || EPI == EPI_XPAY_CG;
  static constexpr bool CG = EPI == EPI_XPAY_CG;
  static constexpr int OFF_X = CL * 32;
  static constexpr int OFF_P = OFF_X + (XR ? SPN : 0);
  static constexpr int OFF_CX = OFF_P + (CG ? SPN : 0);
  static constexpr int OFF_CR = OFF_CX + (CG ? 6 * 32 : 0);
  static constexpr int U4 = ON ? OFF_CR + (CG ? 6 * 32 : 0) : 1;  // uint4 elements of the buffer
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ROWS rows of 32 16-byte elements, row j read from src + j * stride; only the first n elements of
// a row (the unit's valid sites) are copied
template <int ROWS>
__device__ __forceinline__ void stage_rows(uint4* dst, const uint4* src, size_t stride, int n) {
#pragma unroll
  for (int k = 0; k < (ROWS * 32 + 127) / 128; k++) {
    const int i = threadIdx.x + 128 * k;
    if (i < ROWS * 32 && (i & 31) < n) cp_async16(dst + i, src + (size_t)(i >> 5) * stride + (i & 31));
  }
}

// a spinor of precision P (RHS r, sites hh0 .. hh0+n-1) and, for FP16, its norms
template <int P>
__device__ __forceinline__ void stage_spinor(uint4* dst, const void* base, const float* nrm, int Vh, int r, int hh0,
                                             int n) {
  constexpr int SP = P == 32 ? 6 : 3;
  stage_rows<SP>(dst, static_cast<const uint4*>(base) + sidx<SP>(0, Vh, r, hh0), Vh, n);
  // 32 norms = 8 16-byte pieces; n is a multiple of 8 (Vh is), the source 16-byte aligned
  if (P == 16 && threadIdx.x < 8 && 4 * (int)threadIdx.x < n)
    cp_async16(dst + SP * 32 + threadIdx.x, nrm + (size_t)r * Vh + hh0 + 4 * threadIdx.x);
}

// One (block of 32 output sites, RHS r) of the hopping operator on a 128-thread block: warp w
// loads the two links along mu = w and computes the two hops for its lane's site (uniform per warp,
// no divergence), the four partial sums meet in shared memory (part), warps 0 and 1 finish chiral
// block 0 and 1 (sum, clover epilogue, gamma_5, norm or CG update) and the warps share the stores.
// COH is the load mode of the spinor fields (LD_NC, or a coherent mode for a persistent kernel
// reading fields that other blocks wrote).  Returns the thread's share of |out|^2 (do_norm) or of
// |r|^2 (EPI_XPAY_CG, with cg_alpha applied when cg_active).  The epilogue's operands are staged in
// stage (Stage<P, EPI>); the clover pair only when fetch_clover (it is kept from an earlier call on
// the same sites otherwise).  All threads must call it; it synchronises the block and leaves part
// and stage free for the next call.
template <int P, int RECON, int EPI, int COH, bool HALO = false>
__device__ __forceinline__ double split_unit(const DslashArgs& A, int hh, bool valid, const Site& s, int r,
                                             bool cg_active, double cg_alpha, cx<typename Real<P>::T> (*part)[12][32],
                                             uint4* stage, bool fetch_clover) {
  using R = typename Real<P>::T;
  using ST = Stage<P, EPI>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (ST::ON) {
    const int hh0 = hh - lane, n = min(32, A.g.Vh - hh0);
    if (fetch_clover) stage_rows<ST::CL>(stage, static_cast<const uint4*>(A.clover) + hh0, A.g.Vh, n);
    if (ST::XR) stage_spinor<P>(stage + ST::OFF_X, A.x, A.x_norm, A.g.Vh, r, hh0, n);
    if (ST::CG && cg_active) {
      stage_spinor<P>(stage + ST::OFF_P, A.cg_p, A.cg_p_norm, A.g.Vh, r, hh0, n);
      stage_spinor<32>(stage + ST::OFF_CX, A.cg_x, nullptr, A.g.Vh, r, hh0, n);
      stage_spinor<32>(stage + ST::OFF_CR, A.cg_r, nullptr, A.g.Vh, r, hh0, n);
    }
    cp_async_commit();
  }
  {
    cx<R> acc[12];
    if (valid) {
      switch (w) {
        case 0: dir_unit<P, RECON, 0, COH>(A, s, r, acc); break;
        case 1: dir_unit<P, RECON, 1, COH>(A, s, r, acc); break;
        case 2: dir_unit<P, RECON, 2, COH>(A, s, r, acc); break;
        default: dir_unit<P, RECON, 3, COH, HALO>(A, s, r, acc); break;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 12; c++) acc[c] = cmk(R(0), R(0));
    }
#pragma unroll
    for (int c = 0; c < 12; c++) part[w][c][lane] = acc[c];
  }
  if (ST::ON) cp_async_wait_all();
  __syncthreads();
  double nrm = 0.0;
  const float* st_xn = reinterpret_cast<const float*>(stage + ST::OFF_X + ST::SP * 32);
  const float* st_pn = reinterpret_cast<const float*>(stage + ST::OFF_P + ST::SP * 32);
  if (w < 2 && valid) {
    const int b = w;
    cx<R> v[6], res[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const int c = 6 * b + k;
      v[k] = (part[0][c][lane] + part[1][c][lane]) + (part[2][c][lane] + part[3][c][lane]);
    }
    if (EPI == EPI_NONE) {
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = v[k];
    } else if (EPI == EPI_CLOVER_INV) {
      if (ST::ON) CloverIO<CloverPrec<P>::CP>::template apply<LD_SM>(stage, 32, lane, b, v, res);
      else CloverIO<CloverPrec<P>::CP>::apply(A.clover, A.g.Vh, hh, b, v, res);
    } else {  // EPI_XPAY, EPI_XPAY_CG
      cx<R> xs[6], cxs[6];
      if (ST::ON) SpinorIO<P>::template load_block<LD_SM>(stage + ST::OFF_X, st_xn, 32, 0, lane, b, xs);
      else SpinorIO<P>::template load_block<COH>(A.x, A.x_norm, A.g.Vh, r, hh, b, xs);
      if (A.x_g5 && b == 1) {
#pragma unroll
        for (int k = 0; k < 6; k++) xs[k] = -xs[k];
      }
      if (ST::ON) CloverIO<CloverPrec<P>::CP>::template apply<LD_SM>(stage, 32, lane, b, xs, cxs);
      else CloverIO<CloverPrec<P>::CP>::apply(A.clover, A.g.Vh, hh, b, xs, cxs);
      const R a = R(A.a);
#pragma unroll
      for (int k = 0; k < 6; k++) {
        res[k].re = fma(a, v[k].re, cxs[k].re);
        res[k].im = fma(a, v[k].im, cxs[k].im);
      }
    }
    if (A.out_g5 && b == 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = -res[k];
    }
    if (EPI == EPI_XPAY_CG) {
      // res = (A p)_b: advance x and r of this RHS with alpha from the <p, A p> reduction
      constexpr int PR = P == 64 ? 64 : 32;
      using RR = typename Real<PR>::T;
      if (cg_active) {
        const RR al = RR(cg_alpha);
        cx<R> ps[6];
        cx<RR> xs[6], rs[6];
        if (ST::ON) {
          SpinorIO<P>::template load_block<LD_SM>(stage + ST::OFF_P, st_pn, 32, 0, lane, b, ps);
          SpinorIO<PR>::template load_block<LD_SM>(stage + ST::OFF_CX, nullptr, 32, 0, lane, b, xs);
          SpinorIO<PR>::template load_block<LD_SM>(stage + ST::OFF_CR, nullptr, 32, 0, lane, b, rs);
        } else {
          SpinorIO<P>::template load_block<COH>(A.cg_p, A.cg_p_norm, A.g.Vh, r, hh, b, ps);
          SpinorIO<PR>::template load_block<COH>(A.cg_x, nullptr, A.g.Vh, r, hh, b, xs);
          SpinorIO<PR>::template load_block<COH>(A.cg_r, nullptr, A.g.Vh, r, hh, b, rs);
        }
        RR n6 = RR(0);  // the site block's |r|^2 in the precision of r (FP32 below FP64)
#pragma unroll
        for (int k = 0; k < 6; k++) {
          xs[k].re = fma(al, RR(ps[k].re), xs[k].re);
          xs[k].im = fma(al, RR(ps[k].im), xs[k].im);
          rs[k].re = fma(-al, RR(res[k].re), rs[k].re);
          rs[k].im = fma(-al, RR(res[k].im), rs[k].im);
          n6 = fma(rs[k].re, rs[k].re, n6);
          n6 = fma(rs[k].im, rs[k].im, n6);
        }
        nrm += double(n6);
        SpinorIO<PR>::store_block(A.cg_x, nullptr, A.g.Vh, r, hh, b, xs);
        SpinorIO<PR>::store_block(A.cg_r, nullptr, A.g.Vh, r, hh, b, rs);
      }
    } else {
      if (A.do_norm) {
        R n6 = R(0);
#pragma unroll
        for (int k = 0; k < 6; k++) {
          n6 = fma(res[k].re, res[k].re, n6);
          n6 = fma(res[k].im, res[k].im, n6);
        }
        nrm += double(n6);
      }
#pragma unroll
      for (int k = 0; k < 6; k++) part[0][6 * b + k][lane] = res[k];
    }
  }
  __syncthreads();
  if (valid && EPI != EPI_XPAY_CG) {
    if (P == 64) {
      double2* q = static_cast<double2*>(A.out);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const cx<R> v = part[0][3 * w + k][lane];
        q[sidx<12>(3 * w + k, A.g.Vh, r, hh)] = make_double2(double(v.re), double(v.im));
      }
    } else if (P == 32) {
      if (w < 3) {
        float4* q = static_cast<float4*>(A.out);
#pragma unroll
        for (int k = 0; k < 2; k++) {
          const cx<R> v0 = part[0][4 * w + 2 * k][lane], v1 = part[0][4 * w + 2 * k + 1][lane];
          q[sidx<6>(2 * w + k, A.g.Vh, r, hh)] =
              make_float4(float(v0.re), float(v0.im), float(v1.re), float(v1.im));
        }
      }
    } else if (w == 0) {
      cx<float> o[12];
#pragma unroll
      for (int c = 0; c < 12; c++) o[c] = cmk(float(part[0][c][lane].re), float(part[0][c][lane].im));
      SpinorIO<16>::store(A.out, A.out_norm, A.g.Vh, r, hh, o);
    }
  }
  __syncthreads();
  return nrm;
}

// ---------------------------------------------------------------------------------------------------
// Pair unit: one block of 32 output sites on two warps.  Warp d of the pair computes the four hops
// along mu = 2d and 2d + 1 for its lane's site, then finishes chiral block d (components 6d .. 6d+5):
// the two warps swap the other halves of their partial sums through shared memory, meet at one
// named barrier of the pair, and run the epilogue of their block (clover, xpay, gamma_5, norm or CG
// update) and its stores side by side, so no warp idles through the epilogue.  With two threads per
// site, a grid of 4 resident blocks per SM covers the 1024 site blocks of a 16^4 parity in one round
// (the four-warp split unit needs two).

// named barrier of the 64 threads of pair q of a block (ids 1 and 2; id 0 is __syncthreads)
__device__ __forceinline__ void pair_sync(int q) { asm volatile("bar.sync %0, 64;" ::"r"(q + 1) : "memory"); }

// Per-warp staging of the epilogue operands of one chiral block (rows of 32 16-byte elements, lane =
// site): the clover block, then the x block and, for EPI_XPAY_CG, the p block (FP16: the two uint4
// rows the block touches -- the end row, then the shared middle row -- and the 32 site norms).
template <int P, int EPI>
struct PairStage {
  static constexpr bool ON = P != 64 && EPI != EPI_NONE;
  static constexpr int CL = P == 32 ? 9 : 5;            // clover rows of one chiral block
  static constexpr int SPB = P == 32 ? 3 : 2;           // rows of one chiral block of a spinor
  static constexpr int SPBN = SPB * 32 + (P == 16 ? 8 : 0);
  static constexpr bool XR = EPI == EPI_XPAY || EPI == EPI_XPAY_CG;
  static constexpr bool CG = EPI == EPI_XPAY_CG;
  static constexpr int OFF_X = CL * 32;
  static constexpr int OFF_P = OFF_X + (XR ? SPBN : 0);
  static constexpr int U4 = ON ? OFF_P + (CG ? SPBN : 0) : 1;
};

// exchange area of one pair for one unit: the partial sums a warp passes to its partner ([block]
// [component][lane]) and, for FP16 output, each block's largest magnitude per site
template <typename R>
struct PairXch {
  cx<R> v[2][6][32];
  float mx[2][32];
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// chiral block b of a spinor of precision P (RHS 0, sites hh0 .. hh0+n-1) into a warp's staging rows;
// lane l copies site l
template <int P>
__device__ __forceinline__ void stage_spinor_block(uint4* dst, const void* base, const float* nrm, int Vh, int hh0,
                                                   int b, int lane, int n) {
  if (lane >= n) return;
  const uint4* src = static_cast<const uint4*>(base);
  if (P == 32) {
#pragma unroll
    for (int j = 0; j < 3; j++) cp_async16(dst + j * 32 + lane, src + sidx<6>(3 * b + j, Vh, 0, hh0 + lane));
  } else {
    cp_async16(dst + lane, src + sidx<3>(b == 0 ? 0 : 2, Vh, 0, hh0 + lane));
    cp_async16(dst + 32 + lane, src + sidx<3>(1, Vh, 0, hh0 + lane));
    cp_async4(reinterpret_cast<float*>(dst + 64) + lane, nrm + hh0 + lane);
  }
}

// chiral block b of a spinor staged by stage_spinor_block (the values of SpinorIO<P>::load_block)
template <int P>
__device__ __forceinline__ void staged_spinor_block(const uint4* st, int lane, int b, cx<float> s[6]) {
  if (P == 32) {
    const float4* q = reinterpret_cast<const float4*>(st);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const float4 v = q[k * 32 + lane];
      s[2 * k] = cmk(v.x, v.y);
      s[2 * k + 1] = cmk(v.z, v.w);
    }
  } else {
    const float n = reinterpret_cast<const float*>(st + 64)[lane];
    const uint4 end = st[lane], mid = st[32 + lane];
    const float2 e0 = h2f(end.x), e1 = h2f(end.y), e2 = h2f(end.z), e3 = h2f(end.w);
    if (b == 0) {
      const float2 m0 = h2f(mid.x), m1 = h2f(mid.y);
      s[0] = cmk(e0.x * n, e0.y * n);
      s[1] = cmk(e1.x * n, e1.y * n);
      s[2] = cmk(e2.x * n, e2.y * n);
      s[3] = cmk(e3.x * n, e3.y * n);
      s[4] = cmk(m0.x * n, m0.y * n);
      s[5] = cmk(m1.x * n, m1.y * n);
    } else {
      const float2 m2 = h2f(mid.z), m3 = h2f(mid.w);
      s[0] = cmk(m2.x * n, m2.y * n);
      s[1] = cmk(m3.x * n, m3.y * n);
      s[2] = cmk(e0.x * n, e0.y * n);
      s[3] = cmk(e1.x * n, e1.y * n);
      s[4] = cmk(e2.x * n, e2.y * n);
      s[5] = cmk(e3.x * n, e3.y * n);
    }
  }
}

// y = C x for chiral block b with the block's clover rows staged (FP32: 9 float4 rows; FP16: 5 uint4)
template <int P>
__device__ __forceinline__ void staged_clover_block(const uint4* st, int lane, int b, const cx<float> x[6],
                                                    cx<float> y[6]) {
  if (P == 32) {
    CloverIO<32>::template apply<LD_SM>(st, 32, lane, 0, x, y);
  } else {
    if (b == 0) CloverIO<16>::template apply_block<0, LD_SM, 0>(st, 32, lane, x, y);
    else CloverIO<16>::template apply_block<1, LD_SM, 0>(st, 32, lane, x, y);
  }
}

// the hops along mu = 2B and 2B + 1 of one output site (acc = their sum)
template <int P, int RECON, int COH, int B, bool LAZY = false>
__device__ __forceinline__ void pair_hops(const DslashArgs& A, const Site& s, cx<typename Real<P>::T> acc[12]) {
  using R = typename Real<P>::T;
  DirLinks<R> L;
  dir_unit<P, RECON, 2 * B, COH, false, LAZY>(A, s, 0, acc);
  load_dir<P, RECON, 2 * B + 1>(A, s, L);
  hop_dir<P, 2 * B + 1, COH, false, false, true, LAZY>(A, L, 0, acc);
}

// The pair unit on warp B of its pair (B is the chiral block the warp finishes; a compile-time
// constant, so that the partial sums stay in registers).
// LAZY (FP32): with EPI_CLOVER_INV the input p' = lz_b p + lz_a r is formed at every neighbour; with
// EPI_XPAY the local term x = p is replaced by p' (formed from the staged p and r blocks) and p' is
// written back over p, which completes the p update of the iteration.
template <int P, int RECON, int EPI, int COH, int B, bool LAZY = false>
__device__ __forceinline__ float pair_unit_b(const DslashArgs& A, int hh, bool valid, const Site& s, int q,
                                             bool cg_active, double cg_alpha, PairXch<float>* xch, uint4* stage) {
  static_assert(P == 32 || P == 16, "the pair unit serves the FP32 and FP16 inner iteration");
  static_assert(!LAZY || (P == 32 && (EPI == EPI_CLOVER_INV || EPI == EPI_XPAY)), "lazy p: FP32 phases 1, 2");
  constexpr bool LZ_HOPS = LAZY && EPI == EPI_CLOVER_INV, LZ_X = LAZY && EPI == EPI_XPAY;
  using ST = PairStage<P, EPI>;
  constexpr int b = B;
  const int lane = threadIdx.x & 31;
  const int Vh = A.g.Vh;
  if (ST::ON) {
    const int hh0 = hh - lane, n = min(32, Vh - hh0);
    if (lane < n) {
      const uint4* cl = static_cast<const uint4*>(A.clover);
      if (P == 32) {
#pragma unroll
        for (int j = 0; j < 9; j++) cp_async16(stage + j * 32 + lane, cl + (size_t)(9 * b + j) * Vh + hh0 + lane);
      } else {
#pragma unroll
        for (int j = 0; j < 5; j++) cp_async16(stage + j * 32 + lane, cl + (size_t)(4 * b + j) * Vh + hh0 + lane);
      }
    }
    if (ST::XR) stage_spinor_block<P>(stage + ST::OFF_X, A.x, A.x_norm, Vh, hh0, b, lane, n);
    if (ST::CG && cg_active) stage_spinor_block<P>(stage + ST::OFF_P, A.cg_p, A.cg_p_norm, Vh, hh0, b, lane, n);
    // (the warp's rows are sized for EPI_XPAY_CG, whose p rows follow x: r takes their place here)
    if (LZ_X) stage_spinor_block<32>(stage + ST::OFF_X + ST::SPBN, A.lz_r, nullptr, Vh, hh0, b, lane, n);
    cp_async_commit();
  }
  cx<float> acc[12];
  if (valid) {
    pair_hops<P, RECON, COH, B, LZ_HOPS>(A, s, acc);
  } else {
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = cmk(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < 6; k++) xch->v[1 - b][k][lane] = acc[6 * (1 - b) + k];
  if (ST::ON) cp_async_wait_all();
  pair_sync(q);
  float nrm = 0.f;
  cx<float> res[6];
  if (valid) {
    cx<float> v[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = acc[6 * b + k] + xch->v[b][k][lane];
    if (EPI == EPI_NONE) {
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = v[k];
    } else if (EPI == EPI_CLOVER_INV) {
      staged_clover_block<P>(stage, lane, b, v, res);
    } else {  // EPI_XPAY, EPI_XPAY_CG
      cx<float> xs[6], cxs[6];
      staged_spinor_block<P>(stage + ST::OFF_X, lane, b, xs);
      if (LZ_X) {
        cx<float> rs[6];
        staged_spinor_block<32>(stage + ST::OFF_X + ST::SPBN, lane, b, rs);
#pragma unroll
        for (int k = 0; k < 6; k++) {
          xs[k].re = fmaf(A.lz_b, xs[k].re, A.lz_a * rs[k].re);
          xs[k].im = fmaf(A.lz_b, xs[k].im, A.lz_a * rs[k].im);
        }
        SpinorIO<32>::store_block(const_cast<void*>(A.x), nullptr, Vh, 0, hh, b, xs);
      }
      if (A.x_g5 && b == 1) {
#pragma unroll
        for (int k = 0; k < 6; k++) xs[k] = -xs[k];
      }
      staged_clover_block<P>(stage, lane, b, xs, cxs);
      const float a = float(A.a);
#pragma unroll
      for (int k = 0; k < 6; k++) {
        res[k].re = fmaf(a, v[k].re, cxs[k].re);
        res[k].im = fmaf(a, v[k].im, cxs[k].im);
      }
    }
    if (A.out_g5 && b == 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = -res[k];
    }
    if (EPI == EPI_XPAY_CG) {
      // res = (A p)_b: advance x and r (FP32) of this RHS with alpha from the <p, A p> reduction
      if (cg_active) {
        const float al = float(cg_alpha);
        cx<float> ps[6], xs[6], rs[6];
        staged_spinor_block<P>(stage + ST::OFF_P, lane, b, ps);
        SpinorIO<32>::template load_block<COH>(A.cg_x, nullptr, Vh, 0, hh, b, xs);
        SpinorIO<32>::template load_block<COH>(A.cg_r, nullptr, Vh, 0, hh, b, rs);
#pragma unroll
        for (int k = 0; k < 6; k++) {
          xs[k].re = fmaf(al, ps[k].re, xs[k].re);
          xs[k].im = fmaf(al, ps[k].im, xs[k].im);
          rs[k].re = fmaf(-al, res[k].re, rs[k].re);
          rs[k].im = fmaf(-al, res[k].im, rs[k].im);
          nrm = fmaf(rs[k].re, rs[k].re, nrm);
          nrm = fmaf(rs[k].im, rs[k].im, nrm);
        }
        SpinorIO<32>::store_block(A.cg_x, nullptr, Vh, 0, hh, b, xs);
        SpinorIO<32>::store_block(A.cg_r, nullptr, Vh, 0, hh, b, rs);
      }
    } else {
      if (A.do_norm) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
          nrm = fmaf(res[k].re, res[k].re, nrm);
          nrm = fmaf(res[k].im, res[k].im, nrm);
        }
      }
      if (P == 32) SpinorIO<32>::store_block(A.out, nullptr, Vh, 0, hh, b, res);
    }
  }
  if (P == 16 && EPI != EPI_XPAY_CG) {
    // the FP16 site norm is the largest magnitude over both blocks: swap the blocks' maxima
    float m = 0.f;
    if (valid) {
#pragma unroll
      for (int k = 0; k < 6; k++) m = fmaxf(m, fmaxf(fabsf(res[k].re), fabsf(res[k].im)));
    }
    xch->mx[b][lane] = m;
    pair_sync(q);
    if (valid) {
      m = fmaxf(m, xch->mx[1 - b][lane]);
      const float inv = m > 0.f ? 1.0f / m : 0.f;
      uint4* o = static_cast<uint4*>(A.out);
      // block 0: uint4 row 0 and the first half of row 1; block 1: the second half of row 1 and row 2
      const uint2 half1 = b == 0 ? make_uint2(f2h(res[4].re * inv, res[4].im * inv), f2h(res[5].re * inv, res[5].im * inv))
                                 : make_uint2(f2h(res[0].re * inv, res[0].im * inv), f2h(res[1].re * inv, res[1].im * inv));
      const int o0 = b == 0 ? 0 : 2;  // first of the four components that fill a whole row
      uint4 full;
      full.x = f2h(res[o0].re * inv, res[o0].im * inv);
      full.y = f2h(res[o0 + 1].re * inv, res[o0 + 1].im * inv);
      full.z = f2h(res[o0 + 2].re * inv, res[o0 + 2].im * inv);
      full.w = f2h(res[o0 + 3].re * inv, res[o0 + 3].im * inv);
      o[sidx<3>(b == 0 ? 0 : 2, Vh, 0, hh)] = full;
      reinterpret_cast<uint2*>(o + sidx<3>(1, Vh, 0, hh))[b] = half1;
      if (b == 0) A.out_norm[hh] = m;
    }
  }
  return nrm;
}

// One pair unit (RHS 0) on warp d of pair q: returns the thread's share of |out|^2 (do_norm) or of
// |r|^2 (EPI_XPAY_CG, with cg_alpha applied when cg_active), summed in FP32 over the site's
// components.  xch: the pair's exchange area for this unit (alternate two per pair between units, so
// that one barrier per unit suffices); stage: the warp's PairStage<P, EPI> rows.  P is 32 or 16.
template <int P, int RECON, int EPI, int COH, bool LAZY = false>
__device__ __forceinline__ float pair_unit(const DslashArgs& A, int hh, bool valid, const Site& s, int d, int q,
                                           bool cg_active, double cg_alpha, PairXch<float>* xch, uint4* stage) {
  if (d == 0)
    return pair_unit_b<P, RECON, EPI, COH, 0, LAZY>(A, hh, valid, s, q, cg_active, cg_alpha, xch, stage);
  return pair_unit_b<P, RECON, EPI, COH, 1, LAZY>(A, hh, valid, s, q, cg_active, cg_alpha, xch, stage);
}

// FP64 pair unit: the hopping operator for one block of 32 output sites on a 64-thread block, warp B
// computing the four hops along mu = 2B, 2B+1 of RHS r and finishing chiral block B (epilogue and
// stores) after the two warps swap half of their partial sums.  Used by the standalone FP64 hopping
// kernel (the reliable updates' passes): with two threads per site and 64-thread blocks, 8 blocks per
// SM hold the 1024 site blocks of a 16^4 parity in one wave, where 128-thread blocks of four warps at 4
// per SM needed 1.7 (the FP64 pipe idled through the second wave's partly filled SMs).
template <int RECON, int EPI, int B>
__device__ __forceinline__ double pair_unit64_b(const DslashArgs& A, int hh, bool valid, const Site& s, int r,
                                                cx<double> (*xch)[6][32]) {
  constexpr int b = B;
  const int lane = threadIdx.x & 31;
  const int Vh = A.g.Vh;
  cx<double> acc[12];
  if (valid) {
    DirLinks<double> L;
    load_dir<64, RECON, 2 * B>(A, s, L);
    hop_dir<64, 2 * B, LD_NC, true>(A, L, r, acc);
    load_dir<64, RECON, 2 * B + 1>(A, s, L);
    hop_dir<64, 2 * B + 1, LD_NC>(A, L, r, acc);
  } else {
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = cmk(0.0, 0.0);
  }
#pragma unroll
  for (int k = 0; k < 6; k++) xch[1 - b][k][lane] = acc[6 * (1 - b) + k];
  __syncthreads();
  double nrm = 0.0;
  if (valid) {
    cx<double> v[6], res[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = acc[6 * b + k] + xch[b][k][lane];
    if (EPI == EPI_NONE) {
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = v[k];
    } else if (EPI == EPI_CLOVER_INV) {
      CloverIO<64>::apply(A.clover, Vh, hh, b, v, res);
    } else {
      cx<double> xs[6], cxs[6];
      SpinorIO<64>::load_block(A.x, nullptr, Vh, r, hh, b, xs);
      if (A.x_g5 && b == 1) {
#pragma unroll
        for (int k = 0; k < 6; k++) xs[k] = -xs[k];
      }
      CloverIO<64>::apply(A.clover, Vh, hh, b, xs, cxs);
#pragma unroll
      for (int k = 0; k < 6; k++) {
        res[k].re = fma(A.a, v[k].re, cxs[k].re);
        res[k].im = fma(A.a, v[k].im, cxs[k].im);
      }
    }
    if (A.out_g5 && b == 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) res[k] = -res[k];
    }
    if (A.do_norm) {
#pragma unroll
      for (int k = 0; k < 6; k++) {
        nrm = fma(res[k].re, res[k].re, nrm);
        nrm = fma(res[k].im, res[k].im, nrm);
      }
    }
    SpinorIO<64>::store_block(A.out, nullptr, Vh, r, hh, b, res);
  }
  __syncthreads();  // the exchange area is rewritten by the next RHS
  return nrm;
}

// Standalone FP64 hopping kernel on pair units (epilogues EPI_NONE, EPI_CLOVER_INV, EPI_XPAY), looping
// over the RHS; one 64-thread block per 32 output sites.
template <int RECON, int EPI>
__global__ void __launch_bounds__(64, 8) dslash_pair64_kernel(DslashArgs A) {
  __shared__ cx<double> xch[2][6][32];
  if ((A.halt && *A.halt) || (A.gate && !*A.gate)) return;
  const int hh = blockIdx.x * 32 + (threadIdx.x & 31);
  const bool valid = hh < A.g.Vh;
  Site s;
  if (valid) s = site_of(A.g, A.p, hh);
  for (int r = 0; r < A.nrhs; r++) {
    const double nrm = (threadIdx.x >> 5) == 0 ? pair_unit64_b<RECON, EPI, 0>(A, hh, valid, s, r, xch)
                                                : pair_unit64_b<RECON, EPI, 1>(A, hh, valid, s, r, xch);
    if (A.do_norm) block_partial<64>(nrm, r, blockIdx.x, gridDim.x, A.red);
  }
  if (A.do_norm) grid_finish<64>(A.nrhs, gridDim.x, gridDim.x, A.red);
}

// The 32-site block that block b of a staged FP32 multi-RHS launch takes: the lattice in chunks of TC
// time slices, each chunk z plane by z plane and, within a plane, slice by slice.  A neighbour spinor
// is read by the blocks of its own slice and of the slices above and below: in lexicographic block
// order those reads lie a whole slice of blocks apart on either side (1024 blocks at 32^3 x 64, where
// 8 RHS of FP32 spinors, links and clover stream 72 MB through L2 in between, and about half of the
// input lines were read from DRAM twice), here 2 TC plane rows apart except across chunk boundaries
// (8 RHS: 689.9 -> 669.4 us at 32^3 x 64, 648.8 -> 635.5 us at 32^3 x 60).  FP16, whose 8-RHS launch
// reads every byte once in lexicographic order, keeps that order (622 against 646 us in this one).
// The identity unless a z plane holds whole blocks and TC > 1 divides T; a permutation of the blocks
// either way (qcd_selftest_site_order checks it on the host).
__host__ __device__ __forceinline__ int site_block_order(const Geom& g, int b) {
  const int plane = g.XY >> 1;  // half sites per z plane
  if (plane & 31) return b;
  int tc = 16;
  while (tc > 1 && g.T % tc) tc >>= 1;
  if (tc == 1) return b;
  const int bz = plane >> 5;
  const int q = b % bz, r1 = b / bz, ti = r1 % tc, r2 = r1 / tc, z = r2 % g.Z, c = r2 / g.Z;
  return ((c * tc + ti) * g.Z + z) * bz + q;
}

// Site of a lane in the block of 32 sites starting at 32 * sb.
__device__ __forceinline__ void split_prologue(const DslashArgs& A, int sb, int& hh, bool& valid, Site& s) {
  hh = sb * 32 + (threadIdx.x & 31);
  valid = hh < A.g.Vh;
  if (valid) s = site_of(A.g, A.p, hh);
}

// Hopping kernel: one block per 32 output sites, looping over the right-hand sides (used for one
// RHS, and for several in FP64; with HALO, for the sites of a t-slab).
template <int P, int RECON, int EPI, bool HALO = false>
__device__ __forceinline__ void dslash_split_body(const DslashArgs& A) {
  using R = typename Real<P>::T;
  __shared__ cx<R> part[4][12][32];
  __shared__ uint4 stage[Stage<P, EPI>::U4];
  if ((A.halt && *A.halt) || (A.gate && !*A.gate)) return;
  int hh;
  bool valid;
  Site s;
  split_prologue(A, blockIdx.x, hh, valid, s);
  const bool reduce = A.do_norm || EPI == EPI_XPAY_CG;
  for (int r = 0; r < A.nrhs; r++) {
    bool act = false;
    double al = 0.0;
    if (EPI == EPI_XPAY_CG) {
      act = A.red.cg[r].active != 0;
      al = A.red.cg[r].alpha;
    }
    const double nrm =
        split_unit<P, RECON, EPI, LD_NC, HALO>(A, hh, valid, s, r, act, al, part, stage, r == 0);
    if (reduce) block_partial<128>(nrm, r, blockIdx.x, gridDim.x, A.red);
  }
  if (reduce) grid_finish<128>(A.nrhs, gridDim.x, gridDim.x, A.red);
}

template <int P, int RECON, int EPI, bool HALO = false>
__global__ void __launch_bounds__(128) dslash_split_kernel(DslashArgs A) {
  dslash_split_body<P, RECON, EPI, HALO>(A);
}

// Staged copies of the site kernel: per site, the 8 links (2 mu, 2 mu + 1: forward, backward) as 10
// complex numbers each (9 and a pad, so that every link starts on 16 bytes) and the clover pair's 72
// values, each site's run padded by 16 bytes so that the 16-byte reads of eight consecutive lanes hit
// distinct banks.
constexpr int STG_LINK_STRIDE = 8 * 20 + 4;  // floats per site of the staged links
constexpr int STG_CLOVER_STRIDE = 72 + 4;     // floats per site of the staged clover pair

// link j (= 2 mu for U_mu(x), 2 mu + 1 for U_mu(x - mu)) of the site in `lane`
template <typename R>
__device__ __forceinline__ void staged_link(const float* sl, int lane, int j, cx<R> u[9]) {
  const float4* q = reinterpret_cast<const float4*>(sl + lane * STG_LINK_STRIDE + 20 * j);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const float4 v = q[k];
    u[2 * k] = cmk(R(v.x), R(v.y));
    u[2 * k + 1] = cmk(R(v.z), R(v.w));
  }
  const float2 v = *reinterpret_cast<const float2*>(q + 4);
  u[8] = cmk(R(v.x), R(v.y));
}

// y = C x for chiral block b of a staged clover pair (values 36 b .. 36 b + 35 of the site's run: 6
// diagonal reals, then 15 strictly-lower complex)
template <typename R>
__device__ __forceinline__ void clover_apply_smem(const float* scl, int lane, int b, const cx<R> x[6], cx<R> y[6]) {
  const float4* q = reinterpret_cast<const float4*>(scl + lane * STG_CLOVER_STRIDE + 36 * b);
  float f[36];
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const float4 v = q[k];
    f[4 * k] = v.x;
    f[4 * k + 1] = v.y;
    f[4 * k + 2] = v.z;
    f[4 * k + 3] = v.w;
  }
  R d[6];
  cx<R> L[15];
#pragma unroll
  for (int i = 0; i < 6; i++) d[i] = R(f[i]);
#pragma unroll
  for (int k = 0; k < 15; k++) L[k] = cmk(R(f[6 + 2 * k]), R(f[7 + 2 * k]));
  hermitian6_accumulate(d, L, x, y);
}

// The eight hops of FP16 site s and RHS r on spin-paired registers (qcd_spinpair.cuh); STAGED: the
// block's links staged as broadcast pairs at lks (the site's run), else loaded here.
template <int RECON, bool STAGED>
__device__ __forceinline__ void hops_fp16_sp(const DslashArgs& A, const Site& s, int r, const float4* lks,
                                             cx<float> acc[12]) {
  const float g = A.in_g5 ? -1.f : 1.f;
  const float2 SG[4] = {make_float2(g, g), make_float2(g, -g), make_float2(-g, g), make_float2(-g, -g)};
  const float2 M1 = make_float2(-1.f, -1.f);
  const int Vh = A.g.Vh;
  SpAcc sa;
  auto dir = [&](auto mu_c, auto f01_c, auto f23_c) {
    constexpr int MU = decltype(mu_c)::value;
    constexpr bool F01 = decltype(f01_c)::value, F23 = decltype(f23_c)::value;
    DirLinks<float> L;
    dir_index<MU>(A.g, s, L);
    SpinorIO<16>::Raw qf, qb;
    load_nb_sp(A.in, A.in_norm, Vh, r, L.nbf, qf);
    load_nb_sp(A.in, A.in_norm, Vh, r, L.nbb, qb);
    if constexpr (STAGED) {
      hop_sp<MU, -1, F01, F23>(qf, StagedLinkSp{lks + 18 * MU}, L.sf, SG, M1, sa);
      hop_sp<MU, +1, false, false>(qb, StagedLinkSp{lks + 18 * MU + 9}, L.sb, SG, M1, sa);
    } else {
      GaugeIO<16, RECON>::load(A.gauge, Vh, A.p, MU, s.i >> 1, L.uf);
      GaugeIO<16, RECON>::load(A.gauge, Vh, 1 - A.p, MU, L.nbb, L.ub);
      hop_sp<MU, -1, F01, F23>(qf, RegLinkSp{L.uf}, L.sf, SG, M1, sa);
      hop_sp<MU, +1, false, false>(qb, RegLinkSp{L.ub}, L.sb, SG, M1, sa);
    }
  };
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using BT = std::true_type;
  using BF = std::false_type;
  if constexpr (!STAGED) {
    // links and neighbours of two directions in flight: those of mu + 1 are fetched before the
    // arithmetic of mu (32^3 x 64, 1 RHS: 107 -> 103 us at 4 blocks of 128 registers per SM; at 5
    // blocks of 96 registers 105 us, without the prefetch 107 us)
    using GIO = GaugeIO<16, RECON>;
    struct DirRaw {
      SpinorIO<16>::Raw qf, qb;
      typename GIO::Raw lf, lb;
    };
    DirLinks<float> L[4];
    auto fetch = [&](auto mu_c, DirRaw& d) {
      constexpr int MU = decltype(mu_c)::value;
      dir_index<MU>(A.g, s, L[MU]);
      load_nb_sp(A.in, A.in_norm, Vh, r, L[MU].nbf, d.qf);
      load_nb_sp(A.in, A.in_norm, Vh, r, L[MU].nbb, d.qb);
      GIO::load_raw(A.gauge, Vh, A.p, MU, s.i >> 1, d.lf);
      GIO::load_raw(A.gauge, Vh, 1 - A.p, MU, L[MU].nbb, d.lb);
    };
    auto compute = [&](auto mu_c, auto f01_c, auto f23_c, const DirRaw& d) {
      constexpr int MU = decltype(mu_c)::value;
      constexpr bool F01 = decltype(f01_c)::value, F23 = decltype(f23_c)::value;
      cx<float> u[9];
      GIO::decode(d.lf, u);
      hop_sp<MU, -1, F01, F23>(d.qf, RegLinkSp{u}, L[MU].sf, SG, M1, sa);
      GIO::decode(d.lb, u);
      hop_sp<MU, +1, false, false>(d.qb, RegLinkSp{u}, L[MU].sb, SG, M1, sa);
    };
    DirRaw d0, d1;
    fetch(I0(), d0);
    fetch(I1(), d1);
    compute(I0(), BT(), BF(), d0);
    fetch(I2(), d0);
    compute(I1(), BF(), BF(), d1);
    fetch(I3(), d1);
    compute(I2(), BF(), BT(), d0);
    compute(I3(), BF(), BF(), d1);
    sp_unpack(sa, acc);
    return;
  }
  dir(I0(), BT(), BF());
  dir(I1(), BF(), BF());
  dir(I2(), BF(), BT());
  dir(I3(), BF(), BF());
  sp_unpack(sa, acc);
}

// Hopping kernel with one thread per (site, RHS).  A block of four warps covers 32 sites (64 when
// nrhs = 2: two site groups of two warps; 128 when nrhs = 1: four groups of one warp); warp k of a
// site group takes RHS k, k + W, ... (W warps per group) and computes all eight hops and the
// epilogue of its RHS, with no block barrier.  The links and the clover pair of the block's sites
// are the same for every RHS: with STAGED (nrhs >= 3, one site group) the block decodes them once
// (12-real links reconstructed, FP16 converted) into shared memory; otherwise every warp reads them
// through L1.  Sums are reduced per warp into the partial slot of (RHS, site group).
template <int P, int RECON, int EPI, bool STAGED>
__device__ __forceinline__ void dslash_site_body(const DslashArgs& A) {
  using R = typename Real<P>::T;
  constexpr int CP = CloverPrec<P>::CP;
  constexpr int PR = P == 64 ? 64 : 32;
  using RR = typename Real<PR>::T;
  // (staging the clover pair as well as the links: 8 RHS FP32 on 32^3 x 64 757 -> 707 us)
  constexpr bool SCL = STAGED && EPI != EPI_NONE;
  static_assert(!STAGED || P != 64, "staging holds FP32 values");
  // [site][link][10 complex]; FP16: [site][link][9 entries as (re, re, im, im)] (spin-paired hops)
  constexpr int LSTRIDE = P == 16 ? SP_LINK_STRIDE : STG_LINK_STRIDE;
  __shared__ __align__(16) float sl[STAGED ? 32 * LSTRIDE : 4];
  __shared__ __align__(16) float scl[SCL ? 32 * STG_CLOVER_STRIDE : 4];     // [site][72 values]
  if ((A.halt && *A.halt) || (A.gate && !*A.gate)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int G = STAGED ? 1 : (A.nrhs == 1 ? 4 : (A.nrhs == 2 ? 2 : 1)), W = 4 / G;
  const int grp = w / W, k = w - grp * W;
  const int sbk = STAGED && P == 32 ? site_block_order(A.g, blockIdx.x) : (int)blockIdx.x;
  const int hh = (sbk * G + grp) * 32 + lane;
  const bool valid = hh < A.g.Vh;
  const int Vh = A.g.Vh;
  if (STAGED) {
    for (int it = threadIdx.x; it < 8 * 32; it += 128) {
      const int j = it >> 5, l = it & 31, hs = sbk * 32 + l, mu = j >> 1;
      if (hs < Vh) {
        const Site ss = site_of(A.g, A.p, hs);
        cx<R> u[9];
        if ((j & 1) == 0) GaugeIO<P, RECON>::load(A.gauge, Vh, A.p, mu, ss.i >> 1, u);
        else GaugeIO<P, RECON>::load(A.gauge, Vh, 1 - A.p, mu, neighbor_bwd(A.g, ss, mu) >> 1, u);
        if (P == 16) {
          float4* q = reinterpret_cast<float4*>(sl + l * LSTRIDE + 36 * j);
#pragma unroll
          for (int e = 0; e < 9; e++)
            q[e] = make_float4(float(u[e].re), float(u[e].re), float(u[e].im), float(u[e].im));
        } else {
          float4* q = reinterpret_cast<float4*>(sl + l * LSTRIDE + 20 * j);
#pragma unroll
          for (int e = 0; e < 4; e++)
            q[e] = make_float4(float(u[2 * e].re), float(u[2 * e].im), float(u[2 * e + 1].re), float(u[2 * e + 1].im));
          *reinterpret_cast<float2*>(q + 4) = make_float2(float(u[8].re), float(u[8].im));
        }
      }
    }
    if (SCL) {
      const int hs0 = sbk * 32;
      if (CP == 32) {
        const float4* q = static_cast<const float4*>(A.clover);
        for (int it = threadIdx.x; it < 18 * 32; it += 128) {
          const int v = it >> 5, l = it & 31;  // float4 v = 9 b + k of the pair
          if (hs0 + l < Vh)  // float4 v holds values 4 v .. 4 v + 3 of the pair (block v / 9)
            *reinterpret_cast<float4*>(scl + l * STG_CLOVER_STRIDE + 4 * v) = __ldg(q + (size_t)v * Vh + hs0 + l);
        }
      } else {
        const uint4* q = static_cast<const uint4*>(A.clover);
        for (int it = threadIdx.x; it < 9 * 32; it += 128) {
          const int v = it >> 5, l = it & 31;  // halves 8 v .. 8 v + 7 of the site's 72
          if (hs0 + l < Vh) {
            const uint4 f = __ldg(q + (size_t)v * Vh + hs0 + l);
            const float2 a = h2f(f.x), b = h2f(f.y), c = h2f(f.z), d = h2f(f.w);
            float4* o = reinterpret_cast<float4*>(scl + l * STG_CLOVER_STRIDE + 8 * v);
            o[0] = make_float4(a.x, a.y, b.x, b.y);
            o[1] = make_float4(c.x, c.y, d.x, d.y);
          }
        }
      }
    }
    __syncthreads();
  }
  Site s;
  if (valid) s = site_of(A.g, A.p, hh);
  const bool reduce = A.do_norm || EPI == EPI_XPAY_CG;
  auto apply_cl = [&](int b, const cx<R> x[6], cx<R> y[6]) {
    if (SCL) clover_apply_smem(scl, lane, b, x, y);
    else CloverIO<CP>::apply(A.clover, Vh, hh, b, x, y);
  };
  for (int r = k; r < A.nrhs; r += W) {
    bool act = true;
    double al = 0.0;
    if (EPI == EPI_XPAY_CG) {
      act = A.red.cg[r].active != 0;
      al = A.red.cg[r].alpha;
    }
    double nrm = 0.0;
    if (valid) {
      cx<R> acc[12];
      if constexpr (P == 16) {
        hops_fp16_sp<RECON, STAGED>(A, s, r, reinterpret_cast<const float4*>(sl + lane * LSTRIDE),
                                    reinterpret_cast<cx<float>*>(acc));
      } else {
        DirLinks<R> L;
        auto links = [&](auto mu_c) {
          constexpr int MU = decltype(mu_c)::value;
          if (STAGED) {
            dir_index<MU>(A.g, s, L);
            staged_link(sl, lane, 2 * MU, L.uf);
            staged_link(sl, lane, 2 * MU + 1, L.ub);
          } else {
            load_dir<P, RECON, MU>(A, s, L);
          }
        };
        links(std::integral_constant<int, 0>());
        hop_dir<P, 0, LD_NC, true, false, !STAGED>(A, L, r, acc);
        links(std::integral_constant<int, 1>());
        hop_dir<P, 1, LD_NC, false, false, !STAGED>(A, L, r, acc);
        links(std::integral_constant<int, 2>());
        hop_dir<P, 2, LD_NC, false, false, !STAGED>(A, L, r, acc);
        links(std::integral_constant<int, 3>());
        hop_dir<P, 3, LD_NC>(A, L, r, acc);
      }
      cx<R> res[12];
#pragma unroll
      for (int b = 0; b < 2; b++) {
        cx<R> v[6], o[6];
#pragma unroll
        for (int j = 0; j < 6; j++) v[j] = acc[6 * b + j];
        if (EPI == EPI_NONE) {
#pragma unroll
          for (int j = 0; j < 6; j++) o[j] = v[j];
        } else if (EPI == EPI_CLOVER_INV) {
          apply_cl(b, v, o);
        } else {
          cx<R> xs[6], cxs[6];
          SpinorIO<P>::load_block(A.x, A.x_norm, Vh, r, hh, b, xs);
          if (A.x_g5 && b == 1) {
#pragma unroll
            for (int j = 0; j < 6; j++) xs[j] = -xs[j];
          }
          apply_cl(b, xs, cxs);
          const R a = R(A.a);
#pragma unroll
          for (int j = 0; j < 6; j++) {
            o[j].re = fma(a, v[j].re, cxs[j].re);
            o[j].im = fma(a, v[j].im, cxs[j].im);
          }
        }
        if (A.out_g5 && b == 1) {
#pragma unroll
          for (int j = 0; j < 6; j++) o[j] = -o[j];
        }
        if (EPI == EPI_XPAY_CG) {
          if (act) {
            const RR alr = RR(al);
            cx<R> ps[6];
            cx<RR> xs[6], rs[6];
            SpinorIO<P>::load_block(A.cg_p, A.cg_p_norm, Vh, r, hh, b, ps);
            SpinorIO<PR>::load_block(A.cg_x, nullptr, Vh, r, hh, b, xs);
            SpinorIO<PR>::load_block(A.cg_r, nullptr, Vh, r, hh, b, rs);
            RR n6 = RR(0);  // the site block's |r|^2 in the precision of r (FP32 below FP64)
#pragma unroll
            for (int j = 0; j < 6; j++) {
              xs[j].re = fma(alr, RR(ps[j].re), xs[j].re);
              xs[j].im = fma(alr, RR(ps[j].im), xs[j].im);
              rs[j].re = fma(-alr, RR(o[j].re), rs[j].re);
              rs[j].im = fma(-alr, RR(o[j].im), rs[j].im);
              n6 = fma(rs[j].re, rs[j].re, n6);
              n6 = fma(rs[j].im, rs[j].im, n6);
            }
            nrm += double(n6);
            SpinorIO<PR>::store_block(A.cg_x, nullptr, Vh, r, hh, b, xs);
            SpinorIO<PR>::store_block(A.cg_r, nullptr, Vh, r, hh, b, rs);
          }
        } else {
          if (A.do_norm) {
            R n6 = R(0);
#pragma unroll
            for (int j = 0; j < 6; j++) {
              n6 = fma(o[j].re, o[j].re, n6);
              n6 = fma(o[j].im, o[j].im, n6);
            }
            nrm += double(n6);
          }
#pragma unroll
          for (int j = 0; j < 6; j++) res[6 * b + j] = o[j];
        }
      }
      if (EPI != EPI_XPAY_CG) {
        if (P == 16) {
          cx<float> of[12];
#pragma unroll
          for (int c = 0; c < 12; c++) of[c] = cmk(float(res[c].re), float(res[c].im));
          SpinorIO<16>::store(A.out, A.out_norm, Vh, r, hh, of);
        } else {
          SpinorIO<P>::store(A.out, A.out_norm, Vh, r, hh, res);
        }
      }
    }
    if (reduce) {
      for (int off = 16; off >= 1; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
      if (lane == 0) {
        const long long slot = (long long)r * (gridDim.x * G) + blockIdx.x * G + grp;
        if (slot < A.red.capacity) A.red.partials[slot] = nrm;
        else A.red.ctl->overflow = 1;
      }
    }
  }
  if (reduce) grid_finish<128>(A.nrhs, gridDim.x, gridDim.x * G, A.red);
}

// FP32: 6 blocks per SM (80 registers).  32^3 x 64 against the compiler's own choice (96 registers
// unstaged, 5 blocks): 1 RHS 159 -> 153.5 us, 4 RHS 418 -> 413 us, 8 RHS 698 -> 688 us; 48^3 x 96,
// 1 RHS 782 -> 744 us.  7 blocks spill (1 RHS 170 us), 5 staged blocks are slower (8 RHS 715 us).
template <int P, int RECON, int EPI, bool STAGED>
__global__ void __launch_bounds__(128, 6) dslash_site_kernel(DslashArgs A) {
  dslash_site_body<P, RECON, EPI, STAGED>(A);
}

// FP16: 4 blocks per SM of up to 128 registers.  Unstaged, the registers hold the links and
// neighbours of two directions at once (5 blocks of 96 registers: 105 us against 103 us at 32^3 x 64,
// 1 RHS; 6 of 80: 108 us); staged, the 47 KB of shared memory (links as broadcast pairs, clover pair)
// allow 4 blocks (5 blocks of 96 registers with the clover read through L1 instead: 32^3 x 64, 8 RHS
// 631 -> 658 us)
template <int RECON, int EPI, bool STAGED>
__global__ void __launch_bounds__(128, 4) dslash_site_fp16_kernel(DslashArgs A) {
  dslash_site_body<16, RECON, EPI, STAGED>(A);
}

// The single-RHS FP16 operator is bound by latency: it is held to 64 registers, so that 8 blocks
// (32 warps) share an SM.
template <int RECON, int EPI, bool HALO = false>
__global__ void __launch_bounds__(128, 8) dslash_split_fp16_kernel(DslashArgs A) {
  dslash_split_body<16, RECON, EPI, HALO>(A);
}

}  // namespace qcd
