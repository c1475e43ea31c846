// The eight hops of one FP16 site and RHS on paired FP32 registers (spin rows paired).
//
// A projected half spinor has two spin rows per colour.  Here the two rows are held as pairs
// (row 0, row 1) of FP32 registers, real and imaginary parts in separate pairs, and the arithmetic
// runs on the paired FP32 instructions of sm_100 and later (fma.rn.f32x2 and mul.rn.f32x2 through
// __ffma2_rn and __fmul2_rn: one issued instruction for both rows, each lane rounded as the scalar
// instruction would round it):
//   * the projection h_s = psi_s + c_s psi_k(s) (s = 0, 1; c = +-1 or +-i) is one paired FMA per
//     colour and part, the factors +-i being a choice of operand and the signs a constant pair;
//   * the link multiply w = U h takes U_ab as broadcast pairs (re, re), (im, im), read from shared
//     memory where the block staged them in that form, or formed from registers;
//   * the reconstruction of spin rows 2 and 3 accumulates (c_l w_jl, c_h w_jh): lanes in the order
//     (row 2, row 3) for mu = z, t and (row 3, row 2) for mu = x, y, two accumulators that are added
//     once at the end.
// FP16 neighbours are converted half by half, so the conversions write the pairs directly.  The
// operator is that of the other hopping kernels (Wilson hopping term with spin projection, DeGrand-
// Rossi basis; the paper's application, Sec. 1).
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

// one colour of two spin rows: re = (Re row s, Re row s'), im likewise
struct sp2 {
  float2 re, im;
};

__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// staged links of the spin-paired FP16 kernel, floats per site: 8 links x 9 entries x (re, re, im,
// im), padded to an odd multiple of 16 bytes (consecutive sites' 16-byte reads in distinct bank groups)
constexpr int SP_LINK_STRIDE = 8 * 9 * 4 + 4;

// The factor of a projection or reconstruction term: 0 = +1, 1 = -1, 2 = +i, 3 = -i.  The real part
// of c x is +-x.re (c real) or -+x.im (c imaginary); neg_re / neg_im: whether it enters negated.
__host__ __device__ constexpr bool c_imag(int c) { return c >= 2; }
__host__ __device__ constexpr bool neg_re(int c) { return c == 1 || c == 2; }
__host__ __device__ constexpr bool neg_im(int c) { return c == 1 || c == 3; }
// index of the sign pair (lane 0 negated, lane 1 negated) in a table {++, +-, -+, --}
__host__ __device__ constexpr int sgn_idx(bool n0, bool n1) { return (n0 ? 2 : 0) + (n1 ? 1 : 0); }

// Factors per direction and sign (SGN < 0: forward hop, 1 - g_mu; SGN > 0: backward hop, 1 + g_mu):
// rows 0, 1 of the projection h0 = s0 + c0 s_k0, h1 = s1 + c1 s_k1; reconstruction of rows 2, 3:
// lo = cl w_jl, hi = ch w_jh.
template <int MU, int SGN>
struct SpTable {
  static constexpr int k0 = (MU == 0 || MU == 1) ? 3 : 2;
  static constexpr int k1 = (MU == 0 || MU == 1) ? 2 : 3;
  static constexpr int c0 = MU == 0 ? (SGN < 0 ? 3 : 2) : MU == 1 ? (SGN < 0 ? 0 : 1)
                          : MU == 2 ? (SGN < 0 ? 3 : 2) : (SGN < 0 ? 1 : 0);
  static constexpr int c1 = MU == 0 ? (SGN < 0 ? 3 : 2) : MU == 1 ? (SGN < 0 ? 1 : 0)
                          : MU == 2 ? (SGN < 0 ? 2 : 3) : (SGN < 0 ? 1 : 0);
  static constexpr bool swapped = MU == 0 || MU == 1;  // jl = 1, jh = 0: lanes (row 3, row 2)
  static constexpr int cl = MU == 0 ? (SGN < 0 ? 2 : 3) : MU == 1 ? (SGN < 0 ? 1 : 0)
                          : MU == 2 ? (SGN < 0 ? 2 : 3) : (SGN < 0 ? 1 : 0);
  static constexpr int ch = MU == 0 ? (SGN < 0 ? 2 : 3) : MU == 1 ? (SGN < 0 ? 0 : 1)
                          : MU == 2 ? (SGN < 0 ? 3 : 2) : (SGN < 0 ? 1 : 0);
};

// link entries as broadcast pairs: from the staged copy (float4 (re, re, im, im) per entry) ...
struct StagedLinkSp {
  const float4* q;
  __device__ __forceinline__ void get(int e, float2& ur, float2& ui) const {
    const float4 v = q[e];
    ur = make_float2(v.x, v.y);
    ui = make_float2(v.z, v.w);
  }
};
// ... or from a link in registers
struct RegLinkSp {
  const cx<float>* u;
  __device__ __forceinline__ void get(int e, float2& ur, float2& ui) const {
    ur = make_float2(u[e].re, u[e].re);
    ui = make_float2(u[e].im, u[e].im);
  }
};

// row a of w = U h (ADJ: U^dag h), both spin rows at once
template <bool ADJ, typename LK>
__device__ __forceinline__ sp2 su3_row_sp(const LK& lk, int a, const sp2 h[3], float2 M1) {
  float2 ur[3], ui[3];
#pragma unroll
  for (int b = 0; b < 3; b++) lk.get(ADJ ? 3 * b + a : 3 * a + b, ur[b], ui[b]);
  sp2 w;
  if (!ADJ) {  // re = sum ur h.re - ui h.im, im = sum ur h.im + ui h.re
    float2 p = p_mul(ur[0], h[0].re), n = p_mul(ui[0], h[0].im), q = p_mul(ur[0], h[0].im);
    q = p_fma(ui[0], h[0].re, q);
#pragma unroll
    for (int b = 1; b < 3; b++) {
      p = p_fma(ur[b], h[b].re, p);
      n = p_fma(ui[b], h[b].im, n);
      q = p_fma(ur[b], h[b].im, q);
      q = p_fma(ui[b], h[b].re, q);
    }
    w.re = p_fma(n, M1, p);
    w.im = q;
  } else {  // conj(u): re = sum ur h.re + ui h.im, im = sum ur h.im - ui h.re
    float2 p = p_mul(ur[0], h[0].re), q = p_mul(ur[0], h[0].im), n = p_mul(ui[0], h[0].re);
    p = p_fma(ui[0], h[0].im, p);
#pragma unroll
    for (int b = 1; b < 3; b++) {
      p = p_fma(ur[b], h[b].re, p);
      p = p_fma(ui[b], h[b].im, p);
      q = p_fma(ur[b], h[b].im, q);
      n = p_fma(ui[b], h[b].re, n);
    }
    w.re = p;
    w.im = p_fma(n, M1, q);
  }
  return w;
}

// half of a stored FP16 word as float: the real (HI = false) or imaginary part of component c
template <bool HI>
__device__ __forceinline__ float half_of(const SpinorIO<16>::Raw& q, int c) {
  const uint4& v = q.v[c >> 2];
  const uint32_t w = (c & 3) == 0 ? v.x : (c & 3) == 1 ? v.y : (c & 3) == 2 ? v.z : v.w;
  const __half2 h = *reinterpret_cast<const __half2*>(&w);
  return HI ? __high2float(h) : __low2float(h);
}

// the pair (component c0, component c1) of a stored site, real or imaginary parts
template <bool HI>
__device__ __forceinline__ float2 pair_of(const SpinorIO<16>::Raw& q, int c0, int c1) {
  return make_float2(half_of<HI>(q, c0), half_of<HI>(q, c1));
}

// Accumulators of one site and RHS: rows (0, 1), rows (2, 3) and rows (3, 2), per colour.
struct SpAcc {
  sp2 a01[3], a23[3], a32[3];
};

// acc (+)= the hop from the stored neighbour q (its norm and the boundary factor bc applied to the
// product) through link lk.  SG: the gamma_5 sign pairs of the input {++, +-, -+, --} x g.
// FIRST01: first term of rows 0, 1 and (3, 2); FIRST23: first term of rows (2, 3).
template <int MU, int SGN, bool FIRST01, bool FIRST23, typename LK>
__device__ __forceinline__ void hop_sp(const SpinorIO<16>::Raw& q, const LK& lk, float bc, const float2 SG[4],
                                       float2 M1, SpAcc& acc) {
  using T = SpTable<MU, SGN>;
  static_assert(c_imag(T::c0) == c_imag(T::c1), "both rows of a projection take the same kind of factor");
  constexpr bool IM = c_imag(T::c0);
  // h = (s0, s1) + (c0 s_k0, c1 s_k1) per colour: the real part takes x.re (x.im for imaginary c)
  constexpr int SRE = sgn_idx(neg_re(T::c0), neg_re(T::c1)), SIM = sgn_idx(neg_im(T::c0), neg_im(T::c1));
  sp2 h[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const float2 sre = pair_of<false>(q, a, 3 + a), sim = pair_of<true>(q, a, 3 + a);
    const float2 xre = pair_of<false>(q, 3 * T::k0 + a, 3 * T::k1 + a);
    const float2 xim = pair_of<true>(q, 3 * T::k0 + a, 3 * T::k1 + a);
    h[a].re = p_fma(IM ? xim : xre, SG[SRE], sre);
    h[a].im = p_fma(IM ? xre : xim, SG[SIM], sim);
  }
  const float f = MU == 3 ? q.n * bc : q.n;
  const float2 F = make_float2(f, f);
  // rows 2, 3: lanes (cl w0, ch w1) into a23, or (ch w0, cl w1) into a32
  constexpr int L0 = T::swapped ? T::ch : T::cl, L1 = T::swapped ? T::cl : T::ch;
  static_assert(c_imag(L0) == c_imag(L1), "both reconstructed rows take the same kind of factor");
  constexpr bool LIM = c_imag(L0);
  constexpr int FRE = sgn_idx(neg_re(L0), neg_re(L1)), FIM = sgn_idx(neg_im(L0), neg_im(L1));
  const float2 fre = FRE == 0 ? F : p_mul(F, make_float2(FRE & 2 ? -1.f : 1.f, FRE & 1 ? -1.f : 1.f));
  const float2 fim = FIM == 0 ? F : p_mul(F, make_float2(FIM & 2 ? -1.f : 1.f, FIM & 1 ? -1.f : 1.f));
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const sp2 w = su3_row_sp<(SGN > 0)>(lk, a, h, M1);
    if (FIRST01) {
      acc.a01[a].re = p_mul(F, w.re);
      acc.a01[a].im = p_mul(F, w.im);
    } else {
      acc.a01[a].re = p_fma(F, w.re, acc.a01[a].re);
      acc.a01[a].im = p_fma(F, w.im, acc.a01[a].im);
    }
    sp2& lo = T::swapped ? acc.a32[a] : acc.a23[a];
    const float2 xr = LIM ? w.im : w.re, xi = LIM ? w.re : w.im;
    if (T::swapped ? FIRST01 : FIRST23) {
      lo.re = p_mul(fre, xr);
      lo.im = p_mul(fim, xi);
    } else {
      lo.re = p_fma(fre, xr, lo.re);
      lo.im = p_fma(fim, xi, lo.im);
    }
  }
}

// the stored neighbour site of RHS r at half index nb
__device__ __forceinline__ void load_nb_sp(const void* in, const float* in_norm, int Vh, int r, int nb,
                                           SpinorIO<16>::Raw& q) {
  SpinorIO<16>::load_raw<LD_NC>(in, in_norm, Vh, r, nb, q);
}

// rows 0..3 of the summed hops as complex components 3 * spin + colour
__device__ __forceinline__ void sp_unpack(const SpAcc& acc, cx<float> out[12]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    out[a] = cmk(acc.a01[a].re.x, acc.a01[a].im.x);
    out[3 + a] = cmk(acc.a01[a].re.y, acc.a01[a].im.y);
    out[6 + a] = cmk(acc.a23[a].re.x + acc.a32[a].re.y, acc.a23[a].im.x + acc.a32[a].im.y);
    out[9 + a] = cmk(acc.a23[a].re.y + acc.a32[a].re.x, acc.a23[a].im.y + acc.a32[a].im.x);
  }
}

}  // namespace qcd
