// Device-side building blocks shared by the CUDA translation units of libqcd:
// lattice geometry, complex arithmetic, and loaders/storers for the
// structure-of-arrays field layouts in every precision.
//
// Layout (all fields checkerboarded: parity p = (x+y+z+t) mod 2, half index
// h = i >> 1 of the lexicographic index i = x + X (y + Y (z + Z t)); X even):
//   spinor FP64 : [rhs][12][Vh] double2     component c = 3*spin + colour
//   spinor FP32 : [rhs][6][Vh]  float4      two complex components per float4
//   spinor FP16 : [rhs][3][Vh]  uint4 (8 halves = 4 complex) + [rhs][Vh] float norm
//   gauge  FP64 : [p][mu][9][Vh] double2    element (i,j) at 3i+j
//   gauge  FP32 : recon 18 [p][mu][9][Vh] float2, recon 12 [p][mu][3][Vh] float4
//   gauge  FP16 : recon 18 [p][mu][9][Vh] half2,  recon 12 [p][mu][3][Vh] uint2
//   clover FP64 : [p][36][Vh] double2, FP32 [p][18][Vh] float4: two chiral
//                 6x6 Hermitian blocks, each 6 real diagonal + 15 complex
//                 strictly-lower entries in row-major order.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qcd {

// Division by a lattice extent d >= 2, for 0 <= n < 2^31, as a multiply and a shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d)
// and m = ceil(2^(31+l) / d) < 2^32, n / d = floor(n m / 2^(31+l)).  It is exact because
// n (m d - 2^(31+l)) < 2^31 d <= 2^(31+l), so the excess of n m / 2^(31+l) over n / d stays below
// 1 / d.  The host evaluates the same expression with a 64-bit product.
struct FastDiv {
  unsigned m;
  int s;  // l - 1
  __host__ __device__ __forceinline__ int div(int n) const {
#ifdef __CUDA_ARCH__
    return (int)(__umulhi((unsigned)n, m) >> s);
#else
    return (int)((((unsigned long long)(unsigned)n * m) >> 32) >> s);
#endif
  }
};

inline FastDiv make_fastdiv(int d) {
  int l = 0;
  while ((1LL << l) < d) l++;
  FastDiv f;
  f.s = l - 1;
  f.m = (unsigned)(((1ULL << (31 + l)) + (unsigned long long)d - 1) / (unsigned long long)d);
  return f;
}

struct Geom {
  int X, Y, Z, T;
  int Vh;                // sites of one parity
  int XY, XYZ;           // lexicographic strides
  double t_bc;           // factor on U_t(x) at global time Tg-1 in the hopping term
  FastDiv dX, dY, dZ;    // division by X, Y, Z
  int t0, Tg;            // global time of local t = 0 and the global time extent (a t-slab of a larger
                         // lattice; 0 and T otherwise)
};

// (x, y, z, t) of the lexicographic index i = x + X (y + Y (z + Z t))
__host__ __device__ __forceinline__ void lattice_coords(const Geom& g, int i, int c[4]) {
  const int q1 = g.dX.div(i);
  c[0] = i - q1 * g.X;
  const int q2 = g.dY.div(q1);
  c[1] = q1 - q2 * g.Y;
  const int q3 = g.dZ.div(q2);
  c[2] = q2 - q3 * g.Z;
  c[3] = q3;
}

// ---------------------------------------------------------------- complex ----
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> cmk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> times_i(cx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cx<R> times_mi(cx<R> a) { return {a.im, -a.re}; }
// acc + a*b
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a)*b
template <typename R>
__device__ __forceinline__ cx<R> cfmac(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename R>
__device__ __forceinline__ R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }

// ------------------------------------------------------------- geometry ----
struct Site {
  int x, y, z, t;
  int i;  // lexicographic index
};

__device__ __forceinline__ Site site_of(const Geom& g, int p, int h) {
  Site s;
  int c[4];
  lattice_coords(g, 2 * h, c);
  s.y = c[1];
  s.z = c[2];
  s.t = c[3];
  s.x = c[0] + ((p + s.y + s.z + s.t) & 1);
  s.i = s.x + g.X * (s.y + g.Y * (s.z + g.Z * s.t));
  return s;
}

// lexicographic index of the neighbour x + dir*mu_hat (dir = +1 or -1)
__device__ __forceinline__ int neighbor_fwd(const Geom& g, const Site& s, int mu) {
  switch (mu) {
    case 0: return s.x == g.X - 1 ? s.i - (g.X - 1) : s.i + 1;
    case 1: return s.y == g.Y - 1 ? s.i - (g.XY - g.X) : s.i + g.X;
    case 2: return s.z == g.Z - 1 ? s.i - (g.XYZ - g.XY) : s.i + g.XY;
    default: return s.t == g.T - 1 ? s.i - (g.T - 1) * g.XYZ : s.i + g.XYZ;
  }
}
__device__ __forceinline__ int neighbor_bwd(const Geom& g, const Site& s, int mu) {
  switch (mu) {
    case 0: return s.x == 0 ? s.i + (g.X - 1) : s.i - 1;
    case 1: return s.y == 0 ? s.i + (g.XY - g.X) : s.i - g.X;
    case 2: return s.z == 0 ? s.i + (g.XYZ - g.XY) : s.i - g.XY;
    default: return s.t == 0 ? s.i + (g.T - 1) * g.XYZ : s.i - g.XYZ;
  }
}

// ------------------------------------------------------------ debug checks ----
// Builds with QCD_DEBUG=1 (libqcd_debug.so) check the indices every field accessor below is given: the
// site (0 <= h < Vh, or the face index against its face), the RHS (r >= 0), the link's parity and
// direction and the clover block.  A failed check sets a bit of this translation unit's violation word
// (DBG_SPINOR, DBG_LINK, DBG_CLOVER, DBG_HALO) and the access is skipped: a load returns zeros, a
// store writes nothing.  The host collects the words with qcd_debug_violations.  Release builds
// compile the checks away.
enum : unsigned { DBG_SPINOR = 1u, DBG_LINK = 2u, DBG_CLOVER = 4u, DBG_HALO = 8u };
#ifndef QCD_DEBUG
#define QCD_DEBUG 0
#endif
#if QCD_DEBUG
static __device__ unsigned qcd_dbg_word;
#endif
__device__ __forceinline__ bool dbg_check(bool ok, unsigned bit) {
#if QCD_DEBUG
  if (!ok) atomicOr(&qcd_dbg_word, bit);
  return ok;
#else
  (void)bit;
  return true;
#endif
}
__device__ __forceinline__ bool dbg_spinor(int Vh, int r, int h) { return dbg_check(h >= 0 && h < Vh && r >= 0, DBG_SPINOR); }
__device__ __forceinline__ bool dbg_link(int Vh, int p, int mu, int h) {
  return dbg_check(h >= 0 && h < Vh && (p == 0 || p == 1) && mu >= 0 && mu < 4, DBG_LINK);
}
__device__ __forceinline__ bool dbg_clover(int Vh, int h, int b) {
  return dbg_check(h >= 0 && h < Vh && (b == 0 || b == 1), DBG_CLOVER);
}
// A host function `unsigned name()` that returns and clears this translation unit's violation word
// (0 in release builds); every translation unit with kernels defines one.
#if QCD_DEBUG
#define QCD_DEBUG_TAKE(name)                                                         \
  unsigned name() {                                                                  \
    unsigned v = 0, z = 0;                                                           \
    if (cudaMemcpyFromSymbol(&v, qcd_dbg_word, sizeof v) != cudaSuccess) v = ~0u;    \
    cudaMemcpyToSymbol(qcd_dbg_word, &z, sizeof z);                                  \
    return v;                                                                        \
  }
#else
#define QCD_DEBUG_TAKE(name) \
  unsigned name() { return 0; }
#endif

// ------------------------------------------------------------ precision ----
template <int P>
struct Real;
template <>
struct Real<64> { using T = double; };
template <>
struct Real<32> { using T = float; };
template <>
struct Real<16> { using T = float; };

// Load modes of the field accessors: LD_NC through the read-only path (fields no block of the
// kernel writes); LD_CG through L2 only; LD_CA an ordinary load cached in L1 and L2, for fields
// that other blocks of the same (persistent) kernel wrote before a grid barrier whose GPU-scope
// acquire makes their writes visible; LD_SM a plain load, for copies staged in shared memory.
enum : int { LD_NC = 0, LD_CG = 1, LD_SM = 2, LD_CA = 3 };
template <int LD, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if (LD == LD_CG) return __ldcg(p);
  if (LD == LD_CA) return __ldca(p);
  if (LD == LD_SM) return *p;
  return __ldg(p);
}

// spinor accessors: 12 complex components, component c = 3*spin + colour.  A field of nrhs
// right-hand sides is stored RHS-major: vector k of (RHS r, site h) at (r * NVEC + k) * Vh + h, so
// the lanes of a warp (consecutive sites of one RHS) read one contiguous run.
template <int NV>
__device__ __forceinline__ size_t sidx(int k, int Vh, int r, int h) {
  return ((size_t)r * NV + k) * Vh + h;
}

template <int P>
struct SpinorIO;

template <>
struct SpinorIO<64> {
  static constexpr int NVEC = 12;  // double2 per site
  template <int LD = LD_NC>
  __device__ static void load(const void* base, const float*, int Vh, int r, int h, cx<double> s[12]) {
    if (!dbg_spinor(Vh, r, h)) {
      for (int c = 0; c < 12; c++) s[c] = {};
      return;
    }
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      double2 v = ldv<LD>(p + sidx<NVEC>(c, Vh, r, h));
      s[c] = cmk(v.x, v.y);
    }
  }
  __device__ static void store(void* base, float*, int Vh, int r, int h, const cx<double> s[12]) {
    if (!dbg_spinor(Vh, r, h)) return;
    double2* p = static_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 12; c++) p[sidx<NVEC>(c, Vh, r, h)] = make_double2(s[c].re, s[c].im);
  }
  // components 6b..6b+5 (chiral block b: spins 2b, 2b+1)
  template <int LD = LD_NC>
  __device__ static void load_block(const void* base, const float*, int Vh, int r, int h, int b,
                                    cx<double> s[6]) {
    if (!dbg_spinor(Vh, r, h)) {
      for (int c = 0; c < 6; c++) s[c] = {};
      return;
    }
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++) {
      double2 v = ldv<LD>(p + sidx<NVEC>(6 * b + c, Vh, r, h));
      s[c] = cmk(v.x, v.y);
    }
  }
  __device__ static void store_block(void* base, float*, int Vh, int r, int h, int b,
                                     const cx<double> s[6]) {
    if (!dbg_spinor(Vh, r, h)) return;
    double2* p = static_cast<double2*>(base);
#pragma unroll
    for (int c = 0; c < 6; c++) p[sidx<NVEC>(6 * b + c, Vh, r, h)] = make_double2(s[c].re, s[c].im);
  }
};

template <>
struct SpinorIO<32> {
  static constexpr int NVEC = 6;  // float4 per site
  template <int LD = LD_NC>
  __device__ static void load(const void* base, const float*, int Vh, int r, int h, cx<float> s[12]) {
    if (!dbg_spinor(Vh, r, h)) {
      for (int c = 0; c < 12; c++) s[c] = {};
      return;
    }
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = ldv<LD>(p + sidx<NVEC>(k, Vh, r, h));
      s[2 * k] = cmk(v.x, v.y);
      s[2 * k + 1] = cmk(v.z, v.w);
    }
  }
  __device__ static void store(void* base, float*, int Vh, int r, int h, const cx<float> s[12]) {
    if (!dbg_spinor(Vh, r, h)) return;
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++)
      p[sidx<NVEC>(k, Vh, r, h)] = make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
  }
  template <int LD = LD_NC>
  __device__ static void load_block(const void* base, const float*, int Vh, int r, int h, int b,
                                    cx<float> s[6]) {
    if (!dbg_spinor(Vh, r, h)) {
      for (int c = 0; c < 6; c++) s[c] = {};
      return;
    }
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = ldv<LD>(p + sidx<NVEC>(3 * b + k, Vh, r, h));
      s[2 * k] = cmk(v.x, v.y);
      s[2 * k + 1] = cmk(v.z, v.w);
    }
  }
  __device__ static void store_block(void* base, float*, int Vh, int r, int h, int b,
                                     const cx<float> s[6]) {
    if (!dbg_spinor(Vh, r, h)) return;
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++)
      p[sidx<NVEC>(3 * b + k, Vh, r, h)] =
          make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
  }
};

__device__ __forceinline__ float2 h2f(uint32_t u) {
  __half2 h = *reinterpret_cast<__half2*>(&u);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// FP16 spinor: each real is stored as half(v / n) with n = max |v| over the site's 24 reals;
// the norms of a field are stored [nrhs][Vh]
template <>
struct SpinorIO<16> {
  static constexpr int NVEC = 3;  // uint4 per site
  template <int LD = LD_NC>
  __device__ static void load(const void* base, const float* nrm, int Vh, int r, int h, cx<float> s[12]) {
    if (!dbg_spinor(Vh, r, h)) {
      for (int c = 0; c < 12; c++) s[c] = {};
      return;
    }
    const uint4* p = static_cast<const uint4*>(base);
    const float n = ldv<LD>(nrm + (size_t)r * Vh + h);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 v = ldv<LD>(p + sidx<NVEC>(k, Vh, r, h));
      float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
      s[4 * k + 0] = cmk(a.x * n, a.y * n);
      s[4 * k + 1] = cmk(b.x * n, b.y * n);
      s[4 * k + 2] = cmk(c.x * n, c.y * n);
      s[4 * k + 3] = cmk(d.x * n, d.y * n);
    }
  }
  // a site as stored (24 halves and the norm), so that loads can be issued well before the
  // values are used
  struct Raw {
    uint4 v[3];
    float n;
  };
  template <int LD = LD_NC>
  __device__ static void load_raw(const void* base, const float* nrm, int Vh, int r, int h, Raw& q) {
    if (!dbg_spinor(Vh, r, h)) {
      q = {};
      return;
    }
    const uint4* p = static_cast<const uint4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++) q.v[k] = ldv<LD>(p + sidx<NVEC>(k, Vh, r, h));
    q.n = ldv<LD>(nrm + (size_t)r * Vh + h);
  }
  // the stored values v / n without the per-site scale n, which is returned
  __device__ static float unpack_unscaled(const Raw& q, cx<float> s[12]) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float2 a = h2f(q.v[k].x), b = h2f(q.v[k].y), c = h2f(q.v[k].z), d = h2f(q.v[k].w);
      s[4 * k + 0] = cmk(a.x, a.y);
      s[4 * k + 1] = cmk(b.x, b.y);
      s[4 * k + 2] = cmk(c.x, c.y);
      s[4 * k + 3] = cmk(d.x, d.y);
    }
    return q.n;
  }
  template <int LD = LD_NC>
  __device__ static float load_unscaled(const void* base, const float* nrm, int Vh, int r, int h, cx<float> s[12]) {
    Raw q;
    load_raw<LD>(base, nrm, Vh, r, h, q);
    return unpack_unscaled(q, s);
  }
  __device__ static void store(void* base, float* nrm, int Vh, int r, int h, const cx<float> s[12]) {
    if (!dbg_spinor(Vh, r, h)) return;
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; c++) m = fmaxf(m, fmaxf(fabsf(s[c].re), fabsf(s[c].im)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4* p = static_cast<uint4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 v;
      v.x = f2h(s[4 * k + 0].re * inv, s[4 * k + 0].im * inv);
      v.y = f2h(s[4 * k + 1].re * inv, s[4 * k + 1].im * inv);
      v.z = f2h(s[4 * k + 2].re * inv, s[4 * k + 2].im * inv);
      v.w = f2h(s[4 * k + 3].re * inv, s[4 * k + 3].im * inv);
      p[sidx<NVEC>(k, Vh, r, h)] = v;
    }
    nrm[(size_t)r * Vh + h] = m;
  }
  // block 0 = chunk 0 and the first half of chunk 1; block 1 = the second half of chunk 1 and chunk 2
  template <int LD = LD_NC>
  __device__ static void load_block(const void* base, const float* nrm, int Vh, int r, int h, int b,
                                    cx<float> s[6]) {
    if (!dbg_spinor(Vh, r, h)) {
      for (int c = 0; c < 6; c++) s[c] = {};
      return;
    }
    const uint4* p = static_cast<const uint4*>(base);
    const float n = ldv<LD>(nrm + (size_t)r * Vh + h);
    const uint4 mid = ldv<LD>(p + sidx<NVEC>(1, Vh, r, h));
    const uint4 end = ldv<LD>(p + sidx<NVEC>(b == 0 ? 0 : 2, Vh, r, h));
    float2 e0 = h2f(end.x), e1 = h2f(end.y), e2 = h2f(end.z), e3 = h2f(end.w);
    if (b == 0) {
      float2 m0 = h2f(mid.x), m1 = h2f(mid.y);
      s[0] = cmk(e0.x * n, e0.y * n);
      s[1] = cmk(e1.x * n, e1.y * n);
      s[2] = cmk(e2.x * n, e2.y * n);
      s[3] = cmk(e3.x * n, e3.y * n);
      s[4] = cmk(m0.x * n, m0.y * n);
      s[5] = cmk(m1.x * n, m1.y * n);
    } else {
      float2 m2 = h2f(mid.z), m3 = h2f(mid.w);
      s[0] = cmk(m2.x * n, m2.y * n);
      s[1] = cmk(m3.x * n, m3.y * n);
      s[2] = cmk(e0.x * n, e0.y * n);
      s[3] = cmk(e1.x * n, e1.y * n);
      s[4] = cmk(e2.x * n, e2.y * n);
      s[5] = cmk(e3.x * n, e3.y * n);
    }
  }
};

// gauge accessors: u[3i+j] = U_ij of the link at (parity p, direction mu, half index h)
template <typename R>
__device__ __forceinline__ void reconstruct_row2(cx<R> u[9]) {
  // row 2 = conj(row 0 x row 1) for a special unitary matrix
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

template <int P, int RECON>
struct GaugeIO;

template <>
struct GaugeIO<64, 18> {
  static constexpr int NVEC = 9;
  __device__ static void load(const void* g, int Vh, int p, int mu, int h, cx<double> u[9]) {
    if (!dbg_link(Vh, p, mu, h)) {
      for (int k = 0; k < 9; k++) u[k] = {};
      return;
    }
    const double2* q = static_cast<const double2*>(g) + (size_t)(p * 4 + mu) * NVEC * Vh + h;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      double2 v = __ldg(q + (size_t)k * Vh);
      u[k] = cmk(v.x, v.y);
    }
  }
};

template <>
struct GaugeIO<32, 18> {
  static constexpr int NVEC = 9;
  __device__ static void load(const void* g, int Vh, int p, int mu, int h, cx<float> u[9]) {
    if (!dbg_link(Vh, p, mu, h)) {
      for (int k = 0; k < 9; k++) u[k] = {};
      return;
    }
    const float2* q = static_cast<const float2*>(g) + (size_t)(p * 4 + mu) * NVEC * Vh + h;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float2 v = __ldg(q + (size_t)k * Vh);
      u[k] = cmk(v.x, v.y);
    }
  }
};

template <>
struct GaugeIO<32, 12> {
  static constexpr int NVEC = 3;
  __device__ static void load(const void* g, int Vh, int p, int mu, int h, cx<float> u[9]) {
    if (!dbg_link(Vh, p, mu, h)) {
      for (int k = 0; k < 9; k++) u[k] = {};
      return;
    }
    const float4* q = static_cast<const float4*>(g) + (size_t)(p * 4 + mu) * NVEC * Vh + h;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = __ldg(q + (size_t)k * Vh);
      u[2 * k] = cmk(v.x, v.y);
      u[2 * k + 1] = cmk(v.z, v.w);
    }
    reconstruct_row2(u);
  }
};

// FP16 links: load_raw fetches the stored halves (so that loads can be issued ahead of their use),
// decode converts them (and reconstructs row 2 of 12-real storage)
template <>
struct GaugeIO<16, 18> {
  static constexpr int NVEC = 9;
  struct Raw {
    uint32_t v[9];
  };
  __device__ static void load_raw(const void* g, int Vh, int p, int mu, int h, Raw& w) {
    if (!dbg_link(Vh, p, mu, h)) {
      w = {};
      return;
    }
    const uint32_t* q = static_cast<const uint32_t*>(g) + (size_t)(p * 4 + mu) * NVEC * Vh + h;
#pragma unroll
    for (int k = 0; k < 9; k++) w.v[k] = __ldg(q + (size_t)k * Vh);
  }
  __device__ static void decode(const Raw& w, cx<float> u[9]) {
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float2 v = h2f(w.v[k]);
      u[k] = cmk(v.x, v.y);
    }
  }
  __device__ static void load(const void* g, int Vh, int p, int mu, int h, cx<float> u[9]) {
    Raw w;
    load_raw(g, Vh, p, mu, h, w);
    decode(w, u);
  }
};

template <>
struct GaugeIO<16, 12> {
  static constexpr int NVEC = 3;
  struct Raw {
    uint2 v[3];
  };
  __device__ static void load_raw(const void* g, int Vh, int p, int mu, int h, Raw& w) {
    if (!dbg_link(Vh, p, mu, h)) {
      w = {};
      return;
    }
    const uint2* q = static_cast<const uint2*>(g) + (size_t)(p * 4 + mu) * NVEC * Vh + h;
#pragma unroll
    for (int k = 0; k < 3; k++) w.v[k] = __ldg(q + (size_t)k * Vh);
  }
  __device__ static void decode(const Raw& w, cx<float> u[9]) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float2 a = h2f(w.v[k].x), b = h2f(w.v[k].y);
      u[2 * k] = cmk(a.x, a.y);
      u[2 * k + 1] = cmk(b.x, b.y);
    }
    reconstruct_row2(u);
  }
  __device__ static void load(const void* g, int Vh, int p, int mu, int h, cx<float> u[9]) {
    Raw w;
    load_raw(g, Vh, p, mu, h, w);
    decode(w, u);
  }
};

// clover accessors: y = A x for chiral block b (x, y: 6 complex, index 3*local_spin + colour)
template <int CP>
struct CloverIO;

template <typename R>
__device__ __forceinline__ void hermitian6_accumulate(const R d[6], const cx<R> L[15], const cx<R> x[6],
                                                      cx<R> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; i++) y[i] = d[i] * x[i];
  int k = 0;
#pragma unroll
  for (int i = 1; i < 6; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      y[i] = cfma(L[k], x[j], y[i]);
      y[j] = cfmac(L[k], x[i], y[j]);
      k++;
    }
  }
}

template <>
struct CloverIO<64> {
  static constexpr int NVEC = 36;  // double2 per site
  template <int LD = LD_NC>
  __device__ static void apply(const void* c, int Vh, int h, int b, const cx<double> x[6], cx<double> y[6]) {
    if (!dbg_clover(Vh, h, b)) {
      for (int k = 0; k < 6; k++) y[k] = {};
      return;
    }
    const double2* q = static_cast<const double2*>(c) + (size_t)(b * 18) * Vh + h;
    double d[6];
    cx<double> L[15];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      double2 v = ldv<LD>(q + (size_t)k * Vh);
      d[2 * k] = v.x;
      d[2 * k + 1] = v.y;
    }
#pragma unroll
    for (int k = 0; k < 15; k++) {
      double2 v = ldv<LD>(q + (size_t)(3 + k) * Vh);
      L[k] = cmk(v.x, v.y);
    }
    hermitian6_accumulate(d, L, x, y);
  }
};

template <>
struct CloverIO<32> {
  static constexpr int NVEC = 18;  // float4 per site
  template <int LD = LD_NC>
  __device__ static void apply(const void* c, int Vh, int h, int b, const cx<float> x[6], cx<float> y[6]) {
    if (!dbg_clover(Vh, h, b)) {
      for (int k = 0; k < 6; k++) y[k] = {};
      return;
    }
    const float4* q = static_cast<const float4*>(c) + (size_t)(b * 9) * Vh + h;
    float f[36];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float4 v = ldv<LD>(q + (size_t)k * Vh);
      f[4 * k] = v.x;
      f[4 * k + 1] = v.y;
      f[4 * k + 2] = v.z;
      f[4 * k + 3] = v.w;
    }
    float d[6];
    cx<float> L[15];
#pragma unroll
    for (int k = 0; k < 6; k++) d[k] = f[k];
#pragma unroll
    for (int k = 0; k < 15; k++) L[k] = cmk(f[6 + 2 * k], f[7 + 2 * k]);
    hermitian6_accumulate(d, L, x, y);
  }
};

// FP16 clover: 72 halves per site (block 0: halves 0..35, block 1: 36..71) in [9][Vh] uint4
template <>
struct CloverIO<16> {
  static constexpr int NVEC = 9;  // uint4 per site
  // block B occupies halves [36B, 36B+36): uint4 4B .. 4B+4 (the middle uint4 is shared).  ROW0: the
  // row of c holding uint4 4B (4B for a whole field; 0 for a copy of the block's five rows alone)
  template <int B, int LD = LD_NC, int ROW0 = 4 * B>
  __device__ static void apply_block(const void* c, int Vh, int h, const cx<float> x[6], cx<float> y[6]) {
    if (!dbg_clover(Vh, h, B)) {
      for (int k = 0; k < 6; k++) y[k] = {};
      return;
    }
    const uint4* q = static_cast<const uint4*>(c) + h;
    float f[40];
#pragma unroll
    for (int k = 0; k < 5; k++) {
      uint4 v = ldv<LD>(q + (size_t)(ROW0 + k) * Vh);
      float2 a0 = h2f(v.x), a1 = h2f(v.y), a2 = h2f(v.z), a3 = h2f(v.w);
      f[8 * k + 0] = a0.x;
      f[8 * k + 1] = a0.y;
      f[8 * k + 2] = a1.x;
      f[8 * k + 3] = a1.y;
      f[8 * k + 4] = a2.x;
      f[8 * k + 5] = a2.y;
      f[8 * k + 6] = a3.x;
      f[8 * k + 7] = a3.y;
    }
    constexpr int o = 4 * B;  // block 1 starts 4 halves into uint4 4
    float d[6];
    cx<float> L[15];
#pragma unroll
    for (int k = 0; k < 6; k++) d[k] = f[o + k];
#pragma unroll
    for (int k = 0; k < 15; k++) L[k] = cmk(f[o + 6 + 2 * k], f[o + 7 + 2 * k]);
    hermitian6_accumulate(d, L, x, y);
  }
  template <int LD = LD_NC>
  __device__ static void apply(const void* c, int Vh, int h, int b, const cx<float> x[6], cx<float> y[6]) {
    if (b == 0) apply_block<0, LD>(c, Vh, h, x, y);
    else apply_block<1, LD>(c, Vh, h, x, y);
  }
};

// ---------------------------------------------------------- CG control ----
// Per right-hand side state of the CG iteration, resident in device memory so
// that the iteration runs without host round trips.
struct CGState {
  double rr;            // |r|^2 of the iterated residual
  double rr_prev;       // |r|^2 one iteration earlier
  double rr_reliable;   // |r|^2 at the last reliable update
  double pAp;           // <p, A p> = |Mhat p|^2
  double alpha, beta;
  double tol2;          // stop when |r|^2 <= tol2 (= tol^2 |b|^2)
  double bnorm2;
  double true_rr;       // last true residual |b - A x|^2 (FP64)
  int active;           // 1 until converged
  int iters;
  int since_reliable;
  int pending;          // reliable update requested
  int reliable_updates;
  int pad_;
};

struct CGControl {
  int halt;             // set when any RHS wants a reliable update or on error
  int nan;              // non-finite reduction or breakdown
  int reliable_every;
  int overflow;         // a reduction launch needed more partial slots than allocated (skipped)
  int rel_go;           // a reliable update is due: its kernels run only while this is set
  int pad_;
  double delta2;        // reliable update when |r|^2 < delta2 * rr_reliable
};

enum FinalizeMode {
  FIN_STORE = 0,     // result[r] = total
  FIN_CG_PAP = 1,    // alpha = rr / pAp
  FIN_CG_RR = 2,     // new |r|^2, beta, reliable-update and convergence triggers
  FIN_CG_TRUE = 3,   // true residual after a reliable update
  FIN_CG_BNORM = 4,  // |b|^2: tol2 *= |b|^2, a zero source is inactive from the start
};

struct ReduceArgs {
  double* partials;        // [nrhs][gridDim.x]
  long long capacity;      // slots in partials; a launch needing more records ctl->overflow
  unsigned int* counter;   // zero before the launch; the last block resets it
  double* result;          // [nrhs], FIN_STORE
  int mode;
  CGState* cg;
  CGControl* ctl;
};

// Per-RHS action of the last block once the grid-wide total is known.
__device__ __forceinline__ void finalize_total(const ReduceArgs& ra, int r, double total) {
  switch (ra.mode) {
    case FIN_STORE:
      ra.result[r] = total;
      break;
    case FIN_CG_PAP: {
      CGState& s = ra.cg[r];
      s.pAp = total;
      if (s.active) {
        if (!(total > 0.0) || !isfinite(total)) {
          ra.ctl->nan = 1;
          ra.ctl->halt = 1;
          s.alpha = 0.0;
        } else {
          s.alpha = s.rr / total;
        }
      } else {
        s.alpha = 0.0;
      }
      break;
    }
    case FIN_CG_RR: {
      CGState& s = ra.cg[r];
      if (!s.active) break;
      if (!isfinite(total)) {
        ra.ctl->nan = 1;
        ra.ctl->halt = 1;
        break;
      }
      s.rr_prev = s.rr;
      s.beta = total / s.rr;
      s.rr = total;
      s.iters += 1;
      s.since_reliable += 1;
      bool want = total <= s.tol2 || s.since_reliable >= ra.ctl->reliable_every ||
                  total < ra.ctl->delta2 * s.rr_reliable;
      if (want) {
        s.pending = 1;
        ra.ctl->halt = 1;
        ra.ctl->rel_go = 1;
      }
      break;
    }
    case FIN_CG_BNORM: {
      CGState& s = ra.cg[r];
      if (!isfinite(total)) {
        ra.ctl->nan = 1;
        ra.ctl->halt = 1;
        s.active = 0;
        break;
      }
      s.bnorm2 = total;
      s.tol2 *= total;
      s.active = total > 0.0 ? 1 : 0;
      break;
    }
    case FIN_CG_TRUE: {
      CGState& s = ra.cg[r];
      if (!isfinite(total)) {
        ra.ctl->nan = 1;
        break;
      }
      s.true_rr = total;
      if (!s.active) break;
      s.beta = s.rr_prev > 0.0 ? total / s.rr_prev : 0.0;
      s.rr = total;
      s.rr_reliable = total;
      s.since_reliable = 0;
      s.pending = 0;
      s.reliable_updates += 1;
      if (total <= s.tol2) s.active = 0;
      break;
    }
  }
}

// Grid-wide deterministic sums, one per right-hand side, in two parts.  block_partial: the block's
// sum of one double per thread for RHS r (warp shuffles, then shared memory) into slot
// r * nblk + blk of the partials.  grid_finish: after all of a block's partials are written, the
// last block of the grid to finish (blk_total blocks) sums every RHS's nblk partials in a fixed
// order and runs finalize_total.  Both are called by all threads of the block.
template <int BLOCK>
__device__ __forceinline__ void block_partial(double v, int r, int blk, int nblk, const ReduceArgs& ra) {
  __shared__ double sm[BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll 1
    for (int w = 0; w < BLOCK / 32; w++) s += sm[w];
    const long long slot = (long long)r * nblk + blk;
    if (slot < ra.capacity) ra.partials[slot] = s;
    else ra.ctl->overflow = 1;
  }
  __syncthreads();
}

template <int BLOCK>
__device__ __forceinline__ void grid_finish(int nrhs, long long blk_total, int nblk, const ReduceArgs& ra) {
  __shared__ double sm[BLOCK / 32];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(ra.counter, 1u);
    is_last = (ticket == blk_total - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int r = 0; r < nrhs; r++) {
    // thread t adds partials t, t + BLOCK, t + 2 BLOCK, ... in that order; the loads of U terms are
    // issued together (a grid of 32768 blocks leaves 256 partials per thread of a 128-thread block)
    constexpr int U = 16;
    double s = 0.0;
    for (int j0 = threadIdx.x; j0 < nblk; j0 += U * BLOCK) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int j = j0 + u * BLOCK;
        const long long slot = (long long)r * nblk + j;
        v[u] = (j < nblk && slot < ra.capacity) ? __ldcg(ra.partials + slot) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; u++) s += v[u];
    }
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __syncthreads();
    if (lane == 0) sm[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < BLOCK / 32; w++) tot += sm[w];
      finalize_total(ra, r, tot);
    }
  }
  if (threadIdx.x == 0) {
    if (ra.mode == FIN_CG_TRUE) {
      // after a residual replacement the inner iteration may run again unless
      // every right-hand side has converged or a non-finite value was seen
      int any = 0;
      for (int r = 0; r < nrhs; r++) any |= ra.cg[r].active;
      ra.ctl->halt = (any && !ra.ctl->nan) ? 0 : 1;
    }
    *ra.counter = 0u;
  }
}

}  // namespace qcd
