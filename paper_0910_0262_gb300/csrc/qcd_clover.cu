// Clover term A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) and its inverse.
//
// Standard Sheikholeslami-Wohlert definition (the paper's application is MILC's
// clover_dynamical, Sec. 1): Q_{mu nu}(x) is the sum of the four plaquette
// leaves around x in the (mu, nu) plane, F = traceless part of (Q - Q^dag)/(8i).
// In the DeGrand-Rossi basis sigma_{mu nu} is block diagonal in chirality, so A
// is two Hermitian 6x6 blocks.  With the 2x2 spin blocks of sigma written as
// Pauli matrices, block b (b = 0: spins 0,1; b = 1: spins 2,3) is
//   A_b = 1 - kappa c_sw [[ B3, B1 - i B2 ], [ B1 + i B2, -B3 ]]
//   b = 0: B1 = F_yz - F_xt, B2 = F_xz + F_yt, B3 = F_xy - F_zt
//   b = 1: B1 = F_yz + F_xt, B2 = F_xz - F_yt, B3 = F_xy + F_zt.
// The inverse is formed once per gauge field in FP64 by a Cholesky factorisation
// A_b = L L^dag and A_b^-1 = L^-dag L^-1; a non-positive pivot raises a flag.
#include "qcd_kernels.h"
#include "qcd_su3.cuh"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_clover)

namespace {

// traceless part of (Q - Q^dag) / (8 i), with Q = L1 + L2 + L3 + L4 the four-leaf sum in the
// (mu, nu) plane.  Only the anti-Hermitian part of Q is needed, and Q - Q^dag = M - M^dag with
// M = (L1 - L4^dag) + (L2 - L3^dag), where L1 and L4^dag both start with U_mu(x) and L2 and L3^dag
// both end with U_mu(x - mu):
//   L1 - L4^dag = U_mu(x) [U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag - U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)]
//   L2 - L3^dag = [U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag - U_nu(x-nu)^dag U_mu(x-mu-nu)^dag U_nu(x-mu-nu)] U_mu(x-mu)
// which takes 10 matrix products instead of the 12 of the four leaves.
__device__ M3 field_strength(const Geom& g, const double2* g64, const int c[4], int mu, int nu) {
  auto at = [&](int dm, int dn, int dir) {
    int q[4] = {c[0], c[1], c[2], c[3]};
    q[mu] += dm;
    q[nu] += dn;
    return link_at(g, g64, q[0], q[1], q[2], q[3], dir);
  };
  M3 M;
  {
    // U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    const M3 A = mul_nd(mul_nd(at(1, 0, nu), at(0, 1, mu)), at(0, 0, nu));
    // U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) = (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
    const M3 B = mul_dn(mul(at(0, -1, mu), at(1, -1, nu)), at(0, -1, nu));
    M3 D;
#pragma unroll
    for (int k = 0; k < 9; k++) D.e[k] = A.e[k] - B.e[k];
    M = mul(at(0, 0, mu), D);
  }
  {
    // U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag
    const M3 A = mul_nd(mul_nd(at(0, 0, nu), at(-1, 1, mu)), at(-1, 0, nu));
    // U_nu(x-nu)^dag U_mu(x-mu-nu)^dag U_nu(x-mu-nu) = (U_mu(x-mu-nu) U_nu(x-nu))^dag U_nu(x-mu-nu)
    const M3 B = mul_dn(mul(at(-1, -1, mu), at(0, -1, nu)), at(-1, -1, nu));
    M3 D;
#pragma unroll
    for (int k = 0; k < 9; k++) D.e[k] = A.e[k] - B.e[k];
    const M3 M2 = mul(D, at(-1, 0, mu));
#pragma unroll
    for (int k = 0; k < 9; k++) M.e[k] = M.e[k] + M2.e[k];
  }
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C d = M.e[3 * i + j] - conj(M.e[3 * j + i]);
      F.e[3 * i + j] = cmk(d.im * 0.125, -d.re * 0.125);  // d / (8 i)
    }
  const double tr = (F.e[0].re + F.e[4].re + F.e[8].re) / 3.0;
  F.e[0].re -= tr;
  F.e[4].re -= tr;
  F.e[8].re -= tr;
  return F;
}

__host__ __device__ constexpr int tri(int i, int j) { return i * (i - 1) / 2 + j; }

// Cholesky-based inverse of a Hermitian positive definite 6x6 matrix given as (diag d,
// strictly-lower L), and log det = sum_j log L_jj^2.  Returns false on a non-positive pivot.  All
// loops are unrolled, so the packed triangles stay in registers: A = l l^dag (l lower, diagonal ld),
// m = l^-1 (lower), A^-1 = m^dag m.
__device__ __forceinline__ bool invert6(const double d[6], const C L[15], double di[6], C Li[15], double* logdet) {
  double ild[6];  // 1 / l_jj: one division per pivot, multiplications elsewhere
  C lo[15];       // strictly-lower part of l
  double ldet = 0.0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; j++) {
    double s = d[j];
#pragma unroll
    for (int k = 0; k < j; k++) s -= norm2(lo[tri(j, k)]);
    ok = ok && s > 0.0;
    s = s > 0.0 ? s : 1.0;  // keeps the arithmetic finite; the result is discarded when !ok
    ldet += log(s);
    ild[j] = 1.0 / sqrt(s);
#pragma unroll
    for (int i = j + 1; i < 6; i++) {
      C v = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; k++) v = v - lo[tri(i, k)] * conj(lo[tri(j, k)]);
      lo[tri(i, j)] = cmk(v.re * ild[j], v.im * ild[j]);
    }
  }
  if (!ok) return false;
  // m = l^-1: m_jj = 1 / l_jj, m_ij = -(sum_{k=j}^{i-1} l_ik m_kj) / l_ii for i > j
  C mo[15];
#pragma unroll
  for (int j = 0; j < 6; j++)
#pragma unroll
    for (int i = j + 1; i < 6; i++) {
      C s = cmk(lo[tri(i, j)].re * ild[j], lo[tri(i, j)].im * ild[j]);
#pragma unroll
      for (int k = j + 1; k < i; k++) s = cfma(lo[tri(i, k)], mo[tri(k, j)], s);
      mo[tri(i, j)] = cmk(-s.re * ild[i], -s.im * ild[i]);
    }
  // A^-1 = m^dag m: (A^-1)_ij = sum_{k >= i} conj(m_ki) m_kj for i >= j
#pragma unroll
  for (int i = 0; i < 6; i++) {
    double sd = ild[i] * ild[i];
#pragma unroll
    for (int k = i + 1; k < 6; k++) sd += norm2(mo[tri(k, i)]);
    di[i] = sd;
#pragma unroll
    for (int j = 0; j < i; j++) {
      C s = cmk(ild[i] * mo[tri(i, j)].re, ild[i] * mo[tri(i, j)].im);  // k = i: m_ii m_ij
#pragma unroll
      for (int k = i + 1; k < 6; k++) s = cfmac(mo[tri(k, i)], mo[tri(k, j)], s);
      Li[tri(i, j)] = s;
    }
  }
  *logdet = ldet;
  return true;
}

__device__ __forceinline__ void store_block64(double2* base, int Vh, int h, int b, const double d[6], const C L[15]) {
  double2* q = base + (size_t)(b * 18) * Vh + h;
#pragma unroll
  for (int k = 0; k < 3; k++) q[(size_t)k * Vh] = make_double2(d[2 * k], d[2 * k + 1]);
#pragma unroll
  for (int k = 0; k < 15; k++) q[(size_t)(3 + k) * Vh] = make_double2(L[k].re, L[k].im);
}

// the 36 values of a block in storage order: 6 diagonal reals, then the 15 lower entries re, im
__device__ __forceinline__ double block_value(const double d[6], const C L[15], int k) {
  return k < 6 ? d[k] : ((k & 1) ? L[(k - 7) / 2].im : L[(k - 6) / 2].re);
}

__device__ __forceinline__ void store_block32(float4* base, int Vh, int h, int b, const double d[6], const C L[15]) {
  float4* q = base + (size_t)(b * 9) * Vh + h;
#pragma unroll
  for (int k = 0; k < 9; k++)
    q[(size_t)k * Vh] = make_float4((float)block_value(d, L, 4 * k), (float)block_value(d, L, 4 * k + 1),
                                    (float)block_value(d, L, 4 * k + 2), (float)block_value(d, L, 4 * k + 3));
}

// 36 halves of block B at halves [36B, 36B+36) of the site's 72 ([9][Vh] uint4 layout): four whole
// uint4 and one half of the uint4 the two blocks share (its low 8 bytes for block 0, high for 1)
template <int B>
__device__ __forceinline__ void store_block16_b(uint4* base, int Vh, int h, const double d[6], const C L[15]) {
  auto pack = [&](int k) { return f2h((float)block_value(d, L, k), (float)block_value(d, L, k + 1)); };
  constexpr int w0 = B == 0 ? 0 : 5;  // first whole uint4 of the block
  constexpr int k0 = B == 0 ? 0 : 4;  // block value stored at its start
#pragma unroll
  for (int w = 0; w < 4; w++) {
    const int k = k0 + 8 * w;
    base[(size_t)(w0 + w) * Vh + h] = make_uint4(pack(k), pack(k + 2), pack(k + 4), pack(k + 6));
  }
  constexpr int ks = B == 0 ? 32 : 0;  // the four values in the shared uint4 4
  *(reinterpret_cast<uint2*>(base + (size_t)4 * Vh + h) + B) = make_uint2(pack(ks), pack(ks + 2));
}

__device__ __forceinline__ void store_block16(uint4* base, int Vh, int h, int b, const double d[6], const C L[15]) {
  if (b == 0) store_block16_b<0>(base, Vh, h, d, L);
  else store_block16_b<1>(base, Vh, h, d, L);
}

// F_{mu nu} for one (site, plane) per thread into Fbuf[plane][9][V] (V = all sites, lexicographic)
__global__ void __launch_bounds__(128) field_strength_kernel(Geom g, const double2* __restrict__ g64, double2* Fbuf) {
  const int V = 2 * g.Vh;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 6LL * V) return;
  const int pl = (int)(tid / V), i = (int)(tid - (long long)pl * V);
  const int PM[6] = {0, 0, 0, 1, 1, 2}, PN[6] = {1, 2, 3, 2, 3, 3};
  int c[4];
  lattice_coords(g, i, c);
  const M3 F = field_strength(g, g64, c, PM[pl], PN[pl]);
  double2* q = Fbuf + (size_t)pl * 9 * V + i;
#pragma unroll
  for (int k = 0; k < 9; k++) q[(size_t)k * V] = make_double2(F.e[k].re, F.e[k].im);
}

// A's chiral block b and its inverse for one (site, block) per thread, from the six F_{mu nu}
__global__ void __launch_bounds__(128) clover_assemble_kernel(Geom g, const double2* __restrict__ Fbuf, double kappa,
                                                              double csw, double2* A64, double2* Ainv64, float4* A32,
                                                              float4* Ainv32, uint4* A16, uint4* Ainv16,
                                                              double* logdet, int* notposdef) {
  const int V = 2 * g.Vh;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * V) return;
  const int b = tid / V, i = tid - b * V;  // block b of lexicographic site i
  int c[4];
  lattice_coords(g, i, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int h = i >> 1;
  auto Fe = [&](int pl, int e) {
    const double2 v = __ldg(Fbuf + ((size_t)pl * 9 + e) * V + i);
    return cmk(v.x, v.y);
  };
  // planes xy xz xt yz yt zt = 0..5
  const double sg = b == 0 ? -1.0 : 1.0;
  C B1[9], B2[9], B3[9];
#pragma unroll
  for (int e = 0; e < 9; e++) {
    B1[e] = Fe(3, e) + sg * Fe(2, e);
    B2[e] = Fe(1, e) - sg * Fe(4, e);
    B3[e] = Fe(0, e) + sg * Fe(5, e);
  }
  const double kc = kappa * csw;
  double d[6];
  C L[15];
#pragma unroll
  for (int ii6 = 0; ii6 < 6; ii6++) {
    const int ii = ii6 % 3;
    d[ii6] = 1.0 - kc * (ii6 < 3 ? B3[4 * ii].re : -B3[4 * ii].re);
#pragma unroll
    for (int j = 0; j < ii6; j++) {
      const int jj = j % 3;
      C hv;
      if (ii6 < 3) hv = B3[3 * ii + jj];
      else if (j < 3) hv = B1[3 * ii + jj] + times_i(B2[3 * ii + jj]);
      else hv = -B3[3 * ii + jj];
      L[tri(ii6, j)] = cmk(-kc * hv.re, -kc * hv.im);
    }
  }
  double di[6];
  C Li[15];
  double ld = 0.0;
  if (!invert6(d, L, di, Li, &ld)) {
    *notposdef = 1;
    ld = 0.0;
    for (int k = 0; k < 6; k++) di[k] = 0.0;
    for (int k = 0; k < 15; k++) Li[k] = cmk(0.0, 0.0);
  }
  logdet[((size_t)p * 2 + b) * g.Vh + h] = ld;
  store_block64(A64 + (size_t)p * 36 * g.Vh, g.Vh, h, b, d, L);
  store_block64(Ainv64 + (size_t)p * 36 * g.Vh, g.Vh, h, b, di, Li);
  if (A32) store_block32(A32 + (size_t)p * 18 * g.Vh, g.Vh, h, b, d, L);
  if (Ainv32) store_block32(Ainv32 + (size_t)p * 18 * g.Vh, g.Vh, h, b, di, Li);
  if (A16) store_block16(A16 + (size_t)p * 9 * g.Vh, g.Vh, h, b, d, L);
  if (Ainv16) store_block16(Ainv16 + (size_t)p * 9 * g.Vh, g.Vh, h, b, di, Li);
}

template <int P>
__global__ void clover_apply_kernel(Geom g, const void* clov, const void* in, const float* in_norm, void* out,
                                    float* out_norm, int nrhs) {
  using R = typename Real<P>::T;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.Vh * nrhs) return;
  const int r = tid / g.Vh, h = tid - r * g.Vh;  // consecutive threads: consecutive sites of one RHS
  cx<R> s[12], o[12];
  SpinorIO<P>::load(in, in_norm, g.Vh, r, h, s);
  constexpr int CP = P;
  CloverIO<CP>::apply(clov, g.Vh, h, 0, s, o);
  CloverIO<CP>::apply(clov, g.Vh, h, 1, s + 6, o + 6);
  SpinorIO<P>::store(out, out_norm, g.Vh, r, h, o);
}

}  // namespace

void launch_clover_build(const Geom& g, const void* g64, double kappa, double csw, void* A64, void* Ainv64, void* A32,
                         void* Ainv32, void* A16, void* Ainv16, void* work, double* logdet, int* notposdef,
                         cudaStream_t st) {
  const int B = 128;
  const long long V = 2LL * g.Vh;
  // F per (site, plane), then one chiral block per thread
  g_kernel_launches += 2;
  field_strength_kernel<<<(int)((6 * V + B - 1) / B), B, 0, st>>>(g, static_cast<const double2*>(g64),
                                                                    static_cast<double2*>(work));
  clover_assemble_kernel<<<(int)((2 * V + B - 1) / B), B, 0, st>>>(
      g, static_cast<const double2*>(work), kappa, csw, static_cast<double2*>(A64), static_cast<double2*>(Ainv64),
      static_cast<float4*>(A32), static_cast<float4*>(Ainv32), static_cast<uint4*>(A16), static_cast<uint4*>(Ainv16),
      logdet, notposdef);
}

void launch_clover_apply(int prec, const Geom& g, const void* clover, const void* in, const float* in_norm, void* out,
                         float* out_norm, int nrhs, cudaStream_t st) {
  g_kernel_launches += 1;
  const int B = 128;
  const int nb = (g.Vh * nrhs + B - 1) / B;
  if (prec == 64) clover_apply_kernel<64><<<nb, B, 0, st>>>(g, clover, in, in_norm, out, out_norm, nrhs);
  else if (prec == 32) clover_apply_kernel<32><<<nb, B, 0, st>>>(g, clover, in, in_norm, out, out_norm, nrhs);
  else clover_apply_kernel<16><<<nb, B, 0, st>>>(g, clover, in, in_norm, out, out_norm, nrhs);
}

}  // namespace qcd
