// FP64 3x3 complex matrix helpers and link access by lattice coordinates, shared by
// the clover-term and fermion-force kernels.
#pragma once

#include "qcd_internal.cuh"

namespace qcd {

using C = cx<double>;

struct M3 {
  C e[9];
};

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C s = a.e[3 * i] * b.e[j];
      s = cfma(a.e[3 * i + 1], b.e[3 + j], s);
      s = cfma(a.e[3 * i + 2], b.e[6 + j], s);
      c.e[3 * i + j] = s;
    }
  return c;
}
// acc + a conj(b) (four FMAs)
__device__ __forceinline__ C cfma_nc(C a, C b, C acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im);
  acc.im = fma(-a.re, b.im, acc.im);
  return acc;
}

// a * b^dag
__device__ __forceinline__ M3 mul_nd(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C s = a.e[3 * i] * conj(b.e[3 * j]);
      s = cfma_nc(a.e[3 * i + 1], b.e[3 * j + 1], s);
      s = cfma_nc(a.e[3 * i + 2], b.e[3 * j + 2], s);
      c.e[3 * i + j] = s;
    }
  return c;
}
// a^dag * b
__device__ __forceinline__ M3 mul_dn(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C s = cmk(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; k++) s = cfmac(a.e[3 * k + i], b.e[3 * k + j], s);
      c.e[3 * i + j] = s;
    }
  return c;
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// U_mu at lexicographic coordinates (x, y, z, t), wrapped periodically
__device__ __forceinline__ M3 link_at(const Geom& g, const double2* g64, int x, int y, int z, int t, int mu) {
  x = wrap(x, g.X);
  y = wrap(y, g.Y);
  z = wrap(z, g.Z);
  t = wrap(t, g.T);
  const int i = x + g.X * (y + g.Y * (z + g.Z * t));
  const int p = (x + y + z + t) & 1;
  const double2* q = g64 + (size_t)(p * 4 + mu) * 9 * g.Vh + (i >> 1);
  M3 u;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 v = __ldg(q + (size_t)k * g.Vh);
    u.e[k] = cmk(v.x, v.y);
  }
  return u;
}


__device__ __forceinline__ M3 m3_add(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int k = 0; k < 9; k++) c.e[k] = a.e[k] + b.e[k];
  return c;
}

__device__ __forceinline__ M3 m3_dag(const M3& a) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) c.e[3 * i + j] = conj(a.e[3 * j + i]);
  return c;
}

}  // namespace qcd
