// t-faces of a field for the neighbouring slabs of a time decomposition.
//
// The paper runs its application as two MPI processes, each holding half of the lattice, that
// exchange their boundary data between kernels (Sec. 4); here a lattice is cut into slabs of
// consecutive time slices, one per GPU.  A hopping pass needs, at the sites of its first and last
// local time slice, the spinors one slice beyond the slab.  Only their spin projections enter the
// time hops, so a slab sends six complex numbers per face site in each direction: (1 - g_t) psi of
// its first slice to the slab below (whose last slice hops forward onto it), and U_t^dag (1 + g_t)
// psi of its last slice, with the link it owns already applied, to the slab above.
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_halo)

namespace {

template <int P, int RECON>
__global__ void halo_pack_kernel(Geom g, const void* gauge, const void* in, const float* in_norm, int q, int in_g5,
                                 void* send_lo, void* send_hi, int nrhs) {
  using R = typename Real<P>::T;
  const int F = g.XYZ / 2;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * F * nrhs) return;
  const int f = tid % F, side = (tid / F) & 1, r = tid / (2 * F);
  const int h = side == 0 ? f : (g.T - 1) * F + f;  // face site f of the first / last local slice
  cx<R> sp[12], hs[6];
  if (P == 16) {
    cx<float> v[12];
    SpinorIO<16>::load(in, in_norm, g.Vh, r, h, v);
#pragma unroll
    for (int c = 0; c < 12; c++) sp[c] = cmk(R(v[c].re), R(v[c].im));
  } else {
    SpinorIO<P>::load(in, in_norm, g.Vh, r, h, sp);
  }
  if (in_g5) apply_g5(sp);
  if (side == 0) {
    project<3, -1>(sp, hs);
    HaloIO<P>::store(send_lo, F, r, f, hs);
  } else {
    project<3, +1>(sp, hs);
    cx<R> u[9], w[6];
    GaugeIO<P, RECON>::load(gauge, g.Vh, q, 3, h, u);
    su3_adj_mul(u, hs, w);
    if (g.t0 + g.T - 1 == g.Tg - 1) {
#pragma unroll
      for (int k = 0; k < 6; k++) w[k] = R(g.t_bc) * w[k];
    }
    HaloIO<P>::store(send_hi, F, r, f, w);
  }
}

}  // namespace

void launch_halo_pack(int prec, int recon, const Geom& g, const void* gauge, const void* in, const float* in_norm,
                      int q, int in_g5, void* send_lo, void* send_hi, int nrhs, cudaStream_t st) {
  g_kernel_launches += 1;
  const int n = g.XYZ * nrhs;  // 2 faces x XYZ/2 sites x nrhs
  const int nb = (n + 127) / 128;
  if (prec == 64)
    halo_pack_kernel<64, 18><<<nb, 128, 0, st>>>(g, gauge, in, in_norm, q, in_g5, send_lo, send_hi, nrhs);
  else if (prec == 32) {
    if (recon == 12)
      halo_pack_kernel<32, 12><<<nb, 128, 0, st>>>(g, gauge, in, in_norm, q, in_g5, send_lo, send_hi, nrhs);
    else
      halo_pack_kernel<32, 18><<<nb, 128, 0, st>>>(g, gauge, in, in_norm, q, in_g5, send_lo, send_hi, nrhs);
  } else {
    if (recon == 12)
      halo_pack_kernel<16, 12><<<nb, 128, 0, st>>>(g, gauge, in, in_norm, q, in_g5, send_lo, send_hi, nrhs);
    else
      halo_pack_kernel<16, 18><<<nb, 128, 0, st>>>(g, gauge, in, in_norm, q, in_g5, send_lo, send_hi, nrhs);
  }
}

}  // namespace qcd
