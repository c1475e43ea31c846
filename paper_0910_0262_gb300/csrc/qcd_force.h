// Fermion-force launchers (internal to libqcd).
#pragma once

#include <atomic>

#include <cuda_runtime.h>

#include "qcd_internal.cuh"

namespace qcd {

extern std::atomic<long long> g_kernel_launches;

// bytes of one per-site, per-plane 3x3 complex field over the full lattice (6 planes)
size_t force_clover_bytes(const Geom& g);

// Force for S = sum_r phi_r^dag (Mhat^dag Mhat)^-1 phi_r, given per RHS the native FP64 fields
// X_e, X_o = A_oo^-1 D_oe X_e, Y_e = Mhat X_e, Y_o = A_oo^-1 D_eo^dag Y_e.
// 1. C_{mu nu} per site and plane into Cbuf (force_clover_bytes).
// The fields of one batch of nrhs right-hand sides; accumulate adds to Cbuf (later batches).
void launch_force_coeff(const Geom& g, double kappa, double csw, int nrhs, const double2* Xe, const double2* Xo,
                        const double2* Ye, const double2* Yo, double2* Cbuf, bool accumulate, cudaStream_t st);
// bytes of the edge insertions E (two per site and plane)
size_t force_edge_bytes(const Geom& g);
// 2. per link and plane containing it, E = C(x) U(x) + U(x) C(x + dir) into Ebuf (force_edge_bytes),
// from the coefficients in Cbuf.
void launch_force_edges(const Geom& g, const void* g64, const double2* Cbuf, double2* Ebuf, cudaStream_t st);
// 3. per link: G, or F = -1/2 P_TA(U G^dag) (linear in G), into out (canonical [V][4][3][3]
// complex128): the hopping part of this batch, plus the clover part from Ebuf when with_clover;
// accumulate adds to out.
void launch_force_links(const Geom& g, double kappa, int nrhs, const void* g64, const double2* Xe, const double2* Xo,
                        const double2* Ye, const double2* Yo, const double2* Ebuf, double2* out, bool gradient,
                        bool with_clover, bool accumulate, cudaStream_t st);
// 4. add to Cbuf the coefficients of the clover determinant term S_det = -2 sum_{x odd} log det A(x)
// (at odd sites), from the FP64 A_oo^-1 blocks ([36][Vh] double2 of the odd parity).
void launch_force_det_coeff(const Geom& g, double kappa, double csw, const double2* Ainv_odd, double2* Cbuf,
                            cudaStream_t st);
// conventional FP64 flop counts: per link of kernel 2, per site of kernel 1
double force_link_flops(int nrhs, bool with_clover);
double force_edge_flops();
double force_coeff_flops(int nrhs);

}  // namespace qcd
