// Host-side launchers of the CUDA kernels (internal to libqcd; not part of the C ABI).
#pragma once

#include <atomic>

#include <cuda_runtime.h>

#include "qcd.h"
#include "qcd_internal.cuh"

namespace qcd {

// Read-only view of a context, for entry points defined outside qcd_api.cu (filled by ctx_view;
// false for a null context)
struct CtxView {
  Geom g;
  cudaStream_t st;
  int device;
  const void* g64;
  const void* A_even64;
  const void* Ainv_odd64;
  double kappa;
  bool have_gauge, have_clover;
  bool slab;
};
bool ctx_view(const qcd_ctx* c, CtxView* v);

// kernels launched by the library since the last reset (profiling)
extern std::atomic<long long> g_kernel_launches;

// ---- persistent single-RHS CG iteration (qcd_cg_persistent.cu)
struct PersistentCGArgs {
  Geom g;
  const void* gauge;           // links of the inner precision
  const void* clover_inv_odd;  // A_oo^-1 of the inner precision
  const void* clover_even;     // A_ee of the inner precision
  void *p, *t, *y;             // inner-precision fields (t odd, p and y even)
  float *p_n, *t_n, *y_n;      // FP16 norms (null otherwise)
  void *x, *r;                 // x_lo, r_lo (FP64 for inner 64, else FP32)
  double k2;                   // kappa^2
  CGState* cg;                 // state of the single RHS
  CGControl* ctl;
  double *part_pap, *part_rr;  // one slot per block
  int slots;                   // slots in each; the grid never exceeds it
  unsigned* bar_count;         // barrier arrivals, zeroed before the launch
  unsigned* bar_flag;          // release word of the summing barriers, zeroed before the launch
  double* totals;              // [2]: the grid totals the summing barriers publish (pAp, |r|^2)
  int* bar_err;                // set when a barrier wait gave up
  int iter_limit;              // total iterations of the RHS (over all launches) at which to stop
  int* round_out;              // non-null: 2 x iterations this launch ran, + 1 if it raised a reliable
                               // update, written at its end
};
cudaError_t launch_cg_persistent(int prec, int recon, const PersistentCGArgs& q, cudaStream_t st);
// one grid barrier that a block never reaches (the wait must give up and set *err)
cudaError_t launch_barrier_probe(unsigned* count, int* err, cudaStream_t st);

// ---- layout (qcd_layout.cu)
void launch_pack_gauge(const Geom& g, const double2* canon, void* g64, void* g32, int recon32, void* g16,
                       int recon16, cudaStream_t st);
void launch_spinor_to_native(int prec, const Geom& g, const double2* canon, void* nat, float* norm, int nrhs,
                             cudaStream_t st);
void launch_spinor_to_canon(int prec, const Geom& g, const void* nat, const float* norm, double2* canon, int nrhs,
                            cudaStream_t st);
void launch_check_finite(const double* data, size_t n, int* flag, cudaStream_t st);

// ---- clover (qcd_clover.cu)
// A (both parities) and A^-1 (both parities) in FP64, FP32 and FP16; flag set if a block is not positive definite.
// work: 6 * 9 * V double2 for the field strengths (two kernels: F per site and plane, then one chiral
// block per thread); logdet: [parity][block][Vh] log det of each 6x6 block.
void launch_clover_build(const Geom& g, const void* g64, double kappa, double csw, void* A64, void* Ainv64,
                         void* A32, void* Ainv32, void* A16, void* Ainv16, void* work, double* logdet,
                         int* notposdef, cudaStream_t st);
// out = C in for a site-local clover field C of parity-matched fields
void launch_clover_apply(int prec, const Geom& g, const void* clover, const void* in, const float* in_norm,
                         void* out, float* out_norm, int nrhs, cudaStream_t st);

// ---- debug builds: each translation unit's index-violation word, returned and cleared (qcd_internal.cuh)
unsigned debug_take_blas();
unsigned debug_take_cg_persistent();
unsigned debug_take_clover();
unsigned debug_take_dslash();
unsigned debug_take_force();
unsigned debug_take_halo();
unsigned debug_take_layout();
unsigned debug_take_md();
unsigned debug_take_probe();
// one thread loads the FP64 spinor at site index Vh (one past the last site) of buf, which holds
// 13 Vh double2, so that the load stays inside buf even unchecked; debug builds record DBG_SPINOR
void launch_debug_index_probe(const Geom& g, const double2* buf, double* out, cudaStream_t st);

// ---- hopping term (qcd_dslash.cu)
struct DslashArgs;
void launch_dslash(int prec, int recon, int epi, const DslashArgs& a, cudaStream_t st);
// the same operators on the sites of a t-slab, time hops that leave the slab taken from a.halo_lo /
// a.halo_hi (epi: EPI_NONE, EPI_CLOVER_INV or EPI_XPAY)
void launch_dslash_halo(int prec, int recon, int epi, const DslashArgs& a, cudaStream_t st);
// t-faces of a field of parity q (precision prec, nrhs RHS, native layout) for the neighbouring slabs:
// send_lo[f] = (1 - g_t) (g5) psi at the face site f of local time 0; send_hi[f] = U_t(x)^dag (1 + g_t)
// (g5) psi at the face site f of the last local time slice, times t_bc if that slice is the global
// time Tg - 1 (HaloIO layout; gauge of the operator's precision)
void launch_halo_pack(int prec, int recon, const Geom& g, const void* gauge, const void* in, const float* in_norm,
                      int q, int in_g5, void* send_lo, void* send_hi, int nrhs, cudaStream_t st);

// ---- BLAS-1 and CG steps (qcd_blas.cu); 2-D grids (sites x RHS)
// gate (these three): non-null, the kernel returns at once unless *gate != 0 (the reliable-update
// steps, enqueued ahead of knowing whether an update is due)
// p = r + beta p
void launch_p_update(int prec_r, int prec_p, const Geom& g, int nrhs, const void* r, const float* rn, void* p,
                     float* pn, const CGState* cg, const int* halt, cudaStream_t st, const int* gate = nullptr);
// x_hi += x_lo ; x_lo = 0
void launch_accumulate_x(int prec_r, const Geom& g, int nrhs, double2* x_hi, void* x_lo, float* x_lon,
                         cudaStream_t st, const int* gate = nullptr);
// r_lo = b - Ap_hi ; |b - Ap_hi|^2 -> reduction (FIN_CG_TRUE)
void launch_true_residual(int prec_r, const Geom& g, int nrhs, const double2* b, const double2* Ap, void* r_lo,
                          float* r_lon, const ReduceArgs& red, cudaStream_t st, const int* gate = nullptr);
// *gate = 0
void launch_gate_clear(int* gate, cudaStream_t st);
// x_lo += alpha p, r_lo -= alpha Ap (alpha from cg), |r_lo|^2 -> reduction (nrhs RHS; prec_r 64: all FP64)
void launch_xr_update(int prec_r, int prec_p, const Geom& g, int nrhs, void* x_lo, void* r_lo, const void* p,
                      const float* pn, const void* ap, const float* apn, const CGState* cg, const ReduceArgs& red,
                      cudaStream_t st);
// finalize_total(red, r, totals[r]) for r < nrhs on the device (totals summed over the slabs)
void launch_finalize(const ReduceArgs& red, const double* totals, int nrhs, cudaStream_t st);
// |v|^2 (FP64 native) -> reduction
void launch_norm2(const Geom& g, int nrhs, const double2* v, const ReduceArgs& red, cudaStream_t st);
// ---- molecular dynamics (qcd_md.cu); canonical link fields [V][4][3][3] complex128
// Wilson gauge force (or gradient) of beta sum (1 - Re tr P / 3) from the FP64 packed links, written
// to or added to out
void launch_gauge_force(const Geom& g, double beta, const void* g64, double2* out, bool gradient, bool accumulate,
                        cudaStream_t st);
// result[0] = sum over sites and planes of Re tr P_{mu nu}(x) / 3 (FIN_STORE)
void launch_plaquette(const Geom& g, const void* g64, const ReduceArgs& red, cudaStream_t st);
// result[0] = sum of |v_j|^2 over n complex numbers (FIN_STORE)
void launch_flat_norm2(size_t n, const double2* v, const ReduceArgs& red, cudaStream_t st);
// result[0] + i result[1] = sum over spatial sites of tr prod_t U_t / 3 (FIN_STORE)
void launch_polyakov(const Geom& g, const void* g64, const ReduceArgs& red, cudaStream_t st);
// result[r] = Re sum_j conj(a_j) b_j over the n complex numbers of RHS r (FIN_STORE)
void launch_flat_redot(size_t n, int nrhs, const double2* a, const double2* b, const ReduceArgs& red,
                       cudaStream_t st);
// U <- reunitarised exp(eps P) U for nlinks canonical links
void launch_link_update(size_t nlinks, double eps, const double2* P, double2* U, cudaStream_t st);

// result[p] = sum of v[p][0 .. 2 Vh) for p = 0, 1 (FIN_STORE)
void launch_parity_sum(const Geom& g, const double* v, const ReduceArgs& red, cudaStream_t st);
// y = a x + b y over n complex numbers
void launch_axpby(size_t n, double a, const double2* x, double b, double2* y, cudaStream_t st);
// Re <a, b> (FP64 native) -> reduction
void launch_redot(const Geom& g, int nrhs, const double2* a, const double2* b, const ReduceArgs& red,
                  cudaStream_t st);
void launch_zero(void* ptr, size_t bytes, cudaStream_t st);

}  // namespace qcd
