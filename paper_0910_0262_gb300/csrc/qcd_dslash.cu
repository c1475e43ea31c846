// Instantiations and launcher of the fused hopping-term kernels.
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"


namespace qcd {

QCD_DEBUG_TAKE(debug_take_dslash)

namespace {

template <int P, int RECON>
void launch_split(int epi, const DslashArgs& a, cudaStream_t st) {
  const int nb = (a.g.Vh + 31) / 32;
  switch (epi) {
    case EPI_NONE: dslash_split_kernel<P, RECON, EPI_NONE><<<nb, 128, 0, st>>>(a); break;
    case EPI_CLOVER_INV: dslash_split_kernel<P, RECON, EPI_CLOVER_INV><<<nb, 128, 0, st>>>(a); break;
    case EPI_XPAY_CG: dslash_split_kernel<P, RECON, EPI_XPAY_CG><<<nb, 128, 0, st>>>(a); break;
    default: dslash_split_kernel<P, RECON, EPI_XPAY><<<nb, 128, 0, st>>>(a); break;
  }
}

// FP64 passes without the fused CG update on pair units (one wave of 64-thread blocks at 16^4; 7 or 6
// blocks per SM instead of 8, with fewer spills: 81.3 / 87.4 against 81.5 us)
template <int RECON>
void launch_pair64(int epi, const DslashArgs& a, cudaStream_t st) {
  const int nb = (a.g.Vh + 31) / 32;
  switch (epi) {
    case EPI_NONE: dslash_pair64_kernel<RECON, EPI_NONE><<<nb, 64, 0, st>>>(a); break;
    case EPI_CLOVER_INV: dslash_pair64_kernel<RECON, EPI_CLOVER_INV><<<nb, 64, 0, st>>>(a); break;
    default: dslash_pair64_kernel<RECON, EPI_XPAY><<<nb, 64, 0, st>>>(a); break;
  }
}

template <int RECON>
void launch_split_fp16(int epi, const DslashArgs& a, cudaStream_t st) {
  const int nb = (a.g.Vh + 31) / 32;
  switch (epi) {
    case EPI_NONE: dslash_split_fp16_kernel<RECON, EPI_NONE><<<nb, 128, 0, st>>>(a); break;
    case EPI_CLOVER_INV: dslash_split_fp16_kernel<RECON, EPI_CLOVER_INV><<<nb, 128, 0, st>>>(a); break;
    case EPI_XPAY_CG: dslash_split_fp16_kernel<RECON, EPI_XPAY_CG><<<nb, 128, 0, st>>>(a); break;
    default: dslash_split_fp16_kernel<RECON, EPI_XPAY><<<nb, 128, 0, st>>>(a); break;
  }
}

template <int P, int RECON, bool STAGED>
void launch_site_k(int epi, const DslashArgs& a, int nb, cudaStream_t st) {
  if constexpr (P == 16) {
    switch (epi) {
      case EPI_NONE: dslash_site_fp16_kernel<RECON, EPI_NONE, STAGED><<<nb, 128, 0, st>>>(a); break;
      case EPI_CLOVER_INV: dslash_site_fp16_kernel<RECON, EPI_CLOVER_INV, STAGED><<<nb, 128, 0, st>>>(a); break;
      case EPI_XPAY_CG: dslash_site_fp16_kernel<RECON, EPI_XPAY_CG, STAGED><<<nb, 128, 0, st>>>(a); break;
      default: dslash_site_fp16_kernel<RECON, EPI_XPAY, STAGED><<<nb, 128, 0, st>>>(a); break;
    }
  } else {
    switch (epi) {
      case EPI_NONE: dslash_site_kernel<P, RECON, EPI_NONE, STAGED><<<nb, 128, 0, st>>>(a); break;
      case EPI_CLOVER_INV: dslash_site_kernel<P, RECON, EPI_CLOVER_INV, STAGED><<<nb, 128, 0, st>>>(a); break;
      case EPI_XPAY_CG: dslash_site_kernel<P, RECON, EPI_XPAY_CG, STAGED><<<nb, 128, 0, st>>>(a); break;
      default: dslash_site_kernel<P, RECON, EPI_XPAY, STAGED><<<nb, 128, 0, st>>>(a); break;
    }
  }
}

template <int P, int RECON>
void launch_site(int epi, const DslashArgs& a, cudaStream_t st) {
  const int G = a.nrhs == 1 ? 4 : (a.nrhs == 2 ? 2 : 1);
  const int nb = (a.g.Vh + 32 * G - 1) / (32 * G);
  // staging pays once its cost is spread over enough RHS: FP32 from 4 RHS (32^3 x 64, 8 RHS: 857 ->
  // 702 us; 48^3 x 96, 4 RHS: 2628 -> 2362 us), FP16 (cheaper links and clover to decode) from 8
  // (48^3 x 96, 4 RHS: 1816 us unstaged, 2025 staged; 32^3 x 64, 8 RHS: 695 -> 680 us)
  if (a.nrhs >= (P == 16 ? 8 : 3)) launch_site_k<P, RECON, true>(epi, a, nb, st);
  else launch_site_k<P, RECON, false>(epi, a, nb, st);
}

// Half volume from which one RHS runs one thread per site: below it the four threads per site of
// the direction-split kernel are needed to fill the GPU (16^4: 32768 sites per parity would give
// 256 blocks), above it the site kernel's lower instruction count and absence of block barriers win
// (32^3 x 64: FP16 147 -> 116 us, FP32 170 -> 164 us per hopping launch).
#ifndef QCD_SITE_KERNEL_MIN_VH
#define QCD_SITE_KERNEL_MIN_VH (1 << 17)
#endif
const int SITE_KERNEL_MIN_VH = QCD_SITE_KERNEL_MIN_VH;

// FP32/FP16: one thread per (site, RHS) for several RHS or large lattices, else the direction-split
// kernel; FP64 (bound by the FP64 pipe): pair units for any number of RHS, the split kernel for the
// fused CG update
template <int P, int RECON>
void launch_prec(int epi, const DslashArgs& a, cudaStream_t st) {
  if constexpr (P == 64) {
    // pair units against the four-warp split kernel, M^dag M passes: 16^4 83.3 vs 84.0 us, 32^3 x 64
    // 2222 vs 2292 us, 8 RHS 17.7 vs 18.7 ms (one thread per site was within 7% of the split kernel
    // either way); the fused CG update stays on the split kernel
    if (epi == EPI_XPAY_CG) launch_split<P, RECON>(epi, a, st);
    else launch_pair64<RECON>(epi, a, st);
  } else {
    if (a.nrhs > 1 || a.g.Vh >= SITE_KERNEL_MIN_VH) launch_site<P, RECON>(epi, a, st);
    else if constexpr (P == 16) launch_split_fp16<RECON>(epi, a, st);
    else launch_split<P, RECON>(epi, a, st);
  }
}

// the split kernel with t-slab halos (no fused CG epilogue)
template <int P, int RECON>
void launch_halo(int epi, const DslashArgs& a, cudaStream_t st) {
  const int nb = (a.g.Vh + 31) / 32;
  if constexpr (P == 16) {
    switch (epi) {
      case EPI_NONE: dslash_split_fp16_kernel<RECON, EPI_NONE, true><<<nb, 128, 0, st>>>(a); break;
      case EPI_CLOVER_INV: dslash_split_fp16_kernel<RECON, EPI_CLOVER_INV, true><<<nb, 128, 0, st>>>(a); break;
      default: dslash_split_fp16_kernel<RECON, EPI_XPAY, true><<<nb, 128, 0, st>>>(a); break;
    }
  } else {
    switch (epi) {
      case EPI_NONE: dslash_split_kernel<P, RECON, EPI_NONE, true><<<nb, 128, 0, st>>>(a); break;
      case EPI_CLOVER_INV: dslash_split_kernel<P, RECON, EPI_CLOVER_INV, true><<<nb, 128, 0, st>>>(a); break;
      default: dslash_split_kernel<P, RECON, EPI_XPAY, true><<<nb, 128, 0, st>>>(a); break;
    }
  }
}

}  // namespace

void launch_dslash_halo(int prec, int recon, int epi, const DslashArgs& a, cudaStream_t st) {
  g_kernel_launches += 1;
  if (prec == 64) launch_halo<64, 18>(epi, a, st);
  else if (prec == 32) {
    if (recon == 12) launch_halo<32, 12>(epi, a, st);
    else launch_halo<32, 18>(epi, a, st);
  } else {
    if (recon == 12) launch_halo<16, 12>(epi, a, st);
    else launch_halo<16, 18>(epi, a, st);
  }
}

void launch_dslash(int prec, int recon, int epi, const DslashArgs& a, cudaStream_t st) {
  g_kernel_launches += 1;
  if (prec == 64) launch_prec<64, 18>(epi, a, st);
  else if (prec == 32) {
    if (recon == 12) launch_prec<32, 12>(epi, a, st);
    else launch_prec<32, 18>(epi, a, st);
  } else {
    if (recon == 12) launch_prec<16, 12>(epi, a, st);
    else launch_prec<16, 18>(epi, a, st);
  }
}

}  // namespace qcd
