// Instantiations and launcher of the fused hopping-term kernels.
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"


namespace qcd {

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

template <int P, int RECON>
void launch_site_multi(int epi, const DslashArgs& a, cudaStream_t st) {
  const int G = a.nrhs == 2 ? 2 : 1;
  const int nb = (a.g.Vh + 32 * G - 1) / (32 * G);
  switch (epi) {
    case EPI_NONE: dslash_site_multi_kernel<P, RECON, EPI_NONE><<<nb, 128, 0, st>>>(a); break;
    case EPI_CLOVER_INV: dslash_site_multi_kernel<P, RECON, EPI_CLOVER_INV><<<nb, 128, 0, st>>>(a); break;
    case EPI_XPAY_CG: dslash_site_multi_kernel<P, RECON, EPI_XPAY_CG><<<nb, 128, 0, st>>>(a); break;
    default: dslash_site_multi_kernel<P, RECON, EPI_XPAY><<<nb, 128, 0, st>>>(a); break;
  }
}

// one RHS: the direction-split kernel (four threads per site); several RHS in FP32/FP16: one thread
// per (site, RHS); FP64 (bound by the FP64 pipe): the split kernel for any number of RHS
template <int P, int RECON>
void launch_prec(int epi, const DslashArgs& a, cudaStream_t st) {
  if constexpr (P == 64) {
    launch_split<P, RECON>(epi, a, st);
  } else {
    if (a.nrhs > 1) launch_site_multi<P, RECON>(epi, a, st);
    else if constexpr (P == 16) launch_split_fp16<RECON>(epi, a, st);
    else launch_split<P, RECON>(epi, a, st);
  }
}

}  // namespace

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
