// Instantiations and launcher of the fused hopping-term kernels.
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"


namespace qcd {

namespace {

template <int P, int RECON, bool MULTI>
void launch_epi(int epi, const DslashArgs& a, cudaStream_t st) {
  const int nb = (a.g.Vh + 31) / 32;
  switch (epi) {
    case EPI_NONE: dslash_split_kernel<P, RECON, EPI_NONE, MULTI><<<nb, 128, 0, st>>>(a); break;
    case EPI_CLOVER_INV: dslash_split_kernel<P, RECON, EPI_CLOVER_INV, MULTI><<<nb, 128, 0, st>>>(a); break;
    case EPI_XPAY_CG: dslash_split_kernel<P, RECON, EPI_XPAY_CG, MULTI><<<nb, 128, 0, st>>>(a); break;
    default: dslash_split_kernel<P, RECON, EPI_XPAY, MULTI><<<nb, 128, 0, st>>>(a); break;
  }
}

template <int P, int RECON>
void launch_epi(int epi, const DslashArgs& a, cudaStream_t st) {
  if (a.nrhs > 1) launch_epi<P, RECON, true>(epi, a, st);
  else launch_epi<P, RECON, false>(epi, a, st);
}

}  // namespace

void launch_dslash(int prec, int recon, int epi, const DslashArgs& a, cudaStream_t st) {
  g_kernel_launches += 1;
  if (prec == 64) launch_epi<64, 18>(epi, a, st);
  else if (prec == 32) {
    if (recon == 12) launch_epi<32, 12>(epi, a, st);
    else launch_epi<32, 18>(epi, a, st);
  } else {
    if (recon == 12) launch_epi<16, 12>(epi, a, st);
    else launch_epi<16, 18>(epi, a, st);
  }
}

}  // namespace qcd
