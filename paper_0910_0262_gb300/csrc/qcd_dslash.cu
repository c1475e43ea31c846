// Instantiations and launcher of the fused hopping-term kernels.
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"

#include <cstdlib>

namespace qcd {

namespace {
constexpr int DB = 128;  // threads per block of the hopping kernels

// 1: direction-split kernel (default); 0: one site per thread (QCD_DSLASH_SPLIT=0)
int split_mode() {
  static int mode = -1;
  if (mode < 0) {
    const char* e = getenv("QCD_DSLASH_SPLIT");
    mode = (e && e[0] == '0') ? 0 : 1;
  }
  return mode;
}

template <int P, int RECON>
void launch_epi(int epi, const DslashArgs& a, cudaStream_t st) {
  if (split_mode()) {
    const int nb = (a.g.Vh * a.nrhs + 31) / 32;
    switch (epi) {
      case EPI_NONE: dslash_split_kernel<P, RECON, EPI_NONE><<<nb, 128, 0, st>>>(a); break;
      case EPI_CLOVER_INV: dslash_split_kernel<P, RECON, EPI_CLOVER_INV><<<nb, 128, 0, st>>>(a); break;
      case EPI_XPAY_CG: dslash_split_kernel<P, RECON, EPI_XPAY_CG><<<nb, 128, 0, st>>>(a); break;
      default: dslash_split_kernel<P, RECON, EPI_XPAY><<<nb, 128, 0, st>>>(a); break;
    }
    return;
  }
  if (epi == EPI_XPAY_CG) {  // only the split kernel carries the fused CG update
    const int nb = (a.g.Vh * a.nrhs + 31) / 32;
    dslash_split_kernel<P, RECON, EPI_XPAY_CG><<<nb, 128, 0, st>>>(a);
    return;
  }
  const int nb = (a.g.Vh * a.nrhs + DB - 1) / DB;
  switch (epi) {
    case EPI_NONE: dslash_kernel<P, RECON, EPI_NONE, DB><<<nb, DB, 0, st>>>(a); break;
    case EPI_CLOVER_INV: dslash_kernel<P, RECON, EPI_CLOVER_INV, DB><<<nb, DB, 0, st>>>(a); break;
    default: dslash_kernel<P, RECON, EPI_XPAY, DB><<<nb, DB, 0, st>>>(a); break;
  }
}
}  // namespace

int dslash_block() { return DB; }

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
