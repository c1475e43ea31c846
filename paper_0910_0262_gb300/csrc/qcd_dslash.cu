// Instantiations and launcher of the fused hopping-term kernels.
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"

namespace qcd {

namespace {
constexpr int DB = 128;  // threads per block of the hopping kernels

template <int P, int RECON>
void launch_epi(int epi, const DslashArgs& a, cudaStream_t st) {
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
