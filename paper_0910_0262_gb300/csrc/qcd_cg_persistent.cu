// Persistent CG iteration for one right-hand side.
//
// On small lattices the inner CG iteration is bound by kernel launch latency and ramp-up, not by
// memory bandwidth: its five launches (four hopping passes, the p update) each touch a working set
// that fits in L2.  This cooperative kernel keeps every block resident and runs the iteration's
// phases back to back, separated by grid barriers, until a reliable-update or convergence trigger (or
// an iteration cap) -- the same arithmetic as the graph of launches.
// At a reliable-update trigger it raises the update's gate (ctl->rel_go), so that the update's
// launches, enqueued behind it before the trigger is known, run; a launch that finds the RHS
// converged or halted returns at once.
//
//   phase 1  t  = A_oo^-1 D_oe p
//   phase 2  y  = A_ee p - kappa^2 D_eo t,     |y|^2 = <p, Mhat^dag Mhat p>  -> alpha
//   phase 3  t  = A_oo^-1 D_oe g5 y
//   phase 4  Ap = g5 (A_ee g5 y - kappa^2 D_eo t), x += alpha p, r -= alpha Ap, |r|^2 -> beta
//   phase 5  p  = r + beta p
//
// FP32 forms phase 5 where phases 1 and 2 of the next iteration read p (p = r + beta p from the
// previous iteration's r, p and beta), so its iteration has four phases; phase 5 runs as a phase only
// when a launch stops at its iteration cap.  Sums are formed per block over a fixed set of site blocks;
// the barrier that closes a sum has the last-arriving block add the per-block partials in block order
// and publish the total, so all blocks hold the same alpha and beta.  Fields written inside
// the kernel are read with ordinary loads after the barrier.  Every barrier wait is bounded: a
// block that has waited too long sets an error word and all blocks return (the host reports
// QCD_ERR_TIMEOUT).
#include <mutex>

#include "qcd_dslash.cuh"
#include "qcd_kernels.h"

namespace qcd {

QCD_DEBUG_TAKE(debug_take_cg_persistent)

namespace {

constexpr unsigned BARRIER_SPIN_LIMIT = 1u << 22;  // polls of an L2 word: about a second or more

// Grid-wide barrier of a cooperative launch.  Arrivals count up one word, which the host zeroes
// before the launch; the k-th barrier of the launch is passed when the word reaches k * gridDim.x.
// target holds that value for this block and is advanced here.  The arrival is a release and the
// poll an acquire at GPU scope, so the block's earlier writes are visible to every block after the
// barrier.  Returns false (on every thread of the block) if this block gave up waiting or another
// block reported an error.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& target, int* err) {
  __shared__ int ok;
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    unsigned spins = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((++spins & 31) == 0) {
        if (*reinterpret_cast<volatile int*>(err)) {
          ok = 0;
          break;
        }
        if (spins > BARRIER_SPIN_LIMIT) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Bounded wait of thread 0 until *word reaches target (an acquire at GPU scope); false if the wait
// gave up (it then sets *err) or another block reported an error.
__device__ __forceinline__ bool wait_word(const unsigned* word, unsigned target, int* err) {
  unsigned spins = 0;
  while (true) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(word) : "memory");
    if ((int)(v - target) >= 0) return true;
    if ((++spins & 31) == 0) {
      if (*reinterpret_cast<volatile int*>(err)) return false;
      if (spins > BARRIER_SPIN_LIMIT) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
}

template <int BLOCK>
__device__ __forceinline__ double grid_total(const double* part);

// Grid-wide barrier that also sums one double per block (`mine`, thread 0's value): every block
// writes its partial and arrives on the counter with an acquire-release add; the block whose arrival
// completes the count reads all partials (the add's acquire makes them visible), sums them in block
// order -- the same bits whichever block arrives last -- publishes the total and releases the others
// through *flag.  The total comes out of the barrier instead of after it (at 16^4 the separate sum of
// 512 partials after a barrier took 2.5 us).  Returns false as grid_barrier does; *total: the sum.
template <int BLOCK>
__device__ __forceinline__ bool grid_barrier_sum(unsigned* count, unsigned* flag, unsigned& target, int* err,
                                                 double* part, double* slot, double mine, double* total) {
  __shared__ int ok, last;
  __shared__ double tot;
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    part[blockIdx.x] = mine;
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
    last = old == target - 1;
    ok = 1;
  }
  __syncthreads();
  if (last) {
    const double t = grid_total<BLOCK>(part);
    if (threadIdx.x == 0) {
      *slot = t;
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(target) : "memory");
    }
  }
  if (threadIdx.x == 0) {
    ok = wait_word(flag, target, err) ? 1 : 0;
    if (ok) tot = __ldcg(slot);
  }
  __syncthreads();
  *total = tot;
  return ok != 0;
}

// sum of one double per thread over the BLOCK threads of the block (thread 0 gets it)
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[BLOCK / 32];
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < BLOCK / 32; w++) s += sm[w];
  }
  __syncthreads();
  return s;
}

// sum of the gridDim.x per-block partials, on every thread: each thread adds a fixed strided
// subset (its loads issued together), then a fixed shuffle / shared-memory tree, so every block
// gets the same bits
template <int BLOCK>
__device__ __forceinline__ double grid_total(const double* part) {
  __shared__ double sm[BLOCK / 32];
  double s = 0.0;
  for (int base = 0; base < (int)gridDim.x; base += 8 * BLOCK) {
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const int j = base + (int)threadIdx.x + BLOCK * i;
      v[i] = j < (int)gridDim.x ? __ldcg(part + j) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) s += v[i];
  }
  for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; w++) t += sm[w];
  __syncthreads();
  return t;
}

// load mode of the fields the kernel writes: cached in L1, which the acquire of each grid barrier
// invalidates, so neighbours shared by the sites of a block are read from L2 once
constexpr int LDM = LD_CA;

// Shape of the persistent kernel.  FP32 / FP16 iterations run each phase as pair units (two warps
// per block of 32 sites, so that the resident grid covers a 16^4 parity in one round), two pairs
// per 128-thread block; FP64 (bound by the FP64 pipe) runs four-warp split units.  Four blocks per
// SM either way.  (One 512-thread block of eight pairs per SM made the grid barrier cheaper, 1.6
// against 2.2 us at 16^4, but the sum of the per-block partials slower, 4.6 against 2.5 us.)
template <int P>
struct PcShape {
  static constexpr bool PAIR = P != 64;
  static constexpr int THREADS = 128;
  static constexpr int MIN_BLOCKS = 4;
  static constexpr int PAIRS = THREADS / 64;
  static constexpr int PAIR_STAGE = PairStage<P == 64 ? 32 : P, EPI_XPAY_CG>::U4;  // per warp
  // pair units: the pairs' exchange areas and the warps' staging rows, in dynamic shared memory
  static constexpr size_t DYN = PAIR ? sizeof(PairXch<float>) * 2 * PAIRS + sizeof(uint4) * (THREADS / 32) * PAIR_STAGE
                                     : 0;
};

// one phase over the site blocks this block owns; returns the thread's share of the phase's sum
template <int P, int RECON, int EPI, bool LAZY = false>
__device__ __forceinline__ double run_phase(const DslashArgs& A, cx<typename Real<P>::T> (*part)[12][32],
                                            PairXch<float> (*xch)[2], uint4* stage, double alpha) {
  const int nsb = (A.g.Vh + 31) / 32;
  double v = 0.0;
  if constexpr (PcShape<P>::PAIR) {
    constexpr int NP = PcShape<P>::PAIRS;
    const int w = threadIdx.x >> 5, q = w >> 1, d = w & 1;
    int slot = 0;
    // site block sb goes to block sb mod grid, pair sb / grid: every SM gets a share of the phase
    for (int sb = q * gridDim.x + blockIdx.x; sb < nsb; sb += NP * gridDim.x) {
      int hh;
      bool valid;
      Site s;
      split_prologue(A, sb, hh, valid, s);
      v += pair_unit<P, RECON, EPI, LDM, LAZY>(A, hh, valid, s, d, q, true, alpha, &xch[q][slot],
                                               stage + w * PcShape<P>::PAIR_STAGE);
      slot ^= 1;
    }
  } else {
    for (int sb = blockIdx.x; sb < nsb; sb += gridDim.x) {
      int hh;
      bool valid;
      Site s;
      split_prologue(A, sb, hh, valid, s);
      v += split_unit<P, RECON, EPI, LDM>(A, hh, valid, s, 0, true, alpha, part, stage, true);
    }
  }
  return v;
}

template <int P, int RECON>
__global__ void __launch_bounds__(PcShape<P>::THREADS, PcShape<P>::MIN_BLOCKS)
    cg_persistent_kernel(PersistentCGArgs Q) {
  using R = typename Real<P>::T;
  constexpr int PR = P == 64 ? 64 : 32;
  using RR = typename Real<PR>::T;
  constexpr bool PAIR = PcShape<P>::PAIR;
  constexpr int BLOCK = PcShape<P>::THREADS;
  __shared__ cx<R> part[PAIR ? 1 : 4][12][32];                            // split unit: partial sums
  __shared__ uint4 split_stage[PAIR ? 1 : Stage<P, EPI_XPAY_CG>::U4];     // split unit: staging
  extern __shared__ __align__(16) unsigned char pc_dyn[];                  // pair units (PcShape::DYN)
  PairXch<float>(*xch)[2] = reinterpret_cast<PairXch<float>(*)[2]>(pc_dyn);
  uint4* stage = PAIR ? reinterpret_cast<uint4*>(pc_dyn + sizeof(PairXch<float>) * 2 * PcShape<P>::PAIRS)
                      : split_stage;
  const CGState st0 = *Q.cg;
  // an earlier launch of the batch whose barrier gave up leaves *bar_err set: do nothing
  if (!st0.active || Q.ctl->halt || st0.iters >= Q.iter_limit || *reinterpret_cast<volatile int*>(Q.bar_err)) {
    if (Q.round_out && blockIdx.x == 0 && threadIdx.x == 0) *Q.round_out = 0;
    return;
  }
  double rr = st0.rr, rr_prev = st0.rr_prev;
  int iters = st0.iters, since = st0.since_reliable;
  const int every = Q.ctl->reliable_every;
  const double delta2 = Q.ctl->delta2;
  const int Vh = Q.g.Vh;

  DslashArgs a1;  // t = A_oo^-1 D_oe (g5) v
  memset(&a1, 0, sizeof a1);
  a1.g = Q.g;
  a1.p = 1;
  a1.nrhs = 1;
  a1.gauge = Q.gauge;
  a1.out = Q.t;
  a1.out_norm = Q.t_n;
  a1.clover = Q.clover_inv_odd;
  DslashArgs a2 = a1;  // even output, clover A_ee
  a2.p = 0;
  a2.clover = Q.clover_even;
  a2.a = -Q.k2;
  a2.in = Q.t;
  a2.in_norm = Q.t_n;

  // FP32: the p update p = r + beta p of iteration k is formed where p is read in phases 1 and 2 of
  // iteration k+1 (phase 2 writes it back), so phase 5 and its grid barrier are not needed; the first
  // iteration of a launch finds p already updated (coefficients 0, 1)
  constexpr bool LAZY = P == 32;
  bool first = true;
  double alpha = 0.0, beta = 0.0, pAp = 0.0;
  unsigned bar_target = 0;
  while (true) {
    // phase 1
    a1.in = Q.p;
    a1.in_norm = Q.p_n;
    a1.in_g5 = 0;
    a1.lz_r = Q.r;
    a1.lz_a = first ? 0.f : 1.f;
    a1.lz_b = first ? 1.f : float(beta);
    run_phase<P, RECON, EPI_CLOVER_INV, LAZY>(a1, part, xch, stage, 0.0);
    if (!grid_barrier(Q.bar_count, bar_target, Q.bar_err)) return;
    // phase 2
    {
      DslashArgs a = a2;
      a.x = Q.p;
      a.x_norm = Q.p_n;
      a.out = Q.y;
      a.out_norm = Q.y_n;
      a.do_norm = 1;
      a.lz_r = a1.lz_r;
      a.lz_a = a1.lz_a;
      a.lz_b = a1.lz_b;
      const double v = block_sum<BLOCK>(run_phase<P, RECON, EPI_XPAY, LAZY>(a, part, xch, stage, 0.0));
      if (!grid_barrier_sum<BLOCK>(Q.bar_count, Q.bar_flag, bar_target, Q.bar_err, Q.part_pap, Q.totals, v, &pAp))
        return;
    }
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        Q.ctl->nan = 1;
        Q.ctl->halt = 1;
        if (Q.round_out) *Q.round_out = 2 * (iters - st0.iters);
      }
      return;
    }
    alpha = rr / pAp;
    // phase 3
    a1.in = Q.y;
    a1.in_norm = Q.y_n;
    a1.in_g5 = 1;
    run_phase<P, RECON, EPI_CLOVER_INV>(a1, part, xch, stage, 0.0);
    if (!grid_barrier(Q.bar_count, bar_target, Q.bar_err)) return;
    // phase 4
    double rr_new;
    {
      DslashArgs a = a2;
      a.x = Q.y;
      a.x_norm = Q.y_n;
      a.x_g5 = 1;
      a.out_g5 = 1;
      a.cg_x = Q.x;
      a.cg_r = Q.r;
      a.cg_p = Q.p;
      a.cg_p_norm = Q.p_n;
      const double v = block_sum<BLOCK>(run_phase<P, RECON, EPI_XPAY_CG>(a, part, xch, stage, alpha));
      if (!grid_barrier_sum<BLOCK>(Q.bar_count, Q.bar_flag, bar_target, Q.bar_err, Q.part_rr, Q.totals + 1, v,
                                   &rr_new))
        return;
    }
    if (!isfinite(rr_new)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        Q.ctl->nan = 1;
        Q.ctl->halt = 1;
        if (Q.round_out) *Q.round_out = 2 * (iters - st0.iters);
      }
      return;
    }
    beta = rr_new / rr;
    rr_prev = rr;
    rr = rr_new;
    iters += 1;
    since += 1;
    const bool want = rr_new <= st0.tol2 || since >= every || rr_new < delta2 * st0.rr_reliable;
    first = false;
    // phase 5 (with LAZY only when the launch ends without a reliable update, so that the next launch
    // finds p updated; at a reliable update the update's own p = r + beta p follows)
    if (!want && (!LAZY || iters >= Q.iter_limit)) {
      // phase 5
      for (int h = blockIdx.x * BLOCK + threadIdx.x; h < Vh; h += gridDim.x * BLOCK) {
        cx<RR> rs[12];
        cx<R> ps[12], out[12];
        SpinorIO<PR>::template load<LDM>(Q.r, nullptr, Vh, 0, h, rs);
        SpinorIO<P>::template load<LDM>(Q.p, Q.p_n, Vh, 0, h, ps);
        const RR b = RR(beta);
#pragma unroll
        for (int c = 0; c < 12; c++) {
          out[c].re = R(fma(b, RR(ps[c].re), rs[c].re));
          out[c].im = R(fma(b, RR(ps[c].im), rs[c].im));
        }
        SpinorIO<P>::store(Q.p, Q.p_n, Vh, 0, h, out);
      }
      if (!grid_barrier(Q.bar_count, bar_target, Q.bar_err)) return;
    }
    if (want || iters >= Q.iter_limit) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        CGState& s = *Q.cg;
        s.rr = rr;
        s.rr_prev = rr_prev;
        s.pAp = pAp;
        s.alpha = alpha;
        s.beta = beta;
        s.iters = iters;
        s.since_reliable = since;
        if (want) {
          s.pending = 1;
          Q.ctl->halt = 1;
          Q.ctl->rel_go = 1;
        }
        if (Q.round_out) *Q.round_out = 2 * (iters - st0.iters) + (want ? 1 : 0);
      }
      return;
    }
  }
}

// Two blocks meet at one grid barrier, except that block `absent` returns first: the other
// block's wait must run out, set *err and return.
__global__ void barrier_probe_kernel(unsigned* count, int* err, int absent) {
  if ((int)blockIdx.x == absent) return;
  unsigned target = 0;
  grid_barrier(count, target, err);
}

// Resident blocks per SM of one kernel instance and the SM count, per device (looked up on a
// device's first launch, under a lock, so that host threads and devices with different SM counts
// each get their own figures).
struct GridShape {
  int per_sm = -1, sms = 0;
};
constexpr int kMaxDevices = 64;

template <int P, int RECON>
cudaError_t launch_pc(const PersistentCGArgs& q, cudaStream_t st) {
  static std::mutex mu;
  static GridShape shape[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int per_sm, sms;
  {
    std::lock_guard<std::mutex> lock(mu);
    GridShape& s = shape[dev];
    if (s.per_sm < 0) {
      int n = 0, k = 0;
      if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if (PcShape<P>::DYN > 0 &&
          (e = cudaFuncSetAttribute(cg_persistent_kernel<P, RECON>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)PcShape<P>::DYN)) != cudaSuccess)
        return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, cg_persistent_kernel<P, RECON>, PcShape<P>::THREADS,
                                                             PcShape<P>::DYN)) != cudaSuccess)
        return e;
      s.sms = n;
      s.per_sm = k < 1 ? 0 : k;
    }
    per_sm = s.per_sm;
    sms = s.sms;
  }
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int nsb = (q.g.Vh + 31) / 32;
  int grid = per_sm * sms;
  const int units_per_block = PcShape<P>::PAIR ? PcShape<P>::PAIRS : 1;
  if (grid > (nsb + units_per_block - 1) / units_per_block) grid = (nsb + units_per_block - 1) / units_per_block;
  if (grid > q.slots) grid = q.slots;
  PersistentCGArgs a = q;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(cg_persistent_kernel<P, RECON>), dim3(grid),
                                     dim3(PcShape<P>::THREADS), args, PcShape<P>::DYN, st);
}

}  // namespace

cudaError_t launch_barrier_probe(unsigned* count, int* err, cudaStream_t st) {
  g_kernel_launches += 1;
  int absent = 1;
  void* args[] = {&count, &err, &absent};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(barrier_probe_kernel), dim3(2), dim3(32), args, 0, st);
}

cudaError_t launch_cg_persistent(int prec, int recon, const PersistentCGArgs& q, cudaStream_t st) {
  g_kernel_launches += 1;
  if (prec == 64) return launch_pc<64, 18>(q, st);
  if (prec == 32) return recon == 12 ? launch_pc<32, 12>(q, st) : launch_pc<32, 18>(q, st);
  return recon == 12 ? launch_pc<16, 12>(q, st) : launch_pc<16, 18>(q, st);
}

}  // namespace qcd
