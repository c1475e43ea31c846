// In-process slab group: the halo exchanges and sums of the time decomposition for several slabs of
// one lattice held by one process on one GPU, each slab driven by a host thread of its own.  The
// callbacks run in the library: a slab records a CUDA event on its stream when its faces (or its
// partial sums) are ready, and the slabs meet once per exchange or sum at a host barrier, only to
// publish those events.  A slab's halo kernel then reads its neighbours' send buffers in place (no
// copy), after waiting for their events on its own stream; the send buffers alternate between two
// sets from one pass to the next, so a slab packs the next pass's faces while its neighbours may
// still read the last ones, and the wait at the next meeting orders its packing after their reads
// of the set before.  Sums stage each slab's values in one of two alternating buffers and add them
// in slab order, so every slab gets the same bits.  No host thread waits for the GPU.  (The paper's
// two MPI processes on one Cell blade exchanged through shared memory, Sec. 4; this is the
// single-process analogue.)
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "qcd.h"
#include "qcd_api_scope.h"
#include "qcd_kernels.h"

namespace {

constexpr int kMaxMembers = 16;
constexpr int kStageDoubles = 64;                             // sums of up to 64 doubles per call
constexpr auto kBarrierTimeout = std::chrono::seconds(120);  // a slab that never arrives fails the call

struct SumArgs {
  const double* src[kMaxMembers];
  int count;
  int n;
  double* out;
};

// out[i] = src[0][i] + src[1][i] + ... in that order
__global__ void local_sum_kernel(SumArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double s = a.src[0][i];
  for (int k = 1; k < a.count; k++) s += a.src[k][i];
  a.out[i] = s;
}

}  // namespace

struct qcd_local_group;

namespace {

struct Member {
  qcd_local_group* grp = nullptr;
  int rank = -1;
  int device = -1;
  cudaStream_t st = nullptr;
  void* buf[4] = {nullptr, nullptr, nullptr, nullptr};  // send sets: (lo, hi) = buf[2 s], buf[2 s + 1]
  size_t cap = 0;
  double* stage = nullptr;                              // two sets of kStageDoubles
  cudaEvent_t ready = nullptr;
  qcd_slab_comm* comm = nullptr;                        // the struct the slab's calls take
  unsigned passes = 0, sums = 0;                        // calls so far: the current set of each
};

}  // namespace

struct qcd_local_group {
  int n = 0;
  std::vector<Member> members;
  std::mutex join_mu;
  std::atomic<int> arrived{0};
  std::atomic<unsigned> generation{0};
  std::atomic<bool> broken{false};
};

namespace {

// A rank whose call fails before the barrier breaks the group, so that the others fail at once
// instead of waiting for it until the timeout.
int fail_group(qcd_local_group* g) {
  g->broken.store(true, std::memory_order_release);
  return 1;
}

// All n slabs meet; false (for every later caller too) if one has not arrived within the timeout or
// the group was aborted.  Each slab has a host thread of its own, so the waiting threads spin on the
// generation word (yielding now and then) rather than sleep: a wake-up through the scheduler costs
// tens of microseconds, several times per CG iteration.  The last arrival resets the count before it
// advances the generation, so no thread enters the next barrier before the count is reset.
bool group_barrier(qcd_local_group* g) {
  if (g->broken.load(std::memory_order_acquire)) return false;
  const unsigned gen = g->generation.load(std::memory_order_acquire);
  if (g->arrived.fetch_add(1, std::memory_order_acq_rel) + 1 == g->n) {
    g->arrived.store(0, std::memory_order_relaxed);
    g->generation.fetch_add(1, std::memory_order_release);
    return true;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned k = 1; g->generation.load(std::memory_order_acquire) == gen; k++) {
    if (g->broken.load(std::memory_order_acquire)) return false;
    if ((k & 1023) == 0) {
      if (std::chrono::steady_clock::now() - t0 > kBarrierTimeout) {
        g->broken.store(true, std::memory_order_release);
        return false;
      }
      std::this_thread::yield();
    }
  }
  return !g->broken.load(std::memory_order_acquire);
}

// After every slab's faces of this pass are packed (its event), the pass's receive buffers are the
// neighbours' send buffers of the current set; the next pass packs into the other set.
int local_exchange(void* user, size_t bytes) {
  Member* m = static_cast<Member*>(user);
  qcd_local_group* g = m->grp;
  if (bytes > m->cap) return fail_group(g);
  const int s = m->passes & 1;
  if (cudaEventRecord(m->ready, m->st) != cudaSuccess) return fail_group(g);
  if (!group_barrier(g)) return 1;
  const Member& up = g->members[(m->rank + 1) % g->n];
  const Member& lo = g->members[(m->rank + g->n - 1) % g->n];
  // (with two slabs both neighbours are the other slab; a slab alone is its own neighbour and its
  // stream is already in order)
  if (&up != m) cudaStreamWaitEvent(m->st, up.ready, 0);
  if (&lo != m && &lo != &up) cudaStreamWaitEvent(m->st, lo.ready, 0);
  m->comm->recv_hi = up.buf[2 * s];      // the slab above's lower face
  m->comm->recv_lo = lo.buf[2 * s + 1];  // the slab below's upper face
  m->passes++;
  m->comm->send_lo = m->buf[2 * (1 - s)];
  m->comm->send_hi = m->buf[2 * (1 - s) + 1];
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// values <- the sum over the slabs in slab order, from the staged copies of the current set
int local_allreduce(void* user, double* values, int n) {
  Member* m = static_cast<Member*>(user);
  qcd_local_group* g = m->grp;
  if (n < 0 || n > kStageDoubles) return fail_group(g);
  if (n == 0) return 0;
  const int s = m->sums & 1;
  m->sums++;
  cudaMemcpyAsync(m->stage + s * kStageDoubles, values, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->st);
  if (cudaEventRecord(m->ready, m->st) != cudaSuccess) return fail_group(g);
  if (!group_barrier(g)) return 1;
  SumArgs a;
  a.count = g->n;
  a.n = n;
  a.out = values;
  for (int k = 0; k < g->n; k++) {
    if (k != m->rank) cudaStreamWaitEvent(m->st, g->members[k].ready, 0);
    a.src[k] = g->members[k].stage + s * kStageDoubles;
  }
  qcd::g_kernel_launches += 1;
  local_sum_kernel<<<(n + 63) / 64, 64, 0, m->st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

void release_member(Member& m) {
  if (m.device < 0) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(m.device);
  for (void*& b : m.buf) {
    cudaFree(b);
    b = nullptr;
  }
  cudaFree(m.stage);
  m.stage = nullptr;
  if (m.ready) cudaEventDestroy(m.ready);
  m.ready = nullptr;
  m.comm = nullptr;
  m.device = -1;
  if (prev >= 0) cudaSetDevice(prev);
  cudaGetLastError();
}

}  // namespace

extern "C" {

qcd_status qcd_local_group_create(qcd_local_group** grp, int n) {
  if (!grp) return qcd::set_error(QCD_ERR_ARG, "null pointer");
  *grp = nullptr;
  if (n < 1 || n > kMaxMembers) return qcd::set_error(QCD_ERR_ARG, "a local group holds 1 to 16 slabs");
  qcd_local_group* g = new qcd_local_group();
  g->n = n;
  g->members.resize(n);
  for (int r = 0; r < n; r++) {
    g->members[r].grp = g;
    g->members[r].rank = r;
  }
  *grp = g;
  return QCD_OK;
}

qcd_status qcd_local_group_join(qcd_local_group* grp, int rank, qcd_ctx* ctx, qcd_slab_comm* comm) {
  qcd::CtxView v;
  const bool have = qcd::ctx_view(ctx, &v);
  qcd::ApiScope scope("qcd_local_group_join", have ? v.device : -1);
  if (scope.status()) return scope.status();
  if (!grp || !comm) return qcd::set_error(QCD_ERR_ARG, "null pointer");
  if (rank < 0 || rank >= grp->n) return qcd::set_error(QCD_ERR_ARG, "rank outside the group");
  if (!v.slab) return qcd::set_error(QCD_ERR_STATE, "local group members are slab contexts");
  std::lock_guard<std::mutex> lock(grp->join_mu);
  Member& m = grp->members[rank];
  if (m.device >= 0) return qcd::set_error(QCD_ERR_STATE, "rank already joined");
  for (const Member& o : grp->members)
    if (o.device >= 0 && o.device != v.device)
      return qcd::set_error(QCD_ERR_ARG, "the slabs of a local group share one device");
  size_t cap = 0;
  qcd_status s = qcd_slab_halo_bytes(ctx, 64, 8, &cap);  // the largest: FP64 passes over 8 RHS
  if (s) return s;
  m.device = v.device;
  m.st = v.st;
  m.cap = cap;
  bool ok = true;
  for (void*& b : m.buf) ok = ok && cudaMalloc(&b, cap) == cudaSuccess;
  ok = ok && cudaMalloc(&m.stage, sizeof(double) * 2 * kStageDoubles) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&m.ready, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release_member(m);
    return qcd::set_error(QCD_ERR_NOMEM, "local group buffers");
  }
  // the first pass packs into set 0; the receive pointers are set by every exchange (until the first,
  // they name this rank's set 1, which nothing reads)
  comm->send_lo = m.buf[0];
  comm->send_hi = m.buf[1];
  comm->recv_lo = m.buf[2];
  comm->recv_hi = m.buf[3];
  m.comm = comm;
  m.passes = m.sums = 0;
  comm->exchange = local_exchange;
  comm->allreduce = local_allreduce;
  comm->user = &m;
  return QCD_OK;
}

qcd_status qcd_local_group_abort(qcd_local_group* grp) {
  if (!grp) return qcd::set_error(QCD_ERR_ARG, "null pointer");
  grp->broken.store(true, std::memory_order_release);
  return QCD_OK;
}

qcd_status qcd_local_group_destroy(qcd_local_group* grp) {
  if (!grp) return QCD_OK;
  for (Member& m : grp->members) release_member(m);
  delete grp;
  return QCD_OK;
}

}  // extern "C"
