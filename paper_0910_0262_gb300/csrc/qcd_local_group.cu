// In-process slab group: the halo exchanges and sums of the time decomposition for several slabs of
// one lattice held by one process (for example all on one GPU), each slab driven by a host thread of
// its own.  The callbacks run in the library: a slab records a CUDA event on its stream when its
// faces (or its partial sums) are ready, the slabs meet at a host barrier only to publish those events,
// and every copy or sum waits for them on the reading slab's stream; the writer's stream then waits
// for its readers' events before it reuses its buffers.  No host thread waits for the GPU, and the
// sums are added in slab order, so every slab gets the same bits.  (The paper's two MPI processes on
// one Cell blade exchanged through shared memory, Sec. 4; this is the single-process analogue.)
#include <atomic>
#include <chrono>
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
  void* buf[4] = {nullptr, nullptr, nullptr, nullptr};  // send_lo, send_hi, recv_lo, recv_hi
  size_t cap = 0;
  double* stage = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
};

}  // namespace

struct qcd_local_group {
  int n = 0;
  std::vector<Member> members;
  std::atomic<int> arrived{0};
  std::atomic<unsigned> generation{0};
  std::atomic<bool> broken{false};
};

namespace {

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

int local_exchange(void* user, size_t bytes) {
  Member* m = static_cast<Member*>(user);
  qcd_local_group* g = m->grp;
  if (bytes > m->cap) return 1;
  if (cudaEventRecord(m->ready, m->st) != cudaSuccess) return 1;
  if (!group_barrier(g)) return 1;
  const Member& up = g->members[(m->rank + 1) % g->n];
  const Member& lo = g->members[(m->rank + g->n - 1) % g->n];
  cudaStreamWaitEvent(m->st, up.ready, 0);
  cudaStreamWaitEvent(m->st, lo.ready, 0);
  cudaMemcpyAsync(m->buf[3], up.buf[0], bytes, cudaMemcpyDeviceToDevice, m->st);  // recv_hi <- upper send_lo
  cudaMemcpyAsync(m->buf[2], lo.buf[1], bytes, cudaMemcpyDeviceToDevice, m->st);  // recv_lo <- lower send_hi
  cudaEventRecord(m->done, m->st);
  if (!group_barrier(g)) return 1;
  // the next packing into this slab's send buffers follows its readers' copies
  cudaStreamWaitEvent(m->st, up.done, 0);
  cudaStreamWaitEvent(m->st, lo.done, 0);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int local_allreduce(void* user, double* values, int n) {
  Member* m = static_cast<Member*>(user);
  qcd_local_group* g = m->grp;
  if (n < 0 || n > kStageDoubles) return 1;
  if (n == 0) return 0;
  cudaMemcpyAsync(m->stage, values, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->st);
  if (cudaEventRecord(m->ready, m->st) != cudaSuccess) return 1;
  if (!group_barrier(g)) return 1;
  SumArgs a;
  a.count = g->n;
  a.n = n;
  a.out = values;
  for (int k = 0; k < g->n; k++) {
    cudaStreamWaitEvent(m->st, g->members[k].ready, 0);
    a.src[k] = g->members[k].stage;
  }
  qcd::g_kernel_launches += 1;
  local_sum_kernel<<<(n + 63) / 64, 64, 0, m->st>>>(a);
  cudaEventRecord(m->done, m->st);
  if (!group_barrier(g)) return 1;
  for (int k = 0; k < g->n; k++) cudaStreamWaitEvent(m->st, g->members[k].done, 0);  // every slab read `stage`
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
  if (m.done) cudaEventDestroy(m.done);
  m.ready = m.done = nullptr;
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
  Member& m = grp->members[rank];
  if (m.device >= 0) return qcd::set_error(QCD_ERR_STATE, "rank already joined");
  size_t cap = 0;
  qcd_status s = qcd_slab_halo_bytes(ctx, 64, 8, &cap);  // the largest: FP64 passes over 8 RHS
  if (s) return s;
  m.device = v.device;
  m.st = v.st;
  m.cap = cap;
  bool ok = true;
  for (void*& b : m.buf) ok = ok && cudaMalloc(&b, cap) == cudaSuccess;
  ok = ok && cudaMalloc(&m.stage, sizeof(double) * kStageDoubles) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&m.ready, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&m.done, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release_member(m);
    return qcd::set_error(QCD_ERR_NOMEM, "local group buffers");
  }
  comm->send_lo = m.buf[0];
  comm->send_hi = m.buf[1];
  comm->recv_lo = m.buf[2];
  comm->recv_hi = m.buf[3];
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
