// C ABI of libqcd (declared in include/qcd.h): context, workspace, operator
// application and the CG driver.
//
// The paper's runtime wraps every compute loop in a PPE-side function that
// fills a task structure, signals the SPEs and waits for completion (Sec. 3).
// Here a call enqueues kernels on one CUDA stream; the CG iteration keeps its
// scalars in device memory (alpha, beta, |r|^2 are produced by the reducing
// kernels themselves), so the host only looks at the solver state once per
// chunk of iterations and when a reliable update is due.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "qcd.h"
#include "qcd_dslash.cuh"
#include "qcd_kernels.h"
#include "qcd_force.h"
#include "qcd_api_scope.h"

using namespace qcd;

namespace {

thread_local std::string g_err;

qcd_status fail(qcd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

// opens the call's ApiScope (NVTX range, the context's device current until the call returns)
#define QCD_API_ENTER(name, ctx)                                      \
  ApiScope api_scope_(name, (ctx) ? (ctx)->device : -1);              \
  if (api_scope_.status() != QCD_OK) return api_scope_.status()

#define CUDA_TRY(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(QCD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

enum Slot {
  S_IN, S_OUT, S_T, S_Y, S_IN_N, S_OUT_N, S_T_N, S_Y_N,   // qcd_dslash
  S_CANON,                                               // canonical staging
  S_B_HI, S_X_HI, S_AP_HI, S_T_HI, S_Y_HI,               // FP64 solver fields
  S_X_LO, S_R_LO, S_P, S_AP, S_TL, S_YL,                 // inner solver fields
  S_X_LO_N, S_R_LO_N, S_P_N, S_AP_N, S_TL_N, S_YL_N,
  S_F_X, S_F_Y, S_F_CL, S_F_E,                           // force work fields
  S_MD_F, S_MD_PHI,                                      // R-algorithm step
  S_PBP,                                                 // psi-bar psi estimate
  S_COUNT
};

struct Buf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct ProfClass {
  std::string name;
  int launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};
struct ProfPending {
  cudaEvent_t a, b;
  int cls;
  double bytes, flops;
};


struct SolverFields {
  int pr, pp;  // precision of x_lo/r_lo and of p/Ap/temporaries
  double2 *b_hi, *x_hi, *ap_hi, *t_hi, *y_hi;
  void *x_lo, *r_lo, *p, *ap, *t, *y;
  float *x_lo_n, *r_lo_n, *p_n, *ap_n, *t_n, *y_n;
};

// one profiled launch inside a captured graph: an event pair recorded by the graph itself
struct ProfSlot {
  int cls;
  cudaEvent_t a, b;
  double bytes, flops;
  int iter;  // CG iteration inside the graph (-1: always runs)
};

// an instantiated CUDA graph of CG work for one set of solver fields
struct ItGraph {
  int kind = 0;  // 0: `len` CG iterations; 1: one reliable update
  int len = 0, nrhs = 0;
  bool prof = false;
  SolverFields f;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  std::vector<cudaEvent_t> events;
  std::vector<ProfSlot> slots;
};

struct CaptureSink {
  ItGraph* g;
  int iter;
  size_t next;
};

}  // namespace

struct qcd_ctx {
  Geom g{};
  cudaStream_t st = nullptr;
  int device = 0;
  // links
  void* g64 = nullptr;
  void* g32 = nullptr;
  void* g16 = nullptr;
  int recon = 18;
  bool have_gauge = false;
  // clover
  void* A64 = nullptr;
  void* Ainv64 = nullptr;
  void* A32 = nullptr;
  void* Ainv32 = nullptr;
  void* A16 = nullptr;
  void* Ainv16 = nullptr;
  double* logdet = nullptr;  // [parity][block][Vh] log det of each clover block
  bool have_clover = false;
  bool have_kappa = false;  // kappa and c_sw of a clover_build are known (the term may be stale)
  double kappa = 0, csw = 0;
  // device status words: [0] clover not positive definite, [1] non-finite input
  int* flags = nullptr;
  int* h_flags = nullptr;
  // reductions and CG state
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* results = nullptr;
  CGState* cg = nullptr;
  CGControl* ctl = nullptr;
  CGState* h_cg = nullptr;
  CGControl* h_ctl = nullptr;
  double* h_results = nullptr;
  long long max_partials = 0;
  Buf ws[S_COUNT];
  // profiling
  bool prof_on = false;
  std::vector<ProfClass> prof;
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> ev_free;
  // launch stream of the moment (the caller's stream, or the capture stream while a graph is recorded)
  cudaStream_t cur = nullptr;
  cudaStream_t cap = nullptr;
  CaptureSink* sink = nullptr;
  std::vector<ItGraph*> graphs;
  struct Launched {
    ItGraph* g;
    int offset;  // CG iteration offset of the graph's first iteration
    int round;   // reliable-update graph of a pipelined round (-1: always counted)
  };
  std::vector<Launched> launched;  // graphs launched since the last collection
  double last_rho = 0.0;                            // per-iteration |r|^2 ratio seen by the last solve
  // persistent single-RHS iteration: per-block partial sums and the grid barrier words
  double* pc_part = nullptr;   // 2 x pc_slots
  int pc_slots = 0;
  unsigned* pc_bar = nullptr;  // [0] barrier arrivals, [1] release word of the summing barriers, [2] error
  bool persistent = true;
  // per round of a batch of persistent launches: 2 x iterations run + 1 if it raised a reliable update
  int* pc_rounds = nullptr;
  int* h_pc_rounds = nullptr;
  struct PcPending {
    cudaEvent_t a, b;
    double bytes_per_iter, flops_per_iter;
  };
  std::vector<PcPending> pc_pending;
  // t-slab of a larger lattice (qcd_create_slab): the extended links (two slices on each side) and the
  // FP64 packed links and clover term of that extended lattice, from which the slab's part is copied
  bool slab = false;
  Geom ge{};
  double2* U_ext = nullptr;
  void* ext_g64 = nullptr;
  void *ext_A64 = nullptr, *ext_Ainv64 = nullptr, *ext_A32 = nullptr, *ext_Ainv32 = nullptr, *ext_A16 = nullptr,
       *ext_Ainv16 = nullptr;
  double* ext_logdet = nullptr;
};

namespace {

const int MAX_RHS = 8;
// rounds (persistent segment + gated reliable update) enqueued per look at the solver state
const int PC_MAX_ROUNDS = 32;

size_t spinor_bytes(const Geom& g, int prec, int nrhs) {
  const size_t per = prec == 64 ? 192 : (prec == 32 ? 96 : 48);
  return per * (size_t)g.Vh * nrhs;
}

qcd_status ws_get(qcd_ctx* c, int slot, size_t bytes, void** out) {
  Buf& b = c->ws[slot];
  if (b.bytes < bytes) {
    if (b.ptr) {
      cudaStreamSynchronize(c->st);
      cudaFree(b.ptr);
      b.ptr = nullptr;
      b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.ptr, bytes);
    if (e != cudaSuccess) {
      b.ptr = nullptr;
      cudaGetLastError();
      return fail(QCD_ERR_NOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
  }
  *out = b.ptr;
  return QCD_OK;
}

// --------------------------------------------------------------- profiling --
int prof_class(qcd_ctx* c, const std::string& name) {
  for (size_t i = 0; i < c->prof.size(); i++)
    if (c->prof[i].name == name) return (int)i;
  ProfClass pc;
  pc.name = name;
  c->prof.push_back(pc);
  return (int)c->prof.size() - 1;
}

cudaEvent_t prof_event(qcd_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  qcd_ctx* c;
  cudaEvent_t a = nullptr;
  int cls = -1;
  double bytes, flops;
  ProfScope(qcd_ctx* c_, const char* name, double bytes_, double flops_) : c(c_), bytes(bytes_), flops(flops_) {
    if (c->sink) {
      // recording a graph: the event pair becomes two event-record nodes of the graph.  Only the
      // first CG iteration of each graph is bracketed (a sample), since every event-record node
      // also serialises the graph at that point.
      if (!c->sink->g->prof || c->sink->iter > 0) return;
      cls = prof_class(c, name);
      a = c->sink->g->events[c->sink->next++];
      cudaEventRecordWithFlags(a, c->cur, cudaEventRecordExternal);
      return;
    }
    if (!c->prof_on) return;
    cls = prof_class(c, name);
    a = prof_event(c);
    cudaEventRecord(a, c->cur);
  }
  ~ProfScope() {
    if (cls < 0) return;
    if (c->sink) {
      cudaEvent_t b = c->sink->g->events[c->sink->next++];
      cudaEventRecordWithFlags(b, c->cur, cudaEventRecordExternal);
      c->sink->g->slots.push_back(ProfSlot{cls, a, b, bytes, flops, c->sink->iter});
      return;
    }
    cudaEvent_t b = prof_event(c);
    cudaEventRecord(b, c->cur);
    c->pending.push_back(ProfPending{a, b, cls, bytes, flops});
  }
};

// collect finished event pairs (the caller has synchronised the stream)
void prof_collect(qcd_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    ProfClass& pc = c->prof[p.cls];
    pc.launches += 1;
    pc.ms += ms;
    pc.bytes += p.bytes;
    pc.flops += p.flops;
    c->ev_free.push_back(p.a);
    c->ev_free.push_back(p.b);
  }
  c->pending.clear();
}

// ------------------------------------------------------ operator helpers --
int real_bytes(int prec) { return prec == 64 ? 8 : (prec == 32 ? 4 : 2); }

void dslash_cost(const qcd_ctx* c, int prec, int epi, int nrhs, double* bytes, double* flops) {
  const double Vh = c->g.Vh;
  const int R = prec == 64 ? 18 : c->recon;
  const double bl = real_bytes(prec);
  const double bc = prec == 64 ? 8 : (prec == 32 ? 4 : 2);
  const double bs = 24.0 * real_bytes(prec) + (prec == 16 ? 4 : 0);
  double site = 8.0 * R * bl + (epi != EPI_NONE ? 72.0 * bc : 0.0);
  double rhs = bs * (epi == EPI_XPAY ? 3.0 : 2.0);
  if (epi == EPI_XPAY_CG) {
    // reads in, x, p; reads and writes x_lo, r_lo; writes nothing else
    const double sr = 24.0 * (prec == 64 ? 8 : 4);
    rhs = 3.0 * bs + 4.0 * sr;
  }
  *bytes = Vh * site + Vh * nrhs * rhs;
  *flops = Vh * nrhs * (1320.0 + (epi != EPI_NONE ? 504.0 : 0.0) + (epi >= EPI_XPAY ? 48.0 : 0.0) +
                        (epi == EPI_XPAY_CG ? 96.0 : 0.0));
}

const void* gauge_ptr(const qcd_ctx* c, int prec) { return prec == 64 ? c->g64 : (prec == 32 ? c->g32 : c->g16); }

const void* clover_ptr(const qcd_ctx* c, int prec, bool inverse, int parity) {
  if (prec == 64) {
    const double2* base = static_cast<const double2*>(inverse ? c->Ainv64 : c->A64);
    return base + (size_t)parity * 36 * c->g.Vh;
  }
  if (prec == 16) {
    const uint4* base = static_cast<const uint4*>(inverse ? c->Ainv16 : c->A16);
    return base + (size_t)parity * 9 * c->g.Vh;
  }
  const float4* base = static_cast<const float4*>(inverse ? c->Ainv32 : c->A32);
  return base + (size_t)parity * 18 * c->g.Vh;
}

DslashArgs base_args(const qcd_ctx* c, int prec, int parity, int nrhs) {
  DslashArgs a;
  memset(&a, 0, sizeof a);
  a.g = c->g;
  a.p = parity;
  a.nrhs = nrhs;
  a.gauge = gauge_ptr(c, prec);
  return a;
}

void run_dslash(qcd_ctx* c, int prec, int epi, const DslashArgs& a) {
  double bytes, flops;
  dslash_cost(c, prec, epi, a.nrhs, &bytes, &flops);
  char name[40];
  snprintf(name, sizeof name, "dslash_p%d_r%d_%s", prec, prec == 64 ? 18 : c->recon,
           epi == EPI_NONE ? "plain" : (epi == EPI_CLOVER_INV ? "cloverinv" : (epi == EPI_XPAY ? "xpay" : "xpaycg")));
  ProfScope ps(c, name, bytes, flops);
  launch_dslash(prec, prec == 64 ? 18 : c->recon, epi, a, c->cur);
}

ReduceArgs reduce_args(qcd_ctx* c, int mode) {
  ReduceArgs r;
  r.partials = c->partials;
  r.capacity = c->max_partials;
  r.counter = c->counter;
  r.result = c->results;
  r.mode = mode;
  r.cg = c->cg;
  r.ctl = c->ctl;
  return r;
}

// out = Mhat in (dagger: Mhat^dag) on even sites, t: odd temporary.
// red (may be null) reduces |out|^2 per RHS.
void apply_mhat(qcd_ctx* c, int prec, int nrhs, bool dagger, const void* in, const float* in_n, void* out,
                float* out_n, void* t, float* t_n, const ReduceArgs* red, const int* halt,
                const int* gate = nullptr) {
  const double k2 = c->kappa * c->kappa;
  DslashArgs a = base_args(c, prec, 1, nrhs);
  a.in = in;
  a.in_norm = in_n;
  a.out = t;
  a.out_norm = t_n;
  a.clover = clover_ptr(c, prec, true, 1);
  a.in_g5 = dagger;
  a.halt = halt;
  a.gate = gate;
  run_dslash(c, prec, EPI_CLOVER_INV, a);
  DslashArgs b = base_args(c, prec, 0, nrhs);
  b.in = t;
  b.in_norm = t_n;
  b.out = out;
  b.out_norm = out_n;
  b.x = in;
  b.x_norm = in_n;
  b.clover = clover_ptr(c, prec, false, 0);
  b.a = -k2;
  b.x_g5 = dagger;
  b.out_g5 = dagger;
  b.halt = halt;
  b.gate = gate;
  if (red) {
    b.do_norm = 1;
    b.red = *red;
  }
  run_dslash(c, prec, EPI_XPAY, b);
}

// out = Mhat^dag Mhat in; y: even temporary, t: odd temporary; pap reduces |Mhat in|^2
void apply_mdagm(qcd_ctx* c, int prec, int nrhs, const void* in, const float* in_n, void* out, float* out_n, void* t,
                 float* t_n, void* y, float* y_n, const ReduceArgs* pap, const int* halt,
                 const int* gate = nullptr) {
  apply_mhat(c, prec, nrhs, false, in, in_n, y, y_n, t, t_n, pap, halt, gate);
  apply_mhat(c, prec, nrhs, true, y, y_n, out, out_n, t, t_n, nullptr, halt, gate);
}

qcd_status sync_and_check(qcd_ctx* c, const char* what) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  if (c->prof_on) prof_collect(c);
  return QCD_OK;
}

bool valid_prec(int p) { return p == 64 || p == 32 || p == 16; }

// largest supported batch (1, 2, 4 or 8) not above n
int batch_of(int n) {
  int b = 1;
  while (b * 2 <= n && b * 2 <= MAX_RHS) b *= 2;
  return b;
}

}  // namespace

// Read-only view of a context and the thread's error message, for entry points defined in other
// translation units of the library (qcd_kernels.h).
namespace qcd {

bool ctx_view(const qcd_ctx* c, CtxView* v) {
  if (!c) return false;
  v->g = c->g;
  v->st = c->st;
  v->device = c->device;
  v->g64 = c->g64;
  v->A_even64 = c->A64 ? clover_ptr(c, 64, false, 0) : nullptr;
  v->Ainv_odd64 = c->Ainv64 ? clover_ptr(c, 64, true, 1) : nullptr;
  v->kappa = c->kappa;
  v->have_gauge = c->have_gauge;
  v->have_clover = c->have_clover;
  v->slab = c->slab;
  return true;
}

qcd_status set_error(qcd_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace qcd

namespace {
qcd_status slab_clover_build(qcd_ctx* c, double kappa, double csw, void* work);
// calls that need an ordinary lattice (or a slab that is the whole lattice) refuse a t-slab
qcd_status slab_refuse(const qcd_ctx* c, const char* what, bool whole_ok) {
  if (!c || !c->slab) return QCD_OK;
  if (whole_ok && c->g.T == c->g.Tg) return QCD_OK;
  return fail(QCD_ERR_STATE, "%s is not available on a t-slab context%s", what,
              whole_ok ? " (use the qcd_slab_* calls)" : "");
}
}  // namespace

// ===================================================================== ABI ==
extern "C" {

const char* qcd_last_error(void) { return g_err.c_str(); }

static qcd_status create_ctx(qcd_ctx** out, const int dims[4], double t_bc, void* stream);

qcd_status qcd_create(qcd_ctx** out, const int dims[4], double t_bc, void* stream) {
  nvtxRangePushA("qcd_create");
  const qcd_status s = create_ctx(out, dims, t_bc, stream);
  nvtxRangePop();
  return s;
}

}  // extern "C"

// the body of qcd_create, on the caller's current device
static qcd_status create_ctx(qcd_ctx** out, const int dims[4], double t_bc, void* stream) {
  if (!out || !dims) return fail(QCD_ERR_ARG, "null argument");
  *out = nullptr;
  for (int k = 0; k < 4; k++)
    if (dims[k] < 2 || dims[k] % 2) return fail(QCD_ERR_ARG, "extent %d = %d must be even and >= 2", k, dims[k]);
  if (t_bc != 1.0 && t_bc != -1.0) return fail(QCD_ERR_ARG, "t_bc must be +1 or -1");
  const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  if (V * 8 >= (1LL << 31)) return fail(QCD_ERR_ARG, "lattice too large (V = %lld)", V);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  qcd_ctx* c = new qcd_ctx();
  c->device = dev;
  c->st = static_cast<cudaStream_t>(stream);
  c->cur = c->st;
  c->g.X = dims[0];
  c->g.Y = dims[1];
  c->g.Z = dims[2];
  c->g.T = dims[3];
  c->g.Vh = (int)(V / 2);
  c->g.XY = dims[0] * dims[1];
  c->g.XYZ = dims[0] * dims[1] * dims[2];
  c->g.t_bc = t_bc;
  c->g.dX = make_fastdiv(dims[0]);
  c->g.dY = make_fastdiv(dims[1]);
  c->g.dZ = make_fastdiv(dims[2]);
  c->g.t0 = 0;
  c->g.Tg = dims[3];
  // partial sums of one reduction: nrhs x (blocks of the launch); the hopping kernel covers 32
  // (site, RHS) pairs per block, the fewest of all reducing kernels, so nrhs <= MAX_RHS needs
  // at most MAX_RHS * ceil(Vh * MAX_RHS / 32) slots
  c->max_partials = (long long)MAX_RHS * ((c->g.Vh * (long long)MAX_RHS + 31) / 32) + 64;
  bool ok = cudaMalloc(&c->flags, 4 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->partials, sizeof(double) * (size_t)c->max_partials) == cudaSuccess &&
            cudaMalloc(&c->counter, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&c->results, sizeof(double) * MAX_RHS) == cudaSuccess &&
            cudaMalloc(&c->cg, sizeof(CGState) * MAX_RHS) == cudaSuccess &&
            cudaMalloc(&c->ctl, sizeof(CGControl)) == cudaSuccess &&
            cudaMallocHost(&c->h_flags, 4 * sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&c->h_cg, sizeof(CGState) * MAX_RHS) == cudaSuccess &&
            cudaMallocHost(&c->h_ctl, sizeof(CGControl)) == cudaSuccess &&
            cudaMallocHost(&c->h_results, sizeof(double) * MAX_RHS) == cudaSuccess &&
            cudaMalloc(&c->pc_rounds, sizeof(int) * PC_MAX_ROUNDS) == cudaSuccess &&
            cudaMallocHost(&c->h_pc_rounds, sizeof(int) * PC_MAX_ROUNDS) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    qcd_destroy(c);
    return fail(QCD_ERR_NOMEM, "context allocation failed");
  }
  cudaMemset(c->counter, 0, sizeof(unsigned));
  cudaMemset(c->flags, 0, 4 * sizeof(int));
  cudaMemset(c->ctl, 0, sizeof(CGControl));
  {
    int sms = 0, coop = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    c->pc_slots = sms * 16;  // 16 resident 128-thread blocks per SM at most
    c->persistent = coop != 0;
    const char* e = getenv("QCD_CG_PERSISTENT");
    if (e && e[0] == '0') c->persistent = false;
    // two sets of per-block partials, then the two grid totals
    if (cudaMalloc(&c->pc_part, sizeof(double) * (2 * c->pc_slots + 2)) != cudaSuccess ||
        cudaMalloc(&c->pc_bar, 4 * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      qcd_destroy(c);
      return fail(QCD_ERR_NOMEM, "context allocation failed");
    }
    cudaMemset(c->pc_bar, 0, 4 * sizeof(unsigned));
  }
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    qcd_destroy(c);
    return fail(QCD_ERR_CUDA, "capture stream creation failed");
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    qcd_destroy(c);
    return fail(QCD_ERR_CUDA, "context init: %s", cudaGetErrorString(e));
  }
  *out = c;
  return QCD_OK;
}

extern "C" {

qcd_status qcd_destroy(qcd_ctx* c) {
  if (!c) return QCD_OK;
  QCD_API_ENTER("qcd_destroy", c);
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  void* dev[] = {c->g64, c->g32, c->g16, c->A64, c->Ainv64, c->A32, c->Ainv32, c->A16, c->Ainv16, c->logdet, c->flags,
                 c->pc_part, c->pc_bar, c->pc_rounds,
                 c->partials, c->counter, c->results, c->cg, c->ctl,
                 c->U_ext, c->ext_g64, c->ext_A64, c->ext_Ainv64, c->ext_A32, c->ext_Ainv32, c->ext_A16, c->ext_Ainv16,
                 c->ext_logdet};
  for (void* p : dev)
    if (p) cudaFree(p);
  for (auto& b : c->ws)
    if (b.ptr) cudaFree(b.ptr);
  void* host[] = {c->h_flags, c->h_cg, c->h_ctl, c->h_results, c->h_pc_rounds};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  for (ItGraph* gph : c->graphs) {
    if (gph->exec) cudaGraphExecDestroy(gph->exec);
    for (auto e : gph->events) cudaEventDestroy(e);
    delete gph;
  }
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
  return QCD_OK;
}

qcd_status qcd_load_gauge(qcd_ctx* c, const double* U, int on_device, int flags) {
  QCD_API_ENTER("qcd_load_gauge", c);
  qcd_status s = QCD_OK;
  if (!U) return fail(QCD_ERR_ARG, "null gauge pointer");
  if (flags & ~QCD_GAUGE_RECON12) return fail(QCD_ERR_ARG, "unknown gauge flags 0x%x", flags);
  const Geom& g = c->g;
  const size_t n_links = (size_t)g.Vh * 2 * 4;
  const size_t canon_bytes = n_links * 9 * sizeof(double2);
  c->recon = (flags & QCD_GAUGE_RECON12) ? 12 : 18;
  if (!c->g64) {
    CUDA_TRY(cudaMalloc(&c->g64, canon_bytes));
    CUDA_TRY(cudaMalloc(&c->g32, n_links * 9 * sizeof(float2)));
    CUDA_TRY(cudaMalloc(&c->g16, n_links * 9 * sizeof(uint32_t)));
  }
  // a t-slab keeps the whole extended field (its clover build reads it); the slab's own links start
  // two time slices in
  const size_t in_links = c->slab ? (size_t)c->ge.Vh * 2 * 4 : n_links;
  const size_t in_bytes = in_links * 9 * sizeof(double2);
  const double2* src = reinterpret_cast<const double2*>(U);
  if (c->slab) {
    if (!c->U_ext) CUDA_TRY(cudaMalloc(&c->U_ext, in_bytes));
    CUDA_TRY(cudaMemcpyAsync(c->U_ext, U, in_bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->st));
    src = c->U_ext;
  } else if (!on_device) {
    void* stage;
    if ((s = ws_get(c, S_CANON, canon_bytes, &stage))) return s;
    CUDA_TRY(cudaMemcpyAsync(stage, U, canon_bytes, cudaMemcpyHostToDevice, c->st));
    src = static_cast<const double2*>(stage);
  }
  CUDA_TRY(cudaMemsetAsync(c->flags, 0, 4 * sizeof(int), c->st));
  launch_check_finite(reinterpret_cast<const double*>(src), in_links * 18, c->flags + 1, c->st);
  launch_pack_gauge(g, src + (c->slab ? (size_t)2 * g.XYZ * 4 * 9 : 0), c->g64, c->g32, c->recon, c->g16, c->recon,
                    c->st);
  CUDA_TRY(cudaMemcpyAsync(c->h_flags, c->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "load_gauge"))) return s;
  c->have_clover = false;
  if (c->h_flags[1]) {
    c->have_gauge = false;
    return fail(QCD_ERR_NAN, "gauge field holds a non-finite value");
  }
  c->have_gauge = true;
  return QCD_OK;
}

qcd_status qcd_clover_build(qcd_ctx* c, double kappa, double csw) {
  QCD_API_ENTER("qcd_clover_build", c);
  qcd_status s = QCD_OK;
  if (!c->have_gauge) return fail(QCD_ERR_STATE, "clover_build before load_gauge");
  if (!(kappa == kappa) || !(csw == csw)) return fail(QCD_ERR_ARG, "kappa/csw not finite");
  const Geom& g = c->g;
  if (!c->A64) {
    CUDA_TRY(cudaMalloc(&c->A64, (size_t)2 * 36 * g.Vh * sizeof(double2)));
    CUDA_TRY(cudaMalloc(&c->Ainv64, (size_t)2 * 36 * g.Vh * sizeof(double2)));
    CUDA_TRY(cudaMalloc(&c->A32, (size_t)2 * 18 * g.Vh * sizeof(float4)));
    CUDA_TRY(cudaMalloc(&c->Ainv32, (size_t)2 * 18 * g.Vh * sizeof(float4)));
    CUDA_TRY(cudaMalloc(&c->A16, (size_t)2 * 9 * g.Vh * sizeof(uint4)));
    CUDA_TRY(cudaMalloc(&c->Ainv16, (size_t)2 * 9 * g.Vh * sizeof(uint4)));
    CUDA_TRY(cudaMalloc(&c->logdet, (size_t)2 * 2 * g.Vh * sizeof(double)));
  }
  void* work;
  if ((s = ws_get(c, S_F_CL, force_clover_bytes(c->slab ? c->ge : g), &work))) return s;
  CUDA_TRY(cudaMemsetAsync(c->flags, 0, 4 * sizeof(int), c->st));
  if (c->slab) {
    if ((s = slab_clover_build(c, kappa, csw, work))) return s;
  } else {
    // 6 planes x 10 products of 3x3 complex matrices per site (two leaves share a product), plus
    // the two inversions
    ProfScope ps(c, "clover_build", 0, 2.0 * g.Vh * (60 * 216.0 + 2 * 1000.0));
    launch_clover_build(g, c->g64, kappa, csw, c->A64, c->Ainv64, c->A32, c->Ainv32, c->A16, c->Ainv16, work,
                        c->logdet, c->flags, c->st);
  }
  CUDA_TRY(cudaMemcpyAsync(c->h_flags, c->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "clover_build"))) return s;
  if (c->h_flags[0]) {
    c->have_clover = false;
    return fail(QCD_ERR_NOT_POSDEF, "a clover block is not positive definite (kappa=%g, csw=%g)", kappa, csw);
  }
  c->kappa = kappa;
  c->csw = csw;
  c->have_clover = true;
  c->have_kappa = true;
  return QCD_OK;
}

qcd_status qcd_dslash(qcd_ctx* c, double* out, const double* in, int op, int dagger, int prec, int nrhs) {
  QCD_API_ENTER("qcd_dslash", c);
  if (qcd_status rs = slab_refuse(c, "qcd_dslash", true)) return rs;
  qcd_status s = QCD_OK;
  if (!out || !in) return fail(QCD_ERR_ARG, "null field pointer");
  if (op < QCD_OP_DSLASH_EO || op > QCD_OP_CLOVER_INV) return fail(QCD_ERR_ARG, "unknown op %d", op);
  if (!valid_prec(prec)) return fail(QCD_ERR_ARG, "precision must be 64, 32 or 16");
  if (nrhs < 1) return fail(QCD_ERR_ARG, "nrhs must be >= 1");
  if (!c->have_gauge) return fail(QCD_ERR_STATE, "dslash before load_gauge");
  const bool needs_clover = op >= QCD_OP_MHAT;
  if (needs_clover && !c->have_clover) return fail(QCD_ERR_STATE, "op %d needs clover_build", op);
  const Geom& g = c->g;
  const size_t canon = (size_t)g.Vh * 12 * sizeof(double2);
  if ((const char*)out < (const char*)in + canon * nrhs && (const char*)in < (const char*)out + canon * nrhs)
    return fail(QCD_ERR_ARG, "in and out overlap");
  int done = 0;
  while (done < nrhs) {
    const int nb = batch_of(nrhs - done);
    const double2* cin = reinterpret_cast<const double2*>(in) + (size_t)done * g.Vh * 12;
    double2* cout = reinterpret_cast<double2*>(out) + (size_t)done * g.Vh * 12;
    void *vin, *vout, *vt, *vy, *nin = nullptr, *nout = nullptr, *nt = nullptr, *ny = nullptr;
    const size_t fb = spinor_bytes(g, prec, nb), nbytes = sizeof(float) * (size_t)g.Vh * nb;
    if ((s = ws_get(c, S_IN, fb, &vin)) || (s = ws_get(c, S_OUT, fb, &vout)) || (s = ws_get(c, S_T, fb, &vt)) ||
        (s = ws_get(c, S_Y, fb, &vy)))
      return s;
    if (prec == 16) {
      if ((s = ws_get(c, S_IN_N, nbytes, &nin)) || (s = ws_get(c, S_OUT_N, nbytes, &nout)) ||
          (s = ws_get(c, S_T_N, nbytes, &nt)) || (s = ws_get(c, S_Y_N, nbytes, &ny)))
        return s;
    }
    float *fin = (float*)nin, *fout = (float*)nout, *ft = (float*)nt, *fy = (float*)ny;
    launch_spinor_to_native(prec, g, cin, vin, fin, nb, c->st);
    switch (op) {
      case QCD_OP_DSLASH_EO:
      case QCD_OP_DSLASH_OE: {
        DslashArgs a = base_args(c, prec, op == QCD_OP_DSLASH_EO ? 0 : 1, nb);
        a.in = vin;
        a.in_norm = fin;
        a.out = vout;
        a.out_norm = fout;
        a.in_g5 = a.out_g5 = dagger ? 1 : 0;
        run_dslash(c, prec, EPI_NONE, a);
        break;
      }
      case QCD_OP_MHAT:
        apply_mhat(c, prec, nb, dagger != 0, vin, fin, vout, fout, vt, ft, nullptr, nullptr);
        break;
      case QCD_OP_MDAGM:
        apply_mdagm(c, prec, nb, vin, fin, vout, fout, vt, ft, vy, fy, nullptr, nullptr);
        break;
      case QCD_OP_CLOVER:
        launch_clover_apply(prec, g, clover_ptr(c, prec, false, 0), vin, fin, vout, fout, nb, c->st);
        break;
      case QCD_OP_CLOVER_INV:
        launch_clover_apply(prec, g, clover_ptr(c, prec, true, 1), vin, fin, vout, fout, nb, c->st);
        break;
    }
    launch_spinor_to_canon(prec, g, vout, fout, cout, nb, c->st);
    done += nb;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "dslash launch: %s", cudaGetErrorString(e));
  return QCD_OK;
}

}  // extern "C"

// ============================================================ CG driver ==
namespace {



qcd_status solver_fields(qcd_ctx* c, int inner, int nrhs, SolverFields* f) {
  const Geom& g = c->g;
  f->pp = inner;
  f->pr = inner == 64 ? 64 : 32;
  qcd_status s;
  void* v;
  const size_t hi = spinor_bytes(g, 64, nrhs), lo_r = spinor_bytes(g, f->pr, nrhs), lo_p = spinor_bytes(g, f->pp, nrhs);
#define GET(slot, bytes, dst, type)                       \
  if ((s = ws_get(c, slot, bytes, &v))) return s; \
  dst = static_cast<type>(v);
  GET(S_B_HI, hi, f->b_hi, double2*);
  GET(S_X_HI, hi, f->x_hi, double2*);
  GET(S_AP_HI, hi, f->ap_hi, double2*);
  GET(S_T_HI, hi, f->t_hi, double2*);
  GET(S_Y_HI, hi, f->y_hi, double2*);
  GET(S_X_LO, lo_r, f->x_lo, void*);
  GET(S_R_LO, lo_r, f->r_lo, void*);
  GET(S_P, lo_p, f->p, void*);
  GET(S_AP, lo_p, f->ap, void*);
  GET(S_TL, lo_p, f->t, void*);
  GET(S_YL, lo_p, f->y, void*);
  f->x_lo_n = f->r_lo_n = f->p_n = f->ap_n = f->t_n = f->y_n = nullptr;
  if (f->pp == 16) {
    const size_t nb = sizeof(float) * (size_t)g.Vh * nrhs;
    GET(S_P_N, nb, f->p_n, float*);
    GET(S_AP_N, nb, f->ap_n, float*);
    GET(S_TL_N, nb, f->t_n, float*);
    GET(S_YL_N, nb, f->y_n, float*);
  }
#undef GET
  return QCD_OK;
}

void update_cost(const Geom& g, int pr, int pp, int nrhs, double* bytes) {
  const double sr = 24.0 * real_bytes(pr), sp = 24.0 * real_bytes(pp) + (pp == 16 ? 4 : 0);
  *bytes = (double)g.Vh * nrhs * (4 * sr + 2 * sp);
}

// --- work of one CG iteration and of one reliable update, enqueued on c->cur ---------------------

// Mhat^dag Mhat p (|Mhat p|^2 -> alpha), x += alpha p, r -= alpha Ap (|r|^2 -> beta and the
// reliable-update / convergence triggers), p = r + beta p.  Every kernel returns at once while
// ctl->halt is set, so iterations enqueued past a trigger cost only their launch.
void enqueue_iteration(qcd_ctx* c, const SolverFields& f, int nrhs) {
  const Geom& g = c->g;
  const int* halt = &c->ctl->halt;
  ReduceArgs red_pap = reduce_args(c, FIN_CG_PAP);
  ReduceArgs red_rr = reduce_args(c, FIN_CG_RR);
  // y = Mhat p with |y|^2 = <p, Mhat^dag Mhat p> -> alpha
  apply_mhat(c, f.pp, nrhs, false, f.p, f.p_n, f.y, f.y_n, f.t, f.t_n, &red_pap, halt);
  // t = A_oo^-1 D_oe g5 y
  DslashArgs a = base_args(c, f.pp, 1, nrhs);
  a.in = f.y;
  a.in_norm = f.y_n;
  a.out = f.t;
  a.out_norm = f.t_n;
  a.clover = clover_ptr(c, f.pp, true, 1);
  a.in_g5 = 1;
  a.halt = halt;
  run_dslash(c, f.pp, EPI_CLOVER_INV, a);
  // Ap = g5 (A_ee g5 y - kappa^2 D_eo t), kept in registers: x += alpha p, r -= alpha Ap,
  // |r|^2 -> beta and the reliable-update / convergence triggers
  DslashArgs b = base_args(c, f.pp, 0, nrhs);
  b.in = f.t;
  b.in_norm = f.t_n;
  b.x = f.y;
  b.x_norm = f.y_n;
  b.clover = clover_ptr(c, f.pp, false, 0);
  b.a = -c->kappa * c->kappa;
  b.x_g5 = 1;
  b.out_g5 = 1;
  b.halt = halt;
  b.red = red_rr;
  b.cg_x = f.x_lo;
  b.cg_r = f.r_lo;
  b.cg_p = f.p;
  b.cg_p_norm = f.p_n;
  run_dslash(c, f.pp, EPI_XPAY_CG, b);
  {
    const double pb = (double)g.Vh * nrhs * (24.0 * real_bytes(f.pr) + 2 * (24.0 * real_bytes(f.pp) + (f.pp == 16 ? 4 : 0)));
    ProfScope ps(c, "p_update", pb, 0);
    launch_p_update(f.pr, f.pp, g, nrhs, f.r_lo, f.r_lo_n, f.p, f.p_n, c->cg, halt, c->cur);
  }
}

// x_hi += x_lo, r = b - Mhat^dag Mhat x_hi in FP64 (true residual, convergence test, halt cleared
// unless every RHS is done), p = r + beta p.  gated: every step returns at once unless a trigger
// raised ctl->rel_go, which the last step lowers (so the update can be enqueued before it is known
// to be due).
void enqueue_reliable(qcd_ctx* c, const SolverFields& f, int nrhs, bool gated) {
  const Geom& g = c->g;
  const int* gate = gated ? &c->ctl->rel_go : nullptr;
  launch_accumulate_x(f.pr, g, nrhs, f.x_hi, f.x_lo, f.x_lo_n, c->cur, gate);
  apply_mdagm(c, 64, nrhs, f.x_hi, nullptr, f.ap_hi, nullptr, f.t_hi, nullptr, f.y_hi, nullptr, nullptr, nullptr,
              gate);
  launch_true_residual(f.pr, g, nrhs, f.b_hi, f.ap_hi, f.r_lo, f.r_lo_n, reduce_args(c, FIN_CG_TRUE), c->cur, gate);
  launch_p_update(f.pr, f.pp, g, nrhs, f.r_lo, f.r_lo_n, f.p, f.p_n, c->cg, nullptr, c->cur, gate);
  if (gated) launch_gate_clear(&c->ctl->rel_go, c->cur);
}

// --- CUDA graphs of that work ----------------------------------------------------------------------

const int MAX_GRAPH_LEN = 64;

qcd_status capture_graph(qcd_ctx* c, ItGraph* gph) {
  if (gph->prof) {
    const size_t need = 14;
    while (gph->events.size() < need) {
      cudaEvent_t e;
      CUDA_TRY(cudaEventCreate(&e));
      gph->events.push_back(e);
    }
  }
  gph->slots.clear();
  CaptureSink sink{gph, -1, 0};
  const long long k0 = g_kernel_launches;
  c->cur = c->cap;
  c->sink = &sink;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (gph->kind == 0) {
      for (int j = 0; j < gph->len; j++) {
        sink.iter = j;
        enqueue_iteration(c, gph->f, gph->nrhs);
      }
    } else {
      enqueue_reliable(c, gph->f, gph->nrhs, true);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->cap, &graph);
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&gph->exec, graph, 0);
      cudaGraphDestroy(graph);
    }
  }
  c->sink = nullptr;
  c->cur = c->st;
  gph->kernels = g_kernel_launches - k0;
  g_kernel_launches = k0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    gph->exec = nullptr;
    return fail(QCD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  return QCD_OK;
}

// cached graph for (kind, len) on these fields, recorded on first use
qcd_status get_graph(qcd_ctx* c, int kind, int len, const SolverFields& f, int nrhs, ItGraph** out) {
  for (ItGraph* gph : c->graphs) {
    if (gph->kind == kind && gph->len == len && gph->nrhs == nrhs && gph->prof == c->prof_on &&
        memcmp(&gph->f, &f, sizeof f) == 0) {
      *out = gph;
      return QCD_OK;
    }
  }
  ItGraph* gph = new ItGraph();
  gph->kind = kind;
  gph->len = len;
  gph->nrhs = nrhs;
  gph->prof = c->prof_on;
  gph->f = f;
  qcd_status s = capture_graph(c, gph);
  if (s) {
    delete gph;
    return s;
  }
  c->graphs.push_back(gph);
  *out = gph;
  return QCD_OK;
}

qcd_status launch_graph(qcd_ctx* c, ItGraph* gph, int iter_offset, int round = -1) {
  CUDA_TRY(cudaGraphLaunch(gph->exec, c->st));
  g_kernel_launches += gph->kernels;
  if (gph->prof) c->launched.push_back({gph, iter_offset, round});
  return QCD_OK;
}

// after a synchronisation: fold the event pairs of the graphs launched since the last call into the
// kernel classes, counting only CG iterations that ran (the first `real_iters` of the segment) and
// only the reliable updates of pipelined rounds whose gate was raised (rounds[k] odd; null: all)
void collect_graphs(qcd_ctx* c, int real_iters, const int* rounds = nullptr) {
  for (auto& lg : c->launched) {
    if (lg.round >= 0 && rounds && !(rounds[lg.round] & 1)) continue;
    for (const ProfSlot& sl : lg.g->slots) {
      if (sl.iter >= 0 && lg.offset + sl.iter >= real_iters) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, sl.a, sl.b) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      ProfClass& pc = c->prof[sl.cls];
      pc.launches += 1;
      pc.ms += ms;
      pc.bytes += sl.bytes;
      pc.flops += sl.flops;
    }
  }
  c->launched.clear();
}

// n CG iterations as graphs of power-of-two lengths (each length at most once, so that a profiled
// graph's events are read before they are recorded again)
qcd_status launch_iterations(qcd_ctx* c, const SolverFields& f, int nrhs, int n) {
  int offset = 0;
  for (int len = MAX_GRAPH_LEN; len >= 1; len >>= 1) {
    if (n & len) {
      ItGraph* gph;
      qcd_status s = get_graph(c, 0, len, f, nrhs, &gph);
      if (s) return s;
      if ((s = launch_graph(c, gph, offset))) return s;
      offset += len;
    }
  }
  return QCD_OK;
}

qcd_status read_state(qcd_ctx* c, int nrhs) {
  cudaMemcpyAsync(c->h_cg, c->cg, sizeof(CGState) * nrhs, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(CGControl), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(c->h_flags + 2, c->pc_bar + 2, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  return sync_and_check(c, "cg state");
}

// Single-RHS iterations run in the persistent kernel at every lattice size: measured against the
// CUDA-graph iteration (site-kernel passes and separate p updates), mixed FP32 solve to 1e-8:
// 16^4 6.09 vs 6.13 ms, 24^4 24.1 vs 25.6, 32^4 70.4 vs 74.7, 32^3 x 64 139.8 vs 148.1,
// 48^3 x 96 732 vs 772 ms.
const int PERSISTENT_MAX_VH = 1 << 30;

// One segment of CG iterations of a single RHS in the persistent kernel: it stops itself at the
// next reliable-update or convergence trigger, or once the RHS has run iter_limit iterations in
// total; round: its slot in pc_rounds.
qcd_status launch_persistent(qcd_ctx* c, const SolverFields& f, int iter_limit, int round) {
  const Geom& g = c->g;
  PersistentCGArgs q;
  memset(&q, 0, sizeof q);
  q.g = g;
  q.gauge = gauge_ptr(c, f.pp);
  q.clover_inv_odd = clover_ptr(c, f.pp, true, 1);
  q.clover_even = clover_ptr(c, f.pp, false, 0);
  q.p = f.p;
  q.t = f.t;
  q.y = f.y;
  q.p_n = f.p_n;
  q.t_n = f.t_n;
  q.y_n = f.y_n;
  q.x = f.x_lo;
  q.r = f.r_lo;
  q.k2 = c->kappa * c->kappa;
  q.cg = c->cg;
  q.ctl = c->ctl;
  q.part_pap = c->pc_part;
  q.part_rr = c->pc_part + c->pc_slots;
  q.slots = c->pc_slots;
  q.bar_count = c->pc_bar;
  q.bar_flag = c->pc_bar + 1;
  q.totals = c->pc_part + 2 * c->pc_slots;
  q.bar_err = reinterpret_cast<int*>(c->pc_bar + 2);
  q.iter_limit = iter_limit;
  q.round_out = c->pc_rounds + round;
  // the arrival counter and the release word restart with every launch; the error word is cleared once per batch of
  // rounds (cg_batch), so that a timed-out round stops every later one at its first barrier
  CUDA_TRY(cudaMemsetAsync(c->pc_bar, 0, 2 * sizeof(unsigned), c->st));
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (c->prof_on) {
    ea = prof_event(c);
    cudaEventRecord(ea, c->st);
  }
  CUDA_TRY(launch_cg_persistent(f.pp, f.pp == 64 ? 18 : c->recon, q, c->st));
  if (c->prof_on) {
    eb = prof_event(c);
    cudaEventRecord(eb, c->st);
    // bytes and flops are attributed per iteration when the segment's length is known
    double b1, f1, b2, f2, bx, fx;
    dslash_cost(c, f.pp, EPI_CLOVER_INV, 1, &b1, &f1);
    dslash_cost(c, f.pp, EPI_XPAY, 1, &b2, &f2);
    dslash_cost(c, f.pp, EPI_XPAY_CG, 1, &bx, &fx);
    const double sp = 24.0 * real_bytes(f.pp) + (f.pp == 16 ? 4 : 0), sr = 24.0 * real_bytes(f.pr);
    c->pc_pending.push_back({ea, eb, 2 * b1 + b2 + bx + (double)g.Vh * (sr + 2 * sp), 2 * f1 + f2 + fx});
  }
  return QCD_OK;
}

// Iterations to enqueue before the next look at the solver state: the fewest, over the active
// right-hand sides, until a reliable-update trigger (|r| down by reliable_delta since the last
// update, reliable_every iterations, or the target residual), predicted from the per-iteration
// ratio rho of |r|^2 seen so far.  One extra iteration is added: overshooting costs a few
// empty launches, undershooting a host round trip.
int predict_iterations(const qcd_ctx* c, int nrhs, const std::vector<double>& rho, bool after_reliable) {
  const CGControl& ctl = *c->h_ctl;
  long long best = 1LL << 30;
  for (int r = 0; r < nrhs; r++) {
    const CGState& st = c->h_cg[r];
    if (!st.active) continue;
    const int since = after_reliable ? 0 : st.since_reliable;
    long long n = (long long)ctl.reliable_every - since;
    const double rh = rho[r];
    if (rh > 0.0 && rh < 1.0) {
      const double lr = log(rh);
      if (ctl.delta2 > 0.0) {
        const long long k = (long long)ceil(log(ctl.delta2) / lr) - since;
        if (k < n) n = k;
      }
      if (st.rr > 0.0 && st.tol2 > 0.0) {
        const long long k = (long long)ceil(log(st.tol2 / st.rr) / lr) - (after_reliable ? 0 : 0);
        if (k < n) n = k;
      }
    } else if (n > 8) {
      n = 8;
    }
    if (n < best) best = n;
  }
  if (best < 1) best = 1;
  best += 1;
  if (best > 2 * MAX_GRAPH_LEN - 1) best = 2 * MAX_GRAPH_LEN - 1;
  return (int)best;
}

// Rounds of the persistent path (segment + reliable update) expected before convergence: each
// reliable update is due once |r|^2 fell by delta2 (or after reliable_every iterations, at the
// per-iteration ratio rho), and the last one confirms |r|^2 <= tol2.  first: before any look at the
// state, with |r_0| = |b| (a zero initial guess).  Too many rounds cost a few empty launches each, too
// few one more look.
int predict_rounds(const qcd_ctx* c, const qcd_solver_params* prm, bool first, double rho) {
  const CGControl& ctl = *c->h_ctl;
  const CGState& st = c->h_cg[0];
  const double ratio = first ? prm->tol * prm->tol : (st.rr_reliable > 0.0 ? st.tol2 / st.rr_reliable : 1.0);
  double n = 1.0;
  if (ratio > 0.0 && ratio < 1.0) {
    if (ctl.delta2 > 0.0 && ctl.delta2 < 1.0) n = std::max(n, ceil(log(ratio) / log(ctl.delta2) - 1e-9));
    if (rho > 0.0 && rho < 1.0 && ctl.reliable_every > 0)
      n = std::max(n, ceil(log(ratio) / log(rho) / ctl.reliable_every - 1e-9));
  }
  return (int)std::min<double>(n, PC_MAX_ROUNDS);
}

// Solve for one batch of nrhs (1, 2, 4 or 8) canonical fields.
qcd_status cg_batch(qcd_ctx* c, double2* x, const double2* b, int nrhs, const qcd_solver_params* prm,
                    qcd_solver_stats* stats) {
  const Geom& g = c->g;
  SolverFields f;
  qcd_status s = solver_fields(c, prm->inner_prec, nrhs, &f);
  if (s) return s;
  const bool mixed = prm->inner_prec != 64;
  for (int r = 0; r < nrhs; r++) {
    CGState st;
    memset(&st, 0, sizeof st);
    st.tol2 = prm->tol * prm->tol;  // scaled by |b|^2 on the device
    st.active = 1;
    st.reliable_updates = -1;
    c->h_cg[r] = st;
  }
  CGControl ctl;
  memset(&ctl, 0, sizeof ctl);
  ctl.reliable_every = mixed ? (prm->reliable_every > 0 ? prm->reliable_every : 50) : (1 << 30);
  ctl.delta2 = mixed ? prm->reliable_delta * prm->reliable_delta : 0.0;
  *c->h_ctl = ctl;
  CUDA_TRY(cudaMemcpyAsync(c->cg, c->h_cg, sizeof(CGState) * nrhs, cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(cudaMemcpyAsync(c->ctl, c->h_ctl, sizeof(CGControl), cudaMemcpyHostToDevice, c->st));
  // b_hi, |b|^2 (tolerance, zero sources), x_hi = x0 or 0, x_lo = 0, p = 0, r = b - A x_hi, p = r
  launch_spinor_to_native(64, g, b, f.b_hi, nullptr, nrhs, c->st);
  launch_norm2(g, nrhs, f.b_hi, reduce_args(c, FIN_CG_BNORM), c->st);
  if (prm->use_x0) launch_spinor_to_native(64, g, x, f.x_hi, nullptr, nrhs, c->st);
  else launch_zero(f.x_hi, spinor_bytes(g, 64, nrhs), c->st);
  launch_zero(f.x_lo, spinor_bytes(g, f.pr, nrhs), c->st);
  launch_zero(f.p, spinor_bytes(g, f.pp, nrhs), c->st);
  if (f.p_n) launch_zero(f.p_n, sizeof(float) * (size_t)g.Vh * nrhs, c->st);
  if (prm->use_x0)
    apply_mdagm(c, 64, nrhs, f.x_hi, nullptr, f.ap_hi, nullptr, f.t_hi, nullptr, f.y_hi, nullptr, nullptr, nullptr);
  else
    launch_zero(f.ap_hi, spinor_bytes(g, 64, nrhs), c->st);
  launch_true_residual(f.pr, g, nrhs, f.b_hi, f.ap_hi, f.r_lo, f.r_lo_n, reduce_args(c, FIN_CG_TRUE), c->st);
  launch_p_update(f.pr, f.pp, g, nrhs, f.r_lo, f.r_lo_n, f.p, f.p_n, c->cg, nullptr, c->st);

  std::vector<double> rho(nrhs, c->last_rho);
  // event pairs of persistent launches and graphs left by a solve that returned early (an error)
  // are dropped
  for (const auto& pp : c->pc_pending) {
    c->ev_free.push_back(pp.a);
    c->ev_free.push_back(pp.b);
  }
  c->pc_pending.clear();
  c->launched.clear();
  // one RHS: the persistent kernel runs each segment of iterations, and the rounds (segment, gated
  // reliable update) expected before convergence are enqueued together, with one look at the state
  // after them
  const bool use_pc = c->persistent && nrhs == 1 && g.Vh <= PERSISTENT_MAX_VH;
  qcd_status result = QCD_OK;
  bool after_reliable = true;
  int done_iters = 0;
  ItGraph* rel = nullptr;
  while (true) {
    // the state is only known after a synchronisation; right after the set-up or a reliable
    // update the host copy is stale, which predict_iterations accounts for
    int rounds = 0;
    if (use_pc) {
      rounds = predict_rounds(c, prm, done_iters == 0, rho[0]);
      CUDA_TRY(cudaMemsetAsync(c->pc_bar + 2, 0, sizeof(unsigned), c->st));
      for (int k = 0; k < rounds; k++) {
        if ((s = launch_persistent(c, f, prm->max_iter, k))) return s;
        ItGraph* rk;
        if ((s = get_graph(c, 1, k, f, nrhs, &rk))) return s;
        if ((s = launch_graph(c, rk, 0, k))) return s;
      }
      CUDA_TRY(cudaMemcpyAsync(c->h_pc_rounds, c->pc_rounds, sizeof(int) * rounds, cudaMemcpyDeviceToHost, c->st));
    } else {
      const int n = std::min(predict_iterations(c, nrhs, rho, after_reliable), std::max(1, prm->max_iter - done_iters));
      if ((s = launch_iterations(c, f, nrhs, n))) return s;
    }
    if ((s = read_state(c, nrhs))) return s;
    if (use_pc && c->h_flags[2]) return fail(QCD_ERR_TIMEOUT, "a grid barrier of the persistent CG kernel timed out");
    int max_it = 0;
    bool active = false, candidate = false;
    for (int r = 0; r < nrhs; r++) {
      const CGState& st = c->h_cg[r];
      max_it = std::max(max_it, st.iters);
      active |= st.active != 0;
      candidate |= st.active && st.pending && st.rr <= st.tol2;
      if (st.active && st.since_reliable > 0 && st.rr_reliable > 0.0 && st.rr > 0.0)
        rho[r] = pow(st.rr / st.rr_reliable, 1.0 / st.since_reliable);
    }
    if (c->prof_on) collect_graphs(c, max_it - done_iters, use_pc ? c->h_pc_rounds : nullptr);
    if (!c->pc_pending.empty()) {
      // the persistent launches of this look, each with the iterations it ran (no-op launches of
      // rounds past convergence are not counted)
      const int cls = prof_class(c, f.pp == 64 ? "cg_persistent_p64"
                                               : (f.pp == 32 ? "cg_persistent_p32" : "cg_persistent_p16"));
      for (size_t k = 0; k < c->pc_pending.size(); k++) {
        const auto& pp = c->pc_pending[k];
        const int n_it = k < (size_t)rounds ? c->h_pc_rounds[k] >> 1 : 0;
        float ms = 0.f;
        if (n_it > 0 && cudaEventElapsedTime(&ms, pp.a, pp.b) == cudaSuccess) {
          ProfClass& pc = c->prof[cls];
          pc.launches += 1;
          pc.ms += ms;
          pc.bytes += n_it * pp.bytes_per_iter;
          pc.flops += n_it * pp.flops_per_iter;
        } else {
          cudaGetLastError();
        }
        c->ev_free.push_back(pp.a);
        c->ev_free.push_back(pp.b);
      }
      c->pc_pending.clear();
    }
    const bool progress = max_it > done_iters;
    done_iters = max_it;
    if (c->h_ctl->overflow) return fail(QCD_ERR_CUDA, "reduction buffer too small (internal sizing error)");
    if (c->h_ctl->nan) {
      result = fail(QCD_ERR_NAN, "non-finite value or breakdown in CG");
      break;
    }
    if (!active) break;
    if (max_it >= prm->max_iter) {
      result = fail(QCD_ERR_NOT_CONVERGED, "CG did not converge in %d iterations", prm->max_iter);
      break;
    }
    if (use_pc && !progress) {
      // every round returned at once with the RHS still active: nothing more would change
      result = fail(QCD_ERR_NOT_CONVERGED, "persistent CG stopped making progress after %d iterations", max_it);
      break;
    }
    after_reliable = false;
    if (c->h_ctl->halt) {
      if (!rel && (s = get_graph(c, 1, 0, f, nrhs, &rel))) return s;
      if ((s = launch_graph(c, rel, 0))) return s;
      after_reliable = true;
      if (candidate) {
        // the update may have finished the solve: look before enqueuing more iterations
        if ((s = read_state(c, nrhs))) return s;
        if (c->prof_on) collect_graphs(c, 0);
        bool any = false;
        for (int r = 0; r < nrhs; r++) any |= c->h_cg[r].active != 0;
        if (c->h_ctl->nan) {
          result = fail(QCD_ERR_NAN, "non-finite value in the reliable update");
          break;
        }
        if (!any) break;
      }
    }
  }
  for (int r = 0; r < nrhs; r++)
    if (rho[r] > 0.0 && rho[r] < 1.0) c->last_rho = rho[r];
  // not converged: fold the progress into x and recompute the true residual for the stats
  if (result == QCD_ERR_NOT_CONVERGED) enqueue_reliable(c, f, nrhs, false);
  // fold the last low-precision increment into x and write out
  launch_accumulate_x(f.pr, g, nrhs, f.x_hi, f.x_lo, f.x_lo_n, c->st);
  launch_spinor_to_canon(64, g, f.x_hi, nullptr, x, nrhs, c->st);
  launch_redot(g, nrhs, f.b_hi, f.x_hi, reduce_args(c, FIN_STORE), c->st);
  CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->st));
  if ((s = read_state(c, nrhs))) return s;
  if (c->prof_on) collect_graphs(c, 0);
  if (stats) {
    for (int r = 0; r < nrhs; r++) {
      const CGState& st = c->h_cg[r];
      stats[r].iters = st.iters;
      stats[r].reliable_updates = st.reliable_updates;
      stats[r].true_rel_resid = st.bnorm2 > 0 ? sqrt(st.true_rr / st.bnorm2) : 0.0;
      stats[r].b_dot_x = c->h_results[r];
    }
  }
  return result;
}

qcd_status check_params(const qcd_solver_params* p) {
  if (!p) return fail(QCD_ERR_ARG, "null solver params");
  if (!(p->tol > 0.0) || p->max_iter < 1) return fail(QCD_ERR_ARG, "tol must be > 0 and max_iter >= 1");
  if (!valid_prec(p->inner_prec)) return fail(QCD_ERR_ARG, "inner_prec must be 64, 32 or 16");
  if (p->inner_prec != 64 && !(p->reliable_delta >= 0.0 && p->reliable_delta < 1.0))
    return fail(QCD_ERR_ARG, "reliable_delta must be in [0, 1)");
  return QCD_OK;
}

}  // namespace

extern "C" {

qcd_status qcd_cg_solve(qcd_ctx* c, double* x, const double* b, int nrhs, const qcd_solver_params* prm,
                        qcd_solver_stats* stats) {
  QCD_API_ENTER("qcd_cg_solve", c);
  if (qcd_status rs = slab_refuse(c, "qcd_cg_solve", true)) return rs;
  qcd_status s = QCD_OK;
  if (!x || !b) return fail(QCD_ERR_ARG, "null field pointer");
  if (nrhs < 1) return fail(QCD_ERR_ARG, "nrhs must be >= 1");
  if ((s = check_params(prm))) return s;
  if (!c->have_clover) return fail(QCD_ERR_STATE, "cg_solve before clover_build");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t fs = (size_t)c->g.Vh * 12;
  qcd_status worst = QCD_OK;
  int done = 0;
  while (done < nrhs) {
    const int nb = batch_of(nrhs - done);
    s = cg_batch(c, reinterpret_cast<double2*>(x) + done * fs, reinterpret_cast<const double2*>(b) + done * fs, nb,
                 prm, stats ? stats + done : nullptr);
    if (s == QCD_ERR_NOT_CONVERGED) worst = s;
    else if (s) return s;
    done += nb;
  }
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int r = 0; r < nrhs; r++) stats[r].seconds = sec;
  return worst;
}

qcd_status qcd_fermion_force(qcd_ctx* c, double* F, const double* phi_or_x, int nrhs, int flags,
                             const qcd_solver_params* prm, qcd_solver_stats* stats) {
  QCD_API_ENTER("qcd_fermion_force", c);
  if (qcd_status rs = slab_refuse(c, "qcd_fermion_force", false)) return rs;
  qcd_status s = QCD_OK;
  const bool det = (flags & QCD_FORCE_CLOVER_DET) != 0;
  if (!F || (!phi_or_x && nrhs > 0)) return fail(QCD_ERR_ARG, "null pointer");
  if (nrhs < (det ? 0 : 1)) return fail(QCD_ERR_ARG, "nrhs must be >= 1 (>= 0 with QCD_FORCE_CLOVER_DET)");
  if (flags & ~(QCD_FORCE_INPUT_IS_SOLUTION | QCD_FORCE_GRADIENT | QCD_FORCE_CLOVER_DET))
    return fail(QCD_ERR_ARG, "unknown force flags");
  if (!c->have_clover) return fail(QCD_ERR_STATE, "fermion_force before clover_build");
  const Geom& g = c->g;
  if (nrhs == 0) {
    // the determinant term alone: its coefficients into a zeroed buffer, then the leaves
    void* clf;
    if ((s = ws_get(c, S_F_CL, force_clover_bytes(g), &clf))) return s;
    CUDA_TRY(cudaMemsetAsync(clf, 0, force_clover_bytes(g), c->st));
    const double V = 2.0 * g.Vh;
    {
      ProfScope ps(c, "force_det_coeff", g.Vh * (72 * 16.0) + V * 6 * 144.0 * 2, 0.0);
      launch_force_det_coeff(g, c->kappa, c->csw, static_cast<const double2*>(clover_ptr(c, 64, true, 1)),
                             static_cast<double2*>(clf), c->st);
    }
    void* ef;
    if ((s = ws_get(c, S_F_E, force_edge_bytes(g), &ef))) return s;
    {
      ProfScope ps(c, "force_edges", V * (6 + 4 + 12) * 144.0, V * force_edge_flops());
      launch_force_edges(g, c->g64, static_cast<const double2*>(clf), static_cast<double2*>(ef), c->st);
    }
    ProfScope ps(c, "force_links", 4 * V * (144.0 + 3 * 144.0 + 144.0), 4 * V * force_link_flops(0, true));
    launch_force_links(g, c->kappa, 0, c->g64, nullptr, nullptr, nullptr, nullptr, static_cast<const double2*>(ef),
                       reinterpret_cast<double2*>(F), (flags & QCD_FORCE_GRADIENT) != 0, true, false, c->st);
    return sync_and_check(c, "fermion_force");
  }
  const size_t fs = (size_t)g.Vh * 12;
  // X (canonical, FP64) for all RHS
  const double2* X = reinterpret_cast<const double2*>(phi_or_x);
  if (!(flags & QCD_FORCE_INPUT_IS_SOLUTION)) {
    if ((s = check_params(prm))) return s;
    void* v;
    if ((s = ws_get(c, S_CANON, fs * nrhs * sizeof(double2), &v))) return s;
    CUDA_TRY(cudaMemsetAsync(v, 0, fs * nrhs * sizeof(double2), c->st));
    qcd_solver_params p2 = *prm;
    p2.use_x0 = 0;
    s = qcd_cg_solve(c, static_cast<double*>(v), phi_or_x, nrhs, &p2, stats);
    if (s && s != QCD_ERR_NOT_CONVERGED) return s;
    X = static_cast<const double2*>(v);
  }
  // native FP64 X_e, Y_e = Mhat X_e, X_o = A^-1 D_oe X_e, Y_o = g5 A^-1 D_oe g5 Y_e; batches of <= 8 RHS
  const size_t hi1 = spinor_bytes(g, 64, 1);
  void *xf, *yf, *clf, *ef;
  if ((s = ws_get(c, S_F_X, 2 * hi1 * nrhs, &xf)) || (s = ws_get(c, S_F_Y, 2 * hi1 * nrhs, &yf)) ||
      (s = ws_get(c, S_F_CL, force_clover_bytes(g), &clf)) || (s = ws_get(c, S_F_E, force_edge_bytes(g), &ef)))
    return s;
  double2* Xe = static_cast<double2*>(xf);
  double2* Xo = Xe + (size_t)nrhs * 12 * g.Vh;
  double2* Ye = static_cast<double2*>(yf);
  double2* Yo = Ye + (size_t)nrhs * 12 * g.Vh;
  // per batch (RHS interleaved within a batch): convert X, then Y_e, X_o, Y_o; the clover
  // coefficients accumulate over the batches
  const double V = 2.0 * g.Vh;
  std::vector<std::pair<size_t, int>> batches;
  for (int done = 0; done < nrhs;) {
    const int nb = batch_of(nrhs - done);
    batches.push_back({(size_t)done * 12 * g.Vh, nb});
    done += nb;
  }
  for (size_t k = 0; k < batches.size(); k++) {
    const size_t off = batches[k].first;
    const int nb = batches[k].second;
    launch_spinor_to_native(64, g, X + off, Xe + off, nullptr, nb, c->st);
    // Y_e = Mhat X_e with X_o = A_oo^-1 D_oe X_e left in the odd temporary
    apply_mhat(c, 64, nb, false, Xe + off, nullptr, Ye + off, nullptr, Xo + off, nullptr, nullptr, nullptr);
    // Y_o = A_oo^-1 D_eo^dag Y_e = g5 A_oo^-1 D_oe g5 Y_e
    DslashArgs a = base_args(c, 64, 1, nb);
    a.in = Ye + off;
    a.out = Yo + off;
    a.clover = clover_ptr(c, 64, true, 1);
    a.in_g5 = 1;
    a.out_g5 = 1;
    run_dslash(c, 64, EPI_CLOVER_INV, a);
    ProfScope ps(c, "force_clover_coeff", V * (nb * 2 * 192.0 + 6 * 144.0), V * force_coeff_flops(nb));
    launch_force_coeff(g, c->kappa, c->csw, nb, Xe + off, Xo + off, Ye + off, Yo + off, static_cast<double2*>(clf),
                       k > 0, c->st);
  }
  if (det) {
    ProfScope ps(c, "force_det_coeff", g.Vh * (72 * 16.0) + V * 6 * 144.0 * 2, 0.0);
    launch_force_det_coeff(g, c->kappa, c->csw, static_cast<const double2*>(clover_ptr(c, 64, true, 1)),
                           static_cast<double2*>(clf), c->st);
  }
  {
    ProfScope ps(c, "force_edges", V * (6 + 4 + 12) * 144.0, V * force_edge_flops());
    launch_force_edges(g, c->g64, static_cast<const double2*>(clf), static_cast<double2*>(ef), c->st);
  }
  // per link: the hopping part of every batch, the clover part once (F is linear in G)
  for (size_t k = 0; k < batches.size(); k++) {
    const size_t off = batches[k].first;
    const int nb = batches[k].second;
    // compulsory bytes per link: the link, its share of the E fields (three per link), the output,
    // and a quarter of each site's four FP64 spinors per RHS
    ProfScope ps(c, "force_links", 4 * V * (144.0 + (k == 0 ? 3 * 144.0 : 0.0) + 144.0 + 192.0 * nb),
                 4 * V * force_link_flops(nb, k == 0));
    launch_force_links(g, c->kappa, nb, c->g64, Xe + off, Xo + off, Ye + off, Yo + off,
                       static_cast<const double2*>(ef), reinterpret_cast<double2*>(F),
                       (flags & QCD_FORCE_GRADIENT) != 0, k == 0, k > 0, c->st);
  }
  return sync_and_check(c, "fermion_force");
}

qcd_status qcd_selftest_barrier_timeout(qcd_ctx* c) {
  QCD_API_ENTER("qcd_selftest_barrier_timeout", c);
  qcd_status s = QCD_OK;
  CUDA_TRY(cudaMemsetAsync(c->pc_bar, 0, 4 * sizeof(unsigned), c->st));
  CUDA_TRY(launch_barrier_probe(c->pc_bar, reinterpret_cast<int*>(c->pc_bar + 2), c->st));
  CUDA_TRY(cudaMemcpyAsync(c->h_flags + 2, c->pc_bar + 2, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "barrier self-test"))) return s;
  CUDA_TRY(cudaMemsetAsync(c->pc_bar, 0, 4 * sizeof(unsigned), c->st));
  if (c->h_flags[2]) return fail(QCD_ERR_TIMEOUT, "grid barrier wait gave up as intended");
  return QCD_OK;
}

static_assert(QCD_DBG_SPINOR == DBG_SPINOR && QCD_DBG_LINK == DBG_LINK && QCD_DBG_CLOVER == DBG_CLOVER &&
                  QCD_DBG_HALO == DBG_HALO,
              "debug bits of the header and the kernels");

qcd_status qcd_debug_violations(qcd_ctx* c, unsigned* violations, int* is_debug) {
  QCD_API_ENTER("qcd_debug_violations", c);
  qcd_status s = QCD_OK;
  if (!violations) return fail(QCD_ERR_ARG, "null pointer");
  if ((s = sync_and_check(c, "debug_violations"))) return s;
  *violations = debug_take_blas() | debug_take_cg_persistent() | debug_take_clover() | debug_take_dslash() |
                debug_take_force() | debug_take_halo() | debug_take_layout() | debug_take_md() |
                debug_take_probe();
  if (is_debug) *is_debug = QCD_DEBUG;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "debug_violations: %s", cudaGetErrorString(e));
  return QCD_OK;
}

qcd_status qcd_selftest_debug_index(qcd_ctx* c) {
  QCD_API_ENTER("qcd_selftest_debug_index", c);
  qcd_status s = QCD_OK;
  double2* buf = nullptr;
  double* out = nullptr;
  const size_t n = (size_t)13 * c->g.Vh;
  if (cudaMalloc(&buf, n * sizeof(double2)) != cudaSuccess || cudaMalloc(&out, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf);
    return fail(QCD_ERR_NOMEM, "debug index self-test: allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(buf, 0, n * sizeof(double2), c->st);
  if (e == cudaSuccess) launch_debug_index_probe(c->g, buf, out, c->st);
  s = e == cudaSuccess ? sync_and_check(c, "debug index self-test") : fail(QCD_ERR_CUDA, "%s", cudaGetErrorString(e));
  cudaFree(buf);
  cudaFree(out);
  return s;
}

qcd_status qcd_clover_logdet(qcd_ctx* c, double out[2]) {
  QCD_API_ENTER("qcd_clover_logdet", c);
  qcd_status s = QCD_OK;
  if (!out) return fail(QCD_ERR_ARG, "null pointer");
  if (!c->have_clover) return fail(QCD_ERR_STATE, "clover_logdet before clover_build");
  launch_parity_sum(c->g, c->logdet, reduce_args(c, FIN_STORE), c->st);
  CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "clover_logdet"))) return s;
  out[0] = c->h_results[0];
  out[1] = c->h_results[1];
  return QCD_OK;
}

// shared checks of the two full-lattice helpers
static qcd_status eo_check(qcd_ctx* c, const void* out, const void* in1, const void* in2, int nrhs) {
  if (!out || !in1) return fail(QCD_ERR_ARG, "null field pointer");
  if (nrhs < 1) return fail(QCD_ERR_ARG, "nrhs must be >= 1");
  if (!c->have_clover) return fail(QCD_ERR_STATE, "needs clover_build");
  const size_t bytes = (size_t)c->g.Vh * 12 * sizeof(double2) * nrhs;
  for (const void* in : {in1, in2})
    if (in && (const char*)out < (const char*)in + bytes && (const char*)in < (const char*)out + bytes)
      return fail(QCD_ERR_ARG, "output overlaps an input");
  return QCD_OK;
}

qcd_status qcd_prepare_source(qcd_ctx* c, double* bhat_e, const double* b_e, const double* b_o, int nrhs) {
  QCD_API_ENTER("qcd_prepare_source", c);
  if (qcd_status rs = slab_refuse(c, "qcd_prepare_source", false)) return rs;
  qcd_status s = eo_check(c, bhat_e, b_e, b_o, nrhs);
  if (s) return s;
  const Geom& g = c->g;
  const size_t n = (size_t)g.Vh * 12;
  for (int done = 0; done < nrhs;) {
    const int nb = batch_of(nrhs - done);
    const double2* ce = reinterpret_cast<const double2*>(b_e) + done * n;
    double2* cout = reinterpret_cast<double2*>(bhat_e) + done * n;
    if (!b_o) {
      CUDA_TRY(cudaMemcpyAsync(cout, ce, n * nb * sizeof(double2), cudaMemcpyDeviceToDevice, c->st));
    } else {
      void *u, *t;
      const size_t fb = spinor_bytes(g, 64, nb);
      if ((s = ws_get(c, S_IN, fb, &u)) || (s = ws_get(c, S_T, fb, &t))) return s;
      // t = A_oo^-1 b_o, u = D_eo t (native), bhat_e = kappa u + b_e (canonical)
      launch_spinor_to_native(64, g, reinterpret_cast<const double2*>(b_o) + done * n, u, nullptr, nb, c->st);
      launch_clover_apply(64, g, clover_ptr(c, 64, true, 1), u, nullptr, t, nullptr, nb, c->st);
      DslashArgs a = base_args(c, 64, 0, nb);
      a.in = t;
      a.out = u;
      run_dslash(c, 64, EPI_NONE, a);
      launch_spinor_to_canon(64, g, u, nullptr, cout, nb, c->st);
      launch_axpby(n * nb, 1.0, ce, c->kappa, cout, c->st);
    }
    done += nb;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "prepare_source launch: %s", cudaGetErrorString(e));
  return QCD_OK;
}

qcd_status qcd_reconstruct_odd(qcd_ctx* c, double* x_o, const double* x_e, const double* b_o, int nrhs) {
  QCD_API_ENTER("qcd_reconstruct_odd", c);
  if (qcd_status rs = slab_refuse(c, "qcd_reconstruct_odd", false)) return rs;
  qcd_status s = eo_check(c, x_o, x_e, b_o, nrhs);
  if (s) return s;
  const Geom& g = c->g;
  const size_t n = (size_t)g.Vh * 12;
  for (int done = 0; done < nrhs;) {
    const int nb = batch_of(nrhs - done);
    void *u, *t;
    const size_t fb = spinor_bytes(g, 64, nb);
    if ((s = ws_get(c, S_IN, fb, &u)) || (s = ws_get(c, S_T, fb, &t))) return s;
    // t = A_oo^-1 D_oe x_e (one fused launch), then x_o = kappa t + A_oo^-1 b_o
    launch_spinor_to_native(64, g, reinterpret_cast<const double2*>(x_e) + done * n, u, nullptr, nb, c->st);
    DslashArgs a = base_args(c, 64, 1, nb);
    a.in = u;
    a.out = t;
    a.clover = clover_ptr(c, 64, true, 1);
    run_dslash(c, 64, EPI_CLOVER_INV, a);
    double2* cout = reinterpret_cast<double2*>(x_o) + done * n;
    launch_spinor_to_canon(64, g, t, nullptr, cout, nb, c->st);
    if (b_o) {
      launch_spinor_to_native(64, g, reinterpret_cast<const double2*>(b_o) + done * n, u, nullptr, nb, c->st);
      launch_clover_apply(64, g, clover_ptr(c, 64, true, 1), u, nullptr, t, nullptr, nb, c->st);
      // x_o = kappa x_o + (A_oo^-1 b_o): the native result goes through the canonical staging
      void* stage;
      if ((s = ws_get(c, S_CANON, n * nb * sizeof(double2), &stage))) return s;
      launch_spinor_to_canon(64, g, t, nullptr, static_cast<double2*>(stage), nb, c->st);
      launch_axpby(n * nb, 1.0, static_cast<const double2*>(stage), c->kappa, cout, c->st);
    } else {
      launch_axpby(n * nb, 0.0, cout, c->kappa, cout, c->st);
    }
    done += nb;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "reconstruct_odd launch: %s", cudaGetErrorString(e));
  return QCD_OK;
}

qcd_status qcd_gauge_force(qcd_ctx* c, double* F, double beta, int flags) {
  QCD_API_ENTER("qcd_gauge_force", c);
  if (qcd_status rs = slab_refuse(c, "qcd_gauge_force", false)) return rs;
  qcd_status s = QCD_OK;
  if (!F) return fail(QCD_ERR_ARG, "null pointer");
  if (flags & ~(QCD_FORCE_GRADIENT | QCD_FORCE_ACCUMULATE)) return fail(QCD_ERR_ARG, "unknown gauge force flags");
  if (!c->have_gauge) return fail(QCD_ERR_STATE, "gauge_force before load_gauge");
  {
    const double V = 2.0 * c->g.Vh;
    ProfScope ps(c, "gauge_force", 4 * V * (18 * 144.0 + 144.0 * ((flags & QCD_FORCE_ACCUMULATE) ? 2 : 1)),
                 4 * V * 13 * 198.0);
    launch_gauge_force(c->g, beta, c->g64, reinterpret_cast<double2*>(F), (flags & QCD_FORCE_GRADIENT) != 0,
                       (flags & QCD_FORCE_ACCUMULATE) != 0, c->st);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "gauge_force launch: %s", cudaGetErrorString(e));
  return QCD_OK;
}

qcd_status qcd_plaquette(qcd_ctx* c, double* mean) {
  QCD_API_ENTER("qcd_plaquette", c);
  if (qcd_status rs = slab_refuse(c, "qcd_plaquette", false)) return rs;
  qcd_status s = QCD_OK;
  if (!mean) return fail(QCD_ERR_ARG, "null pointer");
  if (!c->have_gauge) return fail(QCD_ERR_STATE, "plaquette before load_gauge");
  launch_plaquette(c->g, c->g64, reduce_args(c, FIN_STORE), c->st);
  CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "plaquette"))) return s;
  *mean = c->h_results[0] / (6.0 * 2.0 * c->g.Vh);
  return QCD_OK;
}

qcd_status qcd_kinetic_energy(qcd_ctx* c, const double* P, double* K) {
  QCD_API_ENTER("qcd_kinetic_energy", c);
  if (qcd_status rs = slab_refuse(c, "qcd_kinetic_energy", false)) return rs;
  qcd_status s = QCD_OK;
  if (!P || !K) return fail(QCD_ERR_ARG, "null pointer");
  launch_flat_norm2((size_t)c->g.Vh * 2 * 4 * 9, reinterpret_cast<const double2*>(P), reduce_args(c, FIN_STORE),
                    c->st);
  CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "kinetic_energy"))) return s;
  *K = c->h_results[0];
  return QCD_OK;
}

qcd_status qcd_update_links(qcd_ctx* c, double* U, const double* P, double eps) {
  QCD_API_ENTER("qcd_update_links", c);
  if (qcd_status rs = slab_refuse(c, "qcd_update_links", false)) return rs;
  qcd_status s = QCD_OK;
  if (!U || !P) return fail(QCD_ERR_ARG, "null pointer");
  const size_t nlinks = (size_t)c->g.Vh * 2 * 4;
  if ((const char*)U < (const char*)P + nlinks * 9 * sizeof(double2) &&
      (const char*)P < (const char*)U + nlinks * 9 * sizeof(double2))
    return fail(QCD_ERR_ARG, "U and P overlap");
  {
    ProfScope ps(c, "link_update", nlinks * 3 * 144.0, nlinks * 10 * 198.0);
    launch_link_update(nlinks, eps, reinterpret_cast<const double2*>(P), reinterpret_cast<double2*>(U), c->st);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "update_links launch: %s", cudaGetErrorString(e));
  return QCD_OK;
}

qcd_status qcd_r_step(qcd_ctx* c, double* U, double* P, const double* eta, int nrhs, double eps, double beta,
                      int flags, const qcd_solver_params* prm, qcd_solver_stats* stats) {
  QCD_API_ENTER("qcd_r_step", c);
  if (qcd_status rs = slab_refuse(c, "qcd_r_step", false)) return rs;
  qcd_status s = QCD_OK;
  if (!U || !P || (!eta && nrhs > 0)) return fail(QCD_ERR_ARG, "null pointer");
  if (nrhs < 0) return fail(QCD_ERR_ARG, "nrhs must be >= 0");
  if (flags & ~(QCD_FORCE_CLOVER_DET | QCD_R_STEP_DEFER_CLOVER)) return fail(QCD_ERR_ARG, "unknown r_step flags");
  if (!c->have_kappa) return fail(QCD_ERR_STATE, "r_step needs kappa and c_sw from a clover_build");
  if (nrhs > 0 && (s = check_params(prm))) return s;
  const Geom& g = c->g;
  const double kappa = c->kappa, csw = c->csw;
  const int gflags = c->recon == 12 ? QCD_GAUGE_RECON12 : 0;
  const size_t nlinks = (size_t)g.Vh * 2 * 4;
  void *fv, *phiv = nullptr;
  if ((s = ws_get(c, S_MD_F, nlinks * 9 * sizeof(double2), &fv))) return s;
  if (nrhs > 0 && (s = ws_get(c, S_MD_PHI, (size_t)g.Vh * 12 * sizeof(double2) * nrhs, &phiv))) return s;
  double* F = static_cast<double*>(fv);
  // half step of the links, then the fields at U'
  if ((s = qcd_update_links(c, U, P, 0.5 * eps))) return s;
  if ((s = qcd_load_gauge(c, U, 1, gflags)) || (s = qcd_clover_build(c, kappa, csw))) return s;
  const int fflags = QCD_FORCE_CLOVER_DET & flags;
  if (nrhs > 0) {
    if ((s = qcd_dslash(c, static_cast<double*>(phiv), eta, QCD_OP_MHAT, 1, 64, nrhs))) return s;
    s = qcd_fermion_force(c, F, static_cast<const double*>(phiv), nrhs, fflags, prm, stats);
  } else if (fflags) {
    s = qcd_fermion_force(c, F, nullptr, 0, fflags, nullptr, nullptr);
  } else {
    CUDA_TRY(cudaMemsetAsync(F, 0, nlinks * 9 * sizeof(double2), c->st));
  }
  if (s && s != QCD_ERR_NOT_CONVERGED) return s;
  const qcd_status solve_status = s;
  if ((s = qcd_gauge_force(c, F, beta, QCD_FORCE_ACCUMULATE))) return s;
  // P -= eps F, then the second half step
  launch_axpby(nlinks * 9, -eps, reinterpret_cast<const double2*>(F), 1.0, reinterpret_cast<double2*>(P), c->st);
  if ((s = qcd_update_links(c, U, P, 0.5 * eps))) return s;
  if ((s = qcd_load_gauge(c, U, 1, gflags))) return s;
  if (!(flags & QCD_R_STEP_DEFER_CLOVER) && (s = qcd_clover_build(c, kappa, csw))) return s;
  return solve_status;
}

qcd_status qcd_polyakov(qcd_ctx* c, double out[2]) {
  QCD_API_ENTER("qcd_polyakov", c);
  if (qcd_status rs = slab_refuse(c, "qcd_polyakov", false)) return rs;
  qcd_status s = QCD_OK;
  if (!out) return fail(QCD_ERR_ARG, "null pointer");
  if (!c->have_gauge) return fail(QCD_ERR_STATE, "polyakov before load_gauge");
  launch_polyakov(c->g, c->g64, reduce_args(c, FIN_STORE), c->st);
  CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if ((s = sync_and_check(c, "polyakov"))) return s;
  out[0] = c->h_results[0] / c->g.XYZ;
  out[1] = c->h_results[1] / c->g.XYZ;
  return QCD_OK;
}

qcd_status qcd_pbp(qcd_ctx* c, const double* eta_e, const double* eta_o, int nrhs, double* out,
                   const qcd_solver_params* prm, qcd_solver_stats* stats) {
  QCD_API_ENTER("qcd_pbp", c);
  if (qcd_status rs = slab_refuse(c, "qcd_pbp", false)) return rs;
  qcd_status s = QCD_OK;
  if (!eta_e || !eta_o || !out) return fail(QCD_ERR_ARG, "null pointer");
  if (nrhs < 1 || nrhs > MAX_RHS) return fail(QCD_ERR_ARG, "nrhs must be in 1..%d", MAX_RHS);
  if (!c->have_clover) return fail(QCD_ERR_STATE, "pbp needs a clover term");
  if ((s = check_params(prm))) return s;
  const Geom& g = c->g;
  const size_t n = (size_t)g.Vh * 12, fb = n * nrhs * sizeof(double2);
  void* w;
  if ((s = ws_get(c, S_PBP, 4 * fb, &w))) return s;
  double2* bh = static_cast<double2*>(w);
  double2* rhs = bh + n * nrhs;
  double2* xe = rhs + n * nrhs;
  double2* xo = xe + n * nrhs;
  if ((s = qcd_prepare_source(c, reinterpret_cast<double*>(bh), eta_e, eta_o, nrhs))) return s;
  if ((s = qcd_dslash(c, reinterpret_cast<double*>(rhs), reinterpret_cast<const double*>(bh), QCD_OP_MHAT, 1, 64,
                      nrhs)))
    return s;
  CUDA_TRY(cudaMemsetAsync(xe, 0, fb, c->st));
  qcd_solver_params p2 = *prm;
  p2.use_x0 = 0;
  const qcd_status solve_status = qcd_cg_solve(c, reinterpret_cast<double*>(xe), reinterpret_cast<const double*>(rhs),
                                               nrhs, &p2, stats);
  if (solve_status && solve_status != QCD_ERR_NOT_CONVERGED) return solve_status;
  if ((s = qcd_reconstruct_odd(c, reinterpret_cast<double*>(xo), reinterpret_cast<const double*>(xe), eta_o, nrhs)))
    return s;
  // Re <eta_e, x_e> + Re <eta_o, x_o> per RHS
  std::vector<double> acc(nrhs, 0.0);
  for (int half = 0; half < 2; half++) {
    launch_flat_redot(n, nrhs, reinterpret_cast<const double2*>(half ? eta_o : eta_e), half ? xo : xe,
                      reduce_args(c, FIN_STORE), c->st);
    CUDA_TRY(cudaMemcpyAsync(c->h_results, c->results, nrhs * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if ((s = sync_and_check(c, "pbp"))) return s;
    for (int r = 0; r < nrhs; r++) acc[r] += c->h_results[r];
  }
  for (int r = 0; r < nrhs; r++) out[r] = acc[r] / (2.0 * 2.0 * g.Vh);
  return solve_status;
}

long long qcd_selftest_site_order(void) {
  long long bad = 0;
  std::vector<char> seen;
  auto check = [&](int X, int Y, int Z, int T) {
    Geom g{};
    g.X = X;
    g.Y = Y;
    g.Z = Z;
    g.T = T;
    g.XY = X * Y;
    g.XYZ = X * Y * Z;
    g.Vh = X * Y * Z * T / 2;
    const int nb = (g.Vh + 31) / 32;
    seen.assign(nb, 0);
    for (int b = 0; b < nb; b++) {
      const int s = site_block_order(g, b);
      if (s < 0 || s >= nb || seen[s]) {
        bad++;
        return;
      }
      seen[s] = 1;
    }
  };
  for (int X = 2; X <= 16; X += 2)
    for (int Y = 2; Y <= 16; Y += 2)
      for (int Z = 2; Z <= 16; Z += 2)
        for (int T = 2; T <= 34; T += 2) check(X, Y, Z, T);
  check(32, 32, 32, 64);
  check(32, 32, 32, 60);
  check(48, 48, 48, 96);
  check(16, 16, 16, 16);
  check(8, 8, 16, 16);
  return bad;
}

long long qcd_selftest_fastdiv(void) {
  long long bad = 0;
  unsigned long long state = 0x9E3779B97F4A7C15ULL;  // xorshift64 numerators
  for (int d = 2; d <= 1024; d += 2) {
    const FastDiv f = make_fastdiv(d);
    auto check = [&](long long n) {
      if (n < 0 || n > 0x7fffffffLL) return;
      if (f.div((int)n) != (int)(n / d)) bad++;
    };
    for (long long n = 0; n < 65536; n++) check(n);
    for (long long q = d; q <= 0x7fffffffLL; q = q * 3 + d) {
      const long long m = q / d * d;
      check(m - 1);
      check(m);
      check(m + d - 1);
    }
    check(0x7fffffffLL);
    for (int k = 0; k < 4096; k++) {
      state ^= state << 13;
      state ^= state >> 7;
      state ^= state << 17;
      check((long long)(state & 0x7fffffffULL));
    }
  }
  return bad;
}

qcd_status qcd_profile(qcd_ctx* c, int enable) {
  QCD_API_ENTER("qcd_profile", c);
  qcd_status s = QCD_OK;
  if ((s = sync_and_check(c, "profile"))) return s;
  prof_collect(c);
  if (enable) {
    // counters restart; the classes keep their indices, which the event slots of recorded CUDA
    // graphs hold
    for (ProfClass& pc : c->prof) {
      pc.launches = 0;
      pc.ms = pc.bytes = pc.flops = 0;
    }
    g_kernel_launches = 0;
  }
  c->prof_on = enable != 0;
  return QCD_OK;
}

qcd_status qcd_profile_read(qcd_ctx* c, qcd_kernel_stat* out, int max_entries, int* n_entries) {
  QCD_API_ENTER("qcd_profile_read", c);
  qcd_status s = QCD_OK;
  if (!n_entries || (max_entries > 0 && !out)) return fail(QCD_ERR_ARG, "null output");
  CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_collect(c);
  int n = 0;
  for (auto& p : c->prof) {
    if (p.launches == 0) continue;
    if (n >= max_entries) break;
    memset(&out[n], 0, sizeof(qcd_kernel_stat));
    snprintf(out[n].name, sizeof out[n].name, "%s", p.name.c_str());
    out[n].launches = p.launches;
    out[n].total_ms = p.ms;
    out[n].bytes = p.bytes;
    out[n].flops = p.flops;
    n++;
  }
  if (n < max_entries) {
    // pseudo-entry: every kernel the library launched since qcd_profile(ctx, 1)
    memset(&out[n], 0, sizeof(qcd_kernel_stat));
    snprintf(out[n].name, sizeof out[n].name, "launches_total");
    out[n].launches = (int)g_kernel_launches;
    n++;
  }
  *n_entries = n;
  return QCD_OK;
}

}  // extern "C"

#include "qcd_api_slab.cuh"
