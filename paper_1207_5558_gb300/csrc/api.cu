// libslsht host side: the C ABI of include/slsht.h.
//
// Owns: argument validation, the per-context caches of device tables (Delta,
// d(beta) tables, phase tables, beta weights), scratch workspaces, the chunked
// launch sequence of the forward transform, the inverse, per-stage profiling
// and the continuous-batching request scheduler behind slsht_submit/poll.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/slsht.h"
#include "batch.cuh"
#include "common.cuh"
#include "stages_dev.cuh"
#include "tc.cuh"

// ---------------------------------------------------------------- errors
static std::mutex g_err_mu;
static std::string g_last_err = "no CUDA error recorded";

static void record_cuda_error(const char* what, cudaError_t e) {
  std::lock_guard<std::mutex> g(g_err_mu);
  g_last_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

// Lets other translation units of the library explain their failures through
// slsht_last_error.
void slsht_record_error_text(const char* text) {
  std::lock_guard<std::mutex> g(g_err_mu);
  g_last_err = text;
}

#define CK(call)                                     \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) {                         \
      record_cuda_error(#call, _e);                  \
      return SLSHT_E_CUDA;                           \
    }                                                \
  } while (0)

#define CKS(call)                                    \
  do {                                               \
    int _s = (call);                                 \
    if (_s != SLSHT_OK) return _s;                   \
  } while (0)

// ---------------------------------------------------------------- validation
static int check_desc(const slsht_desc* d) {
  if (!d) return SLSHT_E_ARG;
  if (d->L_f < 1 || d->L_h < 1 || d->L_h > SLSHT_MAX_LH) return SLSHT_E_ARG;
  if (d->L_f > 1 << 15) return SLSHT_E_ARG;
  if (d->n_alpha < 1 || d->n_beta < 1 || d->n_gamma < 1) return SLSHT_E_ARG;
  if (d->n_beta > 65535) return SLSHT_E_ARG;   // beta rows index a grid dimension
  if ((long long)d->n_beta * d->n_gamma > (1LL << 30)) return SLSHT_E_ARG;
  if (d->prec != SLSHT_FP64 && d->prec != SLSHT_FP32_BULK) return SLSHT_E_ARG;
  return SLSHT_OK;
}

static int check_pairs(const slsht_desc* d, const int32_t* lm, int32_t n) {
  if (n < 0) return SLSHT_E_ARG;
  if (n > 0 && !lm) return SLSHT_E_ARG;
  const int lmax = d->L_f + d->L_h - 2;
  for (int32_t i = 0; i < n; ++i) {
    const int l = lm[2 * i], m = lm[2 * i + 1];
    if (l < 0 || l > lmax || m < -l || m > l) return SLSHT_E_ARG;
  }
  return SLSHT_OK;
}

extern "C" int slsht_check_args(const slsht_desc* desc, const int32_t* lm_host, int32_t n_pairs) {
  CKS(check_desc(desc));
  return check_pairs(desc, lm_host, n_pairs);
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------- context
struct TableEntry {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;   // recorded after the generating kernels
};

struct ProfRec {
  int stage;
  cudaEvent_t a, b;
};

struct Workspace {
  // device scratch, grow-only
  void* f = nullptr; size_t f_cap = 0;
  void* h = nullptr; size_t h_cap = 0;
  void* lm = nullptr; size_t lm_cap = 0;
  void* kc = nullptr; size_t kc_cap = 0;
  void* X = nullptr; size_t X_cap = 0;
  void* X2 = nullptr; size_t X2_cap = 0;
  void* C = nullptr; size_t C_cap = 0;
  void* Y = nullptr; size_t Y_cap = 0;
  void* H = nullptr; size_t H_cap = 0;   // rotated window of the call (route 1)
  // Gaunt coefficient table of the last pair list this workspace saw
  void* gt = nullptr; size_t gt_cap = 0;
  void* gtw = nullptr; size_t gtw_cap = 0;   // its work items (pair, mirror pair)
  void* cw = nullptr; size_t cw_cap = 0;     // the 3j-chain coupling's work items (pair, mirror pair)
  std::vector<int32_t> cw_host;
  // real-field calls: the computed pairs, their output slots (host copies kept
  // until the next call: sources of the uploads) and the device slot map
  std::vector<int32_t> rf_lm, rf_slots;
  void* rfs = nullptr; size_t rfs_cap = 0;
  void* ms = nullptr; size_t ms_cap = 0;     // modulated-SHT coupling scratch
  // double-float FP64 engine: scaled k, its exponents, the scaled window, its exponent
  void* kdd = nullptr; size_t kdd_cap = 0;
  void* kexp = nullptr; size_t kexp_cap = 0;
  void* Hdd = nullptr; size_t Hdd_cap = 0;
  void* hexp = nullptr; size_t hexp_cap = 0;
  void* qmask = nullptr; size_t qmask_cap = 0;   // the window's active orders (SLSHT_OPT_WINDOW_ORDERS)
  void* rtw = nullptr; size_t rtw_cap = 0;       // window operand images of the tensor-core rotated window
  std::vector<int32_t> gt_work;              // host copy (source of the upload)
  bool gt_valid = false;
  int gt_Lf = 0, gt_Lh = 0;
  std::vector<int32_t> gt_lm;
  void* stage[2] = {nullptr, nullptr}; size_t stage_cap[2] = {0, 0};
  cudaEvent_t done = nullptr;          // last use of this workspace
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  cudaEvent_t copy_ev[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;  // D2H of host outputs
  cudaStream_t aux = nullptr;          // coupling + beta/gamma of the next chunk
  cudaEvent_t x_ready[2] = {nullptr, nullptr};
  cudaEvent_t x_free[2] = {nullptr, nullptr};
  cudaEvent_t start = nullptr;
  size_t bytes = 0;
};

struct Request {
  uint64_t id = 0;
  slsht_desc desc{};
  std::vector<double> f, h;
  std::vector<int32_t> lm;
  void* g_out = nullptr;
  int n_pairs = 0;
  int next = 0;                        // first pair not yet issued to a tick
  int done = 0;                        // pairs whose tick has completed
  int nt = 0, form = 0, engine = -1;   // alpha tile shape (engine -1: not chosen yet)
  double t_submit = 0, t_admit = -1, t_issue = -1;   // host clock, ms
  double dev_first = 1e300, dev_last = -1e300;       // device clock of its ticks, ms
  int status = SLSHT_OK;
  // its rotated window (once per request, in the context's window pool)
  size_t h_off = 0, h_len = 0;
  bool h_have = false;
  int h_lane = -1;                     // lane of the tick that computes it
  uint64_t h_tick = 0;                 // that lane's tick number
};

// A chunk of consecutive pairs of one request, evaluated in one serving tick.
struct SvChunk {
  Request* r;
  int p0, np;
  bool comp_h;                         // the tick computes the request's rotated window
};

// One serving lane: a stream, a device arena with fixed list regions (the
// addresses the captured graph reads) and a data region, its pinned host
// staging copy, and the graph.  One tick in flight per lane.
struct SvLane {
  cudaStream_t st = nullptr;
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // branches of the captured graph
  cudaEvent_t fork[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  unsigned char* arena = nullptr;
  unsigned char* stage = nullptr;
  bool busy = false;
  uint64_t tick = 0;                   // ticks issued on this lane
  std::vector<SvChunk> chunks;
  double t_assemble = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t g_rot_smem = 0, g_alpha_smem[3] = {0, 0, 0};
};

#define SERVE_LANES 3
#define SERVE_MAX_QUEUE 4096

// Serving arena (per lane): list capacities, sizes of the staged-input and
// device-only data regions, and the tick budget.
#define SV_ITEMS 1024                         // request chunks per tick
static_assert(SV_ITEMS <= SERVE_CPL_MAX, "a tick's coupling index fits its work-item encoding");
#define SV_PAIRS (1 << 17)                    // pairs per tick (coupling lists)
#define SV_RBLK (1 << 18)                     // rotated-window blocks per tick
#define SV_TILES (1 << 20)                    // alpha tiles per tick and precision
#define SV_STAGE_IN ((size_t)64 << 20)        // staged f, h and pair lists per tick
#define SV_DEV_BYTES ((size_t)896 << 20)      // k, H and their double-float forms per tick
#define SV_TICK_SAMPLES (32ll << 20)          // samples per tick (bounds a tick's duration)
#define SV_CHUNK_SAMPLES (8ll << 20)          // first share of one request in a tick
#define SV_HPOOL_BYTES ((size_t)4 << 30)      // rotated windows of the started requests
#define SV_EXPRESS_SAMPLES (4ll << 20)        // requests this small run on the express lane
#define SV_MEDIUM_SAMPLES (64ll << 20)        // bulk lane 1 serves requests up to this size first

// Byte offsets of a serving arena's regions (the same in the pinned stage,
// which mirrors the lists and the staged inputs).
struct SvLayout {
  size_t hdr, cpl, rot, item, cplp[3], kblk, rblk, tiles[3], in, dev, total, stage;
};
static size_t sv_up(size_t n) { return (n + 255) & ~(size_t)255; }
static SvLayout sv_layout() {
  SvLayout L{};
  size_t o = 0;
  L.hdr = o; o += 256;                                   // int counts[8], counters[4]
  L.cpl = o; o += sv_up(sizeof(BCouple) * SV_ITEMS);
  L.rot = o; o += sv_up(sizeof(BRot) * SV_ITEMS);
  L.item = o; o += sv_up(sizeof(BItem) * SV_ITEMS);
  for (int c = 0; c < 3; ++c) { L.cplp[c] = o; o += sv_up(sizeof(int2) * SV_PAIRS); }
  L.kblk = o; o += sv_up(sizeof(BCplBlk) * SV_PAIRS);
  L.rblk = o; o += sv_up(sizeof(BRotBlk) * SV_RBLK);
  for (int c = 0; c < 3; ++c) { L.tiles[c] = o; o += sv_up(sizeof(BTile) * SV_TILES); }
  L.in = o; o += SV_STAGE_IN;
  L.stage = o;
  L.dev = o; o += SV_DEV_BYTES;
  L.total = o;
  return L;
}

struct slsht_batch;

struct slsht_ctx {
  int device = 0;
  size_t budget = 0;
  std::atomic<size_t> used{0};
  std::mutex mu;                       // caches, profile records, counters
  std::mutex sync_mu;                  // serialises users of sync_ws
  std::map<int, TableEntry> delta;                                  // Lh
  std::map<std::tuple<int, int, int>, TableEntry> dtab;             // Lh, Nb, prec
  std::map<std::tuple<int, int>, TableEntry> rtab;                  // Lh, Nb (split-FP16 d images)
  std::map<std::tuple<int, int, int, int>, TableEntry> phase;       // N, R, r0, prec
  std::map<int, TableEntry> wbeta;                                  // Nb
  std::map<std::tuple<int, int>, TableEntry> etab;                  // Na, Lh (tensor-core E blobs)
  // batch-plan autotuner: (prec, Lh, Na, Nb, Ng, engines allowed) -> (columns per tile, alpha form, engine)
  std::map<std::tuple<int, int, int, int, int, int>, std::tuple<int, int, int>> tune;
  std::vector<slsht_batch*> plans;   // live batch plans (freed by slsht_destroy at the latest)
  Workspace sync_ws;
  int opt_beta_route = 0, opt_alpha_engine = 0, opt_gaunt_table = 0, opt_wait_test = 0, opt_real_fields = 0;
  int opt_coupling = 0;
  int opt_fp64_arith = 0;
  int opt_window_orders = 0;
  int opt_rotwin_engine = 0;
  int64_t opt_chunk = 0;
  bool profile = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  uint64_t launches[SLSHT_NSTAGES] = {0};
  double prof_ms[SLSHT_NSTAGES] = {0};
  uint64_t samples = 0;
  int num_sms = 148;
  // serving
  std::mutex smu;
  std::condition_variable scv;
  std::deque<std::unique_ptr<Request>> queue;        // submitted, not started
  std::vector<std::unique_ptr<Request>> active;      // started, not finished (arrival order)
  struct Final { int st; double t[4]; };
  std::map<uint64_t, Final> status;                  // pending (SLSHT_PENDING) or final, per ticket
  SvLane lanes[SERVE_LANES];
  unsigned char* sv_hpool = nullptr;                 // rotated windows of the started requests
  std::map<size_t, size_t> sv_hfree;                 // free blocks of the pool: offset -> length
  cudaEvent_t sv_ref = nullptr;                      // device-clock origin of the serving ticks
  bool sv_ready = false;
  std::thread worker;
  bool stop = false, worker_started = false;
  uint64_t next_id = 1;
  int inflight = 0;                                  // requests in queue or active
  uint64_t sv_ticks = 0, sv_graphs = 0;
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

static int ctx_alloc(slsht_ctx* c, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) return SLSHT_OK;
  size_t cur = c->used.load();
  if (cur + bytes > c->budget) return SLSHT_E_NOMEM;
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    record_cuda_error("cudaMalloc", e);
    return SLSHT_E_NOMEM;
  }
  c->used += bytes;
  return SLSHT_OK;
}

static void ctx_free(slsht_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  c->used -= bytes;
}

// grow-only scratch buffer
static int ws_reserve(slsht_ctx* c, Workspace& w, void** buf, size_t* cap, size_t need) {
  if (need <= *cap) return SLSHT_OK;
  if (*buf) {
    // the previous user of this workspace may still be running
    cudaEventSynchronize(w.done);
    ctx_free(c, *buf, *cap);
    w.bytes -= *cap;
    *buf = nullptr;
    *cap = 0;
  }
  size_t alloc = need + need / 8;
  CKS(ctx_alloc(c, alloc, buf));
  *cap = alloc;
  w.bytes += alloc;
  return SLSHT_OK;
}

static int ws_init(Workspace& w) {
  if (!w.done) {
    CK(cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
    CK(cudaEventRecord(w.done, 0));
    CK(cudaStreamCreateWithFlags(&w.aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&w.start, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) {
      CK(cudaEventCreateWithFlags(&w.x_ready[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&w.x_free[i], cudaEventDisableTiming));
      CK(cudaEventRecord(w.x_free[i], w.aux));
    }
  }
  return SLSHT_OK;
}

static int ws_init_copy(Workspace& w) {
  if (!w.copy_stream) {
    CK(cudaStreamCreateWithFlags(&w.copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CK(cudaEventCreateWithFlags(&w.stage_ev[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&w.copy_ev[i], cudaEventDisableTiming));
      CK(cudaEventRecord(w.copy_ev[i], w.copy_stream));
    }
  }
  return SLSHT_OK;
}

static void ws_release(slsht_ctx* c, Workspace& w) {
  if (w.done) cudaEventSynchronize(w.done);
  if (w.copy_stream) cudaStreamSynchronize(w.copy_stream);
  if (w.aux) cudaStreamSynchronize(w.aux);
  ctx_free(c, w.X2, w.X2_cap);
  for (int i = 0; i < 2; ++i) {
    if (w.x_ready[i]) cudaEventDestroy(w.x_ready[i]);
    if (w.x_free[i]) cudaEventDestroy(w.x_free[i]);
  }
  if (w.start) cudaEventDestroy(w.start);
  if (w.aux) cudaStreamDestroy(w.aux);
  ctx_free(c, w.f, w.f_cap);
  ctx_free(c, w.h, w.h_cap);
  ctx_free(c, w.lm, w.lm_cap);
  ctx_free(c, w.kc, w.kc_cap);
  ctx_free(c, w.X, w.X_cap);
  ctx_free(c, w.C, w.C_cap);
  ctx_free(c, w.Y, w.Y_cap);
  ctx_free(c, w.H, w.H_cap);
  ctx_free(c, w.gt, w.gt_cap);
  ctx_free(c, w.gtw, w.gtw_cap);
  ctx_free(c, w.cw, w.cw_cap);
  ctx_free(c, w.rfs, w.rfs_cap);
  ctx_free(c, w.ms, w.ms_cap);
  ctx_free(c, w.kdd, w.kdd_cap);
  ctx_free(c, w.kexp, w.kexp_cap);
  ctx_free(c, w.Hdd, w.Hdd_cap);
  ctx_free(c, w.hexp, w.hexp_cap);
  ctx_free(c, w.qmask, w.qmask_cap);
  ctx_free(c, w.rtw, w.rtw_cap);
  w.gt_valid = false;
  for (int i = 0; i < 2; ++i) ctx_free(c, w.stage[i], w.stage_cap[i]);
  for (int i = 0; i < 2; ++i) {
    if (w.stage_ev[i]) cudaEventDestroy(w.stage_ev[i]);
    if (w.copy_ev[i]) cudaEventDestroy(w.copy_ev[i]);
  }
  if (w.copy_stream) cudaStreamDestroy(w.copy_stream);
  if (w.done) cudaEventDestroy(w.done);
  w = Workspace();
}

// ---------------------------------------------------------------- profiling
static cudaEvent_t pool_event(slsht_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Brackets one launch with timing events when profiling is on; counts it always.
struct StageTimer {
  slsht_ctx* c;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageTimer(slsht_ctx* c_, int stage_, cudaStream_t st_) : c(c_), stage(stage_), st(st_) {
    std::lock_guard<std::mutex> g(c->mu);
    c->launches[stage]++;
    if (c->profile) {
      a = pool_event(c);
      if (a) cudaEventRecord(a, st);
    }
  }
  ~StageTimer() {
    if (!a) return;
    std::lock_guard<std::mutex> g(c->mu);
    cudaEvent_t b = pool_event(c);
    if (!b) return;
    cudaEventRecord(b, st);
    c->prof.push_back({stage, a, b});
  }
};

#define LAUNCH(stage, st, call)                      \
  do {                                               \
    StageTimer _t(ctx, stage, st);                   \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) {                         \
      record_cuda_error(#call, _e);                  \
      return SLSHT_E_CUDA;                           \
    }                                                \
  } while (0)

// ---------------------------------------------------------------- tables
#define PREC_DD 2   // internal table precision: double-float pairs (batch plans' FP64 engine)

static int make_entry(slsht_ctx* c, TableEntry& e, size_t bytes) {
  CKS(ctx_alloc(c, bytes, &e.ptr));
  e.bytes = bytes;
  CK(cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming));
  return SLSHT_OK;
}

// All table getters run under ctx->mu; they enqueue generation on `st` on a
// miss and make `st` wait for the table in any case.
static int get_delta(slsht_ctx* ctx, int Lh, cudaStream_t st, const double** out) {
  auto it = ctx->delta.find(Lh);
  if (it == ctx->delta.end()) {
    TableEntry e;
    CKS(make_entry(ctx, e, sizeof(double) * (size_t)blk_off(Lh)));
    {
      ctx->launches[SLSHT_STAGE_TABLES]++;
      cudaError_t er = launch_delta((double*)e.ptr, Lh, st);
      if (er != cudaSuccess) { record_cuda_error("launch_delta", er); return SLSHT_E_CUDA; }
    }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->delta.emplace(Lh, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = (const double*)it->second.ptr;
  return SLSHT_OK;
}

static int get_dtab(slsht_ctx* ctx, int Lh, int Nb, int prec, cudaStream_t st, const void** out) {
  auto key = std::make_tuple(Lh, Nb, prec);
  auto it = ctx->dtab.find(key);
  if (it == ctx->dtab.end()) {
    const double* D;
    CKS(get_delta(ctx, Lh, st, &D));
    TableEntry e;
    const size_t el = prec == SLSHT_FP64 ? sizeof(double) : sizeof(float);
    CKS(make_entry(ctx, e, el * (size_t)blk_off(Lh) * Nb));
    ctx->launches[SLSHT_STAGE_TABLES]++;
    cudaError_t er = prec == SLSHT_FP64 ? launch_dtable_f64(D, (double*)e.ptr, Lh, Nb, st)
                                        : launch_dtable_f32(D, (float*)e.ptr, Lh, Nb, st);
    if (er != cudaSuccess) { record_cuda_error("launch_dtable", er); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->dtab.emplace(key, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = it->second.ptr;
  return SLSHT_OK;
}

// Whether the context holds the tensor-core rotated window's d(beta) image of
// (Lh, Nb), or has room for it beside a quarter of its budget left for the
// call's own buffers (the default engine takes the CUDA cores otherwise).
static bool rtab_fits(slsht_ctx* ctx, int Lh, int Nb) {
  std::lock_guard<std::mutex> g(ctx->mu);
  if (ctx->rtab.count(std::make_tuple(Lh, Nb))) return true;
  return ctx->used.load() + rotwin_tc_table_bytes(Lh, Nb) + ctx->budget / 4 <= ctx->budget;
}

// The tensor-core rotated window's split-FP16 d(beta) images (from the FP32
// d table; once per (Lh, Nb)).
static int get_rtab(slsht_ctx* ctx, int Lh, int Nb, cudaStream_t st, const void** out) {
  auto key = std::make_tuple(Lh, Nb);
  auto it = ctx->rtab.find(key);
  if (it == ctx->rtab.end()) {
    const void* dt;
    CKS(get_dtab(ctx, Lh, Nb, SLSHT_FP32_BULK, st, &dt));
    TableEntry e;
    CKS(make_entry(ctx, e, rotwin_tc_table_bytes(Lh, Nb)));
    ctx->launches[SLSHT_STAGE_TABLES]++;
    cudaError_t er = launch_rotwin_tc_table((const float*)dt, Lh, Nb, e.ptr, st);
    if (er != cudaSuccess) { record_cuda_error("launch_rotwin_tc_table", er); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->rtab.emplace(key, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = it->second.ptr;
  return SLSHT_OK;
}

static int get_phase(slsht_ctx* ctx, int N, int R, int r0, int prec, cudaStream_t st, const void** out) {
  auto key = std::make_tuple(N, R, r0, prec);
  auto it = ctx->phase.find(key);
  if (it == ctx->phase.end()) {
    TableEntry e;
    // prec PREC_DD: double-float pairs {cos.h, sin.h, cos.l, sin.l}
    const size_t el = prec == SLSHT_FP32_BULK ? sizeof(float2) : 16;
    CKS(make_entry(ctx, e, el * (size_t)N * R));
    ctx->launches[SLSHT_STAGE_TABLES]++;
    cudaError_t er = prec == SLSHT_FP64 ? launch_phase_f64((double2*)e.ptr, N, R, r0, st)
                     : prec == SLSHT_FP32_BULK ? launch_phase_f32((float2*)e.ptr, N, R, r0, st)
                                               : launch_phase_dd((float4*)e.ptr, N, R, r0, st);
    if (er != cudaSuccess) { record_cuda_error("launch_phase", er); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->phase.emplace(key, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = it->second.ptr;
  return SLSHT_OK;
}

static int get_wbeta(slsht_ctx* ctx, int Nb, cudaStream_t st, const double** out) {
  auto it = ctx->wbeta.find(Nb);
  if (it == ctx->wbeta.end()) {
    TableEntry e;
    CKS(make_entry(ctx, e, sizeof(double) * (size_t)Nb));
    ctx->launches[SLSHT_STAGE_TABLES]++;
    cudaError_t er = launch_beta_weights((double*)e.ptr, Nb, st);
    if (er != cudaSuccess) { record_cuda_error("launch_beta_weights", er); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->wbeta.emplace(Nb, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = (const double*)it->second.ptr;
  return SLSHT_OK;
}

static int get_etab(slsht_ctx* ctx, int Na, int Lh, cudaStream_t st, const void** out) {
  auto key = std::make_tuple(Na, Lh);
  auto it = ctx->etab.find(key);
  if (it == ctx->etab.end()) {
    TableEntry e;
    // narrow windows (L_h <= 16): one K-chunk; wide ones: 2 or 4
    const bool wide = Lh > 16;
    CKS(make_entry(ctx, e, wide ? tcw_etab_bytes(Na, Lh) : tc_etab_bytes(Na, Lh)));
    ctx->launches[SLSHT_STAGE_TABLES]++;
    cudaError_t er = wide ? launch_tcw_etab(e.ptr, Na, Lh, st) : launch_tc_etab(e.ptr, Na, Lh, st);
    if (er != cudaSuccess) { record_cuda_error("launch_tc_etab", er); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->etab.emplace(key, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = it->second.ptr;
  return SLSHT_OK;
}

// The base-256 digit tables of the FP64 tensor-core alpha stage (all |q| <= 15),
// cached per N_alpha beside the FP32 E tables (key (Na, -1)).
static int get_etab64(slsht_ctx* ctx, int Na, cudaStream_t st, const void** out) {
  auto key = std::make_tuple(Na, -1);
  auto it = ctx->etab.find(key);
  if (it == ctx->etab.end()) {
    TableEntry e;
    CKS(make_entry(ctx, e, tc64_etab_bytes(Na)));
    ctx->launches[SLSHT_STAGE_TABLES]++;
    cudaError_t er = launch_tc64_etab(e.ptr, Na, st);
    if (er != cudaSuccess) { record_cuda_error("launch_tc64_etab", er); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(e.ready, st));
    it = ctx->etab.emplace(key, e).first;
  }
  CK(cudaStreamWaitEvent(st, it->second.ready, 0));
  *out = it->second.ptr;
  return SLSHT_OK;
}

// ---------------------------------------------------------------- create/destroy
extern "C" int slsht_create(slsht_ctx** out, int device, size_t budget) {
  if (!out) return SLSHT_E_ARG;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) { record_cuda_error("cudaGetDeviceCount", e); cudaGetLastError(); return SLSHT_E_CUDA; }
  if (device < 0 || device >= n) return SLSHT_E_ARG;
  DeviceGuard g(device);
  CK(cudaFree(0));   // create / bind the primary context
  slsht_ctx* c = new slsht_ctx();
  c->device = device;
  c->budget = budget ? budget : ((size_t)8 << 30);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int s = ws_init(c->sync_ws);
  if (s != SLSHT_OK) { delete c; return s; }
  *out = c;
  return SLSHT_OK;
}

static void free_entry(slsht_ctx* c, TableEntry& e) {
  ctx_free(c, e.ptr, e.bytes);
  if (e.ready) cudaEventDestroy(e.ready);
}

static void batch_free(slsht_batch* b);

extern "C" void slsht_destroy(slsht_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  {
    std::vector<slsht_batch*> plans;
    {
      std::lock_guard<std::mutex> l(c->mu);
      plans.swap(c->plans);
    }
    for (slsht_batch* b : plans) batch_free(b);
  }
  {
    std::unique_lock<std::mutex> l(c->smu);
    c->stop = true;
  }
  c->scv.notify_all();
  if (c->worker.joinable()) c->worker.join();
  for (auto& ln : c->lanes) {
    if (ln.st) cudaStreamSynchronize(ln.st);
    if (ln.exec) cudaGraphExecDestroy(ln.exec);
    if (ln.graph) cudaGraphDestroy(ln.graph);
    if (ln.ev_a) cudaEventDestroy(ln.ev_a);
    if (ln.ev_b) cudaEventDestroy(ln.ev_b);
    for (auto& sd : ln.side)
      if (sd) cudaStreamDestroy(sd);
    for (auto& ev : ln.fork)
      if (ev) cudaEventDestroy(ev);
    if (ln.st) cudaStreamDestroy(ln.st);
    if (ln.stage) cudaFreeHost(ln.stage);
    ctx_free(c, ln.arena, sv_layout().total);
  }
  ctx_free(c, c->sv_hpool, SV_HPOOL_BYTES);
  if (c->sv_ref) cudaEventDestroy(c->sv_ref);
  ws_release(c, c->sync_ws);
  for (auto& kv : c->delta) free_entry(c, kv.second);
  for (auto& kv : c->dtab) free_entry(c, kv.second);
  for (auto& kv : c->rtab) free_entry(c, kv.second);
  for (auto& kv : c->phase) free_entry(c, kv.second);
  for (auto& kv : c->wbeta) free_entry(c, kv.second);
  for (auto& kv : c->etab) free_entry(c, kv.second);
  for (auto& r : c->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

extern "C" int slsht_set_option(slsht_ctx* c, int option, int64_t v) {
  if (!c) return SLSHT_E_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  switch (option) {
    case SLSHT_OPT_BETA_ROUTE:
      if (v < 0 || v > 2) return SLSHT_E_ARG;
      c->opt_beta_route = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_ALPHA_ENGINE:
      if (v < 0 || v > 4) return SLSHT_E_ARG;
      c->opt_alpha_engine = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_CHUNK_PAIRS:
      if (v < 0 || v > (1 << 20)) return SLSHT_E_ARG;
      c->opt_chunk = v;
      return SLSHT_OK;
    case SLSHT_OPT_GAUNT_TABLE:
      if (v < 0 || v > 2) return SLSHT_E_ARG;
      c->opt_gaunt_table = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_WAIT_TEST:
      if (v < 0 || v > 1) return SLSHT_E_ARG;
      c->opt_wait_test = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_REAL_FIELDS:
      if (v < 0 || v > 1) return SLSHT_E_ARG;
      c->opt_real_fields = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_COUPLING:
      if (v < 0 || v > 2) return SLSHT_E_ARG;
      c->opt_coupling = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_FP64_ARITH:
      if (v < 0 || v > 3) return SLSHT_E_ARG;
      c->opt_fp64_arith = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_ROTWIN_ENGINE:
      if (v < 0 || v > 2) return SLSHT_E_ARG;
      c->opt_rotwin_engine = (int)v;
      return SLSHT_OK;
    case SLSHT_OPT_WINDOW_ORDERS:
      if (v < 0 || v > 2) return SLSHT_E_ARG;
      c->opt_window_orders = (int)v;
      return SLSHT_OK;
    default:
      return SLSHT_E_ARG;
  }
}

// ---------------------------------------------------------------- forward
// Copies (or aliases) an input array to device memory of the workspace.
static int stage_input(slsht_ctx* ctx, Workspace& w, void** buf, size_t* cap, const void* src,
                       size_t bytes, cudaStream_t st, const void** dev) {
  if (is_device_ptr(src)) {
    *dev = src;
    return SLSHT_OK;
  }
  CKS(ws_reserve(ctx, w, buf, cap, bytes));
  {
    StageTimer t(ctx, SLSHT_STAGE_COPY, st);
    CK(cudaMemcpyAsync(*buf, src, bytes, cudaMemcpyHostToDevice, st));
  }
  *dev = *buf;
  return SLSHT_OK;
}

static bool use_tensor_cores(slsht_ctx* ctx, const slsht_desc* d) {
  if (d->prec != SLSHT_FP32_BULK) return false;
  if (!tc_supported(d->L_h, d->n_alpha) && !tcw_supported(d->L_h, d->n_alpha)) return false;
  if (ctx->opt_alpha_engine == 1 || ctx->opt_alpha_engine == 4) return false;
  return true;   // default for FP32_BULK when supported
}

// Work items of the Gaunt table: (i, j) with pair j = (l, -m) the mirror of
// pair i = (l, m), m != 0 (one chain fills both), else (i, -1); every pair is
// in exactly one item.
static void mirror_work(const int32_t* lm, int32_t n, std::vector<int32_t>* out) {
  std::map<std::pair<int, int>, std::vector<int32_t>> free_idx;
  for (int32_t i = n - 1; i >= 0; --i) free_idx[{lm[2 * i], lm[2 * i + 1]}].push_back(i);
  std::vector<char> used((size_t)n, 0);
  out->clear();
  for (int32_t i = 0; i < n; ++i) {
    if (used[i]) continue;
    used[i] = 1;
    const int l = lm[2 * i], m = lm[2 * i + 1];
    int32_t j = -1;
    if (m != 0) {
      auto it = free_idx.find({l, -m});
      if (it != free_idx.end()) {
        auto& v = it->second;
        while (!v.empty() && used[v.back()]) v.pop_back();
        if (!v.empty()) { j = v.back(); v.pop_back(); used[j] = 1; }
      }
    }
    out->push_back(i);
    out->push_back(j);
  }
}

static int batch_rule_nt(int kp, int Lh, long long J);

// Columns per tile of the double-float alpha kernel by rule: 32 for at most
// 32 columns, else 64 (two row groups a column), within the shared-memory limit.
static int dd_rule_cols(int Lh, long long J) {
  int nt = J <= 32 ? 32 : 64;
  while (nt > 32 && batch_alpha_smem(2, Lh, nt) > BA_SMEM_LIMIT) nt /= 2;
  return nt;
}

// Pairs a chunk of the wide tensor-core engine (calls, plans, serving): the
// producer reads H from HBM once per group of 16 pairs, and the producer and
// the alpha kernel do not share SMs (the alpha kernel holds a whole SM's
// shared memory), so a chunk's cost is its operand scratch: XW_CHUNK pairs,
// or more when a pair's operand blob is small (up to 256 MB of blobs, 128
// pairs), so that requests of many pairs on small grids do not become
// hundreds of short launches.
#define XW_CHUNK 16
static int xw_chunk_pairs(int Nb, int Ng, int Lh) {
  const size_t per = std::max<size_t>(1, tcw_xblob_bytes(Nb, Ng, Lh));
  return (int)std::max<size_t>(XW_CHUNK, std::min<size_t>(((size_t)256 << 20) / per, 128));
}

// Pairs a chunk of an FP64 tensor-core call or plan item (digit producer +
// alpha kernel).
#define T64_CHUNK 48

// The forward transform on workspace `w` and stream `st` (ctx->mu NOT held).
// slots (device, nullable): per listed pair {output slot, mirror} (see
// launch_alpha_tc); g_out must then be device memory.
static int forward_core(slsht_ctx* ctx, Workspace& w, const slsht_desc* d, const double* f_lm,
                        const double* h_lm, const int32_t* lm, const int32_t* lm_host, int32_t n_pairs,
                        void* g_out, cudaStream_t st, const int2* slots, bool reuse_k) {
  const int Lf = d->L_f, Lh = d->L_h, Na = d->n_alpha, Nb = d->n_beta, Ng = d->n_gamma;
  const int K = 2 * Lh - 1;
  const bool f64 = d->prec == SLSHT_FP64;
  const size_t J = (size_t)Nb * Ng;
  const size_t per_pair_g = (size_t)Na * J * (f64 ? sizeof(double2) : sizeof(float2));
  const bool host_out = !is_device_ptr(g_out);
  CK(cudaStreamWaitEvent(st, w.done, 0));

  int route, tc, engine, gt_opt, wait_test, coupling, fp64_arith, win_orders, rot_engine;
  int64_t chunk_opt;
  int dd_nt = 0, dd_form = -1, tuned_engine = -1;
  int cc_nt = 0, cc_form = -1;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    route = ctx->opt_beta_route ? ctx->opt_beta_route : 1;
    tc = use_tensor_cores(ctx, d) ? 1 : 0;
    engine = ctx->opt_alpha_engine;
    chunk_opt = ctx->opt_chunk;
    gt_opt = ctx->opt_gaunt_table;
    wait_test = ctx->opt_wait_test;
    coupling = ctx->opt_coupling;
    fp64_arith = ctx->opt_fp64_arith;
    win_orders = ctx->opt_window_orders;
    rot_engine = ctx->opt_rotwin_engine;
    // a tile shape the batch-plan tuner measured for this shape, if any
    // (FP64: both arithmetics allowed; FP32: the tensor cores where they apply)
    const int allowed = f64 ? 6 : ((tc_supported(Lh, Na) && Lh <= 16) ? 5 : 4);
    auto tf = ctx->tune.find(std::make_tuple((int)d->prec, Lh, Na, Nb, Ng, allowed));
    if (tf != ctx->tune.end()) {
      tuned_engine = std::get<2>(tf->second);
      if (tuned_engine == 1) {
        dd_nt = std::get<0>(tf->second);
        dd_form = std::get<1>(tf->second);
      } else if (tuned_engine == 0) {
        cc_nt = std::get<0>(tf->second);
        cc_form = std::get<1>(tf->second);
      }
    }
  }
  // rotated-window route on the tensor cores: producer and alpha stage fused
  // into one kernel unless the separate producer kernel was asked for
  // the factoring route's tensor-core producer serves narrow windows only
  if (tc && route == 2 && Lh > 16) tc = 0;
  const bool fused = tc && route == 1 && Lh <= 16 && engine != 2;
  const bool wide = tc && Lh > 16;      // K-chunked two-kernel tensor-core engine
  // CUDA-core alpha stage: split DFT over the alpha index when Na has a small
  // odd factor that saves work (SLSHT_OPT_ALPHA_ENGINE 4 forces the direct sum)
  const bool split = !tc && engine != 4 && alpha_split_factor(Lh, Na) > 0;
  // FP64, rotated-window route: X and the alpha sum in double-float
  // arithmetic (one kernel over (pair, column block) tiles, no X scratch)
  // unless SLSHT_OPT_FP64_ARITH asks for FP64 arithmetic or the tuner found
  // FP64 arithmetic faster for this shape
  // FP64 on the tensor cores (the default, and SLSHT_OPT_FP64_ARITH = 2, for
  // L_h <= 16 unless the alpha engine is held to CUDA cores): X in
  // double-float, the alpha sum from exact base-256 digit products (producer
  // + alpha kernel per chunk of pairs).  Elsewhere double-float (= 3, or the
  // default where the tuner did not find FP64 arithmetic faster).
  const bool t64 = f64 && route == 1 && (fp64_arith == 0 || fp64_arith == 2) && tc64_supported(Lh, Na) &&
                   engine != 1 && engine != 4;
  const bool ddx = f64 && route == 1 && !t64 && (fp64_arith == 3 || (fp64_arith != 1 && tuned_engine != 0));
  if (ddx) {
    if (dd_form < 0 || (engine == 4 && dd_form != 0)) {
      dd_nt = dd_rule_cols(Lh, (long long)J);
      dd_form = engine == 4 ? 0 : alpha_split_factor(Lh, Na);
    }
  }
  // other CUDA-core calls on the rotated-window route: the same tile kernel
  // in the call's own precision (X in shared memory, no X scratch)
  const bool cc1 = !tc && route == 1 && !ddx && !t64;
  if (cc1) {
    if (cc_form < 0 || (engine == 4 && cc_form != 0)) {
      cc_nt = batch_rule_nt(f64 ? 0 : 1, Lh, (long long)J);
      cc_form = engine == 4 ? 0 : alpha_split_factor(Lh, Na);
    }
  }
  // tables
  const double* D = nullptr;
  const void* dt = nullptr;
  const void* csa = nullptr;
  const void* eg = nullptr;
  const void* etab = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    CKS(get_delta(ctx, Lh, st, &D));
    if (route == 1) CKS(get_dtab(ctx, Lh, Nb, d->prec, st, &dt));
    CKS(get_phase(ctx, Ng, K, -(Lh - 1), d->prec, st, &eg));
    if (tc) CKS(get_etab(ctx, Na, Lh, st, &etab));
    else if (t64) CKS(get_etab64(ctx, Na, st, &etab));
    else if (ddx && dd_form > 0) CKS(get_phase(ctx, Na, K, -(Lh - 1), PREC_DD, st, &csa));
    else if (ddx) CKS(get_phase(ctx, Na, Lh, 0, PREC_DD, st, &csa));
    else if (cc1 && cc_form > 0) CKS(get_phase(ctx, Na, K, -(Lh - 1), d->prec, st, &csa));
    else if (cc1) CKS(get_phase(ctx, Na, Lh, 0, d->prec, st, &csa));
    else if (split) CKS(get_phase(ctx, Na, K, -(Lh - 1), d->prec, st, &csa));   // twiddles of the split DFT
    else CKS(get_phase(ctx, Na, Lh, 0, d->prec, st, &csa));
  }
  // inputs
  const void *f_dev, *h_dev, *lm_dev;
  CKS(stage_input(ctx, w, &w.f, &w.f_cap, f_lm, sizeof(double2) * (size_t)Lf * Lf, st, &f_dev));
  CKS(stage_input(ctx, w, &w.h, &w.h_cap, h_lm, sizeof(double2) * (size_t)Lh * Lh, st, &h_dev));
  CKS(stage_input(ctx, w, &w.lm, &w.lm_cap, lm, sizeof(int2) * (size_t)n_pairs, st, &lm_dev));

  // chunking: X scratch of the chunk kept near L2 size
  const size_t x_per_pair = wide  ? tcw_xblob_bytes(Nb, Ng, Lh)
                            : tc  ? tc_xblob_bytes(Nb, Ng, Lh)
                            : t64 ? tc64_xblob_bytes(Nb, Ng)
                                  : (size_t)K * J * (f64 ? sizeof(double2) : sizeof(float2));
  int P;
  if (chunk_opt > 0) {
    P = (int)std::min<int64_t>(chunk_opt, n_pairs);
  } else if (fused || ddx || cc1) {
    P = n_pairs;                 // no X scratch: one launch per call
  } else {
    const size_t target = (size_t)96 << 20;
    P = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_pairs, target / std::max<size_t>(1, x_per_pair)));
    P = std::min(P, 256);
    // the wide engine's producer reads H once per group of 16 pairs, and a
    // chunk is one launch of each of its kernels: xw_chunk_pairs a chunk
    if (wide) P = std::min<int>(n_pairs, xw_chunk_pairs(Nb, Ng, Lh));
    // the FP64 tensor-core kernel is persistent over (pair, tile) items: at
    // least 48 pairs a chunk keep its last wave short (about 20 items a CTA at
    // workload 3's 62 tiles a pair), and on small grids up to 256 MB of digit
    // operands a chunk (fewer launches, each with more items a CTA)
    if (t64)
      P = std::min<int>(n_pairs, (int)std::max<size_t>(T64_CHUNK, std::min<size_t>(((size_t)256 << 20) /
                                                                                     std::max<size_t>(1, x_per_pair),
                                                                                     1024)));
  }
  if (host_out) {
    // staging buffers for the chunk outputs (double-buffered, D2H on the copy stream)
    const size_t stage_limit = (size_t)1 << 30;
    P = (int)std::max<size_t>(1, std::min<size_t>((size_t)P, stage_limit / std::max<size_t>(1, per_pair_g)));
  }
  CKS(ws_reserve(ctx, w, &w.kc, &w.kc_cap, sizeof(double2) * (size_t)n_pairs * Lh * Lh));
  if (!fused && !ddx && !cc1) {
    CKS(ws_reserve(ctx, w, &w.X, &w.X_cap, x_per_pair * (size_t)P));
    CKS(ws_reserve(ctx, w, &w.X2, &w.X2_cap, x_per_pair * (size_t)P));
  }
  const size_t el2 = f64 ? sizeof(double2) : sizeof(float2);
  if (ddx || t64) {
    CKS(ws_reserve(ctx, w, &w.kdd, &w.kdd_cap, sizeof(float4) * (size_t)n_pairs * Lh * Lh));
    CKS(ws_reserve(ctx, w, &w.kexp, &w.kexp_cap, sizeof(int) * (size_t)n_pairs));
    CKS(ws_reserve(ctx, w, &w.Hdd, &w.Hdd_cap, sizeof(float4) * h_elems(J, Lh * Lh)));
    CKS(ws_reserve(ctx, w, &w.hexp, &w.hexp_cap, 16));
  } else if (route == 1) {
    CKS(ws_reserve(ctx, w, &w.H, &w.H_cap, el2 * h_elems(J, Lh * Lh)));
  }
  if (route == 2) {
    CKS(ws_reserve(ctx, w, &w.C, &w.C_cap, sizeof(double2) * (size_t)P * K * K * K));
    CKS(ws_reserve(ctx, w, &w.Y, &w.Y_cap, sizeof(double2) * (size_t)P * Nb * K * K));
  }
  if (host_out) {
    CKS(ws_init_copy(w));
    for (int i = 0; i < 2; ++i) CKS(ws_reserve(ctx, w, &w.stage[i], &w.stage_cap[i], per_pair_g * (size_t)P));
  }

  // Two-stream pipeline: chunk i's coupling and beta/gamma sums run on the
  // workspace's aux stream into X buffer i%2 while the alpha stage of chunk
  // i-1 runs on the caller's stream.
  cudaStream_t ax = w.aux;
  CK(cudaEventRecord(w.start, st));
  CK(cudaStreamWaitEvent(ax, w.start, 0));
  // the coupling of every pair in one launch (one CTA per pair fills the GPU).
  // With the Gaunt table: the 3j part is kept per workspace for its last
  // pair list (signal independent) and only the gather-sum runs per call.
  const size_t gt_bytes = gaunt_table_bytes(Lh, n_pairs);
  const bool use_gt = gt_opt == 1 || (gt_opt == 0 && gt_bytes <= ((size_t)256 << 20));
  if (reuse_k) {
    // k of this signal and pair list is still in w.kc (multi-window calls)
  } else if (coupling == 2) {
    // Appendix A: quadrature of the modulated signal's transform
    int lmax = 0;
    for (int32_t i = 0; i < n_pairs; ++i) lmax = std::max(lmax, (int)lm_host[2 * i]);
    CKS(ws_reserve(ctx, w, &w.ms, &w.ms_cap, msht_scratch_bytes(Lf, Lh, lmax, n_pairs)));
    LAUNCH(SLSHT_STAGE_COUPLE, ax,
           launch_couple_msht((const double2*)f_dev, Lf, Lh, (const int2*)lm_dev, n_pairs, lmax, w.ms,
                              (double2*)w.kc, ax));
  } else if (use_gt) {
    const bool hit = w.gt_valid && w.gt_Lf == Lf && w.gt_Lh == Lh && w.gt_lm.size() == 2 * (size_t)n_pairs &&
                     std::memcmp(w.gt_lm.data(), lm_host, sizeof(int32_t) * 2 * (size_t)n_pairs) == 0;
    if (!hit) {
      w.gt_valid = false;
      CKS(ws_reserve(ctx, w, &w.gt, &w.gt_cap, gt_bytes));
      mirror_work(lm_host, n_pairs, &w.gt_work);
      const int nwork = (int)(w.gt_work.size() / 2);
      CKS(ws_reserve(ctx, w, &w.gtw, &w.gtw_cap, sizeof(int32_t) * w.gt_work.size()));
      CK(cudaMemcpyAsync(w.gtw, w.gt_work.data(), sizeof(int32_t) * w.gt_work.size(), cudaMemcpyHostToDevice, ax));
      LAUNCH(SLSHT_STAGE_COUPLE, ax,
             launch_gaunt_table(Lf, Lh, (const int2*)lm_dev, n_pairs, (const int2*)w.gtw, nwork, w.gt, ax));
      w.gt_Lf = Lf;
      w.gt_Lh = Lh;
      w.gt_lm.assign(lm_host, lm_host + 2 * (size_t)n_pairs);
      w.gt_valid = true;
    }
    LAUNCH(SLSHT_STAGE_COUPLE, ax,
           launch_couple_apply((const double2*)f_dev, Lh, (const int2*)lm_dev, n_pairs, w.gt, (double2*)w.kc, ax));
  } else {
    // 3j chains in the call; a pair and its mirror (l, -m) share theirs
    mirror_work(lm_host, n_pairs, &w.cw_host);
    const int nwork = (int)(w.cw_host.size() / 2);
    CKS(ws_reserve(ctx, w, &w.cw, &w.cw_cap, sizeof(int32_t) * w.cw_host.size()));
    CK(cudaMemcpyAsync(w.cw, w.cw_host.data(), sizeof(int32_t) * w.cw_host.size(), cudaMemcpyHostToDevice, ax));
    LAUNCH(SLSHT_STAGE_COUPLE, ax,
           launch_couple((const double2*)f_dev, Lf, Lh, (const int2*)lm_dev, n_pairs, (double2*)w.kc, ax,
                         (const int2*)w.cw, nwork));
  }
  // route 1: the window rotated to every (beta, gamma) sample, once per call
  // (SLSHT_OPT_WINDOW_ORDERS: over the window's active orders only)
  const uint32_t* qmask = nullptr;
  if (win_orders && (ddx || t64 || route == 1)) {
    CKS(ws_reserve(ctx, w, &w.qmask, &w.qmask_cap, 16));
    // 1: exact zeros; 2: also orders at the rounding level (2^-40 of the
    // largest coefficient for FP32_BULK, 2^-52 for FP64)
    const int rel_exp = win_orders == 1 ? 0 : (f64 ? 52 : 40);
    LAUNCH(SLSHT_STAGE_BETA, ax, launch_order_mask((const double2*)h_dev, Lh, rel_exp, (uint32_t*)w.qmask, ax));
    qmask = (const uint32_t*)w.qmask;
  }
  if (ddx || t64) {
    LAUNCH(SLSHT_STAGE_COUPLE, ax,
           launch_kdd_pairs((const double2*)w.kc, Lh, n_pairs, (float4*)w.kdd, (int*)w.kexp, ax));
    LAUNCH(SLSHT_STAGE_BETA, ax,
           launch_rotwin_dd((const double2*)h_dev, (const double*)dt, (const double2*)eg, Lh, Nb, Ng,
                            (float4*)w.Hdd, (int*)w.hexp, ax, qmask));
  } else if (route == 1) {
    if (f64)
      LAUNCH(SLSHT_STAGE_BETA, ax,
             launch_rotwin_f64((const double2*)h_dev, (const double*)dt, (const double2*)eg, Lh, Nb, Ng,
                               (double2*)w.H, ax, qmask));
    else if ((rot_engine == 2 || (rot_engine == 0 && Lh > 16)) && rotwin_tc_supported(Lh, Ng) &&
             (rot_engine == 2 || rtab_fits(ctx, Lh, Nb))) {
      const void* rtab;
      {
        std::lock_guard<std::mutex> g(ctx->mu);
        CKS(get_rtab(ctx, Lh, Nb, ax, &rtab));
      }
      if (wait_test) {   // SLSHT_OPT_WAIT_TEST: this launch withholds its first d chunk
        tc_arm_wait_test();
        wait_test = 0;
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->opt_wait_test = 0;
      }
      CKS(ws_reserve(ctx, w, &w.rtw, &w.rtw_cap, rotwin_tc_window_bytes(Lh)));
      LAUNCH(SLSHT_STAGE_BETA, ax,
             launch_rotwin_tc_window((const double2*)h_dev, (const float2*)eg, qmask, Lh, Ng, w.rtw, ax));
      LAUNCH(SLSHT_STAGE_BETA, ax,
             launch_rotwin_tc(rtab, w.rtw, Lh, Nb, Ng, (float2*)w.H, ctx->num_sms, ax));
    }
    else
      LAUNCH(SLSHT_STAGE_BETA, ax,
             launch_rotwin_f32((const double2*)h_dev, (const float*)dt, (const float2*)eg, Lh, Nb, Ng,
                               (float2*)w.H, ax, qmask));
  }
  void* Xb[2] = {w.X, w.X2};
  int ci = 0;
  for (int32_t off = 0; off < n_pairs; off += P, ++ci) {
    const int np = std::min<int>(P, n_pairs - off);
    void* X = Xb[ci & 1];
    const double2* kcc = (const double2*)w.kc + (size_t)off * Lh * Lh;
    if (fused || ddx || cc1) {
      // every chunk reads the couplings and H that the aux stream produced once
      if (ci == 0) {
        CK(cudaEventRecord(w.x_ready[0], ax));
        CK(cudaStreamWaitEvent(st, w.x_ready[0], 0));
      }
    } else {
      // ---- producer side (aux stream)
      CK(cudaStreamWaitEvent(ax, w.x_free[ci & 1], 0));
      if (route == 2) {
        LAUNCH(SLSHT_STAGE_CTENSOR, ax,
               launch_ctensor(kcc, (const double2*)h_dev, D, Lh, np, (double2*)w.C, ax));
        LAUNCH(SLSHT_STAGE_CTENSOR, ax, launch_beta_dft((const double2*)w.C, Lh, Nb, np, (double2*)w.Y, ax));
      }
      const double2* Ysrc = route == 2 ? (const double2*)w.Y : nullptr;
      if (route == 1) {
        // (route 1 on CUDA cores forms X inside the alpha tile kernel)
        if (t64)
          LAUNCH(SLSHT_STAGE_BETA, ax,
                 launch_xa64((const float4*)w.kdd + (size_t)off * Lh * Lh, (const int*)w.kexp + off,
                             (const float4*)w.Hdd, (const int*)w.hexp, Lh, Nb, Ng, np, X, ax));
        else if (wide)
          LAUNCH(SLSHT_STAGE_BETA, ax, launch_xaw_from_h(kcc, (const float2*)w.H, Lh, Nb, Ng, np, X, ax));
        else
          LAUNCH(SLSHT_STAGE_BETA, ax, launch_xa_from_h(kcc, (const float2*)w.H, Lh, Nb, Ng, np, X, ax));
      } else if (tc) {
        LAUNCH(SLSHT_STAGE_BETA, ax,
               launch_betagamma_tc(kcc, (const double2*)h_dev, nullptr, Ysrc, (const float2*)eg, Lh, Nb, Ng, np, X, ax));
      } else if (f64) {
        LAUNCH(SLSHT_STAGE_BETA, ax,
               launch_betagamma_f64(kcc, (const double2*)h_dev, nullptr, Ysrc,
                                    (const double2*)eg, Lh, Nb, Ng, np, (double2*)X, ax));
      } else {
        LAUNCH(SLSHT_STAGE_BETA, ax,
               launch_betagamma_f32(kcc, (const double2*)h_dev, nullptr, Ysrc,
                                    (const float2*)eg, Lh, Nb, Ng, np, (float2*)X, ax));
      }
      CK(cudaEventRecord(w.x_ready[ci & 1], ax));
      // ---- consumer side (caller's stream)
      CK(cudaStreamWaitEvent(st, w.x_ready[ci & 1], 0));
    }
    void* gdst;
    if (host_out) {
      CK(cudaStreamWaitEvent(st, w.copy_ev[ci & 1], 0));   // staging buffer free again
      gdst = w.stage[ci & 1];
    } else {
      gdst = slots != nullptr ? g_out : (void*)((char*)g_out + per_pair_g * (size_t)off);
    }
    const int2* sl = slots != nullptr ? slots + off : nullptr;
    if (ddx) {
      BItem item{};
      item.H = w.Hdd;
      item.csa = csa;
      item.g = gdst;
      item.kdd = (const float4*)w.kdd + (size_t)off * Lh * Lh;
      item.kexp = (const int*)w.kexp + off;
      item.hexp = (const int*)w.hexp;
      item.slots = sl;
      item.prec = 2;
      item.Lh = Lh;
      item.Na = Na;
      item.J = (int)J;
      item.nt = dd_nt;
      item.form = dd_form;
      LAUNCH(SLSHT_STAGE_ALPHA, st, launch_alpha_call(item, np, ctx->num_sms, st));
    } else if (cc1) {
      BItem item{};
      item.kc = kcc;
      item.H = w.H;
      item.csa = csa;
      item.g = gdst;
      item.slots = sl;
      item.prec = f64 ? 0 : 1;
      item.Lh = Lh;
      item.Na = Na;
      item.J = (int)J;
      item.nt = cc_nt;
      item.form = cc_form;
      LAUNCH(SLSHT_STAGE_ALPHA, st, launch_alpha_call(item, np, ctx->num_sms, st));
    } else if (fused) {
      LAUNCH(SLSHT_STAGE_ALPHA, st,
             launch_alpha_fused(kcc, (const float2*)w.H, etab, Lh, Na, Nb, Ng, np, (float2*)gdst, ctx->num_sms,
                                ci == 0 ? wait_test : 0, sl, st));
      if (ci == 0 && wait_test) {      // one launch only
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->opt_wait_test = 0;
      }
    } else if (wide || tc || t64) {
      // the separate-producer tensor-core kernels; SLSHT_OPT_WAIT_TEST arms
      // the first launch's withheld operand (thread-local, consumed by it)
      if (ci == 0 && wait_test) {
        tc_arm_wait_test();
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->opt_wait_test = 0;
      }
      if (wide)
        LAUNCH(SLSHT_STAGE_ALPHA, st,
               launch_alpha_tcw(X, etab, Lh, Na, Nb, Ng, np, (float2*)gdst, ctx->num_sms, sl, st));
      else if (tc)
        LAUNCH(SLSHT_STAGE_ALPHA, st,
               launch_alpha_tc(X, etab, Lh, Na, Nb, Ng, np, (float2*)gdst, ctx->num_sms, sl, st));
      else
        LAUNCH(SLSHT_STAGE_ALPHA, st,
               launch_alpha_tc64(X, etab, Lh, Na, Nb, Ng, np, (double2*)gdst, ctx->num_sms, sl, st));
    } else if (f64) {
      LAUNCH(SLSHT_STAGE_ALPHA, st,
             split ? launch_alpha_split_f64((const double2*)X, (const double2*)csa, Lh, Na, (int)J, np,
                                            (double2*)gdst, sl, st)
                   : launch_alpha_f64((const double2*)X, (const double2*)csa, Lh, Na, (int)J, np, (double2*)gdst, sl,
                                      st));
    } else {
      LAUNCH(SLSHT_STAGE_ALPHA, st,
             split ? launch_alpha_split_f32((const float2*)X, (const float2*)csa, Lh, Na, (int)J, np,
                                            (float2*)gdst, sl, st)
                   : launch_alpha_f32((const float2*)X, (const float2*)csa, Lh, Na, (int)J, np, (float2*)gdst, sl,
                                      st));
    }
    if (!fused && !ddx && !cc1) CK(cudaEventRecord(w.x_free[ci & 1], st));
    if (host_out) {
      CK(cudaEventRecord(w.stage_ev[ci & 1], st));
      CK(cudaStreamWaitEvent(w.copy_stream, w.stage_ev[ci & 1], 0));
      {
        StageTimer t(ctx, SLSHT_STAGE_COPY, w.copy_stream);
        CK(cudaMemcpyAsync((char*)g_out + per_pair_g * (size_t)off, gdst, per_pair_g * (size_t)np,
                           cudaMemcpyDeviceToHost, w.copy_stream));
      }
      CK(cudaEventRecord(w.copy_ev[ci & 1], w.copy_stream));
    }
  }
  if (host_out) {
    CK(cudaStreamWaitEvent(st, w.copy_ev[0], 0));
    CK(cudaStreamWaitEvent(st, w.copy_ev[1], 0));
  }
  CK(cudaEventRecord(w.done, st));
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->samples += (uint64_t)n_pairs * (uint64_t)Na * J;
  }
  return SLSHT_OK;
}

// The forward transform with the real-field symmetry when the context's
// option says f and h are real fields (f_{l,-m} = (-1)^m conj f_lm, same for
// h): then g(rho; l, -m) = (-1)^m conj g(rho; l, m) (the integrand of
// Eq. stft_spatial is real apart from conj(Y_l^m), and Y_l^{-m} =
// (-1)^m conj Y_l^m), so of each mirrored pair only (l, m) is computed and the
// alpha stage stores both outputs.  Device outputs only.
static int forward_impl(slsht_ctx* ctx, Workspace& w, const slsht_desc* d, const double* f_lm,
                        const double* h_lm, const int32_t* lm, const int32_t* lm_host, int32_t n_pairs,
                        void* g_out, cudaStream_t st, bool reuse_k = false) {
  int real;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    real = ctx->opt_real_fields;
  }
  if (!real || !is_device_ptr(g_out))
    return forward_core(ctx, w, d, f_lm, h_lm, lm, lm_host, n_pairs, g_out, st, nullptr, reuse_k);
  std::vector<int32_t> pw;
  mirror_work(lm_host, n_pairs, &pw);
  const int32_t nw = (int32_t)(pw.size() / 2);
  if (nw == n_pairs) return forward_core(ctx, w, d, f_lm, h_lm, lm, lm_host, n_pairs, g_out, st, nullptr, reuse_k);
  w.rf_lm.resize(2 * (size_t)nw);
  w.rf_slots.resize(2 * (size_t)nw);
  for (int32_t k = 0; k < nw; ++k) {
    const int32_t i = pw[2 * k], j = pw[2 * k + 1];
    w.rf_lm[2 * k] = lm_host[2 * i];
    w.rf_lm[2 * k + 1] = lm_host[2 * i + 1];
    w.rf_slots[2 * k] = i;
    w.rf_slots[2 * k + 1] = j < 0 ? -1 : 2 * j + (lm_host[2 * i + 1] & 1);
  }
  CK(cudaStreamWaitEvent(st, w.done, 0));
  CKS(ws_reserve(ctx, w, &w.rfs, &w.rfs_cap, sizeof(int32_t) * w.rf_slots.size()));
  CK(cudaMemcpyAsync(w.rfs, w.rf_slots.data(), sizeof(int32_t) * w.rf_slots.size(), cudaMemcpyHostToDevice, st));
  const int s = forward_core(ctx, w, d, f_lm, h_lm, w.rf_lm.data(), w.rf_lm.data(), nw, g_out, st,
                             (const int2*)w.rfs, reuse_k);
  if (s == SLSHT_OK) {
    std::lock_guard<std::mutex> g(ctx->mu);
    const slsht_desc* dd = d;
    ctx->samples += (uint64_t)(n_pairs - nw) * (uint64_t)dd->n_alpha * dd->n_beta * dd->n_gamma;
  }
  return s;
}

extern "C" int slsht_forward(slsht_ctx* ctx, const slsht_desc* desc, const double* f_lm,
                             const double* h_lm, const int32_t* lm, int32_t n_pairs, void* g_out,
                             void* stream) {
  if (!ctx) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  if (n_pairs < 0) return SLSHT_E_ARG;
  if (n_pairs == 0) return SLSHT_OK;
  if (!f_lm || !h_lm || !lm || !g_out) return SLSHT_E_ARG;
  if (((uintptr_t)g_out) & 7) return SLSHT_E_ARG;
  DeviceGuard g(ctx->device);
  // pair validation needs host-visible indices
  std::vector<int32_t> lm_host;
  const int32_t* lmv = lm;
  if (is_device_ptr(lm)) {            // read on the caller's stream, after the work queued there
    lm_host.resize(2 * (size_t)n_pairs);
    CK(cudaMemcpyAsync(lm_host.data(), lm, sizeof(int32_t) * 2 * (size_t)n_pairs, cudaMemcpyDeviceToHost,
                       (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    lmv = lm_host.data();
  }
  CKS(check_pairs(desc, lmv, n_pairs));
  std::lock_guard<std::mutex> serial(ctx->sync_mu);
  return forward_impl(ctx, ctx->sync_ws, desc, f_lm, h_lm, lm, lmv, n_pairs, g_out, (cudaStream_t)stream);
}

extern "C" int slsht_forward_windows(slsht_ctx* ctx, const slsht_desc* desc, const double* f_lm,
                                     int32_t n_windows, const double* h_lms, const int32_t* lm, int32_t n_pairs,
                                     void* g_out, void* stream) {
  if (!ctx) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  if (n_pairs < 0 || n_windows < 0) return SLSHT_E_ARG;
  if (n_pairs == 0 || n_windows == 0) return SLSHT_OK;
  if (!f_lm || !h_lms || !lm || !g_out) return SLSHT_E_ARG;
  if (((uintptr_t)g_out) & 7) return SLSHT_E_ARG;
  DeviceGuard g(ctx->device);
  std::vector<int32_t> lm_host;
  const int32_t* lmv = lm;
  if (is_device_ptr(lm)) {            // read on the caller's stream, after the work queued there
    lm_host.resize(2 * (size_t)n_pairs);
    CK(cudaMemcpyAsync(lm_host.data(), lm, sizeof(int32_t) * 2 * (size_t)n_pairs, cudaMemcpyDeviceToHost,
                       (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    lmv = lm_host.data();
  }
  CKS(check_pairs(desc, lmv, n_pairs));
  const size_t nh = 2 * (size_t)desc->L_h * desc->L_h;                  // doubles per window
  const size_t per_window = (size_t)n_pairs * desc->n_alpha * desc->n_beta * desc->n_gamma *
                            (desc->prec == SLSHT_FP64 ? sizeof(double2) : sizeof(float2));
  std::lock_guard<std::mutex> serial(ctx->sync_mu);
  for (int32_t wi = 0; wi < n_windows; ++wi)
    CKS(forward_impl(ctx, ctx->sync_ws, desc, f_lm, h_lms + nh * wi, lm, lmv, n_pairs,
                     (char*)g_out + per_window * wi, (cudaStream_t)stream, wi > 0));
  return SLSHT_OK;
}

// ---------------------------------------------------------------- window generator
int window_ellipse_run(int L, double theta_c, double a, int n_phi, int n_theta, void* (*alloc)(size_t, void*),
                       void (*release)(void*, size_t, void*), void* actx, cudaStream_t st, std::vector<double>& h,
                       double* lambda_out, char* errbuf, size_t errlen);

static void* win_alloc(size_t bytes, void* c) {
  void* p = nullptr;
  return ctx_alloc((slsht_ctx*)c, bytes, &p) == SLSHT_OK ? p : nullptr;
}
static void win_release(void* p, size_t bytes, void* c) { ctx_free((slsht_ctx*)c, p, bytes); }

extern "C" int slsht_window_ellipse(slsht_ctx* ctx, int32_t L, double theta_c, double a, int32_t n_phi,
                                    int32_t n_theta, double* h_out, double* concentration, void* stream) {
  if (!ctx || !h_out) return SLSHT_E_ARG;
  DeviceGuard g(ctx->device);
  std::lock_guard<std::mutex> serial(ctx->sync_mu);
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> h;
  char err[160] = {0};
  const int s = window_ellipse_run(L, theta_c, a, n_phi, n_theta, win_alloc, win_release, ctx, st, h, concentration,
                                   err, sizeof(err));
  if (s != SLSHT_OK) {
    if (err[0]) slsht_record_error_text(err);
    return s;
  }
  if (is_device_ptr(h_out)) {
    CK(cudaMemcpyAsync(h_out, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::memcpy(h_out, h.data(), sizeof(double) * h.size());
  }
  return SLSHT_OK;
}

// ---------------------------------------------------------------- inverse
extern "C" int slsht_inverse(slsht_ctx* ctx, const slsht_desc* desc, const void* g_in,
                             const double h00[2], const int32_t* lm, int32_t n_pairs, double* f_out,
                             void* stream) {
  if (!ctx) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  if (n_pairs < 0) return SLSHT_E_ARG;
  if (n_pairs == 0) return SLSHT_OK;
  if (!g_in || !h00 || !lm || !f_out) return SLSHT_E_ARG;
  const int Lh = desc->L_h, Na = desc->n_alpha, Nb = desc->n_beta, Ng = desc->n_gamma;
  if (Na < Lh || Nb < Lh || Ng < Lh) return SLSHT_E_ARG;
  if (h00[0] == 0.0 && h00[1] == 0.0) return SLSHT_E_H00;
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(g_in)) return SLSHT_E_ARG;
  std::vector<int32_t> lm_host;
  const int32_t* lmv = lm;
  if (is_device_ptr(lm)) {            // read on the caller's stream, after the work queued there
    lm_host.resize(2 * (size_t)n_pairs);
    CK(cudaMemcpyAsync(lm_host.data(), lm, sizeof(int32_t) * 2 * (size_t)n_pairs, cudaMemcpyDeviceToHost,
                       (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    lmv = lm_host.data();
  }
  CKS(check_pairs(desc, lmv, n_pairs));
  std::lock_guard<std::mutex> serial(ctx->sync_mu);
  Workspace& w = ctx->sync_ws;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamWaitEvent(st, w.done, 0));
  const double* wb;
  {
    std::lock_guard<std::mutex> gl(ctx->mu);
    CKS(get_wbeta(ctx, Nb, st, &wb));
  }
  // CTAs = column blocks x pairs x slabs of alpha rows: slabs only when the
  // first two leave the GPU short of about 16 CTAs per SM
  const int ncb = inverse_col_blocks(Nb, Ng);
  const long long base = (long long)ncb * n_pairs;
  const int want = (int)std::max<long long>(1, (16LL * ctx->num_sms + base - 1) / base);
  const int nslab = std::min(Na, want);
  const size_t nparts = (size_t)n_pairs * nslab * ncb;
  CKS(ws_reserve(ctx, w, &w.kc, &w.kc_cap, sizeof(double2) * (nparts + (size_t)n_pairs)));
  double2* partial = (double2*)w.kc;
  double2* fdev = is_device_ptr(f_out) ? (double2*)f_out : partial + nparts;
  if (desc->prec == SLSHT_FP64) {
    LAUNCH(SLSHT_STAGE_INVERSE, st,
           launch_inverse_f64((const double2*)g_in, wb, Na, Nb, Ng, n_pairs, partial, nslab, st));
  } else {
    LAUNCH(SLSHT_STAGE_INVERSE, st,
           launch_inverse_f32((const float2*)g_in, wb, Na, Nb, Ng, n_pairs, partial, nslab, st));
  }
  // scale = (2 pi/Na)(2 pi/Ng) / (sqrt(16 pi^3) h00)
  const double pi = 3.14159265358979323846;
  const double q = (2.0 * pi / Na) * (2.0 * pi / Ng) / std::sqrt(16.0 * pi * pi * pi);
  const double den = h00[0] * h00[0] + h00[1] * h00[1];
  const double sre = q * h00[0] / den, sim = -q * h00[1] / den;
  LAUNCH(SLSHT_STAGE_INVERSE, st, launch_inverse_final(partial, nslab * ncb, n_pairs, sre, sim, fdev, st));
  if ((void*)fdev != (void*)f_out) {
    StageTimer t(ctx, SLSHT_STAGE_COPY, st);
    CK(cudaMemcpyAsync(f_out, fdev, sizeof(double2) * (size_t)n_pairs, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaEventRecord(w.done, st));
  return SLSHT_OK;
}

// Host copy of a small argument array on the caller's stream (after the
// work queued there) into out; host memory is copied directly.
static int read_arg(const void* src, size_t bytes, cudaStream_t st, void* out) {
  if (is_device_ptr(src)) {
    CK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::memcpy(out, src, bytes);
  }
  return SLSHT_OK;
}

extern "C" int slsht_inverse_alt(slsht_ctx* ctx, const slsht_desc* desc, const void* g_in, const double* h_lm,
                                 const int32_t* lm_in, int32_t n_in, int32_t p, const int32_t* lm_out,
                                 int32_t n_out, double* f_out, void* stream) {
  if (!ctx) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  if (n_in < 0 || n_out < 0) return SLSHT_E_ARG;
  if (n_out == 0) return SLSHT_OK;
  if (!g_in || !h_lm || !lm_in || !lm_out || !f_out || n_in == 0) return SLSHT_E_ARG;
  const int Lf = desc->L_f, Lh = desc->L_h, Na = desc->n_alpha, Nb = desc->n_beta, Ng = desc->n_gamma;
  if (p < 0 || p >= Lh) return SLSHT_E_ARG;
  if (Na < Lh + p || Nb < Lh + p || Ng < Lh + p) return SLSHT_E_ARG;
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(g_in)) return SLSHT_E_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int K = 2 * p + 1;
  std::vector<int32_t> lin(2 * (size_t)n_in), lout(2 * (size_t)n_out);
  std::vector<double> h(2 * (size_t)Lh * Lh);
  CKS(read_arg(lm_in, sizeof(int32_t) * lin.size(), st, lin.data()));
  CKS(read_arg(lm_out, sizeof(int32_t) * lout.size(), st, lout.data()));
  CKS(read_arg(h_lm, sizeof(double) * h.size(), st, h.data()));
  CKS(check_pairs(desc, lin.data(), n_in));
  // the window's degree-p coefficients and energy (the condition replacing h_0^0 != 0)
  std::vector<double2> hp(K);
  double Ep = 0.0;
  for (int q = -p; q <= p; ++q) {
    const size_t i = (size_t)p * p + p + q;
    hp[q + p] = make_double2(h[2 * i], h[2 * i + 1]);
    Ep += h[2 * i] * h[2 * i] + h[2 * i + 1] * h[2 * i + 1];
  }
  if (!(Ep > 0.0)) {
    slsht_record_error_text("slsht_inverse_alt: the window has no energy at degree p");
    return SLSHT_E_H00;
  }
  // every output needs the rows of (L + p, M + q), |q| <= p
  std::map<std::pair<int, int>, int> row;
  for (int32_t i = 0; i < n_in; ++i) row.emplace(std::make_pair(lin[2 * i], lin[2 * i + 1]), i);
  std::vector<int> rows((size_t)n_out * K);
  for (int32_t o = 0; o < n_out; ++o) {
    const int L = lout[2 * o], M = lout[2 * o + 1];
    if (L < 0 || L >= Lf || M < -L || M > L) return SLSHT_E_ARG;
    for (int q = -p; q <= p; ++q) {
      auto it = row.find(std::make_pair(L + p, M + q));
      if (it == row.end()) {
        slsht_record_error_text("slsht_inverse_alt: g lacks a pair (L + p, M + q) that an output needs");
        return SLSHT_E_ARG;
      }
      rows[(size_t)o * K + q + p] = it->second;
    }
  }
  std::lock_guard<std::mutex> serial(ctx->sync_mu);
  Workspace& w = ctx->sync_ws;
  CK(cudaStreamWaitEvent(st, w.done, 0));
  const double *wb, *dt;
  const void *ea, *eg;
  {
    std::lock_guard<std::mutex> gl(ctx->mu);
    CKS(get_wbeta(ctx, Nb, st, &wb));
    const void* d = nullptr;
    CKS(get_dtab(ctx, Lh, Nb, SLSHT_FP64, st, &d));
    dt = (const double*)d;
    CKS(get_phase(ctx, Na, K, -p, desc->prec == SLSHT_FP64 ? SLSHT_FP64 : SLSHT_FP32_BULK, st, &ea));
    CKS(get_phase(ctx, Ng, K, -p, SLSHT_FP64, st, &eg));
  }
  // scratch in the synchronous workspace: partial sums, khat, f (device),
  // then the host-built arrays (window row, outputs, row map)
  const size_t ncb = (size_t)ialt_col_blocks(Nb, Ng);
  const size_t n_part = (size_t)n_in * ncb * K, n_khat = (size_t)n_in * K;
  CKS(ws_reserve(ctx, w, &w.kc, &w.kc_cap, sizeof(double2) * (n_part + n_khat + (size_t)n_out)));
  double2* partial = (double2*)w.kc;
  double2* khat = partial + n_part;
  double2* fdev = is_device_ptr(f_out) ? (double2*)f_out : khat + n_khat;
  const size_t up_bytes = sizeof(double2) * K + sizeof(int32_t) * lout.size() + sizeof(int) * rows.size();
  CKS(ws_reserve(ctx, w, &w.lm, &w.lm_cap, up_bytes));
  double2* hp_d = (double2*)w.lm;
  int2* lout_d = (int2*)(hp_d + K);
  int* rows_d = (int*)(lout_d + n_out);
  {
    StageTimer t(ctx, SLSHT_STAGE_COPY, st);
    CK(cudaMemcpyAsync(hp_d, hp.data(), sizeof(double2) * K, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(lout_d, lout.data(), sizeof(int32_t) * lout.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(rows_d, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, st));
  }
  const double pi = 3.14159265358979323846;
  const double scale = (2.0 * pi / Na) * (2.0 * pi / Ng) * (2.0 * p + 1.0) / (8.0 * pi * pi * Ep);
  LAUNCH(SLSHT_STAGE_INVERSE, st,
         launch_inverse_alt(g_in, desc->prec == SLSHT_FP64 ? 0 : 1, wb, dt, Lh, hp_d, ea, (const double2*)eg, Na, Nb,
                            Ng, p, n_in, partial, scale, khat, lout_d, rows_d, n_out, fdev, st));
  if ((void*)fdev != (void*)f_out) {
    StageTimer t(ctx, SLSHT_STAGE_COPY, st);
    CK(cudaMemcpyAsync(f_out, fdev, sizeof(double2) * (size_t)n_out, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaEventRecord(w.done, st));
  // the host arrays above are read by the stream's copies: wait for them
  CK(cudaStreamSynchronize(st));
  return SLSHT_OK;
}

extern "C" int slsht_steer_gamma(slsht_ctx* ctx, const slsht_desc* desc, const void* g_in, int32_t n_pairs,
                                 const double* gammas, int32_t n_g, int32_t Q, void* g_out, void* stream) {
  if (!ctx) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  if (n_pairs < 0 || n_g < 0) return SLSHT_E_ARG;
  if (n_pairs == 0 || n_g == 0) return SLSHT_OK;
  if (!g_in || !gammas || !g_out) return SLSHT_E_ARG;
  if (Q < 0 || Q >= desc->L_h || desc->n_gamma < 2 * Q + 1) return SLSHT_E_ARG;
  DeviceGuard g(ctx->device);
  if (!is_device_ptr(g_in) || !is_device_ptr(g_out)) return SLSHT_E_ARG;
  std::lock_guard<std::mutex> serial(ctx->sync_mu);
  Workspace& w = ctx->sync_ws;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamWaitEvent(st, w.done, 0));
  const size_t wbytes = sizeof(double) * ((size_t)n_g * desc->n_gamma + (size_t)n_g);
  CKS(ws_reserve(ctx, w, &w.ms, &w.ms_cap, wbytes));
  double* W = (double*)w.ms;
  double* gam = W + (size_t)n_g * desc->n_gamma;
  {
    StageTimer t(ctx, SLSHT_STAGE_COPY, st);
    CK(cudaMemcpyAsync(gam, gammas, sizeof(double) * (size_t)n_g,
                       is_device_ptr(gammas) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  }
  const long long rows = (long long)n_pairs * desc->n_alpha * desc->n_beta;
  LAUNCH(SLSHT_STAGE_OTHER, st,
         launch_steer_gamma(g_in, desc->prec == SLSHT_FP64 ? 0 : 1, rows, desc->n_gamma, gam, n_g, Q, W, g_out, st));
  CK(cudaEventRecord(w.done, st));
  if (!is_device_ptr(gammas)) CK(cudaStreamSynchronize(st));   // the host angles are read by the copy
  return SLSHT_OK;
}

// ---------------------------------------------------------------- batch plans
// A plan binds many analyses (items) and evaluates them with a fixed launch
// sequence: k_batch_couple (k of every distinct (signal, pair list)),
// k_batch_rotwin (every distinct rotated window), one persistent
// k_batch_alpha per precision over the CUDA-core items' tiles, and one fused
// tensor-core launch per item the tuner gave to the tensor cores.  The
// sequence is captured once into a CUDA graph.
struct BatchItemHost {
  slsht_desc d{};
  const double2* f = nullptr;
  const double2* h = nullptr;
  void* g = nullptr;
  int npairs = 0;
  int gaunt = -1, cpl = -1, rot = -1;
  int nt = 0, form = 0, tuned = 0;     // form -1: fused tensor-core kernel
  int engine = 0;                      // 0 CUDA cores in the item's precision, 1 double-float, 2 tensor cores
  const void* etab = nullptr;
  void* xw = nullptr;                  // wide tensor-core items: A-operand scratch of xw_pairs pairs
  int xw_pairs = 0;
};

#define ENG_NATIVE 0
#define ENG_DD 1
#define ENG_TC 2

struct BatchGaunt {
  int Lf = 0, Lh = 0;
  std::vector<int32_t> lm;
  void* lm_dev = nullptr;
  void* table = nullptr;
};

struct slsht_batch {
  slsht_ctx* ctx = nullptr;
  int flags = 0;
  std::mutex mu;
  cudaStream_t cs = nullptr;            // creation, tuning and capture
  cudaEvent_t done = nullptr;           // last launch
  cudaEvent_t ta = nullptr, tb = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<std::pair<void*, size_t>> mem;
  std::vector<BatchItemHost> items;
  std::vector<BatchGaunt> gaunt;
  std::vector<BCouple> cpl;
  std::vector<BCplBlk> cblk;
  std::vector<BRot> rot;
  std::vector<BRotBlk> rblk;
  std::vector<BCplBlk> kblk;            // double-float k: {couple, pair}
  std::vector<BItem> bitem;             // alpha view of every item (index = item)
  std::vector<BTile> tiles[3];          // CUDA-core tiles per kernel (0 FP64, 1 FP32, 2 double-float)
  std::vector<int> tc_items;
  struct RotTc { int rot; const void* tab; void* wbuf; };
  std::vector<RotTc> rot_tc;            // rotated windows on the tensor cores (FP32, wide windows)
  void *d_cpl = nullptr, *d_cblk = nullptr, *d_rot = nullptr, *d_rblk = nullptr, *d_bitem = nullptr;
  void* d_kblk = nullptr;
  void* d_tiles[3] = {nullptr, nullptr, nullptr};
  int* d_counter = nullptr;             // one tile counter per kernel
  size_t rot_smem = 0, alpha_smem[3] = {0, 0, 0};
  int alpha_grid[3] = {0, 0, 0};
  int kernels = 0, k_couple = 0, k_rot = 0, k_alpha = 0;
  uint64_t samples = 0;
  size_t bytes = 0;
};

static int batch_alloc(slsht_batch* b, size_t bytes, void** out) {
  CKS(ctx_alloc(b->ctx, bytes, out));
  b->mem.push_back({*out, bytes});
  b->bytes += bytes;
  return SLSHT_OK;
}

// Device copy of a host array that the plan keeps (stream-ordered on cs).
static int batch_upload(slsht_batch* b, const void* src, size_t bytes, void** dev) {
  *dev = nullptr;
  if (bytes == 0) return SLSHT_OK;
  CKS(batch_alloc(b, bytes, dev));
  CK(cudaMemcpyAsync(*dev, src, bytes, cudaMemcpyHostToDevice, b->cs));
  return SLSHT_OK;
}

static void batch_free(slsht_batch* b) {
  if (!b) return;
  if (b->cs) cudaStreamSynchronize(b->cs);
  if (b->done) cudaEventSynchronize(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& m : b->mem) ctx_free(b->ctx, m.first, m.second);
  if (b->ta) cudaEventDestroy(b->ta);
  if (b->tb) cudaEventDestroy(b->tb);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

static size_t el2_of(int prec) { return prec == SLSHT_FP64 ? sizeof(double2) : sizeof(float2); }

// Alpha-stage arithmetic per sample of a form (multiply-adds), for ordering tiles.
static double alpha_form_cost(int Lh, int form) {
  if (form <= 0) return 4.0 * (Lh - 1) + 2.0;
  return 4.0 * (2 * Lh - 1) / form + form + 3.0;
}

// Columns per tile by rule: the smallest of 32/64/128 covering min(J, 128),
// halved while its X tile exceeds 48 KB (so that four CTAs fit an SM; kp:
// alpha kernel 0 FP64, 1 FP32, 2 double-float).
static int batch_rule_nt(int kp, int Lh, long long J) {
  int nt = J <= 32 ? 32 : (J <= 64 ? 64 : 128);
  while (nt > 32 && batch_alpha_smem(kp, Lh, nt) > (size_t)48 * 1024) nt /= 2;
  return nt;
}

static bool batch_tc_ok(const slsht_batch* b, const slsht_desc& d) {
  if (b->flags & SLSHT_BATCH_NO_TC) return false;
  if (d.prec == SLSHT_FP64)   // exact digit products from the double-float X (needs its k and H)
    return tc64_supported(d.L_h, d.n_alpha) && !(b->flags & (SLSHT_BATCH_NO_DD | SLSHT_BATCH_FP64_DD));
  return (tc_supported(d.L_h, d.n_alpha) && d.L_h <= 16) || tcw_supported(d.L_h, d.n_alpha);
}

// The tensor-core launches of one item, chunk by chunk: the fused kernel
// (L_h <= 16), or the wide engine's producer and alpha kernels; FP64 items:
// the digit producer and the FP64 alpha kernel.
static cudaError_t batch_tc_launch(const slsht_batch* b, const BatchItemHost& it, int npairs, int nb, void* xw,
                                   int xw_pairs, void* g, cudaStream_t st) {
  const slsht_desc& d = it.d;
  if (d.prec == SLSHT_FP64) {
    const BCouple& c = b->cpl[it.cpl];
    const BRot& r = b->rot[it.rot];
    if (c.kdd == nullptr || c.kexp == nullptr || r.Hdd == nullptr || r.hexp == nullptr) return cudaErrorInvalidValue;
    const size_t n2 = (size_t)d.L_h * d.L_h, per_pair = (size_t)d.n_alpha * nb * d.n_gamma;
    for (int off = 0; off < npairs; off += xw_pairs) {
      const int np = std::min(xw_pairs, npairs - off);
      cudaError_t e = launch_xa64(c.kdd + off * n2, c.kexp + off, r.Hdd, r.hexp, d.L_h, nb, d.n_gamma, np, xw, st);
      if (e == cudaSuccess)
        e = launch_alpha_tc64(xw, it.etab, d.L_h, d.n_alpha, nb, d.n_gamma, np, (double2*)g + off * per_pair,
                              b->ctx->num_sms, nullptr, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const double2* kc = b->cpl[it.cpl].kc;
  const float2* H = (const float2*)b->rot[it.rot].H;
  if (d.L_h <= 16)
    return launch_alpha_fused(kc, H, it.etab, d.L_h, d.n_alpha, nb, d.n_gamma, npairs, (float2*)g, b->ctx->num_sms,
                              0, nullptr, st);
  const size_t n2 = (size_t)d.L_h * d.L_h, per_pair = (size_t)d.n_alpha * nb * d.n_gamma;
  for (int off = 0; off < npairs; off += xw_pairs) {
    const int np = std::min(xw_pairs, npairs - off);
    cudaError_t e = launch_xaw_from_h(kc + off * n2, H, d.L_h, nb, d.n_gamma, np, xw, st);
    if (e == cudaSuccess)
      e = launch_alpha_tcw(xw, it.etab, d.L_h, d.n_alpha, nb, d.n_gamma, np, (float2*)g + off * per_pair,
                           b->ctx->num_sms, nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Phase table of the alpha stage for a form: the direct sum's (cos, sin)(2 pi r a / Na)
// or the split DFT's twiddles (cos, sin)(2 pi q t / Na); double-float pairs for
// the double-float engine.
static int batch_alpha_table(slsht_batch* b, const slsht_desc& d, int form, int engine, const void** out) {
  std::lock_guard<std::mutex> g(b->ctx->mu);
  const int prec = engine == ENG_DD ? PREC_DD : d.prec;
  if (form > 0) return get_phase(b->ctx, d.n_alpha, 2 * d.L_h - 1, -(d.L_h - 1), prec, b->cs, out);
  return get_phase(b->ctx, d.n_alpha, d.L_h, 0, prec, b->cs, out);
}

// The alpha view of item ii for a CUDA-core engine (its tables not set).
static BItem batch_item_view(const slsht_batch* b, int ii, int engine) {
  const BatchItemHost& it = b->items[ii];
  BItem bi = b->bitem[ii];
  if (engine == ENG_DD) {
    bi.prec = 2;
    bi.H = b->rot[it.rot].Hdd;
    bi.kdd = b->cpl[it.cpl].kdd;
    bi.kexp = b->cpl[it.cpl].kexp;
    bi.hexp = b->rot[it.rot].hexp;
  } else {
    bi.prec = it.d.prec == SLSHT_FP64 ? 0 : 1;
    bi.H = b->rot[it.rot].H;
  }
  return bi;
}

// Times one candidate on the first pairs of item `ii`, into scratch, as it
// would run in the plan: a CUDA-core tile shape (nt, form, engine) inside a
// persistent launch that other items' tiles keep full (the sample pairs are
// replicated `reps` times to fill the GPU), or the fused tensor-core kernel
// as a launch of its own over the item's pairs (np of them, no
// replication).  Returns device milliseconds per sample in *cost.
static int batch_time_candidate(slsht_batch* b, int ii, int nt, int form, int engine, int np, int reps, int nbs,
                                void* scratch, void* xw, void* d_item, void* d_tiles, int* d_ctr, double* cost) {
  slsht_ctx* ctx = b->ctx;
  const BatchItemHost& it = b->items[ii];
  const slsht_desc& d = it.d;
  // the first nbs beta rows of each sampled pair (the tiled H and the row
  // stride of the scratch output both allow a prefix of the columns)
  const long long J = (long long)nbs * d.n_gamma;
  if (engine == ENG_TC) reps = 1;
  const double samples = (double)np * reps * d.n_alpha * J;
  std::vector<BTile> tl;
  BItem bi{};
  size_t smem = 0;
  int grid = 0;
  if (engine != ENG_TC) {
    bi = batch_item_view(b, ii, engine);
    bi.g = scratch;
    bi.J = (int)J;
    bi.nt = nt;
    bi.form = form;
    CKS(batch_alpha_table(b, d, form, engine, &bi.csa));
    for (int r = 0; r < reps; ++r)
      for (int p = 0; p < np; ++p)
        for (long long j0 = 0; j0 < J; j0 += nt) tl.push_back({0, p, r * np + p, (int)j0});
    CK(cudaMemcpyAsync(d_item, &bi, sizeof(BItem), cudaMemcpyHostToDevice, b->cs));
    CK(cudaMemcpyAsync(d_tiles, tl.data(), sizeof(BTile) * tl.size(), cudaMemcpyHostToDevice, b->cs));
    smem = batch_alpha_smem(bi.prec, d.L_h, nt);
    grid = (int)std::min<long long>((long long)ctx->num_sms * batch_alpha_occupancy(bi.prec, smem),
                                    (long long)tl.size());
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {          // one warm-up, three timed
    CK(cudaMemsetAsync(d_ctr, 0, sizeof(int), b->cs));
    CK(cudaEventRecord(b->ta, b->cs));
    cudaError_t e;
    if (engine != ENG_TC)
      e = launch_batch_alpha(bi.prec, (const BItem*)d_item, (const BTile*)d_tiles, (int)tl.size(), d_ctr, grid, smem,
                             b->cs);
    else
      e = batch_tc_launch(b, it, np * reps, nbs, xw, XW_CHUNK, scratch, b->cs);
    if (e != cudaSuccess) { record_cuda_error("batch tuning launch", e); return SLSHT_E_CUDA; }
    CK(cudaEventRecord(b->tb, b->cs));
    CK(cudaEventSynchronize(b->tb));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, b->ta, b->tb));
    if (rep > 0) best = std::min(best, ms);
  }
  *cost = best / samples;
  return SLSHT_OK;
}

// Engines an item may use under the plan's flags.
static bool batch_dd_ok(const slsht_batch* b, const slsht_desc& d) {
  return d.prec == SLSHT_FP64 && !(b->flags & SLSHT_BATCH_NO_DD);
}
static bool batch_native_ok(const slsht_batch* b, const slsht_desc& d) {
  return !(d.prec == SLSHT_FP64 && (b->flags & SLSHT_BATCH_FP64_DD));
}

// Picks (columns per tile, alpha form, engine) for item ii's shape: the
// context's cache, the rule (SLSHT_BATCH_NO_TUNE), or by timing every candidate.
static int batch_tune(slsht_batch* b, int ii) {
  slsht_ctx* ctx = b->ctx;
  BatchItemHost& it = b->items[ii];
  const slsht_desc& d = it.d;
  const int Lh = d.L_h, Na = d.n_alpha;
  const long long J = (long long)d.n_beta * d.n_gamma;
  const bool tc_ok = batch_tc_ok(b, d), dd_ok = batch_dd_ok(b, d), nat_ok = batch_native_ok(b, d);
  const int allowed = (tc_ok ? 1 : 0) | (dd_ok ? 2 : 0) | (nat_ok ? 4 : 0);
  const auto key = std::make_tuple((int)d.prec, Lh, Na, d.n_beta, d.n_gamma, allowed);
  if (b->flags & SLSHT_BATCH_NO_TUNE) {
    // rule: the tensor cores where they apply; FP64 in double-float arithmetic
    // unless excluded; the split factor of alpha_split_factor
    it.engine = tc_ok ? ENG_TC : (dd_ok ? ENG_DD : ENG_NATIVE);
    it.nt = it.engine == ENG_DD ? dd_rule_cols(Lh, J) : batch_rule_nt(d.prec == SLSHT_FP64 ? 0 : 1, Lh, J);
    it.form = it.engine == ENG_TC ? -1 : alpha_split_factor(Lh, Na);
    it.tuned = 0;
    return SLSHT_OK;
  }
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto f = ctx->tune.find(key);
    if (f != ctx->tune.end()) {
      std::tie(it.nt, it.form, it.engine) = f->second;
      it.tuned = 2;
      return SLSHT_OK;
    }
  }
  // candidates (nt, form, engine)
  std::vector<std::tuple<int, int, int>> cand;
  std::vector<int> forms = {0};
  for (int P : {3, 5, 7, 9})
    if (Na % P == 0) forms.push_back(P);
  std::vector<int> engines;
  if (nat_ok) engines.push_back(ENG_NATIVE);
  if (dd_ok) engines.push_back(ENG_DD);
  for (int eng : engines) {
    const int kp = eng == ENG_DD ? 2 : (d.prec == SLSHT_FP64 ? 0 : 1);
    for (int nt : {32, 64, 128}) {
      if (nt > 32 && J <= nt / 2) continue;               // more than half the tile idle
      if (batch_alpha_smem(kp, Lh, nt) > BA_SMEM_LIMIT) continue;
      for (int fm : forms) cand.push_back(std::make_tuple(nt, fm, eng));
    }
  }
  if (tc_ok) cand.push_back(std::make_tuple(0, -1, ENG_TC));
  if (cand.empty()) return SLSHT_E_ARG;
  // sample: the first pairs (all of them up to 16M samples), replicated so
  // the candidate with the widest tiles still has about eight tiles per SM;
  // at most 16M samples; of a pair larger than that, the first beta rows
  // (whole 128-column tiles, at least eight per SM)
  int nbs = d.n_beta;
  if ((double)Na * J > 1.6e7) {
    const long long cols = std::max<long long>((long long)std::ceil(1.6e7 / Na), 8LL * ctx->num_sms * 128);
    nbs = (int)std::min<long long>(d.n_beta, (cols + d.n_gamma - 1) / d.n_gamma);
  }
  const long long Js = (long long)nbs * d.n_gamma;
  const double per_pair = (double)Na * Js;
  int np = (int)std::max<double>(1.0, std::min<double>(it.npairs, std::floor(1.6e7 / per_pair)));
  const long long tiles_np = (long long)np * ((Js + 127) / 128);
  int reps = (int)std::max<long long>(1, (8LL * ctx->num_sms + tiles_np - 1) / tiles_np);
  reps = (int)std::max<double>(1.0, std::min<double>(reps, std::floor(1.6e7 / (per_pair * np))));
  const size_t out_bytes = (size_t)np * reps * Na * Js * el2_of(d.prec);
  const size_t max_tiles = (size_t)np * reps * ((Js + 31) / 32);
  void *scratch = nullptr, *d_item = nullptr, *d_tiles = nullptr, *d_ctr = nullptr, *xw = nullptr;
  const size_t xw_bytes = !tc_ok                    ? 0
                          : d.prec == SLSHT_FP64    ? tc64_xblob_bytes(nbs, d.n_gamma) * XW_CHUNK
                          : Lh > 16                 ? tcw_xblob_bytes(nbs, d.n_gamma, Lh) * XW_CHUNK
                                                    : 0;
  int st = ctx_alloc(ctx, out_bytes, &scratch);
  if (st == SLSHT_OK && xw_bytes) st = ctx_alloc(ctx, xw_bytes, &xw);
  if (st == SLSHT_OK) st = ctx_alloc(ctx, sizeof(BItem), &d_item);
  if (st == SLSHT_OK) st = ctx_alloc(ctx, sizeof(BTile) * max_tiles, &d_tiles);
  if (st == SLSHT_OK) st = ctx_alloc(ctx, 16, &d_ctr);
  double best = 1e300;
  std::tuple<int, int, int> pick = cand[0];
  for (size_t c = 0; c < cand.size() && st == SLSHT_OK; ++c) {
    double cost = 0.0;
    st = batch_time_candidate(b, ii, std::get<0>(cand[c]), std::get<1>(cand[c]), std::get<2>(cand[c]), np, reps,
                              nbs, scratch, xw, d_item, d_tiles, (int*)d_ctr, &cost);
    if (st == SLSHT_OK && cost < best) { best = cost; pick = cand[c]; }
  }
  cudaStreamSynchronize(b->cs);
  ctx_free(ctx, scratch, out_bytes);
  ctx_free(ctx, xw, xw_bytes);
  ctx_free(ctx, d_item, sizeof(BItem));
  ctx_free(ctx, d_tiles, sizeof(BTile) * max_tiles);
  ctx_free(ctx, d_ctr, 16);
  CKS(st);
  std::tie(it.nt, it.form, it.engine) = pick;
  if (it.engine == ENG_TC) it.nt = batch_rule_nt(1, Lh, J);
  it.tuned = 1;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->tune[key] = std::make_tuple(it.nt, it.form, it.engine);
  return SLSHT_OK;
}

// The launch sequence of a plan on `st` (also what the graph captures).
static int batch_enqueue(slsht_batch* b, cudaStream_t st) {
  slsht_ctx* ctx = b->ctx;
  cudaError_t e;
  CK(cudaMemsetAsync(b->d_counter, 0, 4 * sizeof(int), st));
  e = launch_batch_couple((const BCouple*)b->d_cpl, (const BCplBlk*)b->d_cblk, (int)b->cblk.size(), st);
  if (e != cudaSuccess) { record_cuda_error("launch_batch_couple", e); return SLSHT_E_CUDA; }
  e = launch_batch_kdd((const BCouple*)b->d_cpl, (const BCplBlk*)b->d_kblk, (int)b->kblk.size(), st);
  if (e != cudaSuccess) { record_cuda_error("launch_batch_kdd", e); return SLSHT_E_CUDA; }
  e = launch_batch_rotwin((const BRot*)b->d_rot, (const BRotBlk*)b->d_rblk, (int)b->rblk.size(), b->rot_smem, st);
  if (e != cudaSuccess) { record_cuda_error("launch_batch_rotwin", e); return SLSHT_E_CUDA; }
  for (const auto& rt : b->rot_tc) {
    const BRot& r = b->rot[rt.rot];
    e = launch_rotwin_tc_window(r.h, (const float2*)r.eg, r.qmask, r.Lh, r.Ng, rt.wbuf, st);
    if (e == cudaSuccess) e = launch_rotwin_tc(rt.tab, rt.wbuf, r.Lh, r.Nb, r.Ng, (float2*)r.H, ctx->num_sms, st);
    if (e != cudaSuccess) { record_cuda_error("launch_rotwin_tc", e); return SLSHT_E_CUDA; }
  }
  for (int pi = 0; pi < 3; ++pi) {
    e = launch_batch_alpha(pi, (const BItem*)b->d_bitem, (const BTile*)b->d_tiles[pi], (int)b->tiles[pi].size(),
                           b->d_counter + pi, b->alpha_grid[pi], b->alpha_smem[pi], st);
    if (e != cudaSuccess) { record_cuda_error("launch_batch_alpha", e); return SLSHT_E_CUDA; }
  }
  for (int ii : b->tc_items) {
    const BatchItemHost& it = b->items[ii];
    e = batch_tc_launch(b, it, it.npairs, it.d.n_beta, it.xw, it.xw_pairs, it.g, st);
    if (e != cudaSuccess) { record_cuda_error("batch tensor-core launch", e); return SLSHT_E_CUDA; }
  }
  return SLSHT_OK;
}

static void batch_count(slsht_batch* b) {
  slsht_ctx* ctx = b->ctx;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->launches[SLSHT_STAGE_COUPLE] += b->k_couple;
  ctx->launches[SLSHT_STAGE_BETA] += b->k_rot;
  ctx->launches[SLSHT_STAGE_ALPHA] += b->k_alpha;
  ctx->samples += b->samples;
}

static int batch_build(slsht_batch* b, const slsht_batch_item* src, int32_t n, cudaStream_t ust,
                       std::vector<std::vector<int32_t>>& lms) {
  slsht_ctx* ctx = b->ctx;
  CK(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
  CK(cudaEventCreate(&b->ta));
  CK(cudaEventCreate(&b->tb));
  CK(cudaEventRecord(b->done, ust));             // inputs written on the caller's stream
  CK(cudaStreamWaitEvent(b->cs, b->done, 0));
  b->items.resize(n);
  std::map<std::tuple<int, int, std::vector<int32_t>>, int> gkey;
  std::map<std::pair<const void*, int>, int> ckey;
  std::map<std::tuple<const void*, int, int, int, int>, int> rkey;
  for (int32_t i = 0; i < n; ++i) {
    BatchItemHost& it = b->items[i];
    const slsht_desc& d = src[i].desc;
    it.d = d;
    it.f = (const double2*)src[i].f_lm;
    it.h = (const double2*)src[i].h_lm;
    it.g = src[i].g_out;
    it.npairs = src[i].n_pairs;
    const int Lh = d.L_h, n2 = Lh * Lh, K = 2 * Lh - 1;
    const long long J = (long long)d.n_beta * d.n_gamma;
    b->samples += (uint64_t)it.npairs * d.n_alpha * J;
    // Gaunt table of (L_f, L_h, pair list), signal independent (Sec. III-B)
    auto gk = std::make_tuple(d.L_f, Lh, lms[i]);
    auto gf = gkey.find(gk);
    if (gf == gkey.end()) {
      BatchGaunt bg;
      bg.Lf = d.L_f;
      bg.Lh = Lh;
      bg.lm = lms[i];
      CKS(batch_upload(b, bg.lm.data(), sizeof(int32_t) * bg.lm.size(), &bg.lm_dev));
      std::vector<int32_t> work;
      mirror_work(bg.lm.data(), it.npairs, &work);
      void* wdev = nullptr;
      CKS(batch_upload(b, work.data(), sizeof(int32_t) * work.size(), &wdev));
      CKS(batch_alloc(b, gaunt_table_bytes(Lh, it.npairs), &bg.table));
      cudaError_t e = launch_gaunt_table(d.L_f, Lh, (const int2*)bg.lm_dev, it.npairs, (const int2*)wdev,
                                         (int)(work.size() / 2), bg.table, b->cs);
      if (e != cudaSuccess) { record_cuda_error("launch_gaunt_table", e); return SLSHT_E_CUDA; }
      CK(cudaStreamSynchronize(b->cs));          // `work` leaves scope
      gf = gkey.emplace(gk, (int)b->gaunt.size()).first;
      b->gaunt.push_back(std::move(bg));
    }
    it.gaunt = gf->second;
    // k of (signal, Gaunt table)
    auto ck = std::make_pair((const void*)it.f, it.gaunt);
    auto cf = ckey.find(ck);
    if (cf == ckey.end()) {
      const BatchGaunt& bg = b->gaunt[it.gaunt];
      BCouple c{};
      c.f = it.f;
      c.lm = (const int2*)bg.lm_dev;
      c.coef = (const double*)bg.table;
      c.meta = (const int2*)(c.coef + (size_t)it.npairs * Lh * n2);
      void* kc = nullptr;
      CKS(batch_alloc(b, sizeof(double2) * (size_t)it.npairs * n2, &kc));
      c.kc = (double2*)kc;
      c.Lh = Lh;
      c.npairs = it.npairs;
      const int ci = (int)b->cpl.size();
      for (long long f0 = 0; f0 < (long long)it.npairs * n2; f0 += 256) b->cblk.push_back({ci, (int)f0});
      cf = ckey.emplace(ck, ci).first;
      b->cpl.push_back(c);
    }
    it.cpl = cf->second;
    // rotated window of (h, L_h, grid rows, precision)
    auto rk = std::make_tuple((const void*)it.h, Lh, d.n_beta, d.n_gamma, (int)d.prec);
    auto rf = rkey.find(rk);
    if (rf == rkey.end()) {
      BRot r{};
      r.h = it.h;
      r.prec = d.prec == SLSHT_FP64 ? 0 : 1;
      r.Lh = Lh;
      r.Nb = d.n_beta;
      r.Ng = d.n_gamma;
      {
        std::lock_guard<std::mutex> g(ctx->mu);
        CKS(get_dtab(ctx, Lh, d.n_beta, d.prec, b->cs, &r.dt));
        CKS(get_phase(ctx, d.n_gamma, K, -(Lh - 1), d.prec, b->cs, &r.eg));
      }
      CKS(batch_alloc(b, el2_of(d.prec) * h_elems((size_t)J, n2), &r.H));
      const RotChunks ch = rot_chunks(Lh, d.n_gamma, el2_of(d.prec));
      r.QC = ch.QC; r.CC = ch.CC; r.nq = ch.nq; r.nc = ch.nc;
      b->rot_smem = std::max(b->rot_smem, ch.smem(Lh, el2_of(d.prec)));
      const int ri = (int)b->rot.size();
      for (int bb = 0; bb < d.n_beta; bb += ROTWIN_NB)
        for (int p = 0; p < Lh; ++p)
          for (int z = 0; z < ch.nq * ch.nc; ++z)
            if ((z / ch.nc) * ch.QC < 2 * p + 1) b->rblk.push_back({ri, bb, p, z});
      rf = rkey.emplace(rk, ri).first;
      b->rot.push_back(r);
    }
    it.rot = rf->second;
    if (batch_dd_ok(b, d)) {
      // double-float k and H for the double-float engine
      BCouple& c = b->cpl[it.cpl];
      if (c.kdd == nullptr) {
        void *kd = nullptr, *ke = nullptr;
        CKS(batch_alloc(b, sizeof(float4) * (size_t)it.npairs * n2, &kd));
        CKS(batch_alloc(b, sizeof(int) * (size_t)it.npairs, &ke));
        c.kdd = (float4*)kd;
        c.kexp = (int*)ke;
      }
      BRot& r = b->rot[it.rot];
      if (r.Hdd == nullptr) {
        void *hd = nullptr, *he = nullptr;
        CKS(batch_alloc(b, sizeof(float4) * h_elems((size_t)J, n2), &hd));
        CKS(batch_alloc(b, 16, &he));
        r.Hdd = (float4*)hd;
        r.hexp = (int*)he;
      }
    }
    if (batch_tc_ok(b, d)) {
      std::lock_guard<std::mutex> g(ctx->mu);
      if (d.prec == SLSHT_FP64)
        CKS(get_etab64(ctx, d.n_alpha, b->cs, &it.etab));
      else
        CKS(get_etab(ctx, d.n_alpha, Lh, b->cs, &it.etab));
    }
    BItem bi{};
    bi.kc = b->cpl[it.cpl].kc;
    bi.H = b->rot[it.rot].H;
    bi.g = it.g;
    bi.prec = d.prec == SLSHT_FP64 ? 0 : 1;
    bi.Lh = Lh;
    bi.Na = d.n_alpha;
    bi.J = (int)J;
    b->bitem.push_back(bi);
  }
  // k and H once (every engine's form), for the tuner
  for (int ci = 0; ci < (int)b->cpl.size(); ++ci)
    if (b->cpl[ci].kdd != nullptr)
      for (int p = 0; p < b->cpl[ci].npairs; ++p) b->kblk.push_back({ci, p});
  CKS(batch_upload(b, b->cpl.data(), sizeof(BCouple) * b->cpl.size(), &b->d_cpl));
  CKS(batch_upload(b, b->cblk.data(), sizeof(BCplBlk) * b->cblk.size(), &b->d_cblk));
  CKS(batch_upload(b, b->kblk.data(), sizeof(BCplBlk) * b->kblk.size(), &b->d_kblk));
  CKS(batch_upload(b, b->rot.data(), sizeof(BRot) * b->rot.size(), &b->d_rot));
  CKS(batch_upload(b, b->rblk.data(), sizeof(BRotBlk) * b->rblk.size(), &b->d_rblk));
  {
    cudaError_t e = launch_batch_couple((const BCouple*)b->d_cpl, (const BCplBlk*)b->d_cblk, (int)b->cblk.size(),
                                        b->cs);
    if (e == cudaSuccess)
      e = launch_batch_kdd((const BCouple*)b->d_cpl, (const BCplBlk*)b->d_kblk, (int)b->kblk.size(), b->cs);
    if (e == cudaSuccess)
      e = launch_batch_rotwin((const BRot*)b->d_rot, (const BRotBlk*)b->d_rblk, (int)b->rblk.size(), b->rot_smem,
                              b->cs);
    if (e != cudaSuccess) { record_cuda_error("batch k / H", e); return SLSHT_E_CUDA; }
  }
  // tile shapes and engines
  for (int32_t i = 0; i < n; ++i) {
    BatchItemHost& it = b->items[i];
    CKS(batch_tune(b, i));
    BItem& bi = b->bitem[i];
    if (it.engine != ENG_TC) bi = batch_item_view(b, i, it.engine);
    bi.nt = it.nt;
    bi.form = std::max(it.form, 0);
    if (it.engine != ENG_TC) CKS(batch_alpha_table(b, it.d, it.form, it.engine, &bi.csa));
  }
  // only the forms of k and H that the chosen engines read are produced per launch
  {
    std::vector<char> rot_native(b->rot.size(), 0), rot_dd(b->rot.size(), 0), cpl_dd(b->cpl.size(), 0);
    for (const BatchItemHost& it : b->items) {
      // the double-float engine and the FP64 tensor-core engine read the
      // double-float k and H
      if (it.engine == ENG_DD || (it.engine == ENG_TC && it.d.prec == SLSHT_FP64)) {
        rot_dd[it.rot] = 1;
        cpl_dd[it.cpl] = 1;
      } else {
        rot_native[it.rot] = 1;
      }
    }
    for (size_t r = 0; r < b->rot.size(); ++r) {
      if (!rot_native[r]) b->rot[r].H = nullptr;
      if (!rot_dd[r]) b->rot[r].Hdd = nullptr;
    }
    // wide FP32 windows on the tensor cores (SLSHT_OPT_ROTWIN_ENGINE 0 or 2):
    // their blocks leave the CUDA-core rotated-window launch
    int rot_engine;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      rot_engine = ctx->opt_rotwin_engine;
    }
    std::vector<char> on_tc(b->rot.size(), 0);
    for (size_t r = 0; r < b->rot.size(); ++r) {
      const BRot& br = b->rot[r];
      if (br.prec != 1 || br.H == nullptr || !rotwin_tc_supported(br.Lh, br.Ng)) continue;
      if (!(rot_engine == 2 || (rot_engine == 0 && br.Lh > 16 && rtab_fits(ctx, br.Lh, br.Nb)))) continue;
      slsht_batch::RotTc rt{(int)r, nullptr, nullptr};
      {
        std::lock_guard<std::mutex> g(ctx->mu);
        CKS(get_rtab(ctx, br.Lh, br.Nb, b->cs, &rt.tab));
      }
      CKS(batch_alloc(b, rotwin_tc_window_bytes(br.Lh), &rt.wbuf));
      b->rot_tc.push_back(rt);
      on_tc[r] = 1;
    }
    if (!b->rot_tc.empty()) {
      std::vector<BRotBlk> keep;
      for (const BRotBlk& rb : b->rblk)
        if (!on_tc[rb.rot]) keep.push_back(rb);
      b->rblk.swap(keep);
      if (!b->rblk.empty())
        CK(cudaMemcpyAsync(b->d_rblk, b->rblk.data(), sizeof(BRotBlk) * b->rblk.size(), cudaMemcpyHostToDevice,
                           b->cs));
    }
    b->kblk.clear();
    for (int ci = 0; ci < (int)b->cpl.size(); ++ci)
      if (cpl_dd[ci])
        for (int p = 0; p < b->cpl[ci].npairs; ++p) b->kblk.push_back({ci, p});
    CK(cudaMemcpyAsync(b->d_rot, b->rot.data(), sizeof(BRot) * b->rot.size(), cudaMemcpyHostToDevice, b->cs));
    if (!b->kblk.empty())
      CK(cudaMemcpyAsync(b->d_kblk, b->kblk.data(), sizeof(BCplBlk) * b->kblk.size(), cudaMemcpyHostToDevice, b->cs));
  }
  // tiles, largest first
  for (int pi = 0; pi < 3; ++pi) {
    std::vector<std::pair<double, BTile>> tl;
    for (int32_t i = 0; i < n; ++i) {
      const BatchItemHost& it = b->items[i];
      if (it.engine == ENG_TC) continue;
      if (b->bitem[i].prec != pi) continue;
      const long long J = (long long)it.d.n_beta * it.d.n_gamma;
      const double cost = (double)it.nt * (4.0 * it.d.L_h * it.d.L_h + it.d.n_alpha * alpha_form_cost(it.d.L_h, it.form));
      for (int p = 0; p < it.npairs; ++p)
        for (long long j0 = 0; j0 < J; j0 += it.nt) tl.push_back({cost, BTile{i, p, p, (int)j0}});
      b->alpha_smem[pi] = std::max(b->alpha_smem[pi], batch_alpha_smem(pi, it.d.L_h, it.nt));
    }
    std::stable_sort(tl.begin(), tl.end(), [](const std::pair<double, BTile>& x, const std::pair<double, BTile>& y) {
      return x.first > y.first;
    });
    for (auto& t : tl) b->tiles[pi].push_back(t.second);
    if (!b->tiles[pi].empty()) {
      b->alpha_grid[pi] = (int)std::min<long long>(
          (long long)ctx->num_sms * batch_alpha_occupancy(pi, b->alpha_smem[pi]), (long long)b->tiles[pi].size());
      CKS(batch_upload(b, b->tiles[pi].data(), sizeof(BTile) * b->tiles[pi].size(), &b->d_tiles[pi]));
      b->k_alpha++;
    }
  }
  for (int32_t i = 0; i < n; ++i) {
    BatchItemHost& it = b->items[i];
    if (it.engine != ENG_TC) continue;
    b->tc_items.push_back(i);
    if (it.d.prec == SLSHT_FP64) {   // digit producer + FP64 alpha kernel per chunk of T64_CHUNK pairs
      it.xw_pairs = std::min(it.npairs, T64_CHUNK);
      CKS(batch_alloc(b, tc64_xblob_bytes(it.d.n_beta, it.d.n_gamma) * it.xw_pairs, &it.xw));
      b->k_alpha += 2 * ((it.npairs + it.xw_pairs - 1) / it.xw_pairs);
    } else if (it.d.L_h <= 16) {
      b->k_alpha++;
    } else {   // wide: producer + alpha kernel per chunk of xw_chunk_pairs pairs
      it.xw_pairs = std::min(it.npairs, xw_chunk_pairs(it.d.n_beta, it.d.n_gamma, it.d.L_h));
      CKS(batch_alloc(b, tcw_xblob_bytes(it.d.n_beta, it.d.n_gamma, it.d.L_h) * it.xw_pairs, &it.xw));
      b->k_alpha += 2 * ((it.npairs + it.xw_pairs - 1) / it.xw_pairs);
    }
  }
  CKS(batch_upload(b, b->bitem.data(), sizeof(BItem) * b->bitem.size(), &b->d_bitem));
  void* ctr = nullptr;
  CKS(batch_alloc(b, 16, &ctr));
  b->d_counter = (int*)ctr;
  b->k_couple = (b->cblk.empty() ? 0 : 1) + (b->kblk.empty() ? 0 : 1);
  b->k_rot = (b->rblk.empty() ? 0 : 1) + 2 * (int)b->rot_tc.size();
  b->kernels = b->k_couple + b->k_rot + b->k_alpha;
  // one direct run: every g_out holds its result, and every launch path
  // (attributes, the tensor-core error word) is set up before the capture
  CKS(batch_enqueue(b, b->cs));
  CK(cudaStreamSynchronize(b->cs));
  if (!(b->flags & SLSHT_BATCH_NO_GRAPH)) {
    CK(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    const int s = batch_enqueue(b, b->cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cs, &graph);
    b->graph = graph;
    CKS(s);
    if (e != cudaSuccess) { record_cuda_error("cudaStreamEndCapture", e); return SLSHT_E_CUDA; }
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  CK(cudaEventRecord(b->done, b->cs));
  CK(cudaStreamSynchronize(b->cs));
  return SLSHT_OK;
}

extern "C" int slsht_batch_create(slsht_ctx* ctx, int32_t n_items, const slsht_batch_item* items, int32_t flags,
                                  void* stream, slsht_batch** out) {
  if (!out) return SLSHT_E_ARG;
  *out = nullptr;
  if (!ctx || !items || n_items < 1) return SLSHT_E_ARG;
  if (flags & ~(SLSHT_BATCH_NO_GRAPH | SLSHT_BATCH_NO_TUNE | SLSHT_BATCH_NO_TC | SLSHT_BATCH_NO_DD |
                SLSHT_BATCH_FP64_DD))
    return SLSHT_E_ARG;
  if ((flags & SLSHT_BATCH_NO_DD) && (flags & SLSHT_BATCH_FP64_DD)) return SLSHT_E_ARG;
  DeviceGuard g(ctx->device);
  std::vector<std::vector<int32_t>> lms((size_t)n_items);
  for (int32_t i = 0; i < n_items; ++i) {
    const slsht_batch_item& it = items[i];
    CKS(check_desc(&it.desc));
    if (it.n_pairs < 1 || !it.lm) return SLSHT_E_ARG;
    if (!is_device_ptr(it.f_lm) || !is_device_ptr(it.h_lm) || !is_device_ptr(it.g_out)) return SLSHT_E_ARG;
    if (((uintptr_t)it.g_out) & 15) return SLSHT_E_ARG;
    if ((long long)it.n_pairs * it.desc.L_h * it.desc.L_h > (1LL << 30)) return SLSHT_E_ARG;
    lms[i].resize(2 * (size_t)it.n_pairs);
    if (is_device_ptr(it.lm)) {
      CK(cudaMemcpy(lms[i].data(), it.lm, sizeof(int32_t) * lms[i].size(), cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(lms[i].data(), it.lm, sizeof(int32_t) * lms[i].size());
    }
    CKS(check_pairs(&it.desc, lms[i].data(), it.n_pairs));
  }
  slsht_batch* b = new slsht_batch();
  b->ctx = ctx;
  b->flags = flags;
  const int s = batch_build(b, items, n_items, (cudaStream_t)stream, lms);
  if (s != SLSHT_OK) {
    batch_free(b);
    return s;
  }
  {
    std::lock_guard<std::mutex> l(ctx->mu);
    ctx->plans.push_back(b);
  }
  *out = b;
  return SLSHT_OK;
}

extern "C" int slsht_tune(slsht_ctx* ctx, const slsht_desc* desc) {
  if (!ctx) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  DeviceGuard g(ctx->device);
  // seeded synthetic coefficients: f_lm = (cos(0.7 i), sin(1.3 i)) / (l + 1),
  // h the same at the window's band; pairs (L_f - 1, m) for |m| <= min(l, 7)
  const int Lf = desc->L_f, Lh = desc->L_h;
  std::vector<double> f(2 * (size_t)Lf * Lf), h(2 * (size_t)Lh * Lh);
  for (int l = 0; l < Lf; ++l)
    for (int m = -l; m <= l; ++m) {
      const size_t i = (size_t)l * l + l + m;
      f[2 * i] = std::cos(0.7 * i) / (l + 1);
      f[2 * i + 1] = std::sin(1.3 * i) / (l + 1);
    }
  for (int l = 0; l < Lh; ++l)
    for (int m = -l; m <= l; ++m) {
      const size_t i = (size_t)l * l + l + m;
      h[2 * i] = std::cos(0.9 * i + 0.3) / (l + 1);
      h[2 * i + 1] = std::sin(1.1 * i + 0.2) / (l + 1);
    }
  std::vector<int32_t> lm;
  const int l = Lf - 1;
  for (int m = -std::min(l, 7); m <= std::min(l, 7); ++m) { lm.push_back(l); lm.push_back(m); }
  const int np = (int)(lm.size() / 2);
  const size_t gbytes = (size_t)np * desc->n_alpha * desc->n_beta * desc->n_gamma *
                        (desc->prec == SLSHT_FP64 ? sizeof(double2) : sizeof(float2));
  void *fd = nullptr, *hd = nullptr, *gd = nullptr;
  int st = ctx_alloc(ctx, sizeof(double) * f.size(), &fd);
  if (st == SLSHT_OK) st = ctx_alloc(ctx, sizeof(double) * h.size(), &hd);
  if (st == SLSHT_OK) st = ctx_alloc(ctx, gbytes, &gd);
  if (st == SLSHT_OK && (cudaMemcpy(fd, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(hd, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
    cudaGetLastError();
    st = SLSHT_E_CUDA;
  }
  if (st == SLSHT_OK) {
    slsht_batch_item it{};
    it.desc = *desc;
    it.f_lm = (const double*)fd;
    it.h_lm = (const double*)hd;
    it.lm = lm.data();
    it.n_pairs = np;
    it.g_out = gd;
    slsht_batch* b = nullptr;
    // the per-call CUDA-core engines' shapes (FP64: double-float or FP64
    // arithmetic; the tensor-core FP64 engine has no tile shape to tune)
    const int fl = SLSHT_BATCH_NO_GRAPH | (desc->prec == SLSHT_FP64 ? SLSHT_BATCH_NO_TC : 0);
    st = slsht_batch_create(ctx, 1, &it, fl, nullptr, &b);
    if (st == SLSHT_OK) slsht_batch_destroy(b);
    // FP32_BULK: also the CUDA-core shapes alone (the serving path's engines)
    if (st == SLSHT_OK && desc->prec != SLSHT_FP64) {
      b = nullptr;
      st = slsht_batch_create(ctx, 1, &it, SLSHT_BATCH_NO_GRAPH | SLSHT_BATCH_NO_TC, nullptr, &b);
      if (st == SLSHT_OK) slsht_batch_destroy(b);
    }
  }
  ctx_free(ctx, gd, gbytes);
  ctx_free(ctx, hd, sizeof(double) * h.size());
  ctx_free(ctx, fd, sizeof(double) * f.size());
  return st;
}

extern "C" int slsht_batch_launch(slsht_batch* b, void* stream) {
  if (!b) return SLSHT_E_ARG;
  DeviceGuard g(b->ctx->device);
  std::lock_guard<std::mutex> l(b->mu);
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) {
    CK(cudaGraphLaunch(b->exec, st));
  } else {
    CKS(batch_enqueue(b, st));
  }
  CK(cudaEventRecord(b->done, st));
  batch_count(b);
  return SLSHT_OK;
}

extern "C" int slsht_batch_query(const slsht_batch* b, int32_t item, int32_t what, int64_t* value) {
  if (!b || !value) return SLSHT_E_ARG;
  const bool per_item = what == SLSHT_BQ_TILE_COLS || what == SLSHT_BQ_ALPHA_FORM || what == SLSHT_BQ_TUNED ||
                        what == SLSHT_BQ_ENGINE;
  if (per_item && (item < 0 || item >= (int32_t)b->items.size())) return SLSHT_E_ARG;
  switch (what) {
    case SLSHT_BQ_TILE_COLS: *value = b->items[item].form < 0 ? 0 : b->items[item].nt; return SLSHT_OK;
    case SLSHT_BQ_ALPHA_FORM: *value = b->items[item].form; return SLSHT_OK;
    case SLSHT_BQ_TUNED: *value = b->items[item].tuned; return SLSHT_OK;
    case SLSHT_BQ_ENGINE: *value = b->items[item].engine; return SLSHT_OK;
    case SLSHT_BQ_TILES: *value = (int64_t)(b->tiles[0].size() + b->tiles[1].size() + b->tiles[2].size()); return SLSHT_OK;
    case SLSHT_BQ_KERNELS: *value = b->kernels; return SLSHT_OK;
    case SLSHT_BQ_GRAPH: *value = b->exec ? 1 : 0; return SLSHT_OK;
    case SLSHT_BQ_BYTES: *value = (int64_t)b->bytes; return SLSHT_OK;
    case SLSHT_BQ_SAMPLES: *value = (int64_t)b->samples; return SLSHT_OK;
    default: return SLSHT_E_ARG;
  }
}

extern "C" void slsht_batch_destroy(slsht_batch* b) {
  if (!b) return;
  slsht_ctx* ctx = b->ctx;
  DeviceGuard g(ctx->device);
  {
    std::lock_guard<std::mutex> l(ctx->mu);
    auto it = std::find(ctx->plans.begin(), ctx->plans.end(), b);
    if (it == ctx->plans.end()) return;   // already freed with its context
    ctx->plans.erase(it);
  }
  batch_free(b);
}

// ---------------------------------------------------------------- serving
// Continuous batching on persistent batched kernels under a captured graph.
// A worker thread turns the admitted requests into ticks: each tick takes a
// chunk of pairs from every started request (oldest first, at most
// SV_CHUNK_SAMPLES a request, SV_TICK_SAMPLES a tick) and from new requests
// as space allows, so a large request is spread over several ticks and small
// requests that arrive behind it enter the next tick.  A tick's work lists
// (couplings, rotated windows, alpha tiles) are built on the host in a
// pinned stage, copied into the lane's device arena, and evaluated by one
// replay of the lane's captured graph:
//   k_serve_couple x3 (3j chains by window band), k_batch_kdd, k_batch_rotwin,
//   k_batch_alpha x3 (FP64, FP32, double-float; persistent, tiles from a counter),
// whose launch configurations are fixed and whose work counts are read from
// the arena's header.  The graph is captured again only when a tick needs more
// shared memory than the captured configuration holds.  Two lanes alternate,
// so the host builds one tick while the other runs, and their kernels overlap
// on the device.  Admission is by memory: a chunk joins a tick only while its
// inputs, couplings and rotated window fit the lane's arena.  The alpha tile
// shape of a request's grid shape comes from the context's tuner cache
// (CUDA-core engines), else the built-in rule, so that a request's result does
// not depend on the requests it shares ticks with.
static double sv_now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

static int sv_init(slsht_ctx* c) {
  if (c->sv_ready) return SLSHT_OK;
  const SvLayout L = sv_layout();
  int prio_low = 0, prio_high = 0;
  CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  for (auto& ln : c->lanes) {
    // lane 0 is the express lane (small requests, high priority)
    const int prio = &ln == &c->lanes[0] ? prio_high : prio_low;
    CK(cudaStreamCreateWithPriority(&ln.st, cudaStreamNonBlocking, prio));
    for (auto& sd : ln.side) CK(cudaStreamCreateWithPriority(&sd, cudaStreamNonBlocking, prio));
    for (auto& ev : ln.fork) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventCreate(&ln.ev_a));
    CK(cudaEventCreate(&ln.ev_b));
    void* a = nullptr;
    CKS(ctx_alloc(c, L.total, &a));
    ln.arena = (unsigned char*)a;
    CK(cudaHostAlloc((void**)&ln.stage, L.stage, cudaHostAllocDefault));
  }
  {
    void* hp = nullptr;
    CKS(ctx_alloc(c, SV_HPOOL_BYTES, &hp));
    c->sv_hpool = (unsigned char*)hp;
    c->sv_hfree.clear();
    c->sv_hfree[0] = SV_HPOOL_BYTES;
  }
  CK(cudaEventCreate(&c->sv_ref));
  CK(cudaEventRecord(c->sv_ref, c->lanes[0].st));
  CK(cudaEventSynchronize(c->sv_ref));
  c->sv_ready = true;
  return SLSHT_OK;
}

// Bytes a chunk of np pairs needs in the device-only region, and its staged inputs.
// Whether a request reads the double-float forms of k and H (the
// double-float engine, and the FP64 tensor-core engine's digit producer).
static bool sv_ddform(const Request& r) {
  return r.engine == ENG_DD || (r.engine == ENG_TC && r.desc.prec == SLSHT_FP64);
}
// The tensor-core engines' operand scratch of a chunk of np pairs (the FP64
// digits of up to T64_CHUNK pairs, the wide FP32 engine's operand of up to
// xw_chunk_pairs pairs; none for the fused FP32 kernel).
static size_t sv_xw_bytes(const Request& r, int np) {
  const slsht_desc& d = r.desc;
  if (r.engine != ENG_TC) return 0;
  if (d.prec == SLSHT_FP64) return sv_up(tc64_xblob_bytes(d.n_beta, d.n_gamma) * (size_t)std::min(np, T64_CHUNK));
  if (d.L_h > 16)
    return sv_up(tcw_xblob_bytes(d.n_beta, d.n_gamma, d.L_h) *
                 (size_t)std::min(np, xw_chunk_pairs(d.n_beta, d.n_gamma, d.L_h)));
  return 0;
}
// Bytes of a request's rotated window in the pool (with the double-float
// form's scale exponent).
static size_t sv_h_bytes(const Request& r) {
  const slsht_desc& d = r.desc;
  const size_t n2 = (size_t)d.L_h * d.L_h, J = (size_t)d.n_beta * d.n_gamma;
  return sv_ddform(r) ? sv_up(sizeof(float4) * h_elems(J, (int)n2)) + 256
                      : sv_up(el2_of(d.prec) * h_elems(J, (int)n2));
}
static size_t sv_dev_bytes(const Request& r, int np) {
  const size_t n2 = (size_t)r.desc.L_h * r.desc.L_h;
  size_t b = sv_up(sizeof(double2) * np * n2);
  if (sv_ddform(r)) b += sv_up(sizeof(float4) * np * n2) + sv_up(sizeof(int) * np);
  return b + sv_xw_bytes(r, np);
}
// First-fit allocation from the window pool; false when nothing fits.
static bool sv_halloc(slsht_ctx* c, size_t len, size_t* off) {
  for (auto it = c->sv_hfree.begin(); it != c->sv_hfree.end(); ++it) {
    if (it->second < len) continue;
    *off = it->first;
    const size_t rest = it->second - len;
    const size_t at = it->first + len;
    c->sv_hfree.erase(it);
    if (rest) c->sv_hfree[at] = rest;
    return true;
  }
  return false;
}
static void sv_hrelease(slsht_ctx* c, size_t off, size_t len) {
  auto it = c->sv_hfree.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != c->sv_hfree.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    c->sv_hfree.erase(nx);
  }
  if (it != c->sv_hfree.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      c->sv_hfree.erase(it);
    }
  }
}
static size_t sv_in_bytes(const Request& r, int np) {
  return sv_up(sizeof(double2) * (size_t)r.desc.L_f * r.desc.L_f) + sv_up(sizeof(double2) * (size_t)r.desc.L_h * r.desc.L_h) +
         sv_up(sizeof(int2) * (size_t)np);
}
static long long sv_tiles_per_pair(const Request& r) {
  if (r.engine == ENG_TC) return 0;                  // the tensor-core kernels take no tiles
  const long long J = (long long)r.desc.n_beta * r.desc.n_gamma;
  return (J + r.nt - 1) / r.nt;
}
static int sv_rblk_count(const Request& r) {
  const RotChunks ch = rot_chunks(r.desc.L_h, r.desc.n_gamma, sv_ddform(r) || r.desc.prec == SLSHT_FP64
                                                                 ? sizeof(double2) : sizeof(float2));
  return ((r.desc.n_beta + ROTWIN_NB - 1) / ROTWIN_NB) * r.desc.L_h * ch.nq * ch.nc;
}

// The alpha tile shape of a request: the tuner's cache for its grid shape on
// CUDA cores, else the rule of SLSHT_BATCH_NO_TUNE.
static bool sv_tc_ok(const slsht_desc& d) {
  if (d.prec == SLSHT_FP64) return tc64_supported(d.L_h, d.n_alpha);
  return (tc_supported(d.L_h, d.n_alpha) && d.L_h <= 16) || tcw_supported(d.L_h, d.n_alpha);
}
static void sv_choose(slsht_ctx* c, Request& r) {
  const slsht_desc& d = r.desc;
  const long long J = (long long)d.n_beta * d.n_gamma;
  const bool tc = sv_tc_ok(d);
  // engines allowed: the tensor cores where they apply, double-float and FP64
  // for FP64 requests, FP32 CUDA cores for FP32_BULK (the tuner cache's key)
  const int allowed = (tc ? 1 : 0) | (d.prec == SLSHT_FP64 ? 6 : 4);
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto f = c->tune.find(std::make_tuple((int)d.prec, d.L_h, d.n_alpha, d.n_beta, d.n_gamma, allowed));
    if (f != c->tune.end()) {
      std::tie(r.nt, r.form, r.engine) = f->second;
      return;
    }
  }
  r.engine = tc ? ENG_TC : (d.prec == SLSHT_FP64 ? ENG_DD : ENG_NATIVE);
  r.nt = r.engine == ENG_DD ? dd_rule_cols(d.L_h, J) : batch_rule_nt(1, d.L_h, J);
  r.form = r.engine == ENG_TC ? -1 : alpha_split_factor(d.L_h, d.n_alpha);
}

// The tensor-core launches of one chunk (after the graph's coupling and
// rotated window): the fused FP32 kernel (L_h <= 16), the wide engine's
// producer and alpha kernel per xw_chunk_pairs pairs, or the FP64 digit producer and
// alpha kernel per T64_CHUNK pairs.
struct SvTc {
  const double2* kc;
  const float4* kdd;
  const int* kexp;
  const void* H;
  const int* hexp;
  const void* etab;
  void* xw;
  int prec, Lh, Na, Nb, Ng, np;
  void* g;
};
static cudaError_t sv_tc_launch(slsht_ctx* c, const SvTc& t, cudaStream_t st) {
  const int n2 = t.Lh * t.Lh;
  const size_t per_pair = (size_t)t.Na * t.Nb * t.Ng;
  if (t.prec == SLSHT_FP64) {
    for (int off = 0; off < t.np; off += T64_CHUNK) {
      const int n = std::min(T64_CHUNK, t.np - off);
      cudaError_t e = launch_xa64(t.kdd + (size_t)off * n2, t.kexp + off, (const float4*)t.H, t.hexp, t.Lh, t.Nb,
                                  t.Ng, n, t.xw, st);
      if (e == cudaSuccess)
        e = launch_alpha_tc64(t.xw, t.etab, t.Lh, t.Na, t.Nb, t.Ng, n, (double2*)t.g + per_pair * off, c->num_sms,
                              nullptr, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (t.Lh <= 16)
    return launch_alpha_fused(t.kc, (const float2*)t.H, t.etab, t.Lh, t.Na, t.Nb, t.Ng, t.np, (float2*)t.g,
                              c->num_sms, 0, nullptr, st);
  const int xc = xw_chunk_pairs(t.Nb, t.Ng, t.Lh);
  for (int off = 0; off < t.np; off += xc) {
    const int n = std::min(xc, t.np - off);
    cudaError_t e = launch_xaw_from_h(t.kc + (size_t)off * n2, (const float2*)t.H, t.Lh, t.Nb, t.Ng, n, t.xw, st);
    if (e == cudaSuccess)
      e = launch_alpha_tcw(t.xw, t.etab, t.Lh, t.Na, t.Nb, t.Ng, n, (float2*)t.g + per_pair * off, c->num_sms, nullptr,
                           st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Captures the lane's launch sequence with shared-memory sizes rot_smem and
// alpha_smem[3] (the graph reads the arena's fixed list addresses).
static int sv_capture(slsht_ctx* c, SvLane& ln, size_t rot_smem, const size_t* alpha_smem) {
  // the bulk lanes' persistent kernels leave one block slot per SM free, so
  // that the express lane's blocks start without waiting for them to finish
  const bool express = &ln == &c->lanes[0];
  const SvLayout L = sv_layout();
  unsigned char* A = ln.arena;
  const int* hdr = (const int*)(A + L.hdr);
  int* ctr = (int*)(A + L.hdr) + 8;
  const int sms = c->num_sms;
  int agrid[3];
  // (when at least three fit: below that the slot costs the bulk too much)
  auto keep = [&](int occ) { return express || occ < 3 ? occ : occ - 1; };
  for (int pi = 0; pi < 3; ++pi) agrid[pi] = sms * keep(batch_alpha_occupancy(pi, alpha_smem[pi]));
  const int rgrid = sms * keep(batch_rotwin_occupancy(rot_smem));
  const int cgrid = sms * (express ? 4 : 2);
  if (ln.exec) { cudaGraphExecDestroy(ln.exec); ln.exec = nullptr; }
  if (ln.graph) { cudaGraphDestroy(ln.graph); ln.graph = nullptr; }
  // branches: {couplings, double-float k} || {rotated windows}, then the
  // three alpha kernels side by side (each takes tiles of its own list)
  CK(cudaStreamBeginCapture(ln.st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(ctr, 0, 4 * sizeof(int), ln.st);
  if (e == cudaSuccess) e = cudaEventRecord(ln.fork[0], ln.st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ln.side[0], ln.fork[0], 0);
  if (e == cudaSuccess)
    e = launch_batch_rotwin_n((const BRot*)(A + L.rot), (const BRotBlk*)(A + L.rblk), hdr + 4, rgrid, rot_smem,
                              ln.side[0]);
  for (int cls = 0; cls < 3 && e == cudaSuccess; ++cls)
    e = launch_serve_couple(cls, (const BCouple*)(A + L.cpl), (const int2*)(A + L.cplp[cls]), hdr + cls, cgrid,
                            ln.st);
  if (e == cudaSuccess)
    e = launch_batch_kdd_n((const BCouple*)(A + L.cpl), (const BCplBlk*)(A + L.kblk), hdr + 3, cgrid, ln.st);
  if (e == cudaSuccess) e = cudaEventRecord(ln.fork[1], ln.side[0]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ln.st, ln.fork[1], 0);
  if (e == cudaSuccess) e = cudaEventRecord(ln.fork[0], ln.st);
  for (int pi = 0; pi < 3 && e == cudaSuccess; ++pi) {
    cudaStream_t bs = pi == 0 ? ln.st : ln.side[pi];
    if (pi > 0) e = cudaStreamWaitEvent(bs, ln.fork[0], 0);
    if (e == cudaSuccess)
      e = launch_batch_alpha_n(pi, (const BItem*)(A + L.item), (const BTile*)(A + L.tiles[pi]), hdr + 5 + pi,
                               ctr + pi, agrid[pi], alpha_smem[pi], bs);
    if (e == cudaSuccess && pi > 0) e = cudaEventRecord(ln.fork[1 + pi], bs);
  }
  for (int pi = 1; pi < 3 && e == cudaSuccess; ++pi) e = cudaStreamWaitEvent(ln.st, ln.fork[1 + pi], 0);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(ln.st, &graph);
  ln.graph = graph;
  if (e != cudaSuccess) { record_cuda_error("serving graph launch", e); return SLSHT_E_CUDA; }
  if (e2 != cudaSuccess) { record_cuda_error("cudaStreamEndCapture", e2); return SLSHT_E_CUDA; }
  CK(cudaGraphInstantiate(&ln.exec, ln.graph, 0));
  ln.g_rot_smem = rot_smem;
  for (int pi = 0; pi < 3; ++pi) ln.g_alpha_smem[pi] = alpha_smem[pi];
  c->sv_graphs++;
  return SLSHT_OK;
}

// Builds one tick on a free lane from the started and queued requests
// (c->smu held by the caller, released around the CUDA calls).  Returns the
// number of chunks issued (0: nothing to do), or a negative status.
static int sv_tick(slsht_ctx* c, SvLane& ln, std::unique_lock<std::mutex>& lk) {
  const SvLayout L = sv_layout();
  // requests that may join: started ones first (arrival order), then the queue
  while (!c->queue.empty() && c->active.size() < SV_ITEMS) {
    c->active.push_back(std::move(c->queue.front()));
    c->queue.pop_front();
    sv_choose(c, *c->active.back());
  }
  std::vector<SvChunk> ch;
  long long samples = 0, tiles[3] = {0, 0, 0};
  size_t dev = 0, in = 0;
  int npairs[3] = {0, 0, 0}, nkblk = 0, nrblk = 0;
  const bool express = &ln == &c->lanes[0];
  // bulk lane 1 takes the medium requests first (arrival order among them),
  // then the rest, so a medium request does not wait behind the large ones
  // that lane 2 works through first come first served
  std::vector<Request*> cand;
  cand.reserve(c->active.size());
  const bool medium_first = &ln == &c->lanes[1];
  for (int pass = 0; pass < (medium_first ? 2 : 1); ++pass)
    for (auto& up : c->active) {
      const slsht_desc& d = up->desc;
      const bool medium = (long long)up->n_pairs * d.n_alpha * d.n_beta * d.n_gamma <= SV_MEDIUM_SAMPLES;
      if (!medium_first || medium == (pass == 0)) cand.push_back(up.get());
    }
  for (Request* rp : cand) {
    Request& r = *rp;
    if (r.next >= r.n_pairs) continue;
    if (samples >= SV_TICK_SAMPLES || (int)ch.size() >= SV_ITEMS) break;
    const slsht_desc& d = r.desc;
    const long long spp = (long long)d.n_alpha * d.n_beta * d.n_gamma;
    if (((long long)r.n_pairs * spp <= SV_EXPRESS_SAMPLES) != express) continue;   // the other lanes' request
    // express ticks share among their small requests; bulk ticks serve the
    // oldest request first, as much of it as the tick holds (first come,
    // first served: the large requests are not time-sliced against each other)
    int np = (int)std::min<long long>(r.n_pairs - r.next,
                                      std::max<long long>(1, express ? SV_CHUNK_SAMPLES / spp : SV_TICK_SAMPLES / spp));
    np = (int)std::min<long long>(np, std::max<long long>(1, (SV_TICK_SAMPLES - samples) / spp));
    const int cls = d.L_h <= 16 ? 0 : (d.L_h <= 32 ? 1 : 2);
    const int kp = r.engine == ENG_DD ? 2 : (d.prec == SLSHT_FP64 ? 0 : 1);
    // the request's rotated window lives in the window pool from its first
    // tick to its completion (admission by memory: wait for room)
    if (!r.h_have) {
      const size_t hb = sv_h_bytes(r);
      if (!sv_halloc(c, hb, &r.h_off)) continue;
      r.h_len = hb;
      r.h_have = true;
      r.h_lane = -1;
    }
    const bool comp_h = r.h_lane < 0;
    const int rb = comp_h ? sv_rblk_count(r) : 0;
    const long long tpp = sv_tiles_per_pair(r);
    // the largest np that fits every region and list
    auto fits = [&](int n) {
      return dev + sv_dev_bytes(r, n) <= SV_DEV_BYTES && in + sv_in_bytes(r, n) <= SV_STAGE_IN &&
             npairs[cls] + n <= SV_PAIRS && (!sv_ddform(r) || nkblk + n <= SV_PAIRS) && nrblk + rb <= SV_RBLK &&
             tiles[kp] + tpp * n <= SV_TILES;
    };
    while (np > 0 && !fits(np)) np /= 2;
    if (np == 0) break;
    ch.push_back({&r, r.next, np, comp_h});
    dev += sv_dev_bytes(r, np);
    in += sv_in_bytes(r, np);
    npairs[cls] += np;
    if (sv_ddform(r)) nkblk += np;
    nrblk += rb;
    tiles[kp] += tpp * np;
    samples += spp * np;
    if (r.t_admit < 0) r.t_admit = sv_now_ms();
    r.next += np;
  }
  // a tick with room left grows its chunks (oldest request first) up to
  // the tick's budget: a request alone on the GPU is not held to one share
  for (SvChunk& k : ch) {
    Request& r = *k.r;
    const slsht_desc& d = r.desc;
    const long long spp = (long long)d.n_alpha * d.n_beta * d.n_gamma;
    if (samples >= SV_TICK_SAMPLES || r.next >= r.n_pairs) continue;
    int extra = (int)std::min<long long>(r.n_pairs - r.next, (SV_TICK_SAMPLES - samples) / spp);
    const int cls = d.L_h <= 16 ? 0 : (d.L_h <= 32 ? 1 : 2);
    const int kp = r.engine == ENG_DD ? 2 : (d.prec == SLSHT_FP64 ? 0 : 1);
    const long long tpp = sv_tiles_per_pair(r);
    auto fits = [&](int n) {
      return dev - sv_dev_bytes(r, k.np) + sv_dev_bytes(r, k.np + n) <= SV_DEV_BYTES &&
             in - sv_in_bytes(r, k.np) + sv_in_bytes(r, k.np + n) <= SV_STAGE_IN && npairs[cls] + n <= SV_PAIRS &&
             (!sv_ddform(r) || nkblk + n <= SV_PAIRS) && tiles[kp] + tpp * n <= SV_TILES;
    };
    while (extra > 0 && !fits(extra)) extra /= 2;
    if (extra == 0) continue;
    dev += sv_dev_bytes(r, k.np + extra) - sv_dev_bytes(r, k.np);
    in += sv_in_bytes(r, k.np + extra) - sv_in_bytes(r, k.np);
    npairs[cls] += extra;
    if (sv_ddform(r)) nkblk += extra;
    tiles[kp] += tpp * extra;
    samples += spp * extra;
    k.np += extra;
    r.next += extra;
  }
  if (ch.empty()) return 0;
  const double t0 = sv_now_ms();
  lk.unlock();
  // ---- fill the stage: lists and staged inputs; device addresses in the arena
  unsigned char* S = ln.stage;
  unsigned char* A = ln.arena;
  int* hdr = (int*)(S + L.hdr);
  std::memset(hdr, 0, 64);
  BCouple* cpl = (BCouple*)(S + L.cpl);
  BRot* rot = (BRot*)(S + L.rot);
  BItem* item = (BItem*)(S + L.item);
  int2* cplp[3] = {(int2*)(S + L.cplp[0]), (int2*)(S + L.cplp[1]), (int2*)(S + L.cplp[2])};
  BCplBlk* kblk = (BCplBlk*)(S + L.kblk);
  BRotBlk* rblk = (BRotBlk*)(S + L.rblk);
  BTile* tl[3] = {(BTile*)(S + L.tiles[0]), (BTile*)(S + L.tiles[1]), (BTile*)(S + L.tiles[2])};
  size_t in_off = 0, dev_off = 0;
  size_t rot_smem = ln.g_rot_smem, asmem[3] = {ln.g_alpha_smem[0], ln.g_alpha_smem[1], ln.g_alpha_smem[2]};
  int st = SLSHT_OK;
  const int lane_ix = (int)(&ln - c->lanes);
  const uint64_t tick_no = ln.tick + 1;
  int nrot = 0;
  bool wait_lane[SERVE_LANES] = {false};
  std::vector<SvTc> tcs;
  std::vector<int32_t> mw;                               // a chunk's coupling work items
  CK(cudaEventRecord(ln.ev_a, ln.st));
  // items in decreasing tile cost, so the large tiles start first
  std::vector<int> order(ch.size());
  for (size_t i = 0; i < ch.size(); ++i) order[i] = (int)i;
  auto cost = [&](const SvChunk& k) {
    const slsht_desc& d = k.r->desc;
    return (double)k.r->nt * (4.0 * d.L_h * d.L_h + d.n_alpha * alpha_form_cost(d.L_h, k.r->form));
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(ch[a]) > cost(ch[b]); });
  for (size_t ii = 0; ii < ch.size() && st == SLSHT_OK; ++ii) {
    const SvChunk& k = ch[ii];
    Request& r = *k.r;
    const slsht_desc& d = r.desc;
    const int Lh = d.L_h, n2 = Lh * Lh, K = 2 * Lh - 1, np = k.np;
    const size_t J = (size_t)d.n_beta * d.n_gamma;
    const bool dd = sv_ddform(r);                       // double-float k and H
    const bool tcx = r.engine == ENG_TC;
    const int rprec = (dd || d.prec == SLSHT_FP64) ? SLSHT_FP64 : SLSHT_FP32_BULK;   // rotated window's
    // staged inputs
    const size_t fo = in_off, fb = sizeof(double2) * (size_t)d.L_f * d.L_f;
    std::memcpy(S + L.in + fo, r.f.data(), fb);
    in_off += sv_up(fb);
    const size_t ho = in_off, hb = sizeof(double2) * (size_t)n2;
    std::memcpy(S + L.in + ho, r.h.data(), hb);
    in_off += sv_up(hb);
    const size_t lo = in_off, lb = sizeof(int2) * (size_t)np;
    std::memcpy(S + L.in + lo, r.lm.data() + 2 * (size_t)k.p0, lb);
    in_off += sv_up(lb);
    // device-only data
    auto dalloc = [&](size_t bytes) { unsigned char* p = A + L.dev + dev_off; dev_off += sv_up(bytes); return p; };
    BCouple cc{};
    cc.f = (const double2*)(A + L.in + fo);
    cc.lm = (const int2*)(A + L.in + lo);
    cc.kc = (double2*)dalloc(sizeof(double2) * (size_t)np * n2);
    cc.Lh = Lh;
    cc.npairs = np;
    cc.Lf = d.L_f;
    BRot rr{};
    rr.h = (const double2*)(A + L.in + ho);
    rr.prec = rprec == SLSHT_FP64 ? 0 : 1;
    rr.Lh = Lh;
    rr.Nb = d.n_beta;
    rr.Ng = d.n_gamma;
    const RotChunks rc = rot_chunks(Lh, d.n_gamma, el2_of(rprec));
    rr.QC = rc.QC; rr.CC = rc.CC; rr.nq = rc.nq; rr.nc = rc.nc;
    rot_smem = std::max(rot_smem, rc.smem(Lh, el2_of(rprec)));
    unsigned char* hbase = c->sv_hpool + r.h_off;      // the request's rotated window
    if (dd) {
      cc.kdd = (float4*)dalloc(sizeof(float4) * (size_t)np * n2);
      cc.kexp = (int*)dalloc(sizeof(int) * (size_t)np);
      rr.Hdd = (float4*)hbase;
      rr.hexp = (int*)(hbase + r.h_len - 256);
    } else {
      rr.H = hbase;
    }
    if (!k.comp_h && r.h_lane != lane_ix && c->lanes[r.h_lane].busy && c->lanes[r.h_lane].tick == r.h_tick)
      wait_lane[r.h_lane] = true;                        // computed by a tick still on another lane
    BItem bi{};
    const void* etab = nullptr;
    {
      std::lock_guard<std::mutex> g(c->mu);
      const void *dt = nullptr, *eg = nullptr, *csa = nullptr;
      st = get_dtab(c, Lh, d.n_beta, rprec, ln.st, &dt);
      if (st == SLSHT_OK) st = get_phase(c, d.n_gamma, K, -(Lh - 1), rprec, ln.st, &eg);
      const int aprec = dd ? PREC_DD : d.prec;
      if (st == SLSHT_OK && tcx)
        st = d.prec == SLSHT_FP64 ? get_etab64(c, d.n_alpha, ln.st, &etab) : get_etab(c, d.n_alpha, Lh, ln.st, &etab);
      else if (st == SLSHT_OK)
        st = r.form > 0 ? get_phase(c, d.n_alpha, K, -(Lh - 1), aprec, ln.st, &csa)
                        : get_phase(c, d.n_alpha, Lh, 0, aprec, ln.st, &csa);
      rr.dt = dt;
      rr.eg = eg;
      bi.csa = csa;
    }
    const int idx = (int)ii;
    const int cls = Lh <= 16 ? 0 : (Lh <= 32 ? 1 : 2);
    // the chunk's pairs, a pair and its mirror (l, -m) in one work item
    mirror_work(r.lm.data() + 2 * (size_t)k.p0, np, &mw);
    for (size_t wi = 0; wi < mw.size(); wi += 2)
      cplp[cls][hdr[cls]++] = serve_couple_entry(idx, mw[wi], mw[wi + 1]);
    if (dd)
      for (int pr = 0; pr < np; ++pr) kblk[hdr[3]++] = BCplBlk{idx, pr};
    if (k.comp_h) {                                      // the window, once per request
      const int ri = nrot++;
      rot[ri] = rr;
      for (int bb = 0; bb < d.n_beta; bb += ROTWIN_NB)
        for (int pp = 0; pp < Lh; ++pp)
          for (int z = 0; z < rc.nq * rc.nc; ++z) rblk[hdr[4]++] = BRotBlk{ri, bb, pp, z};
      r.h_lane = lane_ix;
      r.h_tick = tick_no;
    }
    bi.kc = cc.kc;
    bi.H = dd ? (const void*)rr.Hdd : (const void*)rr.H;
    const size_t per_pair_g = (size_t)d.n_alpha * J * el2_of(d.prec);
    bi.g = (unsigned char*)r.g_out + per_pair_g * (size_t)k.p0;
    bi.kdd = cc.kdd;
    bi.kexp = cc.kexp;
    bi.hexp = rr.hexp;
    bi.prec = dd ? 2 : (d.prec == SLSHT_FP64 ? 0 : 1);
    bi.Lh = Lh;
    bi.Na = d.n_alpha;
    bi.J = (int)J;
    bi.nt = r.nt;
    bi.form = std::max(r.form, 0);
    cpl[idx] = cc;
    item[idx] = bi;
    if (tcx) {                       // a tensor-core engine, launched after the graph
      SvTc t{};
      t.kc = cc.kc;
      t.kdd = cc.kdd;
      t.kexp = cc.kexp;
      t.H = dd ? (const void*)rr.Hdd : (const void*)rr.H;
      t.hexp = rr.hexp;
      t.etab = etab;
      t.xw = sv_xw_bytes(r, np) ? (void*)dalloc(sv_xw_bytes(r, np)) : nullptr;
      t.prec = d.prec;
      t.Lh = Lh;
      t.Na = d.n_alpha;
      t.Nb = d.n_beta;
      t.Ng = d.n_gamma;
      t.np = np;
      t.g = bi.g;
      tcs.push_back(t);
    } else {
      asmem[bi.prec] = std::max(asmem[bi.prec], batch_alpha_smem(bi.prec, Lh, r.nt));
    }
  }
  for (int oi : order) {          // tiles in decreasing cost
    const SvChunk& k = ch[oi];
    if (k.r->engine == ENG_TC) continue;
    const BItem& bi = item[oi];
    for (int pr = 0; pr < k.np; ++pr)
      for (int j0 = 0; j0 < bi.J; j0 += bi.nt) tl[bi.prec][hdr[5 + bi.prec]++] = BTile{oi, pr, pr, j0};
  }
  // the graph's launch configuration must hold this tick's shared memory
  if (st == SLSHT_OK && (!ln.exec || rot_smem > ln.g_rot_smem || asmem[0] > ln.g_alpha_smem[0] ||
                         asmem[1] > ln.g_alpha_smem[1] || asmem[2] > ln.g_alpha_smem[2])) {
    for (int pi = 0; pi < 3; ++pi)
      if (asmem[pi] == 0) asmem[pi] = batch_alpha_smem(pi, 1, 32);
    if (rot_smem == 0) rot_smem = rot_chunks(1, 1, sizeof(double2)).smem(1, sizeof(double2));
    st = sv_capture(c, ln, rot_smem, asmem);
  }
  // copies of the used parts of the stage, then the graph
  auto put = [&](size_t off, size_t bytes) -> int {
    if (bytes == 0) return SLSHT_OK;
    CK(cudaMemcpyAsync(A + off, S + off, bytes, cudaMemcpyHostToDevice, ln.st));
    return SLSHT_OK;
  };
  const int n = (int)ch.size();
  if (st == SLSHT_OK) st = put(L.hdr, 64);
  if (st == SLSHT_OK) st = put(L.cpl, sizeof(BCouple) * n);
  if (st == SLSHT_OK) st = put(L.rot, sizeof(BRot) * nrot);
  for (int li = 0; li < SERVE_LANES && st == SLSHT_OK; ++li)
    if (wait_lane[li] && cudaStreamWaitEvent(ln.st, c->lanes[li].ev_b, 0) != cudaSuccess) st = SLSHT_E_CUDA;
  if (st == SLSHT_OK) st = put(L.item, sizeof(BItem) * n);
  for (int cl = 0; cl < 3 && st == SLSHT_OK; ++cl) st = put(L.cplp[cl], sizeof(int2) * hdr[cl]);
  if (st == SLSHT_OK) st = put(L.kblk, sizeof(BCplBlk) * hdr[3]);
  if (st == SLSHT_OK) st = put(L.rblk, sizeof(BRotBlk) * hdr[4]);
  for (int pi = 0; pi < 3 && st == SLSHT_OK; ++pi) st = put(L.tiles[pi], sizeof(BTile) * hdr[5 + pi]);
  if (st == SLSHT_OK) st = put(L.in, in_off);
  if (st == SLSHT_OK && cudaGraphLaunch(ln.exec, ln.st) != cudaSuccess) {
    cudaGetLastError();
    st = SLSHT_E_CUDA;
  }
  for (const SvTc& t : tcs) {
    if (st != SLSHT_OK) break;
    if (sv_tc_launch(c, t, ln.st) != cudaSuccess) {
      cudaGetLastError();
      st = SLSHT_E_CUDA;
    }
  }
  if (st == SLSHT_OK && cudaEventRecord(ln.ev_b, ln.st) != cudaSuccess) st = SLSHT_E_CUDA;
  const double t1 = sv_now_ms();
  lk.lock();
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->launches[SLSHT_STAGE_COUPLE] += 4;
    c->launches[SLSHT_STAGE_BETA] += 1;
    c->launches[SLSHT_STAGE_ALPHA] += 3;
    c->samples += (uint64_t)samples;
  }
  c->sv_ticks++;
  for (const SvChunk& k : ch)
    if (k.r->t_issue < 0) k.r->t_issue = t1 - t0;
  if (st != SLSHT_OK) {
    for (const SvChunk& k : ch) k.r->status = st;
    // the lane's stream is left as it is; its chunks fail with the tick
  }
  ln.chunks = std::move(ch);
  ln.busy = true;
  ln.tick = tick_no;
  ln.t_assemble = t0;
  return st == SLSHT_OK ? (int)ln.chunks.size() : st;
}

// Retires a lane whose tick has completed (c->smu held).
static void sv_retire(slsht_ctx* c, SvLane& ln) {
  const cudaError_t q = cudaEventQuery(ln.ev_b);
  if (q == cudaErrorNotReady) return;
  float a = 0.f, b = 0.f;
  int st = SLSHT_OK;
  if (q != cudaSuccess || cudaEventElapsedTime(&a, c->sv_ref, ln.ev_a) != cudaSuccess ||
      cudaEventElapsedTime(&b, c->sv_ref, ln.ev_b) != cudaSuccess) {
    cudaGetLastError();
    record_cuda_error("serving tick", q != cudaSuccess ? q : cudaErrorUnknown);
    st = SLSHT_E_CUDA;
  }
  const double now = sv_now_ms();
  for (const SvChunk& k : ln.chunks) {
    Request& r = *k.r;
    r.done += k.np;
    r.dev_first = std::min(r.dev_first, (double)a);
    r.dev_last = std::max(r.dev_last, (double)b);
    if (st != SLSHT_OK) r.status = st;
  }
  ln.chunks.clear();
  ln.busy = false;
  // finished requests leave the active list with their times
  for (size_t i = 0; i < c->active.size();) {
    Request& r = *c->active[i];
    if (r.done >= r.n_pairs || (r.status != SLSHT_OK && r.next >= r.n_pairs && r.done >= r.next)) {
      if (r.h_have) sv_hrelease(c, r.h_off, r.h_len);
      slsht_ctx::Final fin{r.status, {r.t_admit - r.t_submit, r.t_issue, r.dev_last - r.dev_first, now - r.t_submit}};
      c->status[r.id] = fin;
      c->active.erase(c->active.begin() + (long)i);
      c->inflight--;
      c->scv.notify_all();
    } else {
      ++i;
    }
  }
}

static void worker_loop(slsht_ctx* c) {
  DeviceGuard g(c->device);
  std::unique_lock<std::mutex> l(c->smu);
  int init = sv_init(c);
  while (true) {
    for (auto& ln : c->lanes)
      if (ln.busy) sv_retire(c, ln);
    if (init != SLSHT_OK) {          // fail every request: the serving lanes could not be set up
      while (!c->queue.empty()) {
        c->status[c->queue.front()->id] = slsht_ctx::Final{init, {0, 0, 0, 0}};
        c->queue.pop_front();
        c->inflight--;
      }
      c->scv.notify_all();
    }
    bool issued = false;
    if (init == SLSHT_OK) {
      for (auto& ln : c->lanes) {    // every free lane, the express lane first
        if (ln.busy) continue;
        const int n = sv_tick(c, ln, l);
        if (n > 0) issued = true;
        if (n != 0 && &ln != &c->lanes[0]) break;   // one bulk tick per pass: completions are seen between
      }
    }
    bool busy = false;
    for (auto& ln : c->lanes) busy = busy || ln.busy;
    if (c->stop && c->queue.empty() && c->active.empty() && !busy) break;
    if (issued) continue;
    if (busy) {
      c->scv.wait_for(l, std::chrono::microseconds(50));
    } else {
      c->scv.wait(l, [c] { return c->stop || !c->queue.empty(); });
    }
  }
}

static int copy_in(const double* src, size_t n, std::vector<double>& dst) {
  dst.resize(n);
  if (is_device_ptr(src)) {
    CK(cudaMemcpy(dst.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst.data(), src, n * sizeof(double));
  }
  return SLSHT_OK;
}

extern "C" int slsht_submit(slsht_ctx* c, const slsht_desc* desc, const double* f_lm,
                            const double* h_lm, const int32_t* lm, int32_t n_pairs, void* g_out,
                            uint64_t* ticket) {
  if (!c || !ticket) return SLSHT_E_ARG;
  CKS(check_desc(desc));
  if (n_pairs <= 0 || !f_lm || !h_lm || !lm || !g_out) return SLSHT_E_ARG;
  DeviceGuard g(c->device);
  if (!is_device_ptr(g_out) || (((uintptr_t)g_out) & 7)) return SLSHT_E_ARG;
  std::unique_ptr<Request> r(new Request());
  r->desc = *desc;
  r->g_out = g_out;
  r->n_pairs = n_pairs;
  r->t_submit = sv_now_ms();
  CKS(copy_in(f_lm, 2 * (size_t)desc->L_f * desc->L_f, r->f));
  CKS(copy_in(h_lm, 2 * (size_t)desc->L_h * desc->L_h, r->h));
  r->lm.resize(2 * (size_t)n_pairs);
  if (is_device_ptr(lm)) {
    CK(cudaMemcpy(r->lm.data(), lm, sizeof(int32_t) * 2 * (size_t)n_pairs, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(r->lm.data(), lm, sizeof(int32_t) * 2 * (size_t)n_pairs);
  }
  CKS(check_pairs(desc, r->lm.data(), n_pairs));
  // one pair must fit an empty tick (the double-float form is the larger)
  {
    Request probe = Request();
    probe.desc = *desc;
    probe.engine = ENG_DD;
    probe.nt = 32;
    const long long J = (long long)desc->n_beta * desc->n_gamma;
    if (sv_dev_bytes(probe, 1) > SV_DEV_BYTES || sv_in_bytes(probe, 1) > SV_STAGE_IN ||
        sv_h_bytes(probe) > SV_HPOOL_BYTES ||
        sv_rblk_count(probe) > SV_RBLK || (J + 31) / 32 > SV_TILES) {
      slsht_record_error_text("slsht_submit: one pair of this request exceeds a serving tick's arena");
      return SLSHT_E_NOMEM;
    }
  }
  std::unique_lock<std::mutex> l(c->smu);
  if (c->inflight >= SERVE_MAX_QUEUE) return SLSHT_E_BUSY;
  if (!c->worker_started) {
    c->worker = std::thread(worker_loop, c);
    c->worker_started = true;
  }
  r->id = c->next_id++;
  *ticket = r->id;
  c->status[r->id] = slsht_ctx::Final{SLSHT_PENDING, {0, 0, 0, 0}};
  c->queue.push_back(std::move(r));
  c->inflight++;
  c->scv.notify_all();
  return SLSHT_OK;
}

extern "C" int slsht_poll_times(slsht_ctx* c, uint64_t ticket, double* times) {
  if (!c) return SLSHT_E_ARG;
  std::lock_guard<std::mutex> l(c->smu);
  auto it = c->status.find(ticket);
  if (it == c->status.end()) return SLSHT_E_STATE;
  const int s = it->second.st;
  if (s != SLSHT_PENDING) {
    if (times)
      for (int i = 0; i < 4; ++i) times[i] = it->second.t[i];
    c->status.erase(it);
  }
  return s;
}

extern "C" int slsht_poll(slsht_ctx* c, uint64_t ticket) { return slsht_poll_times(c, ticket, nullptr); }

extern "C" int slsht_drain(slsht_ctx* c, int64_t timeout_ms) {
  if (!c) return SLSHT_E_ARG;
  std::unique_lock<std::mutex> l(c->smu);
  const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  while (c->inflight > 0) {
    if (c->scv.wait_until(l, until) == std::cv_status::timeout && c->inflight > 0) return SLSHT_E_TIMEOUT;
  }
  return SLSHT_OK;
}

// ---------------------------------------------------------------- tools
extern "C" const char* slsht_strerror(int code) {
  switch (code) {
    case SLSHT_OK: return "ok";
    case SLSHT_PENDING: return "request pending";
    case SLSHT_E_ARG: return "invalid argument";
    case SLSHT_E_H00: return "window DC coefficient h_0^0 is zero; the inverse needs it non-zero";
    case SLSHT_E_NOMEM: return "out of device memory or over the context's memory budget";
    case SLSHT_E_BUSY: return "request queue full";
    case SLSHT_E_TIMEOUT: return "bounded wait expired";
    case SLSHT_E_CUDA: return "CUDA call failed (see slsht_last_error)";
    case SLSHT_E_STATE: return "unknown ticket or invalid context state";
    default: return "unknown status code";
  }
}

extern "C" const char* slsht_last_error(void) {
  static thread_local std::string copy;
  std::lock_guard<std::mutex> g(g_err_mu);
  copy = g_last_err;
  return copy.c_str();
}

extern "C" int slsht_profile(slsht_ctx* c, int enable) {
  if (!c) return SLSHT_E_ARG;
  std::lock_guard<std::mutex> g(c->mu);
  c->profile = enable != 0;
  return SLSHT_OK;
}

extern "C" int slsht_get_stats(slsht_ctx* c, slsht_stats* out, int reset) {
  if (!c || !out) return SLSHT_E_ARG;
  DeviceGuard dg(c->device);
  std::lock_guard<std::mutex> g(c->mu);
  for (auto& r : c->prof) {
    float ms = 0.f;
    CK(cudaEventSynchronize(r.b));
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    c->prof_ms[r.stage] += ms;
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof.clear();
  for (int i = 0; i < SLSHT_NSTAGES; ++i) {
    out->launches[i] = c->launches[i];
    out->ms[i] = c->prof_ms[i];
  }
  out->samples_written = c->samples;
  const int dev_err = tc_read_error();
  if (reset) {
    for (int i = 0; i < SLSHT_NSTAGES; ++i) { c->launches[i] = 0; c->prof_ms[i] = 0.0; }
    c->samples = 0;
  }
  return dev_err ? SLSHT_E_TIMEOUT : SLSHT_OK;
}

extern "C" size_t slsht_mem_used(slsht_ctx* c) { return c ? c->used.load() : 0; }

extern "C" const char* slsht_version(void) { return "libslsht 0.1 (sm_103a)"; }
