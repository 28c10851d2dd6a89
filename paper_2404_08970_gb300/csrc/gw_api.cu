// C ABI entry points: context, validation, workspace, dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gw_internal.h"

// Records a pair of CUDA events around every traced launch; totals are folded
// in when the report is read.
struct EventTracer : gw::Tracer {
  struct Rec {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<std::string, cudaEvent_t>> open;
  std::map<std::string, std::pair<long, double>> totals;  // name -> (launches, ms)

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void begin(const char* name, cudaStream_t st) override {
    cudaEvent_t e = get();
    cudaEventRecord(e, st);
    open.push_back({name, e});
  }
  void end(cudaStream_t st) override {
    if (open.empty()) return;
    auto o = open.back();
    open.pop_back();
    cudaEvent_t e = get();
    cudaEventRecord(e, st);
    pending.push_back({o.first, o.second, e});
  }
  void collect() {
    for (auto& r : pending) {
      cudaEventSynchronize(r.b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      auto& t = totals[r.name];
      t.first += 1;
      t.second += ms;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  ~EventTracer() override {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct gw_ctx {
  int device = 0;
  int num_sms = 0;
  std::mutex mu;
  std::string err;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  unsigned* status = nullptr;  // device status word
  EventTracer* tracer = nullptr;  // non-null while profiling is on
  int force_generic = 0;          // GW_FORCE_GENERIC set at creation: block-scan row kernel only
  void* dense = nullptr;          // cuBLAS handle and cached dense distance matrices
  // Graph of the last solve (the whole mirror descent), relaunched while the
  // arguments stay the same.
  cudaStream_t cap = nullptr;
  // Side stream and events for work that overlaps inside one call.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Graphs of recent calls (gradients, solves), keyed by their arguments and
  // relaunched while the arguments match; at most kGraphCache, oldest dropped.
  std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;
  // Batched solves: worker streams (fork/join inside the captured graph), the
  // batch workspace and the last batch graph.
  std::vector<cudaStream_t> bstreams;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  std::vector<cudaEvent_t> mix_ev;  // fork and join events of the mixed sets
  void* bws = nullptr;
  size_t bws_bytes = 0;
  cudaGraphExec_t batch_exec = nullptr;
  std::string batch_key;
  // gw_grad_host: two device slots used in turn, so that one call's copy-in
  // overlaps the previous call's gradient and copy-out; a stream each for
  // copy-in, gradient and copy-out.
  struct HostSlot {
    void* dT = nullptr;
    void* dG = nullptr;
    void* dm = nullptr;  // marginals u (n doubles) then v (m doubles)
    size_t tg_bytes = 0, marg_bytes = 0;
    cudaEvent_t in = nullptr, comp = nullptr, out = nullptr;
    bool used = false;
  };
  HostSlot hslot[2];
  int hnext = 0;
  cudaStream_t h_in = nullptr, h_comp = nullptr, h_out = nullptr;
  gw::Tracer* tr() { return tracer; }
};

namespace {

gw_status fail(gw_ctx* c, gw_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
gw_status fail(gw_ctx* c, gw_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

gw_status cuda_fail(gw_ctx* c, cudaError_t e, const char* what) {
  return fail(c, GW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grows the context workspace to at least `bytes` (synchronises the device
// when it has to reallocate).
gw_status ensure_ws(gw_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return GW_OK;
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&c->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, GW_ERR_OOM, "workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  c->ws_bytes = want;
  return GW_OK;
}

constexpr size_t kGraphCache = 8;

// Runs `enqueue` (a sequence of launches on the stream it is given) on
// `stream` as a CUDA graph: captured on the context's side stream the first
// time a key is seen, relaunched from the cache afterwards.  With profiling on
// the launches go straight to `stream` (per-kernel events need them eager).
template <typename F>
gw_status run_graph(gw_ctx* c, const std::string& key, cudaStream_t stream, F&& enqueue, const char* what) {
  int rc;
  if (c->tracer) {
    rc = enqueue(stream);
  } else {
    // A captured graph holds the row configurations of its time: the tuning
    // table's generation is part of the key.
    const std::string tkey = key + " tune" + std::to_string(gw::tune_generation());
    cudaGraphExec_t exec = nullptr;
    for (size_t i = 0; i < c->graphs.size(); ++i)
      if (c->graphs[i].first == tkey) {
        exec = c->graphs[i].second;
        break;
      }
    if (!exec) {
      if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "capture stream");
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
      rc = enqueue(c->cap);
      e = cudaStreamEndCapture(c->cap, &graph);
      if (rc != GW_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(c, rc != GW_OK ? (gw_status)rc : GW_ERR_CUDA, "%s: capture failed (%s)", what,
                    gw::last_failure());
      }
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
      if (c->graphs.size() >= kGraphCache) {
        cudaGraphExecDestroy(c->graphs.front().second);
        c->graphs.erase(c->graphs.begin());
      }
      c->graphs.emplace_back(tkey, exec);
    }
    rc = cudaGraphLaunch(exec, stream) == cudaSuccess ? GW_OK : GW_ERR_CUDA;
  }
  if (rc != GW_OK) {
    cudaError_t e = cudaGetLastError();
    return fail(c, (gw_status)rc, "%s launch failed: %s (%s)", what, cudaGetErrorString(e), gw::last_failure());
  }
  c->err.clear();
  return GW_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

gw_status check_grid(gw_ctx* c, const gw_problem* p) {
  if (!p) return fail(c, GW_ERR_INVALID, "problem descriptor is NULL");
  if (p->dim < 1 || p->dim > 3) return fail(c, GW_ERR_INVALID, "dim must be 1, 2 or 3 (got %d)", p->dim);
  if (p->nx < 1 || p->ny < 1) return fail(c, GW_ERR_INVALID, "grid sizes must be >= 1 (got %d, %d)", p->nx, p->ny);
  if (!finite_pos(p->hx) || !finite_pos(p->hy)) return fail(c, GW_ERR_INVALID, "grid spacings must be finite and > 0");
  if (p->k < 1) return fail(c, GW_ERR_INVALID, "distance exponent k must be >= 1 (got %d)", p->k);
  if (p->dtype != GW_F32 && p->dtype != GW_F64) return fail(c, GW_ERR_INVALID, "dtype must be GW_F32 or GW_F64");
  if (p->dim == 1) {
    if (p->k > 3) return fail(c, GW_ERR_INVALID, "k must be <= 3 (got %d)", p->k);
    if (p->ny > 16384) return fail(c, GW_ERR_INVALID, "ny must be <= 16384 (got %d)", p->ny);
    if (!gw::mixed_k_supported(p->k, p->ky, p->ny, p->dtype))
      return fail(c, GW_ERR_INVALID,
                  "mixed exponents (k, ky) = (%d, %d): supported are (1, 2) and (2, 1) with ny <= 8192 "
                  "(4096 in double)", p->k, p->ky);
  } else if (p->dim == 3) {
    if (p->ky != 0 && p->ky != p->k)
      return fail(c, GW_ERR_INVALID, "3D grids take one distance exponent (ky = 0 or k)");
    if (!(p->cost == GW_COST_SQEUCLID || (p->cost == GW_COST_POW && p->k == 1)))
      return fail(c, GW_ERR_INVALID, "3D grids take the Manhattan distance with k = 1 or the squared Euclidean "
                                     "distance (got cost %d, k = %d)", p->cost, p->k);
    if (p->nx > gw::kMax3DSide || p->ny > gw::kMax3DSide)
      return fail(c, GW_ERR_INVALID, "3D grid sides must be <= %d (got %d, %d)", gw::kMax3DSide, p->nx, p->ny);
  } else {
    if (p->ky != 0 && p->ky != p->k)
      return fail(c, GW_ERR_INVALID, "2D grids take one distance exponent (ky = 0 or k)");
    if (p->cost != GW_COST_POW && p->cost != GW_COST_SQEUCLID)
      return fail(c, GW_ERR_INVALID, "2D cost must be GW_COST_POW or GW_COST_SQEUCLID (got %d)", p->cost);
    if (p->nx > gw::kMax2DSide || p->ny > gw::kMax2DSide)
      return fail(c, GW_ERR_INVALID, "2D grid sides must be <= %d (got %d, %d)", gw::kMax2DSide, p->nx, p->ny);
    if (p->cost == GW_COST_POW && p->k > 1 && !gw::grad2d_powk_supported(p->nx, p->ny, p->k, p->dtype))
      return fail(c, GW_ERR_INVALID,
                  "2D Manhattan^k with k = %d needs k <= 3 and grid sides <= 128 (float) or a smaller double "
                  "image (got %d, %d)", p->k, p->nx, p->ny);
  }
  return GW_OK;
}

// Points of each space: nx, ny in 1D, nx^dim, ny^dim on 2D and 3D grids.
size_t grid_points(int side, int dim) {
  size_t q = 1;
  for (int d = 0; d < dim; ++d) q *= (size_t)side;
  return q;
}
size_t points_x(const gw_problem* p) { return grid_points(p->nx, p->dim); }
size_t points_y(const gw_problem* p) { return grid_points(p->ny, p->dim); }

}  // namespace

extern "C" {

gw_status gw_ctx_create(gw_ctx** out, int device) {
  if (!out) return GW_ERR_INVALID;
  *out = nullptr;
  gw::tune_autoload();
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GW_ERR_CUDA;
  }
  gw_ctx* c = new gw_ctx();
  c->device = device;
  const char* fg = getenv("GW_FORCE_GENERIC");
  c->force_generic = (fg && fg[0] && fg[0] != '0') ? 1 : 0;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  e = cudaMalloc(&c->status, sizeof(unsigned));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return GW_ERR_OOM;
  }
  cudaMemset(c->status, 0, sizeof(unsigned));
  *out = c;
  return GW_OK;
}

void gw_ctx_destroy(gw_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->ws) cudaFree(c->ws);
  if (c->status) cudaFree(c->status);
  gw::dense_state_destroy(c->dense);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
  for (auto st : c->bstreams) cudaStreamDestroy(st);
  for (auto ev : c->join_ev) cudaEventDestroy(ev);
  for (auto ev : c->mix_ev) cudaEventDestroy(ev);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->bws) cudaFree(c->bws);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (auto& h : c->hslot) {
    for (void* q : {h.dT, h.dG, h.dm})
      if (q) cudaFree(q);
    for (cudaEvent_t q : {h.in, h.comp, h.out})
      if (q) cudaEventDestroy(q);
  }
  for (cudaStream_t q : {c->h_in, c->h_comp, c->h_out})
    if (q) cudaStreamDestroy(q);
  delete c->tracer;
  delete c;
}

gw_status gw_ctx_profile(gw_ctx* c, int enable) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (enable && !c->tracer) c->tracer = new EventTracer();
  if (!enable && c->tracer) {
    cudaDeviceSynchronize();
    delete c->tracer;
    c->tracer = nullptr;
  }
  return GW_OK;
}

gw_status gw_ctx_profile_report(gw_ctx* c, char* buf, size_t len, int reset) {
  if (!c || !buf || len == 0) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  std::string out = "{";
  if (c->tracer) {
    c->tracer->collect();
    bool first = true;
    for (auto& kv : c->tracer->totals) {
      char item[256];
      snprintf(item, sizeof item, "%s\"%s\": {\"launches\": %ld, \"ms\": %.6f}", first ? "" : ", ",
               kv.first.c_str(), kv.second.first, kv.second.second);
      out += item;
      first = false;
    }
    if (reset) c->tracer->totals.clear();
  }
  out += "}";
  if (out.size() + 1 > len) return fail(c, GW_ERR_INVALID, "profile report needs %zu bytes", out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return GW_OK;
}

const char* gw_last_error(const gw_ctx* c) { return c ? c->err.c_str() : "no context"; }

gw_status gw_ctx_check(gw_ctx* c, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  unsigned word = 0;
  e = cudaMemcpy(&word, c->status, sizeof word, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  cudaMemset(c->status, 0, sizeof(unsigned));
  if (word & 1u) return fail(c, GW_ERR_TIMEOUT, "a bounded device wait gave up");
  if (word & 2u) return fail(c, GW_ERR_NONFINITE, "a non-finite value reached an output");
  c->err.clear();
  return GW_OK;
}

}  // extern "C"

namespace {

// Argument checks shared by gw_grad and gw_grad_host (the pointers may be
// device or host pointers; only their presence is checked here).
gw_status check_grad_args(gw_ctx* c, const gw_problem* p, const void* u, const void* v, const void* T, void* G,
                          int marginals) {
  gw_status s = check_grid(c, p);
  if (s != GW_OK) return s;
  if (marginals != GW_MARG_TARGET && marginals != GW_MARG_EXACT)
    return fail(c, GW_ERR_INVALID, "marginals must be GW_MARG_TARGET or GW_MARG_EXACT");
  if (!T || !G) return fail(c, GW_ERR_INVALID, "T and G must not be NULL");
  if (marginals == GW_MARG_TARGET && (!u || !v))
    return fail(c, GW_ERR_INVALID, "target marginals requested but u or v is NULL");
  const size_t esz = p->dtype == GW_F32 ? 4 : 8;
  const size_t nm = points_x(p) * points_y(p);
  const char* t0 = (const char*)T;
  const char* g0 = (const char*)G;
  if (t0 < g0 + nm * esz && g0 < t0 + nm * esz) return fail(c, GW_ERR_INVALID, "T and G overlap");
  return GW_OK;
}

// The gradient on device buffers, enqueued on `stream`; the caller holds
// c->mu and has checked the arguments.
gw_status grad_device(gw_ctx* c, const gw_problem* p, const double* d_u, const double* d_v, const void* d_T,
                      void* d_G, int marginals, void* stream) {
  gw_status s;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GW_ERR_CUDA, "cudaSetDevice failed");

  if (p->dim >= 2) {
    gw::Grad2DArgs a{};
    a.dim = p->dim;
    a.sx = p->nx;
    a.sy = p->ny;
    a.cost = p->cost;
    a.k = p->k;
    a.hx = p->hx;
    a.hy = p->hy;
    a.dtype = p->dtype;
    a.T = d_T;
    a.G = d_G;
    a.u = d_u;
    a.v = d_v;
    a.exact = marginals == GW_MARG_EXACT;
    a.out_scale = 1.0;
    a.stream = (cudaStream_t)stream;
    a.status = c->status;
    a.num_sms = c->num_sms;
    a.tracer = c->tr();
    s = ensure_ws(c, gw::grid_grad_workspace_bytes(a.dim, a.sx, a.sy, a.dtype, a.cost, a.k));
    if (s != GW_OK) return s;
    char key[384];
    snprintf(key, sizeof key, "grad%d %d %d %d %d %.17g %.17g %d %p %p %p %p %d %p %zu", a.dim, a.sx, a.sy, a.cost, a.k,
             a.hx, a.hy, a.dtype, a.T, a.G, (void*)a.u, (void*)a.v, a.exact, c->ws, c->ws_bytes);
    return run_graph(
        c, key, a.stream,
        [&](cudaStream_t st) {
          gw::Grad2DArgs ac = a;
          ac.stream = st;
          return gw::grad2d_launch(ac, c->ws, c->ws_bytes);
        },
        a.dim == 3 ? "gw_grad (3D)" : "gw_grad (2D)");
  }

  gw::Grad1DArgs a{};
  a.n = p->nx;
  a.m = p->ny;
  a.k = p->k;
  a.ky = p->ky == p->k ? 0 : p->ky;
  a.hx = p->hx;
  a.hy = p->hy;
  a.dtype = p->dtype;
  a.T = d_T;
  a.G = d_G;
  a.u = d_u;
  a.v = d_v;
  a.exact = marginals == GW_MARG_EXACT;
  a.out_scale = 1.0;
  a.stream = (cudaStream_t)stream;
  a.status = c->status;
  a.num_sms = c->num_sms;
  a.tracer = c->tr();
  a.force_generic = c->force_generic;
  s = ensure_ws(c, gw::grad1d_workspace_bytes(a.n, a.m, a.k, a.dtype, a.num_sms));
  if (s != GW_OK) return s;
  if (!c->side) {
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(c, cudaGetLastError(), "side stream");
  }
  a.side = c->side;
  a.ev_fork = c->ev_fork;
  a.ev_join = c->ev_join;
  char key[384];
  snprintf(key, sizeof key, "grad1 %d %d %d %d %.17g %.17g %d %p %p %p %p %d %d %p %zu", a.n, a.m, a.k, a.ky, a.hx,
           a.hy, a.dtype, a.T, a.G, (void*)a.u, (void*)a.v, a.exact, a.force_generic, c->ws, c->ws_bytes);
  return run_graph(
      c, key, a.stream,
      [&](cudaStream_t st) {
        gw::Grad1DArgs ac = a;
        ac.stream = st;
        return gw::grad1d_launch(ac, c->ws, c->ws_bytes);
      },
      "gw_grad");
}

// Grows one host-call slot to hold the problem's T and G (device) and its
// marginals; synchronises the device when it has to reallocate.
gw_status ensure_host_slot(gw_ctx* c, gw_ctx::HostSlot& h, size_t tg_bytes, size_t marg_bytes) {
  if (tg_bytes <= h.tg_bytes && marg_bytes <= h.marg_bytes) return GW_OK;
  cudaDeviceSynchronize();
  for (void** q : {&h.dT, &h.dG, &h.dm}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  h.tg_bytes = h.marg_bytes = 0;
  cudaError_t e = cudaMalloc(&h.dT, tg_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h.dG, tg_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h.dm, marg_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, GW_ERR_OOM, "host-call staging of %zu bytes failed: %s", 2 * tg_bytes + marg_bytes,
                cudaGetErrorString(e));
  }
  h.tg_bytes = tg_bytes;
  h.marg_bytes = marg_bytes;
  return GW_OK;
}

}  // namespace

extern "C" {

gw_status gw_grad(gw_ctx* c, const gw_problem* p, const double* d_u, const double* d_v, const void* d_T, void* d_G,
                  int marginals, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  gw_status s = check_grad_args(c, p, d_u, d_v, d_T, d_G, marginals);
  if (s != GW_OK) return s;
  return grad_device(c, p, d_u, d_v, d_T, d_G, marginals, stream);
}

gw_status gw_grad_host(gw_ctx* c, const gw_problem* p, const double* h_u, const double* h_v, const void* h_T,
                       void* h_G, int marginals, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  gw_status s = check_grad_args(c, p, h_u, h_v, h_T, h_G, marginals);
  if (s != GW_OK) return s;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GW_ERR_CUDA, "cudaSetDevice failed");
  if (!c->h_in) {
    for (cudaStream_t* q : {&c->h_in, &c->h_comp, &c->h_out})
      if (cudaStreamCreateWithFlags(q, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "host-call streams");
    for (auto& h : c->hslot)
      for (cudaEvent_t* q : {&h.in, &h.comp, &h.out})
        if (cudaEventCreateWithFlags(q, cudaEventDisableTiming) != cudaSuccess)
          return cuda_fail(c, cudaGetLastError(), "host-call events");
  }
  const size_t esz = p->dtype == GW_F32 ? 4 : 8;
  const size_t n = points_x(p), m = points_y(p);
  const size_t tg = n * m * esz;
  gw_ctx::HostSlot& h = c->hslot[c->hnext];
  s = ensure_host_slot(c, h, tg, (n + m) * sizeof(double));
  if (s != GW_OK) return s;
  c->hnext ^= 1;
  const bool target = marginals == GW_MARG_TARGET;
  double* du = (double*)h.dm;
  double* dv = du + n;
  cudaError_t e = cudaSuccess;
  // Copy in, once the slot's previous gradient has read its T.
  if (h.used) e = cudaStreamWaitEvent(c->h_in, h.comp, 0);
  if (e == cudaSuccess && target) e = cudaMemcpyAsync(du, h_u, n * sizeof(double), cudaMemcpyHostToDevice, c->h_in);
  if (e == cudaSuccess && target) e = cudaMemcpyAsync(dv, h_v, m * sizeof(double), cudaMemcpyHostToDevice, c->h_in);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.dT, h_T, tg, cudaMemcpyHostToDevice, c->h_in);
  if (e == cudaSuccess) e = cudaEventRecord(h.in, c->h_in);
  // The gradient, once T is in and the slot's previous G has been copied out.
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->h_comp, h.in, 0);
  if (e == cudaSuccess && h.used) e = cudaStreamWaitEvent(c->h_comp, h.out, 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "gw_grad_host copy-in");
  s = grad_device(c, p, target ? du : nullptr, target ? dv : nullptr, h.dT, h.dG, marginals, c->h_comp);
  if (s != GW_OK) return s;
  e = cudaEventRecord(h.comp, c->h_comp);
  // Copy out, then order the caller's stream after it.
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->h_out, h.comp, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_G, h.dG, tg, cudaMemcpyDeviceToHost, c->h_out);
  if (e == cudaSuccess) e = cudaEventRecord(h.out, c->h_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, h.out, 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "gw_grad_host copy-out");
  h.used = true;
  c->err.clear();
  return GW_OK;
}

gw_status gw_grad_dense(gw_ctx* c, const gw_problem* p, const double* d_u, const double* d_v, const void* d_T,
                        void* d_G, int marginals, int precision, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  gw_status s = check_grid(c, p);
  if (s != GW_OK) return s;
  if (precision < GW_DENSE_FP32 || precision > GW_DENSE_TC_BF16)
    return fail(c, GW_ERR_INVALID, "gw_grad_dense: unknown precision %d", precision);
  if ((precision == GW_DENSE_FP64) != (p->dtype == GW_F64))
    return fail(c, GW_ERR_INVALID, "gw_grad_dense: dtype must be GW_F64 exactly for GW_DENSE_FP64");
  if (marginals != GW_MARG_TARGET && marginals != GW_MARG_EXACT)
    return fail(c, GW_ERR_INVALID, "marginals must be GW_MARG_TARGET or GW_MARG_EXACT");
  if (!d_T || !d_G) return fail(c, GW_ERR_INVALID, "d_T and d_G must not be NULL");
  if (marginals == GW_MARG_TARGET && (!d_u || !d_v))
    return fail(c, GW_ERR_INVALID, "target marginals requested but d_u or d_v is NULL");
  const size_t esz = p->dtype == GW_F32 ? 4 : 8;
  const size_t nm = points_x(p) * points_y(p);
  const char* t0 = (const char*)d_T;
  const char* g0 = (const char*)d_G;
  if (t0 < g0 + nm * esz && g0 < t0 + nm * esz) return fail(c, GW_ERR_INVALID, "d_T and d_G overlap");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GW_ERR_CUDA, "cudaSetDevice failed");
  if (!c->dense) c->dense = gw::dense_state_create();
  gw::DenseArgs a{};
  a.dim = p->dim;
  a.cost = p->cost;
  a.sx = p->nx;
  a.sy = p->ny;
  a.n = (int)points_x(p);
  a.m = (int)points_y(p);
  a.k = p->k;
  a.ky = p->ky == p->k ? 0 : p->ky;
  a.prec = precision;
  a.exact = marginals == GW_MARG_EXACT;
  a.hx = p->hx;
  a.hy = p->hy;
  a.u = d_u;
  a.v = d_v;
  a.T = d_T;
  a.G = d_G;
  a.stream = (cudaStream_t)stream;
  a.tracer = c->tr();
  a.status = c->status;
  a.num_sms = c->num_sms;
  s = ensure_ws(c, gw::dense_workspace_bytes(a.n, a.m, precision));
  if (s != GW_OK) return s;
  int rc = gw::dense_grad_launch(c->dense, a, c->ws, c->ws_bytes);
  if (rc != GW_OK) {
    cudaError_t e = cudaGetLastError();
    return fail(c, (gw_status)rc, "gw_grad_dense failed: %s (%s)", cudaGetErrorString(e), gw::last_failure());
  }
  c->err.clear();
  return GW_OK;
}

}  // extern "C"

namespace {

gw_status check_solve(gw_ctx* c, const gw_problem* p, const double* d_u, const double* d_v, const double* d_phi,
                      const double* d_psi, const void* d_T, const char* who) {
  gw_status s = check_grid(c, p);
  if (s != GW_OK) return s;
  if (!finite_pos(p->eps)) return fail(c, GW_ERR_INVALID, "%s: eps must be finite and > 0", who);
  if (!(p->tau == 0.0 || finite_pos(p->tau)))
    return fail(c, GW_ERR_INVALID, "%s: tau must be 0 (tau = eps) or finite and > 0", who);
  if (p->warm_start != 0 && p->warm_start != 1) return fail(c, GW_ERR_INVALID, "%s: warm_start must be 0 or 1", who);
  if (!(p->rho == 0.0 || finite_pos(p->rho)))
    return fail(c, GW_ERR_INVALID, "%s: rho must be 0 (balanced) or finite and > 0", who);
  if (p->rho > 0.0 && (p->theta != 1.0 || (p->tau != 0.0 && p->tau != p->eps)))
    return fail(c, GW_ERR_INVALID, "%s: unbalanced GW (rho > 0) takes theta = 1 and tau = eps", who);
  if (p->n_outer < 0 || p->n_inner < 1)
    return fail(c, GW_ERR_INVALID, "%s: need n_outer >= 0 and n_inner >= 1", who);
  if (!(p->theta >= 0.0 && p->theta <= 1.0)) return fail(c, GW_ERR_INVALID, "%s: theta must be in [0, 1]", who);
  if (p->theta != 1.0 && (p->feat_dim < 1 || p->feat_dim > 64 || !d_phi || !d_psi))
    return fail(c, GW_ERR_INVALID, "%s: fused GW (theta < 1) needs 1 <= feat_dim <= 64 and both feature arrays",
                who);
  if (!d_u || !d_v || !d_T) return fail(c, GW_ERR_INVALID, "%s: d_u, d_v and d_T must not be NULL", who);
  if (points_y(p) > 16384)
    return fail(c, GW_ERR_INVALID, "%s: the solver takes at most 16384 points in Y (got %zu)", who, points_y(p));
  if (p->dtype == GW_F64 && points_y(p) > gw::kMaxSolveF64Y)
    return fail(c, GW_ERR_INVALID, "%s: double-precision solves take at most %d points in Y (got %zu)", who,
                gw::kMaxSolveF64Y, points_y(p));
  return GW_OK;
}

gw::SolveArgs solve_args(gw_ctx* c, const gw_problem* p, const double* d_u, const double* d_v, const double* d_phi,
                         const double* d_psi, void* d_T, double* d_f, double* d_g, double* d_stats, void* stream) {
  gw::SolveArgs a{};
  a.dim = p->dim;
  a.cost = p->cost;
  a.nx = p->nx;
  a.ny = p->ny;
  a.n = (int)points_x(p);
  a.m = (int)points_y(p);
  a.k = p->k;
  a.dtype = p->dtype;
  a.hx = p->hx;
  a.hy = p->hy;
  a.eps = p->eps;
  a.tau = p->tau > 0.0 ? p->tau : p->eps;
  a.warm_start = p->warm_start;
  a.rho = p->rho;
  a.ky = p->ky == p->k ? 0 : p->ky;
  a.theta = p->theta;
  a.n_outer = p->n_outer;
  a.n_inner = p->n_inner;
  a.feat_dim = p->theta != 1.0 ? p->feat_dim : 0;
  a.u = d_u;
  a.v = d_v;
  a.phi = d_phi;
  a.psi = d_psi;
  a.T = d_T;
  a.f = d_f;
  a.g = d_g;
  a.stats = d_stats;
  a.stream = (cudaStream_t)stream;
  a.status = c->status;
  a.num_sms = c->num_sms;
  a.tracer = c->tr();
  a.force_generic = c->force_generic;
  return a;
}

}  // namespace

extern "C" {

gw_status gw_solve(gw_ctx* c, const gw_problem* p, const double* d_u, const double* d_v, const double* d_phi,
                   const double* d_psi, void* d_T, double* d_f, double* d_g, double* d_stats, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  gw_status s = check_solve(c, p, d_u, d_v, d_phi, d_psi, d_T, "gw_solve");
  if (s != GW_OK) return s;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GW_ERR_CUDA, "cudaSetDevice failed");
  gw::SolveArgs a = solve_args(c, p, d_u, d_v, d_phi, d_psi, d_T, d_f, d_g, d_stats, stream);
  s = ensure_ws(c, gw::solve_workspace_bytes(a));
  if (s != GW_OK) return s;
  char key[512];
  snprintf(key, sizeof key,
           "solve %d %d %d %d %d %d %d %.17g %.17g %.17g %.17g %.17g %.17g %d %d %d %d %p %p %p %p %p %p %p %p %p %zu",
           a.dim, a.cost, a.n, a.m, a.k, a.ky, a.dtype, a.hx, a.hy, a.eps, a.tau, a.rho, a.theta, a.warm_start, a.n_outer,
           a.n_inner, a.feat_dim,
           (void*)a.u, (void*)a.v, (void*)a.phi, (void*)a.psi, a.T, (void*)a.f, (void*)a.g, (void*)a.stats, c->ws,
           c->ws_bytes);
  return run_graph(
      c, key, a.stream,
      [&](cudaStream_t st) {
        gw::SolveArgs ac = a;
        ac.stream = st;
        return gw::solve_launch(ac, c->ws, c->ws_bytes);
      },
      "gw_solve");
}

gw_status gw_barycenter(gw_ctx* c, const gw_barycenter_problem* p, const int* n, const double* h,
                        const double* lambda, const double* const* d_ps, const double* d_p, void* d_C,
                        double* d_stats, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (!p) return fail(c, GW_ERR_INVALID, "gw_barycenter: problem descriptor is NULL");
  if (p->count < 1 || p->count > 64) return fail(c, GW_ERR_INVALID, "gw_barycenter: count must be in [1, 64]");
  if (p->N < 1 || p->N > 4096) return fail(c, GW_ERR_INVALID, "gw_barycenter: N must be in [1, 4096]");
  if (p->k != 1 && p->k != 2) return fail(c, GW_ERR_INVALID, "gw_barycenter: k must be 1 or 2");
  if (p->dtype != GW_F32 && p->dtype != GW_F64)
    return fail(c, GW_ERR_INVALID, "gw_barycenter: dtype must be GW_F32 or GW_F64");
  if (!finite_pos(p->eps) || p->n_iter < 1 || p->n_outer < 1 || p->n_inner < 1)
    return fail(c, GW_ERR_INVALID, "gw_barycenter: need eps > 0 and n_iter, n_outer, n_inner >= 1");
  if (!n || !h || !lambda || !d_ps || !d_p || !d_C)
    return fail(c, GW_ERR_INVALID, "gw_barycenter: n, h, lambda, d_ps, d_p and d_C must not be NULL");
  double wsum = 0.0;
  const int nmax = p->dtype == GW_F64 ? gw::kMaxSolveF64Y : 16384;
  for (int s = 0; s < p->count; ++s) {
    if (n[s] < 1 || n[s] > nmax) return fail(c, GW_ERR_INVALID, "gw_barycenter: n[%d] must be in [1, %d]", s, nmax);
    if (!finite_pos(h[s])) return fail(c, GW_ERR_INVALID, "gw_barycenter: h[%d] must be finite and > 0", s);
    if (!std::isfinite(lambda[s]) || lambda[s] < 0.0)
      return fail(c, GW_ERR_INVALID, "gw_barycenter: lambda[%d] must be finite and >= 0", s);
    if (!d_ps[s]) return fail(c, GW_ERR_INVALID, "gw_barycenter: d_ps[%d] is NULL", s);
    wsum += lambda[s];
  }
  if (!(wsum > 0.0)) return fail(c, GW_ERR_INVALID, "gw_barycenter: the weights must have a positive sum");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GW_ERR_CUDA, "cudaSetDevice failed");
  const std::vector<int> nv(n, n + p->count);
  const std::vector<double> hv(h, h + p->count), lv(lambda, lambda + p->count);
  const std::vector<const double*> pv(d_ps, d_ps + p->count);
  gw::BarycenterArgs a{};
  a.count = p->count;
  a.N = p->N;
  a.k = p->k;
  a.dtype = p->dtype;
  a.n = nv.data();
  a.h = hv.data();
  a.lambda = lv.data();
  a.ps = pv.data();
  a.p = d_p;
  a.C = d_C;
  a.values = d_stats;
  a.eps = p->eps;
  a.n_iter = p->n_iter;
  a.n_outer = p->n_outer;
  a.n_inner = p->n_inner;
  a.stream = (cudaStream_t)stream;
  a.status = c->status;
  a.num_sms = c->num_sms;
  a.tracer = c->tr();
  gw_status s = ensure_ws(c, gw::barycenter_workspace_bytes(a));
  if (s != GW_OK) return s;
  std::string key = "bary ";
  char buf[256];
  snprintf(buf, sizeof buf, "%d %d %d %d %.17g %d %d %d %p %p %p %p %zu|", a.count, a.N, a.k, a.dtype, a.eps, a.n_iter,
           a.n_outer, a.n_inner, (void*)d_p, d_C, (void*)d_stats, c->ws, c->ws_bytes);
  key += buf;
  for (int q = 0; q < a.count; ++q) {
    snprintf(buf, sizeof buf, "%d %.17g %.17g %p|", nv[q], hv[q], lv[q], (void*)pv[q]);
    key += buf;
  }
  return run_graph(
      c, key, a.stream,
      [&](cudaStream_t st) {
        gw::BarycenterArgs ac = a;
        ac.stream = st;
        return gw::barycenter_launch(ac, c->ws, c->ws_bytes);
      },
      "gw_barycenter");
}

gw_status gw_solve_batch(gw_ctx* c, int count, const gw_problem* probs, const double* const* d_u,
                         const double* const* d_v, const double* const* d_phi, const double* const* d_psi,
                         void* const* d_T, double* const* d_stats, void* stream) {
  if (!c) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (count < 0 || (count > 0 && (!probs || !d_u || !d_v || !d_T)))
    return fail(c, GW_ERR_INVALID, "gw_solve_batch: need count >= 0 and the problem and pointer arrays");
  if (count == 0) return GW_OK;
  std::vector<gw::SolveArgs> args(count);
  std::vector<size_t> off(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const double* phi = d_phi ? d_phi[i] : nullptr;
    const double* psi = d_psi ? d_psi[i] : nullptr;
    char who[48];
    snprintf(who, sizeof who, "gw_solve_batch[%d]", i);
    gw_status s = check_solve(c, &probs[i], d_u[i], d_v[i], phi, psi, d_T[i], who);
    if (s != GW_OK) return s;
    args[i] = solve_args(c, &probs[i], d_u[i], d_v[i], phi, psi, d_T[i], nullptr, nullptr,
                         d_stats ? d_stats[i] : nullptr, nullptr);
    args[i].batch = 1;
    off[i] = total;
    total += (gw::solve_workspace_bytes(args[i]) + 4095) / 4096 * 4096;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GW_ERR_CUDA, "cudaSetDevice failed");
  // Mixed sets: problems of one dtype and schedule whose row configurations
  // run 512-thread blocks advance in lock step with every Sinkhorn pass one
  // launch over all of their row bands (each block runs its own problem's
  // configuration).  The other problems form groups of one row
  // configuration (one launch per pass per 32 problems).  Sets and groups
  // run concurrently on worker streams.
  std::map<std::tuple<int, int, int>, std::vector<int>> mixed;
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
  for (int i = 0; i < count; ++i) {
    if (gw::solve_mixable(args[i]))
      mixed[std::make_tuple(args[i].dtype, args[i].n_outer, args[i].n_inner)].push_back(i);
    else
      groups[std::make_tuple(gw::solve_group_key(args[i]), args[i].dtype, args[i].n_outer, args[i].n_inner)]
          .push_back(i);
  }
  std::vector<std::vector<int>> parts;
  for (auto& g : groups) {
    auto& v = g.second;
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
      return (double)args[x].n * args[x].m > (double)args[y].n * args[y].m;
    });
    for (size_t b = 0; b < v.size(); b += 32) parts.emplace_back(v.begin() + b, v.begin() + std::min(v.size(), b + 32));
  }
  // Each mixed set: a device table after the problems' workspaces, a main
  // stream and up to kMixWorkers worker streams.
  constexpr int kMixWorkers = 8;
  std::vector<std::vector<int>> sets;
  std::vector<size_t> table_off;
  for (auto& kv : mixed) {
    auto& v = kv.second;
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
      return (double)args[x].n * args[x].m > (double)args[y].n * args[y].m;
    });
    sets.push_back(v);
    table_off.push_back(total);
    total += (gw::solve_mixed_table_bytes((int)v.size(), args[v[0]].dtype) + 4095) / 4096 * 4096;
  }
  if (total > c->bws_bytes) {
    if (c->bws) {
      cudaDeviceSynchronize();
      cudaFree(c->bws);
      c->bws = nullptr;
      c->bws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->bws, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, GW_ERR_OOM, "gw_solve_batch: workspace of %zu bytes: %s", total, cudaGetErrorString(e));
    }
    c->bws_bytes = total;
  }
  std::vector<int> set_workers(sets.size());
  int S = (int)std::min<size_t>(parts.size(), 32);
  for (size_t j = 0; j < sets.size(); ++j) {
    set_workers[j] = std::min<int>(kMixWorkers, (int)sets[j].size());
    S += 1 + set_workers[j];
  }
  while ((int)c->bstreams.size() < S) {
    cudaStream_t st;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(c, cudaGetLastError(), "gw_solve_batch: worker streams");
    c->bstreams.push_back(st);
    c->join_ev.push_back(ev);
  }
  while (c->mix_ev.size() < sets.size() * (1 + kMixWorkers)) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(c, cudaGetLastError(), "gw_solve_batch: mixed-set events");
    c->mix_ev.push_back(ev);
  }
  if (!c->fork_ev && cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return cuda_fail(c, cudaGetLastError(), "gw_solve_batch: fork event");
  // Arguments, workspaces and device tables of the mixed sets.
  std::vector<std::vector<const gw::SolveArgs*>> set_args(sets.size());
  std::vector<std::vector<void*>> set_ws(sets.size());
  std::vector<std::vector<size_t>> set_wb(sets.size());
  for (size_t j = 0; j < sets.size(); ++j)
    for (int i : sets[j]) {
      set_args[j].push_back(&args[i]);
      set_ws[j].push_back((char*)c->bws + off[i]);
      set_wb[j].push_back(gw::solve_workspace_bytes(args[i]));
    }
  // The tables are written before the solves are enqueued (or captured); a
  // previous batch on this context may still read them, so the device is
  // synchronised first.
  auto write_tables = [&]() -> int {
    if (sets.empty()) return GW_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return GW_ERR_CUDA;
    for (size_t j = 0; j < sets.size(); ++j) {
      const int cnt = (int)sets[j].size();
      std::vector<char> host(gw::solve_mixed_table_bytes(cnt, args[sets[j][0]].dtype));
      int rc = gw::solve_mixed_table(set_args[j].data(), set_ws[j].data(), set_wb[j].data(), cnt, host.data());
      if (rc != GW_OK) return rc;
      if (cudaMemcpy((char*)c->bws + table_off[j], host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return GW_ERR_CUDA;
    }
    return GW_OK;
  };
  auto enqueue = [&](cudaStream_t origin) -> int {
    if (cudaEventRecord(c->fork_ev, origin) != cudaSuccess) return GW_ERR_CUDA;
    for (int k = 0; k < S; ++k)
      if (cudaStreamWaitEvent(c->bstreams[k], c->fork_ev, 0) != cudaSuccess) return GW_ERR_CUDA;
    int next = 0;
    for (size_t j = 0; j < sets.size(); ++j) {
      const int nw = set_workers[j];
      cudaStream_t main = c->bstreams[next];
      const cudaStream_t* workers = c->bstreams.data() + next + 1;
      next += 1 + nw;
      const cudaEvent_t* ev = c->mix_ev.data() + j * (1 + kMixWorkers);
      int rc = gw::solve_mixed_launch(set_args[j].data(), set_ws[j].data(), set_wb[j].data(), (int)sets[j].size(),
                                      (char*)c->bws + table_off[j], main, workers, nw, ev[0], ev + 1);
      if (rc != GW_OK) return rc;
    }
    const int np = S - next;
    for (size_t g = 0; g < parts.size(); ++g) {
      std::vector<gw::SolveArgs> ga;
      std::vector<const gw::SolveArgs*> gp;
      std::vector<void*> gws;
      std::vector<size_t> gb;
      for (int i : parts[g]) {
        ga.push_back(args[i]);
        gws.push_back((char*)c->bws + off[i]);
        gb.push_back(gw::solve_workspace_bytes(args[i]));
      }
      for (auto& a : ga) gp.push_back(&a);
      int rc = gw::solve_group_launch(gp.data(), gws.data(), gb.data(), (int)gp.size(),
                                      c->bstreams[next + (int)(g % np)]);
      if (rc != GW_OK) return rc;
    }
    for (int k = 0; k < S; ++k) {
      if (cudaEventRecord(c->join_ev[k], c->bstreams[k]) != cudaSuccess) return GW_ERR_CUDA;
      if (cudaStreamWaitEvent(origin, c->join_ev[k], 0) != cudaSuccess) return GW_ERR_CUDA;
    }
    return GW_OK;
  };
  int rc;
  if (c->tracer) {
    rc = write_tables();
    if (rc == GW_OK) rc = enqueue((cudaStream_t)stream);
  } else {
    std::string key;
    char buf[512];
    snprintf(buf, sizeof buf, "%d %p %zu %u|", count, c->bws, c->bws_bytes, gw::tune_generation());
    key += buf;
    for (int i = 0; i < count; ++i) {
      const gw::SolveArgs& a = args[i];
      snprintf(buf, sizeof buf,
               "%d %d %d %d %d %d %d %.17g %.17g %.17g %.17g %.17g %.17g %d %d %d %d %p %p %p %p %p %p|", a.dim,
               a.cost, a.n, a.m, a.k, a.ky, a.dtype, a.hx, a.hy, a.eps, a.tau, a.rho, a.theta, a.warm_start, a.n_outer, a.n_inner,
               a.feat_dim, (void*)a.u, (void*)a.v, (void*)a.phi, (void*)a.psi, a.T, (void*)a.stats);
      key += buf;
    }
    if (!c->batch_exec || c->batch_key != key) {
      if (c->batch_exec) {
        cudaGraphExecDestroy(c->batch_exec);
        c->batch_exec = nullptr;
      }
      if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "capture stream");
      rc = write_tables();
      if (rc != GW_OK) return fail(c, (gw_status)rc, "gw_solve_batch: problem tables: %s", gw::last_failure());
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
      rc = enqueue(c->cap);
      e = cudaStreamEndCapture(c->cap, &graph);
      if (rc != GW_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(c, rc != GW_OK ? (gw_status)rc : GW_ERR_CUDA, "gw_solve_batch capture failed");
      }
      e = cudaGraphInstantiate(&c->batch_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        c->batch_exec = nullptr;
        return cuda_fail(c, e, "batch graph instantiate");
      }
      c->batch_key = key;
    }
    rc = cudaGraphLaunch(c->batch_exec, (cudaStream_t)stream) == cudaSuccess ? GW_OK : GW_ERR_CUDA;
  }
  if (rc != GW_OK) {
    cudaError_t e = cudaGetLastError();
    return fail(c, (gw_status)rc, "gw_solve_batch launch failed: %s", cudaGetErrorString(e));
  }
  c->err.clear();
  return GW_OK;
}

}  // extern "C"
