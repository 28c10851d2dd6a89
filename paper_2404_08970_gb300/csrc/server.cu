// Request server: many independent (fused) GW solves arriving over time,
// admitted under a device-memory budget and run concurrently.
//
// gw_submit copies a request's inputs into host memory owned by the server
// and returns a ticket at once.  Worker threads (one per slot) take the
// oldest queued request that fits in the free part of the budget (continuous
// admission: a finished request frees its memory and its slot for the next
// one, whatever the shapes).  A request too large for the free budget does
// not block smaller ones behind it, but only for a bounded number of
// bypasses: once the oldest request has been passed over kMaxBypass times,
// nothing else is admitted until it fits, so large requests cannot starve.
// Each worker runs on its own CUDA stream: device buffers from the
// stream-ordered allocator, inputs staged in the worker's page-locked buffer
// and copied asynchronously, the solve (the same launch sequence as
// gw_solve), device-to-host copies of the statistics and, if requested, the
// plan.  gw_poll reports completion, statistics and the latency from
// submission to completion.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gw_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// How often the oldest queued request may be passed over by younger ones
// that fit the free budget before admission waits for it.
constexpr int kMaxBypass = 32;

struct Request {
  uint64_t ticket = 0;
  int bypassed = 0;     // younger requests admitted while this one waited
  gw_problem prob{};
  std::vector<double> u, v, phi, psi;
  void* h_T = nullptr;  // caller's plan buffer, or null
  size_t need = 0;      // device bytes while running
  Clock::time_point submitted, finished;
  gw_status status = GW_NOT_READY;
  double stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

size_t grid_points(int side, int dim) {
  size_t q = 1;
  for (int d = 0; d < dim; ++d) q *= (size_t)side;
  return q;
}
size_t points_x(const gw_problem& p) { return grid_points(p.nx, p.dim); }
size_t points_y(const gw_problem& p) { return grid_points(p.ny, p.dim); }

}  // namespace

struct gw_server {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // queue or budget changed
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  size_t used = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::atomic<long> completed{0};
  std::string last_error;  // text of the last failed request
};

namespace {

// Device bytes one request holds while it runs: inputs, plan, statistics,
// status word and the solve workspace.
size_t request_bytes(const gw::SolveArgs& a, const gw_problem& p) {
  const size_t rb = p.dtype == GW_F32 ? 4 : 8;
  const size_t n = points_x(p), m = points_y(p);
  size_t b = (n + m) * 8 + n * m * rb + 8 * 8 + 256;
  if (p.theta != 1.0) b += (n + m) * (size_t)p.feat_dim * 8;
  return b + gw::solve_workspace_bytes(a) + 8 * 256;
}

gw::SolveArgs args_for(const gw_server* s, const gw_problem& p) {
  gw::SolveArgs a{};
  a.dim = p.dim;
  a.cost = p.cost;
  a.nx = p.nx;
  a.ny = p.ny;
  a.n = (int)points_x(p);
  a.m = (int)points_y(p);
  a.k = p.k;
  a.dtype = p.dtype;
  a.hx = p.hx;
  a.hy = p.hy;
  a.eps = p.eps;
  a.tau = p.tau > 0.0 ? p.tau : p.eps;
  a.warm_start = p.warm_start;
  a.rho = p.rho;
  a.ky = p.ky == p.k ? 0 : p.ky;
  a.theta = p.theta;
  a.n_outer = p.n_outer;
  a.n_inner = p.n_inner;
  a.feat_dim = p.theta != 1.0 ? p.feat_dim : 0;
  a.num_sms = s->num_sms;
  return a;
}

// Page-locked staging buffer of one worker, grown on demand, so that the
// input copies are truly asynchronous.
struct Staging {
  double* p = nullptr;
  size_t cap = 0;  // doubles
  ~Staging() {
    if (p) cudaFreeHost(p);
  }
  double* get(size_t count) {
    if (count <= cap) return p;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaMallocHost((void**)&p, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return nullptr;
    }
    cap = count;
    return p;
  }
};

// Runs one request on `st`; returns its status and, on failure, a message.
gw_status run_request(gw_server* s, Request& r, cudaStream_t st, unsigned* d_status, Staging* stage,
                      std::string* msg) {
  gw::SolveArgs a = args_for(s, r.prob);
  const size_t n = a.n, m = a.m;
  const size_t rb = r.prob.dtype == GW_F32 ? 4 : 8;
  const size_t ws_bytes = gw::solve_workspace_bytes(a);
  char* base = nullptr;
  cudaGetLastError();  // start from a clean error state on this thread
  cudaError_t me = cudaMallocAsync((void**)&base, r.need, st);
  if (me != cudaSuccess) {
    cudaGetLastError();
    *msg = std::string("device allocation: ") + cudaGetErrorString(me);
    return GW_ERR_OOM;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off = (off + bytes + 255) / 256 * 256;
    return p;
  };
  double* du = (double*)take(n * 8);
  double* dv = (double*)take(m * 8);
  double* dphi = nullptr;
  double* dpsi = nullptr;
  if (a.feat_dim > 0) {
    dphi = (double*)take(n * a.feat_dim * 8);
    dpsi = (double*)take(m * a.feat_dim * 8);
  }
  void* dT = take(n * m * rb);
  double* dstats = (double*)take(8 * 8);
  void* ws = take(ws_bytes);
  // Inputs go through the page-locked staging buffer (the previous request's
  // copies out of it finished with that request's stream synchronisation).
  const size_t nin = n + m + (a.feat_dim > 0 ? (n + m) * (size_t)a.feat_dim : 0);
  double* h = stage->get(nin);
  if (h) {
    memcpy(h, r.u.data(), n * 8);
    memcpy(h + n, r.v.data(), m * 8);
    if (a.feat_dim > 0) {
      memcpy(h + n + m, r.phi.data(), n * a.feat_dim * 8);
      memcpy(h + n + m + n * a.feat_dim, r.psi.data(), m * a.feat_dim * 8);
    }
    cudaMemcpyAsync(du, h, n * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dv, h + n, m * 8, cudaMemcpyHostToDevice, st);
    if (a.feat_dim > 0) {
      cudaMemcpyAsync(dphi, h + n + m, n * a.feat_dim * 8, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(dpsi, h + n + m + n * a.feat_dim, m * a.feat_dim * 8, cudaMemcpyHostToDevice, st);
    }
  } else {  // no page-locked memory to be had: copy from the request itself
    cudaMemcpyAsync(du, r.u.data(), n * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dv, r.v.data(), m * 8, cudaMemcpyHostToDevice, st);
    if (a.feat_dim > 0) {
      cudaMemcpyAsync(dphi, r.phi.data(), n * a.feat_dim * 8, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(dpsi, r.psi.data(), m * a.feat_dim * 8, cudaMemcpyHostToDevice, st);
    }
  }
  cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
  a.u = du;
  a.v = dv;
  a.phi = dphi;
  a.psi = dpsi;
  a.T = dT;
  a.stats = dstats;
  a.stream = st;
  a.status = d_status;
  int rc = gw::solve_launch(a, ws, ws_bytes);
  unsigned word = 0;
  if (rc == GW_OK) {
    cudaMemcpyAsync(r.stats, dstats, 8 * 8, cudaMemcpyDeviceToHost, st);
    if (r.h_T) cudaMemcpyAsync(r.h_T, dT, n * m * rb, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&word, d_status, sizeof word, cudaMemcpyDeviceToHost, st);
  }
  const cudaError_t le = cudaGetLastError();
  cudaFreeAsync(base, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (rc != GW_OK) {
    cudaGetLastError();
    *msg = std::string("solve launch: ") + cudaGetErrorString(le) + "; " + gw::last_failure();
    return (gw_status)rc;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *msg = std::string("stream: ") + cudaGetErrorString(e);
    return GW_ERR_CUDA;
  }
  if (word & 1u) return GW_ERR_TIMEOUT;  // status bits of the kernels: 1 timeout, 2 non-finite
  if (word & 2u) return GW_ERR_NONFINITE;
  return GW_OK;
}

// The request to admit next: the oldest one that fits in the free budget,
// except that once the oldest has been bypassed kMaxBypass times only it may
// go.  queue.end() if none can go now.  Called with s->mu held.
std::deque<std::shared_ptr<Request>>::iterator admissible(gw_server* s) {
  const size_t free_bytes = s->budget - s->used;
  if (s->queue.empty()) return s->queue.end();
  if (s->queue.front()->need <= free_bytes) return s->queue.begin();
  if (s->queue.front()->bypassed >= kMaxBypass) return s->queue.end();
  for (auto it = s->queue.begin() + 1; it != s->queue.end(); ++it)
    if ((*it)->need <= free_bytes) return it;
  return s->queue.end();
}

void worker_loop(gw_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  unsigned* d_status = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaMalloc(&d_status, sizeof(unsigned));
  Staging stage;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto pick = s->queue.end();
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        pick = admissible(s);
        return pick != s->queue.end();
      });
      if (s->stop) break;
      r = *pick;
      if (pick != s->queue.begin()) s->queue.front()->bypassed += 1;
      s->queue.erase(pick);
      s->used += r->need;
    }
    std::string msg;
    const gw_status rc = run_request(s, *r, st, d_status, &stage, &msg);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc != GW_OK) s->last_error = "ticket " + std::to_string(r->ticket) + ": " + msg;
      s->used -= r->need;
      r->finished = Clock::now();
      r->status = rc;
    }
    s->completed.fetch_add(1);
    s->cv_work.notify_all();
  }
  if (d_status) cudaFree(d_status);
  if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

gw_status gw_server_create(gw_server** out, int device, size_t hbm_budget_bytes, int max_slots) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 64) return GW_ERR_INVALID;
  *out = nullptr;
  gw::tune_autoload();
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GW_ERR_CUDA;
  }
  gw_server* s = new gw_server();
  s->device = device;
  s->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  // Keep freed stream-ordered allocations in the pool for the next requests.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = hbm_budget_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return GW_OK;
}

void gw_server_destroy(gw_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->queue) r->status = GW_ERR_SHUTDOWN;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

gw_status gw_submit(gw_server* s, const gw_problem* p, const double* h_u, const double* h_v, const double* h_phi,
                    const double* h_psi, void* h_T, uint64_t* ticket) {
  if (!s || !p || !h_u || !h_v || !ticket) return GW_ERR_INVALID;
  const gw_problem& q = *p;
  if (q.dim < 1 || q.dim > 3 || q.nx < 1 || q.ny < 1 || !(q.hx > 0) || !(q.hy > 0) || q.k < 1 ||
      (q.dtype != GW_F32 && q.dtype != GW_F64) || !(q.eps > 0) || !(q.tau == 0.0 || q.tau > 0) ||
      (q.warm_start != 0 && q.warm_start != 1) || !(q.rho == 0.0 || q.rho > 0) ||
      (q.rho > 0 && (q.theta != 1.0 || (q.tau != 0.0 && q.tau != q.eps))) || q.n_outer < 0 || q.n_inner < 1 ||
      !(q.theta >= 0.0 && q.theta <= 1.0))
    return GW_ERR_INVALID;
  if (q.dim == 1 && (q.k > 3 || q.ny > 16384 || !gw::mixed_k_supported(q.k, q.ky, q.ny, q.dtype)))
    return GW_ERR_INVALID;
  if (q.dim >= 2 && q.ky != 0 && q.ky != q.k) return GW_ERR_INVALID;
  if (q.dim == 3 && (!(q.cost == GW_COST_SQEUCLID || (q.cost == GW_COST_POW && q.k == 1)) ||
                     q.nx > gw::kMax3DSide || q.ny > gw::kMax3DSide))
    return GW_ERR_INVALID;
  if (q.dim == 2 && ((q.cost != GW_COST_POW && q.cost != GW_COST_SQEUCLID) || q.nx > gw::kMax2DSide ||
                     q.ny > gw::kMax2DSide ||
                     (q.cost == GW_COST_POW && q.k > 1 && !gw::grad2d_powk_supported(q.nx, q.ny, q.k, q.dtype))))
    return GW_ERR_INVALID;
  if (points_y(q) > 16384 || (q.dtype == GW_F64 && points_y(q) > (size_t)gw::kMaxSolveF64Y)) return GW_ERR_INVALID;
  if (q.theta != 1.0 && (q.feat_dim < 1 || q.feat_dim > 64 || !h_phi || !h_psi)) return GW_ERR_INVALID;
  auto r = std::make_shared<Request>();
  r->prob = q;
  const size_t n = points_x(q), m = points_y(q);
  r->u.assign(h_u, h_u + n);
  r->v.assign(h_v, h_v + m);
  if (q.theta != 1.0) {
    r->phi.assign(h_phi, h_phi + n * q.feat_dim);
    r->psi.assign(h_psi, h_psi + m * q.feat_dim);
  }
  r->h_T = h_T;
  r->need = request_bytes(args_for(s, q), q);
  if (r->need > s->budget) return GW_ERR_INVALID;  // could never be admitted
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return GW_ERR_SHUTDOWN;
    r->ticket = s->next_ticket++;
    r->submitted = Clock::now();
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return GW_OK;
}

gw_status gw_poll(gw_server* s, uint64_t ticket, double* stats, double* latency_s) {
  if (!s) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return GW_ERR_INVALID;
  Request& r = *it->second;
  if (r.status == GW_NOT_READY) return GW_NOT_READY;
  if (stats) memcpy(stats, r.stats, sizeof r.stats);
  if (latency_s) *latency_s = std::chrono::duration<double>(r.finished - r.submitted).count();
  const gw_status st = r.status;
  s->all.erase(it);  // a ticket reports once
  return st;
}

const char* gw_server_last_error(gw_server* s) {
  if (!s) return "no server";
  std::lock_guard<std::mutex> lk(s->mu);
  thread_local std::string copy;
  copy = s->last_error;
  return copy.c_str();
}

gw_status gw_server_info(gw_server* s, long* queued, long* completed, size_t* bytes_in_use) {
  if (!s) return GW_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (long)s->queue.size();
  if (completed) *completed = s->completed.load();
  if (bytes_in_use) *bytes_in_use = s->used;
  return GW_OK;
}

}  // extern "C"
