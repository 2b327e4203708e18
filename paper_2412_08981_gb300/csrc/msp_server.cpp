// Serving layer of the msp library: continuous batching of per-parameter
// solves over resident hierarchies (see msp.h, msp_server_*).
//
// Each slot = one instance of one hierarchy + one CUDA stream + one host
// thread that runs the whole per-parameter path for a request.  Slots start
// on demand while the device-memory budget allows another instance; any idle
// slot of a hierarchy takes the oldest queued request of that hierarchy, so
// requests that arrive while others run are admitted as soon as a slot (and
// memory) is free and their device work overlaps.
#include <cuda_runtime_api.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "msp.h"

namespace msp {
int fail(int code, const std::string& msg);
}

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  uint64_t id = 0;
  int hid = 0;
  double mu[8] = {0};
  int n_mu = 0;
  double rtol = 1e-8;
  std::vector<double> x;
  msp_stats st{};
  int status = MSP_PENDING;
  bool done = false;
  Clock::time_point t_submit, t_start, t_done;
};

struct Slot {
  msp_instance* inst = nullptr;
  cudaStream_t stream = nullptr;
  std::thread th;
};

struct Entry {
  msp_hierarchy* h = nullptr;
  int n_nodes = 0;
  size_t inst_bytes = 0;
  std::deque<Request*> queue;
  std::vector<std::unique_ptr<Slot>> slots;
  int idle = 0;  // slots waiting for work
};

}  // namespace

struct msp_server {
  msp_server_opts opt{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::unique_ptr<Entry>> hs;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_id = 1;
  size_t used_bytes = 0;
  bool stop = false;
};

namespace {

// Runs one request on a slot: assemble for mu, factor, FGMRES, copy back.
void run_request(msp_server* srv, Entry& E, Slot& S, Request* r) {
  msp_stats st{};
  int rc = MSP_OK;
  if (!S.inst) rc = msp_assemble(E.h, r->mu, r->n_mu, S.stream, &S.inst);
  if (rc == MSP_OK) rc = msp_solve_host(S.inst, r->mu, r->n_mu, nullptr, r->x.data(), r->rtol, &st);
  std::lock_guard<std::mutex> lk(srv->mu);
  r->st = st;
  r->status = rc;
  if (rc != MSP_OK) r->st.status = rc;
  r->t_done = Clock::now();
  r->done = true;
  srv->cv_done.notify_all();
}

void worker(msp_server* srv, Entry* E, Slot* S) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    E->idle++;
    srv->cv_work.wait(lk, [&] { return srv->stop || !E->queue.empty(); });
    E->idle--;
    if (srv->stop) return;
    Request* r = E->queue.front();
    E->queue.pop_front();
    r->t_start = Clock::now();
    lk.unlock();
    run_request(srv, *E, *S, r);
    lk.lock();
  }
}

// Starts another slot for E if the budget allows (called with srv->mu held).
bool try_add_slot(msp_server* srv, Entry* E) {
  if ((int)E->slots.size() >= srv->opt.slots_per_hierarchy) return false;
  if (srv->opt.mem_budget_bytes && srv->used_bytes + E->inst_bytes > srv->opt.mem_budget_bytes)
    return false;
  std::unique_ptr<Slot> S(new Slot());
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  srv->used_bytes += E->inst_bytes;
  Slot* raw = S.get();
  E->slots.push_back(std::move(S));
  raw->th = std::thread(worker, srv, E, raw);
  return true;
}

}  // namespace

extern "C" {

void msp_server_default_options(msp_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->slots_per_hierarchy = 4;
  o->mem_budget_bytes = 0;
  o->rtol_default = 1e-8;
}

int msp_server_create(const msp_server_opts* o, msp_server** out) {
  if (!o || !out) return msp::fail(MSP_ERR_INVALID, "NULL argument");
  if (o->slots_per_hierarchy < 1 || o->slots_per_hierarchy > 64)
    return msp::fail(MSP_ERR_INVALID, "slots_per_hierarchy must be in 1..64");
  std::unique_ptr<msp_server> srv(new msp_server());
  srv->opt = *o;
  if (!(srv->opt.rtol_default > 0)) srv->opt.rtol_default = 1e-8;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    cudaGetLastError();
    return msp::fail(MSP_ERR_CUDA, "cudaGetDevice failed");
  }
  *out = srv.release();
  return MSP_OK;
}

int msp_server_add_hierarchy(msp_server* srv, msp_hierarchy* h, int* id) {
  if (!srv || !h || !id) return msp::fail(MSP_ERR_INVALID, "NULL argument");
  std::unique_ptr<Entry> E(new Entry());
  E->h = h;
  int rc = msp_instance_bytes(h, &E->inst_bytes);
  if (rc) return rc;
  msp_level_info info;
  rc = msp_hierarchy_info(h, 0, &info);
  if (rc) return rc;
  E->n_nodes = info.n_dofs;  // solution length
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->opt.mem_budget_bytes && E->inst_bytes > srv->opt.mem_budget_bytes)
    return msp::fail(MSP_ERR_OOM, "one instance of this hierarchy exceeds the server budget");
  *id = (int)srv->hs.size();
  srv->hs.push_back(std::move(E));
  return MSP_OK;
}

int msp_submit(msp_server* srv, int hierarchy_id, const double* mu, int n_mu, double rtol,
               uint64_t* req_id) {
  if (!srv || !req_id) return msp::fail(MSP_ERR_INVALID, "NULL argument");
  if (n_mu < 0 || n_mu > 8 || (n_mu > 0 && !mu)) return msp::fail(MSP_ERR_INVALID, "n_mu must be 0..8");
  std::unique_ptr<Request> r(new Request());
  for (int j = 0; j < n_mu; ++j) r->mu[j] = mu[j];
  r->n_mu = n_mu;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (hierarchy_id < 0 || hierarchy_id >= (int)srv->hs.size())
    return msp::fail(MSP_ERR_INVALID, "unknown hierarchy id");
  Entry* E = srv->hs[hierarchy_id].get();
  r->id = srv->next_id++;
  r->hid = hierarchy_id;
  r->rtol = rtol > 0 ? rtol : srv->opt.rtol_default;
  r->x.assign(E->n_nodes, 0.0);
  r->t_submit = Clock::now();
  E->queue.push_back(r.get());
  *req_id = r->id;
  srv->reqs[r->id] = std::move(r);
  // admission: add a slot when none is idle and the budget has room
  if (E->idle < (int)E->queue.size()) try_add_slot(srv, E);
  if (E->slots.empty()) {
    E->queue.pop_back();
    srv->reqs.erase(*req_id);
    return msp::fail(MSP_ERR_OOM, "the memory budget cannot hold an instance of this hierarchy");
  }
  srv->cv_work.notify_all();
  return MSP_OK;
}

int msp_poll(msp_server* srv, uint64_t req_id, double* x_host, msp_stats* st, int timeout_ms) {
  if (!srv) return msp::fail(MSP_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) return msp::fail(MSP_ERR_INVALID, "unknown request id");
  Request* r = it->second.get();
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
  else if (timeout_ms > 0) srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  if (!r->done) {
    if (st) {
      std::memset(st, 0, sizeof(*st));
      st->status = MSP_PENDING;
    }
    return MSP_PENDING;
  }
  if (x_host) std::memcpy(x_host, r->x.data(), r->x.size() * sizeof(double));
  if (st) {
    *st = r->st;
    st->ms_queue = ms_between(r->t_submit, r->t_start);
    st->ms_total = ms_between(r->t_submit, r->t_done);
  }
  const int status = r->status;
  srv->reqs.erase(it);
  if (status != MSP_OK) msp::fail(status, "request failed (see msp_stats.status)");
  return status;
}

void msp_server_free(msp_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& E : srv->hs)
    for (auto& S : E->slots)
      if (S->th.joinable()) S->th.join();
  for (auto& E : srv->hs)
    for (auto& S : E->slots) {
      if (S->inst) msp_free_instance(S->inst);
      if (S->stream) cudaStreamDestroy(S->stream);
    }
  delete srv;
}

}  // extern "C"
