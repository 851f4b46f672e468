// Serving: continuous batching of independent solves.
//
// A server thread owns one CUDA stream.  Submitted requests wait in a queue until
// their hierarchy fits the HBM budget (footprint computed from the grid and the
// options); admitted requests get a hierarchy, are set up, and join the running
// batch at the next step boundary, so work from requests that arrived while others
// were on the GPU overlaps with theirs on the device.  After every step (an FP64
// cycle, or a refinement step with its inner FP32 cycles) converged requests
// retire: their statistics are recorded, their hierarchy is released and its
// budget returns to the queue.  The per-request arithmetic is that of a batch, so
// a request's result does not depend on which other requests shared its steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hier.h"

namespace mg {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  const Grid* grid = nullptr;
  const double* eps = nullptr;
  const double* b = nullptr;
  double* u = nullptr;
  double tol = 1e-8;
  int max_cycles = 500;
  size_t footprint = 0;
  Hier* h = nullptr;
  int state = 0;  // 0 queued, 1 setting up, 2 running, 3 done
  cudaEvent_t ev = nullptr;  // completion of the request's setup
  ProblemState ps{};
  mg_status status = MG_OK;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct Server {
  size_t budget = 0, used = 0;
  mg_options opt{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::string error;
  std::thread th;
  cudaStream_t stream = nullptr;
  static constexpr int kSetupStreams = 8;
  cudaStream_t setup_streams[kSetupStreams] = {};
  int next_setup = 0;
  std::vector<Request*> pending;  // setting up (server thread only)
  Batch* batch = nullptr;
  std::vector<Request*> members;  // requests of the current batch, in batch order

  void loop();
  void retire(Request* r, mg_status st);
};

void Server::retire(Request* r, mg_status st) {
  r->status = st;
  r->t_done = Clock::now();
  if (r->ev) {
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
  }
  if (r->h) {
    mg_destroy_hier(reinterpret_cast<mg_hier*>(r->h));
    r->h = nullptr;
  }
  used -= r->footprint;
  r->state = 3;
}

void Server::loop() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || !queue.empty() || !running.empty() || !pending.empty(); });
      if (stop) break;
      // admission by HBM footprint, in arrival order
      while (!queue.empty() && used + queue.front()->footprint <= budget) {
        Request* r = queue.front();
        queue.pop_front();
        used += r->footprint;
        r->state = 1;
        r->t_admit = Clock::now();
        admitted.push_back(r);
      }
    }
    // hierarchies of the admitted requests; their setups run concurrently on a pool of
    // streams, overlapping each other and the running batch
    for (Request* r : admitted) {
      mg_hier* h = nullptr;
      mg_status st = mg_hier_create(reinterpret_cast<const mg_grid*>(r->grid), &opt, &h);
      if (st == MG_OK) {
        r->h = reinterpret_cast<Hier*>(h);
        cudaStream_t ss = setup_streams[next_setup++ % kSetupStreams];
        st = setup_enqueue(*r->h, r->eps, ss);
        if (st == MG_OK && (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventRecord(r->ev, ss) != cudaSuccess))
          st = MG_ERR_CUDA;
      }
      if (st != MG_OK) {
        std::lock_guard<std::mutex> lk(mu);
        retire(r, st);
        cv.notify_all();
        continue;
      }
      pending.push_back(r);
    }
    // requests whose setup finished join the running set
    {
      std::vector<Request*> still;
      bool any_running;
      {
        std::lock_guard<std::mutex> lk(mu);
        any_running = !running.empty();
      }
      for (size_t i = 0; i < pending.size(); ++i) {
        Request* r = pending[i];
        cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady && !any_running && still.empty()) q = cudaEventSynchronize(r->ev);
        if (q == cudaErrorNotReady) {
          still.push_back(r);
          continue;
        }
        int status = 0;
        if (q == cudaSuccess) cudaMemcpy(&status, r->h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
        const mg_status st = q == cudaSuccess ? setup_status(*r->h, status) : MG_ERR_CUDA;
        std::lock_guard<std::mutex> lk(mu);
        if (st != MG_OK) {
          retire(r, st);
          cv.notify_all();
        } else {
          r->state = 2;
          running.push_back(r);
        }
      }
      pending.swap(still);
    }
    // re-form the batch when its membership changed, carrying the state over
    std::vector<Request*> now;
    {
      std::lock_guard<std::mutex> lk(mu);
      now = running;
    }
    if (now.empty()) continue;
    if (now != members) {
      std::vector<ProblemState> carried;
      if (batch) {
        batch_read(*batch, carried, stream);
        for (size_t i = 0; i < members.size(); ++i) members[i]->ps = carried[i];
        batch_destroy(batch);
        batch = nullptr;
      }
      std::vector<Hier*> hs;
      std::vector<double*> us;
      std::vector<const double*> bs;
      std::vector<ProblemState> init;
      std::vector<int> fresh;
      for (Request* r : now) {
        hs.push_back(r->h);
        us.push_back(r->u);
        bs.push_back(r->b);
        const bool is_new = std::find(members.begin(), members.end(), r) == members.end();
        ProblemState ps = r->ps;
        ps.tol = r->tol;
        ps.max_cycles = r->max_cycles;
        init.push_back(ps);
        fresh.push_back(is_new ? 1 : 0);
      }
      mg_status st = batch_create(hs, &batch);
      if (st == MG_OK) batch_set_graph(batch, false);
      if (st == MG_OK) st = batch_begin(*batch, us.data(), bs.data(), init, fresh, stream);
      if (st != MG_OK) {
        std::lock_guard<std::mutex> lk(mu);
        error = std::string("server batch: ") + mg_last_error();
        for (Request* r : now) retire(r, st);
        running.clear();
        members.clear();
        if (batch) {
          batch_destroy(batch);
          batch = nullptr;
        }
        cv.notify_all();
        continue;
      }
      members = now;
    }
    int n_active = 0;
    mg_status st = batch_run(*batch, 1, stream, &n_active);
    std::vector<ProblemState> state;
    if (st == MG_OK) st = batch_read(*batch, state, stream);
    std::lock_guard<std::mutex> lk(mu);
    bool changed = false;
    for (size_t i = 0; i < members.size(); ++i) {
      Request* r = members[i];
      if (st != MG_OK) {
        retire(r, st);
        changed = true;
        continue;
      }
      r->ps = state[i];
      if (!state[i].active) {
        retire(r, status_of(state[i].status));
        changed = true;
      }
    }
    if (changed) {
      std::vector<Request*> keep;
      for (Request* r : running)
        if (r->state == 2) keep.push_back(r);
      running.swap(keep);
      cv.notify_all();
    }
  }
}

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_server_create(size_t hbm_budget_bytes, const mg_options* opt, mg_server** out) {
  if (!out || hbm_budget_bytes == 0) {
    set_error("mg_server_create: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  Server* sv = new (std::nothrow) Server();
  if (!sv) {
    set_error("mg_server_create: out of host memory");
    return MG_ERR_OOM;
  }
  sv->budget = hbm_budget_bytes;
  if (opt)
    sv->opt = *opt;
  else
    mg_default_options(&sv->opt);
  cudaGetDevice(&sv->device);
  bool ok = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < Server::kSetupStreams && ok; ++i)
    ok = cudaStreamCreateWithFlags(&sv->setup_streams[i], cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    delete sv;
    set_error("mg_server_create: cudaStreamCreate failed");
    return MG_ERR_CUDA;
  }
  try {
    sv->th = std::thread([sv] { sv->loop(); });
  } catch (...) {
    cudaStreamDestroy(sv->stream);
    delete sv;
    set_error("mg_server_create: thread start failed");
    return MG_ERR_OOM;
  }
  *out = reinterpret_cast<mg_server*>(sv);
  return MG_OK;
}

mg_status mg_server_submit(mg_server* server, const mg_request* req, uint64_t* ticket) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || !req || !ticket || !req->grid || !req->eps || !req->b || !req->u || !(req->rel_tol >= 0.0) ||
      req->max_cycles < 0) {
    set_error("mg_server_submit: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  const Grid* g = reinterpret_cast<const Grid*>(req->grid);
  if (!g->uniform || sv->opt.coarsest_level >= g->L) {
    set_error("mg_server_submit: the grid needs a uniform hierarchy above the coarsest level");
    return MG_ERR_UNSUPPORTED;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) {
    set_error("mg_server_submit: out of host memory");
    return MG_ERR_OOM;
  }
  r->grid = g;
  r->eps = req->eps;
  r->b = req->b;
  r->u = req->u;
  r->tol = req->rel_tol;
  r->max_cycles = req->max_cycles;
  r->footprint = hier_footprint(*g, sv->opt);
  if (r->footprint > sv->budget) {
    delete r;
    set_error("mg_server_submit: the request's hierarchy (" + std::to_string(hier_footprint(*g, sv->opt)) +
              " bytes) exceeds the server's HBM budget");
    return MG_ERR_BUDGET;
  }
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next_ticket++;
  sv->all[r->ticket] = r;
  sv->queue.push_back(r);
  *ticket = r->ticket;
  sv->cv.notify_all();
  return MG_OK;
}

mg_status mg_server_poll(mg_server* server, uint64_t ticket, int wait, int* done, mg_solve_stats* stats) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || !done) {
    set_error("mg_server_poll: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) {
    set_error("mg_server_poll: unknown ticket");
    return MG_ERR_INVALID_ARG;
  }
  Request* r = it->second;
  if (wait) sv->cv.wait(lk, [&] { return r->state == 3 || sv->stop; });
  *done = r->state == 3 ? 1 : 0;
  if (!*done) return MG_OK;
  if (stats) {
    stats->cycles = r->ps.cycles;
    stats->outer_steps = r->ps.cycles;
    stats->r0_norm = r->ps.r0;
    stats->rel_residual = r->ps.rel;
    stats->solve_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    stats->history_len = 0;
  }
  const mg_status st = r->status;
  sv->all.erase(it);
  delete r;
  if (st != MG_OK) set_error("mg_server_poll: the request did not converge");
  return st;
}

mg_status mg_server_info(mg_server* server, int64_t* queued, int64_t* running, size_t* bytes_in_use) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv) {
    set_error("mg_server_info: NULL server");
    return MG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (queued) *queued = static_cast<int64_t>(sv->queue.size());
  if (running) *running = static_cast<int64_t>(sv->running.size());
  if (bytes_in_use) *bytes_in_use = sv->used;
  return MG_OK;
}

void mg_server_destroy(mg_server* server) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  cudaSetDevice(sv->device);
  if (sv->batch) batch_destroy(sv->batch);
  cudaDeviceSynchronize();
  for (auto& kv : sv->all) {
    if (kv.second->h) mg_destroy_hier(reinterpret_cast<mg_hier*>(kv.second->h));
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    delete kv.second;
  }
  cudaStreamDestroy(sv->stream);
  for (int i = 0; i < Server::kSetupStreams; ++i)
    if (sv->setup_streams[i]) cudaStreamDestroy(sv->setup_streams[i]);
  delete sv;
}

}  // extern "C"
