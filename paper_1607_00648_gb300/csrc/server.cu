// Serving: continuous batching of independent solves.
//
// Submitted requests wait in a queue until their hierarchy fits the HBM budget
// (footprint computed from the grid and the options); admitted requests get a
// hierarchy, are set up on a pool of streams, and join a running batch at its next
// step boundary, so work from requests that arrived while others were on the GPU
// overlaps with theirs on the device.  Requests run in three lanes by size (finest
// level under 2^16 DoFs, under 2^20, larger), each a batch on its own stream at its
// own priority (the smallest highest) and with its own stepping thread: a lane of small
// problems takes many short steps while a step of larger problems is still on the GPU,
// so a small request is held neither to the pace of the largest ones nor to that of
// mid-sized ones, nor to the host work of another lane's re-forms.  After every step of a lane (an FP64 cycle, or a
// refinement step with its inner FP32 cycles) its converged requests retire: their
// statistics are recorded, their hierarchy is released and its budget returns to the
// queue.  The per-request arithmetic is that of a batch, so a request's result does
// not depend on which other requests shared its steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
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
  int lane = 0;   // 0 small, 1 mid-sized, 2 large problems
  // done but still a member of its lane's batch (inactive there): its hierarchy and
  // budget are released when the batch is next re-formed; abandoned: the caller has
  // collected the result meanwhile, so the server deletes the request then
  bool zombie = false, abandoned = false;
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
  std::thread th[3];  // one stepping thread per lane
  // setup streams per lane; a smaller lane's streams (setups and steps) run at a higher
  // priority so that their short kernels are not queued behind larger problems' long ones
  static constexpr int kLanes = 3;
  static constexpr int kSetupStreams = 4;
  cudaStream_t setup_streams[kLanes][kSetupStreams] = {};
  std::atomic<int> next_setup[kLanes] = {0, 0, 0};
  std::vector<Request*> pending;  // set up enqueued, waiting for its event (mu)
  // hierarchy creation and setup enqueue run on one worker thread per lane, so that
  // host-side waits of a creation hold back neither the stepping of running batches
  // nor the small requests behind a large one
  std::deque<Request*> to_create[kLanes];  // admitted, not yet created (mu)
  int creating = 0;                        // requests inside a worker between the two lists (mu)
  static constexpr int kWorkers[kLanes] = {3, 2, 1};  // the small lane's creations run three at a time
  std::thread workers[kLanes][3];
  int prio[kLanes] = {0, 0, 0};            // stream priorities of the lanes (smallest: highest)
  void worker(int lane);
  // a batch of running requests with its own stream; at most one step in flight
  struct Lane {
    Batch* batch = nullptr;
    std::vector<Request*> members;  // requests of the current batch, in batch order
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool in_flight = false;
    Clock::time_point reformed{};
  };
  // a batch is re-formed (new members join, finished ones leave) at most this often
  // while it still has running members: re-forming rebuilds its tables
  static constexpr std::chrono::milliseconds kReformEvery{25};
  static constexpr int64_t kMidDofs = int64_t(1) << 16;    // finest-level DoFs of a mid-sized problem
  static constexpr int64_t kLargeDofs = int64_t(1) << 20;  // finest-level DoFs of a large problem
  Lane lanes[kLanes];

  void loop(int lane);
  void admit(int lane);
  void retire(Request* r, mg_status st, bool release = true);
  void release(Request* r);  // hierarchy and budget of a finished request (mu held)
  bool start_step(Lane& ln, int lane);   // re-form the batch if needed, enqueue a step
  void finish_step(Lane& ln);            // read the states of a completed step, retire
};

void Server::retire(Request* r, mg_status st, bool release_now) {
  r->status = st;
  r->t_done = Clock::now();
  if (r->ev) {
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
  }
  r->state = 3;
  if (release_now)
    release(r);
  else
    r->zombie = true;
}

void Server::release(Request* r) {
  if (r->h) {  // its setup and steps have completed: no device synchronisation needed
    hier_release(r->h);
    r->h = nullptr;
  }
  if (r->footprint) {
    used -= r->footprint;
    r->footprint = 0;
  }
  r->zombie = false;
}

void Server::worker(int lane) {
  cudaSetDevice(device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || !to_create[lane].empty(); });
      if (stop) return;
      r = to_create[lane].front();
      to_create[lane].pop_front();
      ++creating;
    }
    Hier* h = nullptr;
    mg_status st = hier_create(r->grid, opt, prio[lane], &h, false);
    if (st == MG_OK) {
      r->h = h;
      cudaStream_t ss = setup_streams[lane][next_setup[lane]++ % kSetupStreams];
      st = setup_enqueue(*h, r->eps, ss);
      // the setup's status word comes back with it (read at the join without a CUDA call)
      int* status = reinterpret_cast<int*>(h->h_pin + 15);
      if (st == MG_OK &&
          (cudaMemcpyAsync(status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, ss) != cudaSuccess ||
           cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess ||
           cudaEventRecord(r->ev, ss) != cudaSuccess))
        st = MG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(mu);
    --creating;
    if (st != MG_OK)
      retire(r, st);
    else
      pending.push_back(r);
    cv.notify_all();
  }
}

// admission of the queued requests of one lane by the shared HBM budget, in arrival
// order with backfill (a request that does not fit yet keeps its place, later ones that
// fit go ahead of it); mu held
void Server::admit(int lane) {
  bool admitted = false;
  for (auto it = queue.begin(); it != queue.end();) {
    Request* r = *it;
    if (r->lane != lane || used + r->footprint > budget) {
      ++it;
      continue;
    }
    it = queue.erase(it);
    used += r->footprint;
    r->state = 1;
    r->t_admit = Clock::now();
    to_create[r->lane].push_back(r);
    admitted = true;
  }
  if (admitted) cv.notify_all();
}

// One stepping thread per lane: a lane's re-forms (host tables, uploads) and its step
// bookkeeping never hold back another lane's steps.  Each thread admits the queued
// requests of its own lane (by the shared HBM budget, in arrival order with backfill),
// moves its lane's finished setups into the running set, and steps its lane's batch.
void Server::loop(int lane) {
  cudaSetDevice(device);
  Lane& ln = lanes[lane];
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      auto has_work = [&] {
        if (stop) return true;
        for (Request* r : queue)
          if (r->lane == lane && used + r->footprint <= budget) return true;
        for (Request* r : pending)
          if (r->lane == lane) return true;
        for (Request* r : running)
          if (r->lane == lane) return true;
        return !ln.members.empty();
      };
      // pending setups complete without a notification: look again every 100 us
      while (!has_work()) cv.wait_for(lk, std::chrono::microseconds(100));
      if (stop) break;
      admit(lane);
      // requests of this lane whose setup finished join the running set
      std::vector<Request*> still;
      for (Request* r : pending) {
        if (r->lane != lane || cudaEventQuery(r->ev) == cudaErrorNotReady) {
          still.push_back(r);
          continue;
        }
        const mg_status st = setup_status(*r->h, *reinterpret_cast<const int*>(r->h->h_pin + 15));
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
    if (!ln.in_flight && !start_step(ln, lane)) {
      // nothing to step: wait for a setup of this lane or a new request
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    while (cudaEventQuery(ln.done) == cudaErrorNotReady) {
      {
        std::lock_guard<std::mutex> lk(mu);
        if (stop) break;
        admit(lane);  // new requests of the lane start their setups during a long step
      }
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      if (stop) break;
    }
    finish_step(ln);
  }
}

bool Server::start_step(Lane& ln, int lane) {
  std::vector<Request*> now;
  bool joiners = false, members_running = false;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (Request* r : running)
      if (r->lane == lane) {
        now.push_back(r);
        if (std::find(ln.members.begin(), ln.members.end(), r) == ln.members.end()) joiners = true;
      }
    for (Request* r : ln.members) members_running = members_running || r->state == 2;
  }
  const bool reform = (joiners && (!members_running || Clock::now() - ln.reformed >= kReformEvery)) ||
                      (!members_running && !ln.members.empty());
  if (reform) {  // carry the running members' state over, release the finished ones
    const std::vector<Request*> old = ln.members;
    if (ln.batch) {
      std::vector<ProblemState> carried;
      batch_read(*ln.batch, carried, ln.stream);
      for (size_t i = 0; i < old.size(); ++i)
        if (old[i]->state == 2) old[i]->ps = carried[i];
      batch_destroy(ln.batch);
      ln.batch = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      for (Request* r : old)
        if (r->zombie) {
          release(r);
          if (r->abandoned) delete r;
        }
      cv.notify_all();
    }
    ln.members.clear();
    ln.reformed = Clock::now();
    if (now.empty()) return false;
    std::vector<Hier*> hs;
    std::vector<double*> us;
    std::vector<const double*> bs;
    std::vector<ProblemState> init;
    std::vector<int> fresh;
    for (Request* r : now) {
      hs.push_back(r->h);
      us.push_back(r->u);
      bs.push_back(r->b);
      ProblemState ps = r->ps;
      ps.tol = r->tol;
      ps.max_cycles = r->max_cycles;
      init.push_back(ps);
      fresh.push_back(std::find(old.begin(), old.end(), r) == old.end() ? 1 : 0);
    }
    mg_status st = batch_create(hs, &ln.batch, prio[lane], false);
    if (st == MG_OK) batch_set_graph(ln.batch, false);
    if (st == MG_OK) st = batch_begin(*ln.batch, us.data(), bs.data(), init, fresh, ln.stream);
    if (st != MG_OK) {
      std::lock_guard<std::mutex> lk(mu);
      error = std::string("server batch: ") + mg_last_error();
      for (Request* r : now) retire(r, st);
      std::vector<Request*> keep;
      for (Request* r : running)
        if (r->state == 2) keep.push_back(r);
      running.swap(keep);
      if (ln.batch) {
        batch_destroy(ln.batch);
        ln.batch = nullptr;
      }
      cv.notify_all();
      return false;
    }
    ln.members = now;
  } else if (!members_running) {
    return false;
  }
  if (batch_step_enqueue(*ln.batch, ln.stream) != MG_OK || cudaEventRecord(ln.done, ln.stream) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    for (Request* r : ln.members)
      if (r->state == 2) retire(r, MG_ERR_CUDA, false);
    std::vector<Request*> keep;
    for (Request* r : running)
      if (r->state == 2) keep.push_back(r);
    running.swap(keep);
    cv.notify_all();
    return false;
  }
  ln.in_flight = true;
  return true;
}

void Server::finish_step(Lane& ln) {
  ln.in_flight = false;
  std::vector<ProblemState> state;
  const mg_status st = batch_read(*ln.batch, state, ln.stream);
  std::lock_guard<std::mutex> lk(mu);
  bool changed = false;
  for (size_t i = 0; i < ln.members.size(); ++i) {
    Request* r = ln.members[i];
    if (r->state != 2) continue;  // finished at an earlier step, waiting for the re-form
    if (st != MG_OK) {
      retire(r, st, false);
      changed = true;
      continue;
    }
    r->ps = state[i];
    if (!state[i].active) {
      retire(r, status_of(state[i].status), false);
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

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_server_create(size_t hbm_budget_bytes, const mg_options* opt, mg_server** out) {
  if (!out || hbm_budget_bytes == 0) {
    set_error("mg_server_create: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  if (opt && (opt->precision == MG_PREC_MIXED_BPA || opt->smoother != MG_SMOOTH_JACOBI || opt->cycle != MG_CYCLE_V ||
              opt->dynamic_coarsest || opt->tensor_coefficients)) {
    set_error("mg_server_create: the server runs batches: V-cycles, Jacobi smoothing, no bpa codec, a fixed "
              "coarsest level");
    return MG_ERR_UNSUPPORTED;
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
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);  // a numerically lower value is a higher priority
  sv->prio[0] = prio_high;
  sv->prio[1] = prio_high < prio_low ? prio_high + 1 : prio_low;
  sv->prio[2] = prio_low;
  bool ok = true;
  for (int k = 0; k < Server::kLanes && ok; ++k) {
    const int prio = sv->prio[k];
    ok = cudaStreamCreateWithPriority(&sv->lanes[k].stream, cudaStreamNonBlocking, prio) == cudaSuccess &&
         cudaEventCreateWithFlags(&sv->lanes[k].done, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < Server::kSetupStreams && ok; ++i)
      ok = cudaStreamCreateWithPriority(&sv->setup_streams[k][i], cudaStreamNonBlocking, prio) == cudaSuccess;
  }
  if (!ok) {
    delete sv;
    set_error("mg_server_create: cudaStreamCreate failed");
    return MG_ERR_CUDA;
  }
  try {
    for (int k = 0; k < Server::kLanes; ++k) sv->th[k] = std::thread([sv, k] { sv->loop(k); });
    for (int k = 0; k < Server::kLanes; ++k)
      for (int w = 0; w < Server::kWorkers[k]; ++w) sv->workers[k][w] = std::thread([sv, k] { sv->worker(k); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
      sv->cv.notify_all();
    }
    for (auto& t : sv->th)
      if (t.joinable()) t.join();
    for (int k = 0; k < Server::kLanes; ++k)
      for (auto& t : sv->workers[k])
        if (t.joinable()) t.join();
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
  const int64_t nd = g->levels[g->L].n_dofs;
  r->lane = nd >= Server::kLargeDofs ? 2 : nd >= Server::kMidDofs ? 1 : 0;
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
  if (r->zombie)
    r->abandoned = true;  // still a batch member: the server deletes it at the re-form
  else
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
  for (auto& t : sv->th)
    if (t.joinable()) t.join();
  for (int k = 0; k < Server::kLanes; ++k)
    for (auto& t : sv->workers[k])
      if (t.joinable()) t.join();
  cudaSetDevice(sv->device);
  cudaDeviceSynchronize();
  for (int k = 0; k < Server::kLanes; ++k) {
    for (Request* r : sv->lanes[k].members)
      if (r->zombie && r->abandoned) {
        sv->release(r);
        delete r;
      }
    if (sv->lanes[k].batch) batch_destroy(sv->lanes[k].batch);
    if (sv->lanes[k].done) cudaEventDestroy(sv->lanes[k].done);
    if (sv->lanes[k].stream) cudaStreamDestroy(sv->lanes[k].stream);
  }
  for (auto& kv : sv->all) {
    if (kv.second->h) mg_destroy_hier(reinterpret_cast<mg_hier*>(kv.second->h));
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    delete kv.second;
  }
  for (int k = 0; k < Server::kLanes; ++k)
    for (int i = 0; i < Server::kSetupStreams; ++i)
      if (sv->setup_streams[k][i]) cudaStreamDestroy(sv->setup_streams[k][i]);
  delete sv;
}

}  // extern "C"
