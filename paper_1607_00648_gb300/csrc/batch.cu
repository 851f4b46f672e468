// Batched solves of many independent problems of uneven sizes (host driver).
//
// All problems advance through their V-cycles in lockstep, aligned by depth below
// their own finest level: the phase "pre-smoothing at depth j" smooths level
// L_p - j of every problem p that has such a level above its coarsest level.
// Each phase is one launch per brick edge over a work list that holds the items of
// every problem (brick sweeps, slot chunks of transfers), so a phase carries the
// work of the whole batch.  Per-problem convergence flags retire finished
// problems on the device: every item of an inactive problem returns at once, so a
// captured cycle graph stays valid while the batch drains.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "batch_kernels.cuh"
#include "batch_persist.cuh"
#include "hier.h"

namespace mg {

template <>
void blaunch_sweep<2, double>(const BatchArgs<double>&, const BatchGroup&, int, int, int, int, cudaStream_t);
template <>
void blaunch_sweep<3, double>(const BatchArgs<double>&, const BatchGroup&, int, int, int, int, cudaStream_t);
template <>
void blaunch_sweep<2, float>(const BatchArgs<float>&, const BatchGroup&, int, int, int, int, cudaStream_t);
template <>
void blaunch_sweep<3, float>(const BatchArgs<float>&, const BatchGroup&, int, int, int, int, cudaStream_t);
template <>
cudaError_t bpersist_launch<2>(const QueueArgs&, int, int, int, int, cudaStream_t);
template <>
cudaError_t bpersist_launch<3>(const QueueArgs&, int, int, int, int, cudaStream_t);
template <>
void blaunch_transfer<2, double>(const BatchArgs<double>&, const BatchGroup&, bool, int, cudaStream_t);
template <>
void blaunch_transfer<3, double>(const BatchArgs<double>&, const BatchGroup&, bool, int, cudaStream_t);
template <>
void blaunch_transfer<2, float>(const BatchArgs<float>&, const BatchGroup&, bool, int, cudaStream_t);
template <>
void blaunch_transfer<3, float>(const BatchArgs<float>&, const BatchGroup&, bool, int, cudaStream_t);

namespace {

// per-problem convergence test from the partial sums of the norm phase
__global__ void k_bcheck(BatchState s) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < s.n) bcheck_one(s, p);
}

__global__ void k_breset(int* n_active) { *n_active = 0; }

// finest-level chunk items (p, L, chunk)
__global__ void __launch_bounds__(kBlock) k_bzero(const int4* items, const PLevel<double>* lv64, double* const* u64,
                                                   float* const* e32) {
  const int4 it = items[blockIdx.x];
  const int64_t i = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (i >= lv64[it.x * kMaxLevels + it.y].d.n_slots) return;
  u64[it.x][i] = 0.0;
  if (e32) e32[it.x][i] = 0.0f;
}

__global__ void __launch_bounds__(kBlock) k_bzero_masked(const int4* items, const int* mask,
                                                          const PLevel<double>* lv64, double* const* u64,
                                                          float* const* e32) {
  const int4 it = items[blockIdx.x];
  if (!mask[it.x]) return;
  const int64_t i = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (i >= lv64[it.x * kMaxLevels + it.y].d.n_slots) return;
  u64[it.x][i] = 0.0;
  if (e32) e32[it.x][i] = 0.0f;
}

__global__ void __launch_bounds__(kBlock) k_bupdate(const int4* items, const int* active, const PLevel<double>* lv64,
                                                     double* const* u64, float* const* e32, const double* sigma) {
  const int4 it = items[blockIdx.x];
  if (!active[it.x]) return;
  const int64_t i = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (i >= lv64[it.x * kMaxLevels + it.y].d.n_slots) return;
  u64[it.x][i] = fma(sigma[it.x], static_cast<double>(e32[it.x][i]), u64[it.x][i]);
}

__global__ void __launch_bounds__(kBlock) k_bscale(const int4* items, const int* active, const PLevel<double>* lv64,
                                                    float* const* b32, float* const* e32, const double* sigma) {
  const int4 it = items[blockIdx.x];
  if (!active[it.x]) return;
  const PLevel<double>& G = lv64[it.x * kMaxLevels + it.y];
  const int64_t i = static_cast<int64_t>(it.z) * kBlock + threadIdx.x;
  if (i >= G.d.n_slots) return;
  const double sg = sigma[it.x];
  b32[it.x][i] = static_cast<float>(sg > 0.0 ? G.r[i] / sg : 0.0);
  e32[it.x][i] = 0.0f;
}

// coarsest level of every active problem by its FP64 Cholesky factor (one thread each)
template <typename T>
__global__ void k_bcoarse(const PLevel<T>* lv, const int* cp, const int* active, const double* const* chol,
                          const int32_t* const* cslots, const int* nc, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !active[p]) return;
  bcoarse_one<T>(lv, cp, chol, cslots, nc, p);
}

}  // namespace

struct Batch {
  int n = 0, dim = 2, Dmax = 0;
  bool mixed = false;
  int amc64 = 0, pm64 = 0, amc32 = 0, pm32 = 0;
  int nu1 = 2, nu2 = 2, inner = 8;
  double omega = 0.6;
  std::vector<Hier*> H;
  std::vector<void*> allocs;
  PLevel<double>* d_lv64 = nullptr;
  PLevel<float>* d_lv32 = nullptr;
  double** d_u64 = nullptr;
  const double** d_b64 = nullptr;
  float** d_u32 = nullptr;
  float** d_b32 = nullptr;
  int *d_Lp = nullptr, *d_c = nullptr, *d_active = nullptr, *d_cycles = nullptr, *d_status = nullptr;
  int *d_nactive = nullptr, *d_nc = nullptr;
  double *d_r0 = nullptr, *d_rel = nullptr, *d_sigma = nullptr, *d_invc = nullptr, *d_partial = nullptr;
  double* d_tol = nullptr;
  int* d_max = nullptr;
  int2* d_prange = nullptr;
  const double** d_chol = nullptr;
  const int32_t** d_cslots = nullptr;
  int* h_pin = nullptr;
  std::vector<std::vector<BatchGroup>> sw, rs, pr, cp;  // per depth
  std::vector<BatchGroup> fin;                          // finest-level slot chunks
  Graph graph;
  bool use_graph = true;  // the server re-forms batches often and launches steps directly
  BatchState state{};
  // persistent steps (every hierarchy's options.persistent): the step's work queue, its
  // ticket, the per-problem progress counters, the error word and the norm slots
  bool persistent = false;
  QItem* d_queue = nullptr;
  int n_queue = 0;
  unsigned* d_head = nullptr;
  int* d_prog = nullptr;
  int* d_err = nullptr;
  int2* d_prange_q = nullptr;
  cudaStream_t own = nullptr;
  int priority = 0;
  bool blocking = true;
  ~Batch() {  // the caller has made sure no work of the batch is pending
    graph.reset();
    for (void* p : allocs) pool_free(p, own);
    pinned_release(h_pin);
    if (own) cudaStreamDestroy(own);
  }
};

namespace {

template <typename T>
mg_status balloc(Batch& bt, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  void* q = nullptr;
  const cudaError_t e = pool_alloc(&q, n * sizeof(T), bt.own);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("batch: device allocation failed: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
  }
  bt.allocs.push_back(q);
  *p = static_cast<T*>(q);
  return MG_OK;
}

template <typename T>
mg_status bupload(Batch& bt, T** p, const std::vector<T>& v) {
  const mg_status st = balloc(bt, p, v.size());
  if (st != MG_OK) return st;
  if (!v.empty() &&
      cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, bt.own) != cudaSuccess) {
    set_error("batch: upload failed");
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

template <typename T>
PLevel<T> batch_plevel(const Hier& h, int l) {
  const DevLevel& D = h.lv[l];
  PLevel<T> P{};
  P.d = D.d;
  const bool coarse = l < h.top;
  if constexpr (std::is_same<T, double>::value) {
    P.eps = D.eps;
    P.ahat = (coarse && h.galerkin) ? D.ahat : nullptr;
    P.phat = (coarse && h.boxmg) ? D.phat : nullptr;
    P.u = D.u;
    P.b = D.b;
    P.r = D.r;
    P.t = D.t;
  } else {
    P.eps = D.eps32;
    P.ahat = (coarse && h.galerkin) ? D.a16 : nullptr;
    P.ascale = (coarse && h.galerkin) ? D.ascale : nullptr;
    P.phat = (coarse && h.boxmg) ? D.p16 : nullptr;
    P.pscale = (coarse && h.boxmg) ? D.pscale : nullptr;
    P.u = D.u32;
    P.b = D.b32;
    P.r = D.r32;
    P.t = D.t32;
  }
  P.R = D.d.B;  // whole bricks: the batch supplies the parallelism
  P.nitems = static_cast<int>(D.d.n_bricks);
  return P;
}

// groups items by key, uploads them, appends groups (part offsets from `part`)
mg_status make_groups(Batch& bt, std::map<std::pair<int, int>, std::vector<int4>>& by, std::vector<BatchGroup>& out,
                      int* part, bool sweep) {
  for (auto& kv : by) {
    BatchGroup g{};
    if (sweep) {
      g.B = kv.first.first;
    } else {
      g.BC = kv.first.first;
      g.BF = kv.first.second;
    }
    g.count = static_cast<int>(kv.second.size());
    g.part_off = part ? *part : 0;
    if (part) *part += g.count;
    const mg_status st = bupload(bt, &g.items, kv.second);
    if (st != MG_OK) return st;
    out.push_back(g);
  }
  return MG_OK;
}

// Paired smoothing (FP32 V(2,2) cycles, 2D): the groups of brick edge 27 and 9 smooth with two
// sweeps per launch, u -> t before the coarse correction (the residual reads t, the
// prolongation adds into t) and t -> u after it; the other groups sweep one at a time.
template <int DIM, typename T>
static bool emit_paired_cycle(Batch& bt, const BatchArgs<T>& ba, int amc, int pm, cudaStream_t s) {
  if constexpr (DIM == 2 && std::is_same<T, float>::value) {
    if (bt.nu1 != 2 || bt.nu2 != 2) return false;
    BatchArgs<T> nb = ba;
    nb.partial = nullptr;
    nb.pair_t = 1;
    for (int j = 0; j < bt.Dmax; ++j) {
      for (const BatchGroup& g : bt.sw[j])
        if (g.B == 27 || g.B == 9) blaunch_sweep_pair_2d_f32(nb, g, amc, kSelU, kSelT, s);
      for (int k = 0; k < 2; ++k)
        for (const BatchGroup& g : bt.sw[j])
          if (g.B != 27 && g.B != 9) blaunch_sweep<DIM, T>(nb, g, kJacobi, amc, k == 0 ? kSelU : kSelT, k == 0 ? kSelT : kSelU, s);
      for (const BatchGroup& g : bt.sw[j])
        blaunch_sweep<DIM, T>(nb, g, kResidual, amc, (g.B == 27 || g.B == 9) ? kSelT : kSelU, kSelR, s);
      for (const BatchGroup& g : bt.rs[j]) blaunch_transfer<DIM, T>(nb, g, true, pm, s);
    }
    k_bcoarse<T><<<static_cast<unsigned>((bt.n + 127) / 128), 128, 0, s>>>(
        ba.lv, bt.d_c, ba.active, bt.d_chol, bt.d_cslots, bt.d_nc, bt.n);
    for (int j = bt.Dmax - 1; j >= 0; --j) {
      for (const BatchGroup& g : bt.pr[j]) blaunch_transfer<DIM, T>(nb, g, false, pm, s);
      for (const BatchGroup& g : bt.sw[j])
        if (g.B == 27 || g.B == 9) blaunch_sweep_pair_2d_f32(nb, g, amc, kSelT, kSelU, s);
      for (int k = 0; k < 2; ++k)
        for (const BatchGroup& g : bt.sw[j])
          if (g.B != 27 && g.B != 9) blaunch_sweep<DIM, T>(nb, g, kJacobi, amc, k == 0 ? kSelU : kSelT, k == 0 ? kSelT : kSelU, s);
    }
    return true;
  }
  return false;
}

template <int DIM, typename T>
void emit_cycle(Batch& bt, const BatchArgs<T>& ba, int amc, int pm, bool first_done, cudaStream_t s) {
  if (!first_done && emit_paired_cycle<DIM, T>(bt, ba, amc, pm, s)) return;
  BatchArgs<T> nb = ba;
  nb.partial = nullptr;
  for (int j = 0; j < bt.Dmax; ++j) {
    int cur = kSelU, oth = kSelT, k0 = 0;
    if (j == 0 && first_done) {
      cur = kSelT;
      oth = kSelU;
      k0 = 1;
    }
    for (int k = k0; k < bt.nu1; ++k) {
      for (const BatchGroup& g : bt.sw[j]) blaunch_sweep<DIM, T>(nb, g, kJacobi, amc, cur, oth, s);
      std::swap(cur, oth);
    }
    if (cur != kSelU)
      for (const BatchGroup& g : bt.cp[j])
        k_bcopy<T><<<static_cast<unsigned>(g.count), kBlock, 0, s>>>(nb, g.items, cur, kSelU);
    for (const BatchGroup& g : bt.sw[j]) blaunch_sweep<DIM, T>(nb, g, kResidual, amc, kSelU, kSelR, s);
    for (const BatchGroup& g : bt.rs[j]) blaunch_transfer<DIM, T>(nb, g, true, pm, s);
  }
  k_bcoarse<T><<<static_cast<unsigned>((bt.n + 127) / 128), 128, 0, s>>>(
      ba.lv, bt.d_c, ba.active, bt.d_chol, bt.d_cslots, bt.d_nc, bt.n);
  for (int j = bt.Dmax - 1; j >= 0; --j) {
    for (const BatchGroup& g : bt.pr[j]) blaunch_transfer<DIM, T>(nb, g, false, pm, s);
    int cur = kSelU, oth = kSelT;
    for (int k = 0; k < bt.nu2; ++k) {
      for (const BatchGroup& g : bt.sw[j]) blaunch_sweep<DIM, T>(nb, g, kJacobi, amc, cur, oth, s);
      std::swap(cur, oth);
    }
    if (cur != kSelU)
      for (const BatchGroup& g : bt.cp[j])
        k_bcopy<T><<<static_cast<unsigned>(g.count), kBlock, 0, s>>>(nb, g.items, cur, kSelU);
  }
}

template <int DIM>
void emit_fp64_step(Batch& bt, const BatchState& st, cudaStream_t s) {
  BatchArgs<double> ba{bt.d_lv64, bt.d_u64, bt.d_b64, bt.d_Lp, bt.d_active, bt.d_partial, bt.omega};
  k_breset<<<1, 1, 0, s>>>(bt.d_nactive);
  for (const BatchGroup& g : bt.sw[0]) blaunch_sweep<DIM, double>(ba, g, kJacobiNorm, bt.amc64, kSelU, kSelT, s);
  k_bcheck<<<static_cast<unsigned>((bt.n + 127) / 128), 128, 0, s>>>(st);
  emit_cycle<DIM, double>(bt, ba, bt.amc64, bt.pm64, true, s);
  cudaMemcpyAsync(bt.h_pin, bt.d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s);
}

template <int DIM>
void emit_mixed_step(Batch& bt, const BatchState& st, cudaStream_t s) {
  BatchArgs<double> b64{bt.d_lv64, bt.d_u64, bt.d_b64, bt.d_Lp, bt.d_active, bt.d_partial, bt.omega};
  BatchArgs<float> b32{bt.d_lv32, bt.d_u32, bt.d_b32, bt.d_Lp, bt.d_active, nullptr, static_cast<float>(bt.omega)};
  k_breset<<<1, 1, 0, s>>>(bt.d_nactive);
  for (const BatchGroup& g : bt.fin)
    k_bupdate<<<static_cast<unsigned>(g.count), kBlock, 0, s>>>(g.items, bt.d_active, bt.d_lv64, bt.d_u64, bt.d_u32,
                                                                  bt.d_sigma);
  for (const BatchGroup& g : bt.sw[0]) blaunch_sweep<DIM, double>(b64, g, kResidual, 0, kSelU, kSelR, s);
  k_bcheck<<<static_cast<unsigned>((bt.n + 127) / 128), 128, 0, s>>>(st);
  for (const BatchGroup& g : bt.fin)
    k_bscale<<<static_cast<unsigned>(g.count), kBlock, 0, s>>>(g.items, bt.d_active, bt.d_lv64, bt.d_b32, bt.d_u32,
                                                                 bt.d_sigma);
  for (int k = 0; k < bt.inner; ++k) emit_cycle<DIM, float>(bt, b32, bt.amc32, bt.pm32, false, s);
  cudaMemcpyAsync(bt.h_pin, bt.d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s);
}

// The queue of one step: every problem's phases in the order of emit_fp64_step /
// emit_mixed_step, merged phase-major (phase k of every problem before phase k + 1 of
// any); an entry's `need` is the number of its problem's entries in earlier phases.
struct QueueBuilder {
  const Batch& bt;
  std::vector<std::vector<std::vector<QItem>>> ph;  // [problem][phase] entries
  std::vector<int2> prange;
  int part = 0;
  explicit QueueBuilder(const Batch& b) : bt(b), ph(b.n), prange(b.n, make_int2(0, 0)) {}
  std::vector<QItem>& phase(int p) {
    ph[p].emplace_back();
    return ph[p].back();
  }
  static int code(int qop, bool f32, int sop = 0, int src = 0, int dst = 0) {
    return qop | (f32 ? 16 : 0) | (sop << 8) | (src << 12) | (dst << 16);
  }
  void sweeps(int p, int l, bool f32, int sop, int src, int dst, bool norm) {
    const LevelDesc& D = bt.H[p]->lv[l].d;
    auto& v = phase(p);
    if (norm) prange[p].x = part;
    for (int64_t b = 0; b < D.n_bricks; ++b)
      v.push_back(QItem{code(kQSweep, f32, sop, src, dst), p, l, static_cast<int>(b), 0, norm ? part++ : -1});
    if (norm) prange[p].y = part;
  }
  void chunks(int p, int l, int qop, bool f32, int src = 0, int dst = 0) {
    const LevelDesc& D = bt.H[p]->lv[l].d;
    auto& v = phase(p);
    for (int64_t c = 0; c < (D.n_slots + kBlock - 1) / kBlock; ++c)
      v.push_back(QItem{code(qop, f32, 0, src, dst), p, l, static_cast<int>(c), 0, -1});
  }
  void single(int p, int qop, bool f32) { phase(p).push_back(QItem{code(qop, f32), p, 0, 0, 0, -1}); }
  // one V-cycle of problem p (emit_cycle's schedule restricted to p)
  void cycle(int p, bool f32, bool first_done) {
    const Hier& h = *bt.H[p];
    const int D = h.L - h.c;
    for (int j = 0; j < D; ++j) {
      const int l = h.L - j;
      int cur = kSelU, oth = kSelT, k0 = 0;
      if (j == 0 && first_done) {
        cur = kSelT;
        oth = kSelU;
        k0 = 1;
      }
      for (int k = k0; k < bt.nu1; ++k) {
        sweeps(p, l, f32, kJacobi, cur, oth, false);
        std::swap(cur, oth);
      }
      if (cur != kSelU) chunks(p, l, kQCopy, f32, cur, kSelU);
      sweeps(p, l, f32, kResidual, kSelU, kSelR, false);
      chunks(p, l - 1, kQRestrict, f32);
    }
    single(p, kQCoarse, f32);
    for (int j = D - 1; j >= 0; --j) {
      const int l = h.L - j;
      chunks(p, l, kQProlong, f32);
      int cur = kSelU, oth = kSelT;
      for (int k = 0; k < bt.nu2; ++k) {
        sweeps(p, l, f32, kJacobi, cur, oth, false);
        std::swap(cur, oth);
      }
      if (cur != kSelU) chunks(p, l, kQCopy, f32, cur, kSelU);
    }
  }
  std::vector<QItem> build() {
    for (int p = 0; p < bt.n; ++p) {
      const int L = bt.H[p]->L;
      if (bt.mixed) {
        chunks(p, L, kQUpdate, false);
        sweeps(p, L, false, kResidual, kSelU, kSelR, true);
        single(p, kQCheck, false);
        chunks(p, L, kQScale, false);
        for (int k = 0; k < bt.inner; ++k) cycle(p, true, false);
      } else {
        sweeps(p, L, false, kJacobiNorm, kSelU, kSelT, true);
        single(p, kQCheck, false);
        cycle(p, false, true);
      }
    }
    std::vector<QItem> out;
    std::vector<int> done(bt.n, 0);
    size_t maxph = 0;
    for (auto& v : ph) maxph = std::max(maxph, v.size());
    for (size_t k = 0; k < maxph; ++k)
      for (int p = 0; p < bt.n; ++p) {
        if (k >= ph[p].size()) continue;
        for (QItem it : ph[p][k]) {
          it.need = done[p];
          out.push_back(it);
        }
        done[p] += static_cast<int>(ph[p][k].size());
      }
    return out;
  }
};

// one persistent step: reset the ticket, the counters and the active count, run the
// queue, bring back the active count and the error word
mg_status persist_step(Batch& bt, cudaStream_t s) {
  QueueArgs q{};
  q.b64 = BatchArgs<double>{bt.d_lv64, bt.d_u64, bt.d_b64, bt.d_Lp, bt.d_active, bt.d_partial, bt.omega};
  if (bt.mixed)
    q.b32 = BatchArgs<float>{bt.d_lv32, bt.d_u32, bt.d_b32, bt.d_Lp, bt.d_active, nullptr,
                             static_cast<float>(bt.omega)};
  q.st = bt.state;
  q.st.prange = bt.d_prange_q;
  q.cp = bt.d_c;
  q.chol = bt.d_chol;
  q.cslots = bt.d_cslots;
  q.nc = bt.d_nc;
  q.items = bt.d_queue;
  q.n_items = bt.n_queue;
  q.head = bt.d_head;
  q.prog = bt.d_prog;
  q.err = bt.d_err;
  if (cudaMemsetAsync(bt.d_head, 0, sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(bt.d_prog, 0, static_cast<size_t>(bt.n) * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(bt.d_nactive, 0, sizeof(int), s) != cudaSuccess) {
    set_error("batch: persistent step reset failed");
    return MG_ERR_CUDA;
  }
  const cudaError_t e = bt.dim == 2 ? bpersist_launch<2>(q, bt.amc64, bt.pm64, bt.amc32, bt.pm32, s)
                                    : bpersist_launch<3>(q, bt.amc64, bt.pm64, bt.amc32, bt.pm32, s);
  if (e != cudaSuccess || cudaMemcpyAsync(bt.h_pin, bt.d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(bt.h_pin + 1, bt.d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
    set_error(std::string("batch: persistent step: ") + cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

mg_status build_batch(Batch& bt) {
  if (cudaStreamCreateWithPriority(&bt.own, bt.blocking ? cudaStreamDefault : cudaStreamNonBlocking, bt.priority) !=
      cudaSuccess) {
    set_error("mg_batch_create: cudaStreamCreate failed");
    return MG_ERR_CUDA;
  }
  const int n = bt.n;
  const Hier& h0 = *bt.H[0];
  bt.dim = h0.dim;
  bt.mixed = h0.mixed;
  bt.nu1 = h0.opt.nu1;
  bt.nu2 = h0.opt.nu2;
  bt.omega = h0.opt.omega;
  bt.inner = h0.opt.inner_cycles > 0 ? h0.opt.inner_cycles : 8;
  bt.amc64 = h0.galerkin ? 1 : 0;
  bt.pm64 = h0.boxmg ? 1 : 0;
  bt.amc32 = h0.galerkin ? (h0.fmt == 1 ? 2 : 3) : 0;
  bt.pm32 = h0.boxmg ? (h0.fmt == 1 ? 2 : 3) : 0;
  for (const Hier* h : bt.H) {
    if (h->dim != bt.dim || h->mixed != bt.mixed || h->galerkin != h0.galerkin || h->boxmg != h0.boxmg ||
        h->fmt != h0.fmt || h->opt.nu1 != bt.nu1 || h->opt.nu2 != bt.nu2 || h->opt.omega != bt.omega) {
      set_error("mg_batch_create: every hierarchy of a batch needs the same dimension and options");
      return MG_ERR_INVALID_ARG;
    }
    if (h->opt.smoother != MG_SMOOTH_JACOBI || h->opt.cycle != MG_CYCLE_V || h->opt.dynamic_coarsest ||
        h->tensor) {
      set_error("mg_batch_create: batches run V-cycles with the Jacobi smoother and a fixed coarsest level only");
      return MG_ERR_UNSUPPORTED;
    }
    if (h->fmt == 4) {
      set_error("mg_batch_create: bpa-coded hierarchies (MG_PREC_MIXED_BPA) are single-problem only");
      return MG_ERR_UNSUPPORTED;
    }
    if (!h->ready || h->adaptive || h->n_c > 64 || h->L >= kMaxLevels) {
      set_error("mg_batch_create: hierarchies must be set up, with at most 64 coarsest DoFs");
      return MG_ERR_INVALID_ARG;
    }
    bt.Dmax = std::max(bt.Dmax, h->L - h->c);
  }
  std::vector<PLevel<double>> lv64(static_cast<size_t>(n) * kMaxLevels);
  std::vector<PLevel<float>> lv32(bt.mixed ? static_cast<size_t>(n) * kMaxLevels : 0);
  std::vector<int> Lp(n), cp(n), nc(n);
  std::vector<double> invc(n);
  std::vector<const double*> chol(n);
  std::vector<const int32_t*> cslots(n);
  std::vector<float*> u32(n), b32(n);
  for (int p = 0; p < n; ++p) {
    const Hier& h = *bt.H[p];
    for (int l = h.c; l <= h.L; ++l) {
      lv64[p * kMaxLevels + l] = batch_plevel<double>(h, l);
      if (bt.mixed) lv32[p * kMaxLevels + l] = batch_plevel<float>(h, l);
    }
    Lp[p] = h.L;
    cp[p] = h.c;
    nc[p] = h.n_c;
    chol[p] = h.c_mat;
    cslots[p] = h.c_slots;
    invc[p] = h.lv[h.L].n_dofs > 0 ? 1.0 / static_cast<double>(h.lv[h.L].n_dofs) : 0.0;
    if (bt.mixed) {
      u32[p] = h.lv[h.L].u32;
      b32[p] = h.lv[h.L].b32;
    }
  }
  mg_status st;
  if ((st = bupload(bt, &bt.d_lv64, lv64)) != MG_OK) return st;
  if (bt.mixed) {
    if ((st = bupload(bt, &bt.d_lv32, lv32)) != MG_OK) return st;
    if ((st = bupload(bt, &bt.d_u32, u32)) != MG_OK) return st;
    if ((st = bupload(bt, &bt.d_b32, b32)) != MG_OK) return st;
  }
  if ((st = bupload(bt, &bt.d_Lp, Lp)) != MG_OK) return st;
  if ((st = bupload(bt, &bt.d_c, cp)) != MG_OK) return st;
  if ((st = bupload(bt, &bt.d_nc, nc)) != MG_OK) return st;
  if ((st = bupload(bt, &bt.d_invc, invc)) != MG_OK) return st;
  if ((st = bupload(bt, &bt.d_chol, chol)) != MG_OK) return st;
  if ((st = bupload(bt, &bt.d_cslots, cslots)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_u64, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_b64, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_active, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_cycles, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_status, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_r0, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_rel, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_sigma, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_nactive, 1)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_tol, n)) != MG_OK) return st;
  if ((st = balloc(bt, &bt.d_max, n)) != MG_OK) return st;

  // work lists, per depth
  bt.sw.assign(bt.Dmax, {});
  bt.rs.assign(bt.Dmax, {});
  bt.pr.assign(bt.Dmax, {});
  bt.cp.assign(bt.Dmax, {});
  int part = 0;
  std::vector<int2> prange(n, make_int2(0, 0));
  for (int j = 0; j < bt.Dmax; ++j) {
    std::map<std::pair<int, int>, std::vector<int4>> sw, rs, pr, cpy;
    for (int p = 0; p < n; ++p) {
      const Hier& h = *bt.H[p];
      const int l = h.L - j;
      if (l <= h.c) continue;
      const LevelDesc& F = h.lv[l].d;
      const LevelDesc& C = h.lv[l - 1].d;
      for (int64_t b = 0; b < F.n_bricks; ++b) sw[{F.B, 0}].push_back(make_int4(p, l, static_cast<int>(b), 0));
      for (int64_t c = 0; c < (C.n_slots + kBlock - 1) / kBlock; ++c)
        rs[{C.B, F.B}].push_back(make_int4(p, l - 1, static_cast<int>(c), 0));
      for (int64_t c = 0; c < (F.n_slots + kBlock - 1) / kBlock; ++c) {
        pr[{C.B, F.B}].push_back(make_int4(p, l, static_cast<int>(c), 0));
        cpy[{0, 0}].push_back(make_int4(p, l, static_cast<int>(c), 0));
      }
    }
    if (j == 0) {  // per-problem ranges of the norm phase (items of a problem are contiguous in its group)
      int off = 0;
      for (auto& kv : sw) {
        int k = 0;
        while (k < static_cast<int>(kv.second.size())) {
          const int p = kv.second[k].x;
          int e = k;
          while (e < static_cast<int>(kv.second.size()) && kv.second[e].x == p) ++e;
          prange[p] = make_int2(off + k, off + e);
          k = e;
        }
        off += static_cast<int>(kv.second.size());
      }
      if ((st = make_groups(bt, sw, bt.sw[0], &part, true)) != MG_OK) return st;
      if ((st = make_groups(bt, cpy, bt.fin, nullptr, false)) != MG_OK) return st;
    } else {
      if ((st = make_groups(bt, sw, bt.sw[j], nullptr, true)) != MG_OK) return st;
    }
    if ((st = make_groups(bt, rs, bt.rs[j], nullptr, false)) != MG_OK) return st;
    if ((st = make_groups(bt, pr, bt.pr[j], nullptr, false)) != MG_OK) return st;
    if ((st = make_groups(bt, cpy, bt.cp[j], nullptr, false)) != MG_OK) return st;
  }
  if ((st = balloc(bt, &bt.d_partial, std::max(part, 1))) != MG_OK) return st;
  if ((st = bupload(bt, &bt.d_prange, prange)) != MG_OK) return st;
  // persistent steps: every hierarchy asks for them and the batch's storage modes have
  // an instantiated queue kernel (BoxMG + Galerkin with BF16 codes, or geometric)
  bool want = true;
  for (const Hier* h : bt.H) want = want && h->opt.persistent;
  const bool modes = (bt.amc64 == 1 && bt.pm64 == 1 && bt.amc32 == 2 && bt.pm32 == 2) ||
                     (bt.amc64 == 0 && bt.pm64 == 0 && bt.amc32 == 0 && bt.pm32 == 0);
  if (want && modes) {
    QueueBuilder qb(bt);
    const std::vector<QItem> q = qb.build();
    if ((st = bupload(bt, &bt.d_queue, q)) != MG_OK) return st;
    if ((st = bupload(bt, &bt.d_prange_q, qb.prange)) != MG_OK) return st;
    if ((st = balloc(bt, &bt.d_head, 1)) != MG_OK) return st;
    if ((st = balloc(bt, &bt.d_prog, n)) != MG_OK) return st;
    if ((st = balloc(bt, &bt.d_err, 1)) != MG_OK) return st;
    if (qb.part > part) {  // the norm slots of the queue
      if ((st = balloc(bt, &bt.d_partial, qb.part)) != MG_OK) return st;
    }
    if (cudaMemsetAsync(bt.d_err, 0, sizeof(int), bt.own) != cudaSuccess) {
      set_error("mg_batch_create: upload failed");
      return MG_ERR_CUDA;
    }
    bt.n_queue = static_cast<int>(q.size());
    bt.persistent = true;
  }
  bt.h_pin = static_cast<int*>(pinned_slot());
  if (!bt.h_pin) {
    set_error("mg_batch_create: pinned host memory unavailable");
    return MG_ERR_OOM;
  }
  if (cudaStreamSynchronize(bt.own) != cudaSuccess) {  // tables in place before other streams use them
    set_error("mg_batch_create: upload failed");
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

}  // namespace

mg_status status_of(int st) {
  return st == 0 ? MG_OK : st == 2 ? MG_ERR_NONFINITE : st == 3 ? MG_ERR_DIVERGED : MG_ERR_NOT_CONVERGED;
}

void batch_set_graph(Batch* bt, bool use_graph) { bt->use_graph = use_graph; }

mg_status batch_create(const std::vector<Hier*>& hs, Batch** out, int priority, bool blocking) {
  *out = nullptr;
  if (hs.empty()) {
    set_error("batch: no problems");
    return MG_ERR_INVALID_ARG;
  }
  Batch* bt = new (std::nothrow) Batch();
  if (!bt) {
    set_error("batch: out of host memory");
    return MG_ERR_OOM;
  }
  bt->n = static_cast<int>(hs.size());
  bt->H = hs;
  bt->priority = priority;
  bt->blocking = blocking;
  const mg_status st = build_batch(*bt);
  if (st != MG_OK) {
    delete bt;
    return st;
  }
  *out = bt;
  return MG_OK;
}

void batch_destroy(Batch* bt) { delete bt; }

// Uploads the pointer tables and per-problem state; problems with fresh[p] start from
// u = 0 (their state is reset), the others continue from `init` (carried over).
mg_status batch_begin(Batch& bt, double* const* u, const double* const* b, const std::vector<ProblemState>& init,
                      const std::vector<int>& fresh, cudaStream_t s) {
  const int n = bt.n;
  std::vector<int> active(n), cycles(n), status(n), mx(n);
  std::vector<double> r0(n), rel(n), sigma(n), tol(n);
  for (int p = 0; p < n; ++p) {
    if (!u[p] || !b[p]) {
      set_error("batch: NULL vector");
      return MG_ERR_INVALID_ARG;
    }
    const ProblemState& ps = init[p];
    active[p] = fresh[p] ? 1 : ps.active;
    cycles[p] = fresh[p] ? 0 : ps.cycles;
    status[p] = fresh[p] ? 1 : ps.status;
    r0[p] = fresh[p] ? -1.0 : ps.r0;
    rel[p] = fresh[p] ? 1.0 : ps.rel;
    sigma[p] = fresh[p] ? 0.0 : ps.sigma;
    tol[p] = ps.tol;
    mx[p] = ps.max_cycles;
  }
  const bool ok =
      cudaMemcpyAsync(bt.d_u64, u, n * sizeof(double*), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_b64, b, n * sizeof(double*), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_active, active.data(), n * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_cycles, cycles.data(), n * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_status, status.data(), n * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_r0, r0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_rel, rel.data(), n * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_sigma, sigma.data(), n * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_tol, tol.data(), n * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess &&
      cudaMemcpyAsync(bt.d_max, mx.data(), n * sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (!ok) {
    set_error("batch: state upload failed");
    return MG_ERR_CUDA;
  }
  // zero the iterates of fresh problems: a temporary active mask that selects them
  std::vector<int> zmask(fresh.begin(), fresh.end());
  int* d_mask = nullptr;
  if (cudaMallocAsync(&d_mask, n * sizeof(int), s) != cudaSuccess) {
    set_error("batch: mask allocation failed");
    return MG_ERR_OOM;
  }
  cudaMemcpyAsync(d_mask, zmask.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
  for (const BatchGroup& g : bt.fin)
    k_bzero_masked<<<static_cast<unsigned>(g.count), kBlock, 0, s>>>(g.items, d_mask, bt.d_lv64, bt.d_u64,
                                                                      bt.mixed ? bt.d_u32 : nullptr);
  cudaFreeAsync(d_mask, s);
  bt.state = BatchState{bt.d_active, bt.d_cycles, bt.d_status, bt.d_r0, bt.d_rel, bt.d_sigma, bt.d_invc,
                        bt.d_nactive, bt.d_prange, bt.d_partial, bt.d_tol, bt.d_max, bt.mixed ? bt.inner : 1, n};
  if (bt.use_graph && !bt.persistent && !bt.graph.exec) {
    const BatchState& st = bt.state;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      set_error("batch: stream capture failed to start");
      return MG_ERR_CUDA;
    }
    if (bt.mixed) {
      if (bt.dim == 2) emit_mixed_step<2>(bt, st, s); else emit_mixed_step<3>(bt, st, s);
    } else {
      if (bt.dim == 2) emit_fp64_step<2>(bt, st, s); else emit_fp64_step<3>(bt, st, s);
    }
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt.graph.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      bt.graph.exec = nullptr;
      set_error(std::string("batch: graph capture: ") + cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
  }
  return MG_OK;
}

// Runs up to max_steps steps (FP64: a cycle; mixed: a refinement step with its inner
// cycles), stopping early once no problem is active.
mg_status batch_run(Batch& bt, int max_steps, cudaStream_t s, int* n_active) {
  *n_active = bt.n;
  if (bt.persistent) {
    for (int it = 0; it < max_steps; ++it) {
      const mg_status ps = persist_step(bt, s);
      if (ps != MG_OK) return ps;
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error(std::string("batch: ") + cudaGetErrorString(cudaGetLastError()));
        return MG_ERR_CUDA;
      }
      if (bt.h_pin[1] != 0) {
        set_error("batch: a persistent step's wait for a problem's earlier phase timed out");
        return MG_ERR_TIMEOUT;
      }
      *n_active = bt.h_pin[0];
      if (*n_active == 0) break;
    }
    return MG_OK;
  }
  for (int it = 0; it < max_steps; ++it) {
    if (!bt.use_graph) {
      if (bt.mixed) {
        if (bt.dim == 2) emit_mixed_step<2>(bt, bt.state, s); else emit_mixed_step<3>(bt, bt.state, s);
      } else {
        if (bt.dim == 2) emit_fp64_step<2>(bt, bt.state, s); else emit_fp64_step<3>(bt, bt.state, s);
      }
    }
    if ((bt.use_graph && cudaGraphLaunch(bt.graph.exec, s) != cudaSuccess) || cudaStreamSynchronize(s) != cudaSuccess) {
      set_error(std::string("batch: ") + cudaGetErrorString(cudaGetLastError()));
      return MG_ERR_CUDA;
    }
    *n_active = bt.h_pin[0];
    if (*n_active == 0) break;
  }
  return MG_OK;
}

// Enqueues one step on s (direct launches) without waiting for it; batch_read after the
// stream has reached it gives the problems' states.
mg_status batch_step_enqueue(Batch& bt, cudaStream_t s) {
  if (bt.persistent) return persist_step(bt, s);
  if (bt.mixed) {
    if (bt.dim == 2) emit_mixed_step<2>(bt, bt.state, s); else emit_mixed_step<3>(bt, bt.state, s);
  } else {
    if (bt.dim == 2) emit_fp64_step<2>(bt, bt.state, s); else emit_fp64_step<3>(bt, bt.state, s);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("batch: ") + cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

mg_status batch_read(Batch& bt, std::vector<ProblemState>& out, cudaStream_t s) {
  const int n = bt.n;
  std::vector<int> active(n), cycles(n), status(n), mx(n);
  std::vector<double> r0(n), rel(n), sigma(n), tol(n);
  const bool ok =
      cudaMemcpyAsync(active.data(), bt.d_active, n * sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(cycles.data(), bt.d_cycles, n * sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(status.data(), bt.d_status, n * sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(r0.data(), bt.d_r0, n * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(rel.data(), bt.d_rel, n * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(sigma.data(), bt.d_sigma, n * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(tol.data(), bt.d_tol, n * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaMemcpyAsync(mx.data(), bt.d_max, n * sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    set_error("batch: state download failed");
    return MG_ERR_CUDA;
  }
  out.resize(n);
  for (int p = 0; p < n; ++p) out[p] = ProblemState{active[p], cycles[p], status[p], r0[p], rel[p], sigma[p], tol[p], mx[p]};
  return MG_OK;
}

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_batch_create(int n, mg_hier* const* hiers, mg_batch** out) {
  if (!out || n <= 0 || !hiers) {
    set_error("mg_batch_create: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::vector<Hier*> hs;
  for (int p = 0; p < n; ++p) {
    if (!hiers[p]) {
      set_error("mg_batch_create: NULL hierarchy");
      return MG_ERR_INVALID_ARG;
    }
    hs.push_back(reinterpret_cast<Hier*>(hiers[p]));
  }
  Batch* bt = nullptr;
  const mg_status st = batch_create(hs, &bt);
  if (st != MG_OK) return st;
  *out = reinterpret_cast<mg_batch*>(bt);
  return MG_OK;
}

mg_status mg_batch_solve(mg_batch* batch, double* const* u, const double* const* b, double rel_tol, int max_cycles,
                         mg_solve_stats* stats, void* stream) {
  Batch* bt = reinterpret_cast<Batch*>(batch);
  if (!bt || !u || !b || max_cycles < 0 || !(rel_tol >= 0.0)) {
    set_error("mg_batch_solve: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : bt->own;
  const int n = bt->n;
  std::vector<ProblemState> init(n);
  for (int p = 0; p < n; ++p) {
    init[p].tol = rel_tol;
    init[p].max_cycles = max_cycles;
  }
  std::vector<int> fresh(n, 1);
  mg_status st = batch_begin(*bt, u, b, init, fresh, s);
  if (st != MG_OK) return st;
  const auto t0 = std::chrono::steady_clock::now();
  int n_active = 0;
  st = batch_run(*bt, max_cycles + 2, s, &n_active);
  if (st != MG_OK) return st;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  std::vector<ProblemState> out;
  st = batch_read(*bt, out, s);
  if (st != MG_OK) return st;
  mg_status worst = MG_OK;
  for (int p = 0; p < n; ++p) {
    if (stats) {
      stats[p].cycles = out[p].cycles;
      stats[p].outer_steps = bt->mixed ? out[p].cycles / std::max(bt->inner, 1) + 1 : out[p].cycles;
      stats[p].r0_norm = out[p].r0;
      stats[p].rel_residual = out[p].rel;
      stats[p].solve_ms = ms;
      stats[p].history_len = 0;
    }
    const mg_status sp = status_of(out[p].status);
    if (sp != MG_OK && worst == MG_OK) worst = sp;
  }
  if (worst != MG_OK) set_error("mg_batch_solve: some problems did not converge (see stats)");
  return worst;
}

mg_status mg_batch_setup(mg_batch* batch, const double* const* eps, void* stream) {
  Batch* bt = reinterpret_cast<Batch*>(batch);
  if (!bt || !eps) {
    set_error("mg_batch_setup: invalid argument");
    return MG_ERR_INVALID_ARG;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : bt->own;
  for (int p = 0; p < bt->n; ++p)
    if (!eps[p]) {
      set_error("mg_batch_setup: NULL coefficients");
      return MG_ERR_INVALID_ARG;
    }
  // fork: every problem's setup on its hierarchy's own stream, after the work already on
  // s (the coefficients); the small setups of many problems then overlap on the GPU.
  // Each status word comes back into the hierarchy's pinned slot; join on s.
  std::vector<cudaEvent_t> ev(static_cast<size_t>(bt->n) + 1, nullptr);
  auto release = [&] {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  };
  mg_status st = MG_OK;
  bool ok = true;
  for (size_t i = 0; i < ev.size() && ok; ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventRecord(ev[bt->n], s) == cudaSuccess;
  for (int p = 0; p < bt->n && ok && st == MG_OK; ++p) {
    Hier& H = *bt->H[p];
    ok = cudaStreamWaitEvent(H.own, ev[bt->n], 0) == cudaSuccess;
    if (ok) st = setup_enqueue(H, eps[p], H.own);
    ok = ok && cudaMemcpyAsync(reinterpret_cast<int*>(H.h_pin + 15), H.d_status, sizeof(int),
                               cudaMemcpyDeviceToHost, H.own) == cudaSuccess &&
         cudaEventRecord(ev[p], H.own) == cudaSuccess && cudaStreamWaitEvent(s, ev[p], 0) == cudaSuccess;
  }
  if (st != MG_OK) {
    cudaStreamSynchronize(s);
    release();
    return st;
  }
  if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
    release();
    set_error(std::string("mg_batch_setup: ") + cudaGetErrorString(cudaGetLastError()));
    return MG_ERR_CUDA;
  }
  release();
  for (int p = 0; p < bt->n; ++p) {
    st = setup_status(*bt->H[p], *reinterpret_cast<const int*>(bt->H[p]->h_pin + 15));
    if (st != MG_OK) return st;
  }
  return MG_OK;
}

void mg_batch_destroy(mg_batch* batch) {
  if (batch) cudaDeviceSynchronize();  // it may still be in use on any stream
  delete reinterpret_cast<Batch*>(batch);
}

}  // extern "C"
