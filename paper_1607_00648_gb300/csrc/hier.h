// Device-resident multigrid hierarchy (shared by the libmg CUDA translation units).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "device.cuh"
#include "internal.h"

namespace mg {

constexpr int kHistCap = 4096;

struct DevLevel {
  LevelDesc d{};
  int32_t* brick_nbr = nullptr;
  int32_t* brick_roots = nullptr;
  int32_t* brick_rank = nullptr;
  uint8_t* vflags = nullptr;
  uint8_t* cflags = nullptr;
  int32_t* hang_idx = nullptr;
  double* hang_w = nullptr;
  double* eps = nullptr;
  float* eps32 = nullptr;
  double* ahat = nullptr;
  uint16_t* a16 = nullptr;
  float* ascale = nullptr;
  double* phat = nullptr;
  uint16_t* p16 = nullptr;
  float* pscale = nullptr;
  uint64_t* abpa_rec = nullptr;  // bpa codec: per-slot records and byte streams of A_hat, P_hat
  uint8_t* abpa = nullptr;
  uint64_t* pbpa_rec = nullptr;
  uint8_t* pbpa = nullptr;
  double *u = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
  float *u32 = nullptr, *b32 = nullptr, *r32 = nullptr, *t32 = nullptr;
  double* aniso = nullptr;   // finest level of a tensor hierarchy: per-axis coefficient deviations
  float* aniso32 = nullptr;  // (axis-major, cell slots) and their FP32 copy
  double* dinv = nullptr;  // FP64 hierarchies: omega / diag(A) for the Jacobi sweeps
  double* eps_pair = nullptr;   // float-float finest sweeps: eps and omega / diag(A) as
  double* dinv_pair = nullptr;  // (h, l) float pairs in binary64 containers
  double *ad = nullptr, *ar = nullptr;  // additive cycle: correction d_l, surplus residual rh_l
  double* ai = nullptr;                 // BPX: injected skipped c-point updates i_l
  int32_t* child = nullptr;             // additive cycle: level-(l+1) slot at position 3x (injection)
  int R64 = 0, R32 = 0;    // slab depths picked by mg_autotune (0: the default rule)
  double* partial = nullptr;
  unsigned* counter = nullptr;
  int64_t n_dofs = 0;
};

struct Graph {
  cudaGraphExec_t exec = nullptr;
  const void* key0 = nullptr;
  const void* key1 = nullptr;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key0 = key1 = nullptr;
  }
};

// the dynamic coarsest level (Sect. 4.3) keeps the directly solved level at most this
// many unknowns
constexpr int kMaxDynCoarse = 1024;

struct Hier {
  const Grid* g = nullptr;
  mg_options opt{};
  int L = 0, c = 1, dim = 2;
  int c_user = 1, c_max = 1;  // the options' coarsest level; the finest the dynamic rule may take
  int c_setup = 1;            // the coarsest level the last setup chose (dynamic rule (a))
  std::vector<int32_t*> cs_lv, cm_lv;  // per candidate coarsest level: DoF slots, slot -> row map
  std::vector<int> nc_lv;              // and its number of unknowns
  int* d_audit = nullptr;              // dynamic rule: per level, 1 where the audit failed
  int top = 0;            // finest complete level (= L on uniform grids, L - 1 on adaptive ones)
  bool adaptive = false;  // level L only partly refined: composite solve
  int32_t* child_top = nullptr;  // level-top slot -> level-L slot at the same position
  float* c32 = nullptr;   // mixed composite solve: FP32 level-top correction and its right-hand side
  float* cb32 = nullptr;
  int64_t n_comp_dofs = 0;  // composite unknowns: level-L DoFs + unrefined level-(L-1) DoFs
  // composite slot lists: refined level-top DoFs, level-L DoFs, level-L hanging vertices
  int32_t *ref_top = nullptr, *dof_L = nullptr, *hang_L = nullptr;
  int64_t n_ref_top = 0, n_dof_L = 0, n_hang_L = 0;
  bool galerkin = false, boxmg = false, mixed = false;
  bool tensor = false;  // diagonal-tensor coefficients (mg_setup_tensor)
  int fmt = 1;  // 1 bf16, 2 fp16, 4 bpa codec
  uint64_t* bpa_used = nullptr;  // bpa codec: stream lengths per level, [2 l] A_hat, [2 l + 1] P_hat
  std::vector<DevLevel> lv;
  std::vector<void*> allocs;
  int n_c = 0;
  int32_t* c_slots = nullptr;
  int32_t* c_map = nullptr;
  double* c_mat = nullptr;
  double* ap3 = nullptr;  // 3D Galerkin setup: A_f P of the fine level (two-stage product)
  int64_t ap3_len = 0;
  int* d_status = nullptr;
  double* d_scal = nullptr;  // [0] norm2 fp64, [1] norm2 fp32 inner, [2] sigma
  double* h_pin = nullptr;   // pinned mirror of d_scal
  double* d_hist = nullptr;  // persistent solve: history, outputs, parameter block
  int* d_pint = nullptr;
  double* d_pdbl = nullptr;
  void* d_psolve = nullptr;
  cudaStream_t own = nullptr;
  bool ready = false;
  Graph g_cycle64, g_outer, g_inner, g_comp64, g_comp_outer, g_comp_inner, g_add;
  Graph g_cycle_ff, g_comp_ff;  // FP64 solves: cycles with float-float finest sweeps
  Graph g_fused[2][2];  // FP64 solves, norm fused into the next first sweep: [float-float][leading sweep]
  bool ff_active = true;   // float-float finest sweeps in use (when the setup split the pairs)
};

// ---- device memory of hierarchies and batches (solver.cu) ----
// Allocations come from a per-device stream-ordered pool that keeps freed memory
// (release threshold = max), so that creating and destroying hierarchies in a serving
// loop neither calls into the driver's allocator nor synchronises the device (as
// cudaFree does).  Allocation and free are ordered on stream s.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);
// 128 bytes of pinned host memory from a process-wide slab (never returned to the driver)
void* pinned_slot();
void pinned_release(void* p);
// destroy a hierarchy whose work is known to be complete (no device synchronisation)
void hier_release(Hier* H);
// mg_hier_create with the hierarchy's stream at a given priority; blocking false gives it
// a non-blocking stream (for hierarchies that only ever run on explicit streams)
mg_status hier_create(const Grid* g, const mg_options& o, int priority, Hier** out, bool blocking = true);

// enqueue a hierarchy's setup without synchronising; setup_status interprets d_status
mg_status setup_enqueue(Hier& H, const double* eps, cudaStream_t s);
mg_status setup_status(Hier& H, int status);

// ---- batched solves (batch.cu), used by the batch C ABI and the server ----
struct Batch;
struct ProblemState {
  int active, cycles, status;  // status: 0 converged, 1 not converged (yet), 2 non-finite, 3 diverged
  double r0, rel, sigma, tol;
  int max_cycles;
};
mg_status batch_create(const std::vector<Hier*>& hs, Batch** out, int priority = 0,
                       bool blocking = true);  // priority / blocking: of its own stream
void batch_destroy(Batch* bt);
void batch_set_graph(Batch* bt, bool use_graph);
mg_status batch_begin(Batch& bt, double* const* u, const double* const* b, const std::vector<ProblemState>& init,
                      const std::vector<int>& fresh, cudaStream_t s);
mg_status batch_run(Batch& bt, int max_steps, cudaStream_t s, int* n_active);
mg_status batch_step_enqueue(Batch& bt, cudaStream_t s);  // one step, no synchronisation
mg_status batch_read(Batch& bt, std::vector<ProblemState>& out, cudaStream_t s);
mg_status status_of(int st);
size_t hier_footprint(const Grid& g, const mg_options& o);

}  // namespace mg
