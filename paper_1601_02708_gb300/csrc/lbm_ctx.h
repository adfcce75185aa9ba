// lbm_ctx.h -- the library's private context struct, shared by the
// translation units that launch on a context (lbm_api.cu, lbm_batch.cu).
#pragma once
#include <cuda_runtime.h>

#include "lbm_ade.h"
#include "lbm_tma.cuh"

struct DiagDev {
  double mass, J;
  long long infeasible;
};

struct lbm_ctx {
  lbm_params p;
  int pitch = 0;
  long long plane = 0;  // pitch * rows
  size_t esize = 4;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  void* f[2] = {nullptr, nullptr};  // Real [9][rows][pitch]
  int cur = 0;                      // buffer holding the current f*
  uint32_t* link = nullptr;  // [rows][pitch] link words
  void* vel = nullptr;     // Real [2][rows][pitch]
  void* kf = nullptr;      // Real [rows][pitch] or null
  void* u = nullptr;       // Real [rows][pitch]
  void* ureact = nullptr;  // Real [rows][pitch] (dissolution)
  double* mineral = nullptr;
  double* edge = nullptr;  // [3][nedge]: u_dir_t0, u_dir_t1, q
  float* edge32 = nullptr;  // FP32 copy of edge (FP32 lattices)
  long long* infeasible = nullptr;  // [nedge]
  double* jnode = nullptr;          // [ny]
  double* partial = nullptr;        // [max(blocks)]
  int nparts = 0;                   // partials written by the last final step
  int* flip_list = nullptr;
  int* flip_count = nullptr;      // [0] count, [1] done counter, [2] surface list length
  int* slist = nullptr;           // dissolution surface list (padded node indices)
  double* smin = nullptr;         // mineral of the listed nodes
  long long* counters = nullptr;  // [0] flips total, [1] solid count at init,
                                  // [2] wall solves without a root
  int wall_mode = 0;              // LBM_WALL_BOUNCE or LBM_WALL_MAXENT
  int* status = nullptr;          // device error word
  DiagDev* diag = nullptr;
  void* scratch = nullptr;  // staging for host outputs
  size_t scratch_bytes = 0;
  long long steps = 0;
  int nedge = 0;
  dim3 grid, block;
  int dgrid = 0;  // persistent blocks of the dissolution pass
  bool use_tma = false;  // the FP32 step runs the tile pipeline
  bool tma_ready = false;
  int tma_grid = 0, ntx = 0, nty = 0;
  lbm::TmaMaps maps[2];  // pop map of f[0] / f[1]; other maps identical
  // kernel timing (lbm_kernel_timing): event pairs per launch, folded into
  // the sums whenever the pool fills or the times are read
  bool timing = false;
  static constexpr int kPool = 512;
  cudaEvent_t ev[2][kPool][2] = {};
  int ev_used[2] = {0, 0};
  double ms_sum[2] = {0.0, 0.0};
  long long launches[2] = {0, 0};
  struct AdjWork* adj = nullptr;  // adjoint buffers (lbm_adjoint.cu), kept between calls
};

// Services of lbm_api.cu for the other translation units of the library.
lbm_status ctx_fail(lbm_status s, const char* fmt, ...);  // message of lbm_last_error
lbm_status ctx_check(const lbm_ctx* c);                    // null context
lbm_status ctx_status(lbm_ctx* c);   // waits for the stream, reads the device error word
bool ctx_on_device(const void* p);
// Copies the edge data of one call (NULL = zeros) into c->edge.
lbm_status ctx_stage_edges(lbm_ctx* c, const double* ua, const double* ub, const double* q);
// Refreshes the FP32 copy of the edge data after c->edge changed.
lbm_status ctx_edges_changed(lbm_ctx* c);
// One step launch with explicit arguments (fin = c->f[c->cur] for the tile
// pipeline's tensor maps).
template <typename Real>
lbm_status ctx_launch_step(lbm_ctx* c, const lbm::StepArgs<Real>& a, bool final_step);
// Padded [rows][pitch] FP64 field -> caller's [ny][nx] array (host or device).
lbm_status ctx_field_out_f64(lbm_ctx* c, const double* padded, double* out);
void ctx_adjoint_free(lbm_ctx* c);  // lbm_adjoint.cu


// Kernel arguments of a context's next step (fin = the current buffer) and
// of its dissolution pass.
template <typename Real>
inline lbm::StepArgs<Real> step_args(lbm_ctx* c, double frac) {
  lbm::StepArgs<Real> a;
  a.fin = (const Real*)c->f[c->cur];
  a.fout = (Real*)c->f[c->cur ^ 1];
  a.link = c->link;
  a.vel = (const Real*)c->vel;
  a.kf = (const Real*)c->kf;
  a.u_out = (Real*)c->u;
  a.ureact = (Real*)c->ureact;
  a.ua = c->edge;
  a.ub = c->edge + c->nedge;
  a.q = c->edge + 2 * c->nedge;
  a.ua32 = c->edge32;
  a.ub32 = c->edge32 ? c->edge32 + c->nedge : nullptr;
  a.q32 = c->edge32 ? c->edge32 + 2 * c->nedge : nullptr;
  a.infeasible = c->infeasible;
  a.jnode = c->jnode;
  a.partial = c->partial;
  a.status = c->status;
  a.bc_root = nullptr;
  a.wall_infeasible = c->counters + 2;
  a.wall_maxent = c->wall_mode == LBM_WALL_MAXENT;
  a.plane = c->plane;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.pitch = c->pitch;
  a.per_x = c->p.edge[0] == LBM_EDGE_PERIODIC;
  a.per_y = c->p.edge[2] == LBM_EDGE_PERIODIC;
  for (int s = 0; s < 4; ++s) a.edge[s] = c->p.edge[s];
  a.react_mode = c->p.react_mode;
  a.dissolution = c->p.dissolution;
  a.omega = (Real)(1.0 / c->p.tau);
  a.k_scalar = (Real)c->p.k_scalar;
  a.frac = frac;
  return a;
}

inline lbm::DissolveArgs dissolve_args(lbm_ctx* c) {
  lbm::DissolveArgs d;
  d.link = c->link;
  d.mineral = c->mineral;
  d.flip_list = c->flip_list;
  d.flip_count = c->flip_count;
  d.done = (unsigned*)(c->flip_count + 1);
  d.scount = c->flip_count + 2;
  d.slist = c->slist;
  d.smin = c->smin;
  d.flips_total = c->counters;
  d.status = c->status;
  d.nx = c->p.nx;
  d.ny = c->p.ny;
  d.pitch = c->pitch;
  d.per_x = c->p.edge[0] == LBM_EDGE_PERIODIC;
  d.per_y = c->p.edge[2] == LBM_EDGE_PERIODIC;
  d.check_all = 0;
  return d;
}

