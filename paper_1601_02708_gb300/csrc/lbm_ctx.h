// lbm_ctx.h -- the library's private context struct, shared by the
// translation units that launch on a context (lbm_api.cu, lbm_batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <set>
#include <tuple>

#include "lbm_ade.h"
#include "lbm_tma.cuh"

struct DiagDev {
  double mass, J, flux;
  long long infeasible;
};

struct lbm_ctx {
  lbm_params p;
  // A slab of a lattice split by rows (lbm_init_slab): rows y0 .. y0 + p.ny - 1
  // of a lattice of ny_global rows (periodic in y: per_y_global); sides of
  // kind LBM_EDGE_EXCHANGE get their ghost rows from the halo exchange.  An
  // unsplit lattice has y0 = 0, ny_global = p.ny.
  int y0 = 0, ny_global = 0, per_y_global = 0;
  bool first_pass_due = false;  // the first dissolution pass waits for the halo
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
  void* ureact = nullptr;  // [rows][pitch] reaction shares, 8 bytes a node (dissolution)
  double* mineral = nullptr;
  int* flip_step = nullptr;  // [rows][pitch] pass that turned a node fluid (-1: none)
  double* edge = nullptr;  // [3][nedge]: u_dir_t0, u_dir_t1, q
  long long* infeasible = nullptr;  // [nedge]
  double* jnode = nullptr;          // [ny]
  double* jflux = nullptr;          // [ny] east-column first moment of the last step
  double* partial = nullptr;        // [partial_cap]
  int partial_cap = 0;
  int nparts = 0;                   // partials written by the last final step
  int* open_nodes = nullptr;        // padded indices of the nodes on non-periodic sides
  int n_open = 0;
  int* flip_list = nullptr;
  int* flip_count = nullptr;      // [0] count, [1] done counter, [2] surface list length,
                                  // [3] dissolution passes run
  int* slist = nullptr;           // dissolution surface list (padded node indices)
  double* smin = nullptr;         // mineral of the listed nodes
  long long* counters = nullptr;  // [0] flips total, [1] solid count at init,
                                  // [2] wall solves without a root, [3] wall solves
                                  // whose Newton iteration stopped short
  long long warned_infeasible = 0;  // counts already reported by lbm_synchronize or
  long long warned_newton = 0;      // lbm_diagnostics
  int wall_mode = 0;              // lbm_wall_mode
  int* status = nullptr;          // device error word
  DiagDev* diag = nullptr;
  void* scratch = nullptr;  // staging for host outputs
  void* pinned = nullptr;   // page-locked host words: status and blob-header read-backs
  size_t scratch_bytes = 0;
  long long steps = 0;
  int nedge = 0;
  dim3 grid, block;    // 32 x 8 blocks over the lattice (init, adjoint, read-outs)
  dim3 sgrid, sblock;  // blocks of the plain step kernel (lbm::step_rows rows)
  int dgrid = 0;  // persistent blocks of the dissolution pass
  bool use_tma = false;  // the FP32 step runs the tile pipeline
  bool kernel_auto = true;  // the library chooses the FP32 step kernel
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
  // Recorded launch sequences (CUDA graphs) of repeated calls: lbm_substeps
  // and lbm_adjoint record a sequence the second time they see its key and
  // replay it from then on (the first call runs the launches directly, so a
  // one-off call never pays for the recording).  The recording stream is the
  // context's own (created lazily); replays go to the context's stream.
  using GraphKey = std::tuple<int, int, int, int, int, int, int>;  // kind, n, eta, stride,
                                                                    // parity, walls, kernel
  struct Recorded {
    cudaGraphExec_t exec;
    int nparts;  // partials the last recorded step leaves
  };
  std::map<GraphKey, Recorded> graphs;
  std::set<GraphKey> seen;
  cudaStream_t rec_stream = nullptr;
};

// Graph replay of a context's launch sequence (lbm_api.cu): replays `key`
// if it was recorded, records it if it was seen before (enqueue(c) issues
// the launches on c->stream, which points at the recording stream meanwhile,
// and advances the context's bookkeeping), else runs enqueue directly.  The
// context's cur, steps and nparts end as enqueue leaves them.
lbm_status ctx_run_recorded(lbm_ctx* c, const lbm_ctx::GraphKey& key,
                            lbm_status (*enqueue)(lbm_ctx*, void*), void* arg);
// Forget the recorded sequences of one kind (key element 0), e.g. when the
// buffers they write were reallocated.
void ctx_drop_recorded(lbm_ctx* c, int kind);

// Services of lbm_api.cu for the other translation units of the library.
lbm_status ctx_fail(lbm_status s, const char* fmt, ...);  // message of lbm_last_error
// A tiled tensor map (no swizzle, no interleave, L2 promotion 128 B) of a
// rank-2 or rank-3 array; LBM_ERR_CUDA naming `what` if it cannot be made.
lbm_status ctx_make_map(const char* what, CUtensorMap* m, CUtensorMapDataType dt, int rank,
                        void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                        const cuuint32_t* box);
lbm_status ctx_check(const lbm_ctx* c);                    // null context
lbm_status ctx_status(lbm_ctx* c);   // waits for the stream, reads the device error word
bool ctx_on_device(const void* p);
// Copies the edge data of one call (NULL = zeros) into c->edge.
lbm_status ctx_stage_edges(lbm_ctx* c, const double* ua, const double* ub, const double* q);
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
  a.u_hist = nullptr;
  a.ureact = c->ureact;
  a.ua = c->edge;
  a.ub = c->edge + c->nedge;
  a.q = c->edge + 2 * c->nedge;
  a.infeasible = c->infeasible;
  a.jnode = c->jnode;
  a.jflux = c->jflux;
  a.partial = c->partial;
  a.status = c->status;
  a.bc_root = nullptr;
  a.wall_infeasible = c->counters + 2;
  a.newton_fail = c->counters + 3;
  a.open_nodes = c->open_nodes;
  a.n_open = c->n_open;
  a.open_mask = 0;
  for (int s = 0; s < 4; ++s)
    if (c->p.edge[s] == LBM_EDGE_DIRICHLET || c->p.edge[s] == LBM_EDGE_NEUMANN)
      a.open_mask |= 1 << s;
  a.wall_maxent = c->wall_mode != LBM_WALL_BOUNCE;
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

// Template argument kWalls of the step kernels for the context's wall mode:
// 0 without maximum-entropy walls, 2 for FP64 Newton solves on the FP32
// lattice, 1 for solves in the lattice's own precision.
inline int walls_variant(const lbm_ctx* c) {
  if (c->wall_mode == LBM_WALL_BOUNCE) return 0;
  return (c->wall_mode == LBM_WALL_MAXENT && c->esize == 4) ? 2 : 1;
}

inline lbm::DissolveArgs dissolve_args(lbm_ctx* c) {
  lbm::DissolveArgs d;
  d.link = c->link;
  d.mineral = c->mineral;
  d.flip_list = c->flip_list;
  d.flip_count = c->flip_count;
  d.done = (unsigned*)(c->flip_count + 1);
  d.scount = c->flip_count + 2;
  d.pass = c->flip_count + 3;
  d.flip_step = c->flip_step;
  d.kf32 = c->esize == 4 ? (const float*)c->kf : nullptr;
  d.k_scalar = c->p.k_scalar;
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

