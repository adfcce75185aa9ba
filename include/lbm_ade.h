/*
 * lbm_ade.h -- C ABI of the GB300 lattice Boltzmann advection-diffusion-
 * reaction library (liblbmade.so).
 *
 * The library advances the pore-scale subdomain of the hybrid FEM/LBM
 * multi-time-step method of Karimi & Nakshatrala (arXiv 1601.02708): a D2Q9
 * BGK lattice Boltzmann scheme for the advection-diffusion equation
 * (Sec. 4.1, Eqs. "LBE", "Collision", "LBM_feq", "LBM_Macro") with the
 * maximum-entropy Dirichlet and Neumann boundary conditions of Sec. 4.1.1,
 * halfway bounce-back at solid nodes, a first-order reaction sink with
 * optional mineral dissolution, the multi-time-step interpolation of
 * interface data (Sec. 6.2 (iii), Eq. "MTS") and the LBM -> FEM trace
 * (Sec. 6.2 (ii)).
 *
 * Conventions shared by every call
 *  - Lattice units: h = dt = 1, c_s^2 = 1/3, D = (tau - 1/2) / 3.
 *  - D2Q9 direction order: 0 rest, 1 E(+1,0), 2 N(0,+1), 3 W(-1,0), 4 S(0,-1),
 *    5 NE, 6 NW, 7 SW, 8 SE; weights 4/9, 1/9 (1-4), 1/36 (5-8).
 *  - Node fields are row-major [ny][nx] (x fastest), populations
 *    [9][ny][nx], velocity [2][ny][nx] (v_x plane, then v_y plane).
 *  - Edge data (Dirichlet values, Neumann fluxes) use the edge layout
 *    [W: ny][E: ny][S: nx][N: nx], length 2 (nx + ny); W is x = 0, E is
 *    x = nx - 1, S is y = 0, N is y = ny - 1.  A corner node takes its value
 *    from the first side in the order W, E, S, N whose kind applies.
 *  - Every pointer argument may point to host memory or to device memory of
 *    the context's device; the library detects which.  Inputs are copied (or
 *    read on the context's stream before the call's work completes); the
 *    library never keeps or frees caller memory.  Results written to host
 *    memory are complete when the call returns; results written to device
 *    memory are ordered on the context's stream.
 *  - Every call returns an lbm_status; no call aborts, exits or traps.  On an
 *    error, lbm_last_error() describes it (per thread).
 */
#ifndef LBM_ADE_H
#define LBM_ADE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ADE_ABI_VERSION 2

typedef struct lbm_ctx lbm_ctx; /* opaque; owned by the library until lbm_destroy */

typedef enum {
  LBM_OK = 0,
  LBM_WARN_BC_INFEASIBLE = 1, /* success, but boundary solves met data with no
                                 non-negative solution (Sec. 4.1.1: Dirichlet data
                                 below the known populations' sum are applied
                                 literally, Neumann data without a root set the
                                 unknowns to zero); reported once per new count by
                                 the calls that wait for the stream
                                 (lbm_synchronize, lbm_diagnostics); the running
                                 count is lbm_diag.bc_infeasible */
  LBM_ERR_ARG = -1,     /* invalid argument (size, tau <= 1/2, edge kinds, NULL) */
  LBM_ERR_CUDA = -2,    /* a CUDA call failed; the message names it */
  LBM_ERR_NEWTON = -3,  /* a maximum-entropy wall solve stopped short of its Newton
                           tolerance (the last iterate was used); reported like the
                           warning above, counted in lbm_diag.newton_fail */
  LBM_ERR_TIMEOUT = -4, /* a kernel's bounded wait expired; the context's
                           results since the last good call are invalid */
  LBM_ERR_STATE = -5,   /* context misuse (e.g. restore from a foreign blob) */
  LBM_ERR_NOMEM = -6    /* device allocation failed */
} lbm_status;

typedef enum {
  LBM_EDGE_PERIODIC = 0,  /* wraps to the opposite side (both sides must be periodic) */
  LBM_EDGE_DIRICHLET = 1, /* max-entropy Dirichlet, Sec. 4.1.1 (a) */
  LBM_EDGE_NEUMANN = 2,   /* max-entropy Neumann on the first moment, Sec. 4.1.1 (b) */
  LBM_EDGE_EXCHANGE = 3   /* set by lbm_init_slab only: the S or N side a slab shares
                             with its neighbour; its ghost row comes from the halo
                             exchange (lbm_init refuses it) */
} lbm_edge_kind;

typedef enum {
  LBM_REACT_NONE = 0,
  LBM_REACT_SURFACE = 1, /* sink at fluid nodes with a solid D2Q9 neighbour */
  LBM_REACT_BULK = 2     /* sink at every fluid node */
} lbm_react_mode;

typedef enum {
  LBM_WALL_BOUNCE = 0,        /* pore walls: halfway bounce-back (the default) */
  LBM_WALL_MAXENT = 1,        /* pore walls as zero-flux boundaries of the maximum-entropy
                                 kind, Sec. 4.1.1 (b), the Lagrange multiplier found by
                                 Newton's method in FP64 on either lattice (see
                                 lbm_set_wall_mode) */
  LBM_WALL_MAXENT_LATTICE = 2 /* the same walls with Newton's method in the lattice's
                                 own precision (FP32 on an FP32 lattice: faster) */
} lbm_wall_mode;

enum { LBM_SIDE_W = 0, LBM_SIDE_E = 1, LBM_SIDE_S = 2, LBM_SIDE_N = 3 };

typedef struct {
  int nx, ny;        /* lattice nodes, each >= 2; ny <= 65535 (a launch's
                        block index in y numbers the rows) */
  int precision;     /* 32: FP32 populations and arithmetic (FP64 boundary
                        solves, reaction shares, mineral and sums); 64: FP64
                        throughout */
  int edge[4];       /* lbm_edge_kind of the W, E, S, N sides */
  double tau;        /* BGK relaxation time (Eq. "Collision"), > 1/2 */
  int react_mode;    /* lbm_react_mode */
  double k_scalar;   /* first-order rate where k_field is NULL */
  int dissolution;   /* nonzero (surface mode only): the sink removes mineral
                        from the solid neighbours in proportion to the link
                        weights; a solid node whose mineral reaches <= 0
                        becomes fluid with zero populations */
} lbm_params;

typedef struct {
  double mass;             /* sum of u over the lattice at the current time */
  double outlet_J;         /* sum over all steps of the east-edge (x = nx-1)
                              fluid-node concentrations */
  double outlet_flux;      /* first moment sum_i f_i e_ix over the east-edge fluid
                              nodes at the last step (after the boundary
                              conditions, before collision; Eq. "LBM_Macro") */
  double min_f;            /* smallest stored population over the fluid nodes
                              (as lbm_min_population; +inf without fluid) */
  long long steps;         /* time steps taken since lbm_init */
  long long bc_infeasible; /* boundary solves whose data had no non-negative
                              solution (Dirichlet: applied literally; Neumann:
                              unknowns set to zero) */
  long long newton_fail;   /* wall solves whose Newton iteration stopped short of
                              its tolerance */
  long long flips;         /* solid nodes turned fluid by dissolution */
  long long n_solid;       /* solid nodes at the current time */
} lbm_diag;

/* Create a context and initialise the populations to the equilibrium of u0,
 * f_i(x, 0) = f_i^eq(x, 0; u0(x)) (Sec. 6.2 (i), Eq. "LBM_feq").
 *   solid   [ny][nx] nonzero = solid node (NULL: all fluid)
 *   vel     [2][ny][nx] advection velocity, lattice units (NULL: zero);
 *           the caller zeroes it in solids
 *   k_field [ny][nx] per-node rate (NULL: p->k_scalar everywhere)
 *   mineral [ny][nx] mineral mass of solid nodes (NULL: 1.0)
 *   u0      [ny][nx] initial concentration (NULL: zero)
 *   stream  cudaStream_t the context launches on (NULL: legacy default)
 * Device memory is allocated by the library and released by lbm_destroy. */
lbm_status lbm_init(lbm_ctx** out, const lbm_params* p, const uint8_t* solid,
                    const double* vel, const double* k_field,
                    const double* mineral, const double* u0, void* stream);

/* Advance n time steps: substeps j = 1..n of a coarse step split eta ways
 * (Algorithm 1, inner loop).  Each step streams, applies bounce-back and the
 * boundary conditions, takes the moments, reacts and collides.  Dirichlet
 * data at substep j are (1 - j/eta) u_dir_t0 + (j/eta) u_dir_t1 (Eq. "MTS");
 * q_neu are the Neumann first-moment values e.n-weighted, outward positive.
 * Edge arrays use the edge layout; NULL means zero (u_dir_t1 NULL: equal to
 * u_dir_t0).  n = 0 is a no-op.  Asynchronous on the context's stream. */
lbm_status lbm_substeps(lbm_ctx* c, int n, int eta, const double* u_dir_t0,
                        const double* u_dir_t1, const double* q_neu);

/* LBM -> FEM transfer, Sec. 6.2 (ii): bilinear value of the current u at
 * npts points xy[npts][2] given in lattice coordinates.  A point outside
 * [0, nx-1] x [0, ny-1] across a non-periodic side yields NaN.  With xy and
 * u_out both in device memory the call is asynchronous on the context's
 * stream; otherwise it waits. */
lbm_status lbm_interface_trace(lbm_ctx* c, int npts, const double* xy,
                               double* u_out);

/* Current concentration u = sum_i f_i (Eq. "LBM_Macro"), [ny][nx], written
 * as float (out_precision 32) or double (64); zero at solid nodes. */
lbm_status lbm_get_concentration(lbm_ctx* c, void* out, int out_precision);

/* Stored populations [9][ny][nx] as double.  They are post-collision: the
 * values the next step streams. */
lbm_status lbm_get_populations(lbm_ctx* c, double* out);

/* Current solid mask [ny][nx] (1 = solid) and mineral mass [ny][nx].  The
 * mineral already carries the sink of the stored post-collision populations,
 * i.e. one reaction step beyond the returned concentration. */
lbm_status lbm_get_solid(lbm_ctx* c, uint8_t* out);
lbm_status lbm_get_mineral(lbm_ctx* c, double* out);

/* Reductions over the lattice in FP64, in a fixed order (deterministic).
 * Waits for the stream; may return LBM_WARN_BC_INFEASIBLE or LBM_ERR_NEWTON
 * (out is filled either way). */
lbm_status lbm_diagnostics(lbm_ctx* c, lbm_diag* out);
/* Dissolution record [ny][nx]: for every node turned fluid so far the number
 * of steps after which it was first fluid (the step whose dissolution
 * exhausted its mineral, plus one: a node exhausted by the consumption of
 * the first step reads 1), -1 for nodes never turned fluid.  This is the
 * integer record the FP32 and FP64 lattices, and the oracle, compare for
 * the exact mask (Sec. 7.4 narrates dissolution; the rule is that of
 * lbm_params.dissolution).  LBM_ERR_STATE without dissolution. */
lbm_status lbm_get_flip_steps(lbm_ctx* c, int32_t* out);
/* The smallest stored (post-collision) population over the fluid nodes: the
 * check that the populations stay non-negative (Sec. 4.1, Eq. "NN_Cond", and
 * the maximum-entropy boundary data).  +infinity without fluid nodes.  Waits
 * for the context's stream.  Errors: LBM_ERR_ARG (NULL out), LBM_ERR_NOMEM,
 * LBM_ERR_CUDA. */
lbm_status lbm_min_population(lbm_ctx* c, double* out);

/* Treatment of the pore walls from the next step on (Sec. 4.1.1 (b) and the
 * comparison of wall treatments after it).  LBM_WALL_BOUNCE: halfway
 * bounce-back.  LBM_WALL_MAXENT: at a fluid node beside solid ones (and off
 * the non-periodic lattice sides, whose nodes keep bounce-back at their solid
 * links) the populations whose source is solid follow from the zero-flux
 * maximum-entropy condition with the lattice-weighted normal to the solid
 * neighbours, n = -sum w_i e_i over those directions (normalised); unknowns
 * with e_i.n >= 0 keep bounce-back, as does a node where the sum cancels.
 * The Lagrange multiplier is found by Newton's method in FP64 (tolerance
 * 1e-15) and the populations are rounded to the lattice's precision once.
 * LBM_WALL_MAXENT_LATTICE: the same with the Newton iteration in the
 * lattice's precision (on an FP32 lattice: FP32, tolerance 1e-7; GB300 runs
 * FP64 at 1/64 of the FP32 rate, so this mode is the faster one there).
 * Solves with no root set their unknowns to zero and count in
 * lbm_diag.bc_infeasible; solves short of the tolerance count in
 * lbm_diag.newton_fail.  The adjoint (lbm_adjoint) covers bounce-back walls
 * only and returns LBM_ERR_STATE otherwise.  A batch (lbm_batch_create) takes
 * its members' wall modes when it is created; set them before.  Errors:
 * LBM_ERR_ARG for an unknown mode. */
lbm_status lbm_set_wall_mode(lbm_ctx* c, int mode);

/* Instantaneous bimolecular reaction n_A A + n_B B -> n_C C (Sec. 7.2): the
 * invariants alpha = u_A + (n_A / n_C) u_C and beta = u_B + (n_B / n_C) u_C
 * carry no reaction (two lattices transport them like any concentration),
 * and the species follow node by node:
 *   u_A = max(alpha - (n_A / n_B) beta, 0),
 *   u_B = (n_B / n_A) max((n_A / n_B) beta - alpha, 0),
 *   u_C = (n_C / n_A) (alpha - u_A).
 * Arrays of n FP64 values, host or device memory (host arrays are staged
 * and the call returns once the results are written; with device arrays it
 * is asynchronous on `stream`).  Each operation is rounded on its own (no
 * fused multiply-add).  Errors: LBM_ERR_ARG (n < 0, a coefficient not finite
 * and positive, a NULL array), LBM_ERR_NOMEM, LBM_ERR_CUDA. */
lbm_status lbm_species_from_invariants(long long n, double nA, double nB, double nC,
                                       const double* alpha, const double* beta, double* uA,
                                       double* uB, double* uC, void* stream);
/* The invariants of given species concentrations (initial data). */
lbm_status lbm_invariants_from_species(long long n, double nA, double nB, double nC,
                                       const double* uA, const double* uB, const double* uC,
                                       double* alpha, double* beta, void* stream);

/* Calcite at equilibrium, CaCO3 <-> Ca2+ + CO3^2- (Sec. 7.4): with u1, u2, u3
 * the concentrations of CaCO3, Ca2+, CO3^2-, K_sp = u2 u3 / u1 (Eq.
 * "Hybrid_Ksp"), and the invariants psi1 = u1 + u2, psi2 = u3 - u2 (Eq.
 * "Carbonate_uncoupled"; the printed u1 - u2 is not conserved by the
 * reaction, u1 + u2 is and leads to the printed root), which two lattices
 * transport without a reaction term.  lbm_calcite_species returns
 *   u2 = (-(psi2 + K_sp) + sqrt((psi2 + K_sp)^2 + 4 K_sp psi1)) / 2,
 *   u1 = psi1 - u2,  u3 = psi2 + u2,
 * evaluating the root as 2 K_sp psi1 / ((psi2 + K_sp) + sqrt(...)) where
 * psi2 + K_sp > 0 (the same root, without the cancellation of the printed
 * form when K_sp psi1 is small).  Invariants of non-negative species
 * (psi1 >= 0, psi1 + psi2 >= 0) give non-negative species; elsewhere the
 * discriminant may be negative and the node's outputs NaN.
 * lbm_calcite_invariants is the inverse map.
 * Arrays of n FP64 values, host or device, as lbm_species_from_invariants.
 * Errors: LBM_ERR_ARG (n < 0, K_sp not finite and positive, a NULL array),
 * LBM_ERR_NOMEM, LBM_ERR_CUDA. */
lbm_status lbm_calcite_species(long long n, double ksp, const double* psi1, const double* psi2,
                               double* u1, double* u2, double* u3, void* stream);
lbm_status lbm_calcite_invariants(long long n, const double* u1, const double* u2,
                                  const double* u3, double* psi1, double* psi2, void* stream);

/* Two fields on one geometry (the invariants alpha, beta of Sec. 7.2 or
 * psi1, psi2 of Sec. 7.4: two concentrations carried by one flow through one
 * pore space).  lbm_pair_create binds two existing contexts that have the
 * same size, sides, solid mask and velocity field, FP32 populations, the
 * same stream and step parity, bounce-back walls and no dissolution (their
 * relaxation time, rate field, edge data and initial data may differ; the
 * masks and velocities are compared on the device, a call that waits for
 * the stream).  lbm_pair_substeps then advances both by n substeps of eta
 * with one kernel launch a substep: each lattice computes exactly what
 * lbm_substeps on it alone computes (the same Eq. "MTS" edge data, the same
 * mass partials), while the velocity and link words are read once for both.
 * Edge arguments as lbm_substeps, one set per lattice (a_* for the first).
 * The contexts stay usable on their own (lbm_get_u, lbm_mass, lbm_save ...);
 * a pair whose lattices were stepped apart since is refused
 * (LBM_ERR_STATE).  The pair holds no device memory; destroy it before its
 * contexts.  Errors: LBM_ERR_ARG (the lattices do not qualify, n < 0,
 * eta < 1), LBM_ERR_STATE, LBM_ERR_NOMEM, LBM_ERR_CUDA. */
typedef struct lbm_pair lbm_pair;
lbm_status lbm_pair_create(lbm_pair** out, lbm_ctx* a, lbm_ctx* b);
lbm_status lbm_pair_substeps(lbm_pair* p, int n, int eta, const double* a_dir_t0,
                             const double* a_dir_t1, const double* a_q, const double* b_dir_t0,
                             const double* b_dir_t1, const double* b_q);
void lbm_pair_destroy(lbm_pair* p);

/* Schwarz rollback (Algorithm 1 restarts every sub-iteration from the state
 * at the start of the coarse step): lbm_state_bytes gives the size of a
 * state blob; lbm_save writes the full state into a caller-owned buffer of
 * at least that size; lbm_restore reads it back into the same context.
 * lbm_save into device memory is asynchronous on the context's stream (the
 * blob is complete when the stream reaches that point); into host memory it
 * waits.  lbm_restore waits for the stream to read the blob's header (a
 * blob of another lattice is LBM_ERR_STATE), then queues the copies; from
 * host memory it waits for them too. */
lbm_status lbm_state_bytes(lbm_ctx* c, size_t* bytes);
lbm_status lbm_save(lbm_ctx* c, void* buf, size_t bytes);
lbm_status lbm_restore(lbm_ctx* c, const void* buf, size_t bytes);

/* Kernel timing for performance reports.  While enabled, lbm_substeps
 * records a CUDA event pair on the context's stream around every launch of
 * the fused step kernel and of the dissolution kernel;
 * lbm_kernel_times_read waits for the stream and returns the summed device
 * milliseconds and launch counts since the last enable (step kernel first,
 * then dissolution), then keeps timing.  Timing adds two event records per
 * launch and nothing else to the launch sequence. */
lbm_status lbm_kernel_timing(lbm_ctx* c, int enable);
lbm_status lbm_kernel_times_read(lbm_ctx* c, double* step_ms, long long* step_launches,
                                 double* dissolve_ms, long long* dissolve_launches);

/* Kernel variant of the step: LBM_KERNEL_AUTO (default: in FP32 mode the
 * tile pipeline below 8 M nodes or with maximum-entropy pore walls, the
 * generic kernel for larger lattices with bounce-back walls -- the faster of
 * the two on GB300 in each case; the generic kernel in FP64 mode), LBM_KERNEL_GENERIC (one thread per node reading global memory) or
 * LBM_KERNEL_TMA (persistent TMA-fed tile pipeline, FP32 only).  All variants compute the same update;
 * the choice only changes speed.  LBM_ERR_ARG for an unknown or unsupported
 * variant. */
enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_GENERIC = 1, LBM_KERNEL_TMA = 2 };
lbm_status lbm_set_kernel(lbm_ctx* c, int variant);
/* The variant the context's steps run now (LBM_KERNEL_GENERIC or
 * LBM_KERNEL_TMA) into *variant. */
lbm_status lbm_get_kernel(lbm_ctx* c, int* variant);

/* Change the stream the context launches on; wait for its work. */
lbm_status lbm_set_stream(lbm_ctx* c, void* stream);
lbm_status lbm_synchronize(lbm_ctx* c);

/* Replace the per-node rate field k(x) ([ny][nx], host or device, copied
 * before return) of a context created with one (LBM_ERR_STATE otherwise);
 * the next step uses it. */
lbm_status lbm_set_rate_field(lbm_ctx* c, const double* k_field);

/* ---- adjoint: gradients of the outlet breakthrough (reverse mode) ---------
 * The paper computes no gradients; this is the discrete adjoint of the step
 * of lbm_substeps -- pull streaming with bounce-back, the max-entropy
 * boundary conditions of Sec. 4.1.1 (Eq. "LBM_Dir", "LBM_Neu", the time
 * interpolation of Eq. "MTS"), the collision of Eq. "Collision" with the
 * sink -- which for a fixed solid mask is affine in the populations and the
 * edge data (a Neumann node's root / zero-limit branch is recorded in the
 * forward run).  lbm_adjoint advances the context by n substeps exactly as
 * lbm_substeps(c, n, eta, u_dir_t0, u_dir_t1, q_neu) would and returns the
 * outlet breakthrough
 *     J = sum_{j=1..n} sum_{fluid nodes with x = nx - 1} u^j
 * with its gradients, holding the pre-collision state at the start of the
 * call fixed:
 *   grad_k  [ny][nx]: dJ/dk(x), the rate of every node (0 where no reaction
 *           applies: solid nodes, and non-surface nodes in surface mode);
 *   grad_ua, grad_ub [n_edge]: dJ/d(Dirichlet data at the start / the end of
 *           the coarse step), edge layout as in lbm_substeps;
 *   grad_q  [n_edge]: dJ/d(Neumann data);
 *   grad_side [4]: dJ/d(one Dirichlet value held on the whole side W, E, S,
 *           N over the call), i.e. the sum of grad_ua and grad_ub over that
 *           side's slots (0 for a side that is not Dirichlet): the gradient
 *           with respect to a uniform inlet concentration.
 * J and every gradient are FP64; any
 * output may be NULL; outputs may be host or device memory and are complete
 * when the call returns.
 * Work and memory: with stride >= n the forward run stores u and the
 * Neumann branches of every step (n concentration planes of device memory)
 * and the reverse sweep runs one adjoint step per step: about two forward
 * passes.  With 0 < stride < n the state is kept every `stride` steps, each
 * segment is recomputed once during the reverse sweep storing u and the
 * branches of its steps: about three forward passes, with ceil(n / stride)
 * + 3 population sets and `stride` concentration planes.  stride <= 0
 * chooses the whole history when it takes at most a quarter of the free
 * device memory, else stride = ceil(sqrt(n)).  The buffers stay in the
 * context for the next call.
 * Errors: LBM_ERR_STATE if dissolution is on (a flip is not differentiable)
 * or the pore walls are of the maximum-entropy kind (not affine in f);
 * LBM_ERR_ARG for n < 1 or eta < 1, or two Neumann sides that meet at a
 * corner (that root is not affine); LBM_ERR_NOMEM; LBM_ERR_TIMEOUT as for
 * lbm_substeps. */
lbm_status lbm_adjoint(lbm_ctx* c, int n, int eta, int stride, const double* u_dir_t0,
                       const double* u_dir_t1, const double* q_neu, double* J, double* grad_k,
                       double* grad_ua, double* grad_ub, double* grad_q, double* grad_side);

/* ---- batches: many lattices advanced together (Sec. 6.3, Algorithm 2 runs
 * several pore-scale subdomains; each member steps as lbm_substeps does) -----
 * A batch is built from contexts made by lbm_init that share precision,
 * device, step parity and a created (non-default) stream; the contexts stay
 * owned by the caller and usable on their own (read-out, diagnostics, save /
 * restore), but while they are in a batch they should be stepped only
 * through it, and they must outlive it.  One time step of the whole batch is
 * two launches: a persistent step kernel over a tile list spanning every
 * member and one dissolution pass over every member's surface list.  Each
 * (n, eta, parity, shape) sequence is recorded once into a CUDA graph and
 * replayed.  A member's results are bit-identical to stepping it alone.
 * Errors: LBM_ERR_ARG for bad arguments (message in lbm_batch_last_error),
 * LBM_ERR_CUDA / LBM_ERR_NOMEM from the runtime; a bounded wait that expired
 * inside the pipelined kernel sets the status word of every member that CTA
 * served, reported as LBM_ERR_TIMEOUT by that member's next read-out. */
typedef struct lbm_batch lbm_batch;
/* members: n context pointers (n >= 1, no repeats); the batch copies the
 * pointer array and allocates its own device tables. */
lbm_status lbm_batch_create(lbm_batch** out, int n, lbm_ctx* const* members);
/* n steps of every member; edge-data arguments are arrays of one pointer per
 * member, each laid out as in lbm_substeps (an array or entry may be NULL:
 * zero data), host or device memory, read before the call returns. */
lbm_status lbm_batch_substeps(lbm_batch* b, int n, int eta, const double* const* u_dir_t0,
                              const double* const* u_dir_t1, const double* const* q_neu);
/* Tile shape of the step kernel.  Shapes 0 .. 5: one thread per node, tiles
 * of 32 x tile_h nodes, `threads` threads per block, each thread
 * 32 * tile_h / threads rows apart.  Shape 6 (pipelined = 1): the TMA-fed pipeline of the
 * single-lattice FP32 kernel over 96 x 8 tiles, one CTA per SM, available
 * for FP32 members (LBM_ERR_ARG otherwise) and the default where available.
 * Results do not depend on the shape; the speed does.  lbm_batch_time_steps
 * times n steps (eta = 1, the current edge data) in milliseconds, advancing
 * the members: an autotuner saves and restores them around it.
 * lbm_batch_shape_info returns LBM_ERR_ARG past the last shape. */
lbm_status lbm_batch_set_shape(lbm_batch* b, int shape);
lbm_status lbm_batch_get_shape(const lbm_batch* b, int* shape);
lbm_status lbm_batch_shape_info(int shape, int* tile_w, int* tile_h, int* threads,
                                int* pipelined);
lbm_status lbm_batch_time_steps(lbm_batch* b, int n, float* ms);
void lbm_batch_destroy(lbm_batch* b);  /* does not destroy the members */
const char* lbm_batch_last_error(void);

/* ---- the continuum solver of the hybrid method: Q1 finite elements --------
 * Sec. 3 (Galerkin, Sec. 3.1.1; SUPG, Sec. 3.1.2 Eq. "SUPG", "SUPG_tau") and
 * Sec. 6.1.1 (generalized trapezoidal rule, Eq. "FEM_discrete"): the
 * advection-diffusion equation dc/dt + v.grad c - D lap c = 0 with uniform D
 * and v on a structured mesh of nex x ney bilinear elements covering
 * [x0, x0 + nex hx] x [y0, y0 + ney hy], elements optionally switched off
 * (a hole where a lattice lives).  Each step solves
 *     (M + theta dt K) d^{n+1} = (M - (1 - theta) dt K) d^n
 * with the listed Dirichlet nodes at their prescribed values; every other
 * boundary (the mesh edge, the edge of switched-off elements) is zero-flux.
 * Nodes are numbered j (nex + 1) + i; nodal vectors are FP64.
 * The linear system is solved on the GPU (Jacobi-preconditioned BiCGSTAB,
 * FP64, to the relative residual tol), starting from the last converged
 * solution (after lbm_fem_set, the previous Schwarz iterate: a close guess),
 * or from d^n before the first.  Pointers may be host or device
 * memory; everything runs on `stream`.  Errors: LBM_ERR_ARG (bad parameters or
 * node ids), LBM_ERR_STATE (no convergence / breakdown of the linear solve),
 * LBM_ERR_NOMEM, LBM_ERR_CUDA; the message is in lbm_last_error(). */
typedef struct lbm_fem lbm_fem;
typedef struct {
  int nex, ney;            /* elements along x and y */
  double x0, y0, hx, hy;   /* origin and element size */
  double D, vx, vy;        /* diffusivity, velocity */
  double theta, dt;        /* trapezoidal weight in [0, 1], time step */
  int supg;                /* 1: SUPG test functions, 0: Galerkin */
  double tol;              /* relative residual of the solve (<= 0: 1e-12) */
  int max_iter;            /* solver iterations per step (<= 0: 1000) */
} lbm_fem_params;
/* elem_active [ney][nex] (NULL: all on); dir_nodes [n_dir] node ids of the
 * Dirichlet nodes, in the order of the values lbm_fem_step takes; d0 the
 * initial nodal values (NULL: zero). */
lbm_status lbm_fem_init(lbm_fem** out, const lbm_fem_params* p, const uint8_t* elem_active,
                        int n_dir, const int* dir_nodes, const double* d0, void* stream);
/* One time step; dir_values [n_dir] are the Dirichlet values at t^{n+1}. */
lbm_status lbm_fem_step(lbm_fem* f, const double* dir_values);
/* Finite-element (bilinear) interpolant of the current d at npts points
 * xy [npts][2] (physical coordinates; points outside are clamped to the
 * nearest element): the coarse-to-fine transfer of Sec. 5.1 / 6.2 (iii). */
lbm_status lbm_fem_interpolate(lbm_fem* f, int npts, const double* xy, double* out);
/* d [(ney+1)(nex+1)]: into device memory asynchronous on the solver's
 * stream, into host memory it waits. */
lbm_status lbm_fem_get(lbm_fem* f, double* d);
lbm_status lbm_fem_set(lbm_fem* f, const double* d);  /* e.g. the Schwarz rollback */
/* Iterations and relative residual of the last solve. */
lbm_status lbm_fem_solver_info(lbm_fem* f, int* iters, double* rel_resid);
void lbm_fem_destroy(lbm_fem* f);

/* FP64 sum of a concentration field that allocates nothing -- the paper has
 * no counterpart; this entry point exists for callers that cannot allocate
 * device memory when they need the sum: code running inside a device-memory
 * budget fixed at start-up (a later allocation may fail), or a host framework
 * that owns every allocation and forbids libraries to call cudaMalloc.
 *   u          device pointer to n values (float if precision is 32, double
 *              if 64), e.g. the [ny][nx] field of lbm_get_concentration
 *   n          1 .. 67,108,864 (8192 x 8192 nodes); larger n -> LBM_ERR_ARG
 *   mass_out   host or device pointer to one double; a host result is
 *              complete when the call returns (the call waits for the
 *              stream), a device result is ordered on `stream`.  A host
 *              mass_out on a stream in capture mode, where no wait is
 *              allowed, is refused with LBM_ERR_ARG
 *   stream     cudaStream_t of the work (NULL: legacy default stream)
 * The partial sums live in a fixed 64 KB array in the library's device
 * memory (every GPU that loads the library keeps it until the process exits);
 * the sum is taken in a fixed order, so repeated calls give identical
 * results.  The first call on a device looks up that array's device address
 * (with that device current), so make one call before recording any stream
 * capture.  All calls on a device share the array: calls that overlap on the
 * GPU (different streams without ordering between them) race.  On error,
 * lbm_mass_noalloc_error() describes it (per thread). */
lbm_status lbm_mass_noalloc(const void* u, int precision, long long n, double* mass_out,
                            void* stream);
const char* lbm_mass_noalloc_error(void);

/* ---- one lattice split into row slabs --------------------------------------
 * Sec. 5 decomposes a domain into overlapping subdomains that exchange data
 * on their interfaces; the lattice step reaches one node, so a lattice split
 * by rows needs an overlap of one row.  Each slab is a context of its own,
 * on its own GPU or several on one, and the caller moves two small messages
 * across every shared side per time step; the split lattice computes bit for
 * bit what the whole one does (populations, concentration, solid mask,
 * mineral, flip record), only the reductions of lbm_diagnostics are per
 * slab.
 *
 * lbm_init_slab makes the slab of rows y0 .. y1 - 1 (at least 2) of the
 * lattice p describes; every input array is the WHOLE lattice's ([ny][nx],
 * velocity [2][ny][nx]); the slab reads its rows, and the mask's rows next to
 * them.  A side inside the lattice (and both S and N of a y-periodic lattice
 * split in two or more) becomes LBM_EDGE_EXCHANGE.  Edge data of a slab use
 * its own edge layout [W: y1-y0][E: y1-y0][S: nx][N: nx].
 *
 * A time step of the split lattice, with the messages of each shared side
 * moved from the sender's pack buffer to the neighbour's unpack buffer:
 *   lbm_step_stream on every slab;
 *   phase 0: lbm_halo_pack(side, 0) on every shared side of every slab, then
 *            lbm_halo_unpack(side, 0) with the neighbour's message;
 *   lbm_step_dissolve on every slab;
 *   phase 1: the same with phase 1.
 * After lbm_init_slab, before the first step: phase 0, lbm_step_dissolve
 * (the first dissolution pass), phase 1.  lbm_substeps refuses a slab
 * (LBM_ERR_STATE): its halo must move between the halves of each step.
 *
 * A message of phase 0 carries the three populations that stream across the
 * side from the boundary row and, with dissolution, that row's reaction
 * shares; phase 1 carries the boundary row's solid and turning-fluid flags,
 * from which the receiver sets its links across the cut and lists the solid
 * nodes a neighbour's flip exposed.  lbm_halo_bytes gives a message's size
 * (the same for both sides).  Buffers are device memory of the slab's
 * device, caller-owned; pack and unpack are asynchronous on the slab's
 * stream.  Errors: LBM_ERR_ARG (a side that is not shared, a phase other
 * than 0 or 1, a host buffer), LBM_ERR_STATE (lbm_step_stream before the
 * first dissolution pass), LBM_ERR_CUDA. */
lbm_status lbm_init_slab(lbm_ctx** out, const lbm_params* p, int y0, int y1,
                         const uint8_t* solid, const double* vel, const double* k_field,
                         const double* mineral, const double* u0, void* stream);
lbm_status lbm_halo_bytes(lbm_ctx* c, int phase, size_t* bytes);
lbm_status lbm_halo_pack(lbm_ctx* c, int side, int phase, void* buf);
/* side: the side the message crossed (its neighbour's opposite side packed it) */
lbm_status lbm_halo_unpack(lbm_ctx* c, int side, int phase, const void* buf);
/* The two halves of one substep j of eta (lbm_substeps runs both for every
 * step of an unsplit lattice): the fused step -- streaming, boundary
 * conditions, collision; final_step nonzero also writes u and the mass
 * partials -- with the edge data of the last lbm_stage_edges, and the
 * dissolution pass (a no-op without dissolution). */
lbm_status lbm_stage_edges(lbm_ctx* c, const double* u_dir_t0, const double* u_dir_t1,
                           const double* q_neu);
lbm_status lbm_step_stream(lbm_ctx* c, int j, int eta, int final_step);
lbm_status lbm_step_dissolve(lbm_ctx* c);

/* ---- the D1Q2 lattice of the one-dimensional hybrid (Sec. 7.1) ------------
 * Nodes j = 0 .. n-1 of a line; velocities +-c (c = h / dt), weights 1/2,
 * c_s^2 = c^2, so in lattice units D dt / h^2 = tau - 1/2 and the equilibrium
 * (Eq. "LBM_feq") is f_+- = (u/2)(1 +- vl) with vl = v dt / h, |vl| < 1.  A
 * step streams the stored post-collision populations, sets the one unknown
 * population at each end by the maximum-entropy conditions of Sec. 4.1.1 --
 * a Dirichlet end (LBM_EDGE_DIRICHLET): the unknown takes the missing mass,
 * f = u^p - (the known one); a Neumann end (LBM_EDGE_NEUMANN): its unknown
 * has e.n = -1, so f = (the known one) - q^p, and zero flux is bounce-back --
 * takes u = f_+ + f_- and collides.  FP64 throughout; all n substeps of a
 * call run in one kernel launch.
 *   lbm1d_init: u0 [n] (NULL: zero), host or device; f = f^eq(u0).
 *   lbm1d_substeps: substeps j = 1..n of eta with the end data (left,
 *     right) interpolated as (1 - j/eta) ends_t0 + (j/eta) ends_t1 (Eq.
 *     "MTS"; ends_t1 NULL: equal to ends_t0; NULL: zero), q (left, right)
 *     the Neumann data, outward first moments; each a 2-element array, host
 *     or device.  Returns once the steps are done.
 *   lbm1d_get: u [n] at the current time (host or device).
 *   lbm1d_state_bytes / save / restore: the whole state (the Schwarz
 *     rollback of Algorithm 1), caller-owned buffer, host or device.
 * Errors: LBM_ERR_ARG (n < 2, tau <= 1/2, |vl| >= 1, an end kind other than
 * Dirichlet or Neumann, a null argument), LBM_ERR_NOMEM, LBM_ERR_CUDA. */
typedef struct lbm1d lbm1d;
lbm_status lbm1d_init(lbm1d** out, int n, double tau, double vl, int left, int right,
                      const double* u0, void* stream);
lbm_status lbm1d_substeps(lbm1d* c, int n, int eta, const double* ends_t0,
                          const double* ends_t1, const double* q);
lbm_status lbm1d_get(lbm1d* c, double* u);
lbm_status lbm1d_state_bytes(lbm1d* c, size_t* bytes);
lbm_status lbm1d_save(lbm1d* c, void* buf, size_t bytes);
lbm_status lbm1d_restore(lbm1d* c, const void* buf, size_t bytes);
void lbm1d_destroy(lbm1d* c);

/* Release the context's device memory (waits for its stream first). */
void lbm_destroy(lbm_ctx* c);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

/* LBM_ADE_ABI_VERSION of the loaded library. */
int lbm_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_ADE_H */
