/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle of the pore-scale lattice
 * Boltzmann advection-diffusion(-reaction) update with maximum-entropy
 * Dirichlet / Neumann boundary conditions.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library: the lattice constants below are typed out here on their own.
 *
 * One time step follows the order the paper prints it (Sec. 4.1 and
 * Algorithm 1): collide every fluid node (Eq. "Collision", with the
 * equilibrium of Eq. "LBM_feq"), stream by pushing each post-collision
 * population to its neighbour (Eq. "LBE"), impose the boundary conditions on
 * the populations that streaming left unknown (Sec. 4.1.1 (a) and (b)), then
 * take the moments (Eq. "LBM_Macro").
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes):
 *  - the equilibrium's last term is v.v/(2 c_s^2); the printed v.v/c_s^2 would
 *    make the collision destroy mass, against u = sum_i f_i (Sec. 4.1);
 *  - D2Q9 uses the textbook velocities and weights 4/9, 1/9, 1/36, c_s^2 = 1/3;
 *  - boundary nodes are wet nodes on the edge; the unknown populations are the
 *    ones whose upstream neighbour lies outside the lattice, which on a straight
 *    edge is exactly the set M^- of Eq. "Boundary_Vel";
 *  - Dirichlet data that leave no non-negative solution are applied literally
 *    (unknowns may go negative) and counted; Neumann data with no root are met
 *    by the gamma -> -infinity limit (unknowns set to zero) and counted;
 *  - at a corner of two Neumann edges the normal is the normalised sum of the
 *    two outward normals; unknowns with e_i.n = 0 are filled by halfway
 *    bounce-back; a corner that touches a Dirichlet edge is Dirichlet over all
 *    of its unknowns;
 *  - the reaction is an explicit first-order sink applied after collision,
 *    f*_i -= w_i k u, at reactive fluid nodes (fluid nodes with a solid D2Q9
 *    neighbour, or every fluid node in bulk mode);
 *  - with dissolution on, the mass removed at a fluid node is taken from its
 *    solid neighbours in proportion to the link weights w_j; a solid node whose
 *    mineral mass reaches zero or less after a step becomes fluid with all
 *    populations zero;
 *  - Dirichlet data inside a run of eta substeps are interpolated linearly in
 *    time: substep j uses (1 - j/eta) a + (j/eta) b (Eq. "MTS");
 *  - pore walls take halfway bounce-back by default; as the option of the
 *    paper's own kind (Sec. 4.1.1 (b) with zero flux) their normal is the
 *    lattice-weighted direction to the node's solid neighbours, unknowns
 *    tangent to it take bounce-back, a cancelling sum (one-node channel)
 *    takes bounce-back throughout, and nodes on an open lattice side keep
 *    bounce-back at their solid links (their edge condition sets the rest).
 *
 * Memory: the oracle owns copies of everything it is given.  Arrays are
 * row-major [ny][nx]; populations are [9][ny][nx].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- D2Q9 lattice (textbook), c_s^2 = 1/3 -------------------------------- */
enum { NQ = 9 };
static const int CX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* direction pointing the other way: CX[REV[i]] == -CX[i], CY[REV[i]] == -CY[i] */
static int reverse_of(int i) {
  for (int j = 0; j < NQ; ++j)
    if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
  return -1;
}

enum { EDGE_PERIODIC = 0, EDGE_DIRICHLET = 1, EDGE_NEUMANN = 2 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { REACT_NONE = 0, REACT_SURFACE = 1, REACT_BULK = 2 };
enum { WALL_BOUNCE = 0, WALL_MAXENT = 1 };

typedef struct {
  int nx, ny;
  int edge[4];
  double tau;
  int react_mode;
  double k_scalar;
  int dissolution;
  int wall_mode;   /* WALL_BOUNCE or WALL_MAXENT (pore walls)      */
  double *k;       /* [ny][nx] rate, used where reactive          */
  double *vel;     /* [2][ny][nx]                                  */
  uint8_t *solid;  /* [ny][nx] 1 = solid                           */
  double *mineral; /* [ny][nx] mineral mass of solid nodes         */
  int *flip_step;  /* [ny][nx] steps after which a node was first fluid
                      by dissolution (-1: never) -- bookkeeping only */
  double *f;       /* [9][ny][nx] populations after BC (state)     */
  double *fpost;   /* [9][ny][nx] post-collision populations       */
  double *fnew;    /* [9][ny][nx] streamed populations             */
  uint8_t *known;  /* [9][ny][nx] 1 = set by streaming             */
  double *u;       /* [ny][nx] concentration at the current time   */
  long long steps;
  long long bc_infeasible;
  long long flips;
  long long newton_iters;
  long long newton_fail;
  double J;        /* sum over steps of the east-edge fluid concentrations */
  double reacted;  /* total mass removed by the sink                        */
} or_lbm;

static size_t nn(const or_lbm *o) { return (size_t)o->nx * (size_t)o->ny; }
static size_t at(const or_lbm *o, int x, int y) {
  return (size_t)y * (size_t)o->nx + (size_t)x;
}

/* Wrap (x, y) through periodic edges.  Returns 0 if the point lies outside
 * the lattice across a non-periodic edge. */
static int locate(const or_lbm *o, int x, int y, int *ox, int *oy) {
  if (x < 0 || x >= o->nx) {
    if (o->edge[SIDE_W] != EDGE_PERIODIC) return 0;
    x = ((x % o->nx) + o->nx) % o->nx;
  }
  if (y < 0 || y >= o->ny) {
    if (o->edge[SIDE_S] != EDGE_PERIODIC) return 0;
    y = ((y % o->ny) + o->ny) % o->ny;
  }
  *ox = x;
  *oy = y;
  return 1;
}

static int is_solid(const or_lbm *o, int x, int y) {
  int a, b;
  if (!locate(o, x, y, &a, &b)) return 0;
  return o->solid[at(o, a, b)] != 0;
}

/* Second-order equilibrium, Eq. "LBM_feq" with the v.v/(2 c_s^2) reading. */
static double feq(int i, double u, double vx, double vy) {
  double ev = CX[i] * vx + CY[i] * vy;
  double vv = vx * vx + vy * vy;
  return WT[i] * u *
         (1.0 + ev / CS2 + 0.5 * ev * ev / (CS2 * CS2) - 0.5 * vv / CS2);
}

/* A fluid node is reactive in surface mode when one of its 8 neighbours is
 * solid; in bulk mode every fluid node is reactive. */
static int reactive(const or_lbm *o, int x, int y) {
  if (o->solid[at(o, x, y)]) return 0;
  if (o->react_mode == REACT_BULK) return 1;
  if (o->react_mode != REACT_SURFACE) return 0;
  for (int i = 1; i < NQ; ++i)
    if (is_solid(o, x + CX[i], y + CY[i])) return 1;
  return 0;
}

/* Sum of the link weights from fluid node (x,y) to its solid neighbours. */
static double solid_link_weight(const or_lbm *o, int x, int y) {
  double s = 0.0;
  for (int i = 1; i < NQ; ++i)
    if (is_solid(o, x + CX[i], y + CY[i])) s += WT[i];
  return s;
}

static void moments(or_lbm *o) {
  size_t N = nn(o);
#pragma omp parallel for schedule(static)
  for (size_t n = 0; n < N; ++n) {
    double s = 0.0;
    if (!o->solid[n])
      for (int i = 0; i < NQ; ++i) s += o->f[(size_t)i * N + n];
    o->u[n] = s;
  }
}

/* ---- single-node maximum-entropy solutions (Sec. 4.1.1) ------------------ */

/* Dirichlet, Sec. 4.1.1 (a): the unknowns (mask unk[i] = 1) that minimise
 * H = sum f log(f/w) with sum_i f_i = up are f_i = w_i / sum_unk w *
 * (up - sum_known f).  Returns 1 if the data leave no non-negative solution. */
int or_maxent_dirichlet(double *f, const int *unk, double up) {
  double wu = 0.0, known = 0.0;
  for (int i = 0; i < NQ; ++i) {
    if (unk[i]) wu += WT[i];
    else known += f[i];
  }
  double rest = up - known;
  for (int i = 0; i < NQ; ++i)
    if (unk[i]) f[i] = WT[i] / wu * rest;
  return rest < 0.0;
}

/* Neumann, Sec. 4.1.1 (b): unknowns in M^- = {i: unk[i], e_i.n < 0} take
 * f_i = w_i exp(-1 - gamma e_i.n), with gamma the root of
 *   sum_{M^-} w_i (e_i.n) exp(-1 - gamma e_i.n) = q - sum_{not M^-} (e_j.n) f_j.
 * Unknowns with e_i.n >= 0 must already hold a value (the caller fills them).
 * The left side runs over (-inf, 0) and falls strictly with gamma, so a root
 * exists iff the right side R < 0; it is found by Newton's method kept inside
 * a bracket (bisection when a Newton step leaves it).  For R >= 0 the M^-
 * unknowns are set to 0, the limit gamma -> -inf.  Returns 1 when R > 0
 * (infeasible data), 0 otherwise; *iters receives the Newton iterations, and
 * *fail is set if the iteration did not converge. */
int or_maxent_neumann(double *f, const int *unk, double nxn, double nyn,
                      double q, long long *iters, int *fail) {
  double a[NQ];
  int inm[NQ];
  double R = q;
  int any = 0;
  *fail = 0;
  for (int i = 0; i < NQ; ++i) {
    a[i] = CX[i] * nxn + CY[i] * nyn;
    inm[i] = unk[i] && a[i] < 0.0;
    if (inm[i]) any = 1;
    else R -= a[i] * f[i];
  }
  if (!any) return 0;
  if (!(R < 0.0)) {
    for (int i = 0; i < NQ; ++i)
      if (inm[i]) f[i] = 0.0;
    return R > 0.0;
  }
  /* g(gamma) = sum_{M^-} w a exp(-1 - gamma a) - R ; g decreasing. */
  double lo = -1.0, hi = 1.0;
#define G_OF(gm, gout, dout)                                   \
  do {                                                         \
    double s_ = 0.0, d_ = 0.0;                                 \
    for (int i_ = 0; i_ < NQ; ++i_)                            \
      if (inm[i_]) {                                           \
        double e_ = WT[i_] * exp(-1.0 - (gm) * a[i_]);         \
        s_ += a[i_] * e_;                                      \
        d_ -= a[i_] * a[i_] * e_;                              \
      }                                                        \
    gout = s_ - R;                                             \
    dout = d_;                                                 \
  } while (0)
  double glo, ghi, dd;
  G_OF(lo, glo, dd);
  while (glo < 0.0) { lo = 2.0 * lo - 1.0; G_OF(lo, glo, dd); }
  G_OF(hi, ghi, dd);
  while (ghi > 0.0) { hi = 2.0 * hi + 1.0; G_OF(hi, ghi, dd); }
  double gm = 0.5 * (lo + hi);
  int it = 0, done = 0;
  for (; it < 200; ++it) {
    double g, dg;
    G_OF(gm, g, dg);
    if (g == 0.0) { done = 1; break; }
    if (g > 0.0) lo = gm; else hi = gm;
    double nx_ = gm - g / dg;
    if (!(nx_ > lo && nx_ < hi)) nx_ = 0.5 * (lo + hi);
    if (fabs(nx_ - gm) <= 1e-15 * (1.0 + fabs(gm))) { gm = nx_; done = 1; break; }
    gm = nx_;
  }
#undef G_OF
  *iters += it + 1;
  if (!done) *fail = 1;
  for (int i = 0; i < NQ; ++i)
    if (inm[i]) f[i] = WT[i] * exp(-1.0 - gm * a[i]);
  return 0;
}

/* ---- construction -------------------------------------------------------- */

or_lbm *or_lbm_new(int nx, int ny, const int *edge, double tau,
                   int react_mode, double k_scalar, const double *k_field,
                   int dissolution, const uint8_t *solid, const double *vel,
                   const double *mineral, const double *u0) {
  or_lbm *o = (or_lbm *)calloc(1, sizeof(or_lbm));
  if (!o) return NULL;
  o->nx = nx;
  o->ny = ny;
  memcpy(o->edge, edge, sizeof(o->edge));
  o->tau = tau;
  o->react_mode = react_mode;
  o->k_scalar = k_scalar;
  o->dissolution = dissolution;
  size_t N = nn(o);
  o->k = (double *)malloc(N * sizeof(double));
  o->vel = (double *)malloc(2 * N * sizeof(double));
  o->solid = (uint8_t *)malloc(N);
  o->mineral = (double *)malloc(N * sizeof(double));
  o->flip_step = (int *)malloc(N * sizeof(int));
  o->f = (double *)calloc(NQ * N, sizeof(double));
  o->fpost = (double *)calloc(NQ * N, sizeof(double));
  o->fnew = (double *)calloc(NQ * N, sizeof(double));
  o->known = (uint8_t *)calloc(NQ * N, 1);
  o->u = (double *)calloc(N, sizeof(double));
  for (size_t n = 0; n < N; ++n) {
    o->k[n] = k_field ? k_field[n] : k_scalar;
    o->solid[n] = solid ? (solid[n] ? 1 : 0) : 0;
    o->mineral[n] = mineral ? mineral[n] : 1.0;
    o->flip_step[n] = -1;
    o->vel[n] = vel ? vel[n] : 0.0;
    o->vel[N + n] = vel ? vel[N + n] : 0.0;
  }
  /* Initialisation, Sec. 6.2 (i): f_i(x, 0) = f_i^eq(x, 0; u_0(x)). */
  for (size_t n = 0; n < N; ++n) {
    if (o->solid[n]) continue;
    for (int i = 0; i < NQ; ++i)
      o->f[(size_t)i * N + n] = feq(i, u0 ? u0[n] : 0.0, o->vel[n], o->vel[N + n]);
  }
  moments(o);
  return o;
}

void or_lbm_free(or_lbm *o) {
  if (!o) return;
  free(o->k); free(o->vel); free(o->solid); free(o->mineral); free(o->flip_step);
  free(o->f); free(o->fpost); free(o->fnew); free(o->known); free(o->u);
  free(o);
}

/* ---- one time step -------------------------------------------------------- */

/* Value index of edge node (x, y) on side s in the edge-data layout
 * [W: ny][E: ny][S: nx][N: nx]. */
static size_t edge_slot(const or_lbm *o, int s, int x, int y) {
  switch (s) {
    case SIDE_W: return (size_t)y;
    case SIDE_E: return (size_t)o->ny + (size_t)y;
    case SIDE_S: return 2 * (size_t)o->ny + (size_t)x;
    default: return 2 * (size_t)o->ny + (size_t)o->nx + (size_t)x;
  }
}

/* Collision with reaction sink; mineral bookkeeping. */
static double collide(or_lbm *o, double *fout) {
  size_t N = nn(o);
  const double omega = 1.0 / o->tau;
  double removed = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : removed)
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      size_t n = at(o, x, y);
      if (o->solid[n]) continue;
      double u = 0.0;
      for (int i = 0; i < NQ; ++i) u += o->f[(size_t)i * N + n];
      double kr = reactive(o, x, y) ? o->k[n] : 0.0;
      for (int i = 0; i < NQ; ++i) {
        double fi = o->f[(size_t)i * N + n];
        double post = fi + omega * (feq(i, u, o->vel[n], o->vel[N + n]) - fi);
        fout[(size_t)i * N + n] = post - WT[i] * kr * u;
      }
      removed += kr * u;
    }
  return removed;
}

/* Mineral decrement: the sink k u at a reactive fluid node x is taken from
 * its solid neighbours y = x + e_j in proportion to w_j.  Gathered per solid
 * node so that each node's update is one plain sum. */
static void dissolve_gather(or_lbm *o) {
  size_t N = nn(o);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      size_t n = at(o, x, y);
      if (!o->solid[n]) continue;
      double take = 0.0;
      for (int j = 1; j < NQ; ++j) {
        int sx, sy; /* the fluid node whose link j points at (x, y) */
        if (!locate(o, x - CX[j], y - CY[j], &sx, &sy)) continue;
        size_t s = at(o, sx, sy);
        if (o->solid[s] || !reactive(o, sx, sy)) continue;
        double us = 0.0;
        for (int i = 0; i < NQ; ++i) us += o->f[(size_t)i * N + s];
        take += o->k[s] * us * WT[j] / solid_link_weight(o, sx, sy);
      }
      o->mineral[n] -= take;
    }
  (void)N;
}

/* True at nodes on a side that is not periodic (they have pulls from outside
   the lattice). */
static int on_open_side(const or_lbm *o, int x, int y) {
  return (x == 0 && o->edge[SIDE_W] != EDGE_PERIODIC) ||
         (x == o->nx - 1 && o->edge[SIDE_E] != EDGE_PERIODIC) ||
         (y == 0 && o->edge[SIDE_S] != EDGE_PERIODIC) ||
         (y == o->ny - 1 && o->edge[SIDE_N] != EDGE_PERIODIC);
}

/* Push streaming with halfway bounce-back at solid neighbours. */
static void stream(or_lbm *o) {
  size_t N = nn(o);
  memset(o->known, 0, NQ * N);
  memset(o->fnew, 0, NQ * N * sizeof(double));
  /* each (population, node) of fnew has exactly one writer, so rows can be
     streamed in parallel */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      size_t n = at(o, x, y);
      if (o->solid[n]) continue;
      for (int i = 0; i < NQ; ++i) {
        double v = o->fpost[(size_t)i * N + n];
        int tx, ty;
        if (!locate(o, x + CX[i], y + CY[i], &tx, &ty)) continue; /* leaves */
        size_t t = at(o, tx, ty);
        if (o->solid[t]) {
          /* halfway bounce-back; with max-entropy walls the population that
             would come back is left unknown for apply_walls, except at nodes
             on a non-periodic lattice side (their edge condition settles
             them, with bounce-back at their solid links) */
          if (o->wall_mode == WALL_MAXENT && !on_open_side(o, x, y)) continue;
          int r = reverse_of(i);
          o->fnew[(size_t)r * N + n] = v;
          o->known[(size_t)r * N + n] = 1;
        } else {
          o->fnew[(size_t)i * N + t] = v;
          o->known[(size_t)i * N + t] = 1;
        }
      }
    }
}

static void apply_bc(or_lbm *o, int j, int eta, const double *ua,
                     const double *ub, const double *q) {
  size_t N = nn(o);
  const double frac = (double)j / (double)eta;
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      size_t n = at(o, x, y);
      if (o->solid[n]) continue;
      int on[4] = {x == 0 && o->edge[SIDE_W] != EDGE_PERIODIC,
                   x == o->nx - 1 && o->edge[SIDE_E] != EDGE_PERIODIC,
                   y == 0 && o->edge[SIDE_S] != EDGE_PERIODIC,
                   y == o->ny - 1 && o->edge[SIDE_N] != EDGE_PERIODIC};
      if (!(on[0] || on[1] || on[2] || on[3])) continue;
      double f[NQ];
      int unk[NQ], nunk = 0;
      for (int i = 0; i < NQ; ++i) {
        f[i] = o->fnew[(size_t)i * N + n];
        unk[i] = !o->known[(size_t)i * N + n];
        nunk += unk[i];
      }
      if (!nunk) continue;
      int dside = -1, nside = -1;
      for (int s = 0; s < 4; ++s) {
        if (!on[s]) continue;
        if (o->edge[s] == EDGE_DIRICHLET && dside < 0) dside = s;
        if (o->edge[s] == EDGE_NEUMANN && nside < 0) nside = s;
      }
      if (dside >= 0) {
        size_t e = edge_slot(o, dside, x, y);
        double a = ua ? ua[e] : 0.0, b = ub ? ub[e] : 0.0;
        double up = (1.0 - frac) * a + frac * b; /* Eq. "MTS" */
        o->bc_infeasible += or_maxent_dirichlet(f, unk, up);
      } else {
        /* outward normal: normalised sum over the node's Neumann sides */
        double nxn = 0.0, nyn = 0.0;
        static const double SN[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        for (int s = 0; s < 4; ++s)
          if (on[s] && o->edge[s] == EDGE_NEUMANN) {
            nxn += SN[s][0];
            nyn += SN[s][1];
          }
        double len = sqrt(nxn * nxn + nyn * nyn);
        nxn /= len;
        nyn /= len;
        /* unknowns tangent to the normal: halfway bounce-back */
        for (int i = 0; i < NQ; ++i)
          if (unk[i] && CX[i] * nxn + CY[i] * nyn >= 0.0) {
            f[i] = o->fpost[(size_t)reverse_of(i) * N + n];
            unk[i] = 0;
          }
        double qv = q ? q[edge_slot(o, nside, x, y)] : 0.0;
        int fail = 0;
        o->bc_infeasible +=
            or_maxent_neumann(f, unk, nxn, nyn, qv, &o->newton_iters, &fail);
        o->newton_fail += fail;
      }
      for (int i = 0; i < NQ; ++i) o->fnew[(size_t)i * N + n] = f[i];
    }
}

/* Pore walls as zero-flux boundaries of the maximum-entropy kind, Sec. 4.1.1
 * (b) with q = 0 (the paper's reading of a wall as a bath in equilibrium, as
 * against bounce-back).  At a fluid node off the open lattice sides the
 * unknowns are the populations whose source x - e_i is solid.  The outward
 * normal is the lattice-weighted direction to the solid neighbours,
 * n = sum over solid neighbours x + e_k of w_k e_k, normalised; unknowns with
 * e_i . n >= 0 (tangent to the wall or pointing into it) take halfway
 * bounce-back, as at a corner of two Neumann sides, and the rest follow from
 * the Lagrange multiplier of the flux constraint.  Where the weighted
 * directions cancel (a one-node channel) every unknown takes bounce-back. */
static void apply_walls(or_lbm *o) {
  size_t N = nn(o);
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      size_t n = at(o, x, y);
      if (o->solid[n] || on_open_side(o, x, y)) continue;
      double f[NQ];
      /* the normal scaled by 36 (the weights are 4/36 and 1/36): integers, so
         which unknowns are tangent to it, and whether it cancels, is exact */
      int unk[NQ], nunk = 0, mx = 0, my = 0;
      for (int i = 0; i < NQ; ++i) {
        f[i] = o->fnew[(size_t)i * N + n];
        unk[i] = !o->known[(size_t)i * N + n];
        nunk += unk[i];
        if (unk[i]) { /* source x - e_i is solid: the solid neighbour lies along -e_i */
          int w36 = (CX[i] != 0 && CY[i] != 0) ? 1 : 4;
          mx -= w36 * CX[i];
          my -= w36 * CY[i];
        }
      }
      if (!nunk) continue;
      double nxn = 0.0, nyn = 0.0;
      if (mx != 0 || my != 0) {
        double len = sqrt((double)(mx * mx + my * my));
        nxn = mx / len;
        nyn = my / len;
      }
      for (int i = 0; i < NQ; ++i)
        if (unk[i] && CX[i] * mx + CY[i] * my >= 0) {
          f[i] = o->fpost[(size_t)reverse_of(i) * N + n];
          unk[i] = 0;
        }
      int fail = 0;
      o->bc_infeasible += or_maxent_neumann(f, unk, nxn, nyn, 0.0, &o->newton_iters, &fail);
      o->newton_fail += fail;
      for (int i = 0; i < NQ; ++i) o->fnew[(size_t)i * N + n] = f[i];
    }
}

void or_lbm_set_wall_mode(or_lbm *o, int mode) { o->wall_mode = mode; }

/* Run n substeps j = 1..n of a coarse step split eta ways.  ua, ub: Dirichlet
 * data at the start and the end of the coarse step, q: Neumann data, each in
 * the edge layout [W: ny][E: ny][S: nx][N: nx] (NULL means zero). */
void or_lbm_substeps(or_lbm *o, int n, int eta, const double *ua,
                     const double *ub, const double *q) {
  size_t N = nn(o);
  for (int j = 1; j <= n; ++j) {
    /* collide (with the reaction sink) */
    o->reacted += collide(o, o->fpost);
    if (o->dissolution && o->react_mode == REACT_SURFACE) dissolve_gather(o);
    /* stream, then boundary conditions */
    stream(o);
    apply_bc(o, j, eta, ua, ub, q);
    if (o->wall_mode == WALL_MAXENT) apply_walls(o);
    memcpy(o->f, o->fnew, NQ * N * sizeof(double));
    /* dissolution: solid nodes whose mineral is used up become fluid */
    if (o->dissolution && o->react_mode == REACT_SURFACE)
      for (size_t m = 0; m < N; ++m)
        if (o->solid[m] && o->mineral[m] <= 0.0) {
          o->solid[m] = 0;
          o->flip_step[m] = (int)(o->steps + 1);
          for (int i = 0; i < NQ; ++i) o->f[(size_t)i * N + m] = 0.0;
          o->flips += 1;
        }
    moments(o);
    for (int y = 0; y < o->ny; ++y)
      if (!o->solid[at(o, o->nx - 1, y)]) o->J += o->u[at(o, o->nx - 1, y)];
    o->steps += 1;
  }
}

/* ---- read-out ------------------------------------------------------------- */

void or_lbm_get_u(const or_lbm *o, double *out) { memcpy(out, o->u, nn(o) * sizeof(double)); }
void or_lbm_get_f(const or_lbm *o, double *out) { memcpy(out, o->f, NQ * nn(o) * sizeof(double)); }
void or_lbm_get_solid(const or_lbm *o, uint8_t *out) { memcpy(out, o->solid, nn(o)); }
void or_lbm_get_mineral(const or_lbm *o, double *out) { memcpy(out, o->mineral, nn(o) * sizeof(double)); }
void or_lbm_get_flip_steps(const or_lbm *o, int *out) { memcpy(out, o->flip_step, nn(o) * sizeof(int)); }

/* Post-collision populations of the current state (what the next step would
 * stream), for comparing against a solver that stores them. */
void or_lbm_get_fpost(or_lbm *o, double *out) {
  memset(out, 0, NQ * nn(o) * sizeof(double)); /* solid nodes hold no populations */
  (void)collide(o, out);
}

/* diag: [mass, J, reacted, bc_infeasible, flips, newton_iters, newton_fail, steps] */
void or_lbm_diag(const or_lbm *o, double *d) {
  double m = 0.0;
  for (size_t n = 0; n < nn(o); ++n) m += o->u[n];
  d[0] = m;
  d[1] = o->J;
  d[2] = o->reacted;
  d[3] = (double)o->bc_infeasible;
  d[4] = (double)o->flips;
  d[5] = (double)o->newton_iters;
  d[6] = (double)o->newton_fail;
  d[7] = (double)o->steps;
}

/* Boltzmann H of Eq. "BH" summed over fluid nodes; +inf if some f < 0. */
double or_lbm_H(const or_lbm *o) {
  size_t N = nn(o);
  double h = 0.0;
  for (size_t n = 0; n < N; ++n) {
    if (o->solid[n]) continue;
    for (int i = 0; i < NQ; ++i) {
      double v = o->f[(size_t)i * N + n];
      if (v < 0.0) return INFINITY;
      if (v > 0.0) h += v * log(v / WT[i]);
    }
  }
  return h;
}

/* LBM -> FEM transfer, Sec. 6.2 (ii): bilinear value of u at lattice
 * coordinates (px, py) from the four surrounding nodes.  Periodic edges wrap;
 * across a non-periodic edge the point must lie inside [0, n-1]. */
double or_trace_point(const or_lbm *o, double px, double py) {
  int x1 = (int)floor(px), y1 = (int)floor(py);
  if (o->edge[SIDE_W] != EDGE_PERIODIC && x1 >= o->nx - 1) x1 = o->nx - 2;
  if (o->edge[SIDE_S] != EDGE_PERIODIC && y1 >= o->ny - 1) y1 = o->ny - 2;
  double gx = px - x1, gy = py - y1;
  int ax, ay, bx, by;
  locate(o, x1, y1, &ax, &ay);
  locate(o, x1 + 1, y1 + 1, &bx, &by);
  double u1 = o->u[at(o, ax, ay)], u2 = o->u[at(o, bx, ay)];
  double u3 = o->u[at(o, bx, by)], u4 = o->u[at(o, ax, by)];
  return u1 * (1 - gx) * (1 - gy) + u2 * gx * (1 - gy) + u3 * gx * gy +
         u4 * (1 - gx) * gy;
}

/* ---- discrete adjoint of or_lbm_substeps ----------------------------------
 *
 * The paper differentiates nothing; this is the reverse mode of the oracle's
 * own substep, written out by hand, for a fixed solid mask (dissolution off:
 * a flip is not differentiable).  With the mask fixed one substep maps the
 * pre-collision state g^{n-1} to g^n by collision (with the sink), push
 * streaming with bounce-back, the boundary conditions and the moments; it is
 * affine in g and in the edge data, except that a Neumann node switches
 * between the root of Sec. 4.1.1 (b) and the zero limit with the sign of R.
 * The objective is the outlet breakthrough
 *   J = sum_{n=1..N} sum_{east-edge fluid nodes} u^n,
 * and the gradients are taken with respect to the rate k(x) of every node,
 * the Dirichlet data a, b of Eq. "MTS" and the Neumann data q, holding the
 * pre-collision state at the start of the call fixed.
 *
 * Forward: the substeps of or_lbm_substeps, keeping u^{n-1} (the input of
 * each collision) and, at Neumann nodes, whether the root was taken (R < 0).
 * Reverse, n = N .. 1, from gbar = dJ/dg^n (initially the direct term e(x),
 * 1 at east-edge fluid nodes, 0 elsewhere):
 *  - boundary conditions: the unknown entries were set from the known ones,
 *    so their adjoint moves onto the known entries and the data --
 *    Dirichlet f_i = w_i / W_U (u^p - sum_known f):
 *      t = sum_U w_i gbar_i / W_U, pbar_known -= t, d/du^p += t;
 *    Neumann on an axis side with the root, f_i = w_i / W_U (sum a_j f_j - q):
 *      pbar_j += a_j t for the known j, d/dq -= t; with the zero limit the
 *      unknowns depend on nothing;
 *  - streaming: F_i(y) went to y + e_i if that node is fluid, back to y as
 *    direction rev(i) if it is solid, nowhere if it lies outside:
 *      Fbar_i(y) = pbar_i(y + e_i), pbar_rev(i)(y) or 0;
 *  - collision, F_i = (1 - omega) g_i + w_i (omega P_i - k) u, u = sum_j g_j,
 *    with feq_i = w_i P_i u (Eq. "LBM_feq") and the sink of k at reactive
 *    nodes:
 *      gbar_j = (1 - omega) Fbar_j + sum_i w_i (omega P_i - k) Fbar_i
 *               (+ e(x) when n - 1 >= 1),
 *      dJ/dk(x) += -u^{n-1}(x) sum_i w_i Fbar_i at reactive nodes.
 * The state advances by N substeps, as with or_lbm_substeps.  Outputs may be
 * NULL.  Returns 0; -1 if dissolution is on; -2 if two Neumann sides meet at
 * a corner (that root is not affine in the data); -3 if memory ran out.
 */
int or_lbm_adjoint(or_lbm *o, int nsteps, int eta, const double *ua,
                   const double *ub, const double *q, double *J_out,
                   double *grad_k, double *grad_ua, double *grad_ub,
                   double *grad_q) {
  if (o->dissolution) return -1;
  if (o->wall_mode != WALL_BOUNCE) return -4; /* the transpose covers bounce-back walls */
  const int np_x = o->edge[SIDE_W] != EDGE_PERIODIC;
  const int np_y = o->edge[SIDE_S] != EDGE_PERIODIC;
  if (np_x && np_y) {
    const int xs[2] = {SIDE_W, SIDE_E}, ys[2] = {SIDE_S, SIDE_N};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        if (o->edge[xs[a]] == EDGE_NEUMANN && o->edge[ys[b]] == EDGE_NEUMANN) return -2;
  }
  const size_t N = nn(o);
  const size_t ne = 2 * ((size_t)o->nx + (size_t)o->ny);
  const int steps = nsteps > 0 ? nsteps : 0;
  double *uh = (double *)malloc(((size_t)steps + 1) * N * sizeof(double));
  uint8_t *root = (uint8_t *)calloc((size_t)steps * ne + 1, 1);
  double *gbar = (double *)calloc(NQ * N, sizeof(double));
  double *pbar = (double *)calloc(NQ * N, sizeof(double));
  double *Fbar = (double *)calloc(NQ * N, sizeof(double));
  if (!uh || !root || !gbar || !pbar || !Fbar) {
    free(uh); free(root); free(gbar); free(pbar); free(Fbar);
    return -3;
  }
  if (grad_k) memset(grad_k, 0, N * sizeof(double));
  if (grad_ua) memset(grad_ua, 0, ne * sizeof(double));
  if (grad_ub) memset(grad_ub, 0, ne * sizeof(double));
  if (grad_q) memset(grad_q, 0, ne * sizeof(double));
  const double omega = 1.0 / o->tau;
  static const double SN[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};

  /* ---- forward, recording u^{n-1} and the Neumann branches ---- */
  const double J0 = o->J;
  for (int n = 1; n <= steps; ++n) {
    memcpy(uh + (size_t)(n - 1) * N, o->u, N * sizeof(double));
    o->reacted += collide(o, o->fpost);
    stream(o);
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        size_t m = at(o, x, y);
        if (o->solid[m]) continue;
        for (int s = 0; s < 4; ++s) {
          int on = (s == SIDE_W && x == 0) || (s == SIDE_E && x == o->nx - 1) ||
                   (s == SIDE_S && y == 0) || (s == SIDE_N && y == o->ny - 1);
          if (!on || o->edge[s] != EDGE_NEUMANN) continue;
          /* this node is Neumann unless a Dirichlet side also holds it */
          int dir = 0;
          for (int t = 0; t < 4; ++t) {
            int on2 = (t == SIDE_W && x == 0) || (t == SIDE_E && x == o->nx - 1) ||
                      (t == SIDE_S && y == 0) || (t == SIDE_N && y == o->ny - 1);
            if (on2 && o->edge[t] == EDGE_DIRICHLET) dir = 1;
          }
          if (dir) break;
          size_t e = edge_slot(o, s, x, y);
          double R = q ? q[e] : 0.0;
          for (int i = 0; i < NQ; ++i)
            if (o->known[(size_t)i * N + m])
              R -= (CX[i] * SN[s][0] + CY[i] * SN[s][1]) * o->fnew[(size_t)i * N + m];
          root[(size_t)(n - 1) * ne + e] = R < 0.0;
          break;
        }
      }
    apply_bc(o, n, eta, ua, ub, q);
    memcpy(o->f, o->fnew, NQ * N * sizeof(double));
    moments(o);
    for (int y = 0; y < o->ny; ++y)
      if (!o->solid[at(o, o->nx - 1, y)]) o->J += o->u[at(o, o->nx - 1, y)];
    o->steps += 1;
  }
  if (J_out) *J_out = o->J - J0;

  /* ---- reverse sweep ---- */
  for (int y = 0; y < o->ny; ++y) {
    size_t m = at(o, o->nx - 1, y);
    if (!o->solid[m])
      for (int i = 0; i < NQ; ++i) gbar[(size_t)i * N + m] = 1.0;
  }
  for (int n = steps; n >= 1; --n) {
    const double frac = (double)n / (double)eta;
    /* boundary conditions */
    memcpy(pbar, gbar, NQ * N * sizeof(double));
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        size_t m = at(o, x, y);
        if (o->solid[m]) continue;
        int on[4] = {x == 0 && o->edge[SIDE_W] != EDGE_PERIODIC,
                     x == o->nx - 1 && o->edge[SIDE_E] != EDGE_PERIODIC,
                     y == 0 && o->edge[SIDE_S] != EDGE_PERIODIC,
                     y == o->ny - 1 && o->edge[SIDE_N] != EDGE_PERIODIC};
        int unk[NQ], nunk = 0;
        for (int i = 0; i < NQ; ++i) {
          int sx, sy;
          unk[i] = !locate(o, x - CX[i], y - CY[i], &sx, &sy);
          nunk += unk[i];
        }
        if (!nunk) continue;
        int dside = -1, nside = -1;
        for (int s = 0; s < 4; ++s) {
          if (!on[s]) continue;
          if (o->edge[s] == EDGE_DIRICHLET && dside < 0) dside = s;
          if (o->edge[s] == EDGE_NEUMANN && nside < 0) nside = s;
        }
        double wu = 0.0, t = 0.0;
        for (int i = 0; i < NQ; ++i)
          if (unk[i]) wu += WT[i];
        for (int i = 0; i < NQ; ++i)
          if (unk[i]) t += WT[i] * gbar[(size_t)i * N + m] / wu;
        if (dside >= 0) {
          size_t e = edge_slot(o, dside, x, y);
          for (int i = 0; i < NQ; ++i)
            if (!unk[i]) pbar[(size_t)i * N + m] -= t;
          if (grad_ua) grad_ua[e] += (1.0 - frac) * t;
          if (grad_ub) grad_ub[e] += frac * t;
        } else {
          size_t e = edge_slot(o, nside, x, y);
          if (root[(size_t)(n - 1) * ne + e]) {
            for (int i = 0; i < NQ; ++i)
              if (!unk[i])
                pbar[(size_t)i * N + m] +=
                    (CX[i] * SN[nside][0] + CY[i] * SN[nside][1]) * t;
            if (grad_q) grad_q[e] -= t;
          }
        }
        for (int i = 0; i < NQ; ++i)
          if (unk[i]) pbar[(size_t)i * N + m] = 0.0;
      }
    /* streaming */
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        size_t m = at(o, x, y);
        for (int i = 0; i < NQ; ++i) {
          double v = 0.0;
          int tx, ty;
          if (!o->solid[m] && locate(o, x + CX[i], y + CY[i], &tx, &ty)) {
            size_t t = at(o, tx, ty);
            v = o->solid[t] ? pbar[(size_t)reverse_of(i) * N + m] : pbar[(size_t)i * N + t];
          }
          Fbar[(size_t)i * N + m] = v;
        }
      }
    /* collision */
    const double *un = uh + (size_t)(n - 1) * N;
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        size_t m = at(o, x, y);
        if (o->solid[m]) {
          for (int i = 0; i < NQ; ++i) gbar[(size_t)i * N + m] = 0.0;
          continue;
        }
        const int rx = reactive(o, x, y);
        double kr = rx ? o->k[m] : 0.0;
        double s = 0.0, wf = 0.0;
        for (int i = 0; i < NQ; ++i) {
          double Fb = Fbar[(size_t)i * N + m];
          double wP = feq(i, 1.0, o->vel[m], o->vel[N + m]); /* w_i P_i */
          s += (omega * wP - WT[i] * kr) * Fb;
          wf += WT[i] * Fb;
        }
        if (n - 1 >= 1 && x == o->nx - 1) s += 1.0;
        for (int j = 0; j < NQ; ++j)
          gbar[(size_t)j * N + m] = (1.0 - omega) * Fbar[(size_t)j * N + m] + s;
        if (grad_k && rx) grad_k[m] -= un[m] * wf;
      }
  }
  free(uh); free(root); free(gbar); free(pbar); free(Fbar);
  return 0;
}

/* ---- snapshots for the Schwarz rollback ------------------------------------
 * Every Schwarz iteration of a coarse step restarts the fine solver from its
 * state at t_n (Algorithm 1 repeats the substeps of one coarse step).  A
 * snapshot is a deep copy of the evolving state: populations, concentration,
 * mask, mineral and the counters. */
or_lbm *or_lbm_clone(const or_lbm *o) {
  or_lbm *c = or_lbm_new(o->nx, o->ny, o->edge, o->tau, o->react_mode, o->k_scalar,
                         o->k, o->dissolution, o->solid, o->vel, o->mineral, NULL);
  if (!c) return NULL;
  c->wall_mode = o->wall_mode;
  size_t N = nn(o);
  memcpy(c->f, o->f, NQ * N * sizeof(double));
  memcpy(c->u, o->u, N * sizeof(double));
  memcpy(c->flip_step, o->flip_step, N * sizeof(int));
  c->steps = o->steps; c->bc_infeasible = o->bc_infeasible; c->flips = o->flips;
  c->newton_iters = o->newton_iters; c->newton_fail = o->newton_fail;
  c->J = o->J; c->reacted = o->reacted;
  return c;
}

/* Overwrite the evolving state of dst (same lattice) with that of src. */
void or_lbm_assign(or_lbm *dst, const or_lbm *src) {
  size_t N = nn(src);
  memcpy(dst->f, src->f, NQ * N * sizeof(double));
  memcpy(dst->u, src->u, N * sizeof(double));
  memcpy(dst->solid, src->solid, N);
  memcpy(dst->mineral, src->mineral, N * sizeof(double));
  memcpy(dst->flip_step, src->flip_step, N * sizeof(int));
  memcpy(dst->k, src->k, N * sizeof(double));
  dst->steps = src->steps; dst->bc_infeasible = src->bc_infeasible; dst->flips = src->flips;
  dst->newton_iters = src->newton_iters; dst->newton_fail = src->newton_fail;
  dst->J = src->J; dst->reacted = src->reacted;
}
