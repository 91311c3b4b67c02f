/*
 * sgml_oracle.c -- plain, slow FP64 CPU oracle of the single-grid multi-level (SGML) method of
 * Becerra-Sagredo, Mandujano and Malaga, "A GPU-based Multi-level Algorithm for Boundary Value
 * Problems" (arXiv 1703.07206).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference against which the CUDA library is checked.
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA path, and the CUDA path never calls it.
 *
 * Everything lives on ONE grid, exactly as the paper describes (Sec. 2): every field is a full
 * array of N^d doubles (N = 2^n + 1 per dimension, row-major [z][y][x], x fastest), and the level-nu
 * subset is the set of nodes whose indices are all multiples of 2^nu.  Level-nu work reads and writes
 * that subset in place.  No blocking, fusion or compact per-level storage is used: the loops follow
 * the paper's routines in the paper's order so that they can be checked against it by eye.
 *
 * Readings of the paper where it is silent or garbled (each also listed in the design notes):
 *   - Algorithm 1 runs its passes m = 0 .. nu-1 (restriction(0) is the identity), evaluated at the
 *     level-(m+1) nodes only; values there are those of the every-node evaluation.
 *   - Algorithm 3 line 3 is read as the zig-zag "visit nu1, then nu1-1", followed by lines 6-8's
 *     second visit to nu1; a level below 0 is skipped.
 *   - The stencil of Eq. 5 is normalised with kappa_d = 2 / sum_o w_o o_1^2 so that it is exact on
 *     quadratics ("consistent"); the printed 3/(13h) (and the 2-D analogue 1/(2h)) is kept as the
 *     "literal" option.
 *   - The pseudo-time step is theta * (kappa_d S_d / 2) / D_i, D_i the diagonal of delta L at the
 *     node (Jacobi-scaled); for constant sigma and a = 0 this is theta * H^2 / (2 sigma), the bound
 *     of Sec. 2 and Sec. 3.4 times theta.  The node-local form theta * H^2 / (2 sigma_i) of Sec. 3.4
 *     is kept as an option.
 *   - The interpolation of Algorithm 2 is applied to the whole change of a visit once its sweeps
 *     end (the variation of the last sweep is not dropped).
 *   - Dirichlet values are lifted into u before the first cycle; every cycle is homogeneous.
 *   - Images: indices that leave [0, N-1] are reflected (-k -> k, N-1+k -> N-1-k).  On a Neumann
 *     face the image of u carries the prescribed outward derivative g: u_ghost = u_mirror + 2 k h g.
 *     Coefficients (sigma, a) are reflected on every face.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Loops over nodes run on several host threads when the oracle is built with OpenMP: each node's
 * value is computed by the same arithmetic whichever thread computes it, and the only reduction
 * shared between threads is a maximum, so results do not depend on the thread count.  The two
 * order-dependent sums (the trapezoid mean and integral) stay serial. */
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
#define ORC_PARALLEL_FOR ORC_PRAGMA(omp parallel for schedule(static))
#else
#define ORC_PARALLEL_FOR
#endif

/* Host threads used by the parallel loops (1 without OpenMP); n < 1 keeps the current count. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

#define ORC_DIRICHLET 0
#define ORC_NEUMANN 1

/* Problem description.  The Python wrapper mirrors this layout with ctypes. */
typedef struct {
  int dim;               /* 2 or 3 */
  int n;                 /* N = 2^n + 1 nodes per dimension */
  int face_type[6];      /* -x,+x,-y,+y,-z,+z : ORC_DIRICHLET or ORC_NEUMANN */
  double face_value[6];  /* Dirichlet value, or outward normal derivative g on a Neumann face */
  const double* sigma;   /* N^d node values of sigma, or NULL for sigma = 1 */
  const double* a;       /* N^d node values of a, or NULL for a = a_scalar everywhere */
  double a_scalar;
  int n_r;               /* maximum relaxation-interpolations per visit (Algorithm 3) */
  double theta;          /* fraction of the maximum stable pseudo-time step */
  int stencil;           /* 0 consistent kappa_d, 1 literal Eq. 5 constant */
  int dt_mode;           /* 0 Jacobi-scaled step, 1 node-local sigma step (Sec. 3.4) */
} orc_problem;

/* ------------------------------------------------------------------------------------------ */
/* Grid helpers                                                                                 */
/* ------------------------------------------------------------------------------------------ */

static int npts(const orc_problem* p) { return (1 << p->n) + 1; }

static long nnodes(const orc_problem* p) {
  long N = npts(p);
  return p->dim == 3 ? N * N * N : N * N;
}

static long at(const orc_problem* p, const int c[3]) {
  long N = npts(p);
  return ((long)c[2] * N + c[1]) * N + c[0];
}

static double grid_h(const orc_problem* p) { return 1.0 / (double)(npts(p) - 1); }

static void coords(const orc_problem* p, long idx, int c[3]) {
  long N = npts(p);
  c[0] = (int)(idx % N);
  c[1] = (int)((idx / N) % N);
  c[2] = p->dim == 3 ? (int)(idx / (N * N)) : 0;
}

/* A node on a Dirichlet face is fixed; every other node is an unknown (Dirichlet wins at a corner
 * shared with a Neumann face). */
static int is_dirichlet(const orc_problem* p, const int c[3]) {
  int N = npts(p);
  for (int k = 0; k < p->dim; ++k) {
    if (c[k] == 0 && p->face_type[2 * k] == ORC_DIRICHLET) return 1;
    if (c[k] == N - 1 && p->face_type[2 * k + 1] == ORC_DIRICHLET) return 1;
  }
  return 0;
}

static int on_level(const int c[3], int dim, int nu) {
  int s = 1 << nu;
  for (int k = 0; k < dim; ++k)
    if (c[k] % s != 0) return 0;
  return 1;
}

/* Even image of an index outside [0, N-1]; *out_by gets how many fine nodes it lay outside and
 * *face the face it crossed (-1 if inside). */
static int reflect(int i, int N, int k, int* out_by, int* face) {
  *out_by = 0;
  *face = -1;
  if (i < 0) {
    *out_by = -i;
    *face = 2 * k;
    return -i;
  }
  if (i > N - 1) {
    *out_by = i - (N - 1);
    *face = 2 * k + 1;
    return 2 * (N - 1) - i;
  }
  return i;
}

/* Offsets o in {-1,0,1}^d \ {0}: the 8 (2-D) or 26 (3-D) neighbours of the radial stencil. */
static int offsets(int dim, int o[26][3]) {
  int m = 0;
  for (int z = (dim == 3 ? -1 : 0); z <= (dim == 3 ? 1 : 0); ++z)
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        if (x == 0 && y == 0 && z == 0) continue;
        o[m][0] = x;
        o[m][1] = y;
        o[m][2] = z;
        ++m;
      }
  return m;
}

/* Eq. 5: the radial difference to a neighbour at distance h*l is divided by l, with l = 1, sqrt(2),
 * sqrt(3) for face, edge and corner neighbours: w_o = 1 / l_o = 1 / sqrt(#non-zero components). */
static double weight(const int o[3]) {
  int nz = (o[0] != 0) + (o[1] != 0) + (o[2] != 0);
  return 1.0 / sqrt((double)nz);
}

/* Constant in front of Eq. 5.  Consistent: kappa_d = 2 / sum_o w_o o_1^2, which makes the stencil
 * exact on quadratics.  Literal: 3/13 in 3-D as printed, and the same construction in 2-D (the
 * perimeter/area ratio 4/h of the disc of radius h/2 spread over 8 directions) gives 1/2. */
static double kappa(const orc_problem* p) {
  if (p->stencil == 1) return p->dim == 3 ? 3.0 / 13.0 : 0.5;
  int o[26][3];
  int m = offsets(p->dim, o);
  double s = 0.0;
  for (int q = 0; q < m; ++q) s += weight(o[q]) * (double)(o[q][0] * o[q][0]);
  return 2.0 / s;
}

/* kappa_d S_d / 2 with the consistent kappa_d and S_d = sum_o w_o: the product delta_tau * D_i of
 * the Jacobi-scaled step for theta = 1 (sqrt(2) in 2-D). */
static double jacobi_gain(const orc_problem* p) {
  int o[26][3];
  int m = offsets(p->dim, o);
  double s = 0.0, s1 = 0.0;
  for (int q = 0; q < m; ++q) {
    s += weight(o[q]);
    s1 += weight(o[q]) * (double)(o[q][0] * o[q][0]);
  }
  return (2.0 / s1) * s / 2.0;
}

/* ------------------------------------------------------------------------------------------ */
/* Radial finite-difference operator delta L at level nu (Eq. 5, Sec. 3 L = div(sigma grad) + a) */
/* ------------------------------------------------------------------------------------------ */

/* (delta L_nu u) at the level-nu unknown c.  sig and a hold the level-nu (restricted) coefficients
 * at level-nu nodes (NULL: 1 and a_scalar).  Neighbours are level-nu nodes at distance 2^nu h.
 * With with_flux set, a Neumann image carries the prescribed outward derivative (used for the
 * outer residual only; inside a cycle the images are homogeneous). */
static double op_at(const orc_problem* p, int nu, const double* sig, const double* a, const double* u,
                    const int c[3], int with_flux) {
  int N = npts(p);
  int s = 1 << nu;
  double H = s * grid_h(p);
  int o[26][3];
  int m = offsets(p->dim, o);
  long ic = at(p, c);
  double sc = sig ? sig[ic] : 1.0;
  double uc = u[ic];
  double sum = 0.0;
  for (int q = 0; q < m; ++q) {
    int nb[3] = {0, 0, 0};
    double ghost = 0.0;
    for (int k = 0; k < p->dim; ++k) {
      int by, face;
      nb[k] = reflect(c[k] + s * o[q][k], N, k, &by, &face);
      if (face >= 0 && with_flux && p->face_type[face] == ORC_NEUMANN)
        ghost += 2.0 * (double)by * grid_h(p) * p->face_value[face];
    }
    long in = at(p, nb);
    double sn = sig ? sig[in] : 1.0;
    double un = u[in] + ghost;
    sum += weight(o[q]) * 0.5 * (sc + sn) * (un - uc);
  }
  double ac = a ? a[ic] : p->a_scalar;
  return kappa(p) / (H * H) * sum + ac * uc;
}

/* delta L_nu applied at every level-nu unknown; 0 at every other node. */
void orc_apply_op(const orc_problem* p, int nu, const double* sig, const double* a, const double* u,
                  int with_flux, double* out) {
  long M = nnodes(p);
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    out[i] = (on_level(c, p->dim, nu) && !is_dirichlet(p, c)) ? op_at(p, nu, sig, a, u, c, with_flux) : 0.0;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Restriction (Algorithm 1, Eqs. 3-4)                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Hat function of Sec. 2: 1 at 0, 1/2 at +-1/2, support [-1, 1]. */
static double hat(double x) {
  double t = 1.0 - fabs(x);
  return t > 0.0 ? t : 0.0;
}

/* One pass of Algorithm 1 with lambda = 2^m: at every level-(m+1) node,
 * out = 2^-d sum_{p in {-1,0,1}^d} prod_k hat(-p_k/2) in(i + lambda p)   (Eq. 3 in 2-D, Eq. 4 in 3-D).
 * Indices leaving the domain take the even image. */
static void restrict_pass(const orc_problem* p, int m, const double* in, double* out) {
  int N = npts(p);
  int lam = 1 << m;
  long M = nnodes(p);
  double norm = p->dim == 3 ? 1.0 / 8.0 : 1.0 / 4.0;
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    if (!on_level(c, p->dim, m + 1)) continue;
    double acc = 0.0;
    for (int pz = (p->dim == 3 ? -1 : 0); pz <= (p->dim == 3 ? 1 : 0); ++pz)
      for (int py = -1; py <= 1; ++py)
        for (int px = -1; px <= 1; ++px) {
          int pp[3] = {px, py, pz};
          int nb[3] = {0, 0, 0};
          double w = 1.0;
          for (int k = 0; k < p->dim; ++k) {
            int by, face;
            nb[k] = reflect(c[k] + lam * pp[k], N, k, &by, &face);
            w *= hat(-0.5 * pp[k]);
          }
          acc += w * in[at(p, nb)];
        }
    out[i] = norm * acc;
  }
}

/* restriction(nu) of Algorithm 1: g = f, then passes m = 0 .. nu-1.  The result is valid at the
 * level-nu nodes of g (other entries are left as scratch). */
void orc_restriction(const orc_problem* p, int nu, const double* f, double* g) {
  long M = nnodes(p);
  memcpy(g, f, sizeof(double) * M);
  if (nu == 0) return;
  double* t = (double*)malloc(sizeof(double) * M);
  for (int m = 0; m < nu; ++m) {
    memcpy(t, g, sizeof(double) * M);
    restrict_pass(p, m, t, g);
  }
  free(t);
}

/* ------------------------------------------------------------------------------------------ */
/* Pseudo-time step (Sec. 2 stability bound, Sec. 3.4 local step)                              */
/* ------------------------------------------------------------------------------------------ */

/* D_i = kappa/H^2 sum_o w_o (sigma_i + sigma_o)/2 - a_i: minus the diagonal of delta L_nu. */
static double diag_at(const orc_problem* p, int nu, const double* sig, const double* a, const int c[3]) {
  int N = npts(p);
  int s = 1 << nu;
  double H = s * grid_h(p);
  int o[26][3];
  int m = offsets(p->dim, o);
  long ic = at(p, c);
  double sc = sig ? sig[ic] : 1.0;
  double sum = 0.0;
  for (int q = 0; q < m; ++q) {
    int nb[3] = {0, 0, 0};
    for (int k = 0; k < p->dim; ++k) {
      int by, face;
      nb[k] = reflect(c[k] + s * o[q][k], N, k, &by, &face);
    }
    double sn = sig ? sig[at(p, nb)] : 1.0;
    sum += weight(o[q]) * 0.5 * (sc + sn);
  }
  double ac = a ? a[ic] : p->a_scalar;
  return kappa(p) / (H * H) * sum - ac;
}

static double step_at(const orc_problem* p, int nu, const double* sig, const double* a, const int c[3]) {
  if (p->dt_mode == 1) {
    double H = (1 << nu) * grid_h(p);
    double sc = sig ? sig[at(p, c)] : 1.0;
    return p->theta * H * H / (2.0 * sc);
  }
  return p->theta * jacobi_gain(p) / diag_at(p, nu, sig, a, c);
}

/* Local pseudo-time step at every level-nu unknown (0 elsewhere). */
void orc_local_step(const orc_problem* p, int nu, const double* sig, const double* a, double* out) {
  long M = nnodes(p);
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    out[i] = (on_level(c, p->dim, nu) && !is_dirichlet(p, c)) ? step_at(p, nu, sig, a, c) : 0.0;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Interpolation I_lambda (Sec. 2, Algorithm 2 line 6)                                          */
/* ------------------------------------------------------------------------------------------ */

/* For every node x NOT in the level-nu subset: e_x += sum over the corners c of x's level-nu cell of
 * prod_k hat((x_k - c_k) / 2^nu) * delta_c, with delta given at level-nu nodes. */
void orc_interpolate_add(const orc_problem* p, int nu, const double* delta, double* e) {
  int N = npts(p);
  int s = 1 << nu;
  long M = nnodes(p);
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int x[3];
    coords(p, i, x);
    if (on_level(x, p->dim, nu)) continue;
    int lo[3] = {0, 0, 0};
    for (int k = 0; k < p->dim; ++k) lo[k] = (x[k] / s) * s;
    double acc = 0.0;
    for (int cz = 0; cz <= (p->dim == 3 ? 1 : 0); ++cz)
      for (int cy = 0; cy <= 1; ++cy)
        for (int cx = 0; cx <= 1; ++cx) {
          int cc[3] = {lo[0] + cx * s, lo[1] + cy * s, lo[2] + cz * s};
          double w = 1.0;
          int inside = 1;
          for (int k = 0; k < p->dim; ++k) {
            if (cc[k] > N - 1) inside = 0;
            w *= hat((double)(x[k] - cc[k]) / (double)s);
          }
          if (inside && w != 0.0) acc += w * delta[at(p, cc)];
        }
    e[i] += acc;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Relaxation-interpolation visit (Algorithm 2) and the single cycle (Algorithm 3)               */
/* ------------------------------------------------------------------------------------------ */

/* One visit of level nu: k forward-Euler (Jacobi) steps of Eq. 2 on the level-nu unknowns with the
 * restricted source r_nu and coefficients, then the change of the visit is interpolated to every
 * node outside the level-nu subset.  e holds the level-nu values in place on the single grid.
 * If diag is given, diag[nu] is raised to the largest |delta L_nu e - r_nu| met by the sweeps: the
 * diagnostic pseudo-residual of Sec. 3.1 ("the coarsened residual computed while applying the
 * relaxation at every level with restricted sources and coefficients"). */
void orc_visit(const orc_problem* p, int nu, int k, const double* r_nu, const double* sig_nu,
               const double* a_nu, double* e, double* diag) {
  long M = nnodes(p);
  double* saved = (double*)malloc(sizeof(double) * M);
  double* next = (double*)malloc(sizeof(double) * M);
  memcpy(saved, e, sizeof(double) * M);
  for (int sweep = 0; sweep < k; ++sweep) {
    memcpy(next, e, sizeof(double) * M);
    double dmax = diag ? diag[nu] : 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : dmax)
#endif
    for (long i = 0; i < M; ++i) {
      int c[3];
      coords(p, i, c);
      if (!on_level(c, p->dim, nu) || is_dirichlet(p, c)) continue;
      double dtau = step_at(p, nu, sig_nu, a_nu, c);
      double pseudo = op_at(p, nu, sig_nu, a_nu, e, c, 0) - r_nu[i];
      next[i] = e[i] + dtau * pseudo;
      if (fabs(pseudo) > dmax) dmax = fabs(pseudo);
    }
    if (diag) diag[nu] = dmax;
    memcpy(e, next, sizeof(double) * M);
  }
  if (nu > 0) {
    ORC_PARALLEL_FOR
    for (long i = 0; i < M; ++i) {
      int c[3];
      coords(p, i, c);
      next[i] = on_level(c, p->dim, nu) ? e[i] - saved[i] : 0.0;
    }
    orc_interpolate_add(p, nu, next, e);
  }
  free(saved);
  free(next);
}

static int min_int(int a, int b) { return a < b ? a : b; }

/* Number of relaxation-interpolations of a visit in tooth nu1 (Algorithm 3 lines 5, 8, 10). */
static int sweeps_for(const orc_problem* p, int nu1_exp) {
  long full = 1L << (nu1_exp > 30 ? 30 : nu1_exp);
  return (long)p->n_r < full ? p->n_r : (int)full;
}

/* One visit of Algorithm 3: restriction(nu) of the cycle's source and of the coefficients
 * (lines 4, 7), then k relaxation-interpolations (lines 5, 8, 10). */
static void restrict_and_visit(const orc_problem* p, int nu, int k, const double* r, double* e,
                               double* r_nu, double* sig_nu, double* a_nu, double* diag) {
  orc_restriction(p, nu, r, r_nu);
  if (p->sigma) orc_restriction(p, nu, p->sigma, sig_nu);
  if (p->a) orc_restriction(p, nu, p->a, a_nu);
  orc_visit(p, nu, k, r_nu, p->sigma ? sig_nu : NULL, p->a ? a_nu : NULL, e, diag);
}

/* The single cycle (Algorithm 3) solving delta L e = r from e = 0.  Teeth nu1 = n-1 .. 0 each visit
 * nu1, nu1-1 (skipped when negative) and nu1 again with min(n_r, 2^(n-nu1)) sweeps per visit; the
 * cycle ends with min(n_r, 2^n) sweeps on level 0. */
static void cycle_impl(const orc_problem* p, const double* r, double* e, double* diag) {
  long M = nnodes(p);
  double* r_nu = (double*)malloc(sizeof(double) * M);
  double* sig_nu = (double*)malloc(sizeof(double) * M);
  double* a_nu = (double*)malloc(sizeof(double) * M);
  memset(e, 0, sizeof(double) * M);
  for (int nu1 = p->n - 1; nu1 >= 0; --nu1) {
    int k = sweeps_for(p, p->n - nu1);
    for (int nu = nu1; nu >= nu1 - 1; --nu) {
      if (nu < 0) continue;
      restrict_and_visit(p, nu, k, r, e, r_nu, sig_nu, a_nu, diag);
    }
    restrict_and_visit(p, nu1, k, r, e, r_nu, sig_nu, a_nu, diag);
  }
  restrict_and_visit(p, 0, sweeps_for(p, p->n), r, e, r_nu, sig_nu, a_nu, diag);
  free(r_nu);
  free(sig_nu);
  free(a_nu);
}

void orc_cycle(const orc_problem* p, const double* r, double* e) { cycle_impl(p, r, e, NULL); }

/* The cycle, also returning diag[nu] (nu = 0 .. n-1): the largest diagnostic pseudo-residual
 * |delta L_nu e - r_nu| over the sweeps of level nu in this cycle. */
void orc_cycle_diag(const orc_problem* p, const double* r, double* e, double* diag) {
  for (int nu = 0; nu < p->n; ++nu) diag[nu] = 0.0;
  cycle_impl(p, r, e, diag);
}

/* Visit sequence of one cycle (levels, in order); returns the count.  Used to check the schedule. */
int orc_schedule(const orc_problem* p, int* levels, int* sweeps, int cap) {
  int m = 0;
  for (int nu1 = p->n - 1; nu1 >= 0; --nu1) {
    int k = sweeps_for(p, p->n - nu1);
    for (int nu = nu1; nu >= nu1 - 1; --nu) {
      if (nu < 0) continue;
      if (m < cap) { levels[m] = nu; sweeps[m] = k; }
      ++m;
    }
    if (m < cap) { levels[m] = nu1; sweeps[m] = k; }
    ++m;
  }
  if (m < cap) { levels[m] = 0; sweeps[m] = sweeps_for(p, p->n); }
  ++m;
  return m;
}

/* ------------------------------------------------------------------------------------------ */
/* Outer recurrence on accumulated residuals (Sec. 2, last paragraphs; Sec. 3.1 residual norm)   */
/* ------------------------------------------------------------------------------------------ */

/* Dirichlet value of a fixed node: the first Dirichlet face (order -x,+x,-y,+y,-z,+z) holding it. */
static double dirichlet_value(const orc_problem* p, const int c[3]) {
  int N = npts(p);
  for (int k = 0; k < p->dim; ++k) {
    if (c[k] == 0 && p->face_type[2 * k] == ORC_DIRICHLET) return p->face_value[2 * k];
    if (c[k] == N - 1 && p->face_type[2 * k + 1] == ORC_DIRICHLET) return p->face_value[2 * k + 1];
  }
  return 0.0;
}

/* u = Dirichlet values on fixed nodes, 0 on unknowns. */
void orc_lift(const orc_problem* p, double* u) {
  long M = nnodes(p);
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    u[i] = is_dirichlet(p, c) ? dirichlet_value(p, c) : 0.0;
  }
}

/* r = f - delta L_0 u at unknowns (Neumann images carry the prescribed derivative), 0 at fixed
 * nodes. */
void orc_residual(const orc_problem* p, const double* u, const double* f, double* r) {
  long M = nnodes(p);
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    r[i] = is_dirichlet(p, c) ? 0.0 : f[i] - op_at(p, 0, p->sigma, p->a, u, c, 1);
  }
}

/* r = f - delta L_0 u at the listed nodes only (flat indices), 0 at fixed nodes: the residual of
 * Sec. 2 evaluated one node at a time, for checks on grids too large for a full pass. */
void orc_residual_at(const orc_problem* p, const double* u, const double* f, const long* idx, long count, double* r) {
  ORC_PARALLEL_FOR
  for (long q = 0; q < count; ++q) {
    int c[3];
    coords(p, idx[q], c);
    r[q] = is_dirichlet(p, c) ? 0.0 : f[idx[q]] - op_at(p, 0, p->sigma, p->a, u, c, 1);
  }
}

/* Maximum norm over the unknowns. */
double orc_max_norm(const orc_problem* p, const double* v) {
  long M = nnodes(p);
  double m = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : m)
#endif
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    if (!is_dirichlet(p, c) && fabs(v[i]) > m) m = fabs(v[i]);
  }
  return m;
}

/* Repeat the cycle on the residual of the accumulated solution until ||r||_inf / ||f||_inf <= tol
 * (Sec. 3.1; when f vanishes on the unknowns the initial residual is the scale).  The residual is
 * recomputed from u each time (equal to the recurrence r_i = r_{i-1} - delta L e_{i-1} in exact
 * arithmetic).  u is lifted first.  Returns the number of cycles run, or -1 if max_cycles cycles did
 * not reach tol.  hist (may be NULL) receives the relative residual before each cycle and after the
 * last (max_cycles + 1 entries). */
/* ------------------------------------------------------------------------------------------ */
/* Pure-Neumann problems (Sec. 3.2, Eq. 10): every face Neumann with zero normal derivative and    */
/* a >= 0 (a constant), where L u = f has no solution or an unstable constant mode.  The equation   */
/* solved is L u = f - <f> for the zero-mean u, <v> the mean over the unit square / cube by the     */
/* trapezoid rule (node weight 1/2 per coordinate on a face).  The constant mode is projected out   */
/* of u after every cycle: for a = 0 it is the operator's null space, for a > 0 the pseudo-time      */
/* iteration would let it grow.  (With a < 0 everywhere an all-Neumann problem is well posed and is */
/* solved as given.)                                                                                 */
/* ------------------------------------------------------------------------------------------ */
int orc_projects_mean(const orc_problem* p) {
  for (int k = 0; k < 2 * p->dim; ++k)
    if (p->face_type[k] != ORC_NEUMANN) return 0;
  return p->a == NULL && p->a_scalar >= 0.0;
}

double orc_mean(const orc_problem* p, const double* v) {
  int N = npts(p);
  long M = nnodes(p);
  double sw = 0.0, s = 0.0;
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    double w = 1.0;
    for (int k = 0; k < p->dim; ++k)
      if (c[k] == 0 || c[k] == N - 1) w *= 0.5;
    sw += w;
    s += w * v[i];
  }
  return s / sw;
}

void orc_project_mean(const orc_problem* p, double* v) {
  long M = nnodes(p);
  double m = orc_mean(p, v);
  for (long i = 0; i < M; ++i) v[i] -= m;
}

int orc_solve(const orc_problem* p, const double* f_in, double tol, int max_cycles, double* u, double* hist) {
  long M = nnodes(p);
  double* r = (double*)malloc(sizeof(double) * M);
  double* e = (double*)malloc(sizeof(double) * M);
  double* fp = (double*)malloc(sizeof(double) * M);
  const int project = orc_projects_mean(p);
  memcpy(fp, f_in, sizeof(double) * M);
  if (project) orc_project_mean(p, fp);
  const double* f = fp;
  orc_lift(p, u);
  double scale = orc_max_norm(p, f);
  int cycles = -1;
  for (int c = 0;; ++c) {
    orc_residual(p, u, f, r);
    double rn = orc_max_norm(p, r);
    if (c == 0 && scale == 0.0) scale = rn;
    double rel = scale > 0.0 ? rn / scale : 0.0;
    if (hist) hist[c] = rel;
    if (rel <= tol) {
      cycles = c;
      break;
    }
    if (c == max_cycles) break;
    orc_cycle(p, r, e);
    ORC_PARALLEL_FOR
    for (long i = 0; i < M; ++i) u[i] += e[i];
    if (project) orc_project_mean(p, u);
  }
  free(r);
  free(e);
  free(fp);
  return cycles;
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint gradient for J(u(sigma, f)) with delta L_0(sigma) u = f, all faces Dirichlet           */
/* ------------------------------------------------------------------------------------------ */

/* Given the forward solution u and the adjoint lambda (delta L_0^T lambda = dJ/du on the unknowns,
 * lambda = 0 on fixed nodes), dJ/dsigma_m = kappa/(2h^2) sum_{o: m+o inside} w_o
 * (lambda_{m+o} - lambda_m)(u_{m+o} - u_m): the derivative of Eq. 5's link coefficient
 * (sigma_i + sigma_j)/2 with respect to sigma_m, contracted with -lambda^T (d delta L/d sigma_m) u.
 * dJ/df = lambda. */
void orc_sigma_gradient(const orc_problem* p, const double* lambda, const double* u, double* g) {
  int N = npts(p);
  long M = nnodes(p);
  double h = grid_h(p);
  int o[26][3];
  int m = offsets(p->dim, o);
  double c0 = kappa(p) / (2.0 * h * h);
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3];
    coords(p, i, c);
    double acc = 0.0;
    for (int q = 0; q < m; ++q) {
      int nb[3] = {0, 0, 0};
      int inside = 1;
      for (int k = 0; k < p->dim; ++k) {
        nb[k] = c[k] + o[q][k];
        if (nb[k] < 0 || nb[k] > N - 1) inside = 0;
      }
      if (!inside) continue;
      long j = at(p, nb);
      acc += weight(o[q]) * (lambda[j] - lambda[i]) * (u[j] - u[i]);
    }
    g[i] = c0 * acc;
  }
}

/* ------------------------------------------------------------------------------------------------
 * Post-processing of Sec. 3.3: velocity v = curl psi (Eq. 14) of the stream vector potential, and
 * streamlines of v.  The paper leaves the discretisation to its visualisation tool; the readings
 * taken here: derivatives by second-order central differences at interior nodes and second-order
 * one-sided differences (-3 f0 + 4 f1 - f2) / (2h) on the faces; streamlines by the classical
 * fourth-order Runge-Kutta method with a fixed step in the velocity field interpolated trilinearly
 * between nodes, stopped when a stage point or the next position leaves the unit cube.
 * ---------------------------------------------------------------------------------------------- */

/* d f / d x_axis at node (i, j, k) of an N^3 array (axis 0: x, 1: y, 2: z). */
static double orc_deriv(const double* f, int N, double h, int i, int j, int k, int axis) {
  int idx[3] = {i, j, k};
  const int m = idx[axis];
  double a, b, c;
  int q[3] = {i, j, k};
#define ORC_AT(t) (q[axis] = (t), f[((long)q[2] * N + q[1]) * N + q[0]])
  if (m == 0) {
    a = ORC_AT(0), b = ORC_AT(1), c = ORC_AT(2);
    return (-3.0 * a + 4.0 * b - c) / (2.0 * h);
  }
  if (m == N - 1) {
    a = ORC_AT(N - 1), b = ORC_AT(N - 2), c = ORC_AT(N - 3);
    return (3.0 * a - 4.0 * b + c) / (2.0 * h);
  }
  a = ORC_AT(m + 1), b = ORC_AT(m - 1);
  return (a - b) / (2.0 * h);
#undef ORC_AT
}

/* psi, v: three components, each an N^3 array, stored one after the other (x, y, z). */
void orc_curl(int n, const double* psi, double* v) {
  const int N = (1 << n) + 1;
  const double h = 1.0 / (double)(N - 1);
  const long M = (long)N * N * N;
  const double* px = psi;
  const double* py = psi + M;
  const double* pz = psi + 2 * M;
  ORC_PARALLEL_FOR
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const long c = ((long)k * N + j) * N + i;
        v[c] = orc_deriv(pz, N, h, i, j, k, 1) - orc_deriv(py, N, h, i, j, k, 2);
        v[M + c] = orc_deriv(px, N, h, i, j, k, 2) - orc_deriv(pz, N, h, i, j, k, 0);
        v[2 * M + c] = orc_deriv(py, N, h, i, j, k, 0) - orc_deriv(px, N, h, i, j, k, 1);
      }
}

/* Trilinear interpolation of the three components of v at x (inside the closed unit cube). */
static void orc_interp_v(const double* v, int N, const double x[3], double out[3]) {
  const long M = (long)N * N * N;
  const double s = (double)(N - 1);
  int i0[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    double g = x[a] * s;
    int i = (int)floor(g);
    if (i < 0) i = 0;
    if (i > N - 2) i = N - 2;
    i0[a] = i;
    t[a] = g - (double)i;
  }
  for (int comp = 0; comp < 3; ++comp) {
    const double* f = v + comp * M;
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dz ? t[2] : 1.0 - t[2]);
          acc += w * f[((long)(i0[2] + dz) * N + (i0[1] + dy)) * N + (i0[0] + dx)];
        }
    out[comp] = acc;
  }
}

static int orc_inside(const double x[3]) {
  for (int a = 0; a < 3; ++a)
    if (!(x[a] >= 0.0 && x[a] <= 1.0)) return 0;
  return 1;
}

/* RK4 streamlines from nseeds seed points (x, y, z each), nsteps steps of size dt.  paths holds
 * nseeds x (nsteps + 1) x 3 positions (unused entries untouched); lengths[s] = positions written
 * (1 + completed steps). */
void orc_streamlines(int n, const double* v, const double* seeds, int nseeds, double dt, int nsteps, double* paths,
                     int* lengths) {
  const int N = (1 << n) + 1;
  ORC_PARALLEL_FOR
  for (int sd = 0; sd < nseeds; ++sd) {
    double x[3] = {seeds[3 * sd], seeds[3 * sd + 1], seeds[3 * sd + 2]};
    double* out = paths + (long)sd * (nsteps + 1) * 3;
    int len = 0;
    if (orc_inside(x)) {
      out[0] = x[0], out[1] = x[1], out[2] = x[2];
      len = 1;
      for (int st = 0; st < nsteps; ++st) {
        double k1[3], k2[3], k3[3], k4[3], y[3], xn[3];
        orc_interp_v(v, N, x, k1);
        for (int a = 0; a < 3; ++a) y[a] = x[a] + 0.5 * dt * k1[a];
        if (!orc_inside(y)) break;
        orc_interp_v(v, N, y, k2);
        for (int a = 0; a < 3; ++a) y[a] = x[a] + 0.5 * dt * k2[a];
        if (!orc_inside(y)) break;
        orc_interp_v(v, N, y, k3);
        for (int a = 0; a < 3; ++a) y[a] = x[a] + dt * k3[a];
        if (!orc_inside(y)) break;
        orc_interp_v(v, N, y, k4);
        for (int a = 0; a < 3; ++a) xn[a] = x[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        if (!orc_inside(xn)) break;
        for (int a = 0; a < 3; ++a) x[a] = xn[a], out[3 * len + a] = xn[a];
        ++len;
      }
    }
    lengths[sd] = len;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Grid motion of Sec. 3.2: the nodes of the grid are advanced by forward Euler in a pseudo-time t */
/* along dx/dt = v with v = -grad u / (t f + int f dOmega) (Eq. 11), u the force potential of      */
/* Eq. 10 (zero normal derivative on every face) and f its source.  Readings (the paper gives only */
/* the formula and "finite differences of the potential"):                                        */
/*   - grad u at the nodes by central differences with the Neumann images u(-1) = u(1),            */
/*     u(N) = u(N-2), so its normal component is zero on the faces;                               */
/*   - grad u and f at a moving node by multilinear interpolation of their node values in the     */
/*     cell that holds it (cells clamped to the grid);                                            */
/*   - int f dOmega by the trapezoid rule on the unit square / cube (V = 1);                       */
/*   - nsteps equal steps from t0 to t1 (the paper's deformation runs t from 0 to 1); every      */
/*     coordinate is clamped to [0, 1] before the first step and after each step.                 */
/* Positions: x[a * M + node], a = 0 .. dim-1 the coordinate, node row-major [z][y][x].            */
/* ------------------------------------------------------------------------------------------ */
static long orc_node_index(int dim, int N, const int c[3]) {
  long i = 0;
  for (int a = dim - 1; a >= 0; --a) i = i * N + c[a];
  return i;
}

double orc_trapezoid(int dim, int n, const double* f) {
  const int N = (1 << n) + 1;
  const double h = 1.0 / (double)(N - 1);
  long M = 1;
  for (int a = 0; a < dim; ++a) M *= N;
  double s = 0.0;
  for (long i = 0; i < M; ++i) {
    long r = i;
    double w = 1.0;
    for (int a = 0; a < dim; ++a) {
      const int c = (int)(r % N);
      r /= N;
      w *= (c == 0 || c == N - 1) ? 0.5 * h : h;
    }
    s += w * f[i];
  }
  return s;
}

/* grad u at every node: g[a * M + node] = (u(c + e_a) - u(c - e_a)) / (2h), Neumann images. */
void orc_neumann_gradient(int dim, int n, const double* u, double* g) {
  const int N = (1 << n) + 1;
  const double h = 1.0 / (double)(N - 1);
  long M = 1;
  for (int a = 0; a < dim; ++a) M *= N;
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    int c[3] = {0, 0, 0};
    long r = i;
    for (int a = 0; a < dim; ++a) c[a] = (int)(r % N), r /= N;
    for (int a = 0; a < dim; ++a) {
      int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
      cp[a] = c[a] + 1 > N - 1 ? N - 2 : c[a] + 1;
      cm[a] = c[a] - 1 < 0 ? 1 : c[a] - 1;
      g[a * M + i] = (u[orc_node_index(dim, N, cp)] - u[orc_node_index(dim, N, cm)]) / (2.0 * h);
    }
  }
}

/* Multilinear interpolation of the node field v (N^dim values) at the point x. */
static double orc_interp_nodes(int dim, int N, const double* v, const double* x) {
  int i0[3] = {0, 0, 0};
  double t[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < dim; ++a) {
    const double gx = x[a] * (double)(N - 1);
    int i = (int)floor(gx);
    if (i < 0) i = 0;
    if (i > N - 2) i = N - 2;
    i0[a] = i;
    t[a] = gx - (double)i;
  }
  double acc = 0.0;
  for (int corner = 0; corner < (1 << dim); ++corner) {
    int c[3] = {0, 0, 0};
    double w = 1.0;
    for (int a = 0; a < dim; ++a) {
      const int up = (corner >> a) & 1;
      c[a] = i0[a] + up;
      w *= up ? t[a] : 1.0 - t[a];
    }
    acc += w * v[orc_node_index(dim, N, c)];
  }
  return acc;
}

void orc_grid_motion(int dim, int n, const double* u, const double* f, double t0, double t1, int nsteps, double* x) {
  const int N = (1 << n) + 1;
  long M = 1;
  for (int a = 0; a < dim; ++a) M *= N;
  double* g = (double*)malloc(sizeof(double) * dim * M);
  orc_neumann_gradient(dim, n, u, g);
  const double F = orc_trapezoid(dim, n, f);
  const double dt = nsteps > 0 ? (t1 - t0) / (double)nsteps : 0.0;
  ORC_PARALLEL_FOR
  for (long i = 0; i < M; ++i) {
    double p[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; ++a) p[a] = x[a * M + i] < 0.0 ? 0.0 : (x[a * M + i] > 1.0 ? 1.0 : x[a * M + i]);
    for (int k = 0; k < nsteps; ++k) {
      const double t = t0 + (double)k * dt;
      double v[3];
      const double den = t * orc_interp_nodes(dim, N, f, p) + F;
      for (int a = 0; a < dim; ++a) v[a] = -orc_interp_nodes(dim, N, g + a * M, p) / den;
      for (int a = 0; a < dim; ++a) {
        p[a] = p[a] + dt * v[a];
        if (p[a] < 0.0) p[a] = 0.0;
        if (p[a] > 1.0) p[a] = 1.0;
      }
    }
    for (int a = 0; a < dim; ++a) x[a * M + i] = p[a];
  }
  free(g);
}
