/*
 * sgml.h -- C ABI of libsgml, a GB300 (sm_103a) implementation of the single-grid multi-level
 * (SGML) method of Becerra-Sagredo, Mandujano and Malaga, "A GPU-based Multi-level Algorithm for
 * Boundary Value Problems" (arXiv 1703.07206).
 *
 * The library solves, for a batch of independent problems on the unit square (dim = 2) or cube
 * (dim = 3) with N = 2^n + 1 nodes per side,
 *
 *     L u = f,   L = div(sigma grad) + a                                  (Sec. 2 Eq. 1, Sec. 3)
 *
 * discretised with the radial 9-point (2-D) / 27-point (3-D) stencil of Eq. 5, by repeating the
 * saw-like single cycle of Algorithm 3 (restriction, Algorithm 1 / Eqs. 3-4, and relaxation-
 * interpolation, Algorithm 2) on the residual of the accumulated solution (Sec. 2, last
 * paragraphs) until ||f - delta L u||_inf / ||f||_inf <= tol (Sec. 3.1).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an int status (sgml_status); no exception crosses the ABI.  On failure
 *     sgml_last_error() returns a message for the calling thread.
 *   - Node arrays hold N^dim doubles, row-major [z][y][x] with x fastest, boundary nodes included;
 *     node i sits at x_i = i / (N - 1).
 *   - Array pointers may be host or device pointers (unified addressing decides); the library
 *     copies from / to them and never keeps them.  The grid owns all of its device memory.
 *   - Work is issued on the CUDA stream given to sgml_create_grid.  Calls documented as
 *     synchronising wait for that stream; the others are stream-ordered and return at once.
 *   - Faces are ordered -x, +x, -y, +y, -z, +z (the last two ignored in 2-D).
 */
#ifndef SGML_H
#define SGML_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgml_grid* sgml_grid_t;

typedef enum {
  SGML_OK = 0,
  SGML_ERR_ARG = -1,             /* invalid argument; nothing was changed */
  SGML_ERR_CUDA = -2,            /* a CUDA call failed; the grid should be destroyed */
  SGML_ERR_NOT_CONVERGED = -3,   /* solve_to_tol: max_cycles cycles did not reach the tolerance */
  SGML_ERR_DIVERGED = -4,        /* the residual grew for several cycles above its start value */
  SGML_ERR_BARRIER_TIMEOUT = -5, /* a grid-wide barrier of the cycle kernel gave up waiting */
  SGML_ERR_NONFINITE = -6        /* a residual norm was NaN or infinite */
} sgml_status;

enum { SGML_FP64 = 0, SGML_MIXED = 1 };        /* cycle precision; the outer step is always FP64 */
enum { SGML_DIRICHLET = 0, SGML_NEUMANN = 1 }; /* face types */
enum { SGML_NORM_MAX = 0, SGML_NORM_L2 = 1 };
enum { SGML_STENCIL_CONSISTENT = 0, SGML_STENCIL_LITERAL = 1 };

/* Create a batch of `batch` problems of dimension `dim` (2 or 3); problem b has
 * N_b = 2^n_levels[b] + 1 nodes per side (1 <= n_levels[b] <= 12 in 2-D, <= 10 in 3-D).
 * `precision`: SGML_FP64 runs the whole cycle in FP64; SGML_MIXED runs restriction, relaxation and
 * interpolation in FP32 on a scaled residual, keeping the outer residual and the solution sum in FP64.
 * `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  Initially every face is
 * Dirichlet 0, sigma = 1, a = 0 and f = 0; parameters are those of sgml_set_params' defaults.
 * Allocates device memory; *out receives the handle. */
int sgml_create_grid(int dim, int batch, const int* n_levels, int precision, void* cuda_stream,
                     sgml_grid_t* out);

/* Method parameters (Algorithm 3, Sec. 2): n_r = maximum relaxation-interpolations per visit
 * (default 2, as in Fig. 3); theta in (0, 1] = fraction of the maximum stable pseudo-time step
 * (default 0.7; the step at a node is theta * (kappa_d S_d / 2) / D_i with D_i minus the diagonal of
 * delta L there, equal to theta (2^nu h)^2 / (2 sigma) for constant sigma, the bound of Sec. 2 and
 * Sec. 3.4); schedule must be 0 (the zig-zag reading of Algorithm 3); stencil selects the constant
 * of Eq. 5 (SGML_STENCIL_CONSISTENT: exact on quadratics; SGML_STENCIL_LITERAL: the printed
 * 3/(13h) and its 2-D analogue); dt_mode must be 0 (Jacobi-scaled local step); max_cycles bounds
 * sgml_solve_to_tol (default 200).  Stream-ordered. */
int sgml_set_params(sgml_grid_t g, int n_r, double theta, int schedule, int stencil, int dt_mode,
                    int max_cycles);

/* Coefficients of L = div(sigma grad) + a for one problem (problem >= 0) or for all (problem = -1,
 * arrays concatenated problem after problem).  sigma: N^dim positive node values, or NULL for
 * sigma = 1.  a: N^dim node values (<= 0), or NULL for the constant a_scalar (<= 1; the pseudo-time
 * step needs D_i > 0).  a < 0 everywhere makes an all-Neumann problem well posed as given; an
 * all-Neumann problem with a constant a >= 0 is solved in the form of Eq. 10 (Sec. 3.2):
 * L u = f - <f> with zero normal derivatives, for the u of zero mean (<.>: trapezoid-rule mean over
 * the unit square / cube), the constant mode projected out of u after every cycle and the residual
 * recomputed in FP64 every cycle.  Copies the arrays; the coefficient pyramid is rebuilt before the
 * next cycle. */
int sgml_set_coeffs(sgml_grid_t g, int problem, const double* sigma, const double* a, double a_scalar);

/* Source f of L u = f (the paper's sign: a problem -Lap u = q passes f = -q).  N^dim values for one
 * problem, or all problems concatenated when problem = -1.  Values on Dirichlet nodes are ignored.
 * Copies the array and resets the solution (the next cycle starts from the lifted boundary values). */
int sgml_set_source(sgml_grid_t g, int problem, const double* f);

/* Boundary conditions of one problem (or all, problem = -1): face_type[2*dim] of SGML_DIRICHLET /
 * SGML_NEUMANN and face_value[2*dim] (NULL = 0): the Dirichlet value of the face, or the prescribed
 * outward normal derivative of a Neumann face (Sec. 2, boundary conditions).  A node on a Dirichlet
 * face is fixed (Dirichlet wins where faces of both kinds meet; the first Dirichlet face in face
 * order gives the value).  Neumann faces use even images (-k -> k) with u_image = u_mirror + 2 k h g.
 * All faces Neumann with a constant a >= 0: Eq. 10 (see sgml_set_coeffs); every g must then be 0
 * (else SGML_ERR_ARG at the next solve).  Resets the solution. */
int sgml_set_bc(sgml_grid_t g, int problem, const int* face_type, const double* face_value);

/* Run exactly ncycles cycles of Algorithm 3 for every problem from the current solution (the
 * lifted boundary values after create/set_*), each followed by the FP64 outer step u += e,
 * r = f - delta L u.  One persistent cooperative kernel launch.  Stream-ordered (asynchronous). */
int sgml_run_cycle(sgml_grid_t g, int ncycles);

/* Solve every problem from its lifted boundary values: repeat cycles until
 * ||r||_inf / ||f||_inf <= rtol (Sec. 3.1; when f vanishes on the unknowns the initial residual is
 * the scale) or max_cycles cycles.  One persistent cooperative kernel launch; synchronises.
 * cycles_out[batch] and rel_res_out[batch] (either may be NULL) receive per problem the cycles run
 * and the final relative residual.  Returns SGML_OK when every problem converged,
 * SGML_ERR_NOT_CONVERGED / SGML_ERR_DIVERGED / SGML_ERR_NONFINITE otherwise (worst status). */
int sgml_solve_to_tol(sgml_grid_t g, double rtol, int* cycles_out, double* rel_res_out);

/* Relative residual of the current solution for every problem: ||f - delta L u|| / ||f|| over the
 * unknowns in the max norm (SGML_NORM_MAX) or the Euclidean norm (SGML_NORM_L2).  rel_out[batch].
 * Synchronises. */
int sgml_residual_norm(sgml_grid_t g, int norm, double* rel_out);

/* Copy the FP64 solution of one problem (N^dim values) into u.  Synchronises. */
int sgml_get_solution(sgml_grid_t g, int problem, double* u);

/* Per-problem statistics of the last run: cycles run (cumulative since the last reset), final
 * relative residual (max norm), and the status (sgml_status) of the problem.  Synchronises. */
int sgml_get_stats(sgml_grid_t g, int problem, int* cycles, double* rel_max, int* status);

/* Relative max-norm residual before each cycle of the last sgml_solve_to_tol / sgml_run_cycle call
 * and after its last cycle (cycles + 1 values, at most cap).  Synchronises.  Returns the count
 * written through *count. */
int sgml_get_history(sgml_grid_t g, int problem, double* hist, int cap, int* count);

/* r = f - delta L_0 u for one problem, with u given (N^dim values; the grid's own solution is not
 * touched), the grid's source, coefficients and boundary conditions (Neumann images carry the
 * prescribed derivative); r = 0 on fixed nodes.  FP64.  Device arrays of the grid's device are used in
 * place; host arrays pass through a staging buffer the grid allocates once and keeps.  r must not
 * alias u.  Synchronises. */
int sgml_residual(sgml_grid_t g, int problem, const double* u, double* r);

/* Adjoint gradient of J(u) with respect to sigma for one all-Dirichlet problem: given the forward
 * solution u and the adjoint lambda (the solution of delta L^T lambda = dJ/du on the unknowns,
 * lambda = 0 on fixed nodes; delta L is symmetric there), writes
 * dJ/dsigma_m = kappa/(2h^2) sum_{o, m+o inside} w_o (lambda_{m+o} - lambda_m)(u_{m+o} - u_m)
 * (the derivative of Eq. 5's link coefficient (sigma_i + sigma_j)/2).  dJ/df = lambda.  FP64.
 * Device arrays of the grid's device are used in place, host arrays are staged as for sgml_residual.
 * Returns SGML_ERR_ARG for a problem with a Neumann face, or if grad aliases lambda or u.
 * Synchronises. */
int sgml_sigma_gradient(sgml_grid_t g, int problem, const double* lambda, const double* u, double* grad);

/* Launch shape and work partition of the cycle kernel (256 threads per CTA).
 *   ctas_per_sm: CTAs per SM (0 = as many as fit; the cooperative launch needs all CTAs resident, so
 *     the library clamps to the occupancy limit).
 *   z_waves (>= 1): with the contiguous cut, each level's tile-planes are cut into G * z_waves equal
 *     runs (G = CTAs), run j going to CTA j mod G (1: one contiguous share per CTA).
 *   mode 0 (default): every run_cycle / solve_to_tol / residual_norm call is one persistent
 *     cooperative launch with grid-wide barriers between phases.  mode 1: the same device code with
 *     one ordinary launch per phase (for profiling single phases; run_cycle then needs no host
 *     synchronisation and can be captured in a CUDA graph).
 *   tile_x: the column tiles of the tiled phases, 32 (32 x 16 columns) or 64 (64 x 8, the default).
 *   slab_z (default 32 for SGML_MIXED, 0 for SGML_FP64): 3-D levels large enough to give every CTA two slabs of work are cut into
 *     z-slabs of about slab_z planes; the (slab, tile) pieces are dealt to the CTAs in turn, so that
 *     neighbouring tiles are processed at the same time and their shared halo cells are read from
 *     HBM once.  0: contiguous runs on every level.
 * Used by the autotuner.  Results do not depend on these settings (bit for bit). */
int sgml_set_launch(sgml_grid_t g, int ctas_per_sm, int z_waves, int mode, int tile_x, int slab_z);

/* Bounded grid barriers of the persistent cycle kernel (Sec. 2 runs every level inside one cycle;
 * here one launch holds all of them, with grid-wide barriers between phases).  wait_limit_s (default
 * 2.0, range 1e-4 .. 60) is the longest any CTA waits at one barrier before it records a timeout and
 * the launch returns SGML_ERR_BARRIER_TIMEOUT (sync calls) -- a wait never spins forever.
 * withhold_barrier >= 1 is a test aid: in every following launch CTA 0 withholds its arrival at
 * that barrier (1-based count within the launch), so that all waits run out and the timeout path is
 * exercised without any fault; 0 (the default) turns it off.  The grid stays usable: the next launch
 * starts from cleared barrier words.  Host only; takes effect at the next launch. */
int sgml_set_barrier_test(sgml_grid_t g, double wait_limit_s, int withhold_barrier);

/* Fused sweep pairs (3-D, SGML_MIXED): on levels 0 .. pair_levels - 1 (default 0: off) the
 * k relaxation sweeps of a visit (Algorithm 2, Eq. 2) run two at a time in one pass over the level:
 * the first sweep is evaluated on each tile widened by one cell and kept on chip, the second reads
 * it there, so the level's arrays cross HBM once per pair instead of once per sweep.  The result is
 * the same Jacobi iteration (rounding differs from the unfused form only in the order of the
 * neighbour sums).  0 turns fusion off; ignored for 2-D grids and the FP64 form.  Takes effect at
 * the next cycle. */
int sgml_set_fusion(sgml_grid_t g, int pair_levels);

/* Four-row sweeps (3-D, SGML_MIXED): on levels 0 .. quad_levels - 1 (default 0: off) the
 * relaxation sweeps run on tiles of 64 x 16 (or 32 x 32) columns with four nodes per thread,
 * instead of 64 x 8 (32 x 16) with two: fewer shared-memory loads and less pipeline overhead per
 * node.  The same Jacobi sweep (Eq. 2 with Eq. 5); only the rounding order of the neighbour sums
 * differs.  0 turns it off; ignored for 2-D grids and the FP64 form.  Takes effect at the next
 * cycle. */
int sgml_set_quad(sgml_grid_t g, int quad_levels);

/* Coarse tail (3-D, SGML_MIXED, a grid of one problem with n >= 4; on by default).  The phases of
 * a cycle that touch only the three coarsest levels (9^3, 5^3 and 3^3 nodes: the restriction
 * passes into them and the visits of the teeth nu1 = n - 1, n - 2 and the start of n - 3 of
 * Algorithm 3) run in one CTA with all their arrays in shared memory, instead of as grid phases
 * that each end in a grid barrier.  The same operations in the same order: results are
 * bit-identical either way.  on: 1 (default) or 0.  Ignored for batches, 2-D grids, the FP64 form,
 * the one-launch-per-phase mode and while diagnostics are recorded.  Takes effect at the next
 * launch. */
int sgml_set_coarse_tail(sgml_grid_t g, int on);

/* The cycle's phase table as the library runs it (Algorithm 3's schedule: restriction passes, then
 * the visits with their interpolation / injection steps).  Writes 4 ints per phase to out
 * (op: 0 restrict, 1 sweep, 2 interpolate to the finer level, 3 inject to the coarser level; the
 * level it writes; the index of its first sweep within the visit; the sweeps it performs (1 or 2,
 * 0 for the other ops)) for at most cap phases, and the phase count to *count.  Host only. */
int sgml_get_phases(sgml_grid_t g, int* out, int cap, int* count);

/* Per-phase tracing of the persistent cycle kernel (a profiling aid): with cycles > 0, CTA 0
 * stamps the GPU global timer after every grid barrier of the first `cycles` cycles of each
 * launch; 0 turns it off.  Allocates a small device buffer; synchronises. */
int sgml_set_trace(sgml_grid_t g, int cycles);

/* Durations in microseconds of the traced cycles of the last launch, row-major [cycle][slot] with
 * *nphases slots per cycle: slot 0 is unused (0), slot 1 the residual phase (anchor or recurrence),
 * slot 2 the convergence check, slots 3 .. the phases of the cycle's schedule in order.  Each span
 * includes the grid barrier that ends it.  cap bounds the doubles written.  Synchronises. */
int sgml_get_trace(sgml_grid_t g, double* us, int cap, int* nphases, int* ncycles);

/* Diagnostic pseudo-residual (Sec. 3.1: "the coarsened residual computed while applying the
 * relaxation at every level with restricted sources and coefficients"): with cycles > 0 the next
 * launches record, for each problem, each of the first `cycles` cycles of the launch and each level
 * l, the largest |delta L_l e - r_l| met by that level's sweeps (|e_new - e| / delta tau at a node),
 * in the units of the residual f - delta L u.  At level 0 it is the residual of the correction
 * equation itself.  Costs, while on, a reciprocal and a maximum per node and sweep and a warp
 * reduction per tile (about +40 % solve time on a 129^3 problem); fused pairs and four-row tiles
 * are not used meanwhile.  0 turns it off.  Synchronises. */
int sgml_set_diagnostics(sgml_grid_t g, int cycles);

/* The recorded pseudo-residuals of problem `problem` from the last launch: out[c * 13 + l] for
 * cycle c and level l (0 for levels the problem does not have or cycles not run); at most cap
 * doubles; *cycles_out = rows written.  Synchronises. */
int sgml_get_diagnostics(sgml_grid_t g, int problem, double* out, int cap, int* cycles_out);

/* Launch geometry of the cycle kernel for the grid's current settings: CTAs (all co-resident:
 * SMs x CTAs per SM from the occupancy calculator), threads per CTA, dynamic shared memory per CTA
 * in bytes.  Builds the work tables if needed (synchronises). */
int sgml_get_launch_info(sgml_grid_t g, int* ctas, int* threads_per_cta, int* smem_bytes);

/* Number of kernel launches the library issued on this grid since creation (every kernel,
 * setup included). */
int sgml_launch_count(sgml_grid_t g, long long* count);

/* ---- Post-processing of the vortex application (Sec. 3.3) -------------------------------------
 * Velocity from the stream vector potential, v = curl psi (Eq. 14), on the unit cube with
 * N = 2^n + 1 nodes per side (1 <= n <= 10).  psi and v: device arrays of 3 N^3 doubles, the x, y
 * and z components one after the other, each row-major [z][y][x]; caller-owned, must not alias.
 * The paper leaves the differences to its visualisation tool; read here as second-order central
 * differences inside and second-order one-sided differences (-3 f0 + 4 f1 - f2) / (2h) on the
 * faces.  Asynchronous on cuda_stream.  SGML_ERR_ARG for a bad n, NULL, aliasing or host arrays. */
int sgml_curl(int n, const double* psi, double* v, void* cuda_stream);

/* Streamlines of a node velocity field (Sec. 3.3: "a RK-marching scheme"): the classical
 * fourth-order Runge-Kutta method with fixed step dt, the velocity interpolated trilinearly between
 * the nodes of v (layout as for sgml_curl), from nseeds seed points (device array, x y z per seed)
 * for at most nsteps steps.  paths (device, nseeds x (nsteps + 1) x 3 doubles) receives the
 * positions, seed first; lengths (device, nseeds ints) the number written.  A path ends before a
 * stage point or its next position would leave the closed unit cube (length 0 for a seed outside
 * it).  One thread per seed; asynchronous on cuda_stream. */
int sgml_streamlines(int n, const double* v, const double* seeds, int nseeds, double dt, int nsteps, double* paths,
                     int* lengths, void* cuda_stream);

/* ---- Grid motion of the grid-deformation application (Sec. 3.2, Eq. 11) ----------------------
 * Moves points (normally the grid's nodes) by forward Euler in a pseudo-time t along
 * dx/dt = v = -grad u / (t f + int f dOmega), u the force potential of Eq. 10 (zero normal
 * derivative on every face; e.g. a solution of an all-Neumann grid) and f its source, both
 * N^dim node arrays (N = 2^n + 1; 2-D: 1 <= n <= 14, 3-D: 1 <= n <= 10) on the unit square /
 * cube, row-major ([y][x] or [z][y][x]), device memory.  The paper gives only the formula and
 * "finite differences of the potential"; read here as:
 *   - grad u at the nodes by central differences with the Neumann images u(-1) = u(1),
 *     u(N) = u(N-2) (zero normal component on the faces: face nodes slide along their faces);
 *   - grad u and f at a point by multilinear interpolation in the grid cell holding it;
 *   - int f dOmega by the trapezoid rule (V = 1);
 *   - nsteps equal steps from t0 to t1 (the paper's deformation runs t from 0 to 1), every
 *     coordinate clamped to [0, 1] before the first step and after each step.
 * x (device, in/out): dim x N^dim doubles, x[a * N^dim + node] the a-th coordinate (a = 0: x) of
 * the point that starts at node `node`; initialise it to the node coordinates for the paper's grid
 * deformation.  x must not alias u or f.  Synchronises cuda_stream (reads back int f and min f).
 * SGML_ERR_ARG for a bad dim or n, NULL, aliasing or host arrays, t0 < 0, t1 < t0, nsteps < 0, or
 * a denominator that could reach zero (int f <= 0 or int f + t1 min f <= 0; a non-negative source
 * such as the paper's delta function along a curve always passes). */
int sgml_grid_motion(int dim, int n, const double* u, const double* f, double t0, double t1, int nsteps, double* x,
                     void* cuda_stream);

/* ---- Measurement aid ----------------------------------------------------------------------------
 * Arithmetic throughput of the current GPU, the denominator of the FP64 form's roofline (the FP64
 * form runs Sec. 2's pseudo-time iteration entirely in FP64; on a narrow FP64 pipe that pipe, not
 * HBM, bounds it).  The paper has no counterpart.  Runs a kernel of independent FMA chains on every
 * SM (a warm-up launch, then three timed with CUDA events on cuda_stream) in FP64 and in FP32 and
 * writes thread-level FMA instructions per second to *fp64_fma_per_s and *fp32_fma_per_s.  Allocates
 * and frees a small device buffer; synchronises.  SGML_ERR_ARG for NULL outputs. */
int sgml_measure_fma_rates(void* cuda_stream, double* fp64_fma_per_s, double* fp32_fma_per_s);

/* Message of the last failed sgml_curl / sgml_streamlines / sgml_grid_motion call on this thread. */
const char* sgml_post_last_error(void);

int sgml_destroy(sgml_grid_t g);
const char* sgml_last_error(void);

/* One complete solve that allocates no memory, for callers that cannot allocate device memory where
 * they want to solve: frameworks whose memory pool owns the device and forbids allocations made
 * behind its back, hosts whose device-memory budget is fixed at start-up, and control loops that
 * cannot take the synchronisation of cudaMalloc / cudaFree.  The paper has no counterpart; this
 * packages the same cycle kernel as sgml_solve_to_tol.
 *
 * Solves L u = f (L = div(sigma grad) + a_scalar, paper's sign) for ONE problem of dimension dim with
 * N = 2^n + 1 nodes per side from the lifted boundary values until ||r||_inf / ||f||_inf <= rtol or
 * max_cycles cycles, with the default method parameters (n_r = 2, theta = 0.7, consistent stencil).
 * f (N^dim doubles), sigma (N^dim doubles or NULL for 1) and u (N^dim doubles, written) are DEVICE
 * pointers of the current device owned by the caller (anything else -- host memory, another GPU's
 * memory -- is refused with SGML_ERR_ARG); face_type / face_value (2*dim entries, face_value may be
 * NULL) are host arrays as in sgml_set_bc; a_scalar <= 0 (all-Neumann problems need a_scalar < 0
 * here: the mean projection of all-Neumann problems is a grid-API feature).  cycles_out / rel_out
 * (host, may be NULL) receive the cycles run and the final relative residual.  Work runs on
 * cuda_stream; the call synchronises it and copies its small status back to the host.
 *
 * All intermediate data lives in one file-scope device array of 24 MiB that every GPU loading the
 * library holds until the process exits; problems needing more (e.g. beyond 65^3 in 3-D or 513^2
 * in 2-D) are rejected with SGML_ERR_ARG before any GPU work.  No cudaMalloc, cudaFree or other
 * allocating routine is called.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current.  Every call shares the array and clears
 * what must start at zero; calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller.  Returns SGML_OK on convergence, else an
 * sgml_status; the message is in sgml_noalloc_last_error(). */
int sgml_solve_noalloc(int dim, int n, int precision, const double* f, const double* sigma, double a_scalar,
                       const int* face_type, const double* face_value, double rtol, int max_cycles, double* u,
                       int* cycles_out, double* rel_out, void* cuda_stream);
const char* sgml_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGML_H */
