/*
 * hydro.h -- C ABI of the GB300 (sm_103a) Godunov cell-update library.
 *
 * The library advances the Euler equations with gravity, heating and passive
 * scalars (HERACLES++, arXiv:2503.04428, Sect. 2.1 Eq. 1) by one
 * MUSCL-Hancock time step per call (Sect. 3.2, Eq. 17-19): primitive recovery
 * through the ideal-gas EoS (Sect. 2.3 Eq. 5), limited reconstruction, the
 * Hancock half-step predictor, an HLL/HLLC/exact Riemann solve at every face,
 * the conservative update with Cartesian or spherical geometric sources
 * (Sect. 3.1.2, Eq. 13-16), gravity (Sect. 2.2, Eq. 2-4) and heating
 * (Sect. 2.4, Eq. 8-9), and the CFL time step.  All of it runs in the
 * library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point:
 *   - Every function returns a hydro_status (0 = HYDRO_OK, negative = error)
 *     unless stated otherwise; hydro_last_error() returns a thread-local text
 *     describing the last failure on the calling thread.
 *   - A hydro_t is opaque and owns all of its device memory: a double-buffered
 *     state and small scratch arrays.  It is not thread-safe: one host thread
 *     at a time per handle.
 *   - Caller pointers are borrowed for the duration of the call only.  Where
 *     an argument `where` is HYDRO_DEVICE the pointer is a device address in
 *     the current CUDA context (for example a torch tensor's data_ptr()); with
 *     HYDRO_HOST it is ordinary (ideally pinned) host memory.
 *   - All kernels and copies are issued on the CUDA stream given at creation
 *     (NULL = legacy default stream).  Calls that return data to the host
 *     synchronise that stream.
 *   - State layout: structure of arrays over interior cells, variable-major,
 *     U[v][k][j][i] with i fastest; v runs over (rho, rho u_1..rho u_dim, E,
 *     rho f_1..rho f_S).  In spherical coordinates axes (0,1,2) are
 *     (r, theta, phi) and velocities (u_r, u_theta, u_phi).  Elements are
 *     double for precision 64 and float for precision 32.
 */
#ifndef HYDRO_H
#define HYDRO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydro_ctx* hydro_t;

typedef enum {
  HYDRO_OK = 0,
  HYDRO_ERR_ARG = -1,             /* invalid argument (message says which) */
  HYDRO_ERR_CUDA = -2,            /* a CUDA runtime call failed */
  HYDRO_ERR_NEGATIVE_STATE = -3,  /* a cell reached rho <= 0 or P <= 0 */
  HYDRO_ERR_NONFINITE = -4,       /* NaN or Inf in the state */
  HYDRO_ERR_NEWTON = -5,          /* exact-solver Newton did not converge in 100 iterations */
  HYDRO_ERR_TIMEOUT = -6,         /* a bounded device wait expired (batched: a window copy never landed) */
  HYDRO_ERR_OOM = -7,             /* device allocation failed */
  HYDRO_ERR_VACUUM = -8,          /* exact solver: the data generate vacuum */
  HYDRO_ERR_UNSUPPORTED = -9      /* combination not built (see message) */
} hydro_status;

enum { HYDRO_PERIODIC = 0, HYDRO_TRANSMISSIVE = 1, HYDRO_REFLECTIVE = 2 };  /* Sect. 3.2 */
enum { HYDRO_CARTESIAN = 0, HYDRO_SPHERICAL = 1 };                          /* Sect. 3.1.1 */
enum { HYDRO_HLL = 0, HYDRO_HLLC = 1, HYDRO_EXACT = 2 };                    /* Sect. 3.2, App. C.1 */
enum { HYDRO_FIRST_ORDER = 0, HYDRO_MINMOD = 1, HYDRO_VANLEER = 2, HYDRO_VANALBADA = 3 }; /* Eq. 17 */
enum { HYDRO_GRAV_NONE = 0, HYDRO_GRAV_UNIFORM = 1, HYDRO_GRAV_POINT = 2,
       HYDRO_GRAV_POINT_MONOPOLE = 3 };                                     /* Eq. 2-4 */
enum { HYDRO_HEAT_NONE = 0, HYDRO_HEAT_CONST = 1, HYDRO_HEAT_NI56 = 2 };    /* Sect. 2.4 */
enum { HYDRO_HOST = 0, HYDRO_DEVICE = 1 };
enum { HYDRO_GUESS_TORO = 0, HYDRO_GUESS_MLP = 1 };

#define HYDRO_MAX_SCALARS 3
#define HYDRO_MLP_NPARAM 4673  /* 6->64->64->1: W1[64][6] b1[64] W2[64][64] b2[64] w3[64] b3 */

/* Grid (Sect. 3.1.1): logically Cartesian, 1-3 active axes.  faces[d] holds
 * the n[d]+1 increasing face coordinates of axis d (regular, logarithmic or
 * custom spacing; radians for angles); axes >= dim are ignored.  bc[d] gives
 * the (low, high) boundary kind.  Absent angular axes of a spherical grid
 * span the full sphere.  Every active axis needs n[d] >= 2. */
typedef struct {
  int dim;
  int n[3];
  const double* faces[3];
  int bc[3][2];
} hydro_grid;

/* Ideal-gas EoS (Eq. 5) with n_scalars passive scalars (Eq. 1d), 0..3. */
typedef struct {
  double gamma;
  int n_scalars;
} hydro_eos;

typedef struct {
  long long steps;         /* steps completed on this handle */
  long long faces;         /* Riemann problems solved (owned faces) */
  long long newton_iters;  /* exact solver: Newton iterations summed over faces; with the gas +
                            * radiation EoS: the temperature Newton iterations of every EoS call */
  long long fallbacks;     /* predicted face states replaced by the cell average */
  long long mlp_faces;     /* exact solver: faces whose guess came from the MLP */
  double t;                /* simulation time (grid handles) */
  double last_dt;
  int tile_x, tile_y, zchunk, threads;  /* launch shape chosen by the autotuner */
  double tuned_us_per_step;            /* autotuner's best measured step time */
  /* Batched exact solver, owned faces that ran Newton (not two identical
   * states) and their iterations, by category: [0] started from Toro's guess,
   * [1] from the network's guess, both in the handle's precision; [2] FP32
   * faces solved in FP64 (pressure ratio above 1e6 or within 20 % of the
   * vacuum limit), whatever their guess.  Zero for grid handles. */
  long long newton_faces[3];
  long long newton_iters_by[3];
} hydro_stats_t;

/* Create a grid solver.  precision: 64 (FP64 throughout) or 32 (FP32 bulk
 * arithmetic; FP64 CFL reduction, conserved totals and hard Newton solves).
 * riemann: HYDRO_HLL / HYDRO_HLLC / HYDRO_EXACT.  limiter: Eq. 17 options.
 * stream: a cudaStream_t (NULL allowed).  The state is zero until set. */
int hydro_create(const hydro_grid* grid, int coords, const hydro_eos* eos, int riemann,
                 int limiter, int precision, void* stream, hydro_t* out);

/* Equation of state: switch a grid handle from the ideal gas (Eq. 5) to an
 * ideal gas in equilibrium with radiation (Sect. 2.3, Eq. 6-7):
 *   e = rho R_gas T/(gamma-1) + a_rad T^4,   P = rho R_gas T + a_rad T^4/3,
 *   c^2 = (gamma/(gamma-1) + 20 alpha + 16 alpha^2)/(1/(gamma-1) + 12 alpha)
 *         * P_gas/rho,   alpha = P_rad/P_gas,
 * with R_gas = k_b/(mu m_u) the specific gas constant and a_rad the radiation
 * constant, both in the caller's units (R_gas > 0, a_rad >= 0; a_rad = 0 is
 * the ideal gas computed the same way).  The temperature of every EoS call is
 * found by Newton's method from the upper bound min(gas-only, radiation-only
 * temperature), to a relative step of 1e-13 (FP64) or 1e-6 (FP32) plus one
 * more step.  HLL and HLLC only: with the exact solver the call fails with
 * HYDRO_ERR_UNSUPPORTED.  Call before hydro_set_state. */
int hydro_set_eos_radiation(hydro_t h, double R_gas, double a_rad);

/* Internal-energy monitoring in highly supersonic regions (Sect. 2.5): with
 * eps > 0 every cell whose t^n internal energy e is below eps times its
 * kinetic energy density e_k takes e_new = e + alpha d1 + (1 - alpha) d2,
 * where d1 is the change of e implied by the total-energy update, d2 that of
 * de/dt + div(u e) + P div(u) = 0 integrated with the step's face fluxes
 * (u_f e_f = F_rho (e/rho)_upwind, u_f = F_rho/rho_upwind, upwind by the sign
 * of the mass flux; P the cell's t^n pressure; plus the heating), and alpha =
 * 1 for e >= eps e_k, (e/(eps e_k))^2 down to eps e_k/10, 0 below; the total
 * energy is then e_new + rho|u|^2/2.  Cells with alpha = 1 are untouched.
 * eps = 0 (the default) switches the correction off; the paper uses 1e-6. */
int hydro_set_dual_energy(hydro_t h, double eps);

/* Source terms.  gravity (Eq. 2-4): UNIFORM uses g0 (components along the
 * grid axes); POINT uses -G Mc / r^2 e_r; POINT_MONOPOLE adds the enclosed
 * mass M(r) of the current state (spherically symmetric approximation,
 * Eq. 4), both spherical only.  Sources enter as +rho g and +rho u.g with g
 * the acceleration.  heating (Sect. 2.4): CONST adds heat_params[0] per unit
 * volume and time; NI56 adds Eq. 8 in CGS units with heat_params[0] the index
 * of the scalar holding the Ni-56 mass fraction.  Evaluated at t^n. */
int hydro_set_sources(hydro_t h, int gravity, const double g0[3], double G, double Mc,
                      int heating, const double* heat_params);

/* Domain decomposition (Sect. 3.3.1: one subdomain per process, with ghost
 * layers exchanged between neighbours).  A grid handle may be one slab of a
 * larger grid: the sides of ONE axis can be marked as exchanged, and their
 * ghost cells are then the neighbouring slabs' cells, supplied by the caller
 * before every step, instead of a boundary condition.
 *
 * hydro_set_exchange: mark side `side` (0 low, 1 high) of `axis` as
 * exchanged; ghost_faces[0..1] are the two face coordinates beyond that side,
 * nearest first (the neighbour's cells' geometry, so that a slab gives
 * bit for bit the arithmetic of the whole grid).  Call before
 * hydro_set_state; sides of a second axis are rejected (HYDRO_ERR_ARG).
 * Halos, in the state's precision, are laid out [v][layer][cross section]:
 * layer l is the ghost at distance l+1 from the side, and the cross section
 * runs over the two other axes, the lower one fastest ((k, j) for axis 0,
 * (k, i) for axis 1, (j, i) for axis 2): nv * 2 * cross elements.
 * hydro_set_halo: the ghost layers of an exchanged side (host or device
 * memory, `where`), used by the following steps.
 * hydro_get_boundary: the state's two boundary layers at a side in the same
 * layout (layer l = the cell at distance l from the side) -- exactly the
 * halo the neighbour across that side needs.
 * hydro_shell_masses: m_i = sum_jk rho dV of every radial cell of the
 * current state (FP64, n[0] values, host), for monopole gravity (Eq. 4) on a
 * grid split along r; hydro_set_inner_mass: the mass of all shells inside
 * this slab (the sum of the inner slabs' m_i), where the enclosed-mass sum
 * M_i = Mc + (4 pi/Omega)(sum_{i'<i} m_i' + m_i/2) starts.
 * A step of a split grid is: exchange halos, (monopole) exchange shell
 * masses, take the minimum of every slab's hydro_cfl_dt, hydro_step.
 * hydro_run (device-side dt, graph) returns HYDRO_ERR_UNSUPPORTED on a grid
 * with exchanged sides.  Slabs are built for the ideal gas without the
 * dual-energy correction (HYDRO_ERR_UNSUPPORTED otherwise). */
int hydro_set_exchange(hydro_t h, int axis, int side, const double ghost_faces[2]);
int hydro_set_halo(hydro_t h, int axis, int side, const void* halo, int where);
int hydro_get_boundary(hydro_t h, int axis, int side, void* out, int where);
int hydro_shell_masses(hydro_t h, double* m_out);
int hydro_set_inner_mass(hydro_t h, double mass);

/* Moving grid (Sect. 3.1.1: the grid shifted along one axis during the run,
 * e.g. radially to follow expanding ejecta).  Every face of `axis` moves with
 * velocity w (code units), so each step of size dt shifts them by w dt; the
 * flux through a moving face is F - w U of the Riemann solution on the face's
 * path x/t = w (computed as the fixed-face flux of the states seen from the
 * frame moving with w); the Hancock predictor uses the same fluxes along that
 * axis; on a spherical grid (r only) the face areas of a step are their
 * averages over the step (a radial face r^2 + r D + D^2/3, D = w dt) and a
 * cell's content is spread over its new volume, so that a uniform gas at rest
 * stays uniform; the CFL speed is |u - w| + c along that axis.  Cartesian:
 * any axis, transmissive or periodic ends; spherical: r, transmissive ends.
 * Ideal gas, no dual-energy correction, no exchanged sides
 * (HYDRO_ERR_UNSUPPORTED / HYDRO_ERR_ARG).  hydro_run then drives its steps
 * from the host (each step's geometry follows its dt).  hydro_get_faces
 * copies the current n[axis]+1 face coordinates of an axis to host memory. */
int hydro_set_moving_grid(hydro_t h, int axis, double w);
int hydro_get_faces(hydro_t h, int axis, double* out);

/* Copy a state in (validated on the device: rho > 0, P > 0, finite; on
 * failure the previous state is kept) and compute its CFL signal speed. */
int hydro_set_state(hydro_t h, const void* U, int where);
int hydro_get_state(hydro_t h, void* U_out, int where);
int hydro_set_time(hydro_t h, double t);

/* dt = cfl / max_cells sum_d (|u_d| + c)/h_d for the current state (FP64). */
int hydro_cfl_dt(hydro_t h, double cfl, double* dt_out);

/* One time step of size dt (Eq. 19 plus sources).  Synchronises the stream
 * to read the device status; on error the state is left as before the call. */
int hydro_step(hydro_t h, double dt);

/* nsteps time steps with the time step computed on the device from the CFL
 * condition (dt = cfl/smax, clipped so that t does not pass t_end when
 * t_end > 0), without host round trips (captured as one CUDA graph after
 * the first call).  On error the state rolls back to the last good step.
 * *t_out (may be NULL) receives the time reached. */
int hydro_run(hydro_t h, int nsteps, double cfl, double t_end, double* t_out);

/* Conserved totals sum_cells U dV, FP64, deterministic order; out has nv entries. */
int hydro_totals(hydro_t h, double* out_nv);

/* Conserved totals accumulated inside the step (the FP32 form keeps its
 * bulk arithmetic in FP32 and its conservation sums in FP64).  With on != 0
 * every later step (hydro_step, hydro_run) also sums U dV of the cells it
 * updates: each CTA of the fused sweep in a fixed order over its cells,
 * into its own FP64 partial (the FP32 3D form sums each column of cells as
 * a compensated FP32 pair of exact products and converts the column's sum
 * to FP64; its totals equal the FP64 sums of the FP32 state to ~1e-14
 * relative);
 * hydro_step_totals then sums the partials in a fixed order, so the
 * totals of the new state cost no second pass over it and are deterministic.
 * The partials take nv x (the most CTAs of any launch shape) doubles, and a
 * step with totals uses 8 nv bytes more shared memory per updated cell of a
 * CTA.  Rejected on a moving grid (HYDRO_ERR_UNSUPPORTED). */
int hydro_set_step_totals(hydro_t h, int on);
/* The totals (nv doubles, host) of the current state from the last step's
 * partials; HYDRO_ERR_ARG if the totals are off, or no step has completed
 * since they were turned on or the state was set. */
int hydro_step_totals(hydro_t h, double* out_nv);
int hydro_stats(hydro_t h, hydro_stats_t* out);

/* Batched form: ntubes independent 1D tubes on [0,1] with lengths[b] uniform
 * cells each, transmissive ends, no scalars.  The state is (3 x sum lengths),
 * tubes concatenated per variable.  Every tube takes its own CFL time step. */
int hydro_batch_create(const int* lengths, int ntubes, const hydro_eos* eos, int riemann,
                       int limiter, int precision, void* stream, hydro_t* out);

/* nsteps steps of every tube in one persistent launch: a tube's step waits
 * only for the tube's own previous step (its CFL time step needs that
 * step's maximum over the tube), never for the other tubes, so there is no
 * grid-wide barrier between steps.  The launch is captured as a CUDA graph
 * once per (nsteps, cfl) and replayed.  The first call runs the launch-shape
 * autotuner on scratch copies of the state.  A failing step (invalid state,
 * Newton or a bounded device wait, HYDRO_ERR_TIMEOUT) stops the run: every
 * tube keeps the state of the last step it completed (the failing tube the
 * state before its failing step), so the tubes may then have completed
 * different numbers of steps (hydro_batch_times gives each tube's time; the
 * step count of hydro_stats counts the steps every tube completed). */
int hydro_batch_run(hydro_t h, int nsteps, double cfl);

/* The steps of hydro_batch_run, queued on the handle's stream (one launch)
 * without waiting for them (the first call still runs the autotuner,
 * synchronously).  A step that fails on the device stops its launch, and
 * later queued launches do nothing; the next hydro_batch_run reports the
 * failure and leaves every tube at its last good step as described there
 * (hydro_batch_run(h, 0, cfl) only waits and reports).  The
 * paper has no counterpart: this lets a caller overlap its own work with the
 * steps, or time a single step on the device without the host round trip
 * of the status check. */
int hydro_batch_enqueue(hydro_t h, int nsteps, double cfl);

/* Advance a batch whose state lives in host memory: U_in (3 x total cells,
 * the layout of hydro_batch_set_state) is copied in, every tube advances
 * nsteps of its own CFL steps, and the result is copied to U_out.  The tubes
 * are cut into nparts groups of about equal cell counts (0 = 8) whose input
 * copy, steps and output copy are ordered by events on three streams, so that
 * the copies of one group overlap the computation of the others; the overlap
 * needs U_in and U_out in pinned (page-locked) host memory.  The result equals
 * hydro_batch_set_state + hydro_batch_run + hydro_batch_get_state bit for bit
 * and the handle holds it afterwards.  An invalid input state or a failed
 * step returns its status, and U_out is then unspecified.  The paper has no
 * counterpart: this serves callers whose tubes live in host memory. */
int hydro_batch_run_host(hydro_t h, const void* U_in, void* U_out, int nsteps, double cfl, int nparts);

/* Record (with probability keep_prob, counter-based per face and step) the
 * left/right primitive states (rho,u,P)x2 of faces that pass the network's
 * gate (see hydro_mlp_set), during later hydro_batch_run calls; capacity
 * faces at most. */
int hydro_harvest_begin(hydro_t h, long capacity, double keep_prob, unsigned long long seed);
/* Copy up to cap harvested faces (6 doubles each) to host memory; *n = count. */
int hydro_harvest_get(hydro_t h, double* faces6, long cap, long* n);

/* MLP initial guess for the exact solver (6->64->64->1, SiLU, FP32 weights).
 * Inputs: ln(rho_L/rho_ref), ln(rho_R/rho_ref), ln(P_L/P_ref), ln(P_R/P_ref),
 * u_L/c_ref, u_R/c_ref with rho_ref, P_ref the geometric means of the two
 * sides and c_ref = sqrt(gamma P_ref/rho_ref).  Output y: the guess is
 * P_ref exp(y), i.e. the network predicts ln(p_star/P_ref).  It replaces
 * Toro's adaptive guess only on faces where that rule picks the two-shock
 * (TSRS) estimate and max(P_L,P_R) > 4 min(P_L,P_R) (PVRS serves nearby
 * states, the two-rarefaction estimate is exact when both waves are
 * rarefactions, the two-shock estimate is good for mild jumps).  Newton
 * still runs to convergence: to 1e-10 relative and one polishing step in
 * FP64; in FP32 to 1e-6 relative, the step that reaches it being the last
 * (its iterate is ~1e-12 from the root, below FP32 resolution).  weights:
 * HYDRO_MLP_NPARAM floats (host). */
int hydro_mlp_set(hydro_t h, const float* weights, int enable);
int hydro_mlp_get(hydro_t h, float* weights_out);

/* Train the handle's MLP on the GPU (own forward, backward and Adam
 * kernels): faces6 holds n samples (rho_L,u_L,P_L,rho_R,u_R,P_R), log_pstar
 * their ln(p_star); only samples on which the network would be used (the
 * gate described at hydro_mlp_set) are trained on; MSE on
 * ln(p_star/P_ref); minibatches of `batch`, Adam (beta 0.9/0.999) with a
 * learning rate decaying from lr to 0 on a cosine, shuffled by `seed`.  Host
 * arrays.  *loss_out (may be NULL) receives the last epoch's mean loss. */
int hydro_mlp_train(hydro_t h, const double* faces6, const double* log_pstar, long n, int epochs,
                    int batch, float lr, unsigned long long seed, double* loss_out);

/* GPU forward + backward of the MSE loss for given features x6 (n x 6) and
 * targets (n): gradient (HYDRO_MLP_NPARAM doubles) and loss.  Host arrays. */
int hydro_mlp_loss_grad(const float* weights, const double* x6, const double* target, long n,
                        double* grad_out, double* loss_out);

/* The same gradient as hydro_mlp_loss_grad, without allocating device memory.
 * The paper has no counterpart: this entry point serves callers that must
 * not allocate while they call in -- a host framework that owns all of the
 * GPU's memory through its own pool (an allocation behind its back can fail
 * or fragment that pool), or a code whose device-memory budget is fixed when
 * it starts.
 * Every pointer is a device address in the current context: weights
 * (HYDRO_MLP_NPARAM floats), x6 (n x 6 floats, the network inputs), target
 * (n floats), grad_out (HYDRO_MLP_NPARAM doubles), loss_out (1 double); work
 * is queued on `stream` (a cudaStream_t, NULL = legacy default) and the call
 * returns without synchronising.  The per-CTA partial gradients live in a
 * static device array of 4.79 MB that every GPU loading the library holds
 * until the process exits; hence 1 <= n <= HYDRO_NOALLOC_MAX_SAMPLES, larger n
 * is rejected with HYDRO_ERR_ARG.  The array is shared by all calls: nothing
 * in it has to start at zero, but calls that overlap on the GPU race on it.
 * The first call on a device, with that device current, looks the array's
 * address up and raises the gradient kernel's shared-memory limit (no
 * allocation); make that first call before any stream capture. */
#define HYDRO_NOALLOC_MAX_SAMPLES 16384
int hydro_mlp_loss_grad_device(const float* weights, const float* x6, const float* target, long n,
                               double* grad_out, double* loss_out, void* stream);

/* Exact Riemann star states on the GPU for n independent faces (host arrays
 * WL, WR of n x (rho,u,P)): p_star, u_star and Newton iterations per face.
 * precision 64 or 32; guess HYDRO_GUESS_TORO or HYDRO_GUESS_MLP (weights
 * required then).  Same Newton rule as the solver (App. C.1; Toro ch. 4). */
int hydro_exact_solve(const double* WL, const double* WR, long n, double gamma, int guess,
                      const float* weights, int precision, double* pstar, double* ustar,
                      int* iters);

/* Failure-detection check of the device waits: one thread waits, with the
 * bounded wait the batched kernel uses on its bulk copies, on an mbarrier
 * that nothing completes.  Returns HYDRO_ERR_TIMEOUT (the expected outcome:
 * the wait gave up and reported it, the context stays usable) and the time
 * the wait took in *seconds_out (may be null); HYDRO_OK would mean a wait
 * that cannot complete did. */
int hydro_wait_probe(double* seconds_out);

/* Measured arithmetic peak of the current GPU: dense fused multiply-adds in
 * FP64 (precision 64), FP32 (32) or paired FP32 (HYDRO_FMA_F32X2: one
 * instruction performs two FMAs on a float2), in TFLOP/s (2 flops per FMA), the best
 * of four ~20 ms launches of eight independent FMA chains per thread.  The
 * paper has no counterpart: the FP64 forms of the step are bound by this
 * rate rather than by HBM on this hardware, and their roofline needs it
 * measured on the machine at hand.  Synchronous; allocates a few bytes. */
#define HYDRO_FMA_F32X2 2  /* precision code of hydro_fma_rate: paired FP32 FMAs (f32x2) */
int hydro_fma_rate(int precision, double* tflops_out);

/* Sample the exact Riemann solution (Toro ch. 4; the reference solution of
 * the paper's shock-tube tests, App. C.1) in FP64 on the GPU: WL, WR hold nf
 * faces as (rho,u,P); point k belongs to face face_of[k] (0 <= face_of[k] <
 * nf) and sits at the similarity coordinate xi[k] = (x - x_face)/t; W_out
 * (npts x 3) receives (rho,u,P) there.  Star states come from the Toro guess
 * and the Newton rule of hydro_exact_solve; a face without one (vacuum)
 * fails with HYDRO_ERR_NEWTON.  Host arrays. */
int hydro_exact_sample(const double* WL, const double* WR, long nf, double gamma,
                       const long long* face_of, const double* xi, long npts, double* W_out);

/* Fix the batched launch shape instead of autotuning it: warps per CTA (4 or
 * 8), cells per work item (a positive multiple of 28, the kernel's segment;
 * items longer than every tube make one item per tube) and persistent CTAs
 * per SM (1 up to the kernel's occupancy).  HYDRO_ERR_ARG if out of range.
 * The paper has no counterpart: this serves tests and measurements of
 * particular shapes. */
int hydro_batch_set_launch(hydro_t h, int warps_per_cta, int item_cells, int ctas_per_sm);

/* Simulation time of every tube of a batch (ntubes doubles, host): the sum of
 * its own CFL steps dt_b = cfl / max_i (|u|+c)_i n_b since hydro_set_state. */
int hydro_batch_times(hydro_t h, double* t_out);

const char* hydro_last_error(void);
void hydro_destroy(hydro_t h);

#ifdef __cplusplus
}
#endif
#endif
