/*
 * hydro_oracle.h -- C interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library: the enum
 * values below are restated here (they are part of the public interface
 * contract, not shared code).
 *
 * Method (HERACLES++, arXiv:2503.04428):
 *   Euler equations with gravity, heating and passive scalars  -- Sect. 2.1, Eq. 1
 *   gravity: uniform / point mass / monopole                    -- Sect. 2.2, Eq. 2-4
 *   ideal-gas EoS; gas + radiation EoS                          -- Sect. 2.3, Eq. 5-7
 *   heating/cooling, Ni-56 decay chain                          -- Sect. 2.4, Eq. 8-9
 *   mesh, dS and dV per geometry                                -- Sect. 3.1.1
 *   spherical geometric momentum sources                        -- Sect. 3.1.2, Eq. 13-16
 *   MUSCL-Hancock: limited primitive reconstruction (Eq. 17),
 *   Hancock half-step predictor (Eq. 18), Godunov update (Eq. 19),
 *   HLL / HLLC Riemann solvers, three boundary conditions       -- Sect. 3.2
 *   exact Riemann solution (the "analytical" Sod comparison)    -- App. C.1
 *   Sedov self-similar shock radius                             -- Sect. 4.3, Eq. 25
 *
 * Every array is structure-of-arrays, interior cells only, variable-major:
 *   U[v][k][j][i], i fastest, v in (rho, m_1..m_dim, E, rho f_1..rho f_S).
 * All functions return 0 on success, a negative status on error.
 */
#ifndef HYDRO_ORACLE_H
#define HYDRO_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NEGATIVE_STATE = -3, ORC_ERR_NONFINITE = -4,
       ORC_ERR_NEWTON = -5, ORC_ERR_VACUUM = -8 };
enum { ORC_PERIODIC = 0, ORC_TRANSMISSIVE = 1, ORC_REFLECTIVE = 2 };
enum { ORC_CARTESIAN = 0, ORC_SPHERICAL = 1 };
enum { ORC_HLL = 0, ORC_HLLC = 1, ORC_EXACT = 2 };
enum { ORC_FIRST_ORDER = 0, ORC_MINMOD = 1, ORC_VANLEER = 2, ORC_VANALBADA = 3 };
enum { ORC_GRAV_NONE = 0, ORC_GRAV_UNIFORM = 1, ORC_GRAV_POINT = 2, ORC_GRAV_POINT_MONOPOLE = 3 };
enum { ORC_HEAT_NONE = 0, ORC_HEAT_CONST = 1, ORC_HEAT_NI56 = 2 };
enum { ORC_GUESS_TORO = 0, ORC_GUESS_MLP = 1 };

typedef struct orc_ctx* orc_t;

/* n[3]: cells per axis (inactive axes 1); faces: the n[d]+1 face coordinates of
 * every active axis, concatenated; bc[6]: (lo,hi) per axis. */
int  orc_create(int dim, const int* n, const double* faces, const int* bc, int coords,
                double gamma, int n_scalars, int riemann, int limiter, orc_t* out);
void orc_destroy(orc_t h);
int  orc_set_sources(orc_t h, int gravity, const double* g0, double G, double Mc,
                     int heating, const double* heat_params);
int  orc_set_guess(orc_t h, int guess, const float* mlp_weights);
/* Switch to the gas + radiation EoS of Sect. 2.3 Eq. 6-7 (R = k_b/(mu m_u),
 * a = radiation constant, both in the caller's units); HLL/HLLC only. */
int  orc_set_eos_radiation(orc_t h, double R, double a);
/* Dual-energy internal-energy correction of Sect. 2.5 with criterion eps
 * (0 = off; the paper typically uses 1e-6). */
int  orc_set_dual_energy(orc_t h, double eps);
int  orc_set_state(orc_t h, const double* U);
int  orc_get_state(orc_t h, double* U);
int  orc_set_time(orc_t h, double t);
int  orc_cfl_dt(orc_t h, double cfl, double* dt);
int  orc_step(orc_t h, double dt);
int  orc_totals(orc_t h, double* out);
/* out[0]=Riemann faces solved, [1]=Newton iterations, [2]=first-order fallbacks,
 * [3]=faces that used the MLP guess */
int  orc_stats(orc_t h, long long* out);
int  orc_shell_mass(orc_t h, double* M_out);   /* enclosed mass per radial cell (monopole) */

/* Domain decomposition (Sect. 3.3.1): the sides of one axis may be exchanged
 * with neighbouring subdomains.  set_exchange marks (axis, side) and gives
 * the 2 face coordinates beyond it, nearest first (the neighbour's cells'
 * geometry); set_halo gives its 2 ghost layers [nv][2][cross] (layer l = the
 * ghost at distance l+1; the cross section runs over the two other axes, the
 * lower one fastest); get_boundary returns the 2 boundary layers of the
 * state in the same layout (layer l = the cell at distance l from the side),
 * which is the neighbour's halo.  shell_masses: m_i = sum_jk rho dV per
 * radial cell; set_inner_mass: the mass of the shells inside this subdomain
 * (monopole of an r-split). */
int  orc_set_exchange(orc_t h, int axis, int side, const double* ghost_faces);
int  orc_set_halo(orc_t h, int axis, int side, const double* halo);
int  orc_get_boundary(orc_t h, int axis, int side, double* out);
int  orc_shell_masses(orc_t h, double* m_out);
int  orc_set_inner_mass(orc_t h, double mass);

/* Moving grid (Sect. 3.1.1): the faces of `axis` move with velocity w (each
 * step shifts them by w dt); fluxes through the moving faces are F - w U of
 * the Riemann solution on the face path x/t = w, the predictor uses the same
 * fluxes along that axis, face areas are averaged over the step and the
 * content of a cell is spread over its new volume.  Cartesian: any axis,
 * transmissive or periodic ends; spherical: r only, transmissive ends.
 * get_faces returns the current face coordinates of an axis (n+1). */
int  orc_set_moving_grid(orc_t h, int axis, double w);
int  orc_get_faces(orc_t h, int axis, double* out);

/* Batched 1D tubes on [0,1], transmissive ends, each advanced nsteps at its own
 * CFL time step.  U is (3 x total cells), tubes concatenated per variable. */
int  orc_batch_run(const int* lengths, int ntubes, double* U, double gamma, int riemann,
                   int limiter, double cfl, int nsteps, int guess, const float* mlp_weights,
                   int nthreads, long long* stats_out);

/* Point-wise pieces, exposed for the pins. */
double orc_limiter(int kind, double dm, double dp);
int  orc_flux_1d(int riemann, double gamma, int n_scalars, int dim, const double* UL,
                 const double* UR, double* F);
int  orc_exact_star(double gamma, const double* WL, const double* WR, int guess,
                    const float* mlp_weights, double* pstar, double* ustar, int* iters);
int  orc_exact_sample(double gamma, const double* WL, const double* WR, double xi, double* W);
double orc_guess_toro(double gamma, const double* WL, const double* WR, int* kind);
/* x6: network inputs; *pref: sqrt(P_L P_R) (the target is ln(p_star/pref)) */
int  orc_mlp_features(double gamma, const double* WL, const double* WR, double* x6, double* pref);
int  orc_mlp_forward(const float* w, const double* x6, long n, double* y);
double orc_mlp_loss_grad(const float* w, const double* x6, const double* t, long n, double* grad);
int  orc_adam_step(float* w, float* m, float* v, const double* grad, int nparam, int step,
                   double lr, double beta1, double beta2, double eps);
double orc_sedov_xi0(double gamma);
/* Gas + radiation EoS (Eq. 6-7) at one point: from (rho, e) the temperature,
 * pressure and sound speed; from (rho, P) the temperature and e. */
int  orc_eos_rad(double gamma, double R, double a, double rho, double e, double* T, double* P, double* c);
int  orc_eos_rad_eint(double gamma, double R, double a, double rho, double P, double* T, double* e);
double orc_heating_rate(int heating, const double* heat_params, double t, double rho_f_ni);

#ifdef __cplusplus
}
#endif
#endif
