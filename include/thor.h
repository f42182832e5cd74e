/*
 * libthor: C ABI of a GB300 (sm_103a) implementation of the THOR dynamical
 * core's hot path (Mendonca, Grimm, Grosheintz and Heng 2016, "THOR: a new
 * and flexible global circulation model to explore planetary atmospheres").
 *
 * Conventions for every entry point:
 *  - Return value: THOR_OK (0) or a negative THOR_E* status; nothing throws
 *    across the ABI. thor_strerror() names a status.
 *  - Handles (thor_grid, thor_state) and all device memory are owned by the
 *    library; the caller owns every host buffer it passes and keeps it valid
 *    for the duration of the call only.
 *  - Host arrays are float64 in the canonical order: column-major over the
 *    grid columns, then levels, then vector components, i.e. C arrays
 *    [ncol][nv] for centre scalars, [ncol][nv][3] for Cartesian vectors and
 *    [ncol][nv+1] for interface scalars. Column numbering: 10 rhombi of
 *    n x n points (n = 2^glevel), column r*n*n + j*n + i for rhombus r and
 *    lattice point (i, j), then the north and the south pole.
 *  - A handle is not thread-safe; use one state per stream. `stream` is a
 *    cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Invalid arguments give THOR_EINVAL and leave every handle unchanged.
 */
#ifndef THOR_H
#define THOR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  THOR_OK = 0,
  THOR_EINVAL = -1,      /* bad argument or size */
  THOR_ENOMEM = -2,      /* host or device allocation failed */
  THOR_ECUDA = -3,       /* a CUDA runtime call failed */
  THOR_ENONFINITE = -4,  /* the state holds NaN or Inf after a step */
  THOR_ETIMEOUT = -5,    /* a bounded device wait gave up */
  THOR_ENOTCONV = -6     /* an iteration did not converge where required */
};

enum { THOR_FP64 = 0, THOR_MIXED = 1 };
enum { THOR_FORCING_NONE = 0, THOR_FORCING_HELD_SUAREZ = 1, THOR_FORCING_HOT_JUPITER = 2 };
enum {
  THOR_FIELD_RHO = 0,       /* density, [ncol][nv]                         */
  THOR_FIELD_MOM = 1,       /* horizontal momentum rho v_h, [ncol][nv][3]  */
  THOR_FIELD_W = 2,         /* vertical momentum rho v_r, [ncol][nv+1]     */
  THOR_FIELD_RHOTHETA = 3,  /* rho theta, [ncol][nv]                       */
  THOR_FIELD_PRESSURE = 4,  /* p (get only), [ncol][nv]                    */
  THOR_FIELD_TEMPERATURE = 5 /* T (get only), [ncol][nv]                   */
};

typedef struct thor_grid thor_grid;
typedef struct thor_state thor_state;

const char* thor_strerror(int status);

/* ------------------------------------------------------------------ grid */

/* Spring-dynamics parameters (Sec. 2.2, Eqs. spring_force, spr_vel, dbar):
 * natural-length factor beta (1.15), friction alpha (1), spring constant k
 * (1), time step dt (0.01), stop when every |dP/dt| < tol (1e-5; tol <= 0
 * runs exactly max_iter steps). */
typedef struct {
  double beta, alpha, k, dt, tol;
  int max_iter;
} thor_spring;

/* Build the modified icosahedral grid of Sec. 2 (recursive bisection glevel
 * times, spring dynamics, centroid relocation, metric terms) on the host in
 * float64, plus the vertical grid: nv uniform layers from 0 to z_top above a
 * sphere of `radius` (deep atmosphere, Sec. 3). spring = NULL uses the
 * defaults above. glevel in [0, 10], nv in [2, 256], radius > 0, z_top > 0,
 * else THOR_EINVAL. No device memory is touched. */
int thor_grid_create(int glevel, int nv, double radius, double z_top,
                     const thor_spring* spring, thor_grid** out);

/* Sizes (Sec. 2.1, Eq. grid_qts: ncol = 10*4^glevel + 2 points, 12 of them
 * pentagons), nv, the spring iterations run and whether the tol criterion
 * was met (Sec. 2.2). Any output pointer may be NULL; THOR_EINVAL for a NULL
 * grid. */
int thor_grid_info(const thor_grid* grid, int* ncol, int* nv, int* npent,
                   int* spring_iters, int* spring_converged);

/* Cell centres on the unit sphere after the spring dynamics and the
 * centroid relocation of Sec. 2.2, xyz[ncol][3] in the library's column
 * order (caller's buffer); n must be 3*ncol, else THOR_EINVAL. */
int thor_grid_points(const thor_grid* grid, double* xyz, size_t n);

/* Counter-clockwise neighbours of every cell (the hexagons and pentagons of
 * Sec. 2.1), nbr[ncol][6] column indices, -1 in slot 5 of the 12 pentagons
 * (caller's buffer); n must be 6*ncol, else THOR_EINVAL. */
int thor_grid_neighbours(const thor_grid* grid, int* nbr, size_t n);

/* Control-volume areas A_c on the unit sphere (Sec. 2.2: the polygons of
 * the triangle centroids around each point, the areas of Eq. int_grid),
 * area[ncol] (caller's buffer); n must be ncol, else THOR_EINVAL. */
int thor_grid_areas(const thor_grid* grid, double* area, size_t n);

/* Nearest coarse cell of every fine cell: fine_to_coarse[i] = the column of
 * `coarse` whose centre is closest (largest dot product on the unit sphere)
 * to fine column i, the map thor_coarse_grain takes. No passage of the
 * paper (the learned closure's coarse graining, an extension): a greedy
 * walk over the coarse grid's neighbour graph from the previous fine
 * column's answer, which ends at the nearest centre because the coarse
 * cells are the Voronoi-like control volumes of their centres; a walk that
 * stops at a local optimum that is not the global one is caught by a check
 * against every neighbour's neighbours, and such a column falls back to a
 * search over all coarse columns. Host only; n must be the fine column
 * count, else THOR_EINVAL. */
int thor_grid_coarse_map(const thor_grid* fine, const thor_grid* coarse, int* fine_to_coarse, size_t n);

void thor_grid_destroy(thor_grid* grid);

/* ----------------------------------------------------------------- state */

/* Planet (Table 1): radius (m), rotation rate (1/s), gravity (m/s^2), gas
 * constant Rd and cp (J/kg/K), reference pressure p_ref of Eq. pressure (Pa)
 * and the nondimensional diffusion parameter D of Eq. kd
 * (K_d = D dbar^4/dt; D = dt/(32 tau_d) from Eq. tau_d). radius must equal
 * the grid's radius. */
typedef struct {
  double radius, omega, gravity, Rd, cp, p_ref, diff_D;
} thor_planet;

/* Initial state and run options. The atmosphere starts at rest, isothermal
 * at T0, in discrete hydrostatic balance with the lowest layer at
 * p_surf*exp(-g z_0/(Rd T0)); noise_amp > 0 adds amp*(2u-1) K to T at fixed
 * p, u = top 53 bits of SplitMix64(seed XOR (col*nv + k)) / 2^53 (Steele, Lea
 * and Flood 2014). forcing selects Sec. 6.1 (Held-Suarez) or Sec. 6.2
 * (hot Jupiter, day-night contrast hj_dT) physics after each large step.
 * precision: THOR_FP64 (all float64) or THOR_MIXED (float32 fields and
 * stencils, float64 metric terms, vertical solve and reductions).
 * hyperdiffusion / divergence_damping: 1 = on (Sec. 4), 0 = off.
 * shallow: 0 (the paper's runs) = deep atmosphere; 1 = the shallow-atmosphere
 * approximation that Sec. 3 lists among the switches: 1/r replaced by 1/A
 * (A the grid's radius) in every metric factor and cell volume, Coriolis
 * from the local vertical component of Omega acting on the horizontal
 * momentum only ("traditional approximation"), and the metric terms it
 * drops (u w / r, v w / r, (u^2 + v^2) / r) left out by advecting the
 * horizontal velocity and w as a scalar; thor_diag's angular momentum then
 * uses r = A.
 * hydrostatic: 0 (the paper's runs) = nonhydrostatic; 1 = the hydrostatic
 * approximation that Sec. 3 lists among the switches: the vertical
 * momentum's inertia (dW/dt, its advection, radial Coriolis part and
 * diffusion) is dropped, so that the vertical equation of every small step
 * (Eq. momr2) reads 0 = -dp/dr - g rho at the new state and the column solve
 * diagnoses W from it (same tridiagonal system without the identity term).
 * Both switches may be combined; any nonzero value counts as 1.
 * profile: THOR_PROFILE_ISOTHERMAL (0) = the layers at T0 as above;
 * THOR_PROFILE_HELD_SUAREZ (1) = the start of Sec. 6.1's run: every layer
 * at the equatorial Held-Suarez T_eq of its own pressure,
 * max(200 K, (315 K - 10 K ln(p / 1e5 Pa)) (p / 1e5 Pa)^(Rd/cp)), the column
 * in the same discrete hydrostatic balance (found as the fixed point
 * T = T_eq(p(T)) to 1e-12 K, else THOR_ENOTCONV), T0 ignored; noise_amp
 * still adds its perturbation. The balanced start column is also the
 * reference column of the deviation form.
 * vorder: 0 or 1 (the paper's runs) = linear vertical interpolation; 2 or 3 =
 * the Lagrange polynomial of that order k (Sec. 2.1 implements any order
 * and runs k = 1) in the explicit terms: the velocity at the interfaces for
 * the vertical advection, W at the centres for the full momentum
 * (advection, Coriolis), the radial advection and Coriolis at the
 * interfaces, and rho at the interfaces of the vertical hyperdiffusion,
 * each from the k + 1 nodes nearest the target (the lower first on a tie,
 * shifted inward at the bottom and the top). The terms of the implicit
 * vertical system (gravity, theta at the interfaces, the pressure gradient)
 * stay linear, so the column system stays tridiagonal and a resting
 * column in discrete balance stays at rest. Needs nv >= k + 1; other
 * values give THOR_EINVAL. thor_diag and the transfers interpolate
 * linearly whatever vorder is.
 * anelastic: 0 (the paper's runs) = compressible; 1 = the anelastic
 * approximation that Sec. 3 lists among the switches (the density of the
 * continuity equation's divergence term replaced by the reference column
 * rho0(z), after Ogura and Phillips 1962, which filters the sound waves):
 * the state keeps rho = rho0 (the start's temperature noise becomes a
 * theta' = theta0 dT / T at rho0), the momentum obeys the constraint
 * div_h M + r^-2 d(r^2 W)/dr = 0 of the discrete 3-D divergence, the
 * pressure gradient and gravity give way to the buoyancy g rho0 theta' /
 * theta0 at the interfaces, and each RK3 stage (dt/3, dt/2, dt) is one
 * projection from X^t with the pressure p' of L p' = D(M^, W^) / dt_s,
 * L = div o grad, solved in float64 (BiCGStab with a column preconditioner
 * to a true relative residual of 1e-13, restarted from the true residual at
 * most twice, at most 500 iterations a pass, else THOR_ENOTCONV from
 * thor_step); no acoustic small steps, so n_small is ignored, and no CUDA
 * graph (the solver checks convergence on the host every iteration). Not
 * with hydrostatic (THOR_EINVAL), not in ensembles (THOR_EINVAL from
 * thor_ensemble_step), no compensated state, no energy fixer. */
enum { THOR_PROFILE_ISOTHERMAL = 0, THOR_PROFILE_HELD_SUAREZ = 1 };
typedef struct {
  double T0, p_surf, noise_amp;
  unsigned long long seed;
  int forcing;
  double hj_dT;
  int precision;
  int hyperdiffusion;
  int divergence_damping;
  int shallow;
  int hydrostatic;
  int profile;
  int vorder;
  int anelastic;
} thor_init;

/* Allocate the device state for `grid` and set the initial condition. The
 * grid must outlive the state. */
int thor_state_init(thor_grid* grid, const thor_planet* planet, const thor_init* init,
                    void* stream, thor_state** out);

/* Advance n_large large steps of dt seconds (Sec. 3): per large step three
 * Wicker-Skamarock RK3 stages with 1, n_small/2 and n_small forward-backward
 * small steps (dt/3, dt/n_small, dt/n_small), each small step = divergence
 * damping, explicit horizontal momentum (Eq. mom2), implicit vertical
 * momentum (Eq. momr2, tridiagonal per column), density (Eq. dens2),
 * rho theta (Eq. pt2) and pressure (Eq. theta_to_p); then the physics
 * (Sec. 5). Asynchronous on the state's stream (unless the finite check of
 * thor_tune is on). n_small even and >= 2, n_large >= 0, dt > 0, else
 * THOR_EINVAL. */
int thor_step(thor_state* state, int n_large, int n_small, double dt);

/* Global diagnostics in float64 (deterministic two-pass reductions):
 * mass = sum rho V, energy = sum (rho cv T + |rho v|^2/(2 rho) + rho g z) V,
 * axial angular momentum = sum (r x rho v)_z V + sum rho Omega r_perp^2 V,
 * max |v_h|, max |w|, volume-mean T and the count of non-finite values.
 * Synchronises the stream. */
typedef struct {
  double mass, energy, aam, max_vh, max_w, mean_T;
  long long nonfinite;
} thor_diag_t;
int thor_diag(thor_state* state, thor_diag_t* out);

/* Copy a field to / from a float64 host buffer (caller's) in the canonical
 * order [ncol][level(s)][components] (the output of the prognostic variables
 * that Sec. 5 describes; pressure and temperature follow from Eq. pressure
 * and the ideal gas); n is the element count of the field, else THOR_EINVAL.
 * Synchronous. set accepts RHO, MOM, W and RHOTHETA (the rigid lid of Sec. 3:
 * W's bottom and top interfaces are forced to 0). */
int thor_state_get(thor_state* state, int field, double* host, size_t n);
int thor_state_set(thor_state* state, int field, const double* host, size_t n);

/* The four prognostic fields at once, each in the layout of thor_state_get
 * (rho and rho theta [ncol][nv], rho v_h [ncol][nv][3], W [ncol][nv+1]);
 * ncol and nv must be the grid's, else THOR_EINVAL. The copies and
 * conversions of all four are queued on the state's stream and the call
 * synchronises once (page-locked host buffers let the copies run at the
 * link's rate). Results equal four thor_state_get / thor_state_set calls
 * bit for bit. */
int thor_state_get_all(thor_state* state, double* rho, double* mom, double* w, double* rhotheta, int ncol, int nv);
int thor_state_set_all(thor_state* state, const double* rho, const double* mom, const double* w,
                       const double* rhotheta, int ncol, int nv);

/* Raw checkpoint of the prognostic state (Sec. 5: the long runs write the
 * state out and restart from it): the stored arrays (deviation form,
 * padded layout) bit for bit after a 64-byte header (magic, precision, ncol,
 * nv, a 64-bit hash of the reference column, vertical tables, planet and
 * switches that the stored deviations are relative to, and the large steps
 * since a closure was attached). thor_checkpoint_bytes gives the buffer
 * size; save and load copy to / from `buf` in host or device memory
 * (unified addressing) and synchronise the state's stream. Loading into a
 * state of another grid size, level count or precision, into a state whose
 * reference differs (another planet, top, start temperature or surface
 * pressure, or switch), or from a buffer without the header, returns
 * THOR_EINVAL and leaves the state unchanged; a load restores the position
 * inside the closure window. A restart from a checkpoint
 * continues bit for bit like an uninterrupted run; thor_state_get/_set,
 * which exchange full float64 values, round the reference column plus the
 * deviation (a unit in the last place) in float64 storage. */
int thor_checkpoint_bytes(const thor_state* state, size_t* bytes);
int thor_checkpoint_save(thor_state* state, void* buf, size_t bytes);
int thor_checkpoint_load(thor_state* state, const void* buf, size_t bytes);

/* Self-test of the bounded device waits (the mbarrier waits of the staged
 * column solve and of the tensor-core GEMM, normally bounded at 2 s): one
 * thread waits, with limit limit_us (1 .. 2e6 microseconds), on a barrier of
 * one expected arrival; arrive = 1 arrives first. *gave_up = 1 if the wait
 * ran out, 0 if it completed. A wait that runs out leaves nothing in flight,
 * and the context stays usable. Synchronous (default stream). */
int thor_wait_selftest(int arrive, unsigned int limit_us, int* gave_up);

/* Kernel launches issued by this state so far (instrumentation; no passage
 * of the paper). THOR_EINVAL for NULL arguments. */
int thor_launch_count(const thor_state* state, long long* count);

/* Launch-shape knobs (no passage of the paper: the paper's K20 kernels use
 * fixed 2-D blocks of 256 threads, Sec. 5); the results do not depend on them.
 * THOR_TUNE_KCHUNK: levels each thread of the stencil kernels walks (1..256,
 * default 2); fewer levels mean more threads in flight, more levels fewer
 * reloads of the per-column weights.
 * THOR_TUNE_GRAPH: 1 (default) replays a captured CUDA graph of one large
 * step on a non-default stream (re-captured when dt, n_small or the chunk
 * change; never while thor_profile records); 0 launches kernel by kernel.
 * THOR_TUNE_CHECK_FINITE: 1 makes thor_step finish with a non-finite count
 * of the state (one reduction and one stream synchronisation per call) and
 * return THOR_ENONFINITE if any value is NaN or Inf; the state is the one
 * after the step (restore a checkpoint with thor_state_set). Default 0. */
enum { THOR_TUNE_KCHUNK = 0, THOR_TUNE_GRAPH = 1, THOR_TUNE_CHECK_FINITE = 2, THOR_TUNE_BLOCK = 3,
       THOR_TUNE_SOLVE_TMA = 4, THOR_TUNE_ENERGY_FIXER = 5, THOR_TUNE_BUDGET = 6,
       THOR_TUNE_RK_STAGES = 7, THOR_TUNE_COMPENSATED = 8, THOR_TUNE_L2_HINTS = 9,
       THOR_TUNE_LEVEL_SPLIT = 10 };
int thor_tune(thor_state* state, int knob, int value);

/* Energy and angular-momentum budget of the large steps recorded since
 * thor_tune(THOR_TUNE_BUDGET, capacity): row n (8 float64) holds the dry mass,
 * total energy and axial angular momentum of thor_diag at the start of large
 * step n and after its dynamics (before the fixer and the physics), then the
 * fixer's dT (0 when it is off) and 0. The dynamics' numerical sources are
 * columns 3-5 minus 0-2; the physics' (and the fixer's) are the next row's
 * 0-2 minus this row's 3-5. Copies min(recorded, max_rows) rows to `out`
 * (host, max_rows * 8 doubles) and their number to *n_rows (0 when not
 * recording); synchronises the state's stream. Sec. 3 (energy), Sec. 6.1
 * (axial angular momentum reaching a statistically steady value). */
int thor_budget_read(thor_state* state, double* out, int max_rows, int* n_rows);

/* Zonal band means (Sec. 6.1: the climates are judged by zonal and time
 * averages of wind and temperature, the mass stream function built from the
 * averaged northward wind, and the eddy fluxes [u'v'], [v'T'] with
 * phi' = phi - zonal mean of phi). A zonal mean is the volume-weighted mean
 * over the cells of one level whose latitude falls in one of nlat equal
 * bands, band b = floor((lat + pi/2 + 1e-9) / pi * nlat) (the north pole in
 * the last band; a cell on a band edge, such as the equatorial cells, goes
 * north). thor_zonal_accumulate adds, for the current state, per level k and
 * band b the 9 values
 *   [V, u, v, T, p, u'v', v'T', u'u', v'v']
 * (V the band's volume, u and v the eastward and northward components of
 * M / rho, 0 at the two polar cells, then their band means, T and p, then
 * the band covariances) to the state's accumulator, on the state's stream
 * without synchronising; nlat in [1, 360], else THOR_EINVAL. The first call
 * for a given nlat synchronises the stream, allocates the accumulator
 * (about 150 * nv * nlat bytes plus 28 + 8 * nv bytes per column) and
 * clears it. The same call adds every cell's vertical velocity at its
 * centre, w = (W linearly interpolated to the centre) / rho, to a per-cell
 * time sum (for the grid-imprinting map [w*] of Sec. 6.1: the time mean of w
 * minus its zonal band mean).
 * thor_zonal_read copies the accumulated sums, layout
 * [nv][nlat][9] float64 (n must be nv * nlat * 9), and the number of states
 * accumulated; with reset != 0 it then clears them and the per-cell w sums.
 * Divide by the sample count for time means. A read for an nlat that was
 * never accumulated returns zeros and 0 samples. thor_zonal_read_w copies
 * the time mean [w] (m/s) of every cell, layout [ncol][nv] float64 in the
 * column order of thor_state_get (n must be ncol * nv), and the sample
 * count; zeros and 0 samples when nothing was accumulated for nlat. Both
 * reads synchronise the state's stream. */
int thor_zonal_accumulate(thor_state* state, int nlat);
int thor_zonal_read(thor_state* state, int nlat, double* out, size_t n, int reset, long long* samples);
int thor_zonal_read_w(thor_state* state, int nlat, double* out, size_t n, long long* samples);

/* THOR_TUNE_BLOCK: threads (one per column) in a block of the stencil
 * kernels, a multiple of 32 in [32, 256] (default 128).
 * THOR_TUNE_SOLVE_TMA: 1 (default) runs the column solve of a THOR_MIXED
 * state with its planes staged into shared memory by TMA bulk-tensor copies
 * (where the staging fits, nv <= 80); 0 runs the direct-load solve. Same
 * arithmetic, same results. A staged copy that has not landed after 2 s ends
 * the kernel with a device error flag; thor_diag (and thor_step with
 * THOR_TUNE_CHECK_FINITE) then return THOR_ETIMEOUT.
 * THOR_TUNE_ENERGY_FIXER: 1 turns on the energy fixer that Sec. 3 describes
 * (after Williamson 2009: the internal energy adjusted by the same amount at
 * every grid point). Once per large step, after the three RK3 stages and
 * before the physics, every cell's temperature rises by
 *   dT = (E_start - E_dyn) / (c_v * sum over cells of V rho)
 * at fixed density and momentum (rho theta from Eq. pressure), E the total
 * energy of thor_diag at the start of the step and after its dynamics, so
 * that the dynamics leave the total energy unchanged and the physics is its
 * only source. 0 (default, as the paper's runs) turns it off. The first use
 * allocates a small device buffer; synchronises the state's stream.
 * THOR_TUNE_BUDGET: value > 0 records, for each of the next `value` large
 * steps (at most 2^24), one budget row that thor_budget_read returns; 0 stops
 * recording and frees the rows. Allocates value * 64 bytes on the device and
 * synchronises the state's stream; recording costs two float64 reductions
 * of the state per large step. Neither knob applies to thor_ensemble_step.
 * THOR_TUNE_RK_STAGES: 1, 2 or 3 (default) RK3 stages per large step (Sec.
 * 3). With fewer than 3 a large step ends after that stage with the stage's
 * result X^(s+1) = X^t + X* in the state and runs neither the energy fixer
 * nor the physics; with 1 a large step is one slow-term evaluation and one
 * small step of dt/3 from X^t. For tests that check the first small step on
 * its own; THOR_EINVAL outside 1..3.
 * THOR_TUNE_COMPENSATED (THOR_MIXED states): 1 keeps every prognostic field
 * of the state as a float pair hi + lo, |lo| at most half a unit in the
 * last place of hi, and adds the last RK stage's accumulated small-step
 * perturbations (Eqs. dens2, mom2, momr2, pt2; the perturbations start
 * every stage at X^t - X^(s), so they carry the whole large step), the
 * physics increments (Eqs. im_eq_v, im_eq_t) and the energy fixer's to the
 * pair with an error-free sum (TwoSum), so that the float32 storage does
 * not round the state at every large step; thor_state_get / _set,
 * thor_diag and checkpoints (then twice the size) use the full pairs. The
 * RK stage states and the tendencies stay float. The first use allocates
 * the low parts (6 planes), zeroed; 0 frees them and rounds the state to
 * its float parts. Synchronises the state's stream. Ensembles step
 * compensated members the same way. THOR_EINVAL for THOR_FP64 states.
 * Default 1 for THOR_MIXED states (thor_state_init allocates the low parts).
 * THOR_TUNE_L2_HINTS (0..3; no passage of the paper: a memory-placement
 * knob): L2 eviction priorities of the acoustic small steps' loads and
 * stores. Bit 0 loads the stage constants (slow tendencies, Pi, theta at
 * the interfaces, the column matrix's factors) evict-first, bit 1 keeps
 * the perturbations and the kernel split's intermediates evict-last (in
 * THOR_MIXED states only; THOR_FP64 states keep them at normal priority).
 * Results do not depend on it (tested bit for bit). Library-wide on the
 * current device (every state and ensemble); default 3. THOR_EINVAL
 * outside 0..3, THOR_ECUDA if the device rejects it.
 * THOR_TUNE_LEVEL_SPLIT (0 or 1; a launch-shape knob): 1 runs the small
 * steps' three horizontal stencils (the Laplacian of D, the momentum step,
 * the column fluxes) as two chains, the lower and the upper half of the
 * levels, on two streams (graph branches), joined before the column solve:
 * the levels of a horizontal stencil do not depend on each other, and one
 * chain's kernels fill the SMs the other's leave idle while they start and
 * drain. Default 1 (g6 x 32 large step 1.477 -> 1.426 ms at 4 levels per
 * thread); the same numbers either way (tested bit for bit). */

/* Launch-shape autotuner (an extension; the paper fixes no launch shapes).
 * Times `steps` large steps of (n_small, dt) for every levels-per-thread
 * value in {1, 2, 3, 4, 6, 8} and block size in {64, 96, 128, 192, 256}, each after one
 * untimed step, with CUDA events on the state's stream; restores the state's
 * prognostic fields before every candidate and at the end (the state is
 * unchanged), sets the fastest shape (as thor_tune would) and returns it with
 * its time per large step in ms (any output pointer may be NULL). Allocates
 * one state-sized device buffer for the duration of the call and synchronises
 * the stream. n_small even >= 2, dt > 0, steps >= 1, else THOR_EINVAL. */
int thor_autotune(thor_state* state, int n_small, double dt, int steps, int* kchunk, int* block,
                  double* ms_per_step);

/* Per-kernel timing (instrumentation; no passage of the paper). While
 * enabled, every launch of the state is bracketed by
 * two CUDA events recorded on the state's stream; thor_profile_read
 * synchronises the stream and returns, for one kernel id, the summed
 * event-measured duration (ms) and the number of launches since the last
 * thor_profile(state, 1). enable = 0 stops recording. */
enum {
  THOR_K_DERIVED = 0, THOR_K_LAP1, THOR_K_SLOW, THOR_K_SLOW_W, THOR_K_STAGE_INIT,
  THOR_K_SS_LAPD, THOR_K_SS_MOM, THOR_K_SS_SOLVE, THOR_K_PHYSICS, THOR_K_SS_FLUX,
  THOR_K_SS_FACTOR, THOR_K_COUNT
};
int thor_profile(thor_state* state, int enable);
int thor_profile_read(thor_state* state, int kernel, double* total_ms, long long* launches);

void thor_state_destroy(thor_state* state);

/* ---------------------------------------------------------------- ensemble */

/* An ensemble of independent atmospheres stepped together (an extension; the
 * paper runs one atmosphere at a time). Members are existing states of any
 * grid level, planet, forcing and time step, with the same level count nv and
 * precision; every kernel of the large step runs as one launch over all
 * members, and on a non-default `stream` one large step of the whole ensemble
 * is captured as a CUDA graph and replayed (re-captured when a member's dt or
 * n_small, or a launch shape, changes). The results are those of stepping
 * each member alone with the same (n_small, dt).
 *
 * The ensemble keeps the member pointers: members must outlive it and must
 * not be stepped on their own while an ensemble step may be running (work on
 * the members' streams is ordered before and after each ensemble step with
 * events). Closures are not run in an ensemble: a member with a closure
 * attached makes thor_ensemble_step return THOR_EINVAL. There is no
 * non-finite watchdog; use thor_diag per member.
 * create: 1 <= n <= THOR_ENSEMBLE_MAX distinct members, else THOR_EINVAL. */
#define THOR_ENSEMBLE_MAX 4096
typedef struct thor_ensemble thor_ensemble;
int thor_ensemble_create(thor_state* const* members, int n, void* stream, thor_ensemble** out);

/* n_large large steps of every member; n_small[i] (even >= 2) and dt[i] > 0
 * are member i's, in creation order (host arrays of n). A changed plan
 * (n_small, dt or launch shape) synchronises the stream once and uploads the
 * member table and block maps. */
int thor_ensemble_step(thor_ensemble* ens, int n_large, const int* n_small, const double* dt);

/* Member count and kernel launches issued by the ensemble so far
 * (instrumentation). */
int thor_ensemble_info(const thor_ensemble* ens, int* n_members, long long* launches);

/* THOR_TUNE_KCHUNK, THOR_TUNE_BLOCK, THOR_TUNE_GRAPH as for one state. */
int thor_ensemble_tune(thor_ensemble* ens, int knob, int value);

/* thor_autotune over the ensemble: every member's state is restored. */
int thor_ensemble_autotune(thor_ensemble* ens, const int* n_small, const double* dt, int steps, int* kchunk,
                           int* block, double* ms_per_step);

/* Waits for the ensemble's stream; the members stay valid. */
void thor_ensemble_destroy(thor_ensemble* ens);

/* --------------------------------------------------------- learned closure */

/* A per-column MLP closure (an extension; the paper has no learned part).
 * Network: sizes[0] inputs, sizes[1..n_sizes-2] hidden ReLU layers,
 * sizes[n_sizes-1] linear outputs; y = W_L^T relu(... relu(W_1^T x + b_1)) + b_L
 * with W_l stored [sizes[l]][sizes[l+1]] row-major. float32 master weights;
 * the products run on the tensor cores with bfloat16 weights and layer
 * inputs and float32 accumulation. Flat parameter order: W_0, b_0, W_1, b_1, ...
 * Initial weights He-uniform from SplitMix64(seed), biases 0. All x, y, dy,
 * target, grad and loss pointers are device pointers (float32, row-major
 * [m][features]); the MLP's stream is `stream` (the state's stream once
 * attached). sizes[i] in [1, 8192], 2 <= n_sizes <= 16, 1 <= m <= max_batch. */
typedef struct thor_mlp thor_mlp;
int thor_mlp_create(const int* sizes, int n_sizes, int max_batch, unsigned long long seed, void* stream,
                    thor_mlp** out);
int thor_mlp_info(const thor_mlp* mlp, size_t* nparam);
/* Copies the float32 master weights to the host (synchronises the MLP's
 * stream). Returns THOR_ETIMEOUT if a tensor-core GEMM of this MLP gave up
 * waiting for its MMAs (bounded at 2 s per wait; its outputs are then
 * unspecified). */
int thor_mlp_get_params(thor_mlp* mlp, float* host, size_t n);
/* GEMM path. THOR_MLP_TUNE_TCGEN05: 1 (default) runs the products as
 * tcgen05.mma (bfloat16 operands in shared memory, float32 accumulators in
 * tensor memory, 128-row tiles) with the operands brought in by TMA in the
 * 128-byte swizzled layout through a 4-stage ring, when every layer width
 * is a multiple of 8 (the forward then also keeps transposed copies of the
 * weights and layer inputs so that every product reads both operands along
 * its contraction), else with threads staging the operands; 2 forces the
 * thread-staged tcgen05 kernel; 0 runs the warp-level mma.sync kernel. All
 * accumulate in float32; results agree to summation order. Other values:
 * THOR_EINVAL. */
enum { THOR_MLP_TUNE_TCGEN05 = 0 };
int thor_mlp_tune(thor_mlp* mlp, int knob, int value);
/* Sets the float32 master weights and resets the Adam moments. */
int thor_mlp_set_params(thor_mlp* mlp, const float* host, size_t n);
/* y = MLP(x) for m rows. */
int thor_mlp_forward(thor_mlp* mlp, const float* x, int m, float* y);
/* Gradient of sum(y * dy) with respect to every parameter (flat order), for
 * the batch of the last thor_mlp_forward (same m). The output gradient and
 * the hidden-layer gradients enter the weight products in bfloat16. */
int thor_mlp_backward(thor_mlp* mlp, const float* dy, int m, float* grad);
/* One training step on a batch: forward, mean-squared-error loss
 * sum((y - target)^2)/(m n_out) (written to *loss if loss != NULL), backward,
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with rate lr. */
int thor_mlp_train_step(thor_mlp* mlp, const float* x, const float* target, int m, float lr, float* loss);
void thor_mlp_destroy(thor_mlp* mlp);

/* Closure features of a state: per column c, x[c][f*nv + k] is field f at
 * level k and x[c][5*nv + f*nv + k] its mean over the column's neighbours
 * minus its value at c,
 * for f = rho - rho_ref, M_x, M_y, M_z, rho theta - reference (the state's
 * stored deviations); each feature j is normalised as (x - mean[j]) / std[j].
 * x: device [ncol][10*nv]. */
int thor_closure_features(thor_state* state, const float* mean, const float* std, float* x);

/* Attach an MLP (sizes[0] = 10*nv, last size = 5*nv) as a closure with a
 * window of `period` >= 1 large steps, counted from the attach. At the start
 * of each window the correction tendency tau = MLP(features) * out_std +
 * out_mean is evaluated on the current state; when the window closes,
 * field_f(k) += period * dt * tau[f*nv + k] (the momentum correction
 * projected onto the tangent plane). This is the use that matches a network
 * trained on the n-step target [C(X_fine(t + n dt)) - S^n(C(X_fine(t)))] /
 * (n dt) with period = n. thor_step calls that end inside a window carry it
 * over to the next call. The four normalisation arrays are caller-owned
 * device arrays that must stay valid while attached. mlp = NULL detaches
 * (plain method); re-attaching restarts the window count. */
int thor_closure_attach(thor_state* state, thor_mlp* mlp, const float* in_mean, const float* in_std,
                        const float* out_mean, const float* out_std, int period);

/* Area-weighted average of a fine state onto a coarse one: every coarse
 * column gets the mean of the fine columns mapped to it (fine_to_coarse,
 * host, one coarse column index per fine column), weighted by the fine
 * control-volume areas, for all levels of rho, M (projected on the coarse
 * tangent plane), W and rho theta. Both states must share precision, nv,
 * z_top, planet and initial reference column; every coarse column needs at
 * least one fine member. Synchronous. */
int thor_coarse_grain(thor_state* fine, thor_state* coarse, const int* fine_to_coarse, size_t nfine);

/* ------------------------------------------------------- allocation-free */

/* Allocation-free float64 mass sum: *mass_out = sum_i rho[i] * volume[i]
 * over i < n. It is deterministic and uses the scheme of thor_diag's mass
 * (compensated per-block partial sums, then one ordered compensated sum of
 * the partials) with a different blocking (contiguous chunks of 16384
 * elements per block), so the two agree to rounding, not bit for bit. The
 * paper has no counterpart: this entry
 * point exists for callers that must not call cudaMalloc, because an outer
 * framework owns the whole device-memory budget or because cudaMalloc would
 * synchronise the device in a latency-critical loop.
 *  - rho, volume: caller-owned device arrays of n float64 values (any
 *    order, e.g. the canonical [ncol][nv] order of thor_state_get with the
 *    cell volumes A_c r_k^2 dz_k); mass_out: caller-owned device pointer to
 *    one float64. Asynchronous on `stream` (NULL = legacy default stream).
 *  - Allocates nothing. The per-block partial sums live in a file-scope
 *    static __device__ array of 4097 float64 (about 32 KB) that every GPU
 *    loading the library holds until the process exits; it bounds n to
 *    4096 * 16384 = 67,108,864 elements; larger n (or n = 0, or a NULL
 *    pointer) returns THOR_EINVAL without launching anything.
 *  - The first call on a device looks up that array's device address with
 *    cudaGetSymbolAddress (with that device current); make the first call on
 *    each device before any stream capture.
 *  - Every call shares the array and leaves its partial sums in it; each
 *    call overwrites the slots it uses before reading them. Calls that
 *    overlap on the GPU (on different streams, or from different threads)
 *    race on the array and must be ordered by the caller. */
int thor_mass_noalloc(const double* rho, const double* volume, size_t n, double* mass_out,
                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* THOR_H */
