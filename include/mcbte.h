/*
 * mcbte.h -- C ABI of the GB300 deviational Monte Carlo solver for the
 * linearised phonon Boltzmann transport equation (arXiv:2104.03573, MCBTE).
 *
 * The library traces independent signed deviational energy particles
 * (Sec. 3, Eq. deviational_approx): emission from isothermal walls, an
 * initial condition or a control-gradient body source, straight flights,
 * exponential relaxation clocks, relaxation resampling ~ C/tau, adiabatic /
 * isothermal / periodic boundaries and steady track-length or transient
 * snapshot tallies.  All tracing, table building, source setup and
 * finalisation run in CUDA kernels on one GPU (sm_103a).
 *
 * Conventions for every call:
 *   - Return an mcbte_status; 0 is success.  No call exits, traps or prints.
 *   - mcbte_last_error() gives a message for the last failure of the calling
 *     host thread.
 *   - Handles are opaque, owned by the library, released by *_destroy.
 *   - Descriptor arrays (material columns, wall data, t_meas, n_particles)
 *     are HOST memory, read during the call and not retained.
 *   - Output buffers are owned by the caller.  They are all device memory
 *     (on_host = 0; results are written asynchronously on `stream`) or all
 *     host memory (on_host = 1; the call copies results back and
 *     synchronises `stream` before returning).
 *   - `stream` is a cudaStream_t; NULL is the legacy default stream.
 *   - Units at the boundary are SI (m, s, K, W).
 */
#ifndef MCBTE_H
#define MCBTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mcbte_stream; /* == cudaStream_t */

/* Largest number of transient measurement times: the FP32 tracer keeps them
 * in shared memory (4 bytes each). */
#define MCBTE_MAX_TIMES 16384

/* Largest n_scat_max of a run that returns the N_scat_max convergence curve
 * (Sec. 3.5.6 leaves N_scat_max to a convergence study). */
#define MCBTE_MAX_NSCAT_CURVE 4096

/* Largest number of detector regions of a run (Sec. 4.5). */
#define MCBTE_MAX_REGIONS 16

typedef enum {
  MCBTE_OK = 0,
  MCBTE_ERR_INVALID_ARG = 1,   /* a descriptor or parameter is out of range  */
  MCBTE_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  MCBTE_ERR_OOM = 3,           /* device allocation failed                   */
  MCBTE_ERR_TIMEOUT = 4,       /* the run hit its wall-clock budget          */
  MCBTE_WARN_TRUNCATED = 5,    /* some particles hit max_events (results are
                                  written; the truncated count is in stats)  */
  MCBTE_ERR_WORKSPACE = 6,     /* caller workspace smaller than required     */
  MCBTE_ERR_REPLAY = 7         /* FP32 gradient pass did not reproduce a
                                  particle of the forward pass (internal)    */
} mcbte_status;

/* Message of the last failure on this host thread; returns its length.
 * Writes at most n bytes including the terminating NUL. */
int mcbte_last_error(char* buf, size_t n);

/* Library version as major*10000 + minor*100 + patch. */
int mcbte_version(void);

/* ------------------------------------------------------------------ material
 * Per-bin material table of the paper's mat_data.txt (Sec. 4.1): format 1
 * (omega, DOS D, V_g, d_omega, tau) or format 2 (omega, V_g, tau, C).
 * Create copies the columns to the device and builds, in FP64 on the GPU:
 *   C_i = D_i * dE/dT(omega_i, T_lin) * d_omega_i   (Eq. BE_derivative, Eq. Nbin)
 *         with dE/dT = k_B (x/2)^2 / sinh^2(x/2), x = hbar omega / (k_B T)
 *   alias tables (Walker / Vose) for bins ~ C v (wall and body emission,
 *   Eqs. iso_flux, grad_flux_sim), ~ C (initial condition, Eq. Nbin) and
 *   ~ C / tau (relaxation resampling, Eq. n_scatt).
 * Errors: n_bins < 1, any v <= 0 or tau <= 0, C < 0 (or D, d_omega < 0),
 * sum C == 0, T_lin <= 0 when D is given -> MCBTE_ERR_INVALID_ARG.
 * The call synchronises the device work it launches (legacy stream). */
typedef struct {
  int n_bins;
  const double* omega;   /* [n_bins] rad/s                                  */
  const double* v;       /* [n_bins] m/s, group velocity magnitude          */
  const double* tau;     /* [n_bins] s, relaxation time                     */
  const double* C;       /* [n_bins] J/(m^3 K), format 2; or NULL           */
  const double* D;       /* [n_bins] s/(rad m^3), format 1 (used if C NULL) */
  const double* domega;  /* [n_bins] rad/s, format 1                        */
  double T_lin;          /* K, linearisation temperature (Sec. 4.4)         */
  const double* spec_bin; /* [n_bins] optional per-bin specularity d(omega) in
                            [0, 1] (Sec. 3.5.3), used by faces and walls whose
                            specularity is given as < 0; or NULL          */
  const double* tau_imp; /* [n_bins] s, optional two-phonon (impurity)
                            relaxation times (the optional last column of
                            Sec. 4.1), or NULL; each > 0, +inf for none.
                            With it, two- and three-phonon scattering keep
                            separate clocks (Sec. 3.3): a two-phonon event
                            redraws the direction only; only three-phonon
                            events count toward n_scat_max             */
} mcbte_material_desc;

typedef struct mcbte_material mcbte_material;

mcbte_status mcbte_material_create(const mcbte_material_desc* desc, mcbte_material** out);
void mcbte_material_destroy(mcbte_material* m);
int mcbte_material_n_bins(const mcbte_material* m);

/* Copy the FP64 tables back to HOST buffers (any may be NULL):
 * C[n]; for table k in {0: ~C v, 1: ~C, 2: ~C/tau}: prob[k*n+i] (Vose
 * probability), thr[k*n+i] (64-bit keep threshold), alias[k*n+i];
 * sums[3] = (sum C, sum C v, sum C/tau). Synchronous. */
mcbte_status mcbte_material_tables(const mcbte_material* m, double* C, double* prob,
                                   uint64_t* thr, int32_t* alias, double* sums);

/* ------------------------------------------------------------------ geometry
 * Axis-aligned box [0,Lx]x[0,Ly]x[0,Lz], one corner at the origin (Sec. 4.2),
 * six faces in the paper's Boundary_prop.txt ID order (Sec. 4.3):
 *   index 0..5 = ID 1..6 = y=0, x=Lx, y=Ly, x=0, z=0, z=Lz.
 * Face types: isothermal (absorbing, emits at T_b; Sec. 3.5.4), adiabatic
 * with specularity p (Eq. specular, Sec. 3.5.3), periodic (translation by
 * the box length, spatially varying control, Eq. periodic_lin_final).
 * Optional cylindrical pore parallel to z at (cx, cy) with radius r and
 * specularity p_pore (boundary ID 7).  grad_T is the uniform control
 * gradient of Sec. 2.5 (Eq. lin_spatial), in any direction; it adds the body
 * source of Eq. grad_flux with |grad T|, particles Lambertian about
 * -+grad T / |grad T| (Sec. 3.2.3).  gauss adds an
 * initial-condition source dT exp(-|x-c|^2 / 2 sigma^2) (transient only).
 * Internal walls (Sec. 4.2, In_bnd.txt): up to MCBTE_MAX_INNER adiabatic
 * segments (x1, y1, x2, y2) in the x-y plane running through the thickness,
 * each with a unit normal (nx, ny) pointing into the solid and a specularity
 * (IDs after the cylinder).  They bound holes (the regions they enclose,
 * even-odd rule), which body sources avoid and the solid volume excludes; a
 * wall is met only from its solid side.  A specularity below 0 on an
 * adiabatic face or wall selects the material's per-bin d(omega)
 * (mcbte_material_desc.spec_bin; the run fails with MCBTE_ERR_INVALID_ARG if
 * the material has none).
 * Errors: L <= 0, periodic faces not paired on an axis, p above 1,
 * pore not inside the cell (r >= min(Lx,Ly)/2 or centre off), walls outside
 * the box or normals not of unit length -> MCBTE_ERR_INVALID_ARG. */
enum { MCBTE_FACE_ISOTHERMAL = 0, MCBTE_FACE_ADIABATIC = 1, MCBTE_FACE_PERIODIC = 2 };
#define MCBTE_MAX_INNER 16

typedef struct {
  double L[3];           /* m                                               */
  int face_type[6];
  double face_T[6];      /* K, isothermal faces                             */
  double face_p[6];      /* specularity in [0,1], adiabatic faces           */
  double T_eq;           /* K, control temperature                          */
  double grad_T[3];      /* K/m                                             */
  int pore;              /* 0 / 1                                           */
  double pore_c[2];      /* m                                               */
  double pore_r;         /* m                                               */
  double pore_p;         /* specularity of the pore wall                    */
  int gauss;             /* 0 / 1                                           */
  double gauss_c[3];     /* m                                               */
  double gauss_sigma;    /* m                                               */
  double gauss_dT;       /* K                                               */
  int n_inner;           /* internal walls, 0..MCBTE_MAX_INNER              */
  double inner[MCBTE_MAX_INNER][4];    /* x1, y1, x2, y2 (m)               */
  double inner_n[MCBTE_MAX_INNER][2];  /* unit normal into the solid       */
  double inner_p[MCBTE_MAX_INNER];     /* specularity; < 0: per bin        */
} mcbte_geometry_desc;

typedef struct mcbte_geometry mcbte_geometry;

mcbte_status mcbte_geometry_create(const mcbte_geometry_desc* desc, mcbte_geometry** out);
void mcbte_geometry_destroy(mcbte_geometry* g);

/* ------------------------------------------------------------------ runs */
enum { MCBTE_FP64_PLAIN = 0,      /* one thread per particle, FP64 throughout  */
       MCBTE_FP32_TRACE = 1 };    /* persistent FP32 tracer, FP64 tallies      */

/* stats[] layout of every run (per geometry for steady runs) */
enum {
  MCBTE_STAT_KAPPA = 0,       /* W/m/K, -q_mean / (dT/dx) along tally_axis (solid volume)  */
  MCBTE_STAT_KAPPA_SE,        /* standard error of kappa                                  */
  MCBTE_STAT_Q_MEAN,          /* W/m^2, mean flux along tally_axis over the solid (Eq. flux_x_steady) */
  MCBTE_STAT_Q_SE,
  MCBTE_STAT_SUMX,            /* sum_p X_p, X_p = sum s l_axis of particle p (nm)           */
  MCBTE_STAT_SUMX2,
  MCBTE_STAT_EVENTS,          /* emission + relaxations + boundary interactions           */
  MCBTE_STAT_TRUNCATED,       /* particles stopped by max_events or the time budget       */
  MCBTE_STAT_E_TOT,           /* W (steady) or J (transient): total deviational source     */
  MCBTE_STAT_MAX_EVENTS,      /* largest per-particle event count                         */
  MCBTE_STAT_KAPPA_CELL,      /* kappa normalised by the full cell volume                 */
  MCBTE_STAT_SIGNED_EMITTED,  /* sum of emitted signs                                     */
  MCBTE_STAT_SIGNED_ABSORBED, /* sum of signs absorbed at isothermal walls                */
  MCBTE_STAT_STATUS,          /* 0 ok, 4 timeout, 5 truncated, 7 gradient replay mismatch  */
  MCBTE_STAT_N,               /* particles traced                                         */
  MCBTE_STAT_ABSORBED,        /* particles absorbed at isothermal walls                   */
  MCBTE_NSTATS = 16
};

typedef struct {
  const uint64_t* n_particles; /* HOST [n_geoms], each in [1, 2^32)                      */
  uint64_t seed;               /* Philox key                                             */
  int precision;               /* MCBTE_FP64_PLAIN or MCBTE_FP32_TRACE                    */
  int n_scat_max;              /* terminate after this many relaxations; 0 = unlimited    */
  uint64_t max_events;         /* per-particle event guard (0 = 2^32-1)                   */
  int n_cells;                 /* cells of the 1-D track-length grid (0 = none)           */
  int cell_axis;               /* 0,1,2 */
  int tally_axis;              /* axis of q_mean, kappa, X_p and q_bin                    */
  int per_bin;                 /* 1: frequency-resolved flux q_bin                       */
  int threads_per_block;       /* 0 = default                                            */
  int blocks_per_sm;           /* 0 = default                                            */
  double time_budget_s;        /* 0 = 120 s; the kernel stops and reports TIMEOUT        */
  void* trace_event_start;     /* optional cudaEvent_t recorded on `stream` just before   */
  void* trace_event_stop;      /* and just after the tracing kernel (NULL = none)         */
  const uint64_t* seed_device; /* optional DEVICE pointer: if set, the tracing kernel reads
                                  the Philox key from it when it starts (a captured CUDA
                                  graph then draws a new sample per replay after the caller
                                  updates it); `seed` is ignored                          */
  int refill_threshold;        /* FP32 tracer: a warp refills its finished lanes once at
                                  least this many are idle (0 or 1 = at once, up to 32)   */
  int cell_flux_axis;          /* FP32 tracer, cell tallies: 0 = T and q_x, q_y, q_z;
                                  1 = T and the flux along tally_axis only (the other two
                                  components are returned as 0; Eq. flux_x_steady needs
                                  only that one)                                          */
  int n_regions;               /* steady detector regions (Sec. 4.5), 0..MCBTE_MAX_REGIONS,
                                  one geometry only; results in mcbte_steady_out.det       */
  const double* regions;       /* HOST [n_regions][6] xmin, xmax, ymin, ymax, zmin, zmax (m)  */
  const int* region_grid;      /* HOST [n_regions][3] detectors per axis (half-open cuboids
                                  [min, max), closed on the box's upper faces)              */
  int nscat_curve;             /* 1: also kappa for every N_scat_max' = 1..n_scat_max from the
                                  same trajectories (mcbte_steady_out.kappa_nscat); needs
                                  1 <= n_scat_max <= MCBTE_MAX_NSCAT_CURVE; not with mcbte_grad */
  int det_per_bin;             /* 1: the detector outputs per frequency bin (Sec. 4.5 lists the
                                  steady output of each detector per bin); needs n_regions > 0 */
  int tail_lanes;              /* FP32 tracer, tail of the run: once no particle is left to hand
                                  out, a warp with at most this many particles in flight draws
                                  the random words of their next events on all 32 lanes at once
                                  and then traces them (same results, shorter dependent chain
                                  per event); 0 = default (8), -1 = off, at most 32 */
  const uint64_t* pid_begin;   /* HOST [n_geoms] or NULL (0): this call traces particles
                                  pid_begin .. pid_begin + n_particles - 1 of each geometry's
                                  run (their own Philox streams, so a run split over calls or
                                  GPUs gives the particles of the whole run, Sec. 6)        */
  const uint64_t* n_total;     /* HOST [n_geoms] or NULL (n_particles): particles of each
                                  geometry's whole run; E_eff = E_tot / n_total scales this
                                  call's tallies, so the tallies of calls covering the run
                                  add up to the run's (kappa and q_mean too; standard errors
                                  combine through SUMX, SUMX2 and N)                          */
} mcbte_steady_params;

typedef struct {
  double* T;            /* [n_geoms][n_cells]     K, T - T_eq (Eq. temp_steady) or NULL  */
  double* q;            /* [n_geoms][n_cells][3]  W/m^2 (Eq. flux_x_steady) or NULL      */
  double* q_bin;        /* [n_geoms][n_bins]      W/m^2 per bin along tally_axis or NULL  */
  double* stats;        /* [n_geoms][MCBTE_NSTATS] (required)                            */
  uint32_t* events_pp;  /* [sum n_particles] per-particle event counts, or NULL          */
  double* X_pp;         /* [sum n_particles] per-particle X_p (nm), or NULL              */
  int on_host;          /* 0: device pointers, 1: host pointers                          */
  double* det;          /* [n_detectors][4] T - T_eq (K), q_x, q_y, q_z (W/m^2) per detector of
                           the regions (track length in each, Eqs. temp_steady, flux_x_steady),
                           detectors region by region, x fastest; with det_per_bin
                           [n_detectors][n_bins][4], the contribution of each bin; or NULL */
  double* kappa_nscat;  /* [n_geoms][n_scat_max][2] kappa (W/m/K) and its standard error with
                           N_scat_max' = k + 1 at index k (required with nscat_curve)       */
} mcbte_steady_out;

/* Device scratch a run needs.  Pass a buffer at least this large (256-byte
 * aligned) to the run, or NULL to let the run allocate (cudaMallocAsync on
 * `stream`) and free it. */
mcbte_status mcbte_steady_workspace_size(const mcbte_material* m, const mcbte_geometry* const* geoms,
                                         int n_geoms, const mcbte_steady_params* p, int want_grad,
                                         int n_dirs, size_t* bytes);

/* Steady-state run over n_geoms geometries (1..128) in one launch (the
 * steady estimator of Eq. steady_estimate with track-length tallies,
 * Eqs. temp_steady and flux_x_steady).  Particle k of geometry g draws from
 * Philox4x32-10 with counter (k, g, event, sub-block) and key = seed, so
 * results do not depend on the launch shape or on how a run is split.
 * With device outputs the call is asynchronous; its status lands in
 * stats[MCBTE_STAT_STATUS].  With host outputs it returns TIMEOUT /
 * TRUNCATED itself. */
mcbte_status mcbte_run_steady(const mcbte_material* m, const mcbte_geometry* const* geoms, int n_geoms,
                              const mcbte_steady_params* p, const mcbte_steady_out* out,
                              void* workspace, size_t workspace_bytes, mcbte_stream stream);

/* Steady run that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc (code
 * under an allocation-free contract, a fixed device-memory budget, or a
 * process that must not grow device memory after start-up).  Same inputs,
 * results and asynchronous behaviour as mcbte_run_steady with device
 * outputs, but the run's scratch is a fixed 8 MiB device array inside this
 * library, held on every GPU that loads it until the process exits.
 *   - out->on_host must be 0 (outputs are the caller's device buffers).
 *   - Runs needing more than 8 MiB of scratch (many geometries x bins x
 *     cells) return MCBTE_ERR_WORKSPACE with the size needed.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     With CUDA's lazy module loading that first call, or the first one that
 *     launches a given kernel variant, may load the library's device code,
 *     which itself takes device memory: make one call of each kind of run at
 *     start-up, after which calls allocate nothing.
 *   - Every call shares the one array, which keeps the last call's contents
 *     (each call clears what must start at zero): calls whose GPU work
 *     overlaps, on any streams or host threads, race and corrupt each
 *     other's results.  Serialise them. */
mcbte_status mcbte_run_steady_noalloc(const mcbte_material* m, const mcbte_geometry* const* geoms, int n_geoms,
                                      const mcbte_steady_params* p, const mcbte_steady_out* out,
                                      mcbte_stream stream);

typedef struct {
  uint64_t n_particles;        /* [1, 2^32) */
  uint64_t seed;
  int precision;
  uint64_t max_events;
  double t_max;                /* s, end of the simulated interval (Sec. 3.5.6)          */
  int n_times;                 /* measurement times (Sec. 3.4), 1..MCBTE_MAX_TIMES       */
  const double* t_meas;        /* HOST [n_times] s, ascending, in (0, t_max]             */
  int grid[3];                 /* nx, ny, nz detector cells over the box                 */
  int threads_per_block;        /* 0 (default 1024), 256, 512, 768 or 1024 (FP32 path)    */
  int blocks_per_sm;
  double time_budget_s;
  void* trace_event_start;     /* optional cudaEvent_t pair around the tracing kernel     */
  void* trace_event_stop;
  int window_times;            /* FP32 path: measurement times per time window; 0 picks the
                                  largest window whose tally slice fits a third of the L2;
                                  >= n_times traces in one pass (no state buffer)           */
  int n_regions;               /* detector regions (Sec. 4.5, Measure_region), 0..MCBTE_MAX_REGIONS;
                                  0: the whole box split by grid                            */
  const double* regions;       /* HOST [n_regions][6] xmin, xmax, ymin, ymax, zmin, zmax (m)  */
  const int* region_grid;      /* HOST [n_regions][3] detectors per axis (2^n for the paper's
                                  2^(3n) refinement); every region that contains a particle
                                  tallies it; regions are half-open [min, max), closed on the
                                  box's upper faces, so regions tiling the box partition it */
  int time_average;            /* 0: snapshots at each t_meas (Eq. sampling); 1: averages of T
                                  and q over [t_{m-1}, t_m) (t_0 = 0), from the time each flight
                                  spends in each detector                                  */
} mcbte_transient_params;


typedef struct {
  double* tally;        /* [n_times][n_detectors][4]: T - T_eq (K), q_x, q_y, q_z (W/m^2),
                           Eq. sampling; detectors region by region, x fastest (without
                           regions: [n_times][nz][ny][nx][4])                            */
  double* stats;        /* [MCBTE_NSTATS]                                                */
  uint32_t* events_pp;  /* [n_particles] or NULL                                         */
  int on_host;
} mcbte_transient_out;

mcbte_status mcbte_transient_workspace_size(const mcbte_material* m, const mcbte_geometry* g,
                                            const mcbte_transient_params* p, size_t* bytes);

/* Transient run (Sec. 3.2-3.5): wall sources emit at t0 = R t_max, the
 * initial condition at t0 = 0; at each t_meas inside a particle's life its
 * cell receives s E_eff / (C V_cell) and s E_eff V_g / V_cell (Eq. sampling).
 * Body sources are not allowed (MCBTE_ERR_INVALID_ARG). */
mcbte_status mcbte_run_transient(const mcbte_material* m, const mcbte_geometry* g,
                                 const mcbte_transient_params* p, const mcbte_transient_out* out,
                                 void* workspace, size_t workspace_bytes, mcbte_stream stream);

typedef struct {
  double* dkappa_dlogtau;  /* [n_bins] d kappa / d log tau_i                              */
  double* dkappa_dp;       /* [2] value and standard error of d kappa / d p_pore; NaN
                              when the geometry has no pore, or for the likelihood ratio
                              at p_pore = 0 or 1                                          */
  const double* dirs;      /* [n_dirs][n_bins] probe directions in log-tau space, or NULL */
  int n_dirs;              /* 0..16                                                        */
  double* dkappa_dir;      /* [n_dirs][2] value and SE of d kappa along each direction     */
  int on_host;             /* must equal the forward outputs' on_host                     */
  int dp_estimator;        /* d kappa / d p_pore: 0 = likelihood ratio for 0 < p_pore < 1,
                              measure-valued at p_pore = 0 or 1; 1 = likelihood ratio;
                              2 = measure-valued (any p_pore)                              */
} mcbte_grad_out;

/* Steady run of one geometry that also returns the likelihood-ratio
 * (score-function) gradient of kappa with respect to per-bin log tau scale
 * factors and the pore specularity.  The scores follow from the laws the
 * paper samples: the exponential relaxation distance of Eq. time_to_scat
 * (relaxation-ended flight: -1 + l / Lambda; censored flight: l / Lambda),
 * the resampling law ~ C/tau of Eq. n_scatt (-delta_ij + pi_j) and the
 * specular / diffuse draw of Sec. 3.5.3 (1/p, -1/(1-p)); each score
 * multiplies the tally still to come.  The paper itself has no gradient.
 * The measure-valued estimator of d kappa / d p_pore differentiates the
 * specular / diffuse draw itself (its weak derivative is the difference of
 * the two branches): of a particle's K pore hits one is chosen uniformly (hit
 * j replaces the choice when the 64-bit word of Philox sub-block 257 of its
 * event is at most floor((2^64 - 1) / j)), the particle is traced a second
 * time from its emission with the same random words and that hit's branch
 * flipped, and its score is K (X with the hit specular - X with it diffuse).
 * It stays valid at p_pore = 0 and 1, where the likelihood-ratio score does
 * not; the second traces add to the run time, not to the tallies.
 * FP64_PLAIN keeps each particle's relaxation periods and requires
 * 1 <= n_scat_max <= 64.  FP32_TRACE requires n_scat_max >= 1.  With
 * n_scat_max <= 16, no cells (n_cells = 0) and no detector regions it runs
 * one pass: the forward tallies and the gradient together, each particle
 * listing its relaxation periods' score sums until its final tally is known.
 * Otherwise it runs two passes: the forward run, which records every
 * particle's final tally, then a pass that replays the same particles (same
 * random words) and adds each period's term as it closes; that needs 8 more
 * workspace bytes per particle, and returns MCBTE_ERR_REPLAY in the status
 * statistic should a replayed tally differ from the recorded one. */
mcbte_status mcbte_grad(const mcbte_material* m, const mcbte_geometry* g, const mcbte_steady_params* p,
                        const mcbte_steady_out* fwd, const mcbte_grad_out* grad,
                        void* workspace, size_t workspace_bytes, mcbte_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MCBTE_H */
