/*
 * lbm.h -- C ABI of the GB300 pseudopotential (Shan-Chen) D2Q9 lattice
 * Boltzmann library.
 *
 * The method is the one of Li, Luo & Li, "Forcing scheme in pseudopotential
 * lattice Boltzmann model for multiphase flows": one time step is
 *   (1) streaming of Eq. 1 (pull form: f_a(x, t) = f*_a(x - e_a, t - 1)),
 *   (2) the moments rho = sum f_a, u = sum f_a e_a / rho (Sec. III A),
 *   (3) the potential psi(rho) of Eq. 8 with the Carnahan-Starling p_EOS of
 *       Eq. 23 (a, b, R; c = 1, delta_t = 1, G < 0),
 *   (4) the interaction force of Eq. 3 with w(1) = 1/3, w(2) = 1/12,
 *   (5) BGK collision (Eqs. 1-2) with the chosen forcing scheme (or, for
 *       LBM_SCHEME_MRT, the multiple-relaxation-time form of the improved
 *       scheme).
 * All of it runs in one fused CUDA kernel per step; the host only validates
 * arguments, launches, and copies data in and out.
 *
 * Lattice: D2Q9, e0 = (0,0); e1..e4 = (1,0), (0,1), (-1,0), (0,-1);
 * e5..e8 = (1,1), (-1,1), (-1,-1), (1,-1).  Host arrays are row-major
 * [ny][nx] (x fastest); population arrays are [9][ny][nx].  The domain is
 * periodic in x and y.
 *
 * Memory: a context owns every device allocation it makes (two population
 * buffers, plus a density plane for 16-bit storage, plus small scratch);
 * host pointers passed in are only read or written during the call.
 *
 * Errors: every function returns an lbm_status; on failure the context (if
 * any) records a message readable with lbm_last_error().  No function
 * aborts the process.  Threading: one context must not be used by two host
 * threads at once; distinct contexts may share a device.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_E_INVAL = 1,    /* bad argument (size, scheme, tau, null pointer, ...) */
  LBM_E_NOMEM = 2,    /* device or host allocation failed                  */
  LBM_E_CUDA = 3,     /* a CUDA runtime call failed                         */
  LBM_E_DIVERGED = 4, /* density left the domain of psi (rho <= 0, b rho/4 >= 1,
                         negative radicand in Eq. 8) or became non-finite    */
  LBM_E_TIMEOUT = 5,  /* a bounded device-side wait gave up                 */
  LBM_E_STATE = 6     /* call out of order (e.g. step before init)           */
} lbm_status;

/* Forcing schemes (Table I of the paper). */
enum {
  LBM_SCHEME_SC = 0,       /* Shan-Chen velocity shift: BGK towards
                              f_eq(rho, u + tau F / rho), Eqs. 9-10          */
  LBM_SCHEME_EDM = 1,      /* exact difference method:
                              F_a = f_eq(rho, u + F/rho) - f_eq(rho, u), Eq. 11 */
  LBM_SCHEME_IMPROVED = 2, /* improved scheme, Eq. 31: Guo forcing with
                              v' = v + sigma F / ((tau - 1/2) psi^2);
                              sigma = 0 is Guo's scheme (Eqs. 12-13)         */
  LBM_SCHEME_NOFORCE = 3,  /* F = 0: plain BGK (force-free checks)           */
  LBM_SCHEME_EDM_MOD = 4,  /* EDM with C_e = 1/tau (Sec. III C)             */
  LBM_SCHEME_LADD = 5,     /* Ladd: u in f_eq and in F_a, B_e = C_e = 1
                              (Table I)                                      */
  LBM_SCHEME_MRT = 6       /* the improved scheme in multiple-relaxation-time
                              form (the extension stated at the end of
                              Sec. IV; the paper gives no formula, see
                              lbm_set_mrt_rates): D2Q9 moments relax at their
                              own rates towards f_eq(rho, v), with the improved
                              forcing term's moments (v') added at (1 - s/2);
                              single lattices only, not lbm_batch_*          */
};

/* Storage precision of the populations. */
enum {
  LBM_FP32 = 0,    /* float populations, float arithmetic                   */
  LBM_FP64 = 1,    /* double populations, double arithmetic                 */
  LBM_BF16DEV = 2, /* bf16 deviations d_a = f_a - w_a rho plus a float rho
                      plane; float arithmetic                                */
  LBM_FP16DEV = 3  /* as LBM_BF16DEV with IEEE half deviations               */
};

typedef struct {
  int nx, ny;          /* lattice size, each >= 1                            */
  double T_over_Tc;    /* reduced temperature, > 0                           */
  int tc_mode;         /* 0: exact critical temperature of Eq. 23;
                          1: the rounded Tc = 0.094 printed with Eq. 23      */
  double a, b, R, G;   /* Eq. 23 / Eq. 8 constants; the paper's values are
                          a = 1, b = 4, R = 1, G = -1 (G must be < 0)         */
  int precision;       /* LBM_FP32, LBM_FP64, LBM_BF16DEV, LBM_FP16DEV       */
  int device;          /* CUDA device ordinal                                 */
  void *cuda_stream;   /* cudaStream_t to run on, or NULL for a stream the
                          context creates and owns                           */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Fill p with the paper's defaults: a = 1, b = 4, R = 1, G = -1, exact Tc,
 * FP32, device 0, own stream; nx, ny and T_over_Tc are set to 0. */
void lbm_default_params(lbm_params *p);

/* Allocate a lattice.  Errors: LBM_E_INVAL for nx or ny < 1, T_over_Tc <= 0,
 * G >= 0, b <= 0, unknown precision or tc_mode; LBM_E_NOMEM; LBM_E_CUDA.
 * On success *out owns the context (free it with lbm_destroy). */
lbm_status lbm_create(const lbm_params *p, lbm_ctx **out);

/* ---- domain decomposition in y (one band of rows per rank) ----------------
 * A band context holds p->ny >= 2 rows of a larger lattice that is periodic
 * in y, as one rank's share of a decomposition in y-slabs.  One time step of
 * a row reads the post-collision populations of the rows one above and one
 * below it (the pull of Eq. 1), and its force (Eq. 3) the density of those
 * rows, which needs their pulls from the rows beyond: a band therefore keeps
 * two ghost rows below and two above its own rows, refreshed between steps
 * from the neighbouring bands' two boundary rows (all 9 populations, and for
 * deviation storage the density plane).  Periodicity in y is that exchange
 * (the band below rank 0 is the last rank's); x stays periodic in the band.
 *   - lbm_init_density / lbm_init_density_at_rest take (p->ny + 4) x nx
 *     densities: the band's rows with the two global rows below and above
 *     them (wrapped).  The owned rows are then exact; the ghost rows' own
 *     pulls (and, for deviation storage, the density their deviations refer
 *     to) reach beyond the given rows, so exchange halos once after the
 *     initialisation, before the first step;
 *   - lbm_step / lbm_step_async advance one step per call (n <= 1; larger n
 *     is LBM_E_INVAL); between calls the caller exchanges halos:
 *     lbm_band_halo_pack, send / receive, lbm_band_halo_unpack;
 *   - lbm_get_moments, lbm_get_mass and lbm_get_populations report the
 *     owned rows only ([ny][nx], [9][ny][nx]); lbm_set_populations is
 *     LBM_E_INVAL on a band.
 * Each owned row evaluates exactly what the same row of the whole lattice
 * does, so a decomposed run is bit-identical to an undecomposed one. */
lbm_status lbm_create_band(const lbm_params *p, lbm_ctx **out);

/* Bytes of one halo message of a band: 2 rows x nx x (9 populations of the
 * storage type + 4 bytes of density plane for deviation storage).
 * LBM_E_STATE for a context that is not a band. */
lbm_status lbm_band_halo_bytes(const lbm_ctx *ctx, size_t *bytes);

/* Queue on the context stream the copies of the band's two lowest owned rows
 * into d_lo and its two highest into d_hi (caller-owned device buffers of
 * lbm_band_halo_bytes each; layout [9][2][nx] populations then [2][nx]
 * density plane): the messages for the band below and the band above.
 * Returns without waiting. */
lbm_status lbm_band_halo_pack(lbm_ctx *ctx, void *d_lo, void *d_hi);

/* Queue the copies of the received messages into the ghost rows: d_below is
 * the band below's d_hi, d_above the band above's d_lo.  Returns without
 * waiting; the next step on the context stream reads them. */
lbm_status lbm_band_halo_unpack(lbm_ctx *ctx, const void *d_below, const void *d_above);

/* One step of a band with its halo exchange overlapped with the interior:
 * queues on the context stream the step of the two lowest and the two
 * highest owned rows, their copies into d_lo and d_hi (as
 * lbm_band_halo_pack), an event that comm_stream (a CUDA stream of the
 * caller, may be NULL) is made to wait for, and then the step of the
 * interior rows.  The caller sends d_lo / d_hi and receives the neighbours'
 * on comm_stream, makes the context stream wait for that, and unpacks
 * (lbm_band_halo_unpack) before the next step.  Bands of fewer than 5 rows
 * compute all rows before packing.  Same results as lbm_step + pack: the
 * rows are the same computations, only their order differs.  Returns
 * without waiting; the errors of lbm_step_async and lbm_band_halo_pack. */
lbm_status lbm_band_step_overlap(lbm_ctx *ctx, int scheme, double tau, double sigma,
                                 void *d_lo, void *d_hi, void *comm_stream);

/* Set the state to f_a = f_eq(rho, u) (Eq. 2) at every cell.  rho is a host
 * array of ny*nx doubles; ux and uy may be NULL (zero velocity).  Copied to
 * the device during the call.  LBM_E_INVAL if any rho is outside the domain
 * of psi (rho <= 0, b rho / 4 >= 1 or a negative radicand in Eq. 8). */
lbm_status lbm_init_density(lbm_ctx *ctx, const double *rho, const double *ux,
                            const double *uy);

/* The same density at rest: f_a = f_eq(rho, u) (Eq. 2) with u = -F / (2 rho),
 * F the interaction force of Eq. 3 evaluated (in FP64, on the device) on rho
 * itself, so that the actual fluid velocity v = u + F / (2 rho) of Table I is
 * zero at every cell.  Starting a smooth profile (Eq. 24 droplet, Eq. 36
 * slab) from u = 0 instead gives its interfaces the velocity F / (2 rho) and
 * an initial transient.  rho as for lbm_init_density (host, ny*nx doubles,
 * copied); the same errors. */
lbm_status lbm_init_density_at_rest(lbm_ctx *ctx, const double *rho);

/* Advance n >= 0 time steps with the given scheme and relaxation time
 * tau > 1/2 (sigma is read by LBM_SCHEME_IMPROVED only).  Kernels are queued
 * on the context stream, one per step; on lattices of at most 2048^2 cells
 * runs of 16 steps go through a CUDA graph of 16 step kernels, captured on
 * first use for the current buffer and launch arguments and kept until the
 * context is destroyed (bit-identical to single launches); while the caller
 * captures the context stream into a graph of its own, lbm_step_async records
 * one launch per step instead.  The call then waits for the kernels and
 * reads the device status word once (so lbm_step itself cannot be
 * captured).  LBM_E_DIVERGED if psi became undefined in any step (the state
 * is then unspecified but the context stays usable and destroyable);
 * LBM_E_STATE before lbm_init_density / lbm_set_populations. */
lbm_status lbm_step(lbm_ctx *ctx, int n, int scheme, double tau, double sigma);

/* Queue n steps without waiting and without reading the status (for timing
 * and graph capture); lbm_sync_status() later waits and reports. */
lbm_status lbm_step_async(lbm_ctx *ctx, int n, int scheme, double tau,
                          double sigma);
lbm_status lbm_sync_status(lbm_ctx *ctx);

/* Density and the actual fluid velocity v = u + F / (2 rho) (Table I, every
 * scheme) of the current state, as host FP64 arrays of ny*nx; any pointer
 * may be NULL.  F = 0 (and psi is not evaluated) when the most recent
 * lbm_step used LBM_SCHEME_NOFORCE.  LBM_E_DIVERGED if psi is undefined.
 * The values go through device staging and DMA copies; from 2048^2 cells
 * on, rows are computed and copied in four chunks, each copied while the
 * next is computed (page-locked outputs, e.g. from lbm_host_alloc, let the
 * copies run asynchronously at the link rate). */
lbm_status lbm_get_moments(lbm_ctx *ctx, double *rho, double *vx, double *vy);

/* Total mass sum_x rho(x), reduced on the device in FP64. */
lbm_status lbm_get_mass(lbm_ctx *ctx, double *mass);

/* Checkpoint: copy the populations f_a(x, t) of the current state to / from
 * a host FP64 array [9][ny][nx].  For 16-bit storage lbm_set_populations
 * rounds the deviations to 16 bits. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f);

/* Reduced temperature -> absolute temperature used by the context. */
lbm_status lbm_get_temperature(const lbm_ctx *ctx, double *T);

/* Human-readable message of the last failure on ctx ("" if none); with a
 * NULL ctx, the last failure of lbm_create on this thread. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Free every resource of ctx.  Accepts NULL. */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* ---- host-side equation-of-state helpers (no GPU needed) -------------- */

/* Exact critical point of Eq. 23: dp/drho = d^2p/drho^2 = 0. */
lbm_status lbm_cs_critical_point(double a, double b, double R, double *rho_c,
                                 double *T_c, double *p_c);

/* Maxwell equal-area coexistence densities (Eq. 7) of Eq. 23 at absolute
 * temperature T (0 < T < T_c).  LBM_E_INVAL outside that range. */
lbm_status lbm_cs_maxwell(double T, double a, double b, double R,
                          double *rho_g, double *rho_l, double *p0);

/* Number of kernel launches this process has queued through the library
 * (all contexts), for accounting in benchmarks. */
unsigned long long lbm_kernel_launch_count(void);

/* ---- launch tuning ------------------------------------------------------ */

/* Step kernel variant; all give bit-identical results.  REGISTER: one column
 * per lane, rows loaded into registers one row ahead.  PAIR: two adjacent
 * columns per lane (vector loads and stores of two populations), for even
 * nx.  STAGED: one column per lane, rows brought into shared
 * memory by asynchronous bulk copies several rows ahead (FP32 steps with
 * nx % 4 == 0 and nx >= 64; a bounded wait that gives up makes lbm_step
 * return LBM_E_TIMEOUT).  AUTO (default) = PAIR for even nx except with FP64
 * storage or on lattices too small for its 64-column strips to occupy the
 * GPU (about 512 x 512 and below), else REGISTER.  A variant that does not
 * apply falls back to REGISTER. */
enum { LBM_VARIANT_AUTO = 0, LBM_VARIANT_REGISTER = 1, LBM_VARIANT_STAGED = 2,
       LBM_VARIANT_PAIR = 3 };
lbm_status lbm_set_kernel_variant(lbm_ctx *ctx, int variant);

/* Relaxation rates of LBM_SCHEME_MRT for the energy, energy-square and
 * energy-flux moments (Lallemand-Luo D2Q9 basis); the stresses relax at
 * 1/tau, and a rate <= 0 (the default) means 1/tau, which makes the scheme
 * identical to LBM_SCHEME_IMPROVED (up to rounding).  Rates must be < 2.
 * Applies to later lbm_step calls. */
lbm_status lbm_set_mrt_rates(lbm_ctx *ctx, double s_e, double s_eps, double s_q);

/* Rows per warp band of the step kernel (0 = automatic: one wave of warps,
 * at least 4 rows each).  Changes only speed, never results. */
lbm_status lbm_set_band_rows(lbm_ctx *ctx, int band_rows);

/* The launch geometry lbm_step would use for `scheme`: column strips (32
 * columns wide, 64 with the PAIR variant), rows per band, bands, and CTAs of
 * 128 threads. */
lbm_status lbm_get_launch_geometry(lbm_ctx *ctx, int scheme, int *n_strips,
                                   int *band_rows, int *n_bands, int *grid);

/* The kernel variant lbm_step resolves to (REGISTER, STAGED or PAIR) for the
 * context's storage type, lattice width and requested variant. */
lbm_status lbm_get_kernel_variant(lbm_ctx *ctx, int *variant);

/* ---- batched parameter sweeps ------------------------------------------- */
/*
 * Many independent lattices (instances) with their own size, temperature,
 * tau, sigma and forcing scheme, advanced together in FP32 until each one
 * converges, diverges or reaches a step cap.  Each instance is the method of
 * lbm_step (the same fused kernel body); the batch packs all populations in
 * one buffer pair and runs windows of `window` steps as one CUDA graph:
 * WORKLIST: one launch per step and instance class (two columns per lane
 * for even nx, one for odd nx) over a work list of the active instances'
 * strip x band items; PERSISTENT: one launch per window in which each CTA
 * owns whole instances and synchronises only its own threads between steps;
 * COOPERATIVE: one cooperative launch per window (every CTA resident) whose
 * warps take the work-list items of each step and meet at a bounded grid
 * barrier between steps (LBM_E_TIMEOUT if it ever gives up).  AUTO times the
 * candidates on live windows and keeps the fastest.  After every window an FP64 reduction per instance gives the
 * coexistence densities of the flat interface (Eq. 36 slab: rho_g from rows
 * 0 and ny-1, rho_l from rows ny/2-1 and ny/2), the interface width
 * (rho_l - rho_g) / max_y |d rho_row / dy|, the mass, and the largest density
 * change since the previous window.  When an instance has converged is set
 * by the convergence rule (conv, below: COEX by default).
 */

typedef struct {
  int nx, ny;        /* lattice of this instance, each >= 1                  */
  double T_over_Tc;  /* reduced temperature, > 0                             */
  double tau;        /* relaxation time, > 1/2                               */
  double sigma;      /* improved-scheme constant (read by scheme 2 only)     */
  int scheme;        /* LBM_SCHEME_SC .. LBM_SCHEME_LADD (no MRT in batches)  */
} lbm_instance;

/* Launch modes of a window.  WORKLIST: per step and instance class, one
 * launch whose warps take strip x band items in a fixed round-robin;
 * WORKLIST_DYNAMIC: the same items handed out one at a time from a per-step
 * counter (a warp that finishes early takes more); PERSISTENT: one launch per
 * window and class, each CTA owning whole instances; COOPERATIVE: one
 * cooperative launch per window with a bounded grid barrier between steps;
 * BALANCED: per step and class, one wave of resident warps, each taking an
 * equal share of all the class's rows (the rows of every strip laid end to
 * end and cut into equal pieces, at least 8 rows each; rows_per_item does
 * not apply).  AUTO times the candidates on live windows and keeps the
 * fastest.  Every mode gives the same results bit for bit. */
enum { LBM_BATCH_AUTO = 0, LBM_BATCH_WORKLIST = 1, LBM_BATCH_PERSISTENT = 2,
       LBM_BATCH_COOPERATIVE = 3, LBM_BATCH_WORKLIST_DYNAMIC = 4, LBM_BATCH_BALANCED = 5 };
/* Convergence rules.  CELL: every cell changed by less than
 * max(tol, 8 * 2^-23 * rho) over a window.  COEX: the coexistence densities
 * rho_g and rho_l (FP64 row means) each changed by less than
 * max(tol, conv_rel * value) over two consecutive windows.  In FP32 the
 * interface position of a relaxed slab jitters by ~1e-4 cells per window
 * (rounding noise driving a nearly neutral mode), so CELL is met only by
 * some runs; COEX tests what a sweep reports.  TREND: from the ninth window
 * after a (re)start, each coexistence density is settled within
 * max(tol, trend_tol * value): over its last nine window values, the range
 * of the last six (a slab's standing sound wave has a period of a few
 * windows, so the range bounds its amplitude) and the extrapolated drift of
 * the means of three blocks of three windows (two block changes of one sign,
 * the later smaller, are a geometric decay with ratio r = d / d_prev and
 * remaining distance |d| r / (1 - r); any other pair is noise of amplitude
 * |d| + |d_prev|) are both within it.  COEX's floor sits at FP32 rounding
 * noise, which keeps a settled slab running for tens of thousands of steps;
 * TREND stops it once the answer is known to trend_tol, while a slow
 * monotone drift (r near 1) or a live sound wave keeps it running.  The
 * paper has no convergence test; this one serves the sweeps (steps to
 * convergence, warm against cold starts). */
enum { LBM_CONV_COEX = 0, LBM_CONV_CELL = 1, LBM_CONV_NONE = 2 /* run to max_steps */,
       LBM_CONV_TREND = 3 };
enum { LBM_RUN_ACTIVE = 0, LBM_RUN_CONVERGED = 1, LBM_RUN_DIVERGED = 2, LBM_RUN_CAPPED = 3 };

typedef struct {
  int tc_mode;          /* as in lbm_params                                    */
  double a, b, R, G;    /* as in lbm_params                                    */
  int device;
  void *cuda_stream;    /* NULL: the batch creates and owns a stream          */
  int window;           /* steps per convergence check, even, >= 2 (1000)      */
  double tol;           /* density-change tolerance per window (1e-9)          */
  int max_steps;        /* step cap per instance (200000)                      */
  int mode;             /* LBM_BATCH_AUTO (window-level autotuning), _WORKLIST,
                           _WORKLIST_DYNAMIC, _PERSISTENT, _COOPERATIVE,
                           _BALANCED                                           */
  int rows_per_item;    /* band height of a work-list item; 0 = autotuned      */
  int conv;             /* LBM_CONV_COEX (default), _CELL, _NONE or _TREND      */
  int variant;          /* LBM_VARIANT_AUTO (default) or _PAIR: two columns per
                           lane for even nx; _REGISTER: one column per lane for
                           every instance.  Results are identical.             */
  double conv_rel;      /* COEX: relative floor, changes below
                           max(tol, conv_rel * value) count as calm (8 * 2^-23
                           by default; must be >= 0)                           */
  double trend_tol;     /* TREND: relative bound on the estimated distance of
                           rho_g, rho_l to their limits (1e-4; >= 0)           */
} lbm_batch_params;

typedef struct {
  int status;           /* LBM_RUN_*                                          */
  int steps;            /* steps advanced                                     */
  double rho_g, rho_l;  /* slab coexistence densities (FP64 row means)        */
  double width;         /* interface width                                    */
  double mass;          /* total mass (FP64)                                  */
  double max_drho;      /* largest |rho(t) - rho(t - window)| of the last window */
} lbm_result;

typedef struct {
  int windows;                 /* windows run so far                          */
  unsigned long long launches; /* kernel launches queued                      */
  double gpu_ms;               /* device time of all windows (CUDA events)    */
  int mode;                    /* mode of the last window                      */
  int rows_per_item;           /* work-list band height of the last window     */
  int n_active;                /* instances still running                      */
} lbm_batch_stats;

typedef struct lbm_batch lbm_batch;

/* Fill *p with the defaults named above (a = 1, b = 4, R = 1, G = -1, exact
 * Tc, window 1000, tol 1e-9, max_steps 200000, AUTO mode, COEX rule,
 * conv_rel 8 * 2^-23, trend_tol 1e-4, AUTO variant, device 0, own stream).
 * NULL is ignored. */
void lbm_batch_default_params(lbm_batch_params *p);

/* Allocate a batch of `count` instances.  LBM_E_INVAL for count < 1 or any
 * instance with a bad size, temperature, tau or scheme. */
lbm_status lbm_batch_create(const lbm_batch_params *p, const lbm_instance *inst,
                            int count, lbm_batch **out);

/* Instance i starts at rest from the host density rho (ny*nx doubles,
 * copied); LBM_E_INVAL if it leaves the domain of psi.  Called on an instance
 * that has run, it restarts it from rho (active again, convergence history
 * cleared) while its step count keeps the steps already spent. */
lbm_status lbm_batch_init_density(lbm_batch *b, int i, const double *rho);

/* The same with instance i at zero actual velocity: f = f_eq(rho, u), u =
 * -F / (2 rho) from the Eq. 3 force on rho (Table I; see
 * lbm_init_density_at_rest).  Same arguments, errors and restart rule. */
lbm_status lbm_batch_init_density_at_rest(lbm_batch *b, int i, const double *rho);

/* Every instance starts (all results reset) at rest from the flat-interface
 * profile of Eq. 36 built on the device: rho_g + (rho_l - rho_g)/2
 * [tanh(2(y - ny/4)/W) - tanh(2(y - 3ny/4)/W)] with the per-instance rho_g[i],
 * rho_l[i], W = width[i] (width[i] <= 0: a sharp step, liquid on rows
 * [ny/4, 3ny/4)).  At rest: for W > 0, zero actual velocity
 * v = u + F/(2 rho) (Table I), i.e. f = f_eq(rho, u) with u = -F/(2 rho) from
 * the Eq. 3 force of the initial profile; for the sharp step (and
 * LBM_SCHEME_NOFORCE instances) u = 0. */
lbm_status lbm_batch_init_slabs(lbm_batch *b, const double *rho_g, const double *rho_l,
                                const double *width);

/* Run at most max_windows windows (or until no instance is active); the
 * number still active is written to *n_active (may be NULL). */
lbm_status lbm_batch_run(lbm_batch *b, int max_windows, int *n_active);

/* Copy instance i's result (status, steps, and the observables of its last
 * window) to *r.  Host only (no device work); LBM_E_INVAL for a NULL argument
 * or i outside [0, count). */
lbm_status lbm_batch_get_result(const lbm_batch *b, int i, lbm_result *r);

/* Density of instance i (FP64 host array of ny*nx). */
lbm_status lbm_batch_get_density(lbm_batch *b, int i, double *rho);

/* Density and actual velocity v = u + F/(2 rho) (Table I, every scheme) of
 * instance i, as lbm_get_moments: caller-owned FP64 host arrays of ny*nx,
 * each may be NULL. */
lbm_status lbm_batch_get_moments(lbm_batch *b, int i, double *rho, double *vx, double *vy);

/* Copy the batch's counters (windows, launches, device time, the launch mode
 * of the last window, instances still active) to *s.  Host only;
 * LBM_E_INVAL for a NULL argument. */
lbm_status lbm_batch_get_stats(const lbm_batch *b, lbm_batch_stats *s);

/* Message of the batch's last failed call ("" for NULL or none); owned by
 * the batch, valid until its next call. */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Wait for the batch's stream, then free every device and pinned host
 * buffer, graph, event and owned stream.  Accepts NULL. */
lbm_status lbm_batch_destroy(lbm_batch *b);

/* ---- warm-start network ------------------------------------------------- */
/*
 * A 4 -> 64 -> 64 -> 3 MLP with tanh hidden layers, y = tanh(tanh(x W1 + b1)
 * W2 + b2) W3 + b3, trained on the mean squared error with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  The paper has no network: it maps a
 * sweep point (T/Tc, tau, sigma, scheme, scaled by the caller) to the
 * relaxed slab's (rho_l, log rho_g, width) (standardised by the caller) to
 * start new runs near their answer.  Parameters are one flat FP32 vector
 * W1[4][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3] (row-major,
 * lbm_mlp_num_params() = 4675 values).  X is [n][4], Y is [n][3], host FP32.
 */
typedef struct lbm_mlp lbm_mlp;

/* Number of FP32 parameters of the network (4675). */
int lbm_mlp_num_params(void);

/* Network on `device` with all parameters and Adam moments zero; it works on
 * cuda_stream (NULL: it creates and owns a stream).  LBM_E_INVAL for a NULL
 * out, LBM_E_CUDA for a bad device or stream failure, LBM_E_NOMEM when its
 * device buffers cannot be allocated (nothing is left allocated then). */
lbm_status lbm_mlp_create(int device, void *cuda_stream, lbm_mlp **out);

/* Wait for the network's stream and free its buffers (and owned stream).
 * Accepts NULL. */
lbm_status lbm_mlp_destroy(lbm_mlp *m);

/* Message of the network's last failed call ("" for NULL or none). */
const char *lbm_mlp_last_error(const lbm_mlp *m);

/* Set the parameters (and reset the Adam state) / read them back. */
lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *params);
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *params);

/* Gradient of the loss over the n <= 128 samples (no update); *loss may be
 * NULL. */
lbm_status lbm_mlp_gradient(lbm_mlp *m, const float *X, const float *Y, int n,
                            float *grad, float *loss);

/* Adam over `epochs` epochs; order holds epochs x n sample indices (the
 * caller's shuffles, so runs are reproducible), minibatch k of epoch e is
 * order[e*n + k*batch ...] (1 <= batch <= 128, a short last batch is used as
 * is).  One kernel launch trains all epochs.  *final_loss (nullable) gets the
 * last minibatch's loss. */
lbm_status lbm_mlp_train(lbm_mlp *m, const float *X, const float *Y, int n,
                         const int *order, int epochs, int batch, float lr,
                         float *final_loss);

/* Y = network(X) for n samples. */
lbm_status lbm_mlp_predict(lbm_mlp *m, const float *X, int n, float *Y);

/* ---- self-test of the bounded device waits -------------------------------- */
/* One warp on `device` waits, `polls` times (1 .. 2^20), on a shared-memory
 * mbarrier that nothing arrives on, gives up, records the timeout in a
 * device status word and returns -- the path the staged step kernel takes
 * when its bulk copies do not land.  *result receives LBM_E_TIMEOUT when the
 * wait gave up (expected) or LBM_OK.  Returns LBM_E_INVAL for bad arguments
 * (checked before any CUDA call), LBM_E_CUDA / LBM_E_NOMEM on CUDA errors.
 * Nothing faults or hangs; the context stays usable.  The paper has no
 * counterpart. */
lbm_status lbm_selftest_wait_timeout(int device, long long polls, int *result);

/* The same for the grid barrier of the batch engine's cooperative windows:
 * a cooperative launch of 4 CTAs in which CTA 0 never arrives; the other
 * three give up after the barrier's spin limit (well under a few seconds),
 * record the timeout and return.  *result receives LBM_E_TIMEOUT (expected)
 * or LBM_OK.  LBM_E_INVAL for a NULL result, LBM_E_CUDA when the device has
 * no cooperative launch or a CUDA call fails.  The paper has no
 * counterpart. */
lbm_status lbm_selftest_grid_barrier_timeout(int device, int *result);

/* ---- allocation-free variant ------------------------------------------- */

/* FP64 sum of n FP32 values in device memory (for an FP32 population buffer
 * [9][ny][nx]: its total mass), written to the caller's device slot *d_out.
 * The paper has no counterpart: this is a deployment helper for callers that
 * cannot call cudaMalloc -- code whose device memory belongs to another
 * allocator (a framework's caching pool, a fixed budget) or that must not
 * block on an allocation.  It allocates nothing: its partial sums live in a
 * fixed 8 KB file-scope device array (1024 doubles, one per block), held by
 * every GPU that loads the library until exit.  n may be at most 2^30; larger
 * n returns LBM_E_INVAL, as do NULL pointers (n = 0 writes 0).  The blocks
 * and their value ranges depend only on n, so the result is reproducible.
 * The first call on a device (the one current when called) looks up the
 * array's device address and keeps it for the life of the process; make
 * that first call before any stream capture, and do not reset
 * (cudaDeviceReset) a device this entry point has been used on -- the kept
 * address would be stale.  Kernels are queued on cuda_stream (NULL: the
 * legacy default stream) and the call returns without waiting.  Every call
 * on a device shares the array and overwrites what it uses (nothing needs
 * clearing), so calls whose kernels overlap on the GPU race: order them on
 * one stream. */
lbm_status lbm_mass_f32_noalloc(const float *d_values, size_t n, double *d_out,
                                void *cuda_stream);

/* ---- page-locked host buffers ------------------------------------------ */

/* Host memory for the arrays passed to lbm_init_density, lbm_get_moments,
 * lbm_get/set_populations and their batch counterparts, which DMA copies
 * move at the rate of the CPU-GPU link.  *out receives at least `bytes` of
 * zeroed, page-locked memory: an anonymous mapping registered with the CUDA
 * driver (cudaHostRegister); from one transparent huge page up (2 MiB with
 * 4 KiB base pages, 512 MiB with 64 KiB ones) it is aligned to and rounded
 * up to whole huge pages and advised for them (MADV_HUGEPAGE, used where the
 * kernel provides them).  Buffers from
 * cudaHostAlloc work as well; on a virtualised host whose memory had been
 * used and released by an earlier job, 537 MB copies into them were measured
 * 5-8x slower than the link rate, while copies into these buffers stayed at
 * it.  The paper has no counterpart: a deployment helper.  Errors:
 * LBM_E_INVAL for a NULL out or bytes = 0, LBM_E_NOMEM when the mapping
 * fails, LBM_E_CUDA when the registration fails (nothing is then held).
 * Thread-safe. */
lbm_status lbm_host_alloc(size_t bytes, void **out);

/* Unregister and unmap a buffer from lbm_host_alloc.  NULL is accepted;
 * LBM_E_INVAL for any other pointer that lbm_host_alloc did not return. */
lbm_status lbm_host_free(void *p);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
