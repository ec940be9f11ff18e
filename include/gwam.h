/*
 * gwam.h -- C ABI of the GB300 (sm_103a) MS-GWaM-3D gravity-wave ray-volume tracer.
 *
 * The library advances a population of gravity-wave ray volumes through a gridded
 * background and returns the wave drag on that grid, following Voelker et al.,
 * "MS-GWaM: A 3-dimensional transient gravity wave parametrization for atmospheric
 * models" (arXiv:2309.11257):
 *   Sec. 2a  Eq. dispersion, Eq. eikonal, Eq. group-velocity, Eq. eikonal-sphere:1-3
 *            (ray equations with the scale-height correction and spherical metric terms)
 *   Sec. 2b  Eq. mean-flow-impact, Eq. fluxes:momentum, Eq. fluxes:buoyancy (drag)
 *   Sec. 3a  ray volumes and the per-axis phase-space products (Eq. vpvol_cons_cart)
 *   Sec. 3b  coupling to the grid: interpolation and flux projection
 *   Sec. 3c  background source, saturation (Eq. instability-threshold, Eq. turbulent-diffusivity)
 *   App. B   interpolation, parent-cell storage and RK3, splitting, smoothing, ray caps
 *
 * Conventions
 *   - Every call returns a gwam_status (0 = GWAM_OK); nothing throws or exits.
 *   - Grid fields are C-order [nz][ny][nx] doubles (level 0 at the bottom, the
 *     vertical-flux fields [nz+1][ny][nx]).  Sphere: lambda in [0, 2 pi) with
 *     column i centred at (i + 1/2) 2pi/nx, phi in [-pi/2, pi/2] with row j centred
 *     at -pi/2 + (j + 1/2) pi/ny.  f-plane: doubly periodic, x = (i + 1/2) dx.
 *     Levels: z in [0, nz dz), level k centred at (k + 1/2) dz.  Units are SI,
 *     angles in radians.
 *   - Cell index of a ray volume: cell = (j * nx + i) * nz + k (column-major), the
 *     canonical ray order is ascending (cell, id).
 *   - Pointers without a _host suffix on the function are DEVICE pointers on the
 *     context's device; _host functions take host memory.  The library never frees
 *     or retains caller memory beyond the call.
 *   - All device work is enqueued on the stream given to gwam_init; calls that
 *     return host data synchronise that stream.
 *   - The context owns its device state (ray volumes, background, grid fields,
 *     scratch), allocated in gwam_init and freed in gwam_destroy.
 *   - A device-side failure (capacity exceeded, non-finite state) sets a status
 *     word that the next synchronising call returns; after GWAM_ECAPACITY the ray
 *     population is truncated and the context should be re-initialised.
 */
#ifndef GWAM_H
#define GWAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gwam_ctx gwam_ctx;

typedef enum {
    GWAM_OK = 0,
    GWAM_EINVAL = -1,      /* invalid argument (checked on the host before any work) */
    GWAM_ENOMEM = -2,      /* device allocation failed */
    GWAM_ECAPACITY = -3,   /* more ray volumes than max_rays */
    GWAM_ENUMERIC = -4,    /* non-finite or out-of-range background */
    GWAM_ECUDA = -5,       /* a CUDA runtime call failed */
    GWAM_ETIMEOUT = -6,    /* a bounded device wait gave up */
    GWAM_ESTATE = -7       /* call out of order (e.g. step before set_background) */
} gwam_status;

/* Grid.  geometry 0: doubly periodic f-plane box of nx*dx by ny*dy with Coriolis f0.
 * geometry 1: global lat-lon sphere of radius `radius`, f = 2 omega sin(phi).
 * nx, ny, nz >= 2; dz > 0; z_top = nz * dz. */
typedef struct {
    int geometry;
    int nx, ny, nz;
    double dx, dy;        /* f-plane cell size (m); ignored on the sphere */
    double dz;            /* level thickness (m) */
    double f0;            /* f-plane Coriolis parameter (1/s) */
    double radius;        /* planetary radius a (m); r = a + z */
    double omega;         /* rotation rate (1/s) */
    double g;             /* gravity (m/s^2), elastic term of Eq. fluxes:buoyancy */
} gwam_grid;

/* Method switches (App. B, Sec. 3c) and capacity. */
typedef struct {
    int precision;        /* 0: FP64 throughout; 1: precision form -- ray kinematics in FP32 with
                             positions as cell index + FP32 offsets, FP64 only for the saturation
                             sums, the flux accumulation and the budget */
    int gamma_mode;       /* 0: Gamma = 0; 1: Gamma^2 = (d ln rho/dz)^2 / 4 (Sec. 2a) */
    int saturation;       /* spectral saturation of Sec. 3c on/off */
    int smoothing;        /* horizontal 1-2-1 flux smoothing (App. B.4 on a lat-lon grid) on/off */
    int flux_form;        /* 0: direct fluxes (Eq. fluxes:momentum); 1: pseudomomentum (App. A) */
    int splitting;        /* ray-volume splitting (App. B.3) on/off */
    int cap_per_column;   /* ray volumes kept per column (App. B.5); <= 0: no cap */
    double alpha_s;       /* splitting scale factor (2.5 in App. B.3) */
    double min_split_dz;  /* minimum vertical split threshold (1 km in App. B.3) */
    int64_t max_rays;     /* capacity: live ray volumes plus split children of one step (all members) */
    int members;          /* ensemble members: independent backgrounds and ray populations advanced
                             together (0 or 1: a single member; at most 255) */
} gwam_params;

/* Background source of Sec. 3c: alpha(phi) profile, F_sol = alpha(phi) F_s + alpha(-phi) F_w,
 * seasonal F_am(tau); every column with |phi| <= phi_max_deg launches n_az * n_c bins
 * (azimuth 2 pi a / n_az, ground-based phase speed c_min (c_max/c_min)^(q/(n_c-1))) of
 * horizontal wavelength lambda_h in the slab [z_launch, z_launch + dz_launch]; each bin
 * carries F_am / (n_az n_c).  Sphere only. */
typedef struct {
    double f_s, f_w;          /* Pa */
    double tau;               /* 2 pi (t - t_sol) / 1 yr */
    double z_launch, dz_launch;
    double lambda_h;
    double c_min, c_max;
    int n_az, n_c;
    double spectral_frac;     /* dk = dl = frac |k_h|, dm = frac |m| */
    double phi_max_deg;       /* 85 in Sec. 3c */
    int launch_zero_flux;     /* 1: launch zero-action rays where F_am = 0 */
} gwam_bg_source;

/* One explicit spectral launch in column (i, j) of ensemble member `member` (convective-like sources). */
typedef struct {
    int i, j;
    int member;
    double z_launch, dz_launch, theta, c, lambda_h, flux, spectral_frac;
} gwam_spec;

/* Explicit ray volumes: 13 arrays of n doubles -- position (x|lambda, y|phi, z),
 * wavevector (k, l, m), extents (ex, ey in coordinate units, ez in m),
 * spectral widths (dk, dl, dm) and phase-space wave-action density n. */
typedef struct {
    const double *x, *y, *z, *k, *l, *m, *ex, *ey, *ez, *dk, *dl, *dm, *n;
} gwam_ray_input;

/* Counters are cumulative since gwam_init (ray_steps: ray volumes live at the start of each
 * step, summed over steps); w_* are wave-action contents (N Px Py Pz summed, the Sec. 4 budget)
 * in FP64. */
typedef struct {
    int64_t n_live, n_launched, n_filtered, n_split_v, n_split_h;
    int64_t n_exited, n_capped, n_merged, n_invalid, n_steps, ray_steps;
    double w_total, w_launched, w_saturated, w_exited, w_capped, w_invalid;
} gwam_stats;

/* Create a context on the current CUDA device; `stream` is a cudaStream_t (NULL = legacy
 * default stream).  Allocates all device state for `params->max_rays` ray volumes.
 * Errors: GWAM_EINVAL (bad sizes), GWAM_ENOMEM, GWAM_ECUDA.  *out is NULL on failure. */
int gwam_init(gwam_ctx **out, const gwam_grid *grid, const gwam_params *params, void *stream);
void gwam_destroy(gwam_ctx *ctx);

/* Mean state (Sec. 3b): U, V, N^2, rho, each [nz][ny][nx] doubles, copied into the
 * context's own layout; Gamma^2 is derived from rho.  Device pointers.  Checks (device
 * reduction, synchronising): finite, rho > 0, N^2 > f^2 -> GWAM_ENUMERIC.  gwam_set_background
 * gives every ensemble member this background; gwam_set_member_background one member. */
int gwam_set_background(gwam_ctx *ctx, const double *u, const double *v, const double *n2, const double *rho);
int gwam_set_background_host(gwam_ctx *ctx, const double *u, const double *v, const double *n2,
                             const double *rho);
int gwam_set_member_background(gwam_ctx *ctx, int member, const double *u, const double *v, const double *n2,
                               const double *rho);
int gwam_set_member_background_host(gwam_ctx *ctx, int member, const double *u, const double *v,
                                    const double *n2, const double *rho);

/* Append explicit ray volumes (ids next_id, next_id+1, ...), P_x = hX ex dk, P_y = hY ey dl,
 * P_z = ez dm (Sec. 3a).  A ray outside the domain -> GWAM_EINVAL and nothing is added.
 * Synchronising.  Capacity -> GWAM_ECAPACITY. */
int gwam_add_rays(gwam_ctx *ctx, const gwam_ray_input *rays, int64_t n);
int gwam_add_rays_host(gwam_ctx *ctx, const gwam_ray_input *rays, int64_t n);

/* Launch the background source (Sec. 3c) into every member, at the end of the current ray array,
 * in member order, column order (j, then i) and bin order (azimuth, then phase speed).  Bins with w_hat outside
 * (|f|, N) or m^2 <= 0 are counted in n_filtered.  Stream-ordered (no host sync). */
int gwam_launch_sources(gwam_ctx *ctx, const gwam_bg_source *src);
/* Explicit spectral launches, in array order; `specs` device pointer / host pointer. */
int gwam_launch_spectral(gwam_ctx *ctx, const gwam_spec *specs, int64_t n);
int gwam_launch_spectral_host(gwam_ctx *ctx, const gwam_spec *specs, int64_t n);

/* One full step of dt seconds (dt > 0): RK3 ray propagation (App. B.2), exits, splitting
 * (App. B.3), re-binning by cell, per-column cap (App. B.5), saturation (Sec. 3c), flux
 * projection (Sec. 3b), smoothing (App. B.4), divergence (Eq. mean-flow-impact) into
 * dudt, dvdt ([members][nz][ny][nx] device buffers, may be NULL), wave-action budget (Sec. 4).
 * Stream-ordered: no host synchronisation. */
int gwam_step(gwam_ctx *ctx, double dt, double *dudt, double *dvdt);
/* The same step replayed from a CUDA graph: the first call for a given (dt, dudt, dvdt) captures the
 * step's kernels (two graphs, one per ray-buffer parity) on an internal stream; later calls launch
 * the graph on the context's stream -- one launch per step.  Launches and backgrounds may change
 * between calls (the kernels read counts from device memory).  Per-phase profiling is not recorded
 * inside graphs. */
int gwam_step_graph(gwam_ctx *ctx, double dt, double *dudt, double *dvdt);
/* The same with host output buffers (copied back and synchronised). */
int gwam_step_host(gwam_ctx *ctx, double dt, double *dudt_host, double *dvdt_host);

/* Launch shapes of the three heavy ray kernels (0 advance, 1 materialise, 2 projection): threads
 * per block (64..256, a multiple of 32) and blocks (1..8 x the SM count).  gwam_autotune advances
 * the simulation by (candidates x steps_per_candidate) real steps of dt, timing each kernel with
 * CUDA events under each candidate shape, and keeps the fastest shape per kernel (host-side
 * search; the caller may persist the result and restore it with gwam_set_launch_config). */
int gwam_set_launch_config(gwam_ctx *ctx, int kernel, int threads, int blocks);
int gwam_get_launch_config(gwam_ctx *ctx, int kernel, int *threads, int *blocks);
int gwam_autotune(gwam_ctx *ctx, double dt, int steps_per_candidate, double *dudt, double *dvdt);

/* Number of live ray volumes (synchronising). */
int gwam_num_rays(gwam_ctx *ctx, int64_t *n);
/* Ray volumes in canonical order into host memory: state13_host is 13 blocks of `cap`
 * doubles (x y z k l m ex ey ez Px Py Pz N), ids/cells `cap` entries each (either may be
 * NULL).  Ids carry the ensemble member in their top 8 bits; cells are member * ncell + the
 * member's cell index.  cap < number of rays -> GWAM_ECAPACITY. */
int gwam_get_rays_host(gwam_ctx *ctx, double *state13_host, int64_t *ids_host, int32_t *cells_host,
                       int64_t cap);
/* Counters and budget (synchronising; returns a pending device status). */
int gwam_get_stats(gwam_ctx *ctx, gwam_stats *out);
/* Grid field of the last step into host memory, [members] outermost: 0 Fz_lambda, 1 Fz_phi
 * ([nz+1][ny][nx]), 2 F_ll, 3 F_lp, 4 F_pl, 5 F_pp, 6 E_lambda, 7 E_phi, 8 wave-action density ([nz][ny][nx]);
 * fluxes after smoothing when it is on; E_* without the 1/(g rho) factor. */
int gwam_get_field_host(gwam_ctx *ctx, int which, double *out_host);
/* Gamma^2 node field [members][nz][ny][nx] into host memory. */
int gwam_get_gamma2_host(gwam_ctx *ctx, double *out_host);
int gwam_synchronize(gwam_ctx *ctx);

/* Per-cell segment offsets of a ray array ordered by cell (the parent-cell storage of App. B.2):
 * offsets[c] = number of entries of cells[] smaller than c, offsets[ncell] = n, so the entries of
 * cell c are [offsets[c], offsets[c+1]) when cells[] is sorted.  cells: n int32 device values in
 * [0, ncell); offsets: ncell + 1 int32 device values, overwritten.  Work is enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and the call synchronises it.  The call allocates
 * its block-sum scratch (stream-ordered) and frees it before returning.  Errors: GWAM_EINVAL for
 * bad sizes or null pointers, or when a cell lies outside [0, ncell) (such entries are not
 * counted); GWAM_ENOMEM; GWAM_ECUDA. */
int gwam_cell_offsets(const int32_t *cells, int64_t n, int32_t ncell, int32_t *offsets, void *stream);

/* gwam_cell_offsets for callers that cannot allocate device memory.  (The paper has no counterpart:
 * it concerns how this library is called, not the method.)  Host models that hand all device memory
 * to their own pool allocator at start-up, or run under a fixed device-memory budget, must not call
 * cudaMalloc later; this entry point allocates nothing -- no cudaMalloc/cudaFree and no allocating
 * library routine.  Same arguments, results and errors as gwam_cell_offsets, computed by the same
 * kernels, with the scratch in a fixed array inside the library (about 32 KB, held on every GPU that
 * loads the library until the process exits).
 *   - ncell must not exceed GWAM_NOALLOC_MAX_CELLS, else GWAM_ECAPACITY and nothing is done.
 *   - The first call on a device, with that device current, looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU (concurrent streams, threads or
 *     processes sharing a context) race with each other; serialise them. */
#define GWAM_NOALLOC_MAX_CELLS 16775168
int gwam_cell_offsets_noalloc(const int32_t *cells, int64_t n, int32_t ncell, int32_t *offsets, void *stream);

/* Self-test of the arithmetic helpers the kernels use instead of FP64 division and square root
 * (Newton-Raphson refinement of the hardware approximations): rcp_out[i] ~ 1/x[i],
 * rsqrt_out[i] ~ 1/sqrt(x[i]) for positive normal x.  Device pointers, n values; synchronises. */
int gwam_selftest_math(const double *x, int64_t n, double *rcp_out, double *rsqrt_out, void *stream);

/* Per-phase device timing with CUDA events recorded on the context's stream around each phase
 * of gwam_step (for measurement tools; off by default).  enable != 0 resets and starts the
 * accumulation, 0 stops it.  Phases: 0 advance (RK3, exits, split decisions), 1 re-binning
 * (scans, scatter, cap, segment sort, materialise), 2 saturation, 3 projection, 4 smoothing,
 * divergence and budget.  gwam_profile_read synchronises and returns the accumulated
 * milliseconds per phase (ms_host[5]) and the number of profiled steps. */
int gwam_profile_enable(gwam_ctx *ctx, int enable);
int gwam_profile_read(gwam_ctx *ctx, double *ms_host, int64_t *steps);
/* Human-readable description of the last error on this context (never NULL). */
const char *gwam_last_error(const gwam_ctx *ctx);
/* Library version string. */
const char *gwam_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GWAM_H */
