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
    int columnar;         /* 1: single-column mode of MS-GWaM-1D (the single-column approximation of
                             Sec. 1): no horizontal propagation, advection or refraction -- position,
                             horizontal wavenumber and horizontal extents fixed, dm/dt = -dOmega/dz --
                             and du/dt, dv/dt from the vertical flux divergence and the elastic term
                             only; 0: the 3-D model */
    int theta_flux;       /* 1: also project the potential-temperature flux of Eq. fluxes:temperature
                             (fields 9, 10 of gwam_get_field_host) for gwam_get_theta_tendency_host,
                             in either form (FP64 sums; FP32 integrands in the precision form) */
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
/* Explicit spectral launches, in array order; `specs` device pointer / host pointer.  A spec whose
 * column or member lies outside the grid: GWAM_EINVAL (host specs, nothing launched) or, for device
 * specs, the context status GWAM_EINVAL reported by the next synchronising call. */
int gwam_launch_spectral(gwam_ctx *ctx, const gwam_spec *specs, int64_t n);
int gwam_launch_spectral_host(gwam_ctx *ctx, const gwam_spec *specs, int64_t n);

/* Ghost-layer launch over one launch interval dt > 0 (Sec. 3c: the source layer within which ray
 * volumes propagate vertically only; each interval the part that left it is activated, volumes
 * reflected inside are discarded).  Per bin (same bins, order and filtering as gwam_launch_sources /
 * gwam_launch_spectral) a ghost ray volume in the launch state fills the layer [z_launch, z_launch +
 * dz_launch] and is advanced over dt by the single-column equations (k, l, horizontal position and
 * extents fixed).  If its m is no longer negative it is discarded (counted in n_filtered);
 * otherwise the part above the layer top -- from the top (or the ghost's own bottom, if it left
 * whole) to the ghost's top, with the ghost's m, N, horizontal extents and P_z in proportion to
 * the extent -- is appended as a new ray volume (n_launched, w_launched); a bin from which
 * nothing has left the layer appends nothing.  Called once per model step before gwam_step, this
 * emits the source flux every interval.  The ghost is integrated in the FP64 form's double-float
 * arithmetic in both forms: a precision-form context allocates double-float background nodes
 * (128 B per node) at its first ghost-layer launch and keeps them set from then on.  dt not > 0 or
 * not finite: GWAM_EINVAL.  Stream-ordered like the launches above. */
int gwam_launch_ghost(gwam_ctx *ctx, const gwam_bg_source *src, double dt);
int gwam_launch_ghost_spectral(gwam_ctx *ctx, const gwam_spec *specs, int64_t n, double dt);
int gwam_launch_ghost_spectral_host(gwam_ctx *ctx, const gwam_spec *specs, int64_t n, double dt);

/* One full step of dt seconds (dt > 0): RK3 ray propagation (App. B.2), exits, splitting
 * (App. B.3), re-binning by cell, per-column cap (App. B.5), saturation (Sec. 3c), flux
 * projection (Sec. 3b), smoothing (App. B.4), divergence (Eq. mean-flow-impact) into
 * dudt, dvdt ([members][nz][ny][nx] device buffers, may be NULL), wave-action budget (Sec. 4).
 * Stream-ordered: no host synchronisation. */
int gwam_step(gwam_ctx *ctx, double dt, double *dudt, double *dvdt);

/* Asynchronous host entry points: the host-link copies run on two copy streams of the context (one
 * per direction) and overlap the steps; neither call waits for the device.  gwam_set_background_host_async copies the
 * four page-locked caller fields into one of two device staging slots and sets every member's
 * background from it (as gwam_set_background) into a second background set on a set-up stream of
 * its own, overlapping the step in flight; the next step reads the new set (the two sets swap at
 * every call; the first call allocates the second set, about 180 B per node); an invalid value (as there) becomes the sticky
 * context status GWAM_ENUMERIC, reported by the next synchronising call, and the steps in between
 * do nothing.  gwam_step_host_async runs the step (as gwam_step_graph: one graph per output slot,
 * the slots alternating with the ray buffers) into one of two device output slots and copies
 * du/dt, dv/dt into the page-locked caller buffers (either may be NULL).  The caller keeps the input
 * fields unchanged and reads the outputs only after a synchronising call (gwam_synchronize,
 * gwam_get_stats, ...); buffers that are not page-locked: GWAM_EINVAL. */
int gwam_set_background_host_async(gwam_ctx *ctx, const double *u, const double *v, const double *n2,
                                   const double *rho);
int gwam_step_host_async(gwam_ctx *ctx, double dt, double *dudt, double *dvdt);

/* The same step replayed from a CUDA graph: the first call for a given (dt, dudt, dvdt) captures the
 * step's kernels (two graphs, one per ray-buffer parity) on an internal stream; later calls launch
 * the graph on the context's stream -- one launch per step.  Launches and backgrounds may change
 * between calls (the kernels read counts from device memory).  The graphs carry event nodes at the
 * phase boundaries instead of the per-phase profiling of gwam_profile_enable
 * (gwam_graph_profile_read). */
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
 * ([nz+1][ny][nx]), 2 F_ll, 3 F_lp, 4 F_pl, 5 F_pp, 6 E_lambda, 7 E_phi, 8 wave-action density, 9 T_lambda,
 * 10 T_phi ([nz][ny][nx]; 9 and 10 only with theta_flux = 1: g rho-bar <u'theta'> / theta-bar of Eq.
 * fluxes:temperature); fluxes after smoothing when it is on; E_* without the 1/(g rho) factor. */
int gwam_get_field_host(gwam_ctx *ctx, int which, double *out_host);
/* Reference potential temperature theta-bar of Eq. fluxes:temperature: device array
 * [members][nz][ny][nx], copied; GWAM_ENUMERIC unless every value is positive and finite. */
int gwam_set_theta(gwam_ctx *ctx, const double *theta);
/* Potential-temperature tendency of the last step (Eq. mean-flow-impact-t), d theta/dt =
 * -div <u'theta'> with <u'theta'> = theta-bar / (g rho-bar) times the projected integrals of fields
 * 9, 10 (smoothed when smoothing is on), horizontal centred differences as in the momentum
 * divergence, zero in the columnar mode; into host memory [members][nz][ny][nx].  Needs
 * theta_flux = 1, gwam_set_theta and a background (GWAM_ESTATE otherwise).  Synchronises. */
int gwam_get_theta_tendency_host(gwam_ctx *ctx, double *out_host);
/* Gamma^2 node field [members][nz][ny][nx] into host memory. */
int gwam_get_gamma2_host(gwam_ctx *ctx, double *out_host);
int gwam_synchronize(gwam_ctx *ctx);

/* Checkpoint and resume (an operation of this library, not of the paper).  gwam_save writes the
 * complete state that the next step depends on -- the ray volumes in canonical order, ids,
 * counters, budget terms and the background (FP64 nodes and rho; the derived arrays are rebuilt
 * on load) -- to a binary file in host byte order; gwam_load reads it into a context created with the same grid,
 * parameters, members and precision (GWAM_EINVAL otherwise, or for a missing or truncated file;
 * GWAM_ECAPACITY if the file holds more ray volumes than this context's max_rays).  A step after
 * gwam_load gives bit for bit the results the saved context's next step gives.  The grid fields of
 * the last step (gwam_get_field_host) are not part of the checkpoint.  Both synchronise. */
int gwam_save(gwam_ctx *ctx, const char *path);
int gwam_load(gwam_ctx *ctx, const char *path);

/* Per-cell segment offsets of a ray array ordered by cell (the parent-cell storage of App. B.2):
 * offsets[c] = number of entries of cells[] smaller than c, offsets[ncell] = n, so the entries of
 * cell c are [offsets[c], offsets[c+1]) when cells[] is sorted.  cells: n int32 device values in
 * [0, ncell); offsets: ncell + 1 int32 device values, overwritten.  Work is enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and the call synchronises it.  The call allocates
 * its block-sum scratch (stream-ordered) and frees it before returning.  Errors: GWAM_EINVAL for
 * bad sizes or null pointers, or when a cell lies outside [0, ncell) (such entries are not
 * counted); GWAM_ENOMEM; GWAM_ECUDA when one of its own launches, copies or the stream fails (each
 * launch is checked by its own status: an error left pending by the caller's earlier work is
 * neither reported as this call's nor cleared). */
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
 *     (cudaGetSymbolAddress) and remembers it; make that first call before any stream capture.
 *     With lazy module loading (the CUDA default since 12.2) the array and the kernels are loaded
 *     onto the device at that first call, not when the library is loaded: make the first call
 *     before the host model reserves its device memory, or load modules eagerly
 *     (CUDA_MODULE_LOADING=EAGER) so the array is placed when the library loads.
 *   - The remembered address belongs to the device's context: after cudaDeviceReset it is stale,
 *     so do not call this entry point in a process that has reset the device.
 *   - Errors that the caller's own earlier work left pending are neither reported by this call
 *     nor cleared by it (each launch's own status is checked).
 *   - All calls share the one array: calls that overlap on the GPU (concurrent streams, threads or
 *     processes sharing a context) race with each other; serialise them. */
#define GWAM_NOALLOC_MAX_CELLS 16775168
int gwam_cell_offsets_noalloc(const int32_t *cells, int64_t n, int32_t ncell, int32_t *offsets, void *stream);

/* Self-test of the arithmetic helpers the kernels use instead of FP64 division and square root
 * (Newton-Raphson refinement of the hardware approximations): rcp_out[i] ~ 1/x[i],
 * rsqrt_out[i] ~ 1/sqrt(x[i]) for positive normal x.  Device pointers, n values; synchronises. */
int gwam_selftest_math(const double *x, int64_t n, double *rcp_out, double *rsqrt_out, void *stream);

/* Self-test of the precision form's FP64-free helpers: widened[i] = x[i] as a double by integer
 * re-biasing (must equal the hardware float -> double conversion bit for bit, subnormals, zeros,
 * infinities and NaN classes included); action[i] (or NULL) = x[i] x[i+1] x[i+2] x[i+3] (indices
 * mod n) formed in double-float arithmetic on the FP32 pipes and returned as a double.  Device
 * pointers; synchronises `stream`. */
int gwam_selftest_widen(const float *x, int64_t n, double *widened, double *action, void *stream);
/* Self-test of the integer double -> float narrowing (round to nearest even): out[i] must equal the
 * hardware conversion bit for bit (subnormal results, overflow to infinity, NaN classes included). */
int gwam_selftest_narrow(const double *x, int64_t n, float *out, void *stream);
/* Self-test of the double-float split of the FP64 form: hi[i] = x[i] rounded to FP32 and lo[i] =
 * (x[i] - hi[i]) rounded to FP32 (round to nearest even both), bit for bit, whichever of its two
 * paths (integer-only for 2^-74 <= |x| < 2^127, one FP64 subtraction otherwise) x[i] takes.  Device
 * pointers, n values; synchronises `stream`. */
int gwam_selftest_split(const double *x, int64_t n, float *hi, float *lo, void *stream);
/* Self-test of the double-float logarithm of a ratio that forms Gamma^2 = (d ln rho / dz)^2 / 4 from
 * centred differences of ln rho (Sec. 2a; the differences are taken as ln(rho_up / rho_down)):
 * out[i] = ln(a[i] / b[i]) for positive normal doubles a, b, relative error about 2^-45 (exactly 0
 * when a == b).  Device pointers; synchronises `stream`. */
int gwam_selftest_logratio(const double *a, const double *b, int64_t n, double *out, void *stream);

/* Self-test of the step's exclusive scans (the re-binning's new-id and per-cell offsets, App. B.2
 * parent-cell storage): out0[i] = in0[0] + ... + in0[i-1] for i <= n0 (out0[n0] = the total), by
 * the context's two-pass scan over contiguous parts; with in1 != NULL a second, independent scan of
 * in1[0..n1) into out1 runs in the same two launches (as the step pairs its two scans).  Device
 * int32 arrays of any alignment (16-byte-aligned ones take the vector path); in == out is allowed;
 * out must hold n + 1 values; totals must fit in int32.  Runs on the context's stream and
 * synchronises it.  GWAM_EINVAL for negative sizes or missing arrays. */
int gwam_selftest_scan(gwam_ctx *ctx, const int32_t *in0, int32_t *out0, int64_t n0, const int32_t *in1,
                       int32_t *out1, int64_t n1);

/* Self-test of the surrogate's tensor-core GEMM (tcgen05 + TMA, sm_103a): C = act(A . B^T + bias)
 * with A [M][K] and B [N][K] row-major BF16 device arrays (K contiguous, K a multiple of 64, base
 * addresses 16-byte aligned), bias [N] FP32 or NULL, act = GELU(z) = z Phi(z) when gelu != 0, C
 * [M][N] overwritten: FP32 (out_bf16 = 0) or BF16 rounded to nearest (out_bf16 = 1; written through
 * shared memory by TMA stores when N is a multiple of 8).  Products are exact, sums are FP32.  bn
 * selects the tile width (0 = by N; else 64, 128, 192 or 256).  Synchronises `stream`.  Errors:
 * GWAM_EINVAL (shape, alignment, tile), GWAM_ENOMEM, GWAM_ECUDA, GWAM_ETIMEOUT (a bounded device wait
 * gave up). */
int gwam_gemm_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int gelu, int bn,
                   int out_bf16, void *C, void *stream);

/* Self-test of the GEMM's bounded device waits (the failure detection of every spin-wait in the
 * library's kernels; not in the paper): the gwam_gemm_bf16 kernel with tile width bn (as above) is
 * launched with its TMA producer told to issue no copies and every mbarrier wait limited to
 * wait_us microseconds (1 .. 2 000 000).  The MMA and epilogue warps wait on stages that never fill,
 * give up after wait_us, wait (bounded) for the MMAs they issued -- none -- release their tensor
 * memory and set the error word; the call returns GWAM_ETIMEOUT and the context stays usable (the
 * next GEMM allocates the same tensor memory).  A, B, C as for gwam_gemm_bf16 (C FP32, not
 * written).  Synchronises `stream`.  GWAM_EINVAL for bad arguments. */
int gwam_selftest_gemm_timeout(const void *A, const void *B, int M, int N, int K, int bn, float *C,
                               unsigned int wait_us, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Column drag surrogate (not in the paper: an emulator of the ray tracer's column drag, with the
 * tracer as fallback).  An MLP n_in -> n_hidden (x n_layers, GELU(z) = z Phi(z)) -> n_out with
 * BF16 weights and activations on the tensor cores, FP32 accumulation, FP32 master weights and
 * Adam moments (Kingma & Ba 2015).  Inputs are FP32 column features [n][n_in] (row-major, device),
 * normalised per feature, x_hat = (x - mu) * (1 / sigma); targets FP32 [n][n_out] normalised the
 * same way; the loss is the mean over rows and outputs of (y - t)^2 in normalised units.  A column
 * is inside the envelope when lo[f] <= x_hat[f] <= hi[f] for every feature f (all finite); columns
 * outside it are flagged for the ray tracer.  All work is enqueued on the stream given at creation.
 * ------------------------------------------------------------------------------------------- */
typedef struct gwam_mlp gwam_mlp;
typedef struct {
    int n_in;        /* features per column (368 = u, v, N^2, ln rho on 90 levels + 8 source parameters) */
    int n_hidden;    /* width of every hidden layer, a multiple of 64 (512) */
    int n_layers;    /* hidden layers, 1..7 (4) */
    int n_out;       /* outputs per column (180 = du/dt then dv/dt on nlev levels) */
    int nlev;        /* levels of the drag output for gwam_mlp_infer (2 nlev = n_out), or 0 */
    int max_batch;   /* rows per training step and per inference pass, a multiple of 128 */
    uint64_t seed;   /* initial weights W ~ N(0, 1/n_in) from SplitMix64 + Box-Muller, b = 0 */
    float beta1, beta2, eps;   /* Adam constants (0.9, 0.999, 1e-8) */
} gwam_mlp_config;

/* Create / destroy.  Allocates every buffer (weights, Adam state, activations of max_batch rows,
 * split-K scratch) and the TMA tensor maps once.  GWAM_EINVAL, GWAM_ENOMEM, GWAM_ECUDA. */
int gwam_mlp_create(gwam_mlp **out, const gwam_mlp_config *cfg, void *stream);
void gwam_mlp_destroy(gwam_mlp *m);
const char *gwam_mlp_last_error(const gwam_mlp *m);
/* Normalisation and envelope from host arrays: x_mu, x_sigma, lo, hi [n_in]; y_mu, y_sigma [n_out];
 * sigma > 0 and finite, else GWAM_EINVAL.  Synchronises. */
int gwam_mlp_set_normalization_host(gwam_mlp *m, const float *x_mu, const float *x_sigma, const float *y_mu,
                                    const float *y_sigma, const float *lo, const float *hi);
/* Normalisation fitted to a device data set X [n][n_in], Y [n][n_out] (FP64 sums): features get
 * their mean and population sigma (1 for a constant feature); targets get their mean and one shared
 * sigma, the RMS over outputs of their standard deviations (the loss is then proportional to the
 * drag's own squared error); envelope = [min, max] of x_hat widened by margin * (max - min).
 * stats_host (or NULL) receives 4 n_in + 2 n_out floats: x mu, x sigma, lo, hi, y mu, y sigma. */
int gwam_mlp_fit_normalization(gwam_mlp *m, const float *X, const float *Y, int64_t n, float margin,
                               float *stats_host);
/* Parameters of weight layer 1..n_layers+1 from / to host: W [n_out_l][n_in_l] row-major, b [n_out_l].
 * get: which = 0 the FP32 master weights, 1 the gradients of the last train step (either pointer
 * may be NULL).  Synchronise. */
int gwam_mlp_set_params_host(gwam_mlp *m, int layer, const float *W, const float *b);
int gwam_mlp_get_params_host(gwam_mlp *m, int layer, int which, float *W, float *b);
/* One training step on `batch` rows (a multiple of 64, <= max_batch) of the device data set X, Y
 * of n rows: rows[] (device int32, batch entries in [0, n)) or, when rows is NULL, rows drawn by
 * SplitMix64(seed + (r + 1) * 0x9E3779B97F4A7C15) mod n.  Forward, loss, backward and, when lr > 0,
 * one Adam update with that learning rate (lr = 0: gradients only).  Asynchronous. */
int gwam_mlp_train_step(gwam_mlp *m, const float *X, const float *Y, int64_t n, const int32_t *rows, int batch,
                        uint64_t seed, float lr);
/* Loss of the last train step (synchronises; returns a pending device error: GWAM_ETIMEOUT when a
 * bounded wait in the GEMM gave up, GWAM_EINVAL for a row index outside the data set). */
int gwam_mlp_last_loss_host(gwam_mlp *m, double *loss);
/* Network outputs (normalised units) of the first `rows` rows of the last train step, [rows][n_out]. */
int gwam_mlp_output_host(gwam_mlp *m, float *Y, int rows);
/* Inference on ncol columns of features X [ncol][n_in]: for every column inside the envelope the
 * de-normalised drag y * sigma + mu (one FP32 fused multiply-add, widened exactly) is written to
 * dudt[k * ncol + c] and dvdt[k * ncol + c] (k < nlev, the [nz][ny][nx] layout with ncol = ny nx,
 * FP64); fallback_mask[c] = 1 for columns
 * outside the envelope (their drag entries are not written), else 0; *n_fallback (device int32) =
 * their number.  Needs nlev >= 1 and n_out = 2 nlev.  Asynchronous. */
int gwam_mlp_infer(gwam_mlp *m, const float *X, int64_t ncol, double *dudt, double *dvdt, int32_t *fallback_mask,
                   int32_t *n_fallback);
/* Inference timing with CUDA events on the surrogate's stream (for measurement tools; off by
 * default): enable != 0 resets and starts it.  gwam_mlp_profile_read synchronises and returns the
 * accumulated milliseconds of the input packing (ms_host[0]) and of the GEMM chain (ms_host[1]) and
 * the number of timed passes (one per max_batch chunk). */
int gwam_mlp_profile_enable(gwam_mlp *m, int enable);
int gwam_mlp_profile_read(gwam_mlp *m, double *ms_host, int64_t *passes);
/* Pending device status of the surrogate (synchronises). */
int gwam_mlp_status(gwam_mlp *m);
/* Fallback routing: copy the ray tracer's drag into the columns with mask[c] != 0 (device arrays,
 * [nlev][ncol] FP64). */
int gwam_mlp_merge_fallback(const int32_t *mask, int64_t ncol, int nlev, const double *dudt_tracer,
                            const double *dvdt_tracer, double *dudt, double *dvdt, void *stream);
/* Surrogate data: column features X [ncol][4 nz + n_src] (FP32) from [nz][ncol] FP64 device fields
 * u, v, N^2, rho (features u, v, N^2, ln rho level by level, then the n_src source parameters from
 * src[c * src_stride + j]; src_stride = 0 shares one set), and targets Y [ncol][2 nz] = scale *
 * (du_sum, dv_sum). */
int gwam_column_features(const double *u, const double *v, const double *n2, const double *rho, int nz,
                         int64_t ncol, const float *src, int n_src, int src_stride, float *X, void *stream);
int gwam_column_targets(const double *du_sum, const double *dv_sum, int nz, int64_t ncol, double scale, float *Y,
                        void *stream);

/* Per-phase device timing with CUDA events recorded on the context's stream around each phase
 * of gwam_step (for measurement tools; off by default).  enable != 0 resets and starts the
 * accumulation, 0 stops it.  Phases: 0 advance (RK3, exits, split decisions), 1 re-binning
 * (scans, scatter, cap, segment sort, materialise), 2 saturation, 3 projection, 4 smoothing,
 * divergence and budget.  gwam_profile_read synchronises and returns the accumulated
 * milliseconds per phase (ms_host[5]) and the number of profiled steps. */
int gwam_profile_enable(gwam_ctx *ctx, int enable);
int gwam_profile_read(gwam_ctx *ctx, double *ms_host, int64_t *steps);
/* The same five phase times for graph replays (gwam_step_graph): each step graph carries event nodes
 * at the phase boundaries, overwritten by every replay; this call synchronises and returns the
 * phase times of the last replay of each of the two graphs (one per ray-buffer parity), averaged,
 * in ms_host[5], and in *replays how many graphs contributed (0 before the first replay). */
int gwam_graph_profile_read(gwam_ctx *ctx, double *ms_host, int *replays);
/* Kernel launches of one step graph replay: the number of kernel nodes of the captured step graphs
 * (the largest, if they differ), counted from the graph itself when it was captured; *kernels = 0
 * before the first gwam_step_graph.  Memset and event nodes are not kernels and are not counted. */
int gwam_graph_kernel_count(gwam_ctx *ctx, int *kernels);
/* Human-readable description of the last error on this context (never NULL). */
const char *gwam_last_error(const gwam_ctx *ctx);
/* Library version string. */
const char *gwam_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GWAM_H */
