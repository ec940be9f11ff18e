/*
 * gwam_oracle.h -- plain, slow FP64 CPU oracle of the MS-GWaM-3D ray-volume step
 * (Voelker, Boeloeni, Kim, Zaengl, Achatz: "MS-GWaM: A 3-dimensional transient
 * gravity wave parametrization for atmospheric models", arXiv:2309.11257).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, constant or helper with the CUDA path (paper_2309_11257_gb300/csrc)
 * and neither side includes or links the other.
 *
 * Everything here is host memory, FP64, single threaded, and follows the
 * paper's equations in the paper's notation:
 *   position (lambda, phi, r = a + z) or Cartesian (x, y, z)
 *   wavevector (k, l, m) = (k_lambda, k_phi, k_r)
 *   ray-volume extents (dX, dY, dZ) in coordinate units (radians on the sphere)
 *   per-axis phase-space products P_x = hX dX dk, P_y = hY dY dl, P_z = dZ dm
 *   (Sec. 3a, Eq. vpvol_cons_cart and Eq. dkxdkl)
 *   phase-space wave-action density N (calligraphic N in Eq. wa-6d-conservation).
 *
 * Cell index convention (shared by definition, not by code, with the library):
 *   cell = (j * nx + i) * nz + k   (column-major: all levels of a column adjacent)
 * Grid fields handed in and out are C-order [nz][ny][nx], level 0 at the bottom.
 */
#ifndef GWAM_ORACLE_H
#define GWAM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int geometry;           /* 0 = doubly periodic f-plane box, 1 = lat-lon sphere */
    int nx, ny, nz;         /* columns in x/lambda, rows in y/phi, levels */
    double dx, dy;          /* f-plane cell size (m); ignored on the sphere (2pi/nx, pi/ny) */
    double dz;              /* uniform level thickness (m); z_top = nz * dz */
    double f0;              /* f-plane Coriolis parameter (1/s) */
    double radius;          /* planetary radius a (m) */
    double omega;           /* planetary rotation rate (1/s), f = 2 omega sin(phi) */
    double g;               /* gravity (m/s^2), used by the elastic term */
} orc_grid;

typedef struct {
    int gamma_mode;         /* 0: Gamma = 0; 1: Gamma^2 = (d ln rho / dz)^2 / 4 */
    int saturation;         /* Sec. 3c saturation on/off */
    int smoothing;          /* App. B.4 horizontal flux smoothing on/off */
    int flux_form;          /* 0: direct fluxes (Eq. fluxes:momentum), 1: pseudomomentum (App. A) */
    int splitting;          /* App. B.3 splitting on/off */
    int cap_per_column;     /* max rays per column (Sec. B.5); <= 0 disables */
    double alpha_s;         /* splitting scale factor (2.5 in App. B.3) */
    double min_split_dz;    /* minimum vertical split threshold (1 km in App. B.3) */
    int columnar;           /* 1: single-column mode of MS-GWaM-1D (Sec. 1) -- no horizontal propagation,
                               advection or refraction; drag from the vertical flux divergence */
} orc_params;

typedef struct {
    int64_t n_live, n_launched, n_filtered, n_split_v, n_split_h;
    int64_t n_exited, n_capped, n_merged, n_invalid, n_steps;
    double w_total, w_launched, w_saturated, w_exited, w_capped, w_invalid;
} orc_stats;

/* Background launch (Sec. 3c, background source) */
typedef struct {
    double f_s, f_w;        /* summer / winter solstice flux amplitudes (Pa) */
    double tau;             /* 2 pi (t - t_sol) / 1 yr */
    double z_launch;        /* bottom of the launch slab (m) */
    double dz_launch;       /* slab thickness = initial vertical extent (m) */
    double lambda_h;        /* horizontal wavelength (m) */
    double c_min, c_max;    /* ground-based phase speed range (m/s), log spaced */
    int n_az, n_c;          /* azimuths, phase speeds */
    double spectral_frac;   /* dk = dl = frac*|k_h|, dm = frac*|m| */
    double phi_max_deg;     /* no launch poleward of this latitude (85 deg) */
    int launch_zero_flux;   /* launch rays with zero action in zero-flux columns */
} orc_bg_source;

/* One explicit spectral launch (convective-like sources, tests) */
typedef struct {
    int i, j;               /* launch column */
    int pad_;
    double z_launch, dz_launch, theta, c, lambda_h, flux, spectral_frac;
} orc_spec;

typedef struct orc_model orc_model;

orc_model *orc_create(const orc_grid *grid, const orc_params *params);
void orc_destroy(orc_model *m);
/* fields C-order [nz][ny][nx] */
int orc_set_background(orc_model *m, const double *u, const double *v,
                       const double *n2, const double *rho);
/* explicit rays: positions, wavevector, extents (dX,dY in coordinate units), dk dl dm, N */
int orc_add_rays(orc_model *m, int64_t n, const double *x, const double *y, const double *z,
                 const double *k, const double *l, const double *mm,
                 const double *ex, const double *ey, const double *ez,
                 const double *dk, const double *dl, const double *dm, const double *nn);
int orc_launch_background(orc_model *m, const orc_bg_source *src);
int orc_launch_spectral(orc_model *m, int64_t n, const orc_spec *specs);
/* ghost-layer launch over one launch interval dt > 0 (Sec. 3c): per bin, the part of a layer-filling
 * ghost ray volume that propagated (vertically only) out of the launch layer is activated; ghost
 * volumes reflected within the layer are discarded (counted as filtered) */
int orc_launch_ghost(orc_model *m, const orc_bg_source *src, double dt);
int orc_launch_ghost_spectral(orc_model *m, int64_t n, const orc_spec *specs, double dt);
/* one full step; dudt/dvdt C-order [nz][ny][nx] (may be NULL) */
int orc_step(orc_model *m, double dt, double *dudt, double *dvdt);

/* projection, smoothing and tendencies of the current ray volumes, no advance (NULL: fields only) */
int orc_diagnose(orc_model *m, double *dudt, double *dvdt);
int64_t orc_num_rays(const orc_model *m);
/* state: 13 arrays of n in the order x y z k l m dX dY dZ Px Py Pz N (array order) */
int orc_get_rays(const orc_model *m, double *state13, int64_t *ids, int32_t *cells);
void orc_get_stats(const orc_model *m, orc_stats *out);
/* the three phases of orc_step, for a domain-decomposed driver: advance (RK3, exits, splits; array
 * order), local (canonical order, cap, saturation, projection), grid (smoothing, divergence, budget) */
int orc_step_advance(orc_model *m, double dt);
int orc_step_local(orc_model *m, double dt);
int orc_step_grid(orc_model *m, double *dudt, double *dvdt);
/* latitude band [j0, j1) owned by this model (launches only there); id counter; id remapping; new
 * ids issued by the rays before an array position in the last advance; ray
 * volumes whose carrier row left the band (count, take out: row-major states of 13 values + ids);
 * ray volumes handed over (appended with their ids); projected fields overwritten (halo rows) */
int orc_set_owned_rows(orc_model *m, long j0, long j1);
int64_t orc_get_next_id(const orc_model *m);
void orc_set_next_id(orc_model *m, int64_t id);
void orc_remap_ids(orc_model *m, int64_t lo, int64_t hi, int64_t to);
int64_t orc_issued_before(const orc_model *m, int64_t q);
int64_t orc_count_rays_outside(const orc_model *m);
int64_t orc_take_rays_outside(orc_model *m, double *out_state, int64_t *out_ids, int32_t *out_rows, int64_t cap);
int orc_put_rays(orc_model *m, int64_t n, const double *state, const int64_t *ids);
int orc_set_field(orc_model *m, int which, const double *in);
/* threads for the independent per-ray loops (results bit-identical for any count; returns the count
 * in effect: 1 when built without OpenMP) */
int orc_set_threads(orc_model *m, int threads);
/* per ray volume: the wave-action density before the last step's saturation, or |N| (n values) */
int orc_get_action_scale(const orc_model *m, double *out);
/* grid fields of the last step: which = 0..10 ->
 * Fz_lambda, Fz_phi ([nz+1][ny][nx]), F_ll, F_lp, F_pl, F_pp, E_l, E_p, wave-action density, and the
 * potential-temperature flux integrals T_l, T_p of Eq. fluxes:temperature without theta-bar / (g rho-bar)
 * ([nz][ny][nx]) */
int orc_get_field(const orc_model *m, int which, double *out);
/* error scales: sums of |contribution| of a field (each with the ray volume's wave action before the
 * step's saturation), and the tendency formula applied to them */
int orc_get_field_abs(const orc_model *m, int which, double *out);
int orc_tendency_scale(const orc_model *m, double *du_scale, double *dv_scale);
/* reference potential temperature [nz][ny][nx] (positive; -1 otherwise) and the potential-temperature
 * tendency of the last step (Eq. mean-flow-impact-t) with its error scale (scale may be NULL) */
int orc_set_theta(orc_model *m, const double *theta);
int orc_theta_tendency(const orc_model *m, double *out, double *scale);
/* the same divergence of given integrals T_l, T_p (C-order [nz][ny][nx]) */
int orc_theta_divergence(const orc_model *m, const double *tl, const double *tp, double *out);
/* Gamma^2 node field [nz][ny][nx] */
int orc_get_gamma2(const orc_model *m, double *out);

/* ---- single-ray pieces, exposed for the pins ---- */
/* out[0..3] = U V N2 G2, out[4..15] = their interpolated node gradients d/dX, d/dY, d/dz (field-major) */
void orc_gather(const orc_model *m, double X, double Y, double Z, double *out16);
/* intrinsic frequency and intrinsic group velocity: out = {w, ch_x, ch_y, ch_r, K2} */
void orc_dispersion(double k, double l, double mm, double n2, double g2, double f2, double *out5);
/* ray ODE right-hand side; y = X Y Z k l m dX dY dZ */
void orc_rhs(const orc_model *m, const double *y9, double *f9);
/* absolute frequency Omega = k.U + w at a point (the ray Hamiltonian) */
double orc_omega(const orc_model *m, double X, double Y, double Z, double k, double l, double mm);
/* one RK3 step of a single ray (no exits/splits); y9 in/out */
void orc_rk3(const orc_model *m, double *y9, double dt);
/* advance one ray by a full step incl. spectral extents: state13 in/out */
void orc_advance_ray(const orc_model *m, double *state13, double dt);
/* per-cell integrated density perturbation P_c and Q_c = sum P_j K_j^2 of the current rays */
int orc_cell_pq(const orc_model *m, double *p_cells, double *q_cells);
/* latitudinal profile alpha(phi) and F_am(phi, tau) of Sec. 3c (phi in degrees) */
double orc_alpha_profile(double phi_deg);
double orc_fam(double phi_deg, double tau, double f_s, double f_w);
/* divergence of given flux fields (layout as orc_get_field) into du/dt, dv/dt */
int orc_divergence(const orc_model *m, const double *fz_l, const double *fz_p,
                   const double *f_ll, const double *f_lp, const double *f_pl, const double *f_pp,
                   const double *e_l, const double *e_p, double *dudt, double *dvdt);
/* horizontal smoothing of one [nlev][ny][nx] field in place */
int orc_smooth(const orc_model *m, double *field, int nlev);
/* wave energy used by the per-column cap: w_hat * N * Px * Py * Pz */
double orc_ray_energy(const orc_model *m, const double *state13);

#ifdef __cplusplus
}
#endif
#endif
