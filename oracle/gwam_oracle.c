/*
 * gwam_oracle.c -- plain FP64 CPU oracle of one MS-GWaM-3D ray-volume step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the
 * CPU-baseline leg of bench.py; never by the library.  It shares nothing with
 * the CUDA path.  Slow on purpose: every quantity is computed where the paper
 * defines it, in the order the paper states it, one ray at a time.
 *
 * Passages followed (Voelker et al., arXiv:2309.11257):
 *   dispersion relation with scale-height correction ......... Sec. 2a, Eq. dispersion
 *   group velocity c_g = grad_k Omega, rdot = c_g ........... Eq. eikonal, Eq. group-velocity
 *   spherical refraction with metric terms ................... Eq. eikonal-sphere:1-3
 *   ray volumes, per-axis phase-space products ................ Sec. 3a, Eq. vpvol_cons_cart, Eq. dkxdkl
 *   face group velocities, Taylor interpolation .............. Sec. 3b, App. B.1
 *   low-storage RK3 (Williamson 1980) ......................... App. B.2
 *   splitting thresholds ...................................... App. B.3
 *   per-column ray cap, lowest energy removed ................. App. B.5
 *   background source alpha(phi), F_sol, F_am ................. Sec. 3c
 *   saturation P, kappa, N -> N(1 - 2 kappa K^2 dt) ............ Sec. 3c, Eq. instability-threshold,
 *                                                                Eq. turbulent-diffusivity
 *   momentum / elastic fluxes ................................. Sec. 2b, Eq. fluxes:momentum,
 *                                                                Eq. fluxes:temperature, Eq. fluxes:buoyancy
 *   pseudomomentum approximation .............................. Sec. 2b, App. A
 *   vertical / horizontal projection .......................... Sec. 3b
 *   flux smoothing ............................................ App. B.4 (lat-lon analogue)
 *   tendencies ................................................ Eq. mean-flow-impact
 *   wave-action budget ........................................ Sec. 4, Eq. wave-action-budget
 *
 * Threads (orc_set_threads, default 1): the independent per-ray work -- the RK3 advance, and the
 * per-ray integrands of saturation and projection -- may run in parallel (OpenMP); every sum,
 * every bookkeeping decision and every id is still taken one ray at a time in array order, so the
 * results are bit-identical for any thread count.  This exists only to time the oracle on all host
 * cores.
 *
 * Where the paper is silent the code states the reading it takes ("Reading:").
 * Readings with no number in the paper (the lat-lon smoothing stencil, the edge
 * gradients and clamps of the gather, the boundary exits, the tie-break of the
 * cap) are pinned to what the reading itself fixes.  Parity unpinned: the
 * omitted curvature terms of the tensor divergence (the paper gives no
 * discrete form to pin the omission against).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#include "gwam_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { SX, SY, SZ, SK, SL, SM, SEX, SEY, SEZ, SPX, SPY, SPZ, SN, NSTATE };
enum { NFIELD_H = 9 };

struct orc_model {
    orc_grid G;
    orc_params P;
    int have_bg;
    double *u, *v, *n2, *rho, *g2;      /* node fields [nz][ny][nx] */
    double *grad[4][3];                  /* node gradients of U V N2 G2 along X Y z [nz][ny][nx] */
    int64_t n, cap;                      /* rays in array order */
    double *s[NSTATE];
    int64_t *id;
    int32_t *cell;
    int64_t next_id;
    orc_stats st;
    double *fz[2];                       /* vertical fluxes at level interfaces [nz+1][ny][nx] */
    double *hf[NFIELD_H];                /* F_ll F_lp F_pl F_pp E_l E_p wave-action density, and the
                                            potential-temperature flux integrals T_l T_p [nz][ny][nx] */
    double *theta;                       /* reference potential temperature [nz][ny][nx], or NULL */
    double *fzabs[2], *hfabs[NFIELD_H];  /* sums of |contribution| of the same fields (error scales) */
    double *n_scale;                     /* per ray: wave-action density before this step's saturation */
    int64_t n_scale_cap;
    int n_scale_valid;                   /* set by apply_saturation, consumed by project */
    int n_scale_current;                 /* n_scale belongs to the current ray array (the last step's
                                            saturation; cleared when rays are added or reordered) */
    int threads;                         /* threads for the per-ray loops (<= 1: serial) */
    long row0, row1;                     /* rows [row0, row1) this model launches into (default all);
                                            a latitude band of a domain-decomposed run */
    int64_t *issued;                     /* issued[q]: new ids issued by rays 0..q-1 of the last advance */
    int64_t issued_n;
};

#ifdef _OPENMP
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static) num_threads(m->threads) if(m->threads > 1)")
#else
#define ORC_PARALLEL_FOR
#endif

/* ------------------------------------------------------------------ geometry */

static int is_sphere(const orc_model *m) { return m->G.geometry == 1; }
static double cell_x(const orc_model *m) { return is_sphere(m) ? 2.0 * M_PI / m->G.nx : m->G.dx; }
static double cell_y(const orc_model *m) { return is_sphere(m) ? M_PI / m->G.ny : m->G.dy; }
static double y_origin(const orc_model *m) { return is_sphere(m) ? -0.5 * M_PI : 0.0; }
static double period_x(const orc_model *m) { return is_sphere(m) ? 2.0 * M_PI : m->G.nx * m->G.dx; }
static double period_y(const orc_model *m) { return m->G.ny * m->G.dy; }
static double z_top(const orc_model *m) { return m->G.nz * m->G.dz; }
static size_t node(const orc_model *m, long k, long j, long i)
{
    return ((size_t)k * m->G.ny + (size_t)j) * m->G.nx + (size_t)i;
}
static double row_lat(const orc_model *m, long j) { return y_origin(m) + (j + 0.5) * cell_y(m); }

/* metric factors of the coordinate extents: dx = hX dX, dy = hY dY (Eq. dkxdkl) */
static void metric(const orc_model *m, double Y, double Z, double *hX, double *hY, double *r)
{
    if (is_sphere(m)) {
        *r = m->G.radius + Z;
        *hX = *r * cos(Y);
        *hY = *r;
    } else {
        *r = 1.0;
        *hX = 1.0;
        *hY = 1.0;
    }
}

static double wrap_period(double x, double L)
{
    double w = x - L * floor(x / L);
    if (w < 0.0) w += L;
    if (w >= L) w = 0.0;
    return w;
}

/* ------------------------------------------------------------------ background */

static long wrap_index(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Bracketing node pair along one axis; s is the position in node units (node q at s = q).
 * Reading (App. B.1 gives the interpolation, not the edges): outside the first/last node
 * every interpolated quantity is held at its edge-node value. */
static void bracket(double s, long n, int periodic, long *q0, long *q1, double *t)
{
    if (!isfinite(s)) s = 0.0;
    if (periodic) {
        s = s - (double)n * floor(s / (double)n);
        double fl = floor(s);
        *t = s - fl;
        *q0 = wrap_index((long)fl, n);
        *q1 = wrap_index(*q0 + 1, n);
    } else if (s < 0.0) {
        *q0 = 0; *q1 = 1; *t = 0.0;
    } else if (s >= (double)(n - 1)) {
        *q0 = n - 2; *q1 = n - 1; *t = 1.0;
    } else {
        double fl = floor(s);
        *q0 = (long)fl; *q1 = *q0 + 1; *t = s - fl;
    }
}

/* Linear interpolation of the mean fields and of their gradients to a point (Sec. 3b, App. B.1:
 * "all necessary mean fields and their gradients" are interpolated).  Reading on a lat-lon grid:
 * gradients live on the nodes (cell centres) as centred differences, and values and gradients
 * are interpolated trilinearly from the 8 bracketing nodes, so both are continuous in position.
 * Gradients are per unit of coordinate (radian on the sphere, metre otherwise). */
void orc_gather(const orc_model *m, double X, double Y, double Z, double *o)
{
    long i0, i1, j0, j1, k0, k1;
    double tx, ty, tz;
    double dX = cell_x(m), dY = cell_y(m), dz = m->G.dz;
    bracket(X / dX - 0.5, m->G.nx, 1, &i0, &i1, &tx);
    bracket((Y - y_origin(m)) / dY - 0.5, m->G.ny, !is_sphere(m), &j0, &j1, &ty);
    bracket(Z / dz - 0.5, m->G.nz, 0, &k0, &k1, &tz);
    const double *F[16];
    F[0] = m->u; F[1] = m->v; F[2] = m->n2; F[3] = m->g2;
    for (int f = 0; f < 4; ++f)
        for (int q = 0; q < 3; ++q) F[4 + 3 * f + q] = m->grad[f][q];
    long I[2] = {i0, i1}, J[2] = {j0, j1}, K[2] = {k0, k1};
    double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
    for (int f = 0; f < 16; ++f) {
        double val = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) val += wx[a] * wy[b] * wz[e] * F[f][node(m, K[e], J[b], I[a])];
        o[f] = val;
    }
}

/* f^2 and d(f^2)/dphi at latitude Y; f = 2 Omega sin(phi) on the sphere (Sec. 2a) */
static void coriolis(const orc_model *m, double Y, double *f2, double *df2)
{
    if (is_sphere(m)) {
        double f = 2.0 * m->G.omega * sin(Y);
        *f2 = f * f;
        *df2 = 8.0 * m->G.omega * m->G.omega * sin(Y) * cos(Y);
    } else {
        *f2 = m->G.f0 * m->G.f0;
        *df2 = 0.0;
    }
}

/* ------------------------------------------------------------------ dispersion (Eq. dispersion) */

typedef struct {
    double kh2, mg2, K2, D, w2, w, ch[3];
} disp_t;

/* Positive intrinsic branch of Eq. dispersion:
 *   w^2 = (f^2 (m^2 + Gamma^2) + N^2 (k^2 + l^2)) / K^2,  K^2 = k.k + Gamma^2,
 * and the intrinsic group velocity ch = grad_k w (Eq. eikonal), differentiated by hand:
 *   ch_x = k (N^2 - f^2)(m^2 + Gamma^2) / (w K^4), ch_y likewise with l,
 *   ch_r = -m (N^2 - f^2)(k^2 + l^2) / (w K^4). */
static void dispersion(double k, double l, double mm, double n2, double g2, double f2, disp_t *d)
{
    d->kh2 = k * k + l * l;
    d->mg2 = mm * mm + g2;
    d->K2 = d->kh2 + d->mg2;
    d->D = n2 - f2;
    d->w2 = (f2 * d->mg2 + n2 * d->kh2) / d->K2;
    d->w = sqrt(d->w2);
    d->ch[0] = k * d->D * d->mg2 / (d->w * d->K2 * d->K2);
    d->ch[1] = l * d->D * d->mg2 / (d->w * d->K2 * d->K2);
    d->ch[2] = -mm * d->D * d->kh2 / (d->w * d->K2 * d->K2);
}

void orc_dispersion(double k, double l, double mm, double n2, double g2, double f2, double *out)
{
    disp_t d;
    dispersion(k, l, mm, n2, g2, f2, &d);
    out[0] = d.w;
    out[1] = d.ch[0];
    out[2] = d.ch[1];
    out[3] = d.ch[2];
    out[4] = d.K2;
}

double orc_omega(const orc_model *m, double X, double Y, double Z, double k, double l, double mm)
{
    double b[16], f2, df2;
    disp_t d;
    orc_gather(m, X, Y, Z, b);
    coriolis(m, Y, &f2, &df2);
    dispersion(k, l, mm, b[2], b[3], f2, &d);
    return k * b[0] + l * b[1] + d.w;
}

/* ------------------------------------------------------------------ ray equations */

/* Right-hand side of the ray-volume equations for y = (X, Y, Z, k, l, m, dX, dY, dZ).
 *  - background and gradients at the carrier ray (App. B.1)
 *  - wavenumber tendencies with the centre values, Eq. eikonal-sphere:1-3 on the sphere,
 *    kdot = -grad Omega on the f-plane (Eq. eikonal)
 *  - group velocities at the six face centres from first-order Taylor values
 *    chi_face = chi + grad chi . (r_face - r) (App. B.1); the face mean advances the
 *    carrier, the face difference is the extent rate (Sec. 3b, App. B.1). */
static void rhs_mode(const orc_model *m, const double *y, double *F, int columnar)
{
    double X = y[0], Y = y[1], Z = y[2], k = y[3], l = y[4], mm = y[5];
    double ext[3] = {y[6], y[7], y[8]};
    double b[16];
    orc_gather(m, X, Y, Z, b);
    double U = b[0], V = b[1], N2 = b[2], G2 = b[3];
    const double *dU = b + 4, *dV = b + 7, *dN2 = b + 10, *dG2 = b + 13;
    double f2, df2;
    coriolis(m, Y, &f2, &df2);
    double df2v[3] = {0.0, df2, 0.0};
    double hX, hY, r;
    metric(m, Y, Z, &hX, &hY, &r);

    disp_t d;
    dispersion(k, l, mm, N2, G2, f2, &d);
    double cg[3] = {d.ch[0] + U, d.ch[1] + V, d.ch[2]};   /* c_g = ch + U */

    /* derivative of Omega along coordinate q at fixed wavevector */
    double G[3];
    for (int q = 0; q < 3; ++q) {
        G[q] = k * dU[q] + l * dV[q]
             + d.kh2 / (2.0 * d.w * d.K2) * (dN2[q] - d.D / d.K2 * dG2[q])
             + d.mg2 / (2.0 * d.w * d.K2) * df2v[q];
    }
    if (columnar) {
        /* single-column approximation (MS-GWaM-1D, Sec. 1): horizontal gradients of the resolved
         * flow are neglected, so k and l stay fixed and m follows the vertical gradient alone */
        F[3] = 0.0;
        F[4] = 0.0;
        F[5] = -G[2];
    } else if (is_sphere(m)) {
        double tphi = tan(Y);
        F[3] = -G[0] / hX - k * cg[2] / r + k * tphi * cg[1] / r;   /* Eq. eikonal-sphere:1 */
        F[4] = -G[1] / r - l * cg[2] / r - k * tphi * cg[0] / r;    /* Eq. eikonal-sphere:2 */
        F[5] = -G[2] + k * cg[0] / r + l * cg[1] / r;               /* Eq. eikonal-sphere:3 */
    } else {
        F[3] = -G[0];
        F[4] = -G[1];
        F[5] = -G[2];
    }

    for (int q = 0; q < 3; ++q) {
        if (columnar && q < 2) {
            /* no horizontal propagation or advection: position and horizontal extents fixed */
            F[q] = 0.0;
            F[6 + q] = 0.0;
            continue;
        }
        double vel[2];
        for (int side = 0; side < 2; ++side) {
            double h = (side == 0 ? 0.5 : -0.5) * ext[q];
            double Uf = U + dU[q] * h;
            double Vf = V + dV[q] * h;
            double N2f = N2 + dN2[q] * h;
            double G2f = G2 + dG2[q] * h;
            double f2f = f2 + df2v[q] * h;
            disp_t e;
            dispersion(k, l, mm, N2f, G2f, f2f, &e);
            if (q == 0) vel[side] = (e.ch[0] + Uf) / hX;
            else if (q == 1) vel[side] = (e.ch[1] + Vf) / hY;
            else vel[side] = e.ch[2];
        }
        F[q] = 0.5 * (vel[0] + vel[1]);
        F[6 + q] = vel[0] - vel[1];
    }
}

void orc_rhs(const orc_model *m, const double *y, double *F)
{
    rhs_mode(m, y, F, m->P.columnar);
}

/* Williamson (1980) low-storage third-order Runge-Kutta, background frozen over the step
 * (App. B.2; the coefficients are the published ones of that scheme).  columnar != 0 integrates
 * the single-column form whatever the model's mode (the ghost layer of the launch). */
static void rk3_mode(const orc_model *m, double *y, double dt, int columnar)
{
    static const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
    static const double B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    double q[9] = {0}, F[9];
    for (int s = 0; s < 3; ++s) {
        rhs_mode(m, y, F, columnar);
        for (int c = 0; c < 9; ++c) q[c] = A[s] * q[c] + dt * F[c];
        for (int c = 0; c < 9; ++c) y[c] += B[s] * q[c];
    }
}

void orc_rk3(const orc_model *m, double *y, double dt)
{
    rk3_mode(m, y, dt, m->P.columnar);
}

static void wrap_position(const orc_model *m, double *s)
{
    s[SX] = wrap_period(s[SX], period_x(m));
    if (!is_sphere(m)) s[SY] = wrap_period(s[SY], period_y(m));
}

void orc_advance_ray(const orc_model *m, double *s, double dt)
{
    orc_rk3(m, s, dt);
    wrap_position(m, s);
}

/* spectral extents from the conserved products (Eq. vpvol_cons_cart, Eq. dkxdkl) */
static void spectral_extents(const orc_model *m, const double *s, double *dk, double *dl, double *dm)
{
    double hX, hY, r;
    metric(m, s[SY], s[SZ], &hX, &hY, &r);
    *dk = s[SPX] / (hX * s[SEX]);
    *dl = s[SPY] / (hY * s[SEY]);
    *dm = s[SPZ] / s[SEZ];
}

static double physical_volume(const orc_model *m, const double *s)
{
    double hX, hY, r;
    metric(m, s[SY], s[SZ], &hX, &hY, &r);
    return hX * s[SEX] * hY * s[SEY] * s[SEZ];
}

/* wave action content of a ray volume: N times its 6-D volume = N Px Py Pz */
static double ray_action(const double *s) { return s[SN] * s[SPX] * s[SPY] * s[SPZ]; }

/* 0 = inside, 1 = left the domain, 2 = not a valid ray volume any more.
 * Reading: a carrier at z < 0, z >= z_top, or poleward of the centre of the last row leaves. */
static int ray_status(const orc_model *m, const double *s)
{
    for (int c = 0; c < NSTATE; ++c)
        if (!isfinite(s[c])) return 2;
    if (!(s[SEX] > 0.0 && s[SEY] > 0.0 && s[SEZ] > 0.0)) return 2;
    if (!(s[SZ] >= 0.0 && s[SZ] < z_top(m))) return 1;
    if (is_sphere(m)) {
        double phimax = 0.5 * M_PI - 0.5 * cell_y(m);
        if (!(fabs(s[SY]) <= phimax)) return 1;
    }
    return 0;
}

static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void cell_ijk(const orc_model *m, const double *s, long *i, long *j, long *k)
{
    *i = clampl((long)floor(s[SX] / cell_x(m)), 0, m->G.nx - 1);
    *j = clampl((long)floor((s[SY] - y_origin(m)) / cell_y(m)), 0, m->G.ny - 1);
    *k = clampl((long)floor(s[SZ] / m->G.dz), 0, m->G.nz - 1);
}

static int32_t cell_of(const orc_model *m, const double *s)
{
    long i, j, k;
    cell_ijk(m, s, &i, &j, &k);
    return (int32_t)(((long)j * m->G.nx + i) * m->G.nz + k);
}

/* ------------------------------------------------------------------ model */

static void free_fields(orc_model *m)
{
    free(m->fz[0]); free(m->fz[1]);
    free(m->fzabs[0]); free(m->fzabs[1]);
    for (int f = 0; f < NFIELD_H; ++f) {
        free(m->hf[f]);
        free(m->hfabs[f]);
    }
}

orc_model *orc_create(const orc_grid *grid, const orc_params *params)
{
    if (!grid || !params) return NULL;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || !(grid->dz > 0.0)) return NULL;
    if (grid->geometry == 0 && !(grid->dx > 0.0 && grid->dy > 0.0)) return NULL;
    if (grid->geometry == 1 && !(grid->radius > 0.0)) return NULL;
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    m->G = *grid;
    m->P = *params;
    m->row0 = 0;
    m->row1 = grid->ny;
    size_t nc = (size_t)grid->nx * grid->ny * grid->nz;
    size_t ni = (size_t)grid->nx * grid->ny * (grid->nz + 1);
    m->u = calloc(nc, sizeof(double));
    m->v = calloc(nc, sizeof(double));
    m->n2 = calloc(nc, sizeof(double));
    m->rho = calloc(nc, sizeof(double));
    m->g2 = calloc(nc, sizeof(double));
    for (int f = 0; f < 4; ++f)
        for (int q = 0; q < 3; ++q) m->grad[f][q] = calloc(nc, sizeof(double));
    m->fz[0] = calloc(ni, sizeof(double));
    m->fz[1] = calloc(ni, sizeof(double));
    m->fzabs[0] = calloc(ni, sizeof(double));
    m->fzabs[1] = calloc(ni, sizeof(double));
    for (int f = 0; f < NFIELD_H; ++f) {
        m->hf[f] = calloc(nc, sizeof(double));
        m->hfabs[f] = calloc(nc, sizeof(double));
    }
    return m;
}

static void free_rays(orc_model *m)
{
    for (int c = 0; c < NSTATE; ++c) free(m->s[c]);
    free(m->id);
    free(m->cell);
}

void orc_destroy(orc_model *m)
{
    if (!m) return;
    free(m->u); free(m->v); free(m->n2); free(m->rho); free(m->g2);
    for (int f = 0; f < 4; ++f)
        for (int q = 0; q < 3; ++q) free(m->grad[f][q]);
    free_fields(m);
    free_rays(m);
    free(m->n_scale);
    free(m->issued);
    free(m->theta);
    free(m);
}

/* Reading for the scale-height correction Gamma (Sec. 2a names it, never defines it):
 * Gamma^2 = 1 / (4 H_rho^2) with 1/H_rho = -d ln(rho)/dz, discretised by centred
 * differences of ln(rho) between node levels (one-sided at the bottom and top). */
int orc_set_background(orc_model *m, const double *u, const double *v, const double *n2, const double *rho)
{
    long nx = m->G.nx, ny = m->G.ny, nz = m->G.nz;
    size_t nc = (size_t)nx * ny * nz;
    for (size_t q = 0; q < nc; ++q) {
        if (!isfinite(u[q]) || !isfinite(v[q]) || !isfinite(n2[q]) || !isfinite(rho[q])) return -4;
        if (!(rho[q] > 0.0)) return -1;
    }
    memcpy(m->u, u, nc * sizeof(double));
    memcpy(m->v, v, nc * sizeof(double));
    memcpy(m->n2, n2, nc * sizeof(double));
    memcpy(m->rho, rho, nc * sizeof(double));
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double dlnr;
                if (k == 0) dlnr = (log(rho[node(m, 1, j, i)]) - log(rho[node(m, 0, j, i)])) / m->G.dz;
                else if (k == nz - 1)
                    dlnr = (log(rho[node(m, nz - 1, j, i)]) - log(rho[node(m, nz - 2, j, i)])) / m->G.dz;
                else
                    dlnr = (log(rho[node(m, k + 1, j, i)]) - log(rho[node(m, k - 1, j, i)])) / (2.0 * m->G.dz);
                m->g2[node(m, k, j, i)] = m->P.gamma_mode ? 0.25 * dlnr * dlnr : 0.0;
            }
    /* node gradients: centred differences, periodic in x (and y on the f-plane), one-sided at
     * the pole rows and at the bottom and top levels */
    const double *Fv[4] = {m->u, m->v, m->n2, m->g2};
    double dX = cell_x(m), dY = cell_y(m), dz = m->G.dz;
    for (int f = 0; f < 4; ++f)
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j)
                for (long i = 0; i < nx; ++i) {
                    const double *A = Fv[f];
                    size_t c = node(m, k, j, i);
                    m->grad[f][0][c] = (A[node(m, k, j, wrap_index(i + 1, nx))] - A[node(m, k, j, wrap_index(i - 1, nx))])
                                     / (2.0 * dX);
                    if (!is_sphere(m))
                        m->grad[f][1][c] = (A[node(m, k, wrap_index(j + 1, ny), i)]
                                            - A[node(m, k, wrap_index(j - 1, ny), i)]) / (2.0 * dY);
                    else if (j == 0)
                        m->grad[f][1][c] = (A[node(m, k, 1, i)] - A[node(m, k, 0, i)]) / dY;
                    else if (j == ny - 1)
                        m->grad[f][1][c] = (A[node(m, k, ny - 1, i)] - A[node(m, k, ny - 2, i)]) / dY;
                    else
                        m->grad[f][1][c] = (A[node(m, k, j + 1, i)] - A[node(m, k, j - 1, i)]) / (2.0 * dY);
                    if (k == 0)
                        m->grad[f][2][c] = (A[node(m, 1, j, i)] - A[node(m, 0, j, i)]) / dz;
                    else if (k == nz - 1)
                        m->grad[f][2][c] = (A[node(m, nz - 1, j, i)] - A[node(m, nz - 2, j, i)]) / dz;
                    else
                        m->grad[f][2][c] = (A[node(m, k + 1, j, i)] - A[node(m, k - 1, j, i)]) / (2.0 * dz);
                }
    m->have_bg = 1;
    return 0;
}

int orc_get_gamma2(const orc_model *m, double *out)
{
    memcpy(out, m->g2, (size_t)m->G.nx * m->G.ny * m->G.nz * sizeof(double));
    return 0;
}

static void reserve(orc_model *m, int64_t need)
{
    if (need <= m->cap) return;
    int64_t nc = m->cap ? m->cap : 1024;
    while (nc < need) nc *= 2;
    for (int c = 0; c < NSTATE; ++c) m->s[c] = realloc(m->s[c], (size_t)nc * sizeof(double));
    m->id = realloc(m->id, (size_t)nc * sizeof(int64_t));
    m->cell = realloc(m->cell, (size_t)nc * sizeof(int32_t));
    m->cap = nc;
}

static void append_ray(orc_model *m, const double *s, int64_t id)
{
    m->n_scale_current = 0;
    reserve(m, m->n + 1);
    for (int c = 0; c < NSTATE; ++c) m->s[c][m->n] = s[c];
    m->id[m->n] = id;
    m->cell[m->n] = cell_of(m, s);
    m->n++;
}

static void load_ray(const orc_model *m, int64_t i, double *s)
{
    for (int c = 0; c < NSTATE; ++c) s[c] = m->s[c][i];
}

/* ray volume from its extents and spectral widths: P_x = hX dX dk, P_y = hY dY dl, P_z = dZ dm */
static void make_ray(const orc_model *m, double X, double Y, double Z, double k, double l, double mm,
                     double eX, double eY, double eZ, double dk, double dl, double dm, double nn, double *s)
{
    double hX, hY, r;
    metric(m, Y, Z, &hX, &hY, &r);
    s[SX] = X; s[SY] = Y; s[SZ] = Z;
    s[SK] = k; s[SL] = l; s[SM] = mm;
    s[SEX] = eX; s[SEY] = eY; s[SEZ] = eZ;
    s[SPX] = hX * eX * dk;
    s[SPY] = hY * eY * dl;
    s[SPZ] = eZ * dm;
    s[SN] = nn;
}

int orc_add_rays(orc_model *m, int64_t n, const double *x, const double *y, const double *z,
                 const double *k, const double *l, const double *mm,
                 const double *ex, const double *ey, const double *ez,
                 const double *dk, const double *dl, const double *dm, const double *nn)
{
    for (int64_t q = 0; q < n; ++q) {
        double s[NSTATE];
        make_ray(m, x[q], y[q], z[q], k[q], l[q], mm[q], ex[q], ey[q], ez[q], dk[q], dl[q], dm[q], nn[q], s);
        wrap_position(m, s);
        if (ray_status(m, s) != 0) return -1;
        append_ray(m, s, m->next_id++);
        m->st.n_launched++;
        m->st.w_launched += ray_action(s);
        m->st.w_total += ray_action(s);
    }
    m->st.n_live = m->n;
    return 0;
}

/* ------------------------------------------------------------------ sources (Sec. 3c) */

/* latitudinal profile alpha(phi) of the background source, phi in degrees north */
double orc_alpha_profile(double p)
{
    if (p >= 80.0) return fmin(1.0, fmax(0.0, 1.0 - (p - 80.0) / 5.0));
    if (p >= 50.0) return 1.0;
    if (p >= 20.0) return 0.5 * (1.0 - cos(M_PI * (p - 20.0) / 30.0));
    return 0.0;
}

/* F_sol(phi) = alpha(phi) F_s + alpha(-phi) F_w and its seasonal cycle F_am(phi, tau) */
double orc_fam(double p, double tau, double f_s, double f_w)
{
    double fsol_p = orc_alpha_profile(p) * f_s + orc_alpha_profile(-p) * f_w;
    double fsol_m = orc_alpha_profile(-p) * f_s + orc_alpha_profile(p) * f_w;
    return 0.5 * (fsol_p * (1.0 + cos(tau)) + fsol_m * (1.0 - cos(tau)));
}

/* One spectral ray volume at the centre of column (i, j), its slab [z_launch, z_launch + dz_launch].
 * Reading (Sec. 3c cites the spectrum, not its form): a monochromatic bin of horizontal
 * wavelength lambda_h, azimuth theta and ground-based phase speed c; the intrinsic frequency
 * w = |k_h| c - k.U must satisfy |f| < w < N, and m follows from inverting Eq. dispersion,
 * m^2 = k_h^2 (N^2 - w^2) / (w^2 - f^2) - Gamma^2, with m < 0 (upward group velocity).
 * The bin carries the pseudomomentum flux F = |k_h| ch_r A through the launch level. */
static int launch_state(orc_model *m, long i, long j, double z_launch, double dz_launch, double theta,
                        double c, double lambda_h, double flux, double frac, double *s)
{
    double X = (i + 0.5) * cell_x(m);
    double Y = row_lat(m, j);
    double Z = z_launch + 0.5 * dz_launch;
    double b[16], f2, df2;
    orc_gather(m, X, Y, Z, b);
    coriolis(m, Y, &f2, &df2);
    double U = b[0], V = b[1], N2 = b[2], G2 = b[3];
    double kh = 2.0 * M_PI / lambda_h;
    double k = kh * cos(theta), l = kh * sin(theta);
    double w = kh * c - (k * U + l * V);
    if (!(w > 0.0 && w * w > f2 && w * w < N2)) {
        m->st.n_filtered++;
        return 0;
    }
    double m2 = kh * kh * (N2 - w * w) / (w * w - f2) - G2;
    if (!(m2 > 0.0)) {
        m->st.n_filtered++;
        return 0;
    }
    double mm = -sqrt(m2);
    disp_t d;
    dispersion(k, l, mm, N2, G2, f2, &d);
    double A = flux / (kh * d.ch[2]);
    double dk = frac * kh, dl = frac * kh, dm = frac * fabs(mm);
    make_ray(m, X, Y, Z, k, l, mm, cell_x(m), cell_y(m), dz_launch, dk, dl, dm, A / (dk * dl * dm), s);
    if (ray_status(m, s) != 0) {
        m->st.n_filtered++;
        return 0;
    }
    return 1;
}

static void activate(orc_model *m, const double *s)
{
    append_ray(m, s, m->next_id++);
    m->st.n_launched++;
    m->st.w_launched += ray_action(s);
    m->st.w_total += ray_action(s);
}

static int launch_one(orc_model *m, long i, long j, double z_launch, double dz_launch, double theta,
                      double c, double lambda_h, double flux, double frac)
{
    double s[NSTATE];
    if (!launch_state(m, i, j, z_launch, dz_launch, theta, c, lambda_h, flux, frac, s)) return 0;
    activate(m, s);
    return 1;
}

/* Ghost-layer launch (Sec. 3c): a ghost ray volume fills the launch layer [z_launch, z_launch +
 * dz_launch] in the launch state of the bin and propagates vertically only (the single-column
 * equations) over one launch interval dt.  The part of it above the layer top is separated and
 * activated: same N, wavevector and horizontal extents, vertical extent from the layer top (or its
 * own bottom, if it left the layer whole) to its top, and the vertical phase-space product in
 * proportion, P_z = P_z,ghost * extent / dZ_ghost.  A ghost volume reflected within the layer
 * (m no longer negative: downward group velocity) is discarded and counted as filtered. */
static int ghost_one(orc_model *m, long i, long j, double z_launch, double dz_launch, double theta,
                     double c, double lambda_h, double flux, double frac, double dt)
{
    double s[NSTATE];
    if (!launch_state(m, i, j, z_launch, dz_launch, theta, c, lambda_h, flux, frac, s)) return 0;
    double y[9];
    memcpy(y, s, sizeof(y));
    rk3_mode(m, y, dt, 1);
    if (!(y[SM] < 0.0)) {
        m->st.n_filtered++;
        return 0;
    }
    double layer_top = z_launch + dz_launch;
    double top = y[SZ] + 0.5 * y[SEZ], bot = y[SZ] - 0.5 * y[SEZ];
    if (!(top > layer_top)) return 0;                  /* nothing has left the layer */
    double lo = bot > layer_top ? bot : layer_top;
    double e[NSTATE];
    memcpy(e, s, sizeof(e));
    e[SM] = y[SM];
    e[SZ] = 0.5 * (lo + top);
    e[SEZ] = top - lo;
    e[SPZ] = s[SPZ] * e[SEZ] / y[SEZ];
    if (ray_status(m, e) != 0) {
        m->st.n_filtered++;
        return 0;
    }
    activate(m, e);
    return 1;
}

/* dt > 0: ghost-layer emission over one launch interval; dt == 0: activate the launch states */
static int launch_background_dt(orc_model *m, const orc_bg_source *src, double dt)
{
    if (!is_sphere(m) || !m->have_bg) return -1;
    if (src->n_az < 1 || src->n_c < 1) return -1;
    int nbins = src->n_az * src->n_c;
    for (long j = m->row0; j < m->row1; ++j) {
        double pdeg = row_lat(m, j) * 180.0 / M_PI;
        if (fabs(pdeg) > src->phi_max_deg) continue;      /* no launch poleward of 85 deg */
        double fbin = orc_fam(pdeg, src->tau, src->f_s, src->f_w) / nbins;
        if (fbin == 0.0 && !src->launch_zero_flux) continue;
        for (long i = 0; i < m->G.nx; ++i)
            for (int a = 0; a < src->n_az; ++a)
                for (int q = 0; q < src->n_c; ++q) {
                    double theta = 2.0 * M_PI * a / src->n_az;
                    double c = src->n_c == 1 ? src->c_min
                             : src->c_min * pow(src->c_max / src->c_min, (double)q / (src->n_c - 1));
                    if (dt > 0.0)
                        ghost_one(m, i, j, src->z_launch, src->dz_launch, theta, c, src->lambda_h, fbin,
                                  src->spectral_frac, dt);
                    else
                        launch_one(m, i, j, src->z_launch, src->dz_launch, theta, c, src->lambda_h, fbin,
                                   src->spectral_frac);
                }
    }
    m->st.n_live = m->n;
    return 0;
}

int orc_launch_background(orc_model *m, const orc_bg_source *src)
{
    return launch_background_dt(m, src, 0.0);
}

int orc_launch_ghost(orc_model *m, const orc_bg_source *src, double dt)
{
    if (!(dt > 0.0)) return -1;
    return launch_background_dt(m, src, dt);
}

static int launch_spectral_dt(orc_model *m, int64_t n, const orc_spec *sp, double dt)
{
    if (!m->have_bg) return -1;
    for (int64_t q = 0; q < n; ++q)
        if (sp[q].i < 0 || sp[q].i >= m->G.nx || sp[q].j < 0 || sp[q].j >= m->G.ny) return -1;
    for (int64_t q = 0; q < n; ++q) {
        if (sp[q].j < m->row0 || sp[q].j >= m->row1) continue;     /* another band's column */
        if (dt > 0.0)
            ghost_one(m, sp[q].i, sp[q].j, sp[q].z_launch, sp[q].dz_launch, sp[q].theta, sp[q].c,
                      sp[q].lambda_h, sp[q].flux, sp[q].spectral_frac, dt);
        else
            launch_one(m, sp[q].i, sp[q].j, sp[q].z_launch, sp[q].dz_launch, sp[q].theta, sp[q].c,
                       sp[q].lambda_h, sp[q].flux, sp[q].spectral_frac);
    }
    m->st.n_live = m->n;
    return 0;
}

int orc_launch_spectral(orc_model *m, int64_t n, const orc_spec *sp)
{
    return launch_spectral_dt(m, n, sp, 0.0);
}

int orc_launch_ghost_spectral(orc_model *m, int64_t n, const orc_spec *sp, double dt)
{
    if (!(dt > 0.0)) return -1;
    return launch_spectral_dt(m, n, sp, dt);
}

/* ------------------------------------------------------------------ splitting (App. B.3) */

static void halve(double *s, int axis, int plus)
{
    int e = SEX + axis, p = SPX + axis, x = SX + axis;
    s[x] += (plus ? 0.25 : -0.25) * s[e];
    s[e] *= 0.5;
    s[p] *= 0.5;
}

/* Split the ray volume in s into up to four; returns the count, children in out[] with ids.
 * Vertical: dZ > max(alpha_s h_c, 1 km).  Horizontal: cos(phi) dX or dY above alpha_s sqrt(a_c)/R,
 * or cos(phi) dX dY above alpha_s a_c / R^2, split along the larger of cos(phi) dX and dY.
 * Reading: at most one split per axis per step, vertical first; halves sit at +-1/4 of the
 * extent; the lower/minus half keeps the parent id, new ids are issued in array order. */
static int split_ray(orc_model *m, const double *s, int64_t id, double out[4][NSTATE], int64_t oid[4])
{
    int n = 1;
    memcpy(out[0], s, sizeof(double) * NSTATE);
    oid[0] = id;
    if (!m->P.splitting) return 1;
    long ci, cj, ck;
    cell_ijk(m, s, &ci, &cj, &ck);
    double hthr = fmax(m->P.alpha_s * m->G.dz, m->P.min_split_dz);
    if (s[SEZ] > hthr) {
        memcpy(out[1], s, sizeof(double) * NSTATE);
        halve(out[0], 2, 0);
        halve(out[1], 2, 1);
        oid[1] = m->next_id++;
        n = 2;
        m->st.n_split_v++;
    }
    double xlen, ylen, thr, area, athr;
    double dX = cell_x(m), dY = cell_y(m);
    if (is_sphere(m)) {
        double cj_ = cos(row_lat(m, cj));
        xlen = cos(s[SY]) * s[SEX];
        ylen = s[SEY];
        thr = m->P.alpha_s * sqrt(cj_ * dX * dY);
        area = cos(s[SY]) * s[SEX] * s[SEY];
        athr = m->P.alpha_s * cj_ * dX * dY;
    } else {
        xlen = s[SEX];
        ylen = s[SEY];
        thr = m->P.alpha_s * sqrt(dX * dY);
        area = s[SEX] * s[SEY];
        athr = m->P.alpha_s * dX * dY;
    }
    if (xlen > thr || ylen > thr || area > athr) {
        int axis = (xlen >= ylen) ? 0 : 1;
        for (int c = 0; c < n; ++c) {
            memcpy(out[n + c], out[c], sizeof(double) * NSTATE);
            halve(out[c], axis, 0);
            halve(out[n + c], axis, 1);
            oid[n + c] = m->next_id++;
            m->st.n_split_h++;
        }
        n *= 2;
    }
    for (int c = 0; c < n; ++c) wrap_position(m, out[c]);
    return n;
}

/* ------------------------------------------------------------------ ordering */

typedef struct {
    int32_t cell;
    int64_t id;
    int64_t src;
} key_t_;

static int cmp_key(const void *a, const void *b)
{
    const key_t_ *x = (const key_t_ *)a, *y = (const key_t_ *)b;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* put the rays into the canonical order: ascending (cell, id) */
static void sort_rays(orc_model *m)
{
    int64_t n = m->n;
    m->n_scale_current = 0;
    key_t_ *key = malloc(sizeof(key_t_) * (size_t)(n ? n : 1));
    for (int64_t q = 0; q < n; ++q) {
        double s[NSTATE];
        load_ray(m, q, s);
        key[q].cell = cell_of(m, s);
        key[q].id = m->id[q];
        key[q].src = q;
    }
    qsort(key, (size_t)n, sizeof(key_t_), cmp_key);
    double *ns[NSTATE];
    for (int c = 0; c < NSTATE; ++c) ns[c] = malloc(sizeof(double) * (size_t)(n ? n : 1));
    int64_t *nid = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    for (int64_t q = 0; q < n; ++q) {
        for (int c = 0; c < NSTATE; ++c) ns[c][q] = m->s[c][key[q].src];
        nid[q] = key[q].id;
        m->cell[q] = key[q].cell;
    }
    for (int c = 0; c < NSTATE; ++c) {
        memcpy(m->s[c], ns[c], sizeof(double) * (size_t)n);
        free(ns[c]);
    }
    memcpy(m->id, nid, sizeof(int64_t) * (size_t)n);
    free(nid);
    free(key);
}

/* ------------------------------------------------------------------ intrinsic properties at a ray */

static void ray_disp(const orc_model *m, const double *s, disp_t *d, double *f2, double *n2)
{
    double b[16], df2;
    orc_gather(m, s[SX], s[SY], s[SZ], b);
    coriolis(m, s[SY], f2, &df2);
    *n2 = b[2];
    dispersion(s[SK], s[SL], s[SM], b[2], b[3], *f2, d);
}

/* wave energy of a ray volume = intrinsic frequency times its wave action */
double orc_ray_energy(const orc_model *m, const double *s)
{
    disp_t d;
    double f2, n2;
    ray_disp(m, s, &d, &f2, &n2);
    return d.w * ray_action(s);
}

/* ------------------------------------------------------------------ per-column cap (App. B.5) */

typedef struct {
    double e;
    int64_t id;
    int64_t idx;
} ekey_t;

static int cmp_energy(const void *a, const void *b)
{
    const ekey_t *x = (const ekey_t *)a, *y = (const ekey_t *)b;
    if (x->e != y->e) return x->e < y->e ? -1 : 1;
    if (x->id != y->id) return x->id > y->id ? -1 : 1;   /* tie: larger id removed first */
    return 0;
}

static void apply_cap(orc_model *m)
{
    int cap = m->P.cap_per_column;
    if (cap <= 0 || m->n == 0) return;
    char *dead = calloc((size_t)m->n, 1);
    int64_t a = 0;
    while (a < m->n) {
        int32_t col = m->cell[a] / m->G.nz;
        int64_t b = a;
        while (b < m->n && m->cell[b] / m->G.nz == col) ++b;
        int64_t cnt = b - a;
        if (cnt > cap) {
            ekey_t *ek = malloc(sizeof(ekey_t) * (size_t)cnt);
            for (int64_t q = a; q < b; ++q) {
                double s[NSTATE];
                load_ray(m, q, s);
                ek[q - a].e = orc_ray_energy(m, s);
                ek[q - a].id = m->id[q];
                ek[q - a].idx = q;
            }
            qsort(ek, (size_t)cnt, sizeof(ekey_t), cmp_energy);
            for (int64_t q = 0; q < cnt - cap; ++q) {
                double s[NSTATE];
                load_ray(m, ek[q].idx, s);
                dead[ek[q].idx] = 1;
                m->st.n_capped++;
                m->st.w_capped += ray_action(s);
            }
            free(ek);
        }
        a = b;
    }
    int64_t w = 0;
    for (int64_t q = 0; q < m->n; ++q) {
        if (dead[q]) continue;
        for (int c = 0; c < NSTATE; ++c) m->s[c][w] = m->s[c][q];
        m->id[w] = m->id[q];
        m->cell[w] = m->cell[q];
        ++w;
    }
    m->n = w;
    free(dead);
}

/* ------------------------------------------------------------------ saturation (Sec. 3c) */

/* volume of grid cell (i, j, k): a_c h_c with a_c = r_c^2 cos(phi_j) dlambda dphi on the sphere */
static double cell_volume(const orc_model *m, long j, long k)
{
    if (is_sphere(m)) {
        double rc = m->G.radius + (k + 0.5) * m->G.dz;
        return rc * rc * cos(row_lat(m, j)) * cell_x(m) * cell_y(m) * m->G.dz;
    }
    return m->G.dx * m->G.dy * m->G.dz;
}

/* per-ray saturation quantities: P_j = m^2 |k_h|^2 / (w K^2) A_j alpha_j (Eq. instability-threshold
 * and the discrete sum that follows it), with A_j = N dk dl dm and alpha_j = V_j / V_c */
static void ray_p(const orc_model *m, const double *s, long j, long k, double *pj, double *K2)
{
    disp_t d;
    double f2, n2, dk, dl, dm;
    ray_disp(m, s, &d, &f2, &n2);
    spectral_extents(m, s, &dk, &dl, &dm);
    double A = s[SN] * dk * dl * dm;
    double alpha = physical_volume(m, s) / cell_volume(m, j, k);
    *pj = s[SM] * s[SM] * d.kh2 / (d.w * d.K2) * A * alpha;
    *K2 = d.K2;
}

int orc_cell_pq(const orc_model *m, double *p_cells, double *q_cells)
{
    size_t nc = (size_t)m->G.nx * m->G.ny * m->G.nz;
    memset(p_cells, 0, nc * sizeof(double));
    memset(q_cells, 0, nc * sizeof(double));
    for (int64_t q = 0; q < m->n; ++q) {
        double s[NSTATE], pj, K2;
        long i, j, k;
        load_ray(m, q, s);
        cell_ijk(m, s, &i, &j, &k);
        ray_p(m, s, j, k, &pj, &K2);
        size_t c = node(m, k, j, i);
        p_cells[c] += pj;
        q_cells[c] += pj * K2;
    }
    return 0;
}

/* kappa = max(0, (P - rho/2) / (2 dt sum_j P_j K_j^2)) per cell, then N_j -> N_j (1 - 2 kappa K_j^2 dt)
 * (Eq. turbulent-diffusivity).  Reading: the cell is the carrier cell of each ray ("the cell it is
 * contained in"), rho at the cell centre, and the factor is clamped at 0 (not in the paper). */
static void apply_saturation(orc_model *m, double dt)
{
    if (m->n > m->n_scale_cap) {
        free(m->n_scale);
        m->n_scale = malloc(sizeof(double) * (size_t)m->n);
        m->n_scale_cap = m->n_scale ? m->n : 0;
    }
    m->n_scale_valid = m->n_scale != NULL;
    if (m->n_scale_valid)
        for (int64_t q = 0; q < m->n; ++q) m->n_scale[q] = fabs(m->s[SN][q]);
    m->n_scale_current = m->n_scale_valid;
    /* per-ray P_j and K_j^2 (independent per ray; the rays of a cell share its j, k) */
    int64_t nr = m->n;
    double *PJ = malloc(sizeof(double) * (size_t)(nr ? nr : 1));
    double *KJ = malloc(sizeof(double) * (size_t)(nr ? nr : 1));
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < nr; ++q) {
        double s[NSTATE];
        long i, j, k;
        load_ray(m, q, s);
        cell_ijk(m, s, &i, &j, &k);
        ray_p(m, s, j, k, &PJ[q], &KJ[q]);
    }
    int64_t a = 0;
    while (a < m->n) {
        int32_t cell = m->cell[a];
        int64_t b = a;
        while (b < m->n && m->cell[b] == cell) ++b;
        double s0[NSTATE];
        long i, j, k;
        load_ray(m, a, s0);
        cell_ijk(m, s0, &i, &j, &k);
        double P = 0.0, Q = 0.0;
        for (int64_t q = a; q < b; ++q) {
            P += PJ[q];
            Q += PJ[q] * KJ[q];
        }
        double rho = m->rho[node(m, k, j, i)];
        double kappa = Q > 0.0 ? fmax(0.0, (P - 0.5 * rho) / (2.0 * dt * Q)) : 0.0;
        if (kappa > 0.0) {
            for (int64_t q = a; q < b; ++q) {
                double s[NSTATE];
                load_ray(m, q, s);
                double K2 = KJ[q];
                double fac = fmax(0.0, 1.0 - 2.0 * kappa * K2 * dt);
                double nold = s[SN];
                m->s[SN][q] = nold * fac;
                m->st.w_saturated += (nold - nold * fac) * s[SPX] * s[SPY] * s[SPZ];
            }
        }
        a = b;
    }
    free(PJ);
    free(KJ);
}

/* ------------------------------------------------------------------ projection (Sec. 2b, Sec. 3b) */

/* Fluxes of one ray volume.  Direct form (Eq. fluxes:momentum) with e_r x e_lambda = e_phi and
 * e_r x e_phi = -e_lambda; first index = flux direction, second = momentum component:
 *   T^{ab} = [w^2 ch_a k_b + f^2 (e_r x ch)_a (e_r x k_h)_b] / (w^2 - f^2) A
 * Elastic term (Eq. fluxes:temperature into Eq. fluxes:buoyancy; theta-bar cancels):
 *   (f/g) e_r x <u'b'> = -(1 / (g rho)) f^2 N^2 ch_r / (w^2 - f^2) k_h A
 * (accumulated here without the 1/(g rho) factor, applied with the cell density later).
 * Pseudomomentum form (App. A): T^{ab} = ch_a k_b A, no elastic term. */
/* the ten flux values of one ray volume with wave action A (all linear in A):
 * out = {T_ll, T_lp, T_pl, T_pp, E_l, E_p, Z_l, Z_p, Th_l, Th_p}; the last two are the integrand of
 * Eq. fluxes:temperature without its theta-bar / (g rho-bar) factor (applied with the cell values):
 *   <u'theta'> (g rho / theta) = ch_r f N^2 / (w^2 - f^2) (e_r x k_h) A,  e_r x k_h = (-l, k),
 * f the signed Coriolis parameter at the ray; zero in the pseudomomentum form (App. A). */
static void ray_fluxes(const orc_model *m, const disp_t *d, double f, double f2, double n2, double kk, double ll,
                       double A, double out[10])
{
    const double *ch = d->ch;
    if (m->P.flux_form == 0) {
        double den = d->w2 - f2;
        out[8] = -f * n2 * ch[2] / den * ll * A;
        out[9] = f * n2 * ch[2] / den * kk * A;
        out[0] = (d->w2 * ch[0] * kk + f2 * ch[1] * ll) / den * A;
        out[1] = (d->w2 * ch[0] * ll - f2 * ch[1] * kk) / den * A;
        out[2] = (d->w2 * ch[1] * kk - f2 * ch[0] * ll) / den * A;
        out[3] = (d->w2 * ch[1] * ll + f2 * ch[0] * kk) / den * A;
        out[4] = -f2 * n2 * ch[2] / den * kk * A;
        out[5] = -f2 * n2 * ch[2] / den * ll * A;
        out[6] = d->w2 * ch[2] * kk / den * A;
        out[7] = d->w2 * ch[2] * ll / den * A;
    } else {
        out[0] = ch[0] * kk * A;
        out[1] = ch[0] * ll * A;
        out[2] = ch[1] * kk * A;
        out[3] = ch[1] * ll * A;
        out[4] = 0.0;
        out[5] = 0.0;
        out[6] = ch[2] * kk * A;
        out[7] = ch[2] * ll * A;
        out[8] = 0.0;
        out[9] = 0.0;
    }
}

/* Error scales of the ten flux values of one ray volume (same order as ray_fluxes, all >= 0): each
 * integrand with the horizontal wavenumber and group-velocity components replaced by the magnitudes
 * |k_h| and |ch_h| of their vectors, and ch_r by |ch_r|.  The integrands of Eq. fluxes:momentum and
 * Eq. fluxes:temperature are tensors and vectors built from k_h and ch_h; a component of those
 * vectors carries a rounding error relative to the vector's magnitude, not to itself (a wave vector
 * along one axis has a rounding-level component along the other, e.g. cos(pi/2) |k_h|), so the scale
 * of an integrand is the one that does not depend on the orientation of the wave vector. */
static void ray_flux_scales(const orc_model *m, const disp_t *d, double f, double f2, double n2, double kh,
                            double A, double out[10])
{
    const double chh = hypot(d->ch[0], d->ch[1]), chr = fabs(d->ch[2]);
    if (m->P.flux_form == 0) {
        double den = d->w2 - f2;
        double t = (d->w2 + f2) * chh * kh / den * A;
        out[0] = out[1] = out[2] = out[3] = t;
        out[4] = out[5] = f2 * n2 * chr / den * kh * A;
        out[6] = out[7] = d->w2 * chr * kh / den * A;
        out[8] = out[9] = fabs(f) * n2 * chr / den * kh * A;
    } else {
        out[0] = out[1] = out[2] = out[3] = chh * kh * A;
        out[4] = out[5] = 0.0;
        out[6] = out[7] = chr * kh * A;
        out[8] = out[9] = 0.0;
    }
}

/* Error scales (hfabs, fzabs): sums of |contribution| with the wave action a ray volume had before
 * this step's saturation.  The saturation factor 1 - 2 kappa K^2 dt is a difference of terms of
 * size 1, so its rounding error is of order the unit roundoff relative to 1, not to the factor;
 * a nearly fully damped ray volume therefore carries an error proportional to its action before
 * the damping, and the scale follows that. */
static void project(orc_model *m)
{
    long nx = m->G.nx, ny = m->G.ny, nz = m->G.nz;
    size_t nc = (size_t)nx * ny * nz, ni = (size_t)nx * ny * (nz + 1);
    memset(m->fz[0], 0, ni * sizeof(double));
    memset(m->fz[1], 0, ni * sizeof(double));
    memset(m->fzabs[0], 0, ni * sizeof(double));
    memset(m->fzabs[1], 0, ni * sizeof(double));
    for (int f = 0; f < NFIELD_H; ++f) {
        memset(m->hf[f], 0, nc * sizeof(double));
        memset(m->hfabs[f], 0, nc * sizeof(double));
    }
    double dz = m->G.dz;
    /* per-ray integrands (independent per ray), then the sums in array order */
    typedef struct { double fl[10], fa[10], A, A_scale, alpha, w_h, lo, hi; long i, j, k; } ray_proj_t;
    int64_t nr = m->n;
    ray_proj_t *RP = malloc(sizeof(ray_proj_t) * (size_t)(nr ? nr : 1));
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < nr; ++q) {
        ray_proj_t *rp = &RP[q];
        double s[NSTATE], f2, n2, dk, dl, dm;
        disp_t d;
        load_ray(m, q, s);
        cell_ijk(m, s, &rp->i, &rp->j, &rp->k);
        ray_disp(m, s, &d, &f2, &n2);
        spectral_extents(m, s, &dk, &dl, &dm);
        rp->A = s[SN] * dk * dl * dm;
        rp->A_scale = (m->n_scale_valid ? m->n_scale[q] : fabs(s[SN])) * dk * dl * dm;
        const double fsgn = is_sphere(m) ? 2.0 * m->G.omega * sin(s[SY]) : m->G.f0;
        ray_fluxes(m, &d, fsgn, f2, n2, s[SK], s[SL], rp->A, rp->fl);
        ray_flux_scales(m, &d, fsgn, f2, n2, hypot(s[SK], s[SL]), rp->A_scale, rp->fa);
        /* horizontal fluxes: cell average over the ray volumes whose carrier lies in the cell,
         * each weighted by its share alpha_j = V_j / V_c of the cell volume */
        rp->alpha = physical_volume(m, s) / cell_volume(m, rp->j, rp->k);
        /* horizontal share of the column: solid angle of the ray volume over that of the cell */
        if (is_sphere(m))
            rp->w_h = cos(s[SY]) * s[SEX] * s[SEY] / (cos(row_lat(m, rp->j)) * cell_x(m) * cell_y(m));
        else
            rp->w_h = s[SEX] * s[SEY] / (m->G.dx * m->G.dy);
        rp->lo = s[SZ] - 0.5 * s[SEZ];
        rp->hi = s[SZ] + 0.5 * s[SEZ];
    }
    for (int64_t q = 0; q < nr; ++q) {
        const ray_proj_t *rp = &RP[q];
        const double *fl = rp->fl, *fa = rp->fa;
        long i = rp->i, j = rp->j, k = rp->k;
        double alpha = rp->alpha, A = rp->A;
        size_t c = node(m, k, j, i);
        m->hf[0][c] += alpha * fl[0];
        m->hf[1][c] += alpha * fl[1];
        m->hf[2][c] += alpha * fl[2];
        m->hf[3][c] += alpha * fl[3];
        m->hf[4][c] += alpha * fl[4];
        m->hf[5][c] += alpha * fl[5];
        m->hf[6][c] += alpha * A;
        m->hf[7][c] += alpha * fl[8];
        m->hf[8][c] += alpha * fl[9];
        double hv[NFIELD_H] = {fa[0], fa[1], fa[2], fa[3], fa[4], fa[5], rp->A_scale, fa[8], fa[9]};
        for (int f = 0; f < NFIELD_H; ++f) m->hfabs[f][c] += fabs(alpha * hv[f]);
        /* vertical fluxes at the cell interfaces z = kk dz, 1 <= kk <= nz-1: integrate over the
         * staggered cell [(kk - 1/2) dz, (kk + 1/2) dz] of the carrier column; the weight is the
         * horizontal share times the vertical overlap share.  Reading: F^z = 0 at z = 0, z_top. */
        double w_h = rp->w_h, lo = rp->lo, hi = rp->hi;
        for (long kk2 = 1; kk2 < nz; ++kk2) {
            double slo = (kk2 - 0.5) * dz, shi = (kk2 + 0.5) * dz;
            double ov = fmin(hi, shi) - fmax(lo, slo);
            if (!(ov > 0.0)) continue;
            double w = w_h * ov / dz;
            size_t ci = ((size_t)kk2 * ny + (size_t)j) * nx + (size_t)i;
            m->fz[0][ci] += w * fl[6];
            m->fz[1][ci] += w * fl[7];
            m->fzabs[0][ci] += fabs(w * fa[6]);
            m->fzabs[1][ci] += fabs(w * fa[7]);
        }
    }
    free(RP);
    m->n_scale_valid = 0;
}

/* Reading of App. B.4 for a lat-lon grid: separable 1-2-1 x 1-2-1 weights (4 centre, 2 edge,
 * 1 corner, normalised by 16), periodic in x, reflecting (edge row reused) at the pole rows on
 * the sphere, periodic in y on the f-plane. */
int orc_smooth(const orc_model *m, double *fld, int nlev)
{
    long nx = m->G.nx, ny = m->G.ny;
    /* levels are independent */
    double *tmpall = malloc(sizeof(double) * (size_t)nx * ny * (size_t)(nlev > 0 ? nlev : 1));
    ORC_PARALLEL_FOR
    for (int lev = 0; lev < nlev; ++lev) {
        double *F = fld + (size_t)lev * nx * ny;
        double *tmp = tmpall + (size_t)lev * nx * ny;
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double acc = 0.0;
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        long jj = j + dj, ii = wrap_index(i + di, nx);
                        if (is_sphere(m)) jj = clampl(jj, 0, ny - 1);
                        else jj = wrap_index(jj, ny);
                        double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0);
                        acc += w * F[(size_t)jj * nx + ii];
                    }
                tmp[(size_t)j * nx + i] = acc / 16.0;
            }
        memcpy(F, tmp, sizeof(double) * (size_t)nx * ny);
    }
    free(tmpall);
    return 0;
}

static void smooth_all(orc_model *m)
{
    for (int q = 0; q < 2; ++q) {
        orc_smooth(m, m->fz[q], m->G.nz + 1);
        orc_smooth(m, m->fzabs[q], m->G.nz + 1);
    }
    for (int f = 0; f < NFIELD_H; ++f) {
        orc_smooth(m, m->hf[f], m->G.nz);
        orc_smooth(m, m->hfabs[f], m->G.nz);
    }
}

/* Eq. mean-flow-impact: du/dt = -(1/rho) div(rho <v'u'>) + (f/g) e_r x <u'b'>.
 * Horizontal divergence by centred differences in the cell-centre fields,
 *   (1/(r cos phi)) d/dlambda F^{lambda .} + (1/(r cos phi)) d/dphi (cos phi F^{phi .}),
 * flux zero beyond the pole rows; vertical divergence from the interface fluxes bounding the
 * cell (Sec. 3b).  Reading: the curvature terms of the tensor divergence are not included. */
int orc_divergence(const orc_model *m, const double *fz_l, const double *fz_p,
                   const double *f_ll, const double *f_lp, const double *f_pl, const double *f_pp,
                   const double *e_l, const double *e_p, double *dudt, double *dvdt)
{
    long nx = m->G.nx, ny = m->G.ny, nz = m->G.nz;
    double dX = cell_x(m), dY = cell_y(m), dz = m->G.dz;
    ORC_PARALLEL_FOR
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                size_t c = node(m, k, j, i);
                size_t ce = node(m, k, j, wrap_index(i + 1, nx)), cw = node(m, k, j, wrap_index(i - 1, nx));
                double rho = m->rho[c];
                double fz_top_l = fz_l[((size_t)(k + 1) * ny + j) * nx + i];
                double fz_bot_l = fz_l[((size_t)k * ny + j) * nx + i];
                double fz_top_p = fz_p[((size_t)(k + 1) * ny + j) * nx + i];
                double fz_bot_p = fz_p[((size_t)k * ny + j) * nx + i];
                double div_u, div_v;
                if (is_sphere(m)) {
                    double r = m->G.radius + (k + 0.5) * dz;
                    double cphi = cos(row_lat(m, j));
                    double cn = 0.0, cs = 0.0, pl_n = 0.0, pl_s = 0.0, pp_n = 0.0, pp_s = 0.0;
                    if (j + 1 < ny) {
                        size_t cc = node(m, k, j + 1, i);
                        cn = cos(row_lat(m, j + 1));
                        pl_n = f_pl[cc];
                        pp_n = f_pp[cc];
                    }
                    if (j - 1 >= 0) {
                        size_t cc = node(m, k, j - 1, i);
                        cs = cos(row_lat(m, j - 1));
                        pl_s = f_pl[cc];
                        pp_s = f_pp[cc];
                    }
                    double dl_u = (f_ll[ce] - f_ll[cw]) / (2.0 * dX);
                    double dp_u = (cn * pl_n - cs * pl_s) / (2.0 * dY);
                    double dl_v = (f_lp[ce] - f_lp[cw]) / (2.0 * dX);
                    double dp_v = (cn * pp_n - cs * pp_s) / (2.0 * dY);
                    div_u = (dl_u + dp_u) / (r * cphi) + (fz_top_l - fz_bot_l) / dz;
                    div_v = (dl_v + dp_v) / (r * cphi) + (fz_top_p - fz_bot_p) / dz;
                } else {
                    size_t cn = node(m, k, wrap_index(j + 1, ny), i), cs = node(m, k, wrap_index(j - 1, ny), i);
                    div_u = (f_ll[ce] - f_ll[cw]) / (2.0 * dX) + (f_pl[cn] - f_pl[cs]) / (2.0 * dY)
                          + (fz_top_l - fz_bot_l) / dz;
                    div_v = (f_lp[ce] - f_lp[cw]) / (2.0 * dX) + (f_pp[cn] - f_pp[cs]) / (2.0 * dY)
                          + (fz_top_p - fz_bot_p) / dz;
                }
                if (m->P.columnar) {
                    /* horizontally homogeneous column: the vertical flux divergence alone */
                    div_u = (fz_top_l - fz_bot_l) / dz;
                    div_v = (fz_top_p - fz_bot_p) / dz;
                }
                dudt[c] = -div_u / rho + e_l[c] / (m->G.g * rho);
                dvdt[c] = -div_v / rho + e_p[c] / (m->G.g * rho);
            }
    return 0;
}

/* Error scale of the tendencies: the divergence formula applied to the sums of |contribution|
 * with every term taken in magnitude.  Test infrastructure: rounding of the sums is bounded by
 * a small multiple of the machine epsilon times this. */
int orc_tendency_scale(const orc_model *m, double *du_s, double *dv_s)
{
    long nx = m->G.nx, ny = m->G.ny, nz = m->G.nz;
    double dX = cell_x(m), dY = cell_y(m), dz = m->G.dz;
    const double *A[2][4] = {{m->hfabs[0], m->hfabs[2], m->fzabs[0], m->hfabs[4]},
                             {m->hfabs[1], m->hfabs[3], m->fzabs[1], m->hfabs[5]}};
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                size_t c = node(m, k, j, i);
                size_t ce = node(m, k, j, wrap_index(i + 1, nx)), cw = node(m, k, j, wrap_index(i - 1, nx));
                double hx = 1.0, hy = 1.0, cn = 1.0, cs = 1.0;
                long jn = j + 1, js = j - 1;
                if (is_sphere(m)) {
                    double r = m->G.radius + (k + 0.5) * dz, cphi = cos(row_lat(m, j));
                    hx = r * cphi;
                    hy = r * cphi;
                    cn = jn < ny ? cos(row_lat(m, jn)) : 0.0;
                    cs = js >= 0 ? cos(row_lat(m, js)) : 0.0;
                } else {
                    jn = wrap_index(jn, ny);
                    js = wrap_index(js, ny);
                }
                for (int q = 0; q < 2; ++q) {
                    double yn = (jn >= 0 && jn < ny) ? A[q][1][node(m, k, jn, i)] : 0.0;
                    double ys = (js >= 0 && js < ny) ? A[q][1][node(m, k, js, i)] : 0.0;
                    double v = (A[q][2][((size_t)(k + 1) * ny + j) * nx + i] + A[q][2][((size_t)k * ny + j) * nx + i]) / dz;
                    if (!m->P.columnar)
                        v += (A[q][0][ce] + A[q][0][cw]) / (2.0 * dX * hx) + (cn * yn + cs * ys) / (2.0 * dY * hy);
                    v = v / m->rho[c] + A[q][3][c] / (m->G.g * m->rho[c]);
                    (q == 0 ? du_s : dv_s)[c] = v;
                }
            }
    return 0;
}

/* sums of |contribution| of field `which` (layout as orc_get_field) */
int orc_get_field_abs(const orc_model *m, int which, double *out)
{
    size_t nc = (size_t)m->G.nx * m->G.ny * m->G.nz, ni = (size_t)m->G.nx * m->G.ny * (m->G.nz + 1);
    if (which == 0 || which == 1) {
        memcpy(out, m->fzabs[which], ni * sizeof(double));
        return 0;
    }
    if (which >= 2 && which < 2 + NFIELD_H) {
        memcpy(out, m->hfabs[which - 2], nc * sizeof(double));
        return 0;
    }
    return -1;
}

/* reference potential temperature theta-bar at the nodes, C-order [nz][ny][nx] (positive) */
int orc_set_theta(orc_model *m, const double *theta)
{
    size_t nc = (size_t)m->G.nx * m->G.ny * m->G.nz;
    for (size_t q = 0; q < nc; ++q)
        if (!(theta[q] > 0.0) || !isfinite(theta[q])) return -1;
    if (!m->theta) m->theta = malloc(nc * sizeof(double));
    memcpy(m->theta, theta, nc * sizeof(double));
    return 0;
}

/* Eq. mean-flow-impact-t: d theta / dt = -div <u'theta'>, <u'theta'> horizontal (along e_r x k_h)
 * and equal to theta-bar / (g rho-bar) times the projected integrals T_l, T_p of each cell (Eq.
 * fluxes:temperature).  The horizontal divergence as in orc_divergence: centred differences,
 * (1/(r cos phi)) [d/dlambda Th_l + d/dphi (cos phi Th_p)], flux zero beyond the pole rows; zero in
 * the columnar mode.  With mag != 0 every difference becomes a sum of magnitudes (error scale). */
static void theta_div(const orc_model *m, const double *tl, const double *tp, double *out, int mag)
{
    long nx = m->G.nx, ny = m->G.ny, nz = m->G.nz;
    double dX = cell_x(m), dY = cell_y(m), dz = m->G.dz;
    double sg = mag ? -1.0 : 1.0;     /* (east - sg west): a difference, or a sum of magnitudes */
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                size_t c = node(m, k, j, i);
                if (m->P.columnar) {
                    out[c] = 0.0;
                    continue;
                }
#define THF(arr, cc) ((arr)[cc] * m->theta[cc] / (m->G.g * m->rho[cc]))
                size_t ce = node(m, k, j, wrap_index(i + 1, nx)), cw = node(m, k, j, wrap_index(i - 1, nx));
                double div;
                if (is_sphere(m)) {
                    double r = m->G.radius + (k + 0.5) * dz;
                    double cphi = cos(row_lat(m, j));
                    double yn = 0.0, ys = 0.0;
                    if (j + 1 < ny) yn = cos(row_lat(m, j + 1)) * THF(tp, node(m, k, j + 1, i));
                    if (j - 1 >= 0) ys = cos(row_lat(m, j - 1)) * THF(tp, node(m, k, j - 1, i));
                    double dl = (THF(tl, ce) - sg * THF(tl, cw)) / (2.0 * dX);
                    double dp = (yn - sg * ys) / (2.0 * dY);
                    div = (dl + dp) / (r * cphi);
                } else {
                    size_t cn = node(m, k, wrap_index(j + 1, ny), i), cs = node(m, k, wrap_index(j - 1, ny), i);
                    div = (THF(tl, ce) - sg * THF(tl, cw)) / (2.0 * dX) + (THF(tp, cn) - sg * THF(tp, cs)) / (2.0 * dY);
                }
#undef THF
                out[c] = mag ? div : -div;
            }
}

/* the potential-temperature tendency of given integrals T_l, T_p (C-order [nz][ny][nx]) */
int orc_theta_divergence(const orc_model *m, const double *tl, const double *tp, double *out)
{
    if (!m->theta) return -1;
    theta_div(m, tl, tp, out, 0);
    return 0;
}

/* the tendency of the last step's (smoothed) integrals, and its error scale (may be NULL) */
int orc_theta_tendency(const orc_model *m, double *out, double *scale)
{
    if (!m->theta) return -1;
    theta_div(m, m->hf[7], m->hf[8], out, 0);
    if (scale) theta_div(m, m->hfabs[7], m->hfabs[8], scale, 1);
    return 0;
}

int orc_get_field(const orc_model *m, int which, double *out)
{
    size_t nc = (size_t)m->G.nx * m->G.ny * m->G.nz, ni = (size_t)m->G.nx * m->G.ny * (m->G.nz + 1);
    if (which == 0 || which == 1) {
        memcpy(out, m->fz[which], ni * sizeof(double));
        return 0;
    }
    if (which >= 2 && which < 2 + NFIELD_H) {
        memcpy(out, m->hf[which - 2], nc * sizeof(double));
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------ the step */

/* Phase 1 of a step: advance every ray volume (RK3), remove those that left, split the rest;
 * the array is left in array order (not sorted). */
int orc_step_advance(orc_model *m, double dt)
{
    if (!(dt > 0.0) || !isfinite(dt) || !m->have_bg) return -1;
    int64_t n = m->n;
    /* 1. advance every ray volume (RK3), remove those that left, split the rest (array order) */
    double *ns[NSTATE];
    int64_t ncap = 4 * n + 1, nn = 0;
    for (int c = 0; c < NSTATE; ++c) ns[c] = malloc(sizeof(double) * (size_t)ncap);
    int64_t *nid = malloc(sizeof(int64_t) * (size_t)ncap);
    /* the advance of each ray volume is independent of the others */
    double *adv = malloc(sizeof(double) * NSTATE * (size_t)(n ? n : 1));
    ORC_PARALLEL_FOR
    for (int64_t q = 0; q < n; ++q) {
        double *sq = adv + (size_t)q * NSTATE;
        load_ray(m, q, sq);
        orc_advance_ray(m, sq, dt);
    }
    free(m->issued);
    m->issued = malloc(sizeof(int64_t) * (size_t)(n + 1));
    m->issued_n = n;
    const int64_t id0 = m->next_id;
    for (int64_t q = 0; q < n; ++q) {
        double s[NSTATE];
        m->issued[q] = m->next_id - id0;
        memcpy(s, adv + (size_t)q * NSTATE, sizeof(s));
        int st = ray_status(m, s);
        if (st == 2) {
            m->st.n_invalid++;
            if (isfinite(ray_action(s))) m->st.w_invalid += ray_action(s);
            continue;
        }
        if (st == 1) {
            m->st.n_exited++;
            m->st.w_exited += ray_action(s);
            continue;
        }
        double ch[4][NSTATE];
        int64_t cid[4];
        int nch = split_ray(m, s, m->id[q], ch, cid);
        for (int c = 0; c < nch; ++c) {
            if (ray_status(m, ch[c]) != 0) {
                m->st.n_exited++;
                m->st.w_exited += ray_action(ch[c]);
                continue;
            }
            for (int e = 0; e < NSTATE; ++e) ns[e][nn] = ch[c][e];
            nid[nn] = cid[c];
            ++nn;
        }
    }
    m->issued[n] = m->next_id - id0;
    free(adv);
    m->n = 0;
    reserve(m, nn);
    for (int c = 0; c < NSTATE; ++c) {
        memcpy(m->s[c], ns[c], sizeof(double) * (size_t)nn);
        free(ns[c]);
    }
    memcpy(m->id, nid, sizeof(int64_t) * (size_t)nn);
    free(nid);
    m->n = nn;
    return 0;
}

/* Phase 2 of a step: canonical order, per-column cap, saturation and projection -- all local to a
 * carrier cell or column. */
int orc_step_local(orc_model *m, double dt)
{
    if (!(dt > 0.0) || !isfinite(dt) || !m->have_bg) return -1;
    /* 2. reassign cells, canonical order (App. B.2: rays kept per parent cell) */
    sort_rays(m);
    /* 3. per-column cap */
    apply_cap(m);
    /* 4. saturation with the post-step state */
    if (m->P.saturation) apply_saturation(m, dt);
    project(m);
    return 0;
}

/* Phase 3 of a step: smoothing and divergence of the projected fields, budget. */
int orc_step_grid(orc_model *m, double *dudt, double *dvdt)
{
    /* 5. smoothing, divergence */
    if (m->P.smoothing) smooth_all(m);
    size_t nc = (size_t)m->G.nx * m->G.ny * m->G.nz;
    double *du = dudt ? dudt : malloc(nc * sizeof(double));
    double *dv = dvdt ? dvdt : malloc(nc * sizeof(double));
    orc_divergence(m, m->fz[0], m->fz[1], m->hf[0], m->hf[1], m->hf[2], m->hf[3], m->hf[4], m->hf[5], du, dv);
    if (!dudt) free(du);
    if (!dvdt) free(dv);
    /* 6. budget: total wave action in the ray volumes (Eq. wave-action-budget integrated) */
    double w = 0.0;
    for (int64_t q = 0; q < m->n; ++q) {
        double s[NSTATE];
        load_ray(m, q, s);
        w += ray_action(s);
    }
    m->st.w_total = w;
    m->st.n_live = m->n;
    m->st.n_steps++;
    return 0;
}

int orc_step(orc_model *m, double dt, double *dudt, double *dvdt)
{
    if (orc_step_advance(m, dt)) return -1;
    orc_step_local(m, dt);
    return orc_step_grid(m, dudt, dvdt);
}

/* projection (and smoothing) of the current ray volumes without advancing them */
int orc_diagnose(orc_model *m, double *dudt, double *dvdt)
{
    if (!m->have_bg) return -1;
    sort_rays(m);
    project(m);
    if (m->P.smoothing) smooth_all(m);
    if (dudt && dvdt)
        orc_divergence(m, m->fz[0], m->fz[1], m->hf[0], m->hf[1], m->hf[2], m->hf[3], m->hf[4], m->hf[5],
                       dudt, dvdt);
    return 0;
}

int64_t orc_num_rays(const orc_model *m) { return m->n; }

int orc_get_rays(const orc_model *m, double *state, int64_t *ids, int32_t *cells)
{
    for (int c = 0; c < NSTATE; ++c)
        if (state) memcpy(state + (size_t)c * m->n, m->s[c], sizeof(double) * (size_t)m->n);
    if (ids) memcpy(ids, m->id, sizeof(int64_t) * (size_t)m->n);
    if (cells)
        for (int64_t q = 0; q < m->n; ++q) {
            double s[NSTATE];
            load_ray(m, q, s);
            cells[q] = cell_of(m, s);
        }
    return 0;
}

/* Per ray volume of the current array: its wave-action density before the last step's saturation
 * (the scale of the damped density's rounding error, see project), or |N| when the array changed
 * since that saturation or none ran. */
int orc_get_action_scale(const orc_model *m, double *out)
{
    for (int64_t q = 0; q < m->n; ++q)
        out[q] = (m->n_scale_current && m->n_scale) ? m->n_scale[q] : fabs(m->s[SN][q]);
    return 0;
}

/* ---------------------------------------------- latitude-band decomposition (App. B.2)
 * A model may own the rows [j0, j1) of a latitude band: it launches only there, and after the
 * advance phase the ray volumes whose carrier row left the band are taken out and handed to the
 * band that owns them.  The grid stays whole; only the band's rows (and the halo rows its stencils
 * read) carry meaning. */
int orc_set_owned_rows(orc_model *m, long j0, long j1)
{
    if (j0 < 0 || j1 > m->G.ny || j0 >= j1) return -1;
    m->row0 = j0;
    m->row1 = j1;
    return 0;
}

int64_t orc_get_next_id(const orc_model *m) { return m->next_id; }
void orc_set_next_id(orc_model *m, int64_t id) { m->next_id = id; }

/* ids in [lo, hi) become id - lo + to (provisional ids of a band turned into global ones) */
void orc_remap_ids(orc_model *m, int64_t lo, int64_t hi, int64_t to)
{
    for (int64_t q = 0; q < m->n; ++q)
        if (m->id[q] >= lo && m->id[q] < hi) m->id[q] = m->id[q] - lo + to;
}

/* new ids issued by the rays before array position q (0 <= q <= n) in the last advance */
int64_t orc_issued_before(const orc_model *m, int64_t q)
{
    if (!m->issued || q < 0 || q > m->issued_n) return -1;
    return m->issued[q];
}

static long ray_row(const orc_model *m, int64_t q)
{
    double s[NSTATE];
    long i, j, k;
    load_ray(m, q, s);
    cell_ijk(m, s, &i, &j, &k);
    return j;
}

int64_t orc_count_rays_outside(const orc_model *m)
{
    int64_t c = 0;
    for (int64_t q = 0; q < m->n; ++q) {
        long j = ray_row(m, q);
        if (j < m->row0 || j >= m->row1) ++c;
    }
    return c;
}

/* Remove the ray volumes whose carrier row lies outside the owned rows; their states (row-major,
 * 13 values each), ids and carrier rows go to out_state / out_ids / out_rows in array order (at most
 * cap of them). */
int64_t orc_take_rays_outside(orc_model *m, double *out_state, int64_t *out_ids, int32_t *out_rows, int64_t cap)
{
    int64_t w = 0, t = 0;
    for (int64_t q = 0; q < m->n; ++q) {
        long j = ray_row(m, q);
        if (j < m->row0 || j >= m->row1) {
            if (t >= cap) return -1;
            for (int c = 0; c < NSTATE; ++c) out_state[(size_t)t * NSTATE + c] = m->s[c][q];
            out_rows[t] = (int32_t)j;
            out_ids[t++] = m->id[q];
            continue;
        }
        for (int c = 0; c < NSTATE; ++c) m->s[c][w] = m->s[c][q];
        m->id[w] = m->id[q];
        m->cell[w] = m->cell[q];
        ++w;
    }
    m->n = w;
    m->n_scale_current = 0;
    return t;
}

/* Append ray volumes handed over from another band (states row-major, ids kept; no tallies). */
int orc_put_rays(orc_model *m, int64_t n, const double *state, const int64_t *ids)
{
    for (int64_t q = 0; q < n; ++q) append_ray(m, state + (size_t)q * NSTATE, ids[q]);
    m->st.n_live = m->n;
    return 0;
}

/* Overwrite a projected field (same numbering as orc_get_field): halo rows from a neighbour band */
int orc_set_field(orc_model *m, int which, const double *in)
{
    size_t nc = (size_t)m->G.nx * m->G.ny * m->G.nz, ni = (size_t)m->G.nx * m->G.ny * (m->G.nz + 1);
    if (which == 0 || which == 1) {
        memcpy(m->fz[which], in, ni * sizeof(double));
        return 0;
    }
    if (which >= 2 && which < 2 + NFIELD_H) {
        memcpy(m->hf[which - 2], in, nc * sizeof(double));
        return 0;
    }
    return -1;
}

int orc_set_threads(orc_model *m, int threads)
{
    m->threads = threads > 1 ? threads : 1;
#ifdef _OPENMP
    return m->threads;
#else
    m->threads = 1;
    return 1;
#endif
}

void orc_get_stats(const orc_model *m, orc_stats *out)
{
    *out = m->st;
    out->n_live = m->n;
}
