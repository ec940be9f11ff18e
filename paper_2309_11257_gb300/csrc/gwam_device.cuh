// gwam_device.cuh -- device-side data layout and per-ray-volume arithmetic (FP64 form).
//
// Ray equations of Voelker et al. (arXiv:2309.11257):
//   dispersion relation with scale-height correction ........ Sec. 2a, Eq. dispersion
//   c_g = grad_k Omega, rdot = c_g ........................... Eq. eikonal, Eq. group-velocity
//   wavenumber tendencies with spherical metric terms ......... Eq. eikonal-sphere:1-3
//   face group velocities from first-order Taylor values ...... Sec. 3b, App. B.1
//   per-axis phase-space products P = h dX dk ................. Sec. 3a, Eq. vpvol_cons_cart, Eq. dkxdkl
//   low-storage RK3 (Williamson 1980) ......................... App. B.2
//   splitting thresholds ...................................... App. B.3
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gwam_df.cuh"

namespace gwam {

constexpr double kPi = 3.14159265358979323846;
constexpr int kThreads = 256;

// ---------------------------------------------------------------------------- arithmetic

// Reciprocal: the hardware approximation (PTX rcp.approx.ftz.f64, about 20 correct bits) refined by
// two Newton-Raphson steps y <- y + y (1 - x y), each of which doubles the number of correct bits.
// For the positive, finite, normal-range operands of the ray equations (within an ulp or so of the
// IEEE quotient, tested against it); FP64 division would cost several times as many instructions.
__device__ __forceinline__ double rcp_nr(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// Reciprocal square root: the hardware approximation (PTX rsqrt.approx.ftz.f64) refined by two
// Newton-Raphson steps y <- y + (y/2) (1 - x y^2).
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x * y, y, 1.0);
    y = fma(0.5 * y, e, y);
    e = fma(-x * y, y, 1.0);
    return fma(0.5 * y, e, y);
}

// ---------------------------------------------------------------------------- layouts

// Grid geometry as the kernels see it (derived once on the host).
struct Grid {
    int geometry;          // 0 f-plane, 1 sphere
    int columnar;          // single-column mode (no horizontal propagation, advection or refraction)
    int nx, ny, nz;
    int ncol, ncell;       // per member: nx*ny, nx*ny*nz
    int members;           // ensemble members (independent backgrounds and ray populations)
    int ncol_all, ncell_all;   // members * ncol, members * ncell
    double dX, dY, dz;     // coordinate spacings (radians on the sphere)
    double y0;             // southern edge (-pi/2) or 0
    double Lx, Ly;         // periods in x (2 pi or nx dx) and y (f-plane)
    double ztop;
    double f0, radius, omega, g;
    double phimax;         // carriers poleward of this latitude leave (centre of the last row)
    // precomputed reciprocals and tables (FP64 division is a long instruction sequence)
    double inv_dX, inv_dY, inv_dz, inv_nx, inv_ny, inv_g;
    const double* row_cos;      // cos(phi_j) of every row centre (sphere), 1 on the f-plane
    const double* row_inv_cos;  // 1 / row_cos
    const double* lev_inv_r;    // 1 / (a + z_k) of every level centre (sphere), 1 on the f-plane
    // FP32 copies for the precision form (a float <- double conversion runs at the FP64 rate)
    float f_dX, f_dY, f_dz, f_y0, f_radius, f_omega, f_f0, f_inv_dX, f_inv_dY, f_inv_dz;
    const float* row_cos32;     // [ny]
    const float* ivol32;        // [ny * nz]: 1 / cell volume of row j, level k
    const float* whf32;         // [ny]: row_inv_cos * inv_dX * inv_dY (solid-angle share per unit extent)
    // double-float constants and row tables of the FP64 form's ray equations
    float2 df_radius, df_2omega, df_8omega2, df_f0sq, df_f0;
    const float2* row_sc_df;    // [ny][2]: sin, cos of every row centre (sphere)
    const double* row_lat;      // [ny]: latitude of every row centre
    const float2* whf_df;       // [ny]: row_inv_cos * inv_dX * inv_dY
    const float2* ivol_df;      // [ny * nz]: 1 / cell volume of row j, level k
    const float2* row_lat_df;   // [ny]: latitude of every row centre
    float2 df_inv_dX, df_inv_dY, df_inv_dz, df_y0;
    // split thresholds (App. B.3), computed on the host in the order the device used to:
    // split_thr[2 j] = alpha_s sqrt(cos(phi_j) dX dY), split_thr[2 j + 1] = alpha_s cos(phi_j) dX dY
    const double* split_thr;
    double split_hthr;          // max(alpha_s dz, min_split_dz)
    const double* row_f2;       // [ny]: f^2 of every row centre (f0^2 on the f-plane)
};

struct Params {
    int gamma_mode, saturation, smoothing, flux_form, splitting, cap, theta_flux;
    double alpha_s, min_split_dz;
    float f_alpha_s;
};

// Ray-volume state, structure of arrays of double2 (16-byte vector loads):
//   a[0] = (x, y)  a[1] = (z, k)  a[2] = (l, m)  a[3] = (ex, ey)
//   a[4] = (ez, Px)  a[5] = (Py, Pz)  a[6] = (N, id as int64 bits)
struct RaySoA {
    double2* a[7];
};

enum { SX, SY, SZ, SK, SL, SM, SEX, SEY, SEZ, SPX, SPY, SPZ, SN, NSTATE };

// Ray ids are 64-bit: the ensemble member in the top 8 bits, a running number below.  Cells are
// global: member * ncell + (j * nx + i) * nz + k, so the canonical array is member-major.
constexpr int kMemberShift = 56;
__host__ __device__ __forceinline__ int member_of(long long id) { return (int)((unsigned long long)id >> kMemberShift); }
__host__ __device__ __forceinline__ long long with_member(int m, long long local)
{
    return (long long)(((unsigned long long)m << kMemberShift) | (unsigned long long)local);
}

__device__ __forceinline__ void load_ray(const RaySoA& R, int64_t i, double s[NSTATE], long long& id)
{
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double2 v = __ldg(&R.a[q][i]);
        s[2 * q] = v.x;
        s[2 * q + 1] = v.y;
    }
    double2 v = __ldg(&R.a[6][i]);
    s[SN] = v.x;
    id = __double_as_longlong(v.y);
}

__device__ __forceinline__ void store_ray(const RaySoA& R, int64_t i, const double s[NSTATE], long long id)
{
#pragma unroll
    for (int q = 0; q < 6; ++q) R.a[q][i] = make_double2(s[2 * q], s[2 * q + 1]);
    R.a[6][i] = make_double2(s[SN], __longlong_as_double(id));
}

// Background nodes at cell centres, column-major: node (i, j, k) at (j*nx + i)*nz + k.
// The FP64 node holds U, V, N^2, Gamma^2 (32 bytes); the per-step gathers of the ray equations read
// the copies that also carry the node gradients (NodeDF of the FP64 form, Node32 of the precision
// form), written when the background is set (Sec. 3b, App. B.1).
struct __align__(32) Node {
    double v[4];       // U, V, N^2, Gamma^2
};

// FP32 background node of the precision form: the same 16 quantities in FP32 (64 bytes)
struct __align__(64) Node32 {
    float v[4];
    float d[4][3];
};

// FP32 ray record of the precision form, 64 bytes as four float4 arrays:
//   q[0] = (member-local cell as int bits, ox, oy, oz)    offsets in cell units, in [0, 1)
//   q[1] = (k, l, m, N)
//   q[2] = (eX, eY, eZ, Px)                               extents in coordinate units
//   q[3] = (Py, Pz, id low 32 bits, id high 32 bits)
struct Ray32SoA {
    float4* q[4];
};

__host__ __device__ __forceinline__ int64_t node_index(const Grid& G, int i, int j, int k)
{
    return ((int64_t)j * G.nx + i) * G.nz + k;
}

// ---------------------------------------------------------------------------- background gather

struct Bg {
    double v[4];     // U V N2 G2
    double d[4][3];  // coordinate derivatives of each
};

__device__ __forceinline__ int wrap_int(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// periodic bracketing node pair; s in node units, inv_n = 1/n
__device__ __forceinline__ void bracket_periodic(double s, int n, double inv_n, int& q0, int& q1, double& t)
{
    if (!isfinite(s)) s = 0.0;
    s = s - (double)n * floor(s * inv_n);
    double fl = floor(s);
    t = s - fl;
    q0 = wrap_int((int)fl, n);
    q1 = q0 + 1 == n ? 0 : q0 + 1;
}

// clamped bracketing: every interpolated quantity held at its edge-node value outside
__device__ __forceinline__ void bracket_clamped(double s, int n, int& q0, int& q1, double& t)
{
    if (!isfinite(s)) s = 0.0;
    if (s < 0.0) {
        q0 = 0; q1 = 1; t = 0.0;
    } else if (s >= (double)(n - 1)) {
        q0 = n - 2; q1 = n - 1; t = 1.0;
    } else {
        double fl = floor(s);
        q0 = (int)fl; q1 = q0 + 1; t = s - fl;
    }
}

// The background node as 16 double-float pairs (hi, lo), in the order of Node's 16 doubles: the
// per-step gathers of the FP64 form run on the FP32 pipes (compensated sums), with about 48
// significant bits.  Filled from the FP64 nodes whenever the background is set.
struct __align__(128) NodeDF {
    float4 q[8];   // q[e] = (hi, lo) of value 2e, then (hi, lo) of value 2e + 1
};

// s + c += (wh + wl) (vh + vl): TwoProduct of the high parts, TwoSum into s, all lower-order terms
// into the compensation c
__device__ __forceinline__ void df_acc(float vh, float vl, float wh, float wl, float& s, float& c)
{
    const float p = __fmul_rn(wh, vh);
    const float e = __fmaf_rn(wh, vh, -p);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, __fmaf_rn(wh, vl, __fmaf_rn(wl, vh, e))));
}

// Trilinear interpolation of the FP64 node values (U, V, N^2, Gamma^2) to (X, Y, Z).
__device__ __forceinline__ void gather_values_fp64(const Grid& G, const Node* __restrict__ bg, double X, double Y,
                                                   double Z, double v[4])
{
    int i0, i1, j0, j1, k0, k1;
    double tx, ty, tz;
    bracket_periodic(X * G.inv_dX - 0.5, G.nx, G.inv_nx, i0, i1, tx);
    if (G.geometry == 1) bracket_clamped((Y - G.y0) * G.inv_dY - 0.5, G.ny, j0, j1, ty);
    else bracket_periodic(Y * G.inv_dY - 0.5, G.ny, G.inv_ny, j0, j1, ty);
    bracket_clamped(Z * G.inv_dz - 0.5, G.nz, k0, k1, tz);
    const double ux = 1.0 - tx, uy = 1.0 - ty, uz = 1.0 - tz;
    const int dk = k1 - k0;
    const Node* cn[4] = {bg + node_index(G, i0, j0, k0), bg + node_index(G, i1, j0, k0),
                         bg + node_index(G, i0, j1, k0), bg + node_index(G, i1, j1, k0)};
    const double wc[4] = {ux * uy, tx * uy, ux * ty, tx * ty};
#pragma unroll
    for (int f = 0; f < 4; ++f) v[f] = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const Node* p = cn[q >> 1] + ((q & 1) ? dk : 0);
        const double w = wc[q >> 1] * ((q & 1) ? tz : uz);
        const double2 a = __ldg(reinterpret_cast<const double2*>(p->v));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p->v) + 1);
        v[0] += w * a.x;
        v[1] += w * a.y;
        v[2] += w * b.x;
        v[3] += w * b.y;
    }
}

struct BgDF {
    DF v[4];
    DF d[4][3];
};

// Bracketing in node units on double-float coordinates (FP32 pipes only): u = node coordinate,
// q0 = floor(u) (wrapped or clamped), t = u - floor(u).  A non-finite u maps to node 0.
__device__ __forceinline__ int wrap_fast(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    if (i < 0 && i >= -n) return i + n;
    return wrap_int(i, n);
}

__device__ __forceinline__ void bracket_periodic_df(DF u, int n, int& q0, int& q1, DF& t)
{
    float fl = df_floor(u);
    if (!(fabsf(fl) < 1e9f)) {
        fl = 0.0f;
        u = df_f(0.0f);
    }
    t = df_sub(u, df_f(fl));
    q0 = wrap_fast((int)fl, n);
    q1 = q0 + 1 == n ? 0 : q0 + 1;
}

__device__ __forceinline__ void bracket_clamped_df(DF u, int n, int& q0, int& q1, DF& t)
{
    float fl = df_floor(u);
    if (!(fabsf(fl) < 1e9f)) {
        fl = 0.0f;
        u = df_f(0.0f);
    }
    const int q = (int)fl;
    if (q < 0) {
        q0 = 0; q1 = 1; t = df_f(0.0f);
    } else if (q >= n - 1) {
        q0 = n - 2; q1 = n - 1; t = df_f(1.0f);
    } else {
        q0 = q; q1 = q + 1; t = df_sub(u, df_f(fl));
    }
}

// Trilinear sums of the node quantities held in the float4 elements [E0, E1) of every NodeDF
// (element e holds quantities 2e and 2e + 1), as unevaluated hi + compensation pairs, at the
// double-float position (X, Y, Z).
template <int E0, int E1>
__device__ __forceinline__ void gather_df_sums(const Grid& G, const NodeDF* __restrict__ bg, DF X, DF Y, DF Z,
                                               float (&s)[2 * (E1 - E0)], float (&c)[2 * (E1 - E0)])
{
    int i0, i1, j0, j1, k0, k1;
    DF Tx, Ty, Tz;
    const DF half = df_f(0.5f);
    bracket_periodic_df(df_sub(df_mul2(X, DF{G.df_inv_dX.x, G.df_inv_dX.y}), half), G.nx, i0, i1, Tx);
    if (G.geometry == 1)
        bracket_clamped_df(df_sub(df_mul2(df_sub(Y, DF{G.df_y0.x, G.df_y0.y}), DF{G.df_inv_dY.x, G.df_inv_dY.y}), half),
                           G.ny, j0, j1, Ty);
    else
        bracket_periodic_df(df_sub(df_mul2(Y, DF{G.df_inv_dY.x, G.df_inv_dY.y}), half), G.ny, j0, j1, Ty);
    bracket_clamped_df(df_sub(df_mul2(Z, DF{G.df_inv_dz.x, G.df_inv_dz.y}), half), G.nz, k0, k1, Tz);
    const DF one{1.0f, 0.0f};
    const DF Ux = df_sub(one, Tx), Uy = df_sub(one, Ty), Uz = df_sub(one, Tz);
    const DF w00 = df_mul2(Ux, Uy), w10 = df_mul2(Tx, Uy), w01 = df_mul2(Ux, Ty), w11 = df_mul2(Tx, Ty);
#pragma unroll
    for (int q = 0; q < 2 * (E1 - E0); ++q) s[q] = c[q] = 0.0f;
    const int dk = k1 - k0;
    // corners in the order (i0 j0), (i1 j0), (i0 j1), (i1 j1), each at k0 then k1.  The loop is rolled,
    // the corner's node and weight selected, not indexed: one copy of the eight loads and sixteen
    // accumulations instead of eight keeps the ray-step kernels small (measured faster on GB300 than
    // unrolling by 2 or 8: the kernels were stalling on instruction fetch)
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const int cx = (q >> 1) & 1, cy = q >> 2;
        const NodeDF* p = bg + node_index(G, cx ? i1 : i0, cy ? j1 : j0, k0) + ((q & 1) ? dk : 0);
        const DF wxy = cx ? (cy ? w11 : w10) : (cy ? w01 : w00);
        const DF w = df_mul2(wxy, (q & 1) ? Tz : Uz);
#pragma unroll
        for (int e = E0; e < E1; ++e) {
            const float4 a = __ldg(p->q + e);
            df_acc(a.x, a.y, w.hi, w.lo, s[2 * (e - E0)], c[2 * (e - E0)]);
            df_acc(a.z, a.w, w.hi, w.lo, s[2 * (e - E0) + 1], c[2 * (e - E0) + 1]);
        }
    }
}

// gather with double-float results (no conversion back to FP64)
__device__ __forceinline__ void gather_df(const Grid& G, const NodeDF* __restrict__ bg, DF X, DF Y, DF Z, BgDF& b)
{
    float s[16], c[16];
    gather_df_sums<0, 8>(G, bg, X, Y, Z, s, c);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        b.v[f] = df_norm(s[f], c[f]);
#pragma unroll
        for (int q = 0; q < 3; ++q) b.d[f][q] = df_norm(s[4 + 3 * f + q], c[4 + 3 * f + q]);
    }
}

// gather with FP64 results from the double-float nodes (saturation and cap paths of the FP64 form)
__device__ __forceinline__ void gather(const Grid& G, const NodeDF* __restrict__ bg, double X, double Y, double Z,
                                       Bg& b)
{
    float s[16], c[16];
    gather_df_sums<0, 8>(G, bg, df_split(X), df_split(Y), df_split(Z), s, c);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        b.v[f] = widen(s[f]) + widen(c[f]);
#pragma unroll
        for (int q = 0; q < 3; ++q) b.d[f][q] = widen(s[4 + 3 * f + q]) + widen(c[4 + 3 * f + q]);
    }
}

// N^2 and Gamma^2 alone (the second float4 of each node): what the intrinsic quantities need
__device__ __forceinline__ void gather_n2g2_df(const Grid& G, const NodeDF* __restrict__ bg, DF X, DF Y, DF Z,
                                               DF& n2, DF& g2)
{
    float s[2], c[2];
    gather_df_sums<1, 2>(G, bg, X, Y, Z, s, c);
    n2 = df_norm(s[0], c[0]);
    g2 = df_norm(s[1], c[1]);
}

// f^2 and d(f^2)/dphi (f = 2 Omega sin phi on the sphere, f0 on the f-plane)
__device__ __forceinline__ void coriolis(const Grid& G, double sphi, double cphi, double& f2, double& df2)
{
    if (G.geometry == 1) {
        double f = 2.0 * G.omega * sphi;
        f2 = f * f;
        df2 = 8.0 * G.omega * G.omega * sphi * cphi;
    } else {
        f2 = G.f0 * G.f0;
        df2 = 0.0;
    }
}

// ---------------------------------------------------------------------------- dispersion (Eq. dispersion)

// Positive intrinsic branch: w^2 = (f^2 (m^2 + G^2) + N^2 k_h^2) / K^2, K^2 = k_h^2 + m^2 + G^2.
// The intrinsic group velocity is ch = (k, l) D (m^2 + G^2) / (w K^4), ch_r = -m D k_h^2 / (w K^4),
// D = N^2 - f^2, so each component is (its factor) * c with c = D / (w K^4).
struct Disp {
    double K2, iK2, D, w2, w, iw, c;
};

__device__ __forceinline__ void dispersion(double kh2, double mg2, double n2, double f2, Disp& d)
{
    d.K2 = kh2 + mg2;
    d.D = n2 - f2;
    d.iK2 = rcp_nr(d.K2);
    d.w2 = (f2 * mg2 + n2 * kh2) * d.iK2;
    d.iw = rsqrt_nr(d.w2);
    d.w = d.w2 * d.iw;
    d.c = d.D * d.iK2 * d.iK2 * d.iw;
}

// ---------------------------------------------------------------------------- ray equations

struct Geo {
    double r, ir, hX, ihX, hY, sphi, cphi, tphi;
};

__device__ __forceinline__ void geometry_at(const Grid& G, double Y, double Z, Geo& g)
{
    if (G.geometry == 1) {
        sincos(Y, &g.sphi, &g.cphi);
        g.r = G.radius + Z;
        g.ir = rcp_nr(g.r);
        const double ic = rcp_nr(g.cphi);
        g.hX = g.r * g.cphi;
        g.ihX = g.ir * ic;
        g.hY = g.r;
        g.tphi = g.sphi * ic;
    } else {
        g.sphi = 0.0; g.cphi = 1.0; g.tphi = 0.0;
        g.r = 1.0; g.ir = 1.0; g.hX = 1.0; g.ihX = 1.0; g.hY = 1.0;
    }
}

// ------------------------------------------------------------ the ray equations in double-float
// The ray equations -- the carrier moves with the mean of the opposing face group velocities, the
// extents with their difference (Sec. 3b, App. B.1); the wavenumber follows Eq. eikonal-sphere:1-3
// (sphere) or kdot = -grad Omega (f-plane) with the centre values -- evaluated in double-float on
// the FP32 pipes (GB300's FP64 rate is 1/72 of its FP32 rate): the state enters
// as FP64 and is split (one FP64 subtraction per component), the nine rates leave as FP64.  Every
// intermediate carries about 48 significant bits, the reciprocal and reciprocal square root one
// Newton step in DF from the FP32 hardware approximations (~2^-45).

struct DispDF {
    DF K2, iK2, D, w2, iw, c;
};

__device__ __forceinline__ void dispersion_df(DF kh2, DF mg2, DF n2, DF f2, DispDF& d)
{
    d.K2 = df_add(kh2, mg2);
    d.D = df_sub(n2, f2);
    d.iK2 = df_rcp(d.K2);
    d.w2 = df_mul2(df_add(df_mul2(f2, mg2), df_mul2(n2, kh2)), d.iK2);
    d.iw = df_rsqrt(d.w2);
    d.c = df_mul2(df_mul2(d.D, df_mul2(d.iK2, d.iK2)), d.iw);
}

struct GeoDF {
    DF ir, ihX, sphi, cphi, tphi;
};

// sin and cos of the latitude from the row-centre table and the offset d from the centre
// (|d| <= half a row): sin(p0 + d) = s0 cos d + c0 sin d, cos(p0 + d) = c0 cos d - s0 sin d, with
// sin d and cos d from their Taylor series -- the terms up to d^3 and d^4 in DF, the smaller ones
// (below 3e-8 for rows of up to 9 degrees) in FP32, truncated after d^7 and d^8
__device__ __forceinline__ void lat_sincos_df(const Grid& G, DF Y, DF& sphi, DF& cphi)
{
    // the row only selects the expansion point: a neighbouring row near a boundary is as good
    const float fj = df_floor(df_mul2(df_sub(Y, DF{G.df_y0.x, G.df_y0.y}), DF{G.df_inv_dY.x, G.df_inv_dY.y}));
    const int j = fj < 0.0f ? 0 : (fj >= (float)(G.ny - 1) ? G.ny - 1 : (int)fj);
    const float2 rl = G.row_lat_df[j];
    const DF d = df_sub(Y, DF{rl.x, rl.y});
    const DF dd = df_mul2(d, d);
    constexpr DF sixth{1.0f / 6.0f, (float)(1.0 / 6.0 - (double)(1.0f / 6.0f))};
    constexpr DF twentyfourth{1.0f / 24.0f, (float)(1.0 / 24.0 - (double)(1.0f / 24.0f))};
    const float d2 = dd.hi;
    const float d4 = d2 * d2;
    const DF sind = df_add(df_sub(d, df_mul2(df_mul2(dd, d), sixth)),
                           df_f(d.hi * d4 * (1.0f / 120.0f - d2 * (1.0f / 5040.0f))));
    const DF cosd = df_sub(df_add(df_sub(df_f(1.0f), df_pow2(dd, 0.5f)), df_mul2(df_mul2(dd, dd), twentyfourth)),
                           df_f(d4 * d2 * (1.0f / 720.0f - d2 * (1.0f / 40320.0f))));
    const float2 sc0 = G.row_sc_df[2 * j], sc1 = G.row_sc_df[2 * j + 1];
    const DF s0{sc0.x, sc0.y}, c0{sc1.x, sc1.y};
    sphi = df_add(df_mul2(s0, cosd), df_mul2(c0, sind));
    cphi = df_sub(df_mul2(c0, cosd), df_mul2(s0, sind));
}

__device__ __forceinline__ void geometry_df(const Grid& G, DF Y, DF Z, GeoDF& g)
{
    if (G.geometry == 1) {
        lat_sincos_df(G, Y, g.sphi, g.cphi);
        const DF r = df_add(DF{G.df_radius.x, G.df_radius.y}, Z);
        g.ir = df_rcp(r);
        const DF ic = df_rcp(g.cphi);
        g.ihX = df_mul2(g.ir, ic);
        g.tphi = df_mul2(g.sphi, ic);
    } else {
        g.sphi = df_f(0.0f);
        g.cphi = df_f(1.0f);
        g.tphi = df_f(0.0f);
        g.ir = df_f(1.0f);
        g.ihX = df_f(1.0f);
    }
}

// ext_sh: when given, the three extents are read from there (float2 pairs kThreads apart) instead of
// y[6..8], which the caller then need not hold in registers
__device__ __forceinline__ void ray_rhs_df(const Grid& G, const NodeDF* __restrict__ bg, const DF y[9], DF R[9],
                                           const float2* ext_sh = nullptr)
{
    BgDF b;
    gather_df(G, bg, y[0], y[1], y[2], b);
    GeoDF g;
    geometry_df(G, y[1], y[2], g);
    DF f2, df2;
    if (G.geometry == 1) {
        const DF f = df_mul2(DF{G.df_2omega.x, G.df_2omega.y}, g.sphi);
        f2 = df_mul2(f, f);
        df2 = df_mul2(df_mul2(DF{G.df_8omega2.x, G.df_8omega2.y}, g.sphi), g.cphi);
    } else {
        f2 = DF{G.df_f0sq.x, G.df_f0sq.y};
        df2 = df_f(0.0f);
    }
    const DF k = y[3], l = y[4], m = y[5];
    const DF U = b.v[0], V = b.v[1], N2 = b.v[2], G2 = b.v[3];
    const DF kh2 = df_add(df_mul2(k, k), df_mul2(l, l)), m2 = df_mul2(m, m);
    const DF mg2 = df_add(m2, G2);
    DispDF d;
    dispersion_df(kh2, mg2, N2, f2, d);
    const DF mg2c = df_mul2(mg2, d.c);
    const DF cgx = df_add(df_mul2(k, mg2c), U);
    const DF cgy = df_add(df_mul2(l, mg2c), V);
    const DF cgz = df_neg(df_mul2(df_mul2(m, kh2), d.c));
    const DF hwK = df_pow2(df_mul2(d.iw, d.iK2), 0.5f);   // 1 / (2 w K^2)
    const DF aN = df_mul2(kh2, hwK);
    const DF aG = df_mul2(df_mul2(aN, d.D), d.iK2);
    const DF aF = df_mul2(mg2, hwK);
    DF Gq[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        Gq[q] = df_sub(df_add(df_add(df_mul2(k, b.d[0][q]), df_mul2(l, b.d[1][q])), df_mul2(aN, b.d[2][q])),
                       df_mul2(aG, b.d[3][q]));
    Gq[1] = df_add(Gq[1], df_mul2(aF, df2));
    if (G.columnar) {
        // single-column mode: k and l fixed, m by the vertical gradient of Omega alone
        R[3] = df_f(0.0f);
        R[4] = df_f(0.0f);
        R[5] = df_neg(Gq[2]);
    } else if (G.geometry == 1) {
        const DF ir = g.ir;
        R[3] = df_add(df_neg(df_mul2(Gq[0], g.ihX)), df_mul2(df_mul2(k, ir), df_sub(df_mul2(g.tphi, cgy), cgz)));
        R[4] = df_sub(df_neg(df_mul2(Gq[1], ir)), df_mul2(ir, df_add(df_mul2(l, cgz), df_mul2(df_mul2(k, g.tphi), cgx))));
        R[5] = df_add(df_neg(Gq[2]), df_mul2(ir, df_add(df_mul2(k, cgx), df_mul2(l, cgy))));
    } else {
        R[3] = df_neg(Gq[0]);
        R[4] = df_neg(Gq[1]);
        R[5] = df_neg(Gq[2]);
    }
    // faces: first-order Taylor values along the face's own axis.  The six face evaluations run as
    // one rolled loop (axis q, side sd) with the per-axis operands selected, not indexed: one copy of
    // the dispersion relation in the code instead of six keeps the kernel body small.
    int q0 = 0;
    if (G.columnar) {
        // no horizontal propagation or advection
        R[0] = R[1] = R[6] = R[7] = df_f(0.0f);
        q0 = 2;
    }
    const DF zero = df_f(0.0f);
    const DF mkh2 = df_mul2(m, kh2);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q < q0) continue;
        DF ext;
        if (ext_sh) {
            const float2 e2 = ext_sh[q * kThreads];
            ext = DF{e2.x, e2.y};
        } else {
            ext = q == 0 ? y[6] : (q == 1 ? y[7] : y[8]);
        }
        const DF dn = q == 0 ? b.d[2][0] : (q == 1 ? b.d[2][1] : b.d[2][2]);
        const DF dg = q == 0 ? b.d[3][0] : (q == 1 ? b.d[3][1] : b.d[3][2]);
        const DF dfq = q == 1 ? df2 : zero;     // f^2 varies along the meridional axis only
        const DF A = q == 0 ? k : l;
        const DF W = q == 0 ? U : V;
        const DF dW = q == 0 ? b.d[0][0] : b.d[1][1];
        const DF S = q == 0 ? g.ihX : g.ir;
        // the Taylor increments at the +h face, h = ext / 2; the -h face takes their negations (a
        // product by -h is the negated product by h, bit for bit)
        const DF h = df_pow2(ext, 0.5f);
        const DF tn = df_mul2(dn, h), tg = df_mul2(dg, h), tw = df_mul2(dW, h);
        const DF tf = q == 1 ? df_mul2(dfq, h) : zero;
        DF vel0 = zero, vel1 = zero;
#pragma unroll 1
        for (int sd = 0; sd < 2; ++sd) {
            const DF N2f = df_add(N2, sd == 0 ? tn : df_neg(tn));
            const DF G2f = df_add(G2, sd == 0 ? tg : df_neg(tg));
            const DF f2f = q == 1 ? df_add(f2, sd == 0 ? tf : df_neg(tf)) : f2;
            const DF mg2f = df_add(m2, G2f);
            DispDF e;
            dispersion_df(kh2, mg2f, N2f, f2f, e);
            const DF v = q < 2 ? df_mul2(df_add(df_add(df_mul2(df_mul2(A, mg2f), e.c), W), sd == 0 ? tw : df_neg(tw)), S)
                               : df_neg(df_mul2(mkh2, e.c));
            if (sd == 0)
                vel0 = v;
            else
                vel1 = v;
        }
        const DF rc = df_pow2(df_add(vel0, vel1), 0.5f), re = df_sub(vel0, vel1);
        if (q == 0) {
            R[0] = rc;
            R[6] = re;
        } else if (q == 1) {
            R[1] = rc;
            R[7] = re;
        } else {
            R[2] = rc;
            R[8] = re;
        }
    }
}

// Intrinsic quantities of a ray volume at its carrier position in double-float (the FP64 form's
// saturation and projection): wavenumbers, f^2, N^2 and the dispersion terms, from N^2 and Gamma^2
// interpolated alone.
struct IntrDF {
    DF k, l, m, kh2, m2, mg2, f, f2, n2;   // f: the signed Coriolis parameter at the ray
    DispDF d;
};

__device__ __forceinline__ void intrinsic_df(const Grid& G, const NodeDF* __restrict__ bg, const double s[NSTATE],
                                             IntrDF& in)
{
    DF g2;
    const DF Y = df_split(s[SY]);
    gather_n2g2_df(G, bg, df_split(s[SX]), Y, df_split(s[SZ]), in.n2, g2);
    if (G.geometry == 1) {
        DF sphi, cphi;
        lat_sincos_df(G, Y, sphi, cphi);
        in.f = df_mul2(DF{G.df_2omega.x, G.df_2omega.y}, sphi);
        in.f2 = df_mul2(in.f, in.f);
    } else {
        in.f = DF{G.df_f0.x, G.df_f0.y};
        in.f2 = DF{G.df_f0sq.x, G.df_f0sq.y};
    }
    in.k = df_split(s[SK]);
    in.l = df_split(s[SL]);
    in.m = df_split(s[SM]);
    in.kh2 = df_add(df_mul2(in.k, in.k), df_mul2(in.l, in.l));
    in.m2 = df_mul2(in.m, in.m);
    in.mg2 = df_add(in.m2, g2);
    dispersion_df(in.kh2, in.mg2, in.n2, in.f2, in.d);
}

// Williamson (1980) low-storage RK3 on the 9 propagated components; background frozen.  The rates
// and the low-storage register q are double-float; the step's increments B q of the three stages
// are summed in double-float and added to the FP64 state once, at the end (one FP64 rounding per
// component instead of three: the sum is far smaller than the state, so its 48 bits are ample), and
// a double-float copy of the state, updated by the same B q, feeds the next evaluation.  The FP64
// state and the increment sums wait in shared memory during the stages (sh: this thread's first
// slot, slots kThreads apart: 9 doubles, then 9 float2 sums at sh + 9 kThreads), which keeps them
// out of the registers the ray equations need; with kQShared the low-storage register q waits there
// too (9 float2 at sh + 18 kThreads; 27 kThreads doubles in all).
template <bool kQShared = false, bool kExtShared = false>
__device__ __forceinline__ void rk3(const Grid& G, const NodeDF* __restrict__ bg, double s[NSTATE], double dt,
                                    double* sh)
{
    constexpr DF A1{-5.0f / 9.0f, (float)(-5.0 / 9.0 - (double)(-5.0f / 9.0f))};
    constexpr DF A2{-153.0f / 128.0f, 0.0f};
    constexpr DF B0{1.0f / 3.0f, (float)(1.0 / 3.0 - (double)(1.0f / 3.0f))};
    constexpr DF B1{15.0f / 16.0f, 0.0f};
    constexpr DF B2{8.0f / 15.0f, (float)(8.0 / 15.0 - (double)(8.0f / 15.0f))};
    const DF dtd = df_split(dt);
    DF y[9], q[kQShared ? 1 : 9];
    float2* acc = reinterpret_cast<float2*>(sh + 9 * kThreads);
    float2* qs = acc + 9 * kThreads;
    float2* es = qs + 9 * kThreads;   // the extents' double-float copy (kExtShared)
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        y[c] = df_split(s[c]);
        if (!kQShared) q[c] = df_f(0.0f);
        sh[c * kThreads] = s[c];
        acc[c * kThreads] = make_float2(0.0f, 0.0f);
        if (kExtShared && c >= 6) es[(c - 6) * kThreads] = make_float2(y[c].hi, y[c].lo);
    }
#pragma unroll 1
    for (int st = 0; st < 3; ++st) {
        DF F[9];
        ray_rhs_df(G, bg, y, F, kExtShared ? es : nullptr);
        const DF a = st == 1 ? A1 : A2;
        const DF b = st == 0 ? B0 : (st == 1 ? B1 : B2);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            DF qc;
            if (kQShared) {
                const float2 qo = qs[c * kThreads];
                qc = st == 0 ? df_mul2(dtd, F[c]) : df_add(df_mul2(a, DF{qo.x, qo.y}), df_mul2(dtd, F[c]));
                qs[c * kThreads] = make_float2(qc.hi, qc.lo);
            } else {
                qc = st == 0 ? df_mul2(dtd, F[c]) : df_add(df_mul2(a, q[c]), df_mul2(dtd, F[c]));
                q[c] = qc;
            }
            const DF bq = df_mul2(b, qc);
            const float2 o = acc[c * kThreads];
            const DF na = df_add(DF{o.x, o.y}, bq);
            acc[c * kThreads] = make_float2(na.hi, na.lo);
            if (kExtShared && c >= 6) {
                const float2 ye = es[(c - 6) * kThreads];
                const DF yn = df_add(DF{ye.x, ye.y}, bq);
                es[(c - 6) * kThreads] = make_float2(yn.hi, yn.lo);
            } else {
                y[c] = df_add(y[c], bq);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const float2 o = acc[c * kThreads];
        s[c] = sh[c * kThreads] + df_to_double(DF{o.x, o.y});
    }
}

// ---------------------------------------------------------------------------- bookkeeping

__device__ __forceinline__ double wrap_period(double x, double L)
{
    double w = x - L * floor(x / L);
    if (w < 0.0) w += L;
    if (w >= L) w = 0.0;
    return w;
}

__device__ __forceinline__ void wrap_position(const Grid& G, double s[NSTATE])
{
    // most carriers stay inside the period: skip the division then
    if (!(s[SX] >= 0.0 && s[SX] < G.Lx)) s[SX] = wrap_period(s[SX], G.Lx);
    if (G.geometry == 0 && !(s[SY] >= 0.0 && s[SY] < G.Ly)) s[SY] = wrap_period(s[SY], G.Ly);
}

__device__ __forceinline__ double ray_action(const double s[NSTATE])
{
    return s[SN] * s[SPX] * s[SPY] * s[SPZ];
}

// 0 inside, 1 left the domain, 2 not a valid ray volume
__device__ __forceinline__ int ray_status(const Grid& G, const double s[NSTATE])
{
    // finiteness from the exponent bits (integer pipe): all ones means infinity or NaN
    unsigned allf = 0u;
#pragma unroll
    for (int c = 0; c < NSTATE; ++c) allf |= ((((unsigned)__double2hiint(s[c]) >> 20) & 0x7FFu) + 1u) & 0x800u;
    if (allf) return 2;
    if (!(s[SEX] > 0.0 && s[SEY] > 0.0 && s[SEZ] > 0.0)) return 2;
    if (!(s[SZ] >= 0.0 && s[SZ] < G.ztop)) return 1;
    if (G.geometry == 1 && !(fabs(s[SY]) <= G.phimax)) return 1;
    return 0;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ void cell_ijk(const Grid& G, const double s[NSTATE], int& i, int& j, int& k)
{
    i = clampi((int)floor(s[SX] * G.inv_dX), 0, G.nx - 1);
    j = clampi((int)floor((s[SY] - G.y0) * G.inv_dY), 0, G.ny - 1);
    k = clampi((int)floor(s[SZ] * G.inv_dz), 0, G.nz - 1);
}

__device__ __forceinline__ int cell_of(const Grid& G, const double s[NSTATE])
{
    int i, j, k;
    cell_ijk(G, s, i, j, k);
    return (j * G.nx + i) * G.nz + k;
}

// latitude of row j's centre, multiply then add (never contracted into an FMA)
__device__ __forceinline__ double row_lat(const Grid& G, int j) { return __dadd_rn(G.y0, __dmul_rn(j + 0.5, G.dY)); }

// Split decision (App. B.3): bit 0 vertical, bit 1 horizontal, bit 2 horizontal axis is y.
__device__ __forceinline__ int split_code(const Grid& G, const Params& P, const double s[NSTATE])
{
    if (!P.splitting) return 0;
    int code = 0;
    if (s[SEZ] > G.split_hthr) code |= 1;
    double xlen, ylen, thr, area, athr;
    if (G.geometry == 1) {
        int i, j, k;
        cell_ijk(G, s, i, j, k);
        DF sphi, cphi;
        lat_sincos_df(G, df_split(s[SY]), sphi, cphi);
        const double cp = df_to_double(cphi);
        xlen = cp * s[SEX];
        ylen = s[SEY];
        thr = G.split_thr[2 * j];
        area = cp * s[SEX] * s[SEY];
        athr = G.split_thr[2 * j + 1];
    } else {
        xlen = s[SEX];
        ylen = s[SEY];
        thr = G.split_thr[0];
        area = s[SEX] * s[SEY];
        athr = G.split_thr[1];
    }
    if (xlen > thr || ylen > thr || area > athr) code |= (xlen >= ylen) ? 2 : 6;
    return code;
}

__device__ __forceinline__ int num_children(int code) { return ((code & 1) ? 2 : 1) * ((code & 2) ? 2 : 1); }

// one axis of a split: the half at +-1/4 of the extent, half the extent and half the product
__device__ __forceinline__ void halve(double& x, double& ext, double& P, bool plus)
{
    x += (plus ? 0.25 : -0.25) * ext;
    ext *= 0.5;
    P *= 0.5;
}

// Child c of a split parent: children are ordered (lower, upper) x (minus, plus) with the
// vertical index fastest; child 0 keeps the parent id, child c > 0 takes the (c-1)-th new id.
__device__ __forceinline__ void make_child(const Grid& G, const double p[NSTATE], int code, int c, double s[NSTATE])
{
#pragma unroll
    for (int q = 0; q < NSTATE; ++q) s[q] = p[q];
    const int nv = (code & 1) ? 2 : 1;
    if (code & 1) halve(s[SZ], s[SEZ], s[SPZ], (c % nv) == 1);
    if (code & 2) {
        const bool plus = (c / nv) == 1;
        if (code & 4) halve(s[SY], s[SEY], s[SPY], plus);
        else halve(s[SX], s[SEX], s[SPX], plus);
    }
    if (code) wrap_position(G, s);
}


// Intrinsic properties of a ray volume at its carrier position (saturation, projection, cap).
struct Intr {
    double kh2, m2, mg2, K2, iK2, D, w, iw, w2, c, f2, n2;
};

__device__ __forceinline__ void intrinsic_at(const Grid& G, const NodeDF* __restrict__ bg, const double s[NSTATE],
                                             Geo& g, Intr& in)
{
    Bg b;
    gather(G, bg, s[SX], s[SY], s[SZ], b);
    geometry_at(G, s[SY], s[SZ], g);
    double df2;
    coriolis(G, g.sphi, g.cphi, in.f2, df2);
    in.kh2 = s[SK] * s[SK] + s[SL] * s[SL];
    in.m2 = s[SM] * s[SM];
    in.n2 = b.v[2];
    in.mg2 = in.m2 + b.v[3];
    Disp d;
    dispersion(in.kh2, in.mg2, b.v[2], in.f2, d);
    in.K2 = d.K2;
    in.iK2 = d.iK2;
    in.D = d.D;
    in.w = d.w;
    in.iw = d.iw;
    in.w2 = d.w2;
    in.c = d.c;
}

}  // namespace gwam
