// gwam_fp32.cuh -- the precision form: ray kinematics in FP32 with positions stored as an integer
// cell index plus FP32 offsets in cell units; FP64 only for the saturation sums, the flux
// accumulation and the wave-action budget.  Same equations as the FP64 form (Sec. 2a Eq.
// dispersion, Eq. eikonal, Eq. eikonal-sphere:1-3; Sec. 3a, 3b; App. B.1-B.3).
#pragma once

#include "gwam_ctx.cuh"

namespace gwam {


struct S32 {
    int i, j, k;       // base cell
    float o[3];        // position in cell units relative to the base cell
    float w[3];        // k, l, m
    float e[3];        // extents
    float p[3];        // Px, Py, Pz
    float n;
    long long id;
};

__device__ __forceinline__ void load32(const Grid& G, const Ray32SoA& R, int64_t idx, S32& s)
{
    const float4 a = R.q[0][idx], b = R.q[1][idx], c = R.q[2][idx], d = R.q[3][idx];
    const int cell = __float_as_int(a.x);
    s.k = cell % G.nz;
    const int col = cell / G.nz;
    s.i = col % G.nx;
    s.j = col / G.nx;
    s.o[0] = a.y; s.o[1] = a.z; s.o[2] = a.w;
    s.w[0] = b.x; s.w[1] = b.y; s.w[2] = b.z; s.n = b.w;
    s.e[0] = c.x; s.e[1] = c.y; s.e[2] = c.z; s.p[0] = c.w;
    s.p[1] = d.x; s.p[2] = d.y;
    s.id = (long long)(((unsigned long long)(unsigned)__float_as_int(d.w) << 32) | (unsigned)__float_as_int(d.z));
}

__device__ __forceinline__ void store32(const Grid& G, const Ray32SoA& R, int64_t idx, const S32& s)
{
    const int cell = (s.j * G.nx + s.i) * G.nz + s.k;
    R.q[0][idx] = make_float4(__int_as_float(cell), s.o[0], s.o[1], s.o[2]);
    R.q[1][idx] = make_float4(s.w[0], s.w[1], s.w[2], s.n);
    R.q[2][idx] = make_float4(s.e[0], s.e[1], s.e[2], s.p[0]);
    R.q[3][idx] = make_float4(s.p[1], s.p[2], __int_as_float((int)(unsigned)(unsigned long long)s.id),
                              __int_as_float((int)(unsigned)((unsigned long long)s.id >> 32)));
}

// wave-action content N Px Py Pz of the FP32 fields, formed in FP64 (the budget is FP64)
__device__ __forceinline__ double action32(const S32& s)
{
    return (double)s.n * (double)s.p[0] * (double)s.p[1] * (double)s.p[2];
}

// N Px Py Pz as a double-float (relative error about 2^-47)
__device__ __forceinline__ DF action_df(const S32& s)
{
    return df_mul(df_mul(df_prod(s.n, s.p[0]), s.p[1]), s.p[2]);
}

// ------------------------------------------------------------------------------ gather

struct Bg32 {
    float v[4];
    float d[4][3];
};

// bracketing node pair from base index b and offset o (cell units); node q sits at offset 0.5
__device__ __forceinline__ void bracket32(int b, float o, int n, bool periodic, int& q0, int& q1, float& t)
{
    float s = o - 0.5f;
    if (!isfinite(s)) s = 0.0f;
    const float fl = floorf(s);
    t = s - fl;
    int q = b + (int)fl;
    if (periodic) {
        q0 = wrap_int(q, n);
        q1 = q0 + 1 == n ? 0 : q0 + 1;
    } else if (q < 0) {
        q0 = 0; q1 = 1; t = 0.0f;
    } else if (q >= n - 1) {
        q0 = n - 2; q1 = n - 1; t = 1.0f;
    } else {
        q0 = q; q1 = q + 1;
    }
}

// acc += w * node.  kWide: the node's 64 bytes as two 32-byte loads per lane (ld.global.nc.v8.f32;
// nodes are 64-byte aligned) instead of four 16-byte ones -- half the L1 requests of the gather,
// whose lanes touch up to 32 distinct lines per request (the ray step: 0.63 -> 0.55 ms per step on
// the 512 x 256 sphere; the projection and saturation kernels were measured slightly slower with
// it and keep the 16-byte loads)
template <bool kWide>
__device__ __forceinline__ void accumulate32(const Node32* __restrict__ p, float w, float* acc)
{
    if (kWide) {
        const float* q = reinterpret_cast<const float*>(p);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float a[8];
            asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
                : "l"(q + 8 * h));
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[8 * h + e] = fmaf(w, a[e], acc[8 * h + e]);
        }
    } else {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 a = __ldg(q + e);
            acc[4 * e] = fmaf(w, a.x, acc[4 * e]);
            acc[4 * e + 1] = fmaf(w, a.y, acc[4 * e + 1]);
            acc[4 * e + 2] = fmaf(w, a.z, acc[4 * e + 2]);
            acc[4 * e + 3] = fmaf(w, a.w, acc[4 * e + 3]);
        }
    }
}

template <bool kWide = false>
__device__ __forceinline__ void gather32(const Grid& G, const Node32* __restrict__ bg, const S32& s, const float o[3],
                                         Bg32& b)
{
    int i0, i1, j0, j1, k0, k1;
    float tx, ty, tz;
    bracket32(s.i, o[0], G.nx, true, i0, i1, tx);
    bracket32(s.j, o[1], G.ny, G.geometry == 0, j0, j1, ty);
    bracket32(s.k, o[2], G.nz, false, k0, k1, tz);
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    const float ux = 1.0f - tx, uy = 1.0f - ty, uz = 1.0f - tz;
    const int dk = k1 - k0;
    const Node32* c00 = bg + node_index(G, i0, j0, k0);
    const Node32* c10 = bg + node_index(G, i1, j0, k0);
    const Node32* c01 = bg + node_index(G, i0, j1, k0);
    const Node32* c11 = bg + node_index(G, i1, j1, k0);
    accumulate32<kWide>(c00, ux * uy * uz, acc);
    accumulate32<kWide>(c00 + dk, ux * uy * tz, acc);
    accumulate32<kWide>(c10, tx * uy * uz, acc);
    accumulate32<kWide>(c10 + dk, tx * uy * tz, acc);
    accumulate32<kWide>(c01, ux * ty * uz, acc);
    accumulate32<kWide>(c01 + dk, ux * ty * tz, acc);
    accumulate32<kWide>(c11, tx * ty * uz, acc);
    accumulate32<kWide>(c11 + dk, tx * ty * tz, acc);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        b.v[f] = acc[f];
#pragma unroll
        for (int q = 0; q < 3; ++q) b.d[f][q] = acc[4 + 3 * f + q];
    }
}

// ------------------------------------------------------------------------------ geometry, dispersion

struct Geo32 {
    float r, ir, hX, ihX, sphi, cphi, tphi;
};

__device__ __forceinline__ void geo32(const Grid& G, const S32& s, const float o[3], Geo32& g)
{
    if (G.geometry == 1) {
        const float phi = G.f_y0 + ((float)s.j + o[1]) * G.f_dY;
        sincosf(phi, &g.sphi, &g.cphi);
        g.r = G.f_radius + ((float)s.k + o[2]) * G.f_dz;
        g.ir = __frcp_rn(g.r);
        const float ic = __frcp_rn(g.cphi);
        g.hX = g.r * g.cphi;
        g.ihX = g.ir * ic;
        g.tphi = g.sphi * ic;
    } else {
        g.sphi = 0.0f; g.cphi = 1.0f; g.tphi = 0.0f;
        g.r = 1.0f; g.ir = 1.0f; g.hX = 1.0f; g.ihX = 1.0f;
    }
}

__device__ __forceinline__ void coriolis32(const Grid& G, const Geo32& g, float& f2, float& df2)
{
    if (G.geometry == 1) {
        const float om = G.f_omega;
        const float f = 2.0f * om * g.sphi;
        f2 = f * f;
        df2 = 8.0f * om * om * g.sphi * g.cphi;
    } else {
        f2 = G.f_f0 * G.f_f0;
        df2 = 0.0f;
    }
}

struct Disp32 {
    float K2, iK2, D, w2, w, iw, c;
};

__device__ __forceinline__ void dispersion32(float kh2, float mg2, float n2, float f2, Disp32& d)
{
    d.K2 = kh2 + mg2;
    d.D = n2 - f2;
    d.iK2 = __frcp_rn(d.K2);
    d.w2 = (f2 * mg2 + n2 * kh2) * d.iK2;
    d.iw = rsqrtf(d.w2);
    d.w = d.w2 * d.iw;
    d.c = d.D * d.iK2 * d.iK2 * d.iw;
}

// ------------------------------------------------------------------------------ ray equations

// y = (ox, oy, oz in cell units relative to the base cell, k, l, m, eX, eY, eZ); F the rates
__device__ __forceinline__ void rhs32(const Grid& G, const Node32* __restrict__ bg, const S32& s, const float y[9],
                                      float F[9])
{
    const float k = y[3], l = y[4], m = y[5];
    Bg32 b;
    gather32<true>(G, bg, s, y, b);
    Geo32 g;
    geo32(G, s, y, g);
    float f2, df2;
    coriolis32(G, g, f2, df2);
    const float U = b.v[0], V = b.v[1], N2 = b.v[2], G2 = b.v[3];
    const float kh2 = k * k + l * l, m2 = m * m;
    const float mg2 = m2 + G2;
    Disp32 d;
    dispersion32(kh2, mg2, N2, f2, d);
    const float cgx = k * mg2 * d.c + U;
    const float cgy = l * mg2 * d.c + V;
    const float cgz = -m * kh2 * d.c;
    const float hwK = 0.5f * d.iw * d.iK2;
    const float aN = kh2 * hwK;
    const float aG = aN * d.D * d.iK2;
    const float aF = mg2 * hwK;
    float Gq[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) Gq[q] = k * b.d[0][q] + l * b.d[1][q] + aN * b.d[2][q] - aG * b.d[3][q];
    Gq[1] += aF * df2;
    if (G.columnar) {
        // single-column mode: k and l fixed, m by the vertical gradient of Omega alone
        F[3] = 0.0f;
        F[4] = 0.0f;
        F[5] = -Gq[2];
    } else if (G.geometry == 1) {
        F[3] = -Gq[0] * g.ihX + k * g.ir * (g.tphi * cgy - cgz);
        F[4] = -Gq[1] * g.ir - g.ir * (l * cgz + k * g.tphi * cgx);
        F[5] = -Gq[2] + g.ir * (k * cgx + l * cgy);
    } else {
        F[3] = -Gq[0];
        F[4] = -Gq[1];
        F[5] = -Gq[2];
    }
    // face group velocities -> coordinate rates -> cell units
    const float scale[3] = {g.ihX * G.f_inv_dX, g.ir * G.f_inv_dY, G.f_inv_dz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (G.columnar && q < 2) {
            // no horizontal propagation or advection
            F[q] = 0.0f;
            F[6 + q] = 0.0f;
            continue;
        }
        float vel[2];
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
            const float h = (sd == 0 ? 0.5f : -0.5f) * y[6 + q];
            const float N2f = N2 + b.d[2][q] * h;
            const float G2f = G2 + b.d[3][q] * h;
            const float f2f = (q == 1) ? f2 + df2 * h : f2;
            const float mg2f = m2 + G2f;
            Disp32 e;
            dispersion32(kh2, mg2f, N2f, f2f, e);
            if (q == 0) vel[sd] = k * mg2f * e.c + U + b.d[0][0] * h;
            else if (q == 1) vel[sd] = l * mg2f * e.c + V + b.d[1][1] * h;
            else vel[sd] = -m * kh2 * e.c;
        }
        F[q] = 0.5f * (vel[0] + vel[1]) * scale[q];
        // extent rates in coordinate units
        const float cs = q == 0 ? g.ihX : (q == 1 ? g.ir : 1.0f);
        F[6 + q] = (vel[0] - vel[1]) * cs;
    }
}

__device__ __forceinline__ void rk3_32(const Grid& G, const Node32* __restrict__ bg, S32& s, float dt)
{
    float y[9] = {s.o[0], s.o[1], s.o[2], s.w[0], s.w[1], s.w[2], s.e[0], s.e[1], s.e[2]};
    float q[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) q[c] = 0.0f;
#pragma unroll 1
    for (int st = 0; st < 3; ++st) {
        float F[9];
        rhs32(G, bg, s, y, F);
        // the stage's coefficients selected, not indexed (an array indexed by the rolled stage
        // counter would live in local memory, whose loads share L1 with the gathers)
        const float a = st == 0 ? 0.0f : (st == 1 ? -5.0f / 9.0f : -153.0f / 128.0f);
        const float b = st == 0 ? 1.0f / 3.0f : (st == 1 ? 15.0f / 16.0f : 8.0f / 15.0f);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            q[c] = a * q[c] + dt * F[c];
            y[c] += b * q[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s.o[c] = y[c];
        s.w[c] = y[3 + c];
        s.e[c] = y[6 + c];
    }
}

// Move the base cell so that the offsets fall in [0, 1); returns 0 inside, 1 left the domain,
// 2 invalid.  Sphere: beyond the centre of the last row leaves (as in the FP64 form).
__device__ __forceinline__ int renormalize32(const Grid& G, S32& s)
{
    bool finite = isfinite(s.n) && isfinite(s.p[0]) && isfinite(s.p[1]) && isfinite(s.p[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) finite = finite && isfinite(s.o[c]) && isfinite(s.w[c]) && isfinite(s.e[c]);
    if (!finite) return 2;
    if (!(s.e[0] > 0.0f && s.e[1] > 0.0f && s.e[2] > 0.0f)) return 2;
    if (fabsf(s.o[0]) > 1e6f || fabsf(s.o[1]) > 1e6f || fabsf(s.o[2]) > 1e6f) return 1;
    float fx = floorf(s.o[0]), fy = floorf(s.o[1]), fz = floorf(s.o[2]);
    s.o[0] -= fx;
    s.o[1] -= fy;
    s.o[2] -= fz;
    // rounding can leave exactly 1.0
    if (s.o[0] >= 1.0f) { s.o[0] = 0.0f; fx += 1.0f; }
    if (s.o[1] >= 1.0f) { s.o[1] = 0.0f; fy += 1.0f; }
    if (s.o[2] >= 1.0f) { s.o[2] = 0.0f; fz += 1.0f; }
    s.i = wrap_int(s.i + (int)fx, G.nx);
    const int jj = s.j + (int)fy, kk = s.k + (int)fz;
    if (kk < 0 || kk >= G.nz) return 1;
    s.k = kk;
    if (G.geometry == 1) {
        const float yc = (float)jj + s.o[1];
        if (!(yc >= 0.5f && yc <= (float)G.ny - 0.5f)) return 1;
        s.j = jj;
    } else {
        s.j = wrap_int(jj, G.ny);
    }
    return 0;
}

__device__ __forceinline__ int split_code32(const Grid& G, const Params& P, const S32& s)
{
    if (!P.splitting) return 0;
    int code = 0;
    if (s.e[2] > fmaxf((float)(P.alpha_s * G.dz), (float)P.min_split_dz)) code |= 1;
    float xlen, ylen, thr, area, athr;
    const float a = P.f_alpha_s, dX = G.f_dX, dY = G.f_dY;
    if (G.geometry == 1) {
        const float cj = G.row_cos32[s.j];
        const float cp = cosf(G.f_y0 + ((float)s.j + s.o[1]) * dY);
        xlen = cp * s.e[0];
        ylen = s.e[1];
        thr = a * sqrtf(cj * dX * dY);
        area = cp * s.e[0] * s.e[1];
        athr = a * cj * dX * dY;
    } else {
        xlen = s.e[0];
        ylen = s.e[1];
        thr = a * sqrtf(dX * dY);
        area = s.e[0] * s.e[1];
        athr = a * dX * dY;
    }
    if (xlen > thr || ylen > thr || area > athr) code |= (xlen >= ylen) ? 2 : 6;
    return code;
}

// child c (vertical index fastest, as in the FP64 form); returns its status after renormalising
__device__ __forceinline__ int make_child32(const Grid& G, const S32& p, int code, int c, S32& s)
{
    s = p;
    if (!code) return 0;
    const int nv = (code & 1) ? 2 : 1;
    if (code & 1) {
        const bool plus = (c % nv) == 1;
        s.o[2] += (plus ? 0.25f : -0.25f) * s.e[2] * G.f_inv_dz;
        s.e[2] *= 0.5f;
        s.p[2] *= 0.5f;
    }
    // the halved horizontal axis by branch, not by index: a state indexed at run time would be
    // kept in local memory
    if (code & 2) {
        const float h = (c / nv) == 1 ? 0.25f : -0.25f;
        if (code & 4) {
            s.o[1] += h * s.e[1] * G.f_inv_dY;
            s.e[1] *= 0.5f;
            s.p[1] *= 0.5f;
        } else {
            s.o[0] += h * s.e[0] * G.f_inv_dX;
            s.e[0] *= 0.5f;
            s.p[0] *= 0.5f;
        }
    }
    return renormalize32(G, s);
}

__device__ __forceinline__ int cell32(const Grid& G, const S32& s) { return (s.j * G.nx + s.i) * G.nz + s.k; }

// intrinsic properties of a ray volume at its carrier (saturation, projection, cap)
struct Intr32 {
    float kh2, m2, mg2, K2, iK2, D, w, iw, w2, c, f2, n2;
    Geo32 g;
};

__device__ __forceinline__ void intrinsic32(const Grid& G, const Node32* __restrict__ bg, const S32& s, Intr32& in)
{
    Bg32 b;
    gather32(G, bg, s, s.o, b);
    geo32(G, s, s.o, in.g);
    float df2;
    coriolis32(G, in.g, in.f2, df2);
    in.kh2 = s.w[0] * s.w[0] + s.w[1] * s.w[1];
    in.m2 = s.w[2] * s.w[2];
    in.n2 = b.v[2];
    in.mg2 = in.m2 + b.v[3];
    Disp32 d;
    dispersion32(in.kh2, in.mg2, b.v[2], in.f2, d);
    in.K2 = d.K2;
    in.iK2 = d.iK2;
    in.D = d.D;
    in.w = d.w;
    in.iw = d.iw;
    in.w2 = d.w2;
    in.c = d.c;
}

// FP64 state (absolute coordinates) -> FP32 record fields (base cell + offsets)
__device__ __forceinline__ void from_double(const Grid& G, const double d[NSTATE], long long id, S32& s)
{
    const double cx = d[SX] * G.inv_dX, cy = (d[SY] - G.y0) * G.inv_dY, cz = d[SZ] * G.inv_dz;
    s.i = clampi((int)floor(cx), 0, G.nx - 1);
    s.j = clampi((int)floor(cy), 0, G.ny - 1);
    s.k = clampi((int)floor(cz), 0, G.nz - 1);
    s.o[0] = (float)(cx - s.i);
    s.o[1] = (float)(cy - s.j);
    s.o[2] = (float)(cz - s.k);
    s.w[0] = (float)d[SK]; s.w[1] = (float)d[SL]; s.w[2] = (float)d[SM];
    s.e[0] = (float)d[SEX]; s.e[1] = (float)d[SEY]; s.e[2] = (float)d[SEZ];
    s.p[0] = (float)d[SPX]; s.p[1] = (float)d[SPY]; s.p[2] = (float)d[SPZ];
    s.n = (float)d[SN];
    s.id = id;
}

__device__ __forceinline__ void to_double(const Grid& G, const S32& s, double d[NSTATE])
{
    d[SX] = ((double)s.i + (double)s.o[0]) * G.dX;
    d[SY] = G.y0 + ((double)s.j + (double)s.o[1]) * G.dY;
    d[SZ] = ((double)s.k + (double)s.o[2]) * G.dz;
    d[SK] = s.w[0]; d[SL] = s.w[1]; d[SM] = s.w[2];
    d[SEX] = s.e[0]; d[SEY] = s.e[1]; d[SEZ] = s.e[2];
    d[SPX] = s.p[0]; d[SPY] = s.p[1]; d[SPZ] = s.p[2];
    d[SN] = s.n;
}

}  // namespace gwam
