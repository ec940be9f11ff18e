// gwam_launch.cu -- background upload, explicit ray volumes, and the wave sources.
//
//   background: column-major node fields + Gamma^2 from rho (Sec. 2a; Gamma^2 = (d ln rho / dz)^2 / 4,
//               centred differences between node levels, one-sided at the ends)
//   sources:    background source of Sec. 3c (alpha(phi), F_sol, F_am) and explicit spectral bins;
//               intrinsic frequency w = |k_h| c - k.U, bins outside |f| < w < N or with m^2 <= 0 are
//               filtered, m from the inverted Eq. dispersion, m < 0 (upward group velocity),
//               A = F / (|k_h| ch_r).
#include "gwam_common.cuh"
#include "gwam_fp32.cuh"

namespace gwam {

enum { BG_NONFINITE = 1, BG_RHO = 2, BG_N2F2 = 4 };

// exponent bits all ones: infinity or NaN (integer pipe)
__device__ __forceinline__ bool nonfinite_bits(double x)
{
    return ((((unsigned)__double2hiint(x) >> 20) & 0x7FFu) == 0x7FFu);
}

// caller [nz][ny][nx] -> column-major node values (U, V, N^2, Gamma^2) and rho, transposed through
// shared memory (kBgTile columns of a row per block: 8 columns, 23 KB of shared memory, eight blocks
// per SM; 16 columns, four blocks per SM, took 37 us more of the set-up).  Gamma^2 =
// (d ln rho / dz)^2 / 4 by centred differences of ln rho (one-sided at the bottom and top), each
// difference taken as the logarithm of the density ratio in double-float (df_log_ratio); 1/rho by
// the Newton reciprocal; f^2 of the row from the host table.
constexpr int kBgTile = 8;
__global__ void k_set_background(Grid G, int gamma_mode, const double* __restrict__ u, const double* __restrict__ v,
                                 const double* __restrict__ n2, const double* __restrict__ rho, Node* __restrict__ bg,
                                 double* __restrict__ rho_c, double* __restrict__ rho_inv, int* flags)
{
    extern __shared__ double sh[];   // 4 arrays x nz x kBgTile: U, V, N^2, rho
    const int TW = kBgTile;
    const int nz = G.nz;
    const int ntx = (G.nx + TW - 1) / TW;
    const int j = blockIdx.x / ntx, i0 = (blockIdx.x % ntx) * TW;
    double* su = sh;
    double* sv = sh + nz * TW;
    double* sn = sh + 2 * nz * TW;
    double* sr = sh + 3 * nz * TW;
    int bad = 0;
    for (int t = threadIdx.x; t < nz * TW; t += blockDim.x) {
        const int ii = t % TW, k = t / TW, i = i0 + ii;
        if (i >= G.nx) continue;
        const int64_t o = ((int64_t)k * G.ny + j) * G.nx + i;
        const double a = u[o], b = v[o], c = n2[o], d = rho[o];
        su[k * TW + ii] = a;
        sv[k * TW + ii] = b;
        sn[k * TW + ii] = c;
        sr[k * TW + ii] = d;
        if (nonfinite_bits(a) || nonfinite_bits(b) || nonfinite_bits(c) || nonfinite_bits(d)) bad |= BG_NONFINITE;
        else if (__double_as_longlong(d) <= 0) bad |= BG_RHO;   // rho <= 0 (or -0)
    }
    __syncthreads();
    const double f2 = G.row_f2[j];
    const DF h1{G.df_inv_dz.x, G.df_inv_dz.y};
    const DF h2 = df_pow2(h1, 0.5f);
    for (int t = threadIdx.x; t < nz * TW; t += blockDim.x) {
        const int k = t % nz, ii = t / nz, i = i0 + ii;
        if (i >= G.nx) continue;
        const double r = sr[k * TW + ii];
        const bool rok = __double_as_longlong(r) > 0 && !nonfinite_bits(r);
        double g2 = 0.0;
        if (gamma_mode) {
            const int ku = k == nz - 1 ? k : k + 1, kd = k == 0 ? 0 : k - 1;
            const double ru = sr[ku * TW + ii], rd = sr[kd * TW + ii];
            if (rok && __double_as_longlong(ru) > 0 && __double_as_longlong(rd) > 0 && !nonfinite_bits(ru) &&
                !nonfinite_bits(rd)) {
                const DF dl = df_mul2(df_log_ratio(ru, rd), (k == 0 || k == nz - 1) ? h1 : h2);
                g2 = df_to_double(df_pow2(df_mul2(dl, dl), 0.25f));
            }
        }
        const double nn = sn[k * TW + ii];
        if (!(nn > f2)) bad |= BG_N2F2;
        const int64_t c = node_index(G, i, j, k);
        *reinterpret_cast<double4*>(bg[c].v) = make_double4(su[k * TW + ii], sv[k * TW + ii], nn, g2);
        rho_c[c] = r;
        rho_inv[c] = rok ? rcp_nr(r) : 0.0;
    }
    if (bad) atomicOr(flags, bad);
}

// Node gradients by centred differences: periodic in x (and y on the f-plane), one-sided at the
// pole rows and at the bottom and top levels.  The same pass writes the per-step gather copies of
// the node: double-float pairs (FP64 form, bgdf) or FP32 (precision form, bg32), whichever is given.
// At most 85 registers, three blocks per SM: the pass waits on its neighbour loads (at 88 registers
// and two blocks per SM the whole set-up took 0.267 ms, with three 0.241 ms).
__global__ void __launch_bounds__(256, 3) k_node_gradients(Grid G, Node* __restrict__ bg, NodeDF* __restrict__ bgdf,
                                                          Node32* __restrict__ bg32)
{
    const int64_t total = (int64_t)G.ncell;
    const DF idx{G.df_inv_dX.x, G.df_inv_dX.y}, idy{G.df_inv_dY.x, G.df_inv_dY.y}, idz{G.df_inv_dz.x, G.df_inv_dz.y};
    const DF sx = df_pow2(idx, 0.5f);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(c % G.nz);
        const int col = (int)(c / G.nz);
        const int i = col % G.nx, j = col / G.nx;
        const Node* e = bg + node_index(G, i + 1 == G.nx ? 0 : i + 1, j, k);
        const Node* w = bg + node_index(G, i == 0 ? G.nx - 1 : i - 1, j, k);
        const Node *nn, *ss;
        DF sy;
        if (G.geometry == 0) {
            nn = bg + node_index(G, i, j + 1 == G.ny ? 0 : j + 1, k);
            ss = bg + node_index(G, i, j == 0 ? G.ny - 1 : j - 1, k);
            sy = df_pow2(idy, 0.5f);
        } else if (j == 0) {
            nn = bg + node_index(G, i, 1, k);
            ss = bg + node_index(G, i, 0, k);
            sy = idy;
        } else if (j == G.ny - 1) {
            nn = bg + node_index(G, i, G.ny - 1, k);
            ss = bg + node_index(G, i, G.ny - 2, k);
            sy = idy;
        } else {
            nn = bg + node_index(G, i, j + 1, k);
            ss = bg + node_index(G, i, j - 1, k);
            sy = df_pow2(idy, 0.5f);
        }
        const Node *up, *dn;
        DF sz;
        if (k == 0) {
            up = bg + c + 1; dn = bg + c; sz = idz;
        } else if (k == G.nz - 1) {
            up = bg + c; dn = bg + c - 1; sz = idz;
        } else {
            up = bg + c + 1; dn = bg + c - 1; sz = df_pow2(idz, 0.5f);
        }
        auto vals = [](const Node* p) { return *reinterpret_cast<const double4*>(p->v); };
        const double4 ve = vals(e), vw = vals(w), vn = vals(nn), vs = vals(ss), vu = vals(up), vd = vals(dn),
                      vc = vals(bg + c);
        // differences in FP64 (one rounding), scaled in double-float by the spacing reciprocals
        const double dx[4] = {ve.x - vw.x, ve.y - vw.y, ve.z - vw.z, ve.w - vw.w};
        const double dy[4] = {vn.x - vs.x, vn.y - vs.y, vn.z - vs.z, vn.w - vs.w};
        const double dz[4] = {vu.x - vd.x, vu.y - vd.y, vu.z - vd.z, vu.w - vd.w};
        const double val[4] = {vc.x, vc.y, vc.z, vc.w};
        DF q[16];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            q[f] = df_split(val[f]);
            q[4 + 3 * f] = df_mul2(df_split(dx[f]), sx);
            q[5 + 3 * f] = df_mul2(df_split(dy[f]), sy);
            q[6 + 3 * f] = df_mul2(df_split(dz[f]), sz);
        }
        if (bgdf) {
            NodeDF o;
#pragma unroll
            for (int el = 0; el < 8; ++el) o.q[el] = make_float4(q[2 * el].hi, q[2 * el].lo, q[2 * el + 1].hi, q[2 * el + 1].lo);
            bgdf[c] = o;
        }
        if (bg32) {
            // the FP32 node: each quantity rounded once to nearest (hi + lo rounded as a pair)
            Node32 o;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                o.v[f] = narrow(val[f]);
#pragma unroll
                for (int d = 0; d < 3; ++d) o.d[f][d] = __fadd_rn(q[4 + 3 * f + d].hi, q[4 + 3 * f + d].lo);
            }
            bg32[c] = o;
        }
    }
}

void configure_launch_kernels()
{
    cudaFuncSetAttribute(k_set_background, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_set_background(Context& c, int member, const double* u, const double* v, const double* n2,
                           const double* rho)
{
    const int TW = kBgTile;
    const int ntx = (c.G.nx + TW - 1) / TW;
    const size_t shm = sizeof(double) * 4 * (size_t)c.G.nz * TW;
    const int64_t o = (int64_t)member * c.G.ncell;
    k_set_background<<<ntx * c.G.ny, kThreads, shm, c.stream>>>(c.G, c.P.gamma_mode, u, v, n2, rho, c.bg + o,
                                                                c.rho + o, c.rho_inv + o, c.flag_dev);
    const int blocks = (int)std::min<int64_t>((c.G.ncell + kThreads - 1) / kThreads, 16384);
    k_node_gradients<<<blocks, kThreads, 0, c.stream>>>(c.G, c.bg + o, c.bgdf ? c.bgdf + o : nullptr,
                                                        c.f32 ? c.bg32 + o : nullptr);
}

// double-float nodes of a precision-form context (its ghost-layer launch integrates the ghost in the
// FP64 form's double-float RK3): from the FP64 node values already set
void node_gradients_df(Context& c, int member)
{
    const int64_t o = (int64_t)member * c.G.ncell;
    const int blocks = (int)std::min<int64_t>((c.G.ncell + kThreads - 1) / kThreads, 16384);
    k_node_gradients<<<blocks, kThreads, 0, c.stream>>>(c.G, c.bg + o, c.bgdf + o, nullptr);
}

// asynchronous background: an invalid value becomes the sticky context status (GWAM_ENUMERIC),
// reported by the next synchronising call; the steps in between do nothing
__global__ void k_flag_to_status(const int* flag, Ctl* ctl)
{
    if (*flag) set_status(ctl, GWAM_ENUMERIC);
}

void launch_flag_to_status(Context& c) { k_flag_to_status<<<1, 1, 0, c.stream>>>(c.flag_dev, c.ctl); }

// 1/rho of restored nodes (checkpoint load), by the Newton reciprocal as in k_set_background
__global__ void k_rho_inv(const double* __restrict__ rho, double* __restrict__ rho_inv, int64_t n)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double r = rho[c];
        rho_inv[c] = (__double_as_longlong(r) > 0 && !nonfinite_bits(r)) ? rcp_nr(r) : 0.0;
    }
}

void restore_background(Context& c, int member)
{
    const int64_t o = (int64_t)member * c.G.ncell;
    const int blocks = (int)std::min<int64_t>((c.G.ncell + kThreads - 1) / kThreads, 16384);
    k_rho_inv<<<blocks, kThreads, 0, c.stream>>>(c.rho + o, c.rho_inv + o, c.G.ncell);
    k_node_gradients<<<blocks, kThreads, 0, c.stream>>>(c.G, c.bg + o, c.bgdf ? c.bgdf + o : nullptr,
                                                        c.f32 ? c.bg32 + o : nullptr);
}

// caller [members][nz][ny][nx] -> column-major reference potential temperature; flags values that
// are not positive and finite
__global__ void k_set_theta(Grid G, const double* __restrict__ theta, double* __restrict__ out, int* flags)
{
    const int64_t total = (int64_t)G.ncell_all;
    int bad = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mem = t / G.ncell, r = t - mem * G.ncell;
        const int i = (int)(r % G.nx), j = (int)((r / G.nx) % G.ny), k = (int)(r / G.ncol);
        const double v = theta[t];
        if (!(v > 0.0) || nonfinite_bits(v)) bad = 1;
        out[mem * G.ncell + node_index(G, i, j, k)] = v;
    }
    if (bad) atomicOr(flags, BG_NONFINITE);
}

void launch_set_theta(Context& c, const double* theta)
{
    const int blocks = (int)std::min<int64_t>((c.G.ncell_all + kThreads - 1) / kThreads, 16384);
    k_set_theta<<<blocks, kThreads, 0, c.stream>>>(c.G, theta, c.theta, c.flag_dev);
}

// Eq. mean-flow-impact-t: d theta/dt = -div <u'theta'>, <u'theta'> = theta-bar / (g rho-bar) T per cell
// from the (smoothed) integrals T_l, T_p; horizontal centred differences as in the momentum
// divergence (flux zero beyond the pole rows), zero in the columnar mode.  Output in the caller's
// [members][nz][ny][nx].  FP64: an on-demand diagnostic, not a per-step kernel.
__global__ void k_theta_div(Grid G, const double* __restrict__ tl, const double* __restrict__ tp,
                            const double* __restrict__ theta, const double* __restrict__ rho_inv,
                            double* __restrict__ out)
{
    const int64_t total = (int64_t)G.ncell_all;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mem = t / G.ncell, r = t - mem * G.ncell;
        const int i = (int)(r % G.nx), j = (int)((r / G.nx) % G.ny), k = (int)(r / G.ncol);
        if (G.columnar) {
            out[t] = 0.0;
            continue;
        }
        const int64_t o = mem * G.ncell;
        auto thf = [&](const double* a, int ii, int jj) {
            const int64_t c = o + node_index(G, ii, jj, k);
            return a[c] * theta[c] * rho_inv[c] * G.inv_g;
        };
        const int ie = i + 1 == G.nx ? 0 : i + 1, iw = i == 0 ? G.nx - 1 : i - 1;
        double div;
        if (G.geometry == 1) {
            const double yn = j + 1 < G.ny ? G.row_cos[j + 1] * thf(tp, i, j + 1) : 0.0;
            const double ys = j - 1 >= 0 ? G.row_cos[j - 1] * thf(tp, i, j - 1) : 0.0;
            const double dl = (thf(tl, ie, j) - thf(tl, iw, j)) * (0.5 * G.inv_dX);
            const double dp = (yn - ys) * (0.5 * G.inv_dY);
            div = (dl + dp) * G.row_inv_cos[j] * G.lev_inv_r[k];
        } else {
            const int jn = j + 1 == G.ny ? 0 : j + 1, js = j == 0 ? G.ny - 1 : j - 1;
            div = (thf(tl, ie, j) - thf(tl, iw, j)) * (0.5 * G.inv_dX) + (thf(tp, i, jn) - thf(tp, i, js)) * (0.5 * G.inv_dY);
        }
        out[t] = -div;
    }
}

void launch_theta_div(Context& c, const double* tl, const double* tp, double* out)
{
    const int blocks = (int)std::min<int64_t>((c.G.ncell_all + kThreads - 1) / kThreads, 16384);
    k_theta_div<<<blocks, kThreads, 0, c.stream>>>(c.G, tl, tp, c.theta, c.rho_inv, out);
}

// ----------------------------------------------------------------------------- explicit rays

// pass 0 validates, pass 1 writes at n + q with id next_id + q
struct RayInputPtrs {
    const double* p[13];
};

__global__ void k_add_rays(Grid G, RaySoA A, Ray32SoA A32, bool f32, Ctl* ctl, int64_t max_rays, RayInputPtrs in,
                           int n_add, int pass, int* flags, double* partials, int pstride)
{
    const int n0 = ctl->n;
    const long long next = ctl->next_id;
    double w = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_add; q += gridDim.x * blockDim.x) {
        double s[NSTATE];
        s[SX] = in.p[0][q]; s[SY] = in.p[1][q]; s[SZ] = in.p[2][q];
        s[SK] = in.p[3][q]; s[SL] = in.p[4][q]; s[SM] = in.p[5][q];
        s[SEX] = in.p[6][q]; s[SEY] = in.p[7][q]; s[SEZ] = in.p[8][q];
        Geo g;
        geometry_at(G, s[SY], s[SZ], g);
        s[SPX] = g.hX * s[SEX] * in.p[9][q];
        s[SPY] = g.hY * s[SEY] * in.p[10][q];
        s[SPZ] = s[SEZ] * in.p[11][q];
        s[SN] = in.p[12][q];
        wrap_position(G, s);
        if (ray_status(G, s) != 0) {
            atomicOr(flags, 1);
            continue;
        }
        if (pass == 1) {
            const int64_t pos = (int64_t)n0 + q;
            if (pos >= max_rays) {
                set_status(ctl, GWAM_ECAPACITY);
                continue;
            }
            if (f32) {
                S32 r;
                from_double(G, s, next + q, r);
                store32(G, A32, pos, r);
                w += (double)action32(r);
            } else {
                store_ray(A, pos, s, next + q);
                w += ray_action(s);
            }
        }
    }
    const double wb = block_sum(w);
    if (threadIdx.x == 0 && pass == 1) partials[T_LAUNCH * pstride + blockIdx.x] = wb;
}

__global__ void k_append_close(Ctl* ctl, int64_t max_rays, int added)
{
    int n = ctl->n + added;
    if ((int64_t)n > max_rays) n = (int)max_rays;
    ctl->n = n;
    ctl->next_id += added;
    ctl->n_launched += added;
}

void launch_add_rays(Context& c, const double* const in[13], int64_t n)
{
    RayInputPtrs d_in;
    for (int q = 0; q < 13; ++q) d_in.p[q] = in[q];
    cudaMemsetAsync(c.flag_dev, 0, sizeof(int), c.stream);
    k_add_rays<<<c.grid_blocks, kThreads, 0, c.stream>>>(c.G, c.A, c.A32, c.f32, c.ctl, c.max_rays, d_in, (int)n, 0,
                                                         c.flag_dev, c.partials, c.max_blocks);
    cudaMemcpyAsync(c.flag_host, c.flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    cudaStreamSynchronize(c.stream);
    if (*c.flag_host) {
        c.err = "gwam_add_rays: a ray volume lies outside the domain or is invalid";
        throw (int)GWAM_EINVAL;
    }
    cudaMemsetAsync(c.partials, 0, sizeof(double) * NTALLY * (size_t)c.max_blocks, c.stream);
    k_add_rays<<<c.grid_blocks, kThreads, 0, c.stream>>>(c.G, c.A, c.A32, c.f32, c.ctl, c.max_rays, d_in, (int)n, 1,
                                                         c.flag_dev, c.partials, c.max_blocks);
    finalize_tallies(c, 1 << T_LAUNCH, 0);
    k_append_close<<<1, 1, 0, c.stream>>>(c.ctl, c.max_rays, (int)n);
}

// ----------------------------------------------------------------------------- sources (Sec. 3c)

// latitudinal profile alpha(phi), phi in degrees north
__device__ __forceinline__ double alpha_profile(double p)
{
    if (p >= 80.0) return fmin(1.0, fmax(0.0, 1.0 - (p - 80.0) / 5.0));
    if (p >= 50.0) return 1.0;
    if (p >= 20.0) return 0.5 * (1.0 - cos(kPi * (p - 20.0) / 30.0));
    return 0.0;
}

__device__ __forceinline__ double f_am(double p, double tau, double fs, double fw)
{
    const double sol_p = alpha_profile(p) * fs + alpha_profile(-p) * fw;
    const double sol_m = alpha_profile(-p) * fs + alpha_profile(p) * fw;
    const double ct = cos(tau);
    return 0.5 * (sol_p * (1.0 + ct) + sol_m * (1.0 - ct));
}

struct Bin {
    int i, j, member;
    double z_launch, dz_launch, theta, c, lambda_h, flux, frac;
};

// 0 = filtered, 1 = launched (state in s)
__device__ __forceinline__ int make_launch(const Grid& G, const Node* __restrict__ bg_all, const Bin& b,
                                           double s[NSTATE])
{
    const Node* bg = bg_all + (int64_t)b.member * G.ncell;
    const double X = __dmul_rn(b.i + 0.5, G.dX);
    const double Y = row_lat(G, b.j);
    const double Z = b.z_launch + 0.5 * b.dz_launch;
    Bg bk;
    gather_values_fp64(G, bg, X, Y, Z, bk.v);
    Geo g;
    geometry_at(G, Y, Z, g);
    double f2, df2;
    coriolis(G, g.sphi, g.cphi, f2, df2);
    const double U = bk.v[0], V = bk.v[1], N2 = bk.v[2], G2 = bk.v[3];
    const double kh = 2.0 * kPi / b.lambda_h;
    double st, ct;
    sincos(b.theta, &st, &ct);
    const double k = kh * ct, l = kh * st;
    const double w = kh * b.c - (k * U + l * V);
    if (!(w > 0.0 && w * w > f2 && w * w < N2)) return 0;
    const double m2 = kh * kh * (N2 - w * w) / (w * w - f2) - G2;
    if (!(m2 > 0.0)) return 0;
    const double m = -sqrt(m2);
    Disp d;
    dispersion(kh * kh, m2 + G2, N2, f2, d);
    const double chr = -m * kh * kh * d.c;
    const double A = b.flux / (kh * chr);   // once per launched ray: IEEE division is fine here
    const double dk = b.frac * kh, dl = b.frac * kh, dm = b.frac * fabs(m);
    s[SX] = X; s[SY] = Y; s[SZ] = Z;
    s[SK] = k; s[SL] = l; s[SM] = m;
    s[SEX] = G.dX; s[SEY] = G.dY; s[SEZ] = b.dz_launch;
    s[SPX] = g.hX * G.dX * dk;
    s[SPY] = g.hY * G.dY * dl;
    s[SPZ] = b.dz_launch * dm;
    s[SN] = A / (dk * dl * dm);
    return ray_status(G, s) == 0 ? 1 : 0;
}

__device__ __forceinline__ bool source_bin(const Grid& G, const gwam_bg_source& src, int t, Bin& b)
{
    const int nbins = src.n_az * src.n_c;
    const int gcol = t / nbins, bin = t % nbins;
    b.member = gcol / G.ncol;
    const int col = gcol - b.member * G.ncol;
    b.j = col / G.nx;
    b.i = col % G.nx;
    const double pdeg = row_lat(G, b.j) * (180.0 / kPi);
    if (fabs(pdeg) > src.phi_max_deg) return false;
    const double fbin = f_am(pdeg, src.tau, src.f_s, src.f_w) / nbins;
    if (fbin == 0.0 && !src.launch_zero_flux) return false;
    const int a = bin / src.n_c, q = bin % src.n_c;
    b.theta = 2.0 * kPi * a / src.n_az;
    b.c = src.n_c == 1 ? src.c_min : src.c_min * pow(src.c_max / src.c_min, (double)q / (src.n_c - 1));
    b.z_launch = src.z_launch;
    b.dz_launch = src.dz_launch;
    b.lambda_h = src.lambda_h;
    b.flux = fbin;
    b.frac = src.spectral_frac;
    return true;
}

__device__ __forceinline__ bool spec_bin(const Grid& G, Ctl* ctl, const gwam_spec& sp, Bin& b)
{
    // device-resident specs are not seen by the host: a column or member outside the grid is an
    // input error (status GWAM_EINVAL, read at the next synchronising call), never an index
    if (sp.i < 0 || sp.i >= G.nx || sp.j < 0 || sp.j >= G.ny || sp.member < 0 || sp.member >= G.members) {
        set_status(ctl, GWAM_EINVAL);
        return false;
    }
    b.i = sp.i; b.j = sp.j; b.member = sp.member;
    b.z_launch = sp.z_launch; b.dz_launch = sp.dz_launch; b.theta = sp.theta; b.c = sp.c;
    b.lambda_h = sp.lambda_h; b.flux = sp.flux; b.frac = sp.spectral_frac;
    return true;
}

// Ghost-layer emission (Sec. 3c): the launch state s fills the layer [z_launch, z_launch + dz_launch]
// and propagates vertically only over the launch interval dt (single-column RK3: G.columnar is set
// on the grid this kernel is given).  Returns 1 with s = the part above the layer top (vertical
// extent from the layer top, or the ghost's own bottom if it left whole, to its top; P_z in
// proportion; the ghost's m), 0 when the ghost was reflected in the layer (m no longer negative) or
// the part lies outside the domain, 2 when nothing has left the layer.
__device__ __forceinline__ int ghost_emit(const Grid& G, const NodeDF* __restrict__ bgdf, const Bin& b, double dt,
                                          double s[NSTATE], double* sh)
{
    double y[NSTATE];
#pragma unroll
    for (int c = 0; c < NSTATE; ++c) y[c] = s[c];
    rk3(G, bgdf + (int64_t)b.member * G.ncell, y, dt, sh);
    if (!(y[SM] < 0.0)) return 0;
    const double layer_top = b.z_launch + b.dz_launch;
    const double top = y[SZ] + 0.5 * y[SEZ], bot = y[SZ] - 0.5 * y[SEZ];
    if (!(top > layer_top)) return 2;
    const double lo = bot > layer_top ? bot : layer_top;
    s[SM] = y[SM];
    s[SZ] = 0.5 * (lo + top);
    s[SEZ] = top - lo;
    s[SPZ] = s[SPZ] * s[SEZ] / y[SEZ];   // once per emitted ray: IEEE division is fine here
    return ray_status(G, s) == 0 ? 1 : 0;
}

// pass 0: flag[t] = launches?, count filtered bins; pass 1: write launched rays in order.
// kGhost: emit what left the ghost layer over ghost_dt instead of the launch state itself.
template <bool kSpec, bool kGhost>
__global__ void k_launch(Grid G, const Node* __restrict__ bg, const NodeDF* __restrict__ bgdf, RaySoA A,
                         Ray32SoA A32, bool f32, Ctl* ctl, int64_t max_rays,
                         gwam_bg_source src, const gwam_spec* __restrict__ specs, int total, double ghost_dt,
                         int pass, int* __restrict__ flag, double* __restrict__ partials, int pstride)
{
    __shared__ double sh_state[kGhost ? 18 * kThreads : 1];
    const int n0 = ctl->n;
    const long long next = ctl->next_id;
    double w = 0.0;
    long long filtered = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        Bin b;
        bool eligible = kSpec ? spec_bin(G, ctl, specs[t], b) : source_bin(G, src, t, b);
        double s[NSTATE];
        int ok = 0;
        if (eligible) {
            ok = make_launch(G, bg, b, s);
            if (kGhost && ok) {
                const int e = ghost_emit(G, bgdf, b, ghost_dt, s, sh_state + threadIdx.x);
                ok = e == 1;
                if (e == 2) eligible = false;      // nothing left the layer: neither launched nor filtered
            }
            if (eligible && !ok) ++filtered;
        }
        if (pass == 0) {
            flag[t] = ok;
        } else if (ok) {
            const int64_t pos = (int64_t)n0 + flag[t];
            if (pos >= max_rays) {
                set_status(ctl, GWAM_ECAPACITY);
                continue;
            }
            const long long id = with_member(b.member, next + flag[t]);
            if (f32) {
                S32 r;
                from_double(G, s, id, r);
                store32(G, A32, pos, r);
                w += (double)action32(r);
            } else {
                store_ray(A, pos, s, id);
                w += ray_action(s);
            }
        }
    }
    const double wb = block_sum(w);
    const long long fb = block_sum(filtered);
    if (threadIdx.x == 0) {
        if (pass == 1) partials[T_LAUNCH * pstride + blockIdx.x] = wb;
        if (pass == 0 && fb) atomicAdd((unsigned long long*)&ctl->n_filtered, (unsigned long long)fb);
    }
}

__global__ void k_launch_close(Ctl* ctl, int64_t max_rays, const int* off, int total)
{
    const int added = off[total];
    int n = ctl->n + added;
    if ((int64_t)n > max_rays) n = (int)max_rays;
    ctl->n = n;
    ctl->next_id += added;
    ctl->n_launched += added;
}

static int* launch_scratch(Context& c, int64_t need)
{
    if (need + 1 > c.max_rays + 1) {
        // the per-ray scratch `newid` holds max_rays + 1 ints; larger launches need their own
        int* p = nullptr;
        if (cudaMallocAsync((void**)&p, sizeof(int) * (size_t)(need + 1), c.stream) != cudaSuccess) {
            c.err = "launch: scratch allocation failed";
            throw (int)GWAM_ENOMEM;
        }
        return p;
    }
    return c.newid;
}

static void launch_pass(Context& c, const Grid& G, const gwam_bg_source& s0, const gwam_spec* specs, int total,
                        double ghost_dt, int pass, int* flag)
{
    const int nb = c.grid_blocks;
    const bool ghost = ghost_dt > 0.0;
    if (specs && ghost)
        k_launch<true, true><<<nb, kThreads, 0, c.stream>>>(G, c.bg, c.bgdf, c.A, c.A32, c.f32, c.ctl, c.max_rays, s0,
                                                            specs, total, ghost_dt, pass, flag, c.partials,
                                                            c.max_blocks);
    else if (specs)
        k_launch<true, false><<<nb, kThreads, 0, c.stream>>>(G, c.bg, c.bgdf, c.A, c.A32, c.f32, c.ctl, c.max_rays, s0,
                                                             specs, total, ghost_dt, pass, flag, c.partials,
                                                             c.max_blocks);
    else if (ghost)
        k_launch<false, true><<<nb, kThreads, 0, c.stream>>>(G, c.bg, c.bgdf, c.A, c.A32, c.f32, c.ctl, c.max_rays, s0,
                                                             specs, total, ghost_dt, pass, flag, c.partials,
                                                             c.max_blocks);
    else
        k_launch<false, false><<<nb, kThreads, 0, c.stream>>>(G, c.bg, c.bgdf, c.A, c.A32, c.f32, c.ctl, c.max_rays, s0,
                                                              specs, total, ghost_dt, pass, flag, c.partials,
                                                              c.max_blocks);
}

static void launch_common(Context& c, const gwam_bg_source* src, const gwam_spec* specs, int64_t total,
                          double ghost_dt = 0.0)
{
    if (total <= 0) return;
    int* flag = launch_scratch(c, total);
    gwam_bg_source s0{};
    if (src) s0 = *src;
    // the ghost layer propagates vertically only: the single-column equations on this grid copy
    Grid G = c.G;
    if (ghost_dt > 0.0) G.columnar = 1;
    launch_pass(c, G, s0, specs, (int)total, ghost_dt, 0, flag);
    exclusive_scan(c, flag, flag, total, nullptr);
    cudaMemsetAsync(c.partials, 0, sizeof(double) * NTALLY * (size_t)c.max_blocks, c.stream);
    launch_pass(c, G, s0, specs, (int)total, ghost_dt, 1, flag);
    finalize_tallies(c, 1 << T_LAUNCH, 0);
    k_launch_close<<<1, 1, 0, c.stream>>>(c.ctl, c.max_rays, flag, (int)total);
    if (flag != c.newid) cudaFreeAsync(flag, c.stream);
}

void launch_background_source(Context& c, const gwam_bg_source& src)
{
    const int64_t total = (int64_t)c.G.ncol_all * src.n_az * src.n_c;
    launch_common(c, &src, nullptr, total);
}

void launch_spectral(Context& c, const gwam_spec* specs, int64_t n) { launch_common(c, nullptr, specs, n); }

void launch_ghost_source(Context& c, const gwam_bg_source& src, double dt)
{
    const int64_t total = (int64_t)c.G.ncol_all * src.n_az * src.n_c;
    launch_common(c, &src, nullptr, total, dt);
}

void launch_ghost_spectral(Context& c, const gwam_spec* specs, int64_t n, double dt)
{
    launch_common(c, nullptr, specs, n, dt);
}

}  // namespace gwam
