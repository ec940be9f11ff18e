// gwam_fp32.cu -- kernels and step of the precision form (FP32 kinematics, FP64 accumulation).
// The re-binning (scans, cap bookkeeping, segment sort), smoothing and divergence are shared
// with the FP64 form; only the kernels that touch ray state are specialised here.
#include <algorithm>

#include "gwam_common.cuh"
#include "gwam_fp32.cuh"

namespace gwam {

// FP64 -> FP32, round to nearest, for up to NFIELD arrays in one launch (blockIdx.y = array)
struct NarrowSet {
    const double* in[NFIELD];
    float* out[NFIELD];
    int64_t n[NFIELD];
};

__global__ void k_narrow(NarrowSet s)
{
    const int f = blockIdx.y;
    const int64_t n = s.n[f];
    const double* __restrict__ in = s.in[f];
    float* __restrict__ out = s.out[f];
    // four elements per thread and pass, all loads issued first (bytes in flight)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const double a = in[i], b = in[i + stride], c = in[i + 2 * stride], d = in[i + 3 * stride];
        out[i] = narrow(a);
        out[i + stride] = narrow(b);
        out[i + 2 * stride] = narrow(c);
        out[i + 3 * stride] = narrow(d);
    }
    for (; i < n; i += stride) out[i] = narrow(in[i]);
}

// the FP32 nodes themselves are written by the node-gradient pass; here 1/rho is narrowed
void convert_background32(Context& c, int member)
{
    const int64_t o = (int64_t)member * c.G.ncell;
    const int blocks = (int)std::min<int64_t>((c.G.ncell + kThreads - 1) / kThreads, 16384);
    NarrowSet ns{};
    ns.in[0] = c.rho_inv + o;
    ns.out[0] = c.rho_inv32 + o;
    ns.n[0] = c.G.ncell;
    k_narrow<<<dim3((unsigned)blocks, 1), kThreads, 0, c.stream>>>(ns);
}

// ---------------------------------------------------------------------------- FP32 grid phase
// The precision form keeps the projection sums (and the saturation sums and the budget) in FP64;
// smoothing and divergence run in FP32: GB300's FP64 rate is 1/64 of its FP32 rate, and these
// stencils would otherwise be bound by it.  The smoothing reads the projected FP64 fields and
// narrows them as it loads (no FP32 copy of the raw fields is written and read back); without
// smoothing the fields are narrowed once by k_narrow.  du/dt, dv/dt are widened to the caller's
// FP64 on the way out.

struct FieldSet32 {
    const double* in[NFIELD];
    float* out[NFIELD];
};

// separable 1-2-1 x 1-2-1 smoothing (periodic in lambda, edge row reused at the poles).  A warp
// owns 32 consecutive levels of kRows32 rows over a run of kSpan columns and slides a 3 x 3 window
// along the rows: each new column costs kRows32 + 2 loads (the rows and their two neighbours) for
// kRows32 outputs, and the column sums of the previous two columns stay in registers.  All loads of
// a pass (two columns) are issued before any of them is converted.  Three rows over spans of 32
// columns, reading the FP64 fields: 5/3 loads per output, measured faster than two, four or six
// rows or spans of 16 (more rows hold more registers).  Warp item = (field, member, row group,
// level group, span).
constexpr int kSpan = 32;
constexpr int kRows32 = 3;
__global__ void __launch_bounds__(256) k_smooth_fields32(Grid G, FieldSet32 fs, int f0, int nf)
{
    const int lane = threadIdx.x & 31;
    const int nlg = (G.nz + 1 + 31) / 32;                   // level groups (interface fields have nz + 1)
    const int nsp = (G.nx + kSpan - 1) / kSpan;
    const int nrg = (G.ny + kRows32 - 1) / kRows32;
    const long long per_field = (long long)G.members * nrg * nlg * nsp;
    const long long items = per_field * nf;
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= items) return;
    const int f = f0 + (int)(w / per_field);
    long long r = w % per_field;
    const int sp = (int)(r % nsp);
    r /= nsp;
    const int lg = (int)(r % nlg);
    r /= nlg;
    const int rg = (int)(r % nrg);
    const int mem = (int)(r / nrg);
    const int nlev = f <= F_ZP ? G.nz + 1 : G.nz;
    const int lev = lg * 32 + lane;
    if (lg * 32 >= nlev) return;
    const bool live = lev < nlev;
    const int j0 = rg * kRows32;
    const int nrow = min(kRows32, G.ny - j0);
    const int64_t base = (int64_t)mem * G.ncol;
    const double* __restrict__ F = fs.in[f];
    // source rows j0 - 1 .. j0 + kRows32 (clamped at the poles, wrapped on the f-plane)
    const double* src[kRows32 + 2];
#pragma unroll
    for (int q = 0; q < kRows32 + 2; ++q) {
        int jj = j0 - 1 + q;
        if (G.geometry == 1) jj = jj < 0 ? 0 : (jj >= G.ny ? G.ny - 1 : jj);
        else jj = jj < 0 ? jj + G.ny : (jj >= G.ny ? jj - G.ny : jj);
        src[q] = F + (base + (int64_t)jj * G.nx) * nlev + lev;
    }
    float* O = fs.out[f] + (base + (int64_t)j0 * G.nx) * nlev + lev;
    const int64_t orow = (int64_t)G.nx * nlev;
    // vertical 1-2-1 column sums of the kRows32 rows at column i
    auto loadcol = [&](int i, double (&raw)[kRows32 + 2]) {
        const int64_t o = (int64_t)i * nlev;
#pragma unroll
        for (int q = 0; q < kRows32 + 2; ++q) raw[q] = live ? __ldg(src[q] + o) : 0.0;
    };
    auto sums = [&](const double (&raw)[kRows32 + 2], float (&cs)[kRows32]) {
        float v[kRows32 + 2];
#pragma unroll
        for (int q = 0; q < kRows32 + 2; ++q) v[q] = narrow(raw[q]);
#pragma unroll
        for (int q = 0; q < kRows32; ++q) cs[q] = v[q] + 2.0f * v[q + 1] + v[q + 2];
    };
    auto colsums = [&](int i, float (&cs)[kRows32]) {
        double raw[kRows32 + 2];
        loadcol(i, raw);
        sums(raw, cs);
    };
    const int i0 = sp * kSpan, i1 = min(G.nx, i0 + kSpan);
    float cm[kRows32], c0[kRows32], cp[kRows32], cq[kRows32];
    colsums(i0 == 0 ? G.nx - 1 : i0 - 1, cm);
    colsums(i0, c0);
    int i = i0;
    // two columns per pass with their loads issued together
    for (; i + 2 <= i1; i += 2) {
        {
            double ra[kRows32 + 2], rb[kRows32 + 2];
            loadcol(i + 1 == G.nx ? 0 : i + 1, ra);
            loadcol(i + 2 >= G.nx ? i + 2 - G.nx : i + 2, rb);
            sums(ra, cp);
            sums(rb, cq);
        }
        if (live) {
#pragma unroll
            for (int q = 0; q < kRows32; ++q) {
                if (q < nrow) {
                    O[q * orow + (int64_t)i * nlev] = (cm[q] + 2.0f * c0[q] + cp[q]) * 0.0625f;
                    O[q * orow + (int64_t)(i + 1) * nlev] = (c0[q] + 2.0f * cp[q] + cq[q]) * 0.0625f;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kRows32; ++q) {
            cm[q] = cp[q];
            c0[q] = cq[q];
        }
    }
    for (; i < i1; ++i) {
        colsums(i + 1 == G.nx ? 0 : i + 1, cp);
        if (live) {
#pragma unroll
            for (int q = 0; q < kRows32; ++q)
                if (q < nrow) O[q * orow + (int64_t)i * nlev] = (cm[q] + 2.0f * c0[q] + cp[q]) * 0.0625f;
        }
#pragma unroll
        for (int q = 0; q < kRows32; ++q) {
            cm[q] = c0[q];
            c0[q] = cp[q];
        }
    }
}

// divergence (Eq. mean-flow-impact) in FP32:
//   du/dt = -(1/rho) [ (1/(r cos phi)) (d_lambda F^{ll} + d_phi (cos phi F^{pl})) + d_z F^z_l ] + E_l / (g rho),
// dv/dt likewise (centred differences, flux zero beyond the pole rows; in the columnar mode the
// vertical term alone).  One block per (row, tile of TW columns), results transposed through shared
// memory into the caller's [nz][ny][nx] FP64 layout
__global__ void k_divergence32(Grid G, int TW, const float* __restrict__ fzl, const float* __restrict__ fzp,
                               const float* __restrict__ fll, const float* __restrict__ flp,
                               const float* __restrict__ fpl, const float* __restrict__ fpp,
                               const float* __restrict__ el, const float* __restrict__ ep,
                               const float* __restrict__ rho_inv, double* __restrict__ du, double* __restrict__ dv)
{
    extern __shared__ float tile32[];
    float* tu = tile32;
    float* tv = tile32 + (size_t)TW * G.nz;
    float* lev32 = tile32 + 2 * (size_t)TW * G.nz;   // 1 / (a + z_k) per level
    for (int k = threadIdx.x; k < G.nz; k += blockDim.x) lev32[k] = (float)G.lev_inv_r[k];
    __syncthreads();
    const int ntx = (G.nx + TW - 1) / TW;
    const int mem = blockIdx.x / (ntx * G.ny);
    const int bl = blockIdx.x - mem * ntx * G.ny;
    const int j = bl / ntx;
    const int i0 = (bl % ntx) * TW;
    {
        const int64_t oc = (int64_t)mem * G.ncell, oz = (int64_t)mem * G.ncol * (G.nz + 1);
        fzl += oz; fzp += oz;
        fll += oc; flp += oc; fpl += oc; fpp += oc; el += oc; ep += oc; rho_inv += oc;
        if (du) du += oc;
        if (dv) dv += oc;
    }
    const int nz = G.nz;
    const int n = TW * nz;
    const float h2x = (float)(0.5 * G.inv_dX), h2y = (float)(0.5 * G.inv_dY), idz = (float)G.inv_dz,
                ig = (float)G.inv_g;
    float rcp_cos = 1.0f, cn = 0.0f, cs = 0.0f;
    if (G.geometry == 1) {
        rcp_cos = (float)G.row_inv_cos[j];
        if (j + 1 < G.ny) cn = (float)G.row_cos[j + 1];
        if (j - 1 >= 0) cs = (float)G.row_cos[j - 1];
    }
    const int jn = G.geometry == 1 ? j + 1 : wrap_int(j + 1, G.ny);
    const int js = G.geometry == 1 ? j - 1 : wrap_int(j - 1, G.ny);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int k = t % nz, ii = t / nz;
        const int i = i0 + ii;
        if (i >= G.nx) continue;
        const int ie = i + 1 == G.nx ? 0 : i + 1, iw = i == 0 ? G.nx - 1 : i - 1;
        const int64_t c = ((int64_t)j * G.nx + i) * nz + k;
        const int64_t ce = ((int64_t)j * G.nx + ie) * nz + k;
        const int64_t cw = ((int64_t)j * G.nx + iw) * nz + k;
        const int64_t zc = ((int64_t)j * G.nx + i) * (nz + 1) + k;
        float pl_n = 0.0f, pl_s = 0.0f, pp_n = 0.0f, pp_s = 0.0f;
        if (jn >= 0 && jn < G.ny) {
            const int64_t cc = ((int64_t)jn * G.nx + i) * nz + k;
            pl_n = fpl[cc];
            pp_n = fpp[cc];
        }
        if (js >= 0 && js < G.ny) {
            const int64_t cc = ((int64_t)js * G.nx + i) * nz + k;
            pl_s = fpl[cc];
            pp_s = fpp[cc];
        }
        const float ri = rho_inv[c];
        float div_u, div_v;
        const float dzl = (fzl[zc + 1] - fzl[zc]) * idz;
        const float dzp = (fzp[zc + 1] - fzp[zc]) * idz;
        if (G.geometry == 1) {
            const float mh = rcp_cos * lev32[k];
            div_u = ((fll[ce] - fll[cw]) * h2x + (cn * pl_n - cs * pl_s) * h2y) * mh + dzl;
            div_v = ((flp[ce] - flp[cw]) * h2x + (cn * pp_n - cs * pp_s) * h2y) * mh + dzp;
        } else {
            div_u = (fll[ce] - fll[cw]) * h2x + (pl_n - pl_s) * h2y + dzl;
            div_v = (flp[ce] - flp[cw]) * h2x + (pp_n - pp_s) * h2y + dzp;
        }
        if (G.columnar) {
            // horizontally homogeneous column: the vertical flux divergence alone
            div_u = dzl;
            div_v = dzp;
        }
        tu[k * TW + ii] = (el[c] * ig - div_u) * ri;
        tv[k * TW + ii] = (ep[c] * ig - div_v) * ri;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int ii = t % TW, k = t / TW;
        const int i = i0 + ii;
        if (i >= G.nx) continue;
        const int64_t o = ((int64_t)k * G.ny + j) * G.nx + i;
        // widened by integer operations (the conversion instruction runs at the FP64 rate)
        if (du) du[o] = widen(tu[k * TW + ii]);
        if (dv) dv[o] = widen(tv[k * TW + ii]);
    }
}

__global__ void k_widen(const float* __restrict__ in, double* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = widen(in[i]);
}

// Saturation (Sec. 3c, Eq. turbulent-diffusivity) of the precision form: per carrier cell the
// sums P_c = sum P_j alpha_j and Q_c = sum P_j alpha_j K_j^2 in FP64 (segment head over the
// cell's run of the canonical array), the threshold difference P_c - rho/2 in FP64, then
// kappa = (P_c - rho/2) / (2 dt Q_c) in FP32 for every ray of the cell.
__device__ __forceinline__ void sat_run32(int p, int b, int c, const double* __restrict__ rho,
                                          const double* __restrict__ pj, const float* __restrict__ k2, float dt,
                                          float* __restrict__ kappa)
{
    double Pc = 0.0, Q = 0.0;
    for (int q = p; q < b; ++q) {
        const double v = pj[q];
        Pc += v;
        Q = fma(v, widen(k2[q]), Q);
    }
    const double d = fma(-0.5, rho[c], Pc);
    float kap = 0.0f;
    if (d > 0.0 && Q > 0.0) kap = __fdiv_rn(__double2float_rn(d), 2.0f * dt * __double2float_rn(Q));
    for (int q = p; q < b; ++q) kappa[q] = kap;
}

// the listed runs (k_sat_heads of the FP64 form lists them), one per lane
__global__ void k_sat_kappa32(const Ctl* ctl, const int* __restrict__ off2, const int* __restrict__ runlist,
                              const double* __restrict__ rho, const double* __restrict__ pj,
                              const float* __restrict__ k2, float dt, float* __restrict__ kappa)
{
    const int nl = ctl->status ? 0 : ctl->n_big;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += gridDim.x * blockDim.x) {
        const int c = runlist[t];
        sat_run32(off2[c], off2[c + 1], c, rho, pj, k2, dt, kappa);
    }
}

static void narrow_fields(Context& c, int f0, int f1)
{
    NarrowSet ns{};
    int64_t nmax = 0;
    for (int f = f0; f < f1; ++f) {
        ns.in[f - f0] = c.field[f];
        ns.out[f - f0] = c.nar32[f];
        ns.n[f - f0] = c.field_len(f);
        nmax = std::max(nmax, c.field_len(f));
    }
    const int blocks = (int)std::min<int64_t>((nmax + kThreads - 1) / kThreads, 2 * 152 * 8 / (f1 - f0) + 1);
    k_narrow<<<dim3((unsigned)blocks, (unsigned)(f1 - f0)), kThreads, 0, c.stream>>>(ns);
}

// the projected FP64 fields f0 .. f1-1, smoothed into their FP32 copies
static void smooth32(Context& c, int f0, int f1)
{
    FieldSet32 fs{};
    for (int f = 0; f < NFIELD; ++f) {
        fs.in[f] = c.field[f];
        fs.out[f] = c.sm32[f];
    }
    const long long warps = (long long)(f1 - f0) * c.G.members * ((c.G.ny + kRows32 - 1) / kRows32) *
                            ((c.G.nz + 1 + 31) / 32) * ((c.G.nx + kSpan - 1) / kSpan);
    k_smooth_fields32<<<(unsigned)((warps + 7) / 8), 256, 0, c.stream>>>(c.G, fs, f0, f1 - f0);
}

void smooth_field32(Context& c, int f)
{
    smooth32(c, f, f + 1);
    // widened into the FP64 smoothed copy the field readers use
    const int blocks = (int)std::min<int64_t>((c.field_len(f) + kThreads - 1) / kThreads, 8192);
    k_widen<<<blocks, kThreads, 0, c.stream>>>(c.sm32[f], c.smooth[f], c.field_len(f));
}

static void grid_phase32(Context& c, double* du, double* dv, int mask)
{
    const Grid& G = c.G;
    cudaStream_t s = c.stream;
    double* out_u = du ? du : c.dudt_buf;
    double* out_v = dv ? dv : c.dvdt_buf;
    float* const* fl = c.sm32;
    if (c.P.smoothing) {
        smooth32(c, 0, F_WAD);
    } else {
        narrow_fields(c, 0, F_WAD);
        fl = c.nar32;
    }
    const int TW = G.nz <= 96 ? 32 : 16;
    const size_t shm = sizeof(float) * (2 * (size_t)TW * G.nz + G.nz);
    if (shm > 48 * 1024) cudaFuncSetAttribute(k_divergence32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    const int ntx = (G.nx + TW - 1) / TW;
    k_divergence32<<<ntx * G.ny * G.members, kThreads, shm, s>>>(G, TW, fl[F_ZL], fl[F_ZP], fl[F_LL], fl[F_LP],
                                                                 fl[F_PL], fl[F_PP], fl[F_EL], fl[F_EP], c.rho_inv32,
                                                                 out_u, out_v);
    finalize_tallies(c, mask, 1);
}

// RK3 advance in FP32 (the ray-step kernel of the precision form): state read and written in
// place, exits, split decisions, child cells and slots as in k_advance.
__global__ void __launch_bounds__(kThreads) k_advance32(Grid G, Params P, Ray32SoA A, const Node32* __restrict__ bg,
                                                          Ctl* ctl, float dt, int* __restrict__ info,
                                                          int4* __restrict__ ccell, int4* __restrict__ cslot,
                                                          int* __restrict__ newid, int* __restrict__ cnt,
                                                          double* __restrict__ partials, int pstride, ClearSet zs)
{
    __shared__ __align__(128) float4 zbuf[kClearPiece / 16];
    const int n = ctl->n;
    ClearState cs;
    clear_start(zs, zbuf, n, cs);
    double w_exit = 0.0, w_inv = 0.0;
    long long n_exit = 0, n_inv = 0, n_sv = 0, n_sh = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (threadIdx.x == 0) clear_issue(zs, cs, cs.per);
        S32 s;
        load32(G, A, i, s);
        const int mem = member_of(s.id);
        rk3_32(G, bg + (int64_t)mem * G.ncell, s, dt);
        const int st = renormalize32(G, s);
        int code = 0, nch = 0;
        int cc[4] = {-1, -1, -1, -1}, sl[4] = {0, 0, 0, 0};
        if (st == 2) {
            ++n_inv;
            const double w = action32(s);
            if (isfinite(w)) w_inv += w;
        } else if (st == 1) {
            ++n_exit;
            w_exit += action32(s);
        } else {
            code = split_code32(G, P, s);
            nch = num_children(code);
            if (code & 1) ++n_sv;
            if (code & 2) n_sh += (code & 1) ? 2 : 1;
            // unrolled with a guard, not bounded by nch: cc and sl stay in registers
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c >= nch) break;
                S32 ch;
                if (make_child32(G, s, code, c, ch) != 0) {
                    ++n_exit;
                    w_exit += action32(ch);
                } else {
                    cc[c] = mem * G.ncell + cell32(G, ch);
                    sl[c] = atomicAdd(&cnt[cc[c]], 1);
                }
            }
            store32(G, A, i, s);
        }
        info[i] = code | (nch << 4) | (st << 8);
        ccell[i] = make_int4(cc[0], cc[1], cc[2], cc[3]);
        cslot[i] = make_int4(sl[0], sl[1], sl[2], sl[3]);
        newid[i] = nch > 0 ? nch - 1 : 0;
    }
    clear_finish(zs, cs);
    const double we = block_sum(w_exit);
    const double wi = block_sum(w_inv);
    const long long ne = block_sum(n_exit), ni = block_sum(n_inv), nv = block_sum(n_sv), nh = block_sum(n_sh);
    if (threadIdx.x == 0) {
        partials[T_EXIT * pstride + blockIdx.x] = we;
        partials[T_INVALID * pstride + blockIdx.x] = wi;
        if (ne) atomicAdd((unsigned long long*)&ctl->n_exited, (unsigned long long)ne);
        if (ni) atomicAdd((unsigned long long*)&ctl->n_invalid, (unsigned long long)ni);
        if (nv) atomicAdd((unsigned long long*)&ctl->n_split_v, (unsigned long long)nv);
        if (nh) atomicAdd((unsigned long long*)&ctl->n_split_h, (unsigned long long)nh);
    }
}

__device__ __forceinline__ long long id32(const Ray32SoA& A, int64_t i)
{
    const float4 d = A.q[3][i];
    return (long long)(((unsigned long long)(unsigned)__float_as_int(d.w) << 32) | (unsigned)__float_as_int(d.z));
}

__global__ void k_scatter32(Grid G, Ray32SoA A, Ctl* ctl, int64_t max_rays, const int* __restrict__ info,
                            const int4* __restrict__ ccell, const int4* __restrict__ cslot,
                            const int* __restrict__ newid, const int* __restrict__ off,
                            long long* __restrict__ ent_id, int* __restrict__ ent_src, int* __restrict__ ent_cell)
{
    const int n = ctl->n;
    const long long next = ctl->next_id;
    const int total = off[G.ncell_all];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->n_children = total;
        ctl->new_ids = newid[n];
        if ((int64_t)total > max_rays) set_status(ctl, GWAM_ECAPACITY);
    }
    if ((int64_t)total > max_rays) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int nch = (info[i] >> 4) & 7;
        if (!nch) continue;
        const int4 cc = ccell[i], sl = cslot[i];
        const int cs[4] = {cc.x, cc.y, cc.z, cc.w}, ss[4] = {sl.x, sl.y, sl.z, sl.w};
        const long long pid = id32(A, i);
        for (int c = 0; c < nch; ++c) {
            if (cs[c] < 0) continue;
            const int64_t pos = (int64_t)off[cs[c]] + ss[c];
            if (pos >= max_rays) continue;
            ent_id[pos] = c == 0 ? pid : with_member(member_of(pid), next + newid[i] + c - 1);
            ent_src[pos] = i * 4 + c;
            ent_cell[pos] = cs[c];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_cap_apply32(Grid G, Params P, Ray32SoA A,
                                                            const Node32* __restrict__ bg, Ctl* ctl,
                                                            const int* __restrict__ info, const int* __restrict__ off,
                                                            const int* __restrict__ overlist,
                                                            const long long* __restrict__ ent_id, int* ent_src,
                                                            double* ecap, int* cnt, double* __restrict__ partials,
                                                            int pstride)
{
    double w_cap = 0.0;
    long long n_cap = 0;
    const int nover = ctl->status ? 0 : ctl->n_over;
    for (int w = blockIdx.x; w < nover; w += gridDim.x) {
        const int col = overlist[w];
        const int a = off[col * G.nz], b = off[(col + 1) * G.nz];
        const int count = b - a;
        for (int e = a + threadIdx.x; e < b; e += blockDim.x) {
            const int src = ent_src[e];
            S32 s, ch;
            load32(G, A, src >> 2, s);
            make_child32(G, s, info[src >> 2] & 7, src & 3, ch);
            Intr32 in;
            intrinsic32(G, bg + (int64_t)member_of(s.id) * G.ncell, ch, in);
            ecap[e] = (double)in.w * action32(ch);
        }
        __syncthreads();
        for (int e = a + threadIdx.x; e < b; e += blockDim.x) {
            const double E = ecap[e];
            const long long id = ent_id[e];
            int rank = 0;
            for (int q = a; q < b; ++q) {
                const double Eq = ecap[q];
                rank += (Eq < E) || (Eq == E && ent_id[q] > id);
            }
            if (rank < count - P.cap) {
                const int src = ent_src[e];
                S32 s, ch;
                load32(G, A, src >> 2, s);
                make_child32(G, s, info[src >> 2] & 7, src & 3, ch);
                w_cap += action32(ch);
                ++n_cap;
                atomicSub(&cnt[member_of(s.id) * G.ncell + cell32(G, ch)], 1);
                ent_src[e] = -1 - src;
            }
        }
        __syncthreads();
    }
    const double wc = block_sum(w_cap);
    const long long nc = block_sum(n_cap);
    if (threadIdx.x == 0) {
        partials[T_CAP * pstride + blockIdx.x] = wc;
        if (nc) atomicAdd((unsigned long long*)&ctl->n_capped, (unsigned long long)nc);
    }
}

__global__ void __launch_bounds__(kThreads) k_materialize32(Grid G, Params P, Ray32SoA A, Ray32SoA B,
                                                              const Node32* __restrict__ bg, Ctl* ctl,
                                                              const int* __restrict__ off2,
                                                              const int* __restrict__ sorted_src,
                                                              const int* __restrict__ info,
                                                              const int* __restrict__ newid,
                                                              double* __restrict__ pj, float* __restrict__ k2,
                                                              int* __restrict__ raycell)
{
    if (ctl->status) return;
    const int n_new = off2[G.ncell_all];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->n_new = n_new;   // the live count k_finalize closes the step with
    const int n_old = ctl->n;
    const long long next = ctl->next_id;
    const int stride = gridDim.x * blockDim.x;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int src_next = p < n_new ? sorted_src[p] : 0;
    for (; p < n_new; p += stride) {
        const int src = src_next;
        // the next source index loaded a pass ahead (the parent's record load waits on it)
        if (p + stride < n_new) src_next = sorted_src[p + stride];
        const int i = src >> 2, c = src & 3;
        if (src < 0 || i >= n_old) {
            set_status(ctl, GWAM_ECUDA);
            continue;
        }
        S32 s, ch;
        load32(G, A, i, s);
        make_child32(G, s, info[i] & 7, c, ch);
        if (c != 0) ch.id = with_member(member_of(s.id), next + newid[i] + c - 1);
        store32(G, B, p, ch);
        raycell[p] = member_of(ch.id) * G.ncell + cell32(G, ch);
        if (P.saturation) {
            Intr32 in;
            intrinsic32(G, bg + (int64_t)member_of(ch.id) * G.ncell, ch, in);
            // P_j alpha_j = m^2 k_h^2 / (w K^2) N Px Py Pz / V_c in double-float, one FP64 add at the end
            const DF av = df_mul(action_df(ch), G.ivol32[ch.j * G.nz + ch.k]);
            pj[p] = df_to_double(df_mul(av, in.m2 * in.kh2 * in.iw * in.iK2));
            k2[p] = in.K2;
        }
    }
}

// Saturation N update and flux projection; per-ray terms in FP32, accumulated in FP64.
// THETA: also the potential-temperature flux integrals of Eq. fluxes:temperature (fields F_TL, F_TP)
template <bool THETA>
__global__ void __launch_bounds__(kThreads) k_project32(Grid G, Params P, Ray32SoA B, const Node32* __restrict__ bg,
                                                          const Ctl* ctl, const int* __restrict__ off2,
                                                          const float* __restrict__ kappa,
                                                          const float* __restrict__ k2, double dt,
                                                          double* __restrict__ fz_l, double* __restrict__ fz_p,
                                                          double* __restrict__ f_ll, double* __restrict__ f_lp,
                                                          double* __restrict__ f_pl, double* __restrict__ f_pp,
                                                          double* __restrict__ e_l, double* __restrict__ e_p,
                                                          double* __restrict__ wad, double* __restrict__ f_tl,
                                                          double* __restrict__ f_tp, double* __restrict__ partials,
                                                          int pstride)
{
    constexpr int NH = THETA ? 9 : 7;   // centre fields of the segmented sums
    // FP64 work is kept out of the per-ray path (GB300's FP64 rate is 1/72 of FP32): the action
    // and the budget terms in double-float, float -> double by integer widening, FP64 only in the
    // grid atomics (L2) and one addition per thread for the budget
    const int n = ctl->status ? 0 : off2[G.ncell_all];
    DF w_sat{0.0f, 0.0f}, w_tot{0.0f, 0.0f};
    const float dtf = (float)dt;
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x; p0 < n; p0 += stride) {
        const int p = p0 + threadIdx.x;
        const bool act = p < n;
        int key = -1;
        DF hv[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) hv[q] = {0.0f, 0.0f};
        float zl = 0.0f, zp = 0.0f, wh = 0.0f, lo = 0.0f, hi = 0.0f;
        int col = 0, kk0 = 1, nkk = 0;
        if (act) {
            S32 s;
            load32(G, B, p, s);
            if (P.saturation) {
                const float kap = kappa[p];
                if (kap > 0.0f) {
                    const float fac = fmaxf(0.0f, 1.0f - 2.0f * kap * k2[p] * dtf);
                    const float nold = s.n;
                    s.n = nold * fac;
                    w_sat = df_add(w_sat, df_mul(df_mul(df_mul(df_diff(nold, s.n), s.p[0]), s.p[1]), s.p[2]));
                    float4 q1 = B.q[1][p];
                    q1.w = s.n;
                    B.q[1][p] = q1;
                }
            }
            const DF Wd = action_df(s);
            w_tot = df_add(w_tot, Wd);
            const float W = __fadd_rn(Wd.hi, Wd.lo);
            const int mem = member_of(s.id);
            Intr32 in;
            intrinsic32(G, bg + (int64_t)mem * G.ncell, s, in);
            col = mem * G.ncol + s.j * G.nx + s.i;
            key = col * G.nz + s.k;
            const float Vj = in.g.hX * s.e[0] * (G.geometry == 1 ? in.g.r : 1.0f) * s.e[1] * s.e[2];
            const float A = W * __frcp_rn(Vj);
            const float aw = W * G.ivol32[s.j * G.nz + s.k];
            const float k = s.w[0], l = s.w[1], m = s.w[2];
            const float mg2c = in.mg2 * in.c;
            const float chx = k * mg2c, chy = l * mg2c, chr = -m * in.kh2 * in.c;
            float t_ll, t_lp, t_pl, t_pp, el, ep;
            if (P.flux_form == 0) {
                // 1/(w^2 - f^2) = K^2 / (D k_h^2): the algebraically equal form without the
                // cancellation that FP32 suffers for near-inertial waves
                const float iden = in.K2 * __frcp_rn(in.D * in.kh2);
                t_ll = (in.w2 * chx * k + in.f2 * chy * l) * iden;
                t_lp = (in.w2 * chx * l - in.f2 * chy * k) * iden;
                t_pl = (in.w2 * chy * k - in.f2 * chx * l) * iden;
                t_pp = (in.w2 * chy * l + in.f2 * chx * k) * iden;
                zl = in.w2 * chr * k * iden;
                zp = in.w2 * chr * l * iden;
                el = -in.f2 * in.n2 * chr * iden * k;
                ep = -in.f2 * in.n2 * chr * iden * l;
                if (THETA) {
                    // Eq. fluxes:temperature without theta-bar / (g rho-bar): ch_r f N^2 / (w^2 - f^2)
                    // (e_r x k_h), f signed at the ray
                    const float f = G.geometry == 1 ? 2.0f * G.f_omega * in.g.sphi : G.f_f0;
                    const float tc = f * in.n2 * chr * iden;
                    hv[7 % NH].hi = aw * -(tc * l);
                    hv[8 % NH].hi = aw * (tc * k);
                }
            } else {
                t_ll = chx * k; t_lp = chx * l; t_pl = chy * k; t_pp = chy * l;
                zl = chr * k; zp = chr * l;
                el = 0.0f; ep = 0.0f;
            }
            hv[0].hi = aw * t_ll; hv[1].hi = aw * t_lp; hv[2].hi = aw * t_pl;
            hv[3].hi = aw * t_pp; hv[4].hi = aw * el; hv[5].hi = aw * ep; hv[6].hi = aw;
            zl *= A;
            zp *= A;
            wh = in.g.cphi * s.e[0] * s.e[1] * G.whf32[s.j];
            const float zc = ((float)s.k + s.o[2]) * G.f_dz;
            lo = zc - 0.5f * s.e[2];
            hi = zc + 0.5f * s.e[2];
            kk0 = max(1, (int)floorf(lo * G.f_inv_dz - 0.5f));
            const int kk1 = min(G.nz - 1, (int)ceilf(hi * G.f_inv_dz + 0.5f));
            nkk = kk1 >= kk0 ? kk1 - kk0 + 1 : 0;
        }
        const bool own = warp_run_interior(key);
        if (warp_segment_reduce_df(key, hv) && key >= 0) {
            double* const dst[9] = {f_ll, f_lp, f_pl, f_pp, e_l, e_p, wad, f_tl, f_tp};
#pragma unroll
            for (int q = 0; q < NH; ++q) {
                const double v = df_to_double(hv[q]);
                // the whole cell is this run: store its sum (the ray-step kernel cleared the fields)
                if (own) dst[q][key] = v;
                else atomicAdd(&dst[q][key], v);
            }
        }
        int maxk = nkk;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxk = max(maxk, __shfl_xor_sync(0xffffffffu, maxk, o));
        for (int o = 0; o < maxk; ++o) {
            DF zv[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
            int zkey = -1;
            if (o < nkk) {
                const int kk = kk0 + o;
                const float slo = ((float)kk - 0.5f) * G.f_dz, shi = ((float)kk + 0.5f) * G.f_dz;
                const float ov = fminf(hi, shi) - fmaxf(lo, slo);
                if (ov > 0.0f) {
                    const float w = wh * ov * G.f_inv_dz;
                    zv[0].hi = w * zl;
                    zv[1].hi = w * zp;
                    zkey = col * (G.nz + 1) + kk;
                }
            }
            if (warp_segment_reduce_df(zkey, zv) && zkey >= 0) {
                atomicAdd(&fz_l[zkey], df_to_double(zv[0]));
                atomicAdd(&fz_p[zkey], df_to_double(zv[1]));
            }
        }
    }
    const double ws = block_sum(df_to_double(w_sat));
    const double wt = block_sum(df_to_double(w_tot));
    if (threadIdx.x == 0) {
        partials[T_SAT * pstride + blockIdx.x] = ws;
        partials[T_TOTAL * pstride + blockIdx.x] = wt;
    }
}

__global__ void k_gather_rays32(Grid G, Ray32SoA A, double* __restrict__ out, long long* __restrict__ ids,
                                int* __restrict__ cells, int64_t n)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        S32 s;
        load32(G, A, p, s);
        double d[NSTATE];
        to_double(G, s, d);
        for (int q = 0; q < NSTATE; ++q) out[q * n + p] = d[q];
        ids[p] = s.id;
        cells[p] = member_of(s.id) * G.ncell + cell32(G, s);
    }
}

void launch_gather_rays32(Context& c, double* state13, long long* ids, int* cells, int64_t n)
{
    const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096);
    k_gather_rays32<<<blocks, kThreads, 0, c.stream>>>(c.G, c.A32, state13, ids, cells, n);
}

// kernels shared with the FP64 step (gwam_step.cu)
__global__ void k_step_begin(Ctl* ctl);
__global__ void k_cap_find(Grid G, Params P, Ctl* ctl, const int* __restrict__ off, int* __restrict__ overlist);
__global__ void k_segsort(Grid G, Ctl* ctl, const int* __restrict__ off, const int* __restrict__ off2,
                          const long long* __restrict__ ent_id, const int* __restrict__ ent_src,
                          const int* __restrict__ ent_cell, int* __restrict__ sorted_src);
__global__ void __launch_bounds__(kThreads) k_sat_heads(Ctl* ctl, const int* __restrict__ off2, int ncell_all,
                                                          const int* __restrict__ raycell, int* __restrict__ runlist);

void run_step32(Context& c, double dt, double* du, double* dv)
{
    const Grid& G = c.G;
    const Params& P = c.P;
    cudaStream_t s = c.stream;
    const int nb = c.grid_blocks;
    // the cap's column pass: a thread per column (a grid sized by cells launched ~46 K mostly idle
    // blocks on the 512 x 256 x 90 grid: 26 us a step)
    const int col_blocks = (int)std::min<int64_t>((G.ncol_all + kThreads - 1) / kThreads, 65535LL * 4);
    const LaunchCfg& la = c.lcfg[0];
    const LaunchCfg& lm = c.lcfg[1];
    const LaunchCfg& lp = c.lcfg[2];
    k_step_begin<<<1, 1, 0, s>>>(c.ctl);
    cudaMemsetAsync(c.cnt, 0, sizeof(int) * (size_t)(G.ncell_all + 1), s);
    cudaMemsetAsync(c.partials, 0, sizeof(double) * NTALLY * (size_t)c.max_blocks, s);
    prof_mark(c, 0);
    tune_mark(c, 0);
    k_advance32<<<la.blocks, la.threads, 0, s>>>(G, P, c.A32, c.bg32, c.ctl, (float)dt, c.info, c.ccell, c.cslot,
                                                 c.newid, c.cnt, c.partials, c.max_blocks, clear_set(c));
    tune_mark(c, 1);
    prof_mark(c, 1);
    exclusive_scan2(c, c.newid, c.newid, c.max_rays, &c.ctl->n, c.cnt, c.off, G.ncell_all, nullptr);
    k_scatter32<<<nb, kThreads, 0, s>>>(G, c.A32, c.ctl, c.max_rays, c.info, c.ccell, c.cslot, c.newid, c.off,
                                        c.ent_id, c.ent_src, c.ent_cell);
    int mask = (1 << T_EXIT) | (1 << T_INVALID) | (1 << T_SAT) | (1 << T_TOTAL);
    const int* off2 = c.off;
    if (P.cap > 0) {
        k_cap_find<<<col_blocks, kThreads, 0, s>>>(G, P, c.ctl, c.off, c.overlist);
        k_cap_apply32<<<nb, kThreads, 0, s>>>(G, P, c.A32, c.bg32, c.ctl, c.info, c.off, c.overlist, c.ent_id,
                                              c.ent_src, c.ecap, c.cnt, c.partials, c.max_blocks);
        exclusive_scan(c, c.cnt, c.off2, G.ncell_all, nullptr);
        off2 = c.off2;
        mask |= 1 << T_CAP;
    }
    k_segsort<<<nb, kThreads, 0, s>>>(G, c.ctl, c.off, off2, c.ent_id, c.ent_src, c.ent_cell, c.sorted_src);
    tune_mark(c, 2);
    k_materialize32<<<lm.blocks, lm.threads, 0, s>>>(G, P, c.A32, c.B32, c.bg32, c.ctl, off2, c.sorted_src, c.info,
                                                     c.newid, c.pj, reinterpret_cast<float*>(c.k2), c.raycell);
    tune_mark(c, 3);
    prof_mark(c, 2);
    if (P.saturation) {
        // both saturation passes on the largest grid (eight blocks per SM, all resident): shorter
        // chains of per-block passes (saturation 0.070 -> 0.060 ms on the 512 x 256 sphere)
        k_sat_heads<<<c.max_blocks, kThreads, 0, s>>>(c.ctl, off2, G.ncell_all, c.raycell, c.biglist);
        k_sat_kappa32<<<c.max_blocks, kThreads, 0, s>>>(c.ctl, off2, c.biglist, c.rho, c.pj,
                                              reinterpret_cast<const float*>(c.k2), (float)dt,
                                              reinterpret_cast<float*>(c.kappa));
    }
    prof_mark(c, 3);
    // (the projected fields were cleared by k_advance32)
    tune_mark(c, 4);
    if (P.theta_flux)
        k_project32<true><<<lp.blocks, lp.threads, 0, s>>>(
            G, P, c.B32, c.bg32, c.ctl, off2, reinterpret_cast<const float*>(c.kappa),
            reinterpret_cast<const float*>(c.k2), dt, c.field[F_ZL], c.field[F_ZP], c.field[F_LL], c.field[F_LP],
            c.field[F_PL], c.field[F_PP], c.field[F_EL], c.field[F_EP], c.field[F_WAD], c.field[F_TL], c.field[F_TP],
            c.partials, c.max_blocks);
    else
        k_project32<false><<<lp.blocks, lp.threads, 0, s>>>(
            G, P, c.B32, c.bg32, c.ctl, off2, reinterpret_cast<const float*>(c.kappa),
            reinterpret_cast<const float*>(c.k2), dt, c.field[F_ZL], c.field[F_ZP], c.field[F_LL], c.field[F_LP],
            c.field[F_PL], c.field[F_PP], c.field[F_EL], c.field[F_EP], c.field[F_WAD], nullptr, nullptr,
            c.partials, c.max_blocks);
    tune_mark(c, 5);
    if (c.tune_active) ++c.tune_pending;
    prof_mark(c, 4);
    grid_phase32(c, du, dv, mask);
    prof_mark(c, 5);
    swap_rays(c);
}

}  // namespace gwam
