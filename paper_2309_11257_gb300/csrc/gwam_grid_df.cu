// gwam_grid_df.cu -- smoothing and divergence of the FP64 form in double-float arithmetic.
//
// GB300 executes FP64 at 1/72 of its FP32 rate, and the 9-point smoothing of eight FP64 flux fields
// plus the divergence were bound by it.  Here each FP64 projection sum is split, as it is loaded,
// into a double-float pair hi + lo (hi = x rounded to FP32, lo = the remainder rounded to FP32;
// about 48 significant bits) -- one FP64 subtraction per load -- and the stencil arithmetic runs on
// the FP32 pipes (TwoSum / TwoProduct).  Only the final du/dt, dv/dt are formed in FP64 (one
// addition each).  The result differs from FP64 arithmetic by rounding at the 2^-46 level,
// far below the 1e-9 parity bar of the FP64 form.
#include "gwam_common.cuh"
#include "gwam_fp32.cuh"

namespace gwam {

namespace {

__device__ __forceinline__ DF df_load(const float2* p) { const float2 v = *p; return {v.x, v.y}; }

struct FieldSetDF {
    const double* in[NFIELD];
    float2* out[NFIELD];
};

// 1-2-1 x 1-2-1 smoothing (periodic in lambda, edge row reused at the poles): a warp owns 32
// consecutive levels of kRowsDF rows over kSpanDF columns.  For every column it loads and splits the
// kRowsDF + 2 values of its rows and their two neighbours once (2 loads and splits per output
// instead of 3 for two rows: measured faster than 1, 4 or 8 rows), forms the vertical 1-2-1 sums
// of its rows, and slides a window of three such sums along the row (spans of 16 columns: measured
// faster than 8 or 32).  The raw values of the column after next are loaded while the next one is
// summed, so every warp keeps two columns' loads in flight (grid phase 0.291 -> 0.228 ms on the
// 256 x 128 x 90 sphere; a distance of two columns gained nothing more).  Warp item = (field,
// member, row group, level group, span).
constexpr int kSpanDF = 16;
constexpr int kRowsDF = 2;
__global__ void __launch_bounds__(256) k_smooth_df(Grid G, FieldSetDF fs, int f0, int nf)
{
    const int lane = threadIdx.x & 31;
    const int nlg = (G.nz + 1 + 31) / 32;
    const int nsp = (G.nx + kSpanDF - 1) / kSpanDF;
    const int nrg = (G.ny + kRowsDF - 1) / kRowsDF;
    const long long per_field = (long long)G.members * nrg * nlg * nsp;
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= per_field * nf) return;
    const int f = f0 + (int)(w / per_field);
    long long r = w % per_field;
    const int sp = (int)(r % nsp);
    r /= nsp;
    const int lg = (int)(r % nlg);
    r /= nlg;
    const int rg = (int)(r % nrg);
    const int mem = (int)(r / nrg);
    const int nlev = f <= F_ZP ? G.nz + 1 : G.nz;
    if (lg * 32 >= nlev) return;
    const int lev = lg * 32 + lane;
    const bool live = lev < nlev;
    const int j0 = rg * kRowsDF;
    const int nrow = min(kRowsDF, G.ny - j0);
    // source rows j0 - 1 .. j0 + kRowsDF (clamped at the poles, wrapped on the f-plane)
    const double* src[kRowsDF + 2];
    const int64_t base = (int64_t)mem * G.ncol;
    const double* __restrict__ F = fs.in[f];
#pragma unroll
    for (int q = 0; q < kRowsDF + 2; ++q) {
        int jj = j0 - 1 + q;
        if (G.geometry == 1) jj = jj < 0 ? 0 : (jj >= G.ny ? G.ny - 1 : jj);
        else jj = jj < 0 ? jj + G.ny : (jj >= G.ny ? jj - G.ny : jj);
        src[q] = F + (base + (int64_t)jj * G.nx) * nlev + lev;
    }
    float2* O = fs.out[f] + (base + (int64_t)j0 * G.nx) * nlev + lev;
    const int64_t orow = (int64_t)G.nx * nlev;
    auto wrapc = [&](int i) { return i >= G.nx ? i - G.nx : (i < 0 ? i + G.nx : i); };
    auto loadraw = [&](int i, bool ok, double (&v)[kRowsDF + 2]) {
        const int64_t o = (int64_t)wrapc(i) * nlev;
#pragma unroll
        for (int q = 0; q < kRowsDF + 2; ++q) v[q] = (live && ok) ? src[q][o] : 0.0;
    };
    // Most cells receive no ray volume, so whole columns of a warp's 32 levels are +0.0: their sums
    // are +0.0 without the splits and additions (the same bits), and an output whose three column
    // sums are all +0.0 is stored as such.  The flags are warp-uniform (votes).
    auto sums = [&](const double (&r)[kRowsDF + 2], DF (&cs)[kRowsDF]) -> bool {
        bool zero = true;
#pragma unroll
        for (int q = 0; q < kRowsDF + 2; ++q) zero = zero && __double_as_longlong(r[q]) == 0;
        if (__all_sync(0xffffffffu, zero)) {
#pragma unroll
            for (int q = 0; q < kRowsDF; ++q) cs[q] = df_f(0.0f);
            return true;
        }
        DF v[kRowsDF + 2];
#pragma unroll
        for (int q = 0; q < kRowsDF + 2; ++q) v[q] = df_split(r[q]);
#pragma unroll
        for (int q = 0; q < kRowsDF; ++q) cs[q] = df_add(df_add(v[q], df_pow2(v[q + 1], 2.0f)), v[q + 2]);
        return false;
    };
    auto emit = [&](int i, const DF (&cm)[kRowsDF], const DF (&c0)[kRowsDF], const DF (&cp)[kRowsDF], bool zero) {
        if (zero) {
            if (live)
#pragma unroll
                for (int q = 0; q < kRowsDF; ++q)
                    if (q < nrow) O[q * orow + (int64_t)i * nlev] = make_float2(0.0f, 0.0f);
            return;
        }
        if (live) {
#pragma unroll
            for (int q = 0; q < kRowsDF; ++q) {
                if (q < nrow) {
                    const DF s = df_pow2(df_add(df_add(cm[q], df_pow2(c0[q], 2.0f)), cp[q]), 0.0625f);
                    O[q * orow + (int64_t)i * nlev] = make_float2(s.hi, s.lo);
                }
            }
        }
    };
    const int i0 = sp * kSpanDF, i1 = min(G.nx, i0 + kSpanDF);
    DF cm[kRowsDF], c0[kRowsDF], cp[kRowsDF];
    double ra[kRowsDF + 2], rb[kRowsDF + 2];
    loadraw(i0 - 1, true, ra);
    loadraw(i0, true, rb);
    bool zm = sums(ra, cm);
    loadraw(i0 + 1, true, ra);
    bool z0 = sums(rb, c0);
#pragma unroll 1
    for (int i = i0; i < i1; ++i) {
        double rn[kRowsDF + 2];
        loadraw(i + 2, i + 2 <= i1, rn);
        const bool zp = sums(ra, cp);
        emit(i, cm, c0, cp, zm && z0 && zp);
        zm = z0;
        z0 = zp;
#pragma unroll
        for (int q = 0; q < kRowsDF; ++q) {
            cm[q] = c0[q];
            c0[q] = cp[q];
        }
#pragma unroll
        for (int q = 0; q < kRowsDF + 2; ++q) ra[q] = rn[q];
    }
}

// Divergence (Eq. mean-flow-impact) of the smoothed double-float fields,
//   du/dt = -(1/rho) [ (1/(r cos phi)) (d_lambda F^{ll} + d_phi (cos phi F^{pl})) + d_z F^z_l ] + E_l / (g rho),
// dv/dt likewise (centred differences, flux zero beyond the pole rows; in the columnar mode the
// vertical term alone): one block per (row, tile of TW columns), results transposed through shared
// memory into [nz][ny][nx]; only the final du/dt, dv/dt are formed in FP64.
struct DivConsts {
    DF h2x, h2y, idz, ig;
};

__global__ void k_divergence_df(Grid G, int TW, DivConsts K, const float2* __restrict__ tabs,
                                const float2* __restrict__ fzl, const float2* __restrict__ fzp,
                                const float2* __restrict__ fll, const float2* __restrict__ flp,
                                const float2* __restrict__ fpl, const float2* __restrict__ fpp,
                                const float2* __restrict__ el, const float2* __restrict__ ep,
                                const double* __restrict__ rho_inv, double* __restrict__ du, double* __restrict__ dv)
{
    extern __shared__ double tile_df[];
    double* tu = tile_df;
    double* tv = tile_df + (size_t)TW * G.nz;
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
    // tables: row_cos [ny], row_inv_cos [ny], lev_inv_r [nz] as double-float pairs
    const float2* tcos = tabs;
    const float2* ticos = tabs + G.ny;
    const float2* tlev = tabs + 2 * G.ny;
    DF rcp_cos{1.0f, 0.0f}, cn{0.0f, 0.0f}, cs{0.0f, 0.0f};
    if (G.geometry == 1) {
        rcp_cos = df_load(&ticos[j]);
        if (j + 1 < G.ny) cn = df_load(&tcos[j + 1]);
        if (j - 1 >= 0) cs = df_load(&tcos[j - 1]);
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
        DF pl_n{0.0f, 0.0f}, pl_s{0.0f, 0.0f}, pp_n{0.0f, 0.0f}, pp_s{0.0f, 0.0f};
        if (jn >= 0 && jn < G.ny) {
            const int64_t cc = ((int64_t)jn * G.nx + i) * nz + k;
            pl_n = df_load(&fpl[cc]);
            pp_n = df_load(&fpp[cc]);
        }
        if (js >= 0 && js < G.ny) {
            const int64_t cc = ((int64_t)js * G.nx + i) * nz + k;
            pl_s = df_load(&fpl[cc]);
            pp_s = df_load(&fpp[cc]);
        }
        const DF ri = df_split(rho_inv[c]);
        const DF dzl = df_mul2(df_sub(df_load(&fzl[zc + 1]), df_load(&fzl[zc])), K.idz);
        const DF dzp = df_mul2(df_sub(df_load(&fzp[zc + 1]), df_load(&fzp[zc])), K.idz);
        DF div_u, div_v;
        if (G.geometry == 1) {
            const DF mh = df_mul2(rcp_cos, df_load(&tlev[k]));
            const DF xu = df_mul2(df_sub(df_load(&fll[ce]), df_load(&fll[cw])), K.h2x);
            const DF yu = df_mul2(df_sub(df_mul2(cn, pl_n), df_mul2(cs, pl_s)), K.h2y);
            const DF xv = df_mul2(df_sub(df_load(&flp[ce]), df_load(&flp[cw])), K.h2x);
            const DF yv = df_mul2(df_sub(df_mul2(cn, pp_n), df_mul2(cs, pp_s)), K.h2y);
            div_u = df_add(df_mul2(df_add(xu, yu), mh), dzl);
            div_v = df_add(df_mul2(df_add(xv, yv), mh), dzp);
        } else {
            div_u = df_add(df_add(df_mul2(df_sub(df_load(&fll[ce]), df_load(&fll[cw])), K.h2x),
                                  df_mul2(df_sub(pl_n, pl_s), K.h2y)),
                           dzl);
            div_v = df_add(df_add(df_mul2(df_sub(df_load(&flp[ce]), df_load(&flp[cw])), K.h2x),
                                  df_mul2(df_sub(pp_n, pp_s), K.h2y)),
                           dzp);
        }
        if (G.columnar) {
            // horizontally homogeneous column: the vertical flux divergence alone
            div_u = dzl;
            div_v = dzp;
        }
        const DF ru = df_mul2(df_sub(df_mul2(df_load(&el[c]), K.ig), div_u), ri);
        const DF rv = df_mul2(df_sub(df_mul2(df_load(&ep[c]), K.ig), div_v), ri);
        tu[k * TW + ii] = df_to_double(ru);
        tv[k * TW + ii] = df_to_double(rv);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int ii = t % TW, k = t / TW;
        const int i = i0 + ii;
        if (i >= G.nx) continue;
        const int64_t o = ((int64_t)k * G.ny + j) * G.nx + i;
        if (du) du[o] = tu[k * TW + ii];
        if (dv) dv[o] = tv[k * TW + ii];
    }
}

DF host_split(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

__global__ void k_split_df(FieldSetDF fs, int64_t n0, int64_t n1, int nf)
{
    const int f = blockIdx.y;
    if (f >= nf) return;
    const int64_t n = f <= F_ZP ? n0 : n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const DF v = df_split(fs.in[f][i]);
        fs.out[f][i] = make_float2(v.hi, v.lo);
    }
}

void split_fields_df(Context& c, const double* const* in, float2* const* out, int nf)
{
    FieldSetDF fs{};
    for (int f = 0; f < nf; ++f) {
        fs.in[f] = in[f];
        fs.out[f] = out[f];
    }
    const int blocks = (int)std::min<int64_t>((c.field_len(0) + kThreads - 1) / kThreads, 4 * 152);
    k_split_df<<<dim3((unsigned)blocks, (unsigned)nf), kThreads, 0, c.stream>>>(fs, c.field_len(0),
                                                                              c.field_len(F_LL), nf);
}

}  // namespace

void grid_phase_df(Context& c, double* du, double* dv, int mask)
{
    const Grid& G = c.G;
    cudaStream_t s = c.stream;
    double* out_u = du ? du : c.dudt_buf;
    double* out_v = dv ? dv : c.dvdt_buf;
    const float2* fl[NFIELD];
    // the smoothed double-float fields live in the (otherwise on-demand) FP64 smoothing buffers
    float2* sm[NFIELD];
    for (int f = 0; f < NFIELD; ++f) sm[f] = reinterpret_cast<float2*>(c.smooth[f]);
    if (c.P.smoothing) {
        FieldSetDF fs{};
        for (int f = 0; f < NFIELD; ++f) {
            fs.in[f] = c.field[f];
            fs.out[f] = sm[f];
        }
        const long long warps = (long long)F_WAD * G.members * ((G.ny + kRowsDF - 1) / kRowsDF) *
                                ((G.nz + 1 + 31) / 32) * ((G.nx + kSpanDF - 1) / kSpanDF);
        k_smooth_df<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(G, fs, 0, F_WAD);
        for (int f = 0; f < NFIELD; ++f) fl[f] = sm[f];
    } else {
        // unsmoothed: split in place into the same buffers (one pass per field)
        FieldSetDF fs{};
        for (int f = 0; f < NFIELD; ++f) {
            fs.in[f] = c.field[f];
            fs.out[f] = sm[f];
        }
        split_fields_df(c, fs.in, fs.out, F_WAD);
        for (int f = 0; f < NFIELD; ++f) fl[f] = sm[f];
    }
    DivConsts K;
    K.h2x = host_split(0.5 * G.inv_dX);
    K.h2y = host_split(0.5 * G.inv_dY);
    K.idz = host_split(G.inv_dz);
    K.ig = host_split(G.inv_g);
    const int TW = G.nz <= 96 ? 32 : 16;
    const size_t shm = sizeof(double) * 2 * (size_t)TW * G.nz;
    if (shm > 48 * 1024) cudaFuncSetAttribute(k_divergence_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    const int ntx = (G.nx + TW - 1) / TW;
    k_divergence_df<<<ntx * G.ny * G.members, kThreads, shm, s>>>(
        G, TW, K, c.tables_df, fl[F_ZL], fl[F_ZP], fl[F_LL], fl[F_LP], fl[F_PL], fl[F_PP], fl[F_EL], fl[F_EP],
        c.rho_inv, out_u, out_v);
    finalize_tallies(c, mask, 1);
}

}  // namespace gwam
