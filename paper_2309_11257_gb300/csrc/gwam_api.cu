// gwam_api.cu -- the extern "C" entry points declared in include/gwam.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "gwam_common.cuh"

struct gwam_ctx {
    gwam::Context c;
};

namespace gwam {

#define GWAM_CUDA(call)                                                                                \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            c.err = std::string(#call) + ": " + cudaGetErrorString(e_);                                \
            throw (int)(e_ == cudaErrorMemoryAllocation ? GWAM_ENOMEM : GWAM_ECUDA);                  \
        }                                                                                              \
    } while (0)

template <typename T>
static void dalloc(Context& c, T*& p, size_t count)
{
    GWAM_CUDA(cudaMalloc((void**)&p, sizeof(T) * std::max<size_t>(count, 1)));
}

static void free_all(Context& c)
{
    void* ptrs[] = {c.bg, c.bg32, c.bgdf, c.ray32_mem[0], c.ray32_mem[1], c.rho, c.rho_inv, c.tables, c.tables32, c.tables_df,
                    c.bg_scratch, c.theta,
                    c.ray_mem[0], c.ray_mem[1], c.info, c.ccell, c.cslot, c.newid,
                    c.ent_id, c.ent_src, c.ent_cell, c.sorted_src, c.pj, c.k2, c.kappa, c.raycell, c.ecap, c.cnt, c.off, c.off2,
                    c.overlist, c.biglist, c.scan_tmp, c.dudt_buf, c.dvdt_buf, c.ctl,
                    c.budget, c.partials, c.flag_dev, c.spec_buf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int f = 0; f < NFIELD; ++f) {
        if (c.field[f]) cudaFree(c.field[f]);
        if (c.smooth[f]) cudaFree(c.smooth[f]);
        if (c.nar32[f]) cudaFree(c.nar32[f]);
        if (c.sm32[f]) cudaFree(c.sm32[f]);
    }
    if (c.rho_inv32) cudaFree(c.rho_inv32);
    for (int q = 0; q < Context::kRing; ++q)
        for (int p = 0; p <= Context::kPhases; ++p)
            if (c.prof_ev[q][p]) cudaEventDestroy(c.prof_ev[q][p]);
    for (int q = 0; q < Context::kTuneRing; ++q)
        for (int p = 0; p < 6; ++p)
            if (c.tune_ev[q][p]) cudaEventDestroy(c.tune_ev[q][p]);
    for (int q = 0; q < Context::kGraphs; ++q)
        if (c.gexec[q]) cudaGraphExecDestroy(c.gexec[q]);
    for (int q = 0; q < Context::kGraphs; ++q)
        for (int p = 0; p <= Context::kPhases; ++p)
            if (c.gprof_ev[q][p]) cudaEventDestroy(c.gprof_ev[q][p]);
    {
        void* alt[] = {c.bg_alt, c.bgdf_alt, c.bg32_alt, c.rho_alt, c.rho_inv_alt, c.rho_inv32_alt, c.flag_async};
        for (void* p : alt)
            if (p) cudaFree(p);
        for (int q = 0; q < 2; ++q)
            if (c.ev_rel[q]) cudaEventDestroy(c.ev_rel[q]);
        if (c.ev_setup_done) cudaEventDestroy(c.ev_setup_done);
        if (c.setup_stream) cudaStreamDestroy(c.setup_stream);
    }
    if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
    for (int q = 0; q < 2; ++q) {
        if (c.bg_stage[q]) cudaFree(c.bg_stage[q]);
        if (c.d_out[q]) cudaFree(c.d_out[q]);
        cudaEvent_t* evs[] = {&c.ev_up[q], &c.ev_free[q], &c.ev_dready[q], &c.ev_d2h[q]};
        for (cudaEvent_t* e : evs)
            if (*e) cudaEventDestroy(*e);
    }
    if (c.up_stream) cudaStreamDestroy(c.up_stream);
    if (c.down_stream) cudaStreamDestroy(c.down_stream);
    if (c.ctl_host) cudaFreeHost(c.ctl_host);
    if (c.budget_host) cudaFreeHost(c.budget_host);
    if (c.flag_host) cudaFreeHost(c.flag_host);
}

static void check_pending(Context& c)
{
    // asynchronous host copies
    if (c.up_stream) GWAM_CUDA(cudaStreamSynchronize(c.up_stream));
    if (c.down_stream) GWAM_CUDA(cudaStreamSynchronize(c.down_stream));
    GWAM_CUDA(cudaMemcpyAsync(c.ctl_host, c.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c.stream));
    GWAM_CUDA(cudaMemcpyAsync(c.budget_host, c.budget, sizeof(DevBudget), cudaMemcpyDeviceToHost, c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    GWAM_CUDA(cudaGetLastError());
    if (c.ctl_host->status != 0) {
        const int st = c.ctl_host->status;
        c.err = st == GWAM_ECAPACITY ? "device: ray capacity (max_rays) exceeded" : "device: status set";
        throw st;
    }
}

// Same-extent host/device copy helpers
static void h2d(Context& c, void* dst, const void* src, size_t bytes)
{
    GWAM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c.stream));
}

// Device address of a page-locked, device-mapped host buffer [p, p + bytes) (kernels then read or
// write it directly over the host link, without a staging copy), or null when any part of it is
// pageable or unmapped.
static void* mapped_host(const void* p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    const char* q = static_cast<const char*>(p);
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess || cudaPointerGetAttributes(&b, q + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if (static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
}

}  // namespace gwam

using namespace gwam;

#define API_BEGIN(ctx)                                                                                 \
    if (!(ctx)) return GWAM_EINVAL;                                                                    \
    Context& c = (ctx)->c;                                                                             \
    try {
#define API_END                                                                                        \
    }                                                                                                  \
    catch (int code) { return code; }                                                                  \
    catch (std::bad_alloc&) { c.err = "host allocation failed"; return GWAM_ENOMEM; }                  \
    return GWAM_OK;

extern "C" {

const char* gwam_version(void) { return "gwam-gb300 0.2 (sm_103a; FP64 and FP32-kinematics forms)"; }

int gwam_init(gwam_ctx** out, const gwam_grid* grid, const gwam_params* params, void* stream)
{
    if (!out || !grid || !params) return GWAM_EINVAL;
    *out = nullptr;
    if (grid->geometry != 0 && grid->geometry != 1) return GWAM_EINVAL;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || !(grid->dz > 0.0)) return GWAM_EINVAL;
    if (grid->geometry == 0 && !(grid->dx > 0.0 && grid->dy > 0.0)) return GWAM_EINVAL;
    if (grid->geometry == 1 && !(grid->radius > 0.0)) return GWAM_EINVAL;
    if (!(grid->g > 0.0)) return GWAM_EINVAL;
    if ((int64_t)grid->nx * grid->ny * (grid->nz + 1) >= (int64_t)1 << 31) return GWAM_EINVAL;
    if (grid->nz > 192) return GWAM_EINVAL;   // column tiles of the transposing kernels live in shared memory
    if (params->precision != 0 && params->precision != 1) return GWAM_EINVAL;
    if (params->columnar != 0 && params->columnar != 1) return GWAM_EINVAL;
    if (params->theta_flux != 0 && params->theta_flux != 1) return GWAM_EINVAL;
    if (params->max_rays < 1 || params->max_rays >= ((int64_t)1 << 29)) return GWAM_EINVAL;
    if (!(params->alpha_s > 0.0) || !(params->min_split_dz >= 0.0)) return GWAM_EINVAL;
    if (params->flux_form != 0 && params->flux_form != 1) return GWAM_EINVAL;
    const int members = params->members <= 0 ? 1 : params->members;
    if (members > 255) return GWAM_EINVAL;
    if ((int64_t)grid->nx * grid->ny * (grid->nz + 1) * members >= (int64_t)1 << 31) return GWAM_EINVAL;
    gwam_ctx* h = new (std::nothrow) gwam_ctx();
    if (!h) return GWAM_ENOMEM;
    Context& c = h->c;
    try {
        GWAM_CUDA(cudaGetDevice(&c.device));
        GWAM_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
        c.stream = (cudaStream_t)stream;
        Grid& G = c.G;
        G.geometry = grid->geometry;
        G.nx = grid->nx;
        G.ny = grid->ny;
        G.nz = grid->nz;
        G.ncol = grid->nx * grid->ny;
        G.ncell = G.ncol * grid->nz;
        G.members = members;
        G.ncol_all = G.ncol * members;
        G.ncell_all = G.ncell * members;
        c.member_bg.assign(members, false);
        G.dz = grid->dz;
        G.f0 = grid->f0;
        G.radius = grid->radius;
        G.omega = grid->omega;
        G.g = grid->g;
        G.ztop = grid->nz * grid->dz;
        if (G.geometry == 1) {
            G.dX = 2.0 * kPi / grid->nx;
            G.dY = kPi / grid->ny;
            G.y0 = -0.5 * kPi;
            G.Lx = 2.0 * kPi;
            G.Ly = kPi;
        } else {
            G.dX = grid->dx;
            G.dY = grid->dy;
            G.y0 = 0.0;
            G.Lx = grid->nx * grid->dx;
            G.Ly = grid->ny * grid->dy;
        }
        G.phimax = 0.5 * kPi - 0.5 * G.dY;
        G.inv_dX = 1.0 / G.dX;
        G.inv_dY = 1.0 / G.dY;
        G.inv_dz = 1.0 / G.dz;
        G.inv_nx = 1.0 / G.nx;
        G.inv_ny = 1.0 / G.ny;
        G.inv_g = 1.0 / G.g;
        G.f_dX = (float)G.dX;
        G.f_dY = (float)G.dY;
        G.f_dz = (float)G.dz;
        G.f_y0 = (float)G.y0;
        G.f_radius = (float)G.radius;
        G.f_omega = (float)G.omega;
        G.f_f0 = (float)G.f0;
        G.f_inv_dX = (float)G.inv_dX;
        G.f_inv_dY = (float)G.inv_dY;
        G.f_inv_dz = (float)G.inv_dz;
        Params& P = c.P;
        P.gamma_mode = params->gamma_mode;
        P.saturation = params->saturation;
        P.smoothing = params->smoothing;
        P.flux_form = params->flux_form;
        P.splitting = params->splitting;
        G.columnar = params->columnar;
        P.theta_flux = params->theta_flux;
        P.cap = params->cap_per_column;
        P.alpha_s = params->alpha_s;
        P.f_alpha_s = (float)params->alpha_s;
        P.min_split_dz = params->min_split_dz;
        c.max_rays = params->max_rays;
        // persistent grids: multiples of the SM count; the three heavy ray kernels are autotunable
        c.grid_blocks = c.num_sms * 4;
        c.max_blocks = c.num_sms * 8;
        for (int q = 0; q < 3; ++q) c.lcfg[q] = LaunchCfg{kThreads, c.num_sms * 4};
        GWAM_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));

        const size_t nr = (size_t)c.max_rays;
        const size_t ncell = (size_t)G.ncell_all;
        dalloc(c, c.bg, ncell);
        dalloc(c, c.rho, ncell);
        dalloc(c, c.rho_inv, ncell);
        {
            // row and level tables (host-computed once)
            // split thresholds per row (App. B.3) after the row-centre latitudes: alpha_s sqrt(cos dX dY),
            // alpha_s cos dX dY (cos = 1 on the f-plane), evaluated left to right as the oracle does
            const size_t o_thr = 3 * (size_t)G.ny + G.nz, o_f2 = o_thr + 2 * (size_t)G.ny;
            std::vector<double> tab(o_f2 + G.ny);
            for (int j = 0; j < G.ny; ++j) {
                const double phi = G.y0 + (j + 0.5) * G.dY;
                tab[j] = G.geometry == 1 ? cos(phi) : 1.0;
                tab[G.ny + j] = 1.0 / tab[j];
                tab[2 * (size_t)G.ny + G.nz + j] = phi;   // row-centre latitude
                const double f = G.geometry == 1 ? 2.0 * G.omega * sin(phi) : G.f0;
                tab[o_f2 + j] = f * f;
                if (G.geometry == 1) {
                    tab[o_thr + 2 * j] = P.alpha_s * sqrt(tab[j] * G.dX * G.dY);
                    tab[o_thr + 2 * j + 1] = P.alpha_s * tab[j] * G.dX * G.dY;
                } else {
                    tab[o_thr + 2 * j] = P.alpha_s * sqrt(G.dX * G.dY);
                    tab[o_thr + 2 * j + 1] = P.alpha_s * G.dX * G.dY;
                }
            }
            G.split_hthr = fmax(P.alpha_s * G.dz, P.min_split_dz);
            for (int k = 0; k < G.nz; ++k)
                tab[2 * G.ny + k] = G.geometry == 1 ? 1.0 / (G.radius + (k + 0.5) * G.dz) : 1.0;
            dalloc(c, c.tables, tab.size());
            GWAM_CUDA(cudaMemcpy(c.tables, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
            G.row_cos = c.tables;
            G.row_inv_cos = c.tables + G.ny;
            G.lev_inv_r = c.tables + 2 * G.ny;
            G.row_lat = c.tables + 2 * G.ny + G.nz;
            G.split_thr = c.tables + o_thr;
            G.row_f2 = c.tables + o_f2;
            std::vector<float> t32(2 * (size_t)G.ny + (size_t)G.ny * G.nz);
            for (int j = 0; j < G.ny; ++j) {
                t32[j] = (float)tab[j];
                t32[G.ny + j] = (float)(tab[G.ny + j] * G.inv_dX * G.inv_dY);
                for (int k = 0; k < G.nz; ++k) {
                    const double ir = tab[2 * G.ny + k];
                    const double iv = G.geometry == 1 ? ir * ir * tab[G.ny + j] * G.inv_dX * G.inv_dY * G.inv_dz
                                                      : G.inv_dX * G.inv_dY * G.inv_dz;
                    t32[2 * (size_t)G.ny + (size_t)j * G.nz + k] = (float)iv;
                }
            }
            // double-float tables: row_cos, row_inv_cos [ny], lev_inv_r [nz], then (sin, cos) of every
            // row centre [ny][2], the horizontal share per unit extent [ny] and the inverse cell
            // volumes [ny][nz]
            auto split = [](double x) {
                const float hi = (float)x;
                return make_float2(hi, (float)(x - (double)hi));
            };
            const size_t o_whf = 4 * (size_t)G.ny + G.nz, o_ivol = o_whf + G.ny, o_lat = o_ivol + (size_t)G.ny * G.nz;
            std::vector<float2> tdf(o_lat + G.ny);
            for (int j = 0; j < G.ny; ++j) tdf[o_lat + j] = split(tab[2 * (size_t)G.ny + G.nz + j]);
            for (int j = 0; j < G.ny; ++j) {
                tdf[o_whf + j] = split(tab[G.ny + j] * G.inv_dX * G.inv_dY);
                for (int k = 0; k < G.nz; ++k) {
                    const double ir = tab[2 * G.ny + k];
                    tdf[o_ivol + (size_t)j * G.nz + k] =
                        split(G.geometry == 1 ? ir * ir * tab[G.ny + j] * G.inv_dX * G.inv_dY * G.inv_dz
                                              : G.inv_dX * G.inv_dY * G.inv_dz);
                }
            }
            for (int q = 0; q < 2 * G.ny + G.nz; ++q) tdf[q] = split(tab[q]);
            for (int j = 0; j < G.ny; ++j) {
                const double phi = tab[2 * (size_t)G.ny + G.nz + j];
                tdf[2 * (size_t)G.ny + G.nz + 2 * j] = split(G.geometry == 1 ? sin(phi) : 0.0);
                tdf[2 * (size_t)G.ny + G.nz + 2 * j + 1] = split(G.geometry == 1 ? cos(phi) : 1.0);
            }
            dalloc(c, c.tables_df, tdf.size());
            GWAM_CUDA(cudaMemcpy(c.tables_df, tdf.data(), sizeof(float2) * tdf.size(), cudaMemcpyHostToDevice));
            G.row_sc_df = c.tables_df + 2 * G.ny + G.nz;
            G.whf_df = c.tables_df + o_whf;
            G.ivol_df = c.tables_df + o_ivol;
            G.row_lat_df = c.tables_df + o_lat;
            G.df_inv_dX = split(G.inv_dX);
            G.df_inv_dY = split(G.inv_dY);
            G.df_inv_dz = split(G.inv_dz);
            G.df_y0 = split(G.y0);
            G.df_radius = split(G.radius);
            G.df_2omega = split(2.0 * G.omega);
            G.df_8omega2 = split(8.0 * G.omega * G.omega);
            G.df_f0sq = split(G.f0 * G.f0);
            G.df_f0 = split(G.f0);
            dalloc(c, c.tables32, t32.size());
            GWAM_CUDA(cudaMemcpy(c.tables32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice));
            G.row_cos32 = c.tables32;
            G.whf32 = c.tables32 + G.ny;
            G.ivol32 = c.tables32 + 2 * G.ny;
        }
        c.f32 = params->precision == 1;
        // the precision form's projection (48 registers) gains from eight blocks per SM: 0.275 ->
        // 0.265 ms on the 512 x 256 sphere; the FP64 form's kernels and the materialise pass do not.
        // The FP64 ray step (two resident 256-thread blocks per SM) runs as one wave of blocks:
        // 0.585-0.592 -> 0.574-0.577 ms on the 256 x 128 sphere; the precision form's is slower so
        // (0.532 -> 0.553 ms) and keeps four blocks per SM
        if (c.f32) c.lcfg[2] = LaunchCfg{kThreads, c.num_sms * 8};
        else c.lcfg[0] = LaunchCfg{kThreads, c.num_sms * 2};
        for (int b = 0; b < 2; ++b) {
            if (c.f32) {
                dalloc(c, c.ray32_mem[b], 4 * nr);
                Ray32SoA& R = b == 0 ? c.A32 : c.B32;
                for (int q = 0; q < 4; ++q) R.q[q] = c.ray32_mem[b] + q * nr;
            } else {
                dalloc(c, c.ray_mem[b], 7 * nr);
                RaySoA& R = b == 0 ? c.A : c.B;
                for (int q = 0; q < 7; ++q) R.a[q] = c.ray_mem[b] + q * nr;
            }
        }
        if (c.f32) dalloc(c, c.bg32, ncell);
        else dalloc(c, c.bgdf, ncell);
        dalloc(c, c.info, nr);
        dalloc(c, c.ccell, nr);
        dalloc(c, c.cslot, nr);
        dalloc(c, c.newid, nr + 1);
        dalloc(c, c.ent_id, nr);
        dalloc(c, c.ent_src, nr);
        dalloc(c, c.ent_cell, nr);
        dalloc(c, c.sorted_src, nr);
        dalloc(c, c.pj, nr);
        dalloc(c, c.k2, nr);
        dalloc(c, c.kappa, nr);
        dalloc(c, c.raycell, nr);
        dalloc(c, c.ecap, nr);
        dalloc(c, c.cnt, ncell + 1);
        dalloc(c, c.off, ncell + 1);
        dalloc(c, c.off2, ncell + 1);
        dalloc(c, c.overlist, (size_t)G.ncol_all);
        dalloc(c, c.biglist, ncell);
        const size_t scan_blocks = (std::max(nr, ncell) + 2047) / 2048 + 2;
        dalloc(c, c.scan_tmp, scan_blocks + 1);
        c.scan_tmp_cap = (int64_t)scan_blocks + 1;
        if (c.f32) {
            for (int f = 0; f < NFIELD; ++f) {
                // the narrowed raw fields only without smoothing (the smoothing narrows as it loads)
                if (!c.P.smoothing) dalloc(c, c.nar32[f], (size_t)c.field_len(f));
                dalloc(c, c.sm32[f], (size_t)c.field_len(f));
            }
            dalloc(c, c.rho_inv32, ncell);
        }
        for (int f = 0; f < NFIELD; ++f) {
            dalloc(c, c.field[f], (size_t)c.field_len(f));
            dalloc(c, c.smooth[f], (size_t)c.field_len(f));
            GWAM_CUDA(cudaMemsetAsync(c.field[f], 0, sizeof(double) * (size_t)c.field_len(f), c.stream));
            GWAM_CUDA(cudaMemsetAsync(c.smooth[f], 0, sizeof(double) * (size_t)c.field_len(f), c.stream));
        }
        dalloc(c, c.dudt_buf, ncell);
        dalloc(c, c.dvdt_buf, ncell);
        dalloc(c, c.ctl, 1);
        dalloc(c, c.budget, 1);
        dalloc(c, c.partials, (size_t)NTALLY * c.max_blocks);
        dalloc(c, c.flag_dev, 1);
        GWAM_CUDA(cudaMallocHost((void**)&c.ctl_host, sizeof(Ctl)));
        GWAM_CUDA(cudaMallocHost((void**)&c.budget_host, sizeof(DevBudget)));
        GWAM_CUDA(cudaMallocHost((void**)&c.flag_host, sizeof(int)));
        GWAM_CUDA(cudaMemsetAsync(c.ctl, 0, sizeof(Ctl), c.stream));
        GWAM_CUDA(cudaMemsetAsync(c.budget, 0, sizeof(DevBudget), c.stream));
        GWAM_CUDA(cudaMemsetAsync(c.partials, 0, sizeof(double) * NTALLY * c.max_blocks, c.stream));
        configure_kernels();
        GWAM_CUDA(cudaStreamSynchronize(c.stream));
        GWAM_CUDA(cudaGetLastError());
    } catch (int code) {
        free_all(c);
        delete h;
        return code;
    }
    *out = h;
    return GWAM_OK;
}

void gwam_destroy(gwam_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->c.stream);
    free_all(ctx->c);
    delete ctx;
}

static int set_background_impl(gwam_ctx* ctx, int member, const double* u, const double* v, const double* n2,
                               const double* rho, bool host)
{
    API_BEGIN(ctx)
    if (!u || !v || !n2 || !rho) return GWAM_EINVAL;
    if (member < -1 || member >= c.G.members) return GWAM_EINVAL;
    const size_t nc = (size_t)c.G.ncell;
    const double* src[4] = {u, v, n2, rho};
    if (host) {
        // page-locked caller buffers are read by the set-up kernel directly; pageable ones are staged
        const double* mapped[4];
        bool all = true;
        for (int q = 0; q < 4; ++q) {
            mapped[q] = static_cast<const double*>(mapped_host(src[q], sizeof(double) * nc));
            all = all && mapped[q];
        }
        if (all) {
            for (int q = 0; q < 4; ++q) src[q] = mapped[q];
        } else {
            if (!c.bg_scratch) dalloc(c, c.bg_scratch, 4 * nc);
            for (int q = 0; q < 4; ++q) h2d(c, c.bg_scratch + q * nc, src[q], sizeof(double) * nc);
            for (int q = 0; q < 4; ++q) src[q] = c.bg_scratch + q * nc;
        }
    }
    const int m0 = member < 0 ? 0 : member, m1 = member < 0 ? c.G.members : member + 1;
    GWAM_CUDA(cudaMemsetAsync(c.flag_dev, 0, sizeof(int), c.stream));
    for (int m = m0; m < m1; ++m) {
        launch_set_background(c, m, src[0], src[1], src[2], src[3]);
        if (c.f32) convert_background32(c, m);
    }
    GWAM_CUDA(cudaMemcpyAsync(c.flag_host, c.flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    GWAM_CUDA(cudaGetLastError());
    if (*c.flag_host) {
        c.err = "gwam_set_background: non-finite value, rho <= 0 or N^2 <= f^2";
        for (int m = m0; m < m1; ++m) c.member_bg[m] = false;
        c.have_bg = false;
        return GWAM_ENUMERIC;
    }
    for (int m = m0; m < m1; ++m) c.member_bg[m] = true;
    c.have_bg = true;
    for (int m = 0; m < c.G.members; ++m) c.have_bg = c.have_bg && c.member_bg[m];
    API_END
}

int gwam_set_background(gwam_ctx* ctx, const double* u, const double* v, const double* n2, const double* rho)
{
    return set_background_impl(ctx, -1, u, v, n2, rho, false);
}

int gwam_set_background_host(gwam_ctx* ctx, const double* u, const double* v, const double* n2, const double* rho)
{
    return set_background_impl(ctx, -1, u, v, n2, rho, true);
}

int gwam_set_member_background(gwam_ctx* ctx, int member, const double* u, const double* v, const double* n2,
                               const double* rho)
{
    if (member < 0) return GWAM_EINVAL;
    return set_background_impl(ctx, member, u, v, n2, rho, false);
}

int gwam_set_member_background_host(gwam_ctx* ctx, int member, const double* u, const double* v, const double* n2,
                                    const double* rho)
{
    if (member < 0) return GWAM_EINVAL;
    return set_background_impl(ctx, member, u, v, n2, rho, true);
}

static int add_rays_impl(gwam_ctx* ctx, const gwam_ray_input* r, int64_t n, bool host)
{
    API_BEGIN(ctx)
    if (!r || n < 0) return GWAM_EINVAL;
    if (n == 0) return GWAM_OK;
    if (n > c.max_rays) return GWAM_ECAPACITY;
    const double* in[13] = {r->x, r->y, r->z, r->k, r->l, r->m, r->ex, r->ey, r->ez, r->dk, r->dl, r->dm, r->n};
    for (int q = 0; q < 13; ++q)
        if (!in[q]) return GWAM_EINVAL;
    double* tmp = nullptr;
    if (host) {
        GWAM_CUDA(cudaMalloc((void**)&tmp, sizeof(double) * 13 * (size_t)n));
        for (int q = 0; q < 13; ++q) {
            h2d(c, tmp + q * n, in[q], sizeof(double) * (size_t)n);
            in[q] = tmp + q * n;
        }
    }
    int rc = GWAM_OK;
    try {
        launch_add_rays(c, in, n);
        check_pending(c);
    } catch (int code) {
        rc = code;
    }
    if (tmp) {
        cudaStreamSynchronize(c.stream);
        cudaFree(tmp);
    }
    if (rc) return rc;
    API_END
}

int gwam_add_rays(gwam_ctx* ctx, const gwam_ray_input* r, int64_t n) { return add_rays_impl(ctx, r, n, false); }
int gwam_add_rays_host(gwam_ctx* ctx, const gwam_ray_input* r, int64_t n) { return add_rays_impl(ctx, r, n, true); }

static int check_ghost(gwam_ctx* ctx, double dt)
{
    if (!ctx) return GWAM_EINVAL;
    if (!(dt > 0.0) || !isfinite(dt)) return GWAM_EINVAL;
    return GWAM_OK;
}

// the ghost volume is integrated by the FP64 form's double-float RK3: a precision-form context keeps
// double-float nodes too from its first ghost-layer launch on (set-up writes them from then on)
static void ensure_bgdf(Context& c)
{
    if (c.bgdf) return;
    dalloc(c, c.bgdf, (size_t)c.G.ncell_all);
    // the second background set (asynchronous path) gets its nodes at its next set-up
    if (c.bg_alt && !c.bgdf_alt) dalloc(c, c.bgdf_alt, (size_t)c.G.ncell_all);
    for (int m = 0; m < c.G.members; ++m) node_gradients_df(c, m);
}

// ghost_dt > 0: ghost-layer emission over one launch interval
static int launch_sources_impl(gwam_ctx* ctx, const gwam_bg_source* src, double ghost_dt)
{
    API_BEGIN(ctx)
    if (!src) return GWAM_EINVAL;
    if (!c.have_bg) {
        c.err = "gwam_launch_sources: no background";
        return GWAM_ESTATE;
    }
    if (c.G.geometry != 1 || src->n_az < 1 || src->n_c < 1 || src->n_az * src->n_c > 1024) return GWAM_EINVAL;
    if (!(src->lambda_h > 0.0) || !(src->dz_launch > 0.0) || !(src->c_min > 0.0) || !(src->c_max > 0.0))
        return GWAM_EINVAL;
    if (ghost_dt > 0.0) {
        ensure_bgdf(c);
        launch_ghost_source(c, *src, ghost_dt);
    } else {
        launch_background_source(c, *src);
    }
    GWAM_CUDA(cudaGetLastError());
    API_END
}

int gwam_launch_sources(gwam_ctx* ctx, const gwam_bg_source* src) { return launch_sources_impl(ctx, src, 0.0); }

int gwam_launch_ghost(gwam_ctx* ctx, const gwam_bg_source* src, double dt)
{
    const int rc = check_ghost(ctx, dt);
    return rc ? rc : launch_sources_impl(ctx, src, dt);
}

static int launch_spectral_impl(gwam_ctx* ctx, const gwam_spec* specs, int64_t n, bool host, double ghost_dt = 0.0)
{
    API_BEGIN(ctx)
    if (n < 0 || (n > 0 && !specs)) return GWAM_EINVAL;
    if (!c.have_bg) {
        c.err = "gwam_launch_spectral: no background";
        return GWAM_ESTATE;
    }
    if (n == 0) return GWAM_OK;
    if (n >= ((int64_t)1 << 30)) return GWAM_EINVAL;
    const gwam_spec* d = specs;
    if (host) {
        for (int64_t q = 0; q < n; ++q) {
            const gwam_spec& s = specs[q];
            if (s.i < 0 || s.i >= c.G.nx || s.j < 0 || s.j >= c.G.ny || s.member < 0 || s.member >= c.G.members ||
                !(s.lambda_h > 0.0) || !(s.dz_launch > 0.0))
                return GWAM_EINVAL;
        }
        // a device copy kept between calls (per-step ghost launches from host specs do not allocate
        // or wait): the copy is ordered on the stream after the kernels that read the previous one
        if (n > c.spec_cap) {
            GWAM_CUDA(cudaStreamSynchronize(c.stream));
            if (c.spec_buf) GWAM_CUDA(cudaFree(c.spec_buf));
            c.spec_buf = nullptr;
            c.spec_cap = 0;
            GWAM_CUDA(cudaMalloc((void**)&c.spec_buf, sizeof(gwam_spec) * (size_t)n));
            c.spec_cap = n;
        }
        h2d(c, c.spec_buf, specs, sizeof(gwam_spec) * (size_t)n);
        d = c.spec_buf;
    }
    if (ghost_dt > 0.0) {
        ensure_bgdf(c);
        launch_ghost_spectral(c, d, n, ghost_dt);
    } else {
        launch_spectral(c, d, n);
    }
    GWAM_CUDA(cudaGetLastError());
    API_END
}

int gwam_launch_spectral(gwam_ctx* ctx, const gwam_spec* specs, int64_t n)
{
    return launch_spectral_impl(ctx, specs, n, false);
}

int gwam_launch_spectral_host(gwam_ctx* ctx, const gwam_spec* specs, int64_t n)
{
    return launch_spectral_impl(ctx, specs, n, true);
}

int gwam_launch_ghost_spectral(gwam_ctx* ctx, const gwam_spec* specs, int64_t n, double dt)
{
    const int rc = check_ghost(ctx, dt);
    return rc ? rc : launch_spectral_impl(ctx, specs, n, false, dt);
}

int gwam_launch_ghost_spectral_host(gwam_ctx* ctx, const gwam_spec* specs, int64_t n, double dt)
{
    const int rc = check_ghost(ctx, dt);
    return rc ? rc : launch_spectral_impl(ctx, specs, n, true, dt);
}

int gwam_step(gwam_ctx* ctx, double dt, double* dudt, double* dvdt)
{
    API_BEGIN(ctx)
    if (!(dt > 0.0) || !isfinite(dt)) return GWAM_EINVAL;
    if (!c.have_bg) {
        c.err = "gwam_step: no background";
        return GWAM_ESTATE;
    }
    run_step(c, dt, dudt, dvdt);
    GWAM_CUDA(cudaGetLastError());
    API_END
}

int gwam_step_host(gwam_ctx* ctx, double dt, double* dudt_host, double* dvdt_host)
{
    API_BEGIN(ctx)
    if (!(dt > 0.0) || !isfinite(dt)) return GWAM_EINVAL;
    if (!c.have_bg) {
        c.err = "gwam_step_host: no background";
        return GWAM_ESTATE;
    }
    const size_t bytes = sizeof(double) * (size_t)c.G.ncell_all;
    // page-locked caller buffers receive du/dt, dv/dt straight from the divergence kernel
    double* du_map = static_cast<double*>(mapped_host(dudt_host, bytes));
    double* dv_map = static_cast<double*>(mapped_host(dvdt_host, bytes));
    if (du_map && dv_map) {
        run_step(c, dt, du_map, dv_map);
    } else {
        run_step(c, dt, nullptr, nullptr);
        if (dudt_host) GWAM_CUDA(cudaMemcpyAsync(dudt_host, c.dudt_buf, bytes, cudaMemcpyDeviceToHost, c.stream));
        if (dvdt_host) GWAM_CUDA(cudaMemcpyAsync(dvdt_host, c.dvdt_buf, bytes, cudaMemcpyDeviceToHost, c.stream));
    }
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    GWAM_CUDA(cudaGetLastError());
    API_END
}

static void graph_step(Context& c, double dt, double* dudt, double* dvdt);

// ---------------------------------------------------------------- asynchronous host entry points

// page-locked host memory [p, p + bytes) (cudaHostAlloc / cudaHostRegister)
static bool page_locked(const void* p, size_t bytes)
{
    if (!p) return false;
    const char* q = static_cast<const char*>(p);
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess || cudaPointerGetAttributes(&b, q + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && b.type == cudaMemoryTypeHost;
}

static void async_setup(Context& c)
{
    if (c.up_stream) return;
    GWAM_CUDA(cudaStreamCreateWithFlags(&c.up_stream, cudaStreamNonBlocking));
    GWAM_CUDA(cudaStreamCreateWithFlags(&c.down_stream, cudaStreamNonBlocking));
    GWAM_CUDA(cudaStreamCreateWithFlags(&c.setup_stream, cudaStreamNonBlocking));
    for (int q = 0; q < 2; ++q) {
        dalloc(c, c.bg_stage[q], 4 * (size_t)c.G.ncell);
        dalloc(c, c.d_out[q], 2 * (size_t)c.G.ncell_all);
        cudaEvent_t* evs[] = {&c.ev_up[q], &c.ev_free[q], &c.ev_dready[q], &c.ev_d2h[q], &c.ev_rel[q]};
        for (cudaEvent_t* e : evs) GWAM_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    GWAM_CUDA(cudaEventCreateWithFlags(&c.ev_setup_done, cudaEventDisableTiming));
    // the second background set, shaped like the first
    const size_t nc = (size_t)c.G.ncell_all;
    dalloc(c, c.bg_alt, nc);
    dalloc(c, c.rho_alt, nc);
    dalloc(c, c.rho_inv_alt, nc);
    if (c.bgdf) dalloc(c, c.bgdf_alt, nc);
    if (c.bg32) dalloc(c, c.bg32_alt, nc);
    if (c.rho_inv32) dalloc(c, c.rho_inv32_alt, nc);
    dalloc(c, c.flag_async, 1);
}

// exchange the current and the second background set
static void swap_bg_sets(Context& c)
{
    std::swap(c.bg, c.bg_alt);
    std::swap(c.bgdf, c.bgdf_alt);
    std::swap(c.bg32, c.bg32_alt);
    std::swap(c.rho, c.rho_alt);
    std::swap(c.rho_inv, c.rho_inv_alt);
    std::swap(c.rho_inv32, c.rho_inv32_alt);
    c.cur_set ^= 1;
}

int gwam_set_background_host_async(gwam_ctx* ctx, const double* u, const double* v, const double* n2,
                                   const double* rho)
{
    API_BEGIN(ctx)
    const size_t nc = (size_t)c.G.ncell, bytes = sizeof(double) * nc;
    const double* src[4] = {u, v, n2, rho};
    for (int q = 0; q < 4; ++q)
        if (!page_locked(src[q], bytes)) {
            c.err = "gwam_set_background_host_async: the fields must be page-locked host memory";
            return GWAM_EINVAL;
        }
    async_setup(c);
    if (c.bgdf && !c.bgdf_alt) dalloc(c, c.bgdf_alt, (size_t)c.G.ncell_all);   // grown since (ghost launch)
    const int k = c.stage_k;
    c.stage_k ^= 1;
    double* st = c.bg_stage[k];
    // the copies wait until the set-up two calls back has read this slot
    GWAM_CUDA(cudaStreamWaitEvent(c.up_stream, c.ev_free[k], 0));
    for (int q = 0; q < 4; ++q)
        GWAM_CUDA(cudaMemcpyAsync(st + q * nc, src[q], bytes, cudaMemcpyHostToDevice, c.up_stream));
    GWAM_CUDA(cudaEventRecord(c.ev_up[k], c.up_stream));
    // the current set stops being current after the work issued so far; the other set is written
    // on the set-up stream once its own last readers are done, overlapping the steps in flight
    const int cur = c.cur_set;
    GWAM_CUDA(cudaEventRecord(c.ev_rel[cur], c.stream));
    GWAM_CUDA(cudaStreamWaitEvent(c.setup_stream, c.ev_up[k], 0));
    GWAM_CUDA(cudaStreamWaitEvent(c.setup_stream, c.ev_rel[cur ^ 1], 0));
    swap_bg_sets(c);
    cudaStream_t user = c.stream;
    int* flag = c.flag_dev;
    c.stream = c.setup_stream;
    c.flag_dev = c.flag_async;
    int rc = GWAM_OK;
    try {
        GWAM_CUDA(cudaMemsetAsync(c.flag_dev, 0, sizeof(int), c.stream));
        for (int m = 0; m < c.G.members; ++m) {
            launch_set_background(c, m, st, st + nc, st + 2 * nc, st + 3 * nc);
            if (c.f32) convert_background32(c, m);
        }
        GWAM_CUDA(cudaEventRecord(c.ev_free[k], c.stream));
        launch_flag_to_status(c);
        GWAM_CUDA(cudaEventRecord(c.ev_setup_done, c.stream));
    } catch (int code) {
        rc = code;
    }
    c.stream = user;
    c.flag_dev = flag;
    if (rc) return rc;
    // later work on the context's stream (the next step) waits for the new background
    GWAM_CUDA(cudaStreamWaitEvent(c.stream, c.ev_setup_done, 0));
    GWAM_CUDA(cudaGetLastError());
    for (int m = 0; m < c.G.members; ++m) c.member_bg[m] = true;
    c.have_bg = true;
    API_END
}

int gwam_step_host_async(gwam_ctx* ctx, double dt, double* dudt_host, double* dvdt_host)
{
    API_BEGIN(ctx)
    if (!(dt > 0.0) || !isfinite(dt)) return GWAM_EINVAL;
    if (!c.have_bg) {
        c.err = "gwam_step_host_async: no background";
        return GWAM_ESTATE;
    }
    const size_t n = (size_t)c.G.ncell_all, bytes = sizeof(double) * n;
    if ((dudt_host && !page_locked(dudt_host, bytes)) || (dvdt_host && !page_locked(dvdt_host, bytes))) {
        c.err = "gwam_step_host_async: du/dt, dv/dt must be page-locked host memory";
        return GWAM_EINVAL;
    }
    async_setup(c);
    const int k = c.out_k;
    c.out_k ^= 1;
    double* du = c.d_out[k];
    double* dv = du + n;
    // this slot's previous copies to the host (two calls back) must be done before it is rewritten
    GWAM_CUDA(cudaStreamWaitEvent(c.stream, c.ev_d2h[k], 0));
    graph_step(c, dt, du, dv);   // the slots alternate with the ray-buffer parity: one graph each
    GWAM_CUDA(cudaEventRecord(c.ev_dready[k], c.stream));
    GWAM_CUDA(cudaStreamWaitEvent(c.down_stream, c.ev_dready[k], 0));
    if (dudt_host) GWAM_CUDA(cudaMemcpyAsync(dudt_host, du, bytes, cudaMemcpyDeviceToHost, c.down_stream));
    if (dvdt_host) GWAM_CUDA(cudaMemcpyAsync(dvdt_host, dv, bytes, cudaMemcpyDeviceToHost, c.down_stream));
    GWAM_CUDA(cudaEventRecord(c.ev_d2h[k], c.down_stream));
    GWAM_CUDA(cudaGetLastError());
    API_END
}

// one step as a replay of the step's CUDA graph for (dt, dudt, dvdt), captured on first use per
// ray-buffer parity; throws (int) status on failure
static void graph_step(Context& c, double dt, double* dudt, double* dvdt)
{
    const int par = c.parity();
    const int gi = par + 2 * c.cur_set;   // the graph bakes in the ray buffers and the background set
    if (!c.gexec[gi] || c.gdt[gi] != dt || c.gdu[gi] != dudt || c.gdv[gi] != dvdt) {
        if (c.gexec[gi]) {
            GWAM_CUDA(cudaGraphExecDestroy(c.gexec[gi]));
            c.gexec[gi] = nullptr;
        }
        // capture one step on the internal stream; the ray buffers are swapped back afterwards.  The
        // phase boundaries become event nodes of the graph (gwam_graph_profile_read)
        GWAM_CUDA(cudaStreamSynchronize(c.stream));
        if (!c.gprof_ev[gi][0])
            for (int p = 0; p <= Context::kPhases; ++p) GWAM_CUDA(cudaEventCreate(&c.gprof_ev[gi][p]));
        const bool prof = c.prof, tune = c.tune_active;
        c.prof = false;
        c.tune_active = false;
        c.gcap_prof = true;
        c.gcap_slot = gi;
        c.glaunched[gi] = false;
        cudaStream_t user = c.stream;
        c.stream = c.cap_stream;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            run_step(c, dt, dudt, dvdt);
            e = cudaStreamEndCapture(c.cap_stream, &graph);
            // run_step swapped the ray buffers while capturing: restore the live parity
            swap_rays(c);
        }
        c.stream = user;
        c.prof = prof;
        c.tune_active = tune;
        c.gcap_prof = false;
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            c.err = std::string("graph capture: ") + cudaGetErrorString(e);
            throw (int)GWAM_ECUDA;
        }
        // the kernel nodes the graph launches per replay (gwam_graph_kernel_count)
        size_t nn = 0;
        int kern = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
                for (size_t q = 0; q < nn; ++q) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
                }
        }
        c.gkernels[gi] = kern;
        e = cudaGraphInstantiate(&c.gexec[gi], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c.gexec[gi] = nullptr;
            c.err = std::string("graph instantiate: ") + cudaGetErrorString(e);
            throw (int)GWAM_ECUDA;
        }
        c.gdt[gi] = dt;
        c.gdu[gi] = dudt;
        c.gdv[gi] = dvdt;
    }
    GWAM_CUDA(cudaGraphLaunch(c.gexec[gi], c.stream));
    c.glaunched[gi] = true;
    swap_rays(c);
}

int gwam_step_graph(gwam_ctx* ctx, double dt, double* dudt, double* dvdt)
{
    API_BEGIN(ctx)
    if (!(dt > 0.0) || !isfinite(dt)) return GWAM_EINVAL;
    if (!c.have_bg) {
        c.err = "gwam_step_graph: no background";
        return GWAM_ESTATE;
    }
    graph_step(c, dt, dudt, dvdt);
    API_END
}

int gwam_set_launch_config(gwam_ctx* ctx, int kernel, int threads, int blocks)
{
    API_BEGIN(ctx)
    if (kernel < 0 || kernel > 2 || threads < 64 || threads > kThreads || threads % 32 || blocks < 1 ||
        blocks > c.max_blocks)
        return GWAM_EINVAL;
    c.lcfg[kernel] = LaunchCfg{threads, blocks};
    for (int q = 0; q < Context::kGraphs; ++q)
        if (c.gexec[q]) {
            cudaGraphExecDestroy(c.gexec[q]);
            c.gexec[q] = nullptr;
        }
    API_END
}

int gwam_get_launch_config(gwam_ctx* ctx, int kernel, int* threads, int* blocks)
{
    API_BEGIN(ctx)
    if (kernel < 0 || kernel > 2 || !threads || !blocks) return GWAM_EINVAL;
    *threads = c.lcfg[kernel].threads;
    *blocks = c.lcfg[kernel].blocks;
    API_END
}

int gwam_autotune(gwam_ctx* ctx, double dt, int steps_per_candidate, double* dudt, double* dvdt)
{
    API_BEGIN(ctx)
    if (!(dt > 0.0) || steps_per_candidate < 1 || steps_per_candidate > Context::kTuneRing) return GWAM_EINVAL;
    if (!c.have_bg) return GWAM_ESTATE;
    if (!c.tune_ev[0][0])
        for (int q = 0; q < Context::kTuneRing; ++q)
            for (int p = 0; p < 6; ++p) GWAM_CUDA(cudaEventCreate(&c.tune_ev[q][p]));
    // candidate shapes: threads x blocks-per-SM
    const int cand_threads[] = {256, 128, 256, 128, 256, 128, 64};
    const int cand_per_sm[] = {1, 2, 2, 4, 4, 8, 8};
    const int ncand = 7;
    double best_ms[3] = {1e300, 1e300, 1e300};
    LaunchCfg best[3] = {c.lcfg[0], c.lcfg[1], c.lcfg[2]};
    for (int q = 0; q < ncand; ++q) {
        const LaunchCfg cfg{cand_threads[q], std::min(c.max_blocks, c.num_sms * cand_per_sm[q])};
        for (int k = 0; k < 3; ++k) c.lcfg[k] = cfg;
        c.tune_active = true;
        c.tune_pending = 0;
        for (int st = 0; st < steps_per_candidate; ++st) run_step(c, dt, dudt, dvdt);
        c.tune_active = false;
        GWAM_CUDA(cudaStreamSynchronize(c.stream));
        GWAM_CUDA(cudaGetLastError());
        double ms[3] = {0.0, 0.0, 0.0};
        for (int st = 0; st < c.tune_pending; ++st)
            for (int k = 0; k < 3; ++k) {
                float v = 0.0f;
                GWAM_CUDA(cudaEventElapsedTime(&v, c.tune_ev[st][2 * k], c.tune_ev[st][2 * k + 1]));
                ms[k] += v;
            }
        for (int k = 0; k < 3; ++k)
            if (ms[k] < best_ms[k]) {
                best_ms[k] = ms[k];
                best[k] = cfg;
            }
    }
    for (int k = 0; k < 3; ++k) c.lcfg[k] = best[k];
    for (int q = 0; q < Context::kGraphs; ++q)
        if (c.gexec[q]) {
            cudaGraphExecDestroy(c.gexec[q]);
            c.gexec[q] = nullptr;
        }
    API_END
}

int gwam_num_rays(gwam_ctx* ctx, int64_t* n)
{
    API_BEGIN(ctx)
    if (!n) return GWAM_EINVAL;
    check_pending(c);
    *n = c.ctl_host->n;
    API_END
}

int gwam_get_rays_host(gwam_ctx* ctx, double* state13, int64_t* ids, int32_t* cells, int64_t cap)
{
    API_BEGIN(ctx)
    check_pending(c);
    const int64_t n = c.ctl_host->n;
    if (cap < n) return GWAM_ECAPACITY;
    if (n == 0) return GWAM_OK;
    double* tmp = nullptr;
    long long* tid = nullptr;
    int* tcell = nullptr;
    GWAM_CUDA(cudaMalloc((void**)&tmp, sizeof(double) * 13 * (size_t)n));
    GWAM_CUDA(cudaMalloc((void**)&tid, sizeof(long long) * (size_t)n));
    GWAM_CUDA(cudaMalloc((void**)&tcell, sizeof(int) * (size_t)n));
    if (c.f32)
        launch_gather_rays32(c, tmp, tid, tcell, n);
    else
        launch_gather_rays(c, tmp, tid, tcell, n);
    for (int q = 0; q < 13 && state13; ++q)
        GWAM_CUDA(cudaMemcpyAsync(state13 + q * cap, tmp + q * n, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                                  c.stream));
    if (ids) GWAM_CUDA(cudaMemcpyAsync(ids, tid, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToHost, c.stream));
    if (cells) GWAM_CUDA(cudaMemcpyAsync(cells, tcell, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    cudaFree(tmp);
    cudaFree(tid);
    cudaFree(tcell);
    API_END
}

int gwam_get_stats(gwam_ctx* ctx, gwam_stats* out)
{
    API_BEGIN(ctx)
    if (!out) return GWAM_EINVAL;
    check_pending(c);
    const Ctl& t = *c.ctl_host;
    const DevBudget& b = *c.budget_host;
    out->n_live = t.n;
    out->n_launched = t.n_launched;
    out->n_filtered = t.n_filtered;
    out->n_split_v = t.n_split_v;
    out->n_split_h = t.n_split_h;
    out->n_exited = t.n_exited;
    out->n_capped = t.n_capped;
    out->n_merged = 0;
    out->n_invalid = t.n_invalid;
    out->n_steps = t.n_steps;
    out->ray_steps = t.ray_steps;
    out->w_total = b.w_total;
    out->w_launched = b.w_launched;
    out->w_saturated = b.w_saturated;
    out->w_exited = b.w_exited;
    out->w_capped = b.w_capped;
    out->w_invalid = b.w_invalid;
    API_END
}

int gwam_get_field_host(gwam_ctx* ctx, int which, double* out_host)
{
    API_BEGIN(ctx)
    if (which < 0 || which >= NFIELD || !out_host) return GWAM_EINVAL;
    if (c.P.smoothing) {
        if (c.f32) smooth_field32(c, which);
        else smooth_field(c, which);
    }
    const double* src = c.P.smoothing ? c.smooth[which] : c.field[which];
    const int nlev = which <= F_ZP ? c.G.nz + 1 : c.G.nz;
    double* tmp = nullptr;
    GWAM_CUDA(cudaMalloc((void**)&tmp, sizeof(double) * (size_t)c.field_len(which)));
    launch_field_to_caller(c, src, tmp, nlev);
    GWAM_CUDA(cudaMemcpyAsync(out_host, tmp, sizeof(double) * (size_t)c.field_len(which), cudaMemcpyDeviceToHost,
                              c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    cudaFree(tmp);
    API_END
}

int gwam_set_theta(gwam_ctx* ctx, const double* theta)
{
    API_BEGIN(ctx)
    if (!theta) return GWAM_EINVAL;
    if (!c.theta) dalloc(c, c.theta, (size_t)c.G.ncell_all);
    GWAM_CUDA(cudaMemsetAsync(c.flag_dev, 0, sizeof(int), c.stream));
    launch_set_theta(c, theta);
    GWAM_CUDA(cudaMemcpyAsync(c.flag_host, c.flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    GWAM_CUDA(cudaGetLastError());
    if (*c.flag_host) {
        c.err = "gwam_set_theta: theta must be positive and finite";
        cudaFree(c.theta);
        c.theta = nullptr;
        return GWAM_ENUMERIC;
    }
    API_END
}

int gwam_get_theta_tendency_host(gwam_ctx* ctx, double* out_host)
{
    API_BEGIN(ctx)
    if (!out_host) return GWAM_EINVAL;
    if (!c.P.theta_flux || !c.theta || !c.have_bg) {
        c.err = "gwam_get_theta_tendency_host: needs theta_flux = 1, gwam_set_theta and a background";
        return GWAM_ESTATE;
    }
    check_pending(c);
    const double* tl = c.field[F_TL];
    const double* tp = c.field[F_TP];
    if (c.P.smoothing) {
        smooth_field(c, F_TL);
        smooth_field(c, F_TP);
        tl = c.smooth[F_TL];
        tp = c.smooth[F_TP];
    }
    double* tmp = nullptr;
    GWAM_CUDA(cudaMalloc((void**)&tmp, sizeof(double) * (size_t)c.G.ncell_all));
    launch_theta_div(c, tl, tp, tmp);
    GWAM_CUDA(cudaMemcpyAsync(out_host, tmp, sizeof(double) * (size_t)c.G.ncell_all, cudaMemcpyDeviceToHost,
                              c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    cudaFree(tmp);
    API_END
}

int gwam_get_gamma2_host(gwam_ctx* ctx, double* out_host)
{
    API_BEGIN(ctx)
    if (!out_host) return GWAM_EINVAL;
    double* tmp = nullptr;
    GWAM_CUDA(cudaMalloc((void**)&tmp, sizeof(double) * (size_t)c.G.ncell_all));
    launch_gamma_to_caller(c, tmp);
    GWAM_CUDA(cudaMemcpyAsync(out_host, tmp, sizeof(double) * (size_t)c.G.ncell_all, cudaMemcpyDeviceToHost,
                              c.stream));
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    cudaFree(tmp);
    API_END
}

// ------------------------------------------------------------------------------ checkpoints
// File layout: CkptHeader, one byte per member (background set), the ray arrays of the canonical
// order (FP64 form: 7 x n double2; precision form: 4 x n float4), then, when a background is set,
// the FP64 nodes [members * ncell] and rho [members * ncell].  Host byte order.
namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t precision, geometry, nx, ny, nz, members;
    int32_t gamma_mode, saturation, smoothing, flux_form, splitting, cap, columnar, theta_flux;
    double dX, dY, dz, radius, omega, f0, g, alpha_s, min_split_dz;
    int64_t n;
    int32_t have_bg, pad;
    Ctl ctl;
    DevBudget budget;
};
constexpr char kCkptMagic[8] = {'G', 'W', 'A', 'M', 'C', 'K', 'P', '1'};

void fill_header(const Context& c, CkptHeader& h)
{
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.header_bytes = sizeof(CkptHeader);
    h.precision = c.f32 ? 1 : 0;
    h.geometry = c.G.geometry;
    h.nx = c.G.nx;
    h.ny = c.G.ny;
    h.nz = c.G.nz;
    h.members = c.G.members;
    h.gamma_mode = c.P.gamma_mode;
    h.saturation = c.P.saturation;
    h.smoothing = c.P.smoothing;
    h.flux_form = c.P.flux_form;
    h.splitting = c.P.splitting;
    h.cap = c.P.cap;
    h.columnar = c.G.columnar;
    h.theta_flux = c.P.theta_flux;
    h.dX = c.G.dX;
    h.dY = c.G.dY;
    h.dz = c.G.dz;
    h.radius = c.G.radius;
    h.omega = c.G.omega;
    h.f0 = c.G.f0;
    h.g = c.G.g;
    h.alpha_s = c.P.alpha_s;
    h.min_split_dz = c.P.min_split_dz;
}

// the configuration fields of two headers agree (everything but the state)
bool same_config(const CkptHeader& a, const CkptHeader& b)
{
    return memcmp(a.magic, b.magic, 8) == 0 && a.version == b.version && a.header_bytes == b.header_bytes &&
           a.precision == b.precision && a.geometry == b.geometry && a.nx == b.nx && a.ny == b.ny && a.nz == b.nz &&
           a.members == b.members && a.gamma_mode == b.gamma_mode && a.saturation == b.saturation &&
           a.smoothing == b.smoothing && a.flux_form == b.flux_form && a.splitting == b.splitting &&
           a.cap == b.cap && a.columnar == b.columnar && a.theta_flux == b.theta_flux && a.dX == b.dX && a.dY == b.dY && a.dz == b.dz && a.radius == b.radius &&
           a.omega == b.omega && a.f0 == b.f0 && a.g == b.g && a.alpha_s == b.alpha_s &&
           a.min_split_dz == b.min_split_dz;
}

struct FileCloser {
    FILE* f;
    ~FileCloser()
    {
        if (f) fclose(f);
    }
};
}  // namespace

int gwam_save(gwam_ctx* ctx, const char* path)
{
    API_BEGIN(ctx)
    if (!path) return GWAM_EINVAL;
    check_pending(c);
    CkptHeader h;
    fill_header(c, h);
    h.n = c.ctl_host->n;
    h.have_bg = c.have_bg ? 1 : 0;
    h.ctl = *c.ctl_host;
    h.budget = *c.budget_host;
    const size_t n = (size_t)h.n;
    const size_t nc = (size_t)c.G.ncell_all;
    // device -> host first, so that a failed copy leaves no partial file
    std::vector<unsigned char> rays(n * (c.f32 ? 4 * sizeof(float4) : 7 * sizeof(double2)));
    for (int q = 0; q < (c.f32 ? 4 : 7) && n; ++q) {
        const size_t bytes = n * (c.f32 ? sizeof(float4) : sizeof(double2));
        const void* src = c.f32 ? (const void*)c.A32.q[q] : (const void*)c.A.a[q];
        GWAM_CUDA(cudaMemcpyAsync(rays.data() + q * bytes, src, bytes, cudaMemcpyDeviceToHost, c.stream));
    }
    std::vector<Node> nodes;
    std::vector<double> rho;
    if (h.have_bg) {
        nodes.resize(nc);
        rho.resize(nc);
        GWAM_CUDA(cudaMemcpyAsync(nodes.data(), c.bg, sizeof(Node) * nc, cudaMemcpyDeviceToHost, c.stream));
        GWAM_CUDA(cudaMemcpyAsync(rho.data(), c.rho, sizeof(double) * nc, cudaMemcpyDeviceToHost, c.stream));
    }
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    std::vector<unsigned char> flags(c.G.members);
    for (int m = 0; m < c.G.members; ++m) flags[m] = c.member_bg[m] ? 1 : 0;
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) {
        c.err = "gwam_save: cannot open the file for writing";
        return GWAM_EINVAL;
    }
    bool ok = fwrite(&h, sizeof(h), 1, fc.f) == 1 && fwrite(flags.data(), 1, flags.size(), fc.f) == flags.size() &&
              (rays.empty() || fwrite(rays.data(), 1, rays.size(), fc.f) == rays.size());
    if (ok && h.have_bg)
        ok = fwrite(nodes.data(), sizeof(Node), nc, fc.f) == nc && fwrite(rho.data(), sizeof(double), nc, fc.f) == nc;
    if (!ok) {
        c.err = "gwam_save: write failed";
        return GWAM_EINVAL;
    }
    API_END
}

int gwam_load(gwam_ctx* ctx, const char* path)
{
    API_BEGIN(ctx)
    if (!path) return GWAM_EINVAL;
    check_pending(c);
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) {
        c.err = "gwam_load: cannot open the file";
        return GWAM_EINVAL;
    }
    CkptHeader h, mine;
    fill_header(c, mine);
    if (fread(&h, sizeof(h), 1, fc.f) != 1 || !same_config(h, mine)) {
        c.err = "gwam_load: not a checkpoint of this grid, parameters and precision";
        return GWAM_EINVAL;
    }
    if (h.n < 0 || h.n > c.max_rays || h.ctl.n != h.n || h.ctl.status != 0) {
        c.err = "gwam_load: ray count beyond max_rays or inconsistent header";
        return h.n > c.max_rays ? GWAM_ECAPACITY : GWAM_EINVAL;
    }
    const size_t n = (size_t)h.n;
    const size_t nc = (size_t)c.G.ncell_all;
    std::vector<unsigned char> flags(c.G.members);
    std::vector<unsigned char> rays(n * (c.f32 ? 4 * sizeof(float4) : 7 * sizeof(double2)));
    bool ok = fread(flags.data(), 1, flags.size(), fc.f) == flags.size() &&
              (rays.empty() || fread(rays.data(), 1, rays.size(), fc.f) == rays.size());
    std::vector<Node> nodes;
    std::vector<double> rho;
    if (ok && h.have_bg) {
        nodes.resize(nc);
        rho.resize(nc);
        ok = fread(nodes.data(), sizeof(Node), nc, fc.f) == nc && fread(rho.data(), sizeof(double), nc, fc.f) == nc;
    }
    if (!ok) {
        c.err = "gwam_load: truncated checkpoint";
        return GWAM_EINVAL;
    }
    for (int q = 0; q < (c.f32 ? 4 : 7) && n; ++q) {
        const size_t bytes = n * (c.f32 ? sizeof(float4) : sizeof(double2));
        void* dst = c.f32 ? (void*)c.A32.q[q] : (void*)c.A.a[q];
        GWAM_CUDA(cudaMemcpyAsync(dst, rays.data() + q * bytes, bytes, cudaMemcpyHostToDevice, c.stream));
    }
    *c.ctl_host = h.ctl;
    *c.budget_host = h.budget;
    GWAM_CUDA(cudaMemcpyAsync(c.ctl, c.ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c.stream));
    GWAM_CUDA(cudaMemcpyAsync(c.budget, c.budget_host, sizeof(DevBudget), cudaMemcpyHostToDevice, c.stream));
    if (h.have_bg) {
        GWAM_CUDA(cudaMemcpyAsync(c.bg, nodes.data(), sizeof(Node) * nc, cudaMemcpyHostToDevice, c.stream));
        GWAM_CUDA(cudaMemcpyAsync(c.rho, rho.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, c.stream));
        for (int m = 0; m < c.G.members; ++m)
            if (flags[m]) {
                restore_background(c, m);
                if (c.f32) convert_background32(c, m);
            }
    }
    for (int m = 0; m < c.G.members; ++m) c.member_bg[m] = h.have_bg && flags[m];
    c.have_bg = h.have_bg != 0;
    for (int m = 0; m < c.G.members; ++m) c.have_bg = c.have_bg && c.member_bg[m];
    for (int q = 0; q < Context::kGraphs; ++q)
        if (c.gexec[q]) {
            cudaGraphExecDestroy(c.gexec[q]);
            c.gexec[q] = nullptr;
        }
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    GWAM_CUDA(cudaGetLastError());
    API_END
}

int gwam_synchronize(gwam_ctx* ctx)
{
    API_BEGIN(ctx)
    check_pending(c);
    API_END
}

int gwam_profile_enable(gwam_ctx* ctx, int enable)
{
    API_BEGIN(ctx)
    if (enable && !c.prof_ev[0][0]) {
        for (int q = 0; q < Context::kRing; ++q)
            for (int p = 0; p <= Context::kPhases; ++p) GWAM_CUDA(cudaEventCreate(&c.prof_ev[q][p]));
    }
    if (c.prof) prof_harvest(c);
    c.prof = enable != 0;
    c.prof_pending = 0;
    c.prof_steps = 0;
    for (int p = 0; p < Context::kPhases; ++p) c.prof_ms[p] = 0.0;
    API_END
}

int gwam_profile_read(gwam_ctx* ctx, double* ms_host, int64_t* steps)
{
    API_BEGIN(ctx)
    if (!ms_host || !steps) return GWAM_EINVAL;
    prof_harvest(c);
    for (int p = 0; p < Context::kPhases; ++p) ms_host[p] = c.prof_ms[p];
    *steps = c.prof_steps;
    API_END
}

int gwam_graph_profile_read(gwam_ctx* ctx, double* ms_host, int* replays)
{
    API_BEGIN(ctx)
    if (!ms_host || !replays) return GWAM_EINVAL;
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    for (int p = 0; p < Context::kPhases; ++p) ms_host[p] = 0.0;
    int n = 0;
    for (int gi = 0; gi < Context::kGraphs; ++gi) {
        if (!c.glaunched[gi] || !c.gprof_ev[gi][0]) continue;
        for (int p = 0; p < Context::kPhases; ++p) {
            float ms = 0.0f;
            GWAM_CUDA(cudaEventElapsedTime(&ms, c.gprof_ev[gi][p], c.gprof_ev[gi][p + 1]));
            ms_host[p] += ms;
        }
        ++n;
    }
    for (int p = 0; p < Context::kPhases; ++p) ms_host[p] = n ? ms_host[p] / n : 0.0;
    *replays = n;
    API_END
}

int gwam_selftest_scan(gwam_ctx* ctx, const int32_t* in0, int32_t* out0, int64_t n0, const int32_t* in1,
                       int32_t* out1, int64_t n1)
{
    API_BEGIN(ctx)
    if (!in0 || !out0 || n0 < 0 || n0 > INT32_MAX - 1 || (in1 && (!out1 || n1 < 0 || n1 > INT32_MAX - 1)))
        return GWAM_EINVAL;
    if (in1) exclusive_scan2(c, in0, out0, n0, nullptr, in1, out1, n1, nullptr);
    else exclusive_scan(c, in0, out0, n0, nullptr);
    GWAM_CUDA(cudaStreamSynchronize(c.stream));
    GWAM_CUDA(cudaGetLastError());
    API_END
}

int gwam_graph_kernel_count(gwam_ctx* ctx, int* kernels)
{
    API_BEGIN(ctx)
    if (!kernels) return GWAM_EINVAL;
    int k = 0;
    for (int gi = 0; gi < Context::kGraphs; ++gi)
        if (c.gexec[gi]) k = std::max(k, c.gkernels[gi]);
    *kernels = k;
    API_END
}

const char* gwam_last_error(const gwam_ctx* ctx)
{
    if (!ctx) return "null context";
    return ctx->c.err.c_str();
}

}  // extern "C"
