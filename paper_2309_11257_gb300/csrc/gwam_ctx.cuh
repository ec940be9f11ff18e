// gwam_ctx.cuh -- the context behind the C ABI: device buffers and kernel entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gwam.h"
#include "gwam_device.cuh"

namespace gwam {

// Device control block: counts the host never needs to read inside a step.
struct Ctl {
    int n;               // live ray volumes (array A)
    int n_new;           // ray volumes after this step's re-binning
    int n_children;      // children produced this step (before the cap)
    int n_over;          // columns above the cap this step
    int n_big;           // length of the saturation run list
    int status;          // sticky device status (gwam_status values)
    long long next_id;   // next unused ray id
    long long new_ids;   // ids issued this step
    // cumulative counters
    long long n_launched, n_filtered, n_split_v, n_split_h, n_exited, n_capped, n_invalid, n_steps, ray_steps;
};

// FP64 tallies are reduced deterministically: every kernel that produces one writes one
// partial per block (fixed grid) into its slot; a single-block kernel folds them in order.
enum TallySlot { T_EXIT, T_INVALID, T_CAP, T_SAT, T_LAUNCH, T_TOTAL, NTALLY };

struct DevBudget {
    double w_total, w_launched, w_saturated, w_exited, w_capped, w_invalid;
};

// F_TL, F_TP: the potential-temperature flux integrals (projected only with Params.theta_flux)
enum FieldId { F_ZL, F_ZP, F_LL, F_LP, F_PL, F_PP, F_EL, F_EP, F_WAD, F_TL, F_TP, NFIELD };

struct LaunchCfg {
    int threads, blocks;
};

struct Context {
    int device = 0;
    int num_sms = 0;
    int grid_blocks = 0;            // persistent grid of the lighter ray kernels
    int max_blocks = 0;             // largest grid of a tally-producing kernel (partial-sum stride)
    LaunchCfg lcfg[3] = {};         // advance, materialise, projection (autotuned)
    cudaStream_t stream = nullptr;
    Grid G{};
    Params P{};
    int64_t max_rays = 0;
    bool have_bg = false;
    std::string err;

    // background (column-major)
    Node* bg = nullptr;          // U V N2 G2 per node
    double* rho = nullptr;          // rho per node
    double* rho_inv = nullptr;      // 1 / rho per node
    double* theta = nullptr;        // reference potential temperature per node (gwam_set_theta)
    double* tables = nullptr;       // row_cos[ny], row_inv_cos[ny], lev_inv_r[nz]
    float* tables32 = nullptr;      // row_cos32[ny], whf32[ny], ivol32[ny * nz]
    float2* tables_df = nullptr;    // row_cos, row_inv_cos [ny], lev_inv_r [nz] as double-float pairs
    double* bg_scratch = nullptr;   // staging of caller fields ([nz][ny][nx], 4 fields)
    gwam_spec* spec_buf = nullptr;  // device copy of host spectral launches (grown, kept)
    int64_t spec_cap = 0;

    // ray volumes: A holds the canonical array between steps, B is the re-binned output
    bool f32 = false;               // precision form: FP32 records and background
    RaySoA A{}, B{};
    double2* ray_mem[2] = {nullptr, nullptr};
    Ray32SoA A32{}, B32{};
    float4* ray32_mem[2] = {nullptr, nullptr};
    Node32* bg32 = nullptr;
    NodeDF* bgdf = nullptr;         // FP64 form: the background as double-float pairs (per-step gathers);
                                    // precision form: allocated by its first ghost-layer launch

    // per-ray scratch
    int* info = nullptr;            // split code | children << 4 | status << 8
    int4* ccell = nullptr;          // child cells (-1 = left the domain)
    int4* cslot = nullptr;          // child slot inside its cell
    int* newid = nullptr;           // ids needed per ray -> exclusive prefix
    long long* ent_id = nullptr;    // entry id (in cell-offset order)
    int* ent_src = nullptr;         // entry source: parent * 4 + child, < 0 removed by the cap
    int* ent_cell = nullptr;        // entry cell (global)
    int* sorted_src = nullptr;      // entry source in canonical order
    double* pj = nullptr;           // saturation: P_j (incl. alpha_j)
    double* k2 = nullptr;           // saturation: K_j^2
    double* kappa = nullptr;        // saturation: kappa of the carrier cell, per ray
    int* raycell = nullptr;         // global cell of every ray in the canonical array
    double* ecap = nullptr;         // cap: energies of the entries of over-full columns

    // per-cell scratch
    int* cnt = nullptr;             // entries per cell (then live entries per cell)
    int* off = nullptr;             // exclusive prefix of cnt (ncell + 1)
    int* off2 = nullptr;            // exclusive prefix after the cap (ncell + 1)
    int* overlist = nullptr;        // columns above the cap
    int* biglist = nullptr;         // saturation run list: the cell of every run of equal cells
    int* scan_tmp = nullptr;        // block sums of the scans
    int64_t scan_tmp_cap = 0;

    // grid fields (column-major; interface fields [col][nz+1])
    double* field[NFIELD] = {};
    double* smooth[NFIELD] = {};
    // precision form: FP32 copies of the projected fields (narrowed once per step), their smoothed
    // versions and 1 / rho (narrowed when the background is set)
    float* nar32[NFIELD] = {};
    float* sm32[NFIELD] = {};
    float* rho_inv32 = nullptr;
    double* dudt_buf = nullptr;     // [nz][ny][nx]
    double* dvdt_buf = nullptr;

    // control, tallies
    Ctl* ctl = nullptr;
    DevBudget* budget = nullptr;
    double* partials = nullptr;     // NTALLY * grid_blocks
    Ctl* ctl_host = nullptr;        // pinned mirror
    DevBudget* budget_host = nullptr;
    int* flag_dev = nullptr;        // validation flags
    int* flag_host = nullptr;

    // per-phase timing: a ring of event sets, harvested on read (or when the ring is full)
    static constexpr int kPhases = 5;
    static constexpr int kRing = 128;
    bool prof = false;
    cudaEvent_t prof_ev[kRing][kPhases + 1] = {};
    // the same phase boundaries recorded by the step graphs themselves (one set per graph; each
    // replay overwrites its set), read by gwam_graph_profile_read
    static constexpr int kGraphs = 4;   // ray-buffer parity x background set
    cudaEvent_t gprof_ev[kGraphs][kPhases + 1] = {};
    bool gcap_prof = false;     // capturing: prof_mark records into gprof_ev[gcap_slot]
    int gcap_slot = 0;
    bool glaunched[kGraphs] = {};
    int gkernels[kGraphs] = {};  // kernel nodes of each captured step graph
    int prof_pending = 0;
    int64_t prof_steps = 0;
    double prof_ms[kPhases] = {};

    // asynchronous host entry points: one stream for uploads and one for downloads over the host
    // link (a single in-order copy stream would hold the next upload behind the download that waits
    // for the current step), two device staging slots for the background and two for du/dt, dv/dt,
    // with events ordering slot reuse
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    double* bg_stage[2] = {nullptr, nullptr};   // [4][ncell] each
    double* d_out[2] = {nullptr, nullptr};      // [2][ncell_all] each: du/dt then dv/dt
    cudaEvent_t ev_up[2] = {}, ev_free[2] = {}, ev_dready[2] = {}, ev_d2h[2] = {};
    int stage_k = 0, out_k = 0;

    // second background set of the asynchronous host path (allocated on first use): the set-up of
    // the next background writes it on its own stream while the current step reads the other, and
    // the two are swapped; events order the writes after the last reads
    Node* bg_alt = nullptr;
    NodeDF* bgdf_alt = nullptr;
    Node32* bg32_alt = nullptr;
    double* rho_alt = nullptr;
    double* rho_inv_alt = nullptr;
    float* rho_inv32_alt = nullptr;
    int cur_set = 0;                // which physical set the pointers above name as current
    cudaStream_t setup_stream = nullptr;
    cudaEvent_t ev_rel[2] = {};     // set s no longer read (recorded when it stops being current)
    cudaEvent_t ev_setup_done = nullptr;
    int* flag_async = nullptr;      // validation flag of the asynchronous set-up

    // CUDA graphs of the step, one per (ray-buffer parity, background set), keyed by (dt, dudt, dvdt)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[kGraphs] = {};
    double gdt[kGraphs] = {};
    double* gdu[kGraphs] = {};
    double* gdv[kGraphs] = {};
    std::vector<bool> member_bg;

    // autotuning: event sets around the three heavy kernels, one per step
    static constexpr int kTuneRing = 64;
    bool tune_active = false;
    int tune_pending = 0;
    cudaEvent_t tune_ev[kTuneRing][6] = {};

    // exchange the canonical and the re-binned ray buffers of whichever form the context uses
    void swap_rays_()
    {
        if (f32) {
            Ray32SoA t = A32;
            A32 = B32;
            B32 = t;
        } else {
            RaySoA t = A;
            A = B;
            B = t;
        }
    }
    int parity() const { return f32 ? (A32.q[0] == ray32_mem[0] ? 0 : 1) : (A.a[0] == ray_mem[0] ? 0 : 1); }
    int64_t field_len(int f) const { return (int64_t)G.ncol_all * (f <= F_ZP ? G.nz + 1 : G.nz); }
};

// kernels, launched from the host side (gwam_step.cu / gwam_launch.cu)
// reference potential temperature (caller layout -> column-major) and the theta tendency of the
// last step's T fields into the caller layout
void launch_set_theta(Context& c, const double* theta);
void launch_theta_div(Context& c, const double* tl, const double* tp, double* out);
// derived background arrays (1/rho, gradients, gather copies) from restored nodes and rho
void restore_background(Context& c, int member);
void launch_set_background(Context& c, int member, const double* u, const double* v, const double* n2,
                           const double* rho);
void launch_add_rays(Context& c, const double* const in[13], int64_t n);
void launch_background_source(Context& c, const gwam_bg_source& src);
void launch_spectral(Context& c, const gwam_spec* specs, int64_t n);
void launch_ghost_source(Context& c, const gwam_bg_source& src, double dt);
void launch_flag_to_status(Context& c);
void node_gradients_df(Context& c, int member);
void launch_ghost_spectral(Context& c, const gwam_spec* specs, int64_t n, double dt);
void run_step(Context& c, double dt, double* du, double* dv);
void configure_kernels();
void smooth_field(Context& c, int f);
void smooth_field32(Context& c, int f);
void grid_phase_df(Context& c, double* du, double* dv, int mask);
inline void swap_rays(Context& c) { c.swap_rays_(); }
void run_step32(Context& c, double dt, double* du, double* dv);
void convert_background32(Context& c, int member);
void launch_gather_rays32(Context& c, double* state13, long long* ids, int* cells, int64_t n);
void prof_mark(Context& c, int phase);
void tune_mark(Context& c, int idx);
void prof_harvest(Context& c);
void launch_gather_rays(Context& c, double* state13, long long* ids, int* cells, int64_t cap);
void launch_field_to_caller(Context& c, const double* src, double* dst, int nlev);
void launch_gamma_to_caller(Context& c, double* dst);
void exclusive_scan(Context& c, const int* in, int* out, int64_t n, const int* n_dev);
// two independent exclusive scans in one pair of launches
void exclusive_scan2(Context& c, const int* in0, int* out0, int64_t n0, const int* n_dev0, const int* in1,
                     int* out1, int64_t n1, const int* n_dev1);
int scan_block_count(int64_t n);
// histogram of the cells + exclusive scan (the two offsets entry points); each launch's own status
cudaError_t launch_cell_offsets(const int32_t* cells, int64_t n, int32_t ncell, int* counts, int* scratch, int* flag,
                                cudaStream_t s);
void finalize_tallies(Context& c, int slot_mask, int mode);

}  // namespace gwam
