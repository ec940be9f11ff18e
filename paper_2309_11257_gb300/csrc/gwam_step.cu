// gwam_step.cu -- one ray-volume step of the FP64 form on the device.
//
// Order inside a step (the paper leaves it open; this is the reading taken):
//   advance (RK3, App. B.2) -> exits -> split (App. B.3) -> re-bin by cell (parent-cell
//   storage, App. B.2) -> per-column cap (App. B.5) -> saturation (Sec. 3c) -> projection
//   (Sec. 3b, Eq. fluxes:momentum, Eq. fluxes:buoyancy) -> smoothing (App. B.4) ->
//   divergence (Eq. mean-flow-impact) -> wave-action budget (Sec. 4).
//
// Kernels read the live count from device memory, so a whole step is enqueued without a
// host synchronisation.  Ray kernels run a fixed persistent grid so that the per-block FP64
// partial sums, folded in a fixed order, are deterministic.
#include <algorithm>

#include "gwam_common.cuh"

namespace gwam {

// ============================================================================ scans

// Three-kernel exclusive scan (block sums, their scan, the blocks) of the offsets entry points
// (launch_cell_offsets), whose scratch is sized by scan_block_count; the step's own scans are the
// two-pass part scans below.
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ __forceinline__ int scan_len(int64_t n, const int* n_dev) { return n_dev ? *n_dev : (int)n; }

__global__ void k_scan_reduce(const int* __restrict__ in, int64_t n, const int* n_dev, int* __restrict__ bsum)
{
    const int len = scan_len(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
    for (int q = threadIdx.x; q < kScanTile; q += kThreads) {
        int64_t i = base + q;
        if (i < len) s += in[i];
    }
    long long t = block_sum(s);
    if (threadIdx.x == 0) bsum[blockIdx.x] = (int)t;
}

__global__ void k_scan_blocks(int* bsum, int nb)
{
    // single block: exclusive scan of nb block sums in chunks of 1024; total into bsum[nb]
    __shared__ int sh[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {
            int o = threadIdx.x >= d ? sh[threadIdx.x - d] : 0;
            __syncthreads();
            sh[threadIdx.x] += o;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_apply(const int* in, int* out, int64_t n, const int* n_dev, const int* __restrict__ bsum,
                             int nb)
{
    __shared__ int tile[kScanTile];
    __shared__ int wsum[kThreads / 32];
    const int len = scan_len(n, n_dev);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int q = threadIdx.x; q < kScanTile; q += kThreads) {
        int64_t i = base + q;
        tile[q] = i < len ? in[i] : 0;
    }
    __syncthreads();
    int loc[kScanItems];
    int run = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        loc[q] = run;
        run += tile[threadIdx.x * kScanItems + q];
    }
    // exclusive scan of the thread totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = lane < kThreads / 32 ? wsum[lane] : 0;
        int iv = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, iv, d);
            if (lane >= d) iv += o;
        }
        if (lane < kThreads / 32) wsum[lane] = iv - v;
    }
    __syncthreads();
    const int offset = bsum[blockIdx.x] + wsum[wid] + incl - run;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) tile[threadIdx.x * kScanItems + q] = offset + loc[q];
    __syncthreads();
    for (int q = threadIdx.x; q < kScanTile; q += kThreads) {
        int64_t i = base + q;
        if (i < len) out[i] = tile[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[len] = bsum[nb];
}

int scan_block_count(int64_t n) { return (int)((n + kScanTile - 1) / kScanTile) + 1; }

// The step's scans: two passes over at most two contiguous parts per SM.  k_part_sums sums each
// part; k_part_scan adds up the sums of the parts before its own and scans its part tile by tile
// (one int4 of items per thread, warp shuffles, a carry across tiles).  Few, long parts instead of
// one block per 2048 items: no third kernel to scan the block sums, and no launch of ~1400 blocks.
// Both passes take kPartGroup tiles at a time with all their loads issued first (one tile at a
// time left a single 16-byte load per thread in flight, about half the HBM rate), and the scan
// combines the group's tiles in one block-wide step (the warps' scans interleaved, two barriers per
// group).
constexpr int kPartTile = 4 * kThreads;
constexpr int kPartGroup = 4;

__device__ __forceinline__ int64_t part_chunk(int len, int nparts)
{
    const int64_t per = ((int64_t)len + nparts - 1) / nparts;
    return (per + kPartTile - 1) / kPartTile * kPartTile;
}

// items i .. i + 3 of a part ending at b (zeros past b): one 16-byte load when aligned and whole
__device__ __forceinline__ int4 load4(const int* in, int64_t i, int64_t b, bool vec)
{
    if (vec && i + 3 < b) return *reinterpret_cast<const int4*>(in + i);
    int4 v = make_int4(0, 0, 0, 0);
    if (i < b) v.x = in[i];
    if (i + 1 < b) v.y = in[i + 1];
    if (i + 2 < b) v.z = in[i + 2];
    if (i + 3 < b) v.w = in[i + 3];
    return v;
}

__device__ __forceinline__ void store4(int* out, int64_t i, int64_t b, bool vec, int4 r)
{
    if (vec && i + 3 < b) {
        *reinterpret_cast<int4*>(out + i) = r;
        return;
    }
    if (i < b) out[i] = r.x;
    if (i + 1 < b) out[i + 1] = r.y;
    if (i + 2 < b) out[i + 2] = r.z;
    if (i + 3 < b) out[i + 3] = r.w;
}

// One scan of the launch: in[0..len) -> out, len = *n_dev if given (n its upper bound), its part
// sums in psum[0..nparts).  A launch runs one or two independent scans, the second one's parts in
// the blocks after the first one's.
struct ScanJob {
    const int* in;
    int* out;
    int64_t n;
    const int* n_dev;
    int* psum;
    int nparts;
};

__device__ __forceinline__ const ScanJob& scan_job(const ScanJob& j0, const ScanJob& j1, int& part)
{
    part = blockIdx.x;
    if (part < j0.nparts) return j0;
    part -= j0.nparts;
    return j1;
}

__global__ void __launch_bounds__(kThreads) k_part_sums(ScanJob j0, ScanJob j1)
{
    int part;
    const ScanJob& j = scan_job(j0, j1, part);
    const int len = scan_len(j.n, j.n_dev);
    const int64_t chunk = part_chunk(len, j.nparts);
    const int64_t a = (int64_t)part * chunk, b = a + chunk < len ? a + chunk : (int64_t)len;
    const bool vec = (reinterpret_cast<uintptr_t>(j.in) & 15) == 0;
    long long s = 0;
    for (int64_t i = a + 4 * threadIdx.x; i < b; i += kPartTile * kPartGroup) {
        int4 v[kPartGroup];
#pragma unroll
        for (int u = 0; u < kPartGroup; ++u) v[u] = load4(j.in, i + u * kPartTile, b, vec);
#pragma unroll
        for (int u = 0; u < kPartGroup; ++u) s += (long long)v[u].x + v[u].y + v[u].z + v[u].w;
    }
    const long long t = block_sum(s);
    if (threadIdx.x == 0) j.psum[part] = (int)t;
}

__global__ void __launch_bounds__(kThreads) k_part_scan(ScanJob j0, ScanJob j1)
{
    __shared__ int wsum[kPartGroup][kThreads / 32];
    __shared__ int base;
    int part;
    const ScanJob& j = scan_job(j0, j1, part);
    const int* in = j.in;
    int* out = j.out;
    const int len = scan_len(j.n, j.n_dev);
    const int64_t chunk = part_chunk(len, j.nparts);
    const int64_t a = (int64_t)part * chunk, b = a + chunk < len ? a + chunk : (int64_t)len;
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    long long o = 0;
    for (int q = threadIdx.x; q < part; q += kThreads) o += j.psum[q];
    const long long ot = block_sum(o);
    if (threadIdx.x == 0) base = (int)ot;
    __syncthreads();
    int carry = base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t t0 = a; t0 < b; t0 += kPartTile * kPartGroup) {
        // tile u of the group: items t0 + u * kPartTile .. ; all of them read before any is written
        // (in place, each item is written by the thread that read it)
        int4 v[kPartGroup];
        int tot[kPartGroup], incl[kPartGroup];
#pragma unroll
        for (int u = 0; u < kPartGroup; ++u) v[u] = load4(in, t0 + u * kPartTile + 4 * threadIdx.x, b, vec);
#pragma unroll
        for (int u = 0; u < kPartGroup; ++u) {
            tot[u] = v[u].x + v[u].y + v[u].z + v[u].w;
            incl[u] = tot[u];
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int u = 0; u < kPartGroup; ++u) {
                const int x = __shfl_up_sync(0xffffffffu, incl[u], d);
                if (lane >= d) incl[u] += x;
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int u = 0; u < kPartGroup; ++u) wsum[u][wid] = incl[u];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPartGroup; ++u) {
            int before = 0, all = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                const int x = wsum[u][w];
                before += w < wid ? x : 0;
                all += x;
            }
            int4 r;
            r.x = carry + before + incl[u] - tot[u];
            r.y = r.x + v[u].x;
            r.z = r.y + v[u].y;
            r.w = r.z + v[u].z;
            store4(out, t0 + u * kPartTile + 4 * threadIdx.x, b, vec, r);
            carry += all;
        }
        __syncthreads();
    }
    if (part == j.nparts - 1 && threadIdx.x == 0) out[len] = carry;
}

static ScanJob scan_job_for(const Context& c, const int* in, int* out, int64_t n, const int* n_dev, int* psum,
                            int64_t cap)
{
    int64_t np = std::min<int64_t>(2 * (int64_t)c.num_sms, (n + kPartTile - 1) / kPartTile);
    np = std::max<int64_t>(1, std::min<int64_t>(np, cap));
    return ScanJob{in, out, n, n_dev, psum, (int)np};
}

// Exclusive prefix of in[0..len) into out[0..len], out[len] = total; len = *n_dev if given
// (then n is its upper bound).  in == out is allowed (every part reads its items before writing
// them, and out[len] lies outside every part).
void exclusive_scan(Context& c, const int* in, int* out, int64_t n, const int* n_dev)
{
    const ScanJob j0 = scan_job_for(c, in, out, n, n_dev, c.scan_tmp, c.scan_tmp_cap);
    const ScanJob none{nullptr, nullptr, 0, nullptr, nullptr, 0};
    k_part_sums<<<j0.nparts, kThreads, 0, c.stream>>>(j0, none);
    k_part_scan<<<j0.nparts, kThreads, 0, c.stream>>>(j0, none);
}

// Two independent exclusive scans in the same two launches (the part sums of the second one
// after the first one's in the scratch)
void exclusive_scan2(Context& c, const int* in0, int* out0, int64_t n0, const int* n_dev0, const int* in1,
                     int* out1, int64_t n1, const int* n_dev1)
{
    const int64_t half = c.scan_tmp_cap / 2;
    const ScanJob j0 = scan_job_for(c, in0, out0, n0, n_dev0, c.scan_tmp, half);
    const ScanJob j1 = scan_job_for(c, in1, out1, n1, n_dev1, c.scan_tmp + j0.nparts, c.scan_tmp_cap - j0.nparts);
    k_part_sums<<<j0.nparts + j1.nparts, kThreads, 0, c.stream>>>(j0, j1);
    k_part_scan<<<j0.nparts + j1.nparts, kThreads, 0, c.stream>>>(j0, j1);
}

// ============================================================================ advance

// Shared memory of k_advance, per thread (slots kThreads apart): the RK3 state, increment sums,
// low-storage register and the extents' double-float copy (36 doubles, rk3<true, true>), then the
// exit / invalid action sums and four counters (6) -- out of the 128 registers the ray equations
// need at two blocks per SM (no spills)
constexpr int kAdvanceRkSlots = 36;
constexpr size_t kAdvanceSmem = sizeof(double) * (kAdvanceRkSlots + 6) * kThreads;

__global__ void __launch_bounds__(kThreads, 2) k_advance(Grid G, Params P, RaySoA A, const NodeDF* __restrict__ bg,
                                                        Ctl* ctl, double dt, int* __restrict__ info,
                                                        int4* __restrict__ ccell, int4* __restrict__ cslot,
                                                        int* __restrict__ newid, int* __restrict__ cnt,
                                                        double* __restrict__ partials, int pstride, ClearSet zs)
{
    extern __shared__ double sh_state[];   // kAdvanceSmem bytes
    const int n = ctl->n;
    // this thread's exit / invalid action sums and its exit, invalid, vertical- and horizontal-split
    // counters, updated in shared memory where they occur: not held in registers across the stages
    double* const tw = sh_state + kAdvanceRkSlots * kThreads + threadIdx.x;
    long long* const tn = reinterpret_cast<long long*>(tw + 2 * kThreads);
    tw[0] = 0.0;
    tw[kThreads] = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) tn[c * kThreads] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s[NSTATE];
        long long id;
        // the nine propagated components and the id (its member selects the background) now;
        // P_x, P_y, P_z and N, which the stages do not touch, after them: out of the registers the
        // ray equations need
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 v = __ldg(&A.a[q][i]);
            s[2 * q] = v.x;
            s[2 * q + 1] = v.y;
        }
        s[SEZ] = __ldg(reinterpret_cast<const double*>(&A.a[4][i]));
        id = __ldg(reinterpret_cast<const long long*>(&A.a[6][i]) + 1);
        const int mem = member_of(id);
        const NodeDF* bgm = bg + (int64_t)mem * G.ncell;
        rk3<true, true>(G, bgm, s, dt, sh_state + threadIdx.x);
        s[SPX] = __ldg(reinterpret_cast<const double*>(&A.a[4][i]) + 1);
        {
            const double2 v = __ldg(&A.a[5][i]);
            s[SPY] = v.x;
            s[SPZ] = v.y;
        }
        s[SN] = __ldg(reinterpret_cast<const double*>(&A.a[6][i]));
        wrap_position(G, s);
        const int st = ray_status(G, s);
        int code = 0, nch = 0;
        int cc[4] = {-1, -1, -1, -1}, sl[4] = {0, 0, 0, 0};
        if (st == 2) {
            tn[kThreads] += 1;
            const double w = ray_action(s);
            if (isfinite(w)) tw[kThreads] += w;
        } else if (st == 1) {
            tn[0] += 1;
            tw[0] += ray_action(s);
        } else {
            code = split_code(G, P, s);
            nch = num_children(code);
            if (code & 1) tn[2 * kThreads] += 1;
            if (code & 2) tn[3 * kThreads] += (code & 1) ? 2 : 1;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c >= nch) break;
                double ch[NSTATE];
                make_child(G, s, code, c, ch);
                if (ray_status(G, ch) != 0) {
                    tn[0] += 1;
                    tw[0] += ray_action(ch);
                } else {
                    cc[c] = mem * G.ncell + cell_of(G, ch);
                    sl[c] = atomicAdd(&cnt[cc[c]], 1);
                }
            }
            store_ray(A, i, s, id);
        }
        info[i] = code | (nch << 4) | (st << 8);
        ccell[i] = make_int4(cc[0], cc[1], cc[2], cc[3]);
        cslot[i] = make_int4(sl[0], sl[1], sl[2], sl[3]);
        newid[i] = nch > 0 ? nch - 1 : 0;
    }
    // the projected fields, with stores (bulk copies were measured slower here: 0.680 -> 0.741 ms)
    clear_fields(zs);
    const double we = block_sum(tw[0]);
    const double wi = block_sum(tw[kThreads]);
    const long long ne = block_sum(tn[0]), ni = block_sum(tn[kThreads]), nv = block_sum(tn[2 * kThreads]),
                    nh = block_sum(tn[3 * kThreads]);
    if (threadIdx.x == 0) {
        partials[T_EXIT * pstride + blockIdx.x] = we;
        partials[T_INVALID * pstride + blockIdx.x] = wi;
        if (ne) atomicAdd((unsigned long long*)&ctl->n_exited, (unsigned long long)ne);
        if (ni) atomicAdd((unsigned long long*)&ctl->n_invalid, (unsigned long long)ni);
        if (nv) atomicAdd((unsigned long long*)&ctl->n_split_v, (unsigned long long)nv);
        if (nh) atomicAdd((unsigned long long*)&ctl->n_split_h, (unsigned long long)nh);
    }
}

// ============================================================================ re-binning

__global__ void k_scatter(Grid G, RaySoA A, Ctl* ctl, int64_t max_rays, const int* __restrict__ info,
                          const int4* __restrict__ ccell, const int4* __restrict__ cslot,
                          const int* __restrict__ newid, const int* __restrict__ off, long long* __restrict__ ent_id,
                          int* __restrict__ ent_src, int* __restrict__ ent_cell)
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
        const long long pid = __double_as_longlong(A.a[6][i].y);
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

// columns above the cap (App. B.5)
__global__ void k_cap_find(Grid G, Params P, Ctl* ctl, const int* __restrict__ off, int* __restrict__ overlist)
{
    if (ctl->status) return;
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < G.ncol_all; col += gridDim.x * blockDim.x) {
        const int cnt = off[(col + 1) * G.nz] - off[col * G.nz];
        if (cnt > P.cap) overlist[atomicAdd(&ctl->n_over, 1)] = col;
    }
}

// Remove the lowest-energy ray volumes of each over-full column (energy w_hat * N Px Py Pz;
// ties: the larger id goes first).  One block per column, rank by counting.
__global__ void __launch_bounds__(kThreads) k_cap_apply(Grid G, Params P, RaySoA A, const NodeDF* __restrict__ bg,
                                                          Ctl* ctl, const int* __restrict__ info,
                                                          const int* __restrict__ off,
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
            double s[NSTATE], ch[NSTATE];
            long long id;
            load_ray(A, src >> 2, s, id);
            make_child(G, s, info[src >> 2] & 7, src & 3, ch);
            Geo g;
            Intr in;
            intrinsic_at(G, bg + (int64_t)member_of(id) * G.ncell, ch, g, in);
            ecap[e] = in.w * ray_action(ch);
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
                double s[NSTATE], ch[NSTATE];
                long long pid;
                load_ray(A, src >> 2, s, pid);
                make_child(G, s, info[src >> 2] & 7, src & 3, ch);
                w_cap += ray_action(ch);
                ++n_cap;
                atomicSub(&cnt[member_of(pid) * G.ncell + cell_of(G, ch)], 1);
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

// Sort every cell's entries by id (canonical order) and drop the capped ones: a thread per entry
// counts the valid entries of its cell with a smaller id -- its rank -- and writes its source
// there.  No thread idles on the many empty cells, no per-thread arrays; cell segments are short
// (a few entries, tens in the launch slab and above the ghost layer), so the count per entry is
// cheap, and every entry of a warp reads the same few cells.
__global__ void k_segsort(Grid G, Ctl* ctl, const int* __restrict__ off, const int* __restrict__ off2,
                          const long long* __restrict__ ent_id, const int* __restrict__ ent_src,
                          const int* __restrict__ ent_cell, int* __restrict__ sorted_src)
{
    if (ctl->status) return;
    const int total = off[G.ncell_all];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int src = ent_src[e];
        if (src < 0) continue;
        const int c = ent_cell[e];
        const int a = off[c], b = off[c + 1];
        const long long id = ent_id[e];
        int rank = 0;
        int q = a;
        // four entries per pass, their loads issued together
        for (; q + 4 <= b; q += 4) {
            int sv[4];
            long long iv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sv[u] = ent_src[q + u];
                iv[u] = ent_id[q + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) rank += (sv[u] >= 0) && (iv[u] < id);
        }
        for (; q < b; ++q) rank += (ent_src[q] >= 0) && (ent_id[q] < id);
        sorted_src[off2[c] + rank] = src;
    }
}

// Build the canonical array B from the advanced parents in A; with saturation on, also the
// per-ray saturation terms P_j = m^2 k_h^2 / (w K^2) A_j alpha_j (with A_j alpha_j = N Px Py Pz / V_c)
// and K_j^2 (Eq. instability-threshold).
__global__ void __launch_bounds__(kThreads) k_materialize(Grid G, Params P, RaySoA A, RaySoA B,
                                                            const NodeDF* __restrict__ bg, Ctl* ctl,
                                                            const int* __restrict__ off2,
                                                            const int* __restrict__ sorted_src,
                                                            const int* __restrict__ info,
                                                            const int* __restrict__ newid, double* __restrict__ pj,
                                                            double* __restrict__ k2, int* __restrict__ raycell)
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
        if (src < 0 || i >= n_old) {   // inconsistent re-binning: never read past the parents
            set_status(ctl, GWAM_ECUDA);
            continue;
        }
        double s[NSTATE], ch[NSTATE];
        long long id;
        load_ray(A, i, s, id);
        make_child(G, s, info[i] & 7, c, ch);
        const long long cid = c == 0 ? id : with_member(member_of(id), next + newid[i] + c - 1);
        store_ray(B, p, ch, cid);
        raycell[p] = member_of(id) * G.ncell + cell_of(G, ch);
        if (P.saturation) {
            IntrDF in;
            intrinsic_df(G, bg + (int64_t)member_of(id) * G.ncell, ch, in);
            int ci, cj, ck;
            cell_ijk(G, ch, ci, cj, ck);
            const float2 iv = G.ivol_df[cj * G.nz + ck];
            const DF av = df_mul2(df_split(ray_action(ch)), DF{iv.x, iv.y});
            pj[p] = df_to_double(df_mul2(df_mul2(df_mul2(in.m2, in.kh2), df_mul2(in.d.iw, in.d.iK2)), av));
            k2[p] = df_to_double(in.d.K2);
        }
    }
}

// kappa = max(0, (P - rho/2) / (2 dt sum_j P_j K_j^2)) of every carrier cell (Eq. turbulent-diffusivity).
// Rays are in cell order, so each cell is a contiguous run; a run is summed left to right by one
// thread (deterministic, and the order the factor max(0, 1 - 2 kappa K^2 dt) is computed in: where it
// is of the size of the rounding error, the order decides whether it clamps to zero).  k_sat_heads
// lists the cell of every run (one atomic per block and pass, the counts of its warps aggregated in
// shared memory: a single counter under one atomic per warp serialised; iterating rays, not cells,
// skips the many empty cells) and k_sat_kappa sums the listed runs one per lane: the FP64 additions of 32
// runs share one warp instruction, where a thread per ray left all but the runs' first lanes idle.
// The list order varies from run to run; every run's sum does not.
__global__ void __launch_bounds__(kThreads) k_sat_heads(Ctl* ctl, const int* __restrict__ off2, int ncell_all,
                                                          const int* __restrict__ raycell, int* __restrict__ runlist)
{
    __shared__ int wcount[kThreads / 32], wbase[kThreads / 32];
    if (ctl->status) return;
    const int n = off2[ncell_all];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one atomic per block and pass: the block's warps take consecutive slices of the list
    for (int p0 = blockIdx.x * blockDim.x; p0 < n; p0 += gridDim.x * blockDim.x) {
        const int p = p0 + threadIdx.x;
        int c = -1;
        bool head = false;
        if (p < n) {
            c = raycell[p];
            head = p == 0 || raycell[p - 1] != c;
        }
        const unsigned m = __ballot_sync(0xffffffffu, head);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                wbase[w] = tot;
                tot += wcount[w];
            }
            const int b = tot ? atomicAdd(&ctl->n_big, tot) : 0;
            for (int w = 0; w < kThreads / 32; ++w) wbase[w] += b;
        }
        __syncthreads();
        if (head) runlist[wbase[warp] + __popc(m & ((1u << lane) - 1u))] = c;
    }
}

__device__ __forceinline__ void sat_run(int p, int b, int c, const double* __restrict__ rho,
                                        const double* __restrict__ pj, const double* __restrict__ k2, double dt,
                                        double* __restrict__ kappa)
{
    double Pc = 0.0, Q = 0.0;
    for (int q = p; q < b; ++q) {
        Pc += pj[q];
        Q += pj[q] * k2[q];
    }
    // Newton-refined reciprocal instead of an IEEE division (<= 2 ulp; FP64 division is a long
    // instruction sequence at GB300's FP64 rate)
    const double kap = Q > 0.0 ? fmax(0.0, (Pc - 0.5 * rho[c]) * rcp_nr(2.0 * dt * Q)) : 0.0;
    for (int q = p; q < b; ++q) kappa[q] = kap;
}

// the listed runs, counted in ctl->n_big (cleared by k_step_begin; k_sat_heads lists them)
__global__ void k_sat_kappa(const Ctl* ctl, const int* __restrict__ off2, const int* __restrict__ runlist,
                            const double* __restrict__ rho, const double* __restrict__ pj,
                            const double* __restrict__ k2, double dt, double* __restrict__ kappa)
{
    const int nl = ctl->status ? 0 : ctl->n_big;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += gridDim.x * blockDim.x) {
        const int c = runlist[t];
        sat_run(off2[c], off2[c + 1], c, rho, pj, k2, dt, kappa);
    }
}

// ============================================================================ saturation + projection

// Saturation N -> N max(0, 1 - 2 kappa K^2 dt); then each ray volume's fluxes:
//   direct form (Eq. fluxes:momentum): T^{ab} = [w^2 ch_a k_b + f^2 (e_r x ch)_a (e_r x k_h)_b] / (w^2 - f^2) A
//   elastic term (Eq. fluxes:buoyancy, theta cancels): -f^2 N^2 ch_r / (w^2 - f^2) k_h A (without 1/(g rho))
//   pseudomomentum form (App. A): T^{ab} = ch_a k_b A
// Centre fields: cell averages over the ray volumes whose carrier is in the cell, weight V_j/V_c.
// Interface fields (z = kk dz, 1 <= kk < nz): staggered-cell overlap, weight w_h * overlap / dz.
template <bool THETA>
__global__ void __launch_bounds__(kThreads) k_project(Grid G, Params P, RaySoA B, const NodeDF* __restrict__ bg,
                                                        const Ctl* ctl, const int* __restrict__ off2,
                                                        const double* __restrict__ kappa,
                                                        const double* __restrict__ k2, double dt,
                                                        double* __restrict__ fz_l, double* __restrict__ fz_p,
                                                        double* __restrict__ f_ll, double* __restrict__ f_lp,
                                                        double* __restrict__ f_pl, double* __restrict__ f_pp,
                                                        double* __restrict__ e_l, double* __restrict__ e_p,
                                                        double* __restrict__ wad, double* __restrict__ f_tl,
                                                        double* __restrict__ f_tp, double* __restrict__ partials,
                                                        int pstride)
{
    constexpr int NH = THETA ? 9 : 7;   // centre fields of the segmented sums
    const int n = ctl->status ? 0 : off2[G.ncell_all];
    double w_sat = 0.0, w_tot = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x; p0 < n; p0 += stride) {
        const int p = p0 + threadIdx.x;
        const bool act = p < n;
        int key = -1;
        DF hv[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) hv[q] = df_f(0.0f);
        DF zl = df_f(0.0f), zp = df_f(0.0f), lo = df_f(0.0f), hi = df_f(0.0f);
        int col = 0, kk0 = 1, nkk = 0;
        if (act) {
            double s[NSTATE];
            long long id;
            load_ray(B, p, s, id);
            if (P.saturation) {
                const double kap = kappa[p];
                if (kap > 0.0) {
                    const double fac = fmax(0.0, 1.0 - 2.0 * kap * k2[p] * dt);
                    const double nold = s[SN];
                    s[SN] = nold * fac;
                    w_sat += (nold - s[SN]) * s[SPX] * s[SPY] * s[SPZ];
                    B.a[6][p].x = s[SN];
                }
            }
            const double W = ray_action(s);
            w_tot += W;
            const int mem = member_of(id);
            IntrDF in;
            intrinsic_df(G, bg + (int64_t)mem * G.ncell, s, in);
            int ci, cj, ck;
            cell_ijk(G, s, ci, cj, ck);
            col = mem * G.ncol + cj * G.nx + ci;
            key = col * G.nz + ck;
            const DF Wd = df_split(W);
            const float2 iv = G.ivol_df[cj * G.nz + ck];
            const DF aw = df_mul2(Wd, DF{iv.x, iv.y});            // alpha_j A_j = W / V_c
            const DF mg2c = df_mul2(in.mg2, in.d.c);              // (m^2 + Gamma^2) D / (w K^4)
            const DF chx = df_mul2(in.k, mg2c), chy = df_mul2(in.l, mg2c);
            const DF chr = df_neg(df_mul2(df_mul2(in.m, in.kh2), in.d.c));
            DF t_ll, t_lp, t_pl, t_pp, el, ep, zc;
            if (P.flux_form == 0) {
                // 1 / (w^2 - f^2) as K^2 / ((N^2 - f^2) k_h^2): the same quantity without the cancellation
                const DF iden = df_mul2(in.d.K2, df_rcp(df_mul2(in.d.D, in.kh2)));
                const DF w2x = df_mul2(in.d.w2, chx), w2y = df_mul2(in.d.w2, chy);
                const DF f2x = df_mul2(in.f2, chx), f2y = df_mul2(in.f2, chy);
                t_ll = df_mul2(df_add(df_mul2(w2x, in.k), df_mul2(f2y, in.l)), iden);
                t_lp = df_mul2(df_sub(df_mul2(w2x, in.l), df_mul2(f2y, in.k)), iden);
                t_pl = df_mul2(df_sub(df_mul2(w2y, in.k), df_mul2(f2x, in.l)), iden);
                t_pp = df_mul2(df_add(df_mul2(w2y, in.l), df_mul2(f2x, in.k)), iden);
                zc = df_mul2(df_mul2(in.d.w2, chr), iden);
                const DF ec = df_neg(df_mul2(df_mul2(df_mul2(in.f2, in.n2), chr), iden));
                el = df_mul2(ec, in.k);
                ep = df_mul2(ec, in.l);
                if (THETA) {
                    // Eq. fluxes:temperature without theta-bar / (g rho-bar): ch_r f N^2 / (w^2 - f^2) (e_r x k_h)
                    const DF tc = df_mul2(df_mul2(df_mul2(in.f, in.n2), chr), iden);
                    hv[7 % NH] = df_mul2(aw, df_neg(df_mul2(tc, in.l)));
                    hv[8 % NH] = df_mul2(aw, df_mul2(tc, in.k));
                }
            } else {
                t_ll = df_mul2(chx, in.k);
                t_lp = df_mul2(chx, in.l);
                t_pl = df_mul2(chy, in.k);
                t_pp = df_mul2(chy, in.l);
                zc = chr;
                el = df_f(0.0f);
                ep = df_f(0.0f);
            }
            hv[0] = df_mul2(aw, t_ll);
            hv[1] = df_mul2(aw, t_lp);
            hv[2] = df_mul2(aw, t_pl);
            hv[3] = df_mul2(aw, t_pp);
            hv[4] = df_mul2(aw, el);
            hv[5] = df_mul2(aw, ep);
            hv[6] = aw;
            // vertical fluxes: w_h A = W whf / (r^2 ez) -- the cos(phi) ex ey of the horizontal share
            // and of the ray volume cancel; the overlaps are taken in units of dz
            const DF ez = df_split(s[SEZ]);
            DF r2e = ez;
            if (G.geometry == 1) {
                const DF r = df_add(DF{G.df_radius.x, G.df_radius.y}, df_split(s[SZ]));
                r2e = df_mul2(df_mul2(r, r), ez);
            }
            const float2 wf = G.whf_df[cj];
            const DF zcA = df_mul2(zc, df_mul2(df_mul2(Wd, DF{wf.x, wf.y}), df_rcp(r2e)));
            zl = df_mul2(zcA, in.k);
            zp = df_mul2(zcA, in.l);
            const DF u = df_split(s[SZ] * G.inv_dz), e = df_pow2(df_split(s[SEZ] * G.inv_dz), 0.5f);
            lo = df_sub(u, e);
            hi = df_add(u, e);
            kk0 = max(1, (int)df_floor(df_sub(lo, df_f(0.5f))));
            const int kk1 = min(G.nz - 1, (int)df_ceil(df_add(hi, df_f(0.5f))));
            nkk = kk1 >= kk0 ? kk1 - kk0 + 1 : 0;
        }
        // centre fields: warp-segmented reduction over runs of equal cells, one atomic per run
        const bool own = warp_run_interior(key);
        if (warp_segment_reduce_df(key, hv) && key >= 0) {
            double v[NH];
#pragma unroll
            for (int q = 0; q < NH; ++q) v[q] = df_to_double(hv[q]);
            if (own) {
                // the whole cell is this run: store its sum (the ray-step kernel cleared the fields)
                f_ll[key] = v[0];
                f_lp[key] = v[1];
                f_pl[key] = v[2];
                f_pp[key] = v[3];
                e_l[key] = v[4];
                e_p[key] = v[5];
                wad[key] = v[6];
                if (THETA) {
                    f_tl[key] = v[7 % NH];
                    f_tp[key] = v[8 % NH];
                }
            } else {
                atomicAdd(&f_ll[key], v[0]);
                atomicAdd(&f_lp[key], v[1]);
                atomicAdd(&f_pl[key], v[2]);
                atomicAdd(&f_pp[key], v[3]);
                atomicAdd(&e_l[key], v[4]);
                atomicAdd(&e_p[key], v[5]);
                atomicAdd(&wad[key], v[6]);
                if (THETA) {
                    atomicAdd(&f_tl[key], v[7 % NH]);
                    atomicAdd(&f_tp[key], v[8 % NH]);
                }
            }
        }
        // interface fields
        int maxk = nkk;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxk = max(maxk, __shfl_xor_sync(0xffffffffu, maxk, o));
        for (int o = 0; o < maxk; ++o) {
            DF zv[2] = {df_f(0.0f), df_f(0.0f)};
            int zkey = -1;
            if (o < nkk) {
                const int kk = kk0 + o;
                const DF slo = df_f((float)kk - 0.5f), shi = df_f((float)kk + 0.5f);
                const DF ov = df_sub(df_less(hi, shi) ? hi : shi, df_less(lo, slo) ? slo : lo);
                if (ov.hi > 0.0f) {
                    zv[0] = df_mul2(ov, zl);
                    zv[1] = df_mul2(ov, zp);
                    zkey = col * (G.nz + 1) + kk;
                }
            }
            if (warp_segment_reduce_df(zkey, zv) && zkey >= 0) {
                atomicAdd(&fz_l[zkey], df_to_double(zv[0]));
                atomicAdd(&fz_p[zkey], df_to_double(zv[1]));
            }
        }
    }
    const double ws = block_sum(w_sat);
    const double wt = block_sum(w_tot);
    if (threadIdx.x == 0) {
        partials[T_SAT * pstride + blockIdx.x] = ws;
        partials[T_TOTAL * pstride + blockIdx.x] = wt;
    }
}

// ============================================================================ smoothing + divergence

// 1-2-1 x 1-2-1 horizontal smoothing (App. B.4 on a lat-lon grid): periodic in x, the edge row
// reused beyond the pole rows on the sphere, periodic in y on the f-plane.
__global__ void k_smooth(Grid G, const double* __restrict__ in, double* __restrict__ out, int nlev)
{
    const int64_t total = (int64_t)G.ncol_all * nlev;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int lev = (int)(t % nlev);
        const int gcol = (int)(t / nlev);
        const int mem = gcol / G.ncol, col = gcol - mem * G.ncol;
        const int i = col % G.nx, j = col / G.nx;
        const int64_t base = (int64_t)mem * G.ncol;
        double acc = 0.0;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
            int jj = j + dj;
            if (G.geometry == 1) jj = clampi(jj, 0, G.ny - 1);
            else jj = wrap_int(jj, G.ny);
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                const int ii = wrap_int(i + di, G.nx);
                const double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0);
                acc += w * in[(base + (int64_t)jj * G.nx + ii) * nlev + lev];
            }
        }
        out[t] = acc * (1.0 / 16.0);
    }
}

struct FieldSet {
    const double* in[NFIELD];
    double* out[NFIELD];
};

// The same smoothing for several fields in one launch: block (32 levels, 8 columns) of one row;
// blockIdx.z selects the field.  Neighbour offsets are formed once per thread.
__global__ void __launch_bounds__(256) k_smooth_fields(Grid G, FieldSet fs)
{
    const int f = blockIdx.z;
    const int nlev = f <= F_ZP ? G.nz + 1 : G.nz;
    const int ntx = (G.nx + 7) / 8;
    const int mem = blockIdx.y;
    const int j = blockIdx.x / ntx;
    const int i = (blockIdx.x % ntx) * 8 + threadIdx.y;
    if (i >= G.nx) return;
    const int im = i == 0 ? G.nx - 1 : i - 1, ip = i + 1 == G.nx ? 0 : i + 1;
    int jm = j - 1, jp = j + 1;
    if (G.geometry == 1) {
        jm = jm < 0 ? 0 : jm;
        jp = jp >= G.ny ? G.ny - 1 : jp;
    } else {
        jm = jm < 0 ? G.ny - 1 : jm;
        jp = jp >= G.ny ? 0 : jp;
    }
    const int64_t base = (int64_t)mem * G.ncol;
    const int64_t r0 = (base + (int64_t)jm * G.nx) * nlev, r1 = (base + (int64_t)j * G.nx) * nlev,
                  r2 = (base + (int64_t)jp * G.nx) * nlev;
    const int64_t cm = (int64_t)im * nlev, c0 = (int64_t)i * nlev, cp = (int64_t)ip * nlev;
    const double* __restrict__ F = fs.in[f];
    double* __restrict__ O = fs.out[f];
    for (int lev = threadIdx.x; lev < nlev; lev += 32) {
        const double a = F[r0 + cm + lev] + 2.0 * F[r0 + c0 + lev] + F[r0 + cp + lev];
        const double b = F[r1 + cm + lev] + 2.0 * F[r1 + c0 + lev] + F[r1 + cp + lev];
        const double c = F[r2 + cm + lev] + 2.0 * F[r2 + c0 + lev] + F[r2 + cp + lev];
        O[r1 + c0 + lev] = (a + 2.0 * b + c) * (1.0 / 16.0);
    }
}

// smooth fields 0 .. nf-1 in one launch
void launch_smooth(Context& c, int nf)
{
    FieldSet fs;
    for (int f = 0; f < NFIELD; ++f) {
        fs.in[f] = c.field[f];
        fs.out[f] = c.smooth[f];
    }
    const dim3 grid((unsigned)(((c.G.nx + 7) / 8) * c.G.ny), (unsigned)c.G.members, (unsigned)nf);
    k_smooth_fields<<<grid, dim3(32, 8), 0, c.stream>>>(c.G, fs);
}

// ============================================================================ budget, control

// Fold the per-block partials of the slots in `mask` into the budget (a fixed order:
// deterministic); mode 1 also closes a step (live count, ids, step counter).  One warp per slot,
// the slots side by side: lane l sums partials l, l + 32, ... of its slot, kFinUnroll loads issued
// before they are added, then the lane sums by a fixed shuffle tree.  (A block looping over the
// slots one after another, each ending in a block reduction, chained about 30 memory latencies:
// 20 us a step.)
constexpr int kFinUnroll = 16;
static_assert(NTALLY * 32 <= kThreads, "k_finalize runs one warp per tally slot");
__global__ void k_finalize(Ctl* ctl, DevBudget* bud, const double* __restrict__ partials, int nb, int mask, int mode)
{
    __shared__ double acc[NTALLY];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < NTALLY) {
        double v = 0.0;
        if (mask & (1 << w)) {
            const double* __restrict__ p = partials + (int64_t)w * nb;
            for (int b0 = 0; b0 < nb; b0 += 32 * kFinUnroll) {
                double t[kFinUnroll];
#pragma unroll
                for (int u = 0; u < kFinUnroll; ++u) {
                    const int b = b0 + u * 32 + lane;
                    t[u] = b < nb ? p[b] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kFinUnroll; ++u) v += t[u];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) acc[w] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (mask & (1 << T_EXIT)) bud->w_exited += acc[T_EXIT];
    if (mask & (1 << T_INVALID)) bud->w_invalid += acc[T_INVALID];
    if (mask & (1 << T_CAP)) bud->w_capped += acc[T_CAP];
    if (mask & (1 << T_SAT)) bud->w_saturated += acc[T_SAT];
    if (mask & (1 << T_LAUNCH)) {
        bud->w_launched += acc[T_LAUNCH];
        bud->w_total += acc[T_LAUNCH];
    }
    if (mask & (1 << T_TOTAL)) bud->w_total = acc[T_TOTAL];
    if (mode == 1) {
        // after a device failure the population is not trustworthy: drop it (the status stays set)
        ctl->n = ctl->status ? 0 : ctl->n_new;
        ctl->next_id += ctl->new_ids;
        ctl->n_steps += 1;
    }
}

__global__ void k_step_begin(Ctl* ctl)
{
    ctl->n_over = 0;
    ctl->n_big = 0;
    ctl->n_children = 0;
    ctl->new_ids = 0;
    ctl->ray_steps += ctl->n;
}

// ============================================================================ orchestration


// smoothed copy of field f for a read (the step smooths only the fields the divergence needs)
void smooth_field(Context& c, int f)
{
    const int nlev = f <= F_ZP ? c.G.nz + 1 : c.G.nz;
    const int blocks = (int)std::min<int64_t>((c.field_len(f) + kThreads - 1) / kThreads, 8192);
    k_smooth<<<blocks, kThreads, 0, c.stream>>>(c.G, c.field[f], c.smooth[f], nlev);
}

void finalize_tallies(Context& c, int mask, int mode)
{
    k_finalize<<<1, kThreads, 0, c.stream>>>(c.ctl, c.budget, c.partials, c.max_blocks, mask, mode);
}

void tune_mark(Context& c, int idx)
{
    if (c.tune_active) cudaEventRecord(c.tune_ev[c.tune_pending][idx], c.stream);
}

void configure_launch_kernels();

void configure_kernels()
{
    cudaFuncSetAttribute(k_advance, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdvanceSmem);
    configure_launch_kernels();
}

// event `phase` of the current profiled step (phase 0 = step start, kPhases = step end)
void prof_mark(Context& c, int phase)
{
    if (c.gcap_prof) {
        // an event-record node of the graph (a plain record under capture would only order streams)
        cudaEventRecordWithFlags(c.gprof_ev[c.gcap_slot][phase], c.stream, cudaEventRecordExternal);
        return;
    }
    if (!c.prof) return;
    if (phase == 0 && c.prof_pending == Context::kRing) prof_harvest(c);
    cudaEventRecord(c.prof_ev[c.prof_pending][phase], c.stream);
    if (phase == Context::kPhases) ++c.prof_pending;
}

void prof_harvest(Context& c)
{
    for (int q = 0; q < c.prof_pending; ++q) {
        cudaEventSynchronize(c.prof_ev[q][Context::kPhases]);
        for (int p = 0; p < Context::kPhases; ++p) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, c.prof_ev[q][p], c.prof_ev[q][p + 1]);
            c.prof_ms[p] += ms;
        }
    }
    c.prof_steps += c.prof_pending;
    c.prof_pending = 0;
}

void run_step(Context& c, double dt, double* du, double* dv)
{
    if (c.f32) {
        run_step32(c, dt, du, dv);
        return;
    }
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
    k_advance<<<la.blocks, la.threads, kAdvanceSmem, s>>>(G, P, c.A, c.bgdf, c.ctl, dt, c.info, c.ccell, c.cslot, c.newid, c.cnt,
                                               c.partials, c.max_blocks, clear_set(c));
    tune_mark(c, 1);
    prof_mark(c, 1);
    exclusive_scan2(c, c.newid, c.newid, c.max_rays, &c.ctl->n, c.cnt, c.off, G.ncell_all, nullptr);
    k_scatter<<<nb, kThreads, 0, s>>>(G, c.A, c.ctl, c.max_rays, c.info, c.ccell, c.cslot, c.newid, c.off, c.ent_id,
                                      c.ent_src, c.ent_cell);
    int mask = (1 << T_EXIT) | (1 << T_INVALID) | (1 << T_SAT) | (1 << T_TOTAL);
    const int* off2 = c.off;
    if (P.cap > 0) {
        k_cap_find<<<col_blocks, kThreads, 0, s>>>(G, P, c.ctl, c.off, c.overlist);
        k_cap_apply<<<nb, kThreads, 0, s>>>(G, P, c.A, c.bgdf, c.ctl, c.info, c.off, c.overlist, c.ent_id, c.ent_src,
                                            c.ecap, c.cnt, c.partials, c.max_blocks);
        exclusive_scan(c, c.cnt, c.off2, G.ncell_all, nullptr);
        off2 = c.off2;
        mask |= 1 << T_CAP;
    }
    k_segsort<<<nb, kThreads, 0, s>>>(G, c.ctl, c.off, off2, c.ent_id, c.ent_src, c.ent_cell, c.sorted_src);
    tune_mark(c, 2);
    k_materialize<<<lm.blocks, lm.threads, 0, s>>>(G, P, c.A, c.B, c.bgdf, c.ctl, off2, c.sorted_src, c.info, c.newid,
                                                   c.pj, c.k2, c.raycell);
    tune_mark(c, 3);
    prof_mark(c, 2);
    if (P.saturation) {
        // both saturation passes on the largest grid (eight blocks per SM, all resident): shorter
        // chains of per-block passes (saturation 0.070 -> 0.060 ms on the 512 x 256 sphere)
        k_sat_heads<<<c.max_blocks, kThreads, 0, s>>>(c.ctl, off2, G.ncell_all, c.raycell, c.biglist);
        k_sat_kappa<<<c.max_blocks, kThreads, 0, s>>>(c.ctl, off2, c.biglist, c.rho, c.pj, c.k2, dt, c.kappa);
    }
    prof_mark(c, 3);
    // (the projected fields were cleared by k_advance)
    tune_mark(c, 4);
    if (P.theta_flux)
        k_project<true><<<lp.blocks, lp.threads, 0, s>>>(G, P, c.B, c.bgdf, c.ctl, off2, c.kappa, c.k2, dt,
                                                         c.field[F_ZL], c.field[F_ZP], c.field[F_LL], c.field[F_LP],
                                                         c.field[F_PL], c.field[F_PP], c.field[F_EL], c.field[F_EP],
                                                         c.field[F_WAD], c.field[F_TL], c.field[F_TP], c.partials,
                                                         c.max_blocks);
    else
        k_project<false><<<lp.blocks, lp.threads, 0, s>>>(G, P, c.B, c.bgdf, c.ctl, off2, c.kappa, c.k2, dt,
                                                          c.field[F_ZL], c.field[F_ZP], c.field[F_LL], c.field[F_LP],
                                                          c.field[F_PL], c.field[F_PP], c.field[F_EL], c.field[F_EP],
                                                          c.field[F_WAD], nullptr, nullptr, c.partials, c.max_blocks);
    tune_mark(c, 5);
    if (c.tune_active) ++c.tune_pending;
    prof_mark(c, 4);
    grid_phase_df(c, du, dv, mask);
    prof_mark(c, 5);
    swap_rays(c);
}

}  // namespace gwam
