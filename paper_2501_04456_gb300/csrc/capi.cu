// capi.cu -- runtime behind the C ABI of include/npsim.h: owns the device
// buffers of one simulation, picks the all-pairs launch shape with a timing
// autotuner, captures chunks of steps into CUDA graphs, and implements state
// I/O, force queries, statistics, checkpoints and the test hooks.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "npsim_internal.cuh"

using namespace npsim;

namespace {

thread_local std::string g_err;

int set_err(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define NP_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(e_ == cudaErrorMemoryAllocation ? NPSIM_ERR_OOM : NPSIM_ERR_CUDA, \
                           "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                           __FILE__, __LINE__);                                         \
    } while (0)

#define NP_REQUIRE(cond, ...)                                                           \
    do {                                                                                \
        if (!(cond))                                                                    \
            return set_err(NPSIM_ERR_INVALID_ARG, __VA_ARGS__);                         \
    } while (0)

constexpr int kChunk = 16;      // steps per captured graph
constexpr double kKf = 1.593;   // fractal prefactor, Sec. 3.1

template <class T> cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

template <class T> void dfree(T *&p)
{
    if (p)
        cudaFree((void *)p);
    p = nullptr;
}

void free_cells(CellBufs &b)
{
    dfree(b.key);
    dfree(b.rank);
    dfree(b.count);
    dfree(b.start);
    dfree(b.arrived);
    dfree(b.sorted);
    dfree(b.pos);
    dfree(b.sxq);
    dfree(b.tile_sum);
}

// Scratch of the statistics of Sec. 3 (allocated on first use, grown as needed):
// float64 positions, the cell list of the pair histogram, the histograms, the
// per-CTA partial sums and the box-counting hash table.
struct StatsWork {
    double *x = nullptr; // [3][n] float64 positions (hi + lo), when the owner has none
    int x_cap = 0;
    CellGrid grid{};
    CellBufs cb{};
    int cells_cap = 0, cells_n = 0; // cells and NPs the cell buffers hold
    unsigned long long *hist = nullptr, *rhist = nullptr;
    int hist_cap = 0, rhist_cap = 0;
    double *part = nullptr; // 3 doubles per CTA of 256 threads
    int part_cap = 0;
    double *vec = nullptr;  // centre of mass [3], box origin [3]
    unsigned long long *table = nullptr;
    unsigned long long table_size = 0;
    int *count = nullptr;
    unsigned long long *surf = nullptr; // N_surf counter
};
void free_stats(StatsWork &w)
{
    dfree(w.x);
    free_cells(w.cb);
    dfree(w.hist);
    dfree(w.rhist);
    dfree(w.part);
    dfree(w.vec);
    dfree(w.table);
    dfree(w.count);
    dfree(w.surf);
    w = StatsWork{};
}

int check_device(int *sms)
{
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
        return set_err(NPSIM_ERR_NO_DEVICE, "no CUDA device visible");
    int dev = 0;
    NP_CUDA(cudaGetDevice(&dev));
    int major = 0, minor = 0;
    NP_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    NP_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (!(major == 10 && minor == 3))
        return set_err(NPSIM_ERR_NO_DEVICE,
                       "device %d is sm_%d%d; this library is built for sm_103a only", dev,
                       major, minor);
    if (sms)
        NP_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    return NPSIM_OK;
}

std::mutex g_tune_mu;
// (n, lj, grouped length, neutral NPs elided) -> (launch shape, ranges per CTA)
std::map<std::array<long long, 4>, std::pair<int, int>> g_tune_cache;
// Ranges per CTA the autotuner tries for the grouped kernels (dynamic
// launches), and the one a forced shape gets by default.
constexpr int kRangesPerCta[] = {1, 4, 16};
constexpr int kDefaultRangesPerCta = 4;
// ensembles: (grouped length, LJ on, Coulomb on) of every droplet -> launch shape
std::map<std::vector<long long>, int> g_ens_tune_cache;

void fill_streamk(StreamK &sk, int n, const ApConfig &c, int grid_target)
{
    sk.itile = c.block * c.ki;
    sk.jtile = c.jt;
    sk.n_it = (n + sk.itile - 1) / sk.itile;
    sk.n_jt = (n + c.jt - 1) / c.jt;
    sk.W = (long long)sk.n_it * sk.n_jt;
    sk.grid = (int)std::min<long long>(std::max(grid_target, 1), sk.W);
    sk.ctas = 0;
}

// Floats of stream-K partial slots: one slot per (i-tile row, range) pair a
// row can meet, each (hi x, y, z, lo x, y, z) x itile.
// Verlet skin of the LJ neighbour lists (sigma units of the smallest type = 1),
// and the squared displacement (half the skin, less 1 % for rounding) that
// triggers a rebuild.
constexpr float kSkin = 0.3f;
constexpr float kHalfSkin2 = (0.5f * kSkin * 0.99f) * (0.5f * kSkin * 0.99f);

size_t slots_floats(const StreamK &sk)
{
    return (size_t)(sk.n_it + sk.grid) * 6 * (size_t)sk.itile;
}

} // namespace

namespace npsim {
int report_error(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
} // namespace npsim

struct npsim_sim {
    int n = 0, T = 0, sms = 0;
    npsim_params_t P{};
    npsim_type_t types[NPSIM_MAX_TYPES]{};
    double eps_ov[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES]{};
    bool has_ov = false;
    std::vector<int32_t> h_type;
    std::vector<int32_t> h_rank; // order of each NP inside its type group (grouped kernels)
    double d_mean = 1.0;
    float charge_f[NPSIM_MAX_TYPES]{};

    cudaStream_t user = nullptr, cap = nullptr;

    // State: position = xq.xyz (hi words) + x_lo; velocity and force in float32,
    // forces as (hi, lo) pairs.  x is float64 scratch for uploads and statistics.
    double *x = nullptr;                  // [3][n]
    double *stage = nullptr;              // host-facing AoS copies [x | v | F], 9 n (lazy)
    float *x_lo = nullptr, *v = nullptr;  // [3][n]
    float *F = nullptr, *F_tmp = nullptr; // [6][n]
    float4 *xq = nullptr;
    int *typ = nullptr;
    float *slots = nullptr;
    unsigned *ap_work = nullptr;          // range counters of the grouped kernels [2]
    float *F_lj = nullptr;                // [n][8]: (hi x, y, z, lo x | lo y, z, -, -)
    PairTab *tab_full = nullptr, *tab_lj = nullptr, *tab_coul = nullptr;
    float rc2_lim = 0.0f; // largest LJ rc^2 of the table (x 1.0001): tile-culling bound
    int any_charge = 0;   // Coulomb on and some type charged
    float *d_rcc2 = nullptr; // coulomb mode 2: squared Coulomb cutoff per type pair (8 x 8)
    long long *d_step = nullptr;
    float4 *d_spring = nullptr; // [2][NPSIM_MAX_TYPES] spring radius table (spring_entry)
    int *d_flags = nullptr;
    unsigned *d_done = nullptr;

    CellGrid grid{};
    CellBufs cb{};
    bool cell = false;
    double rlist[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES]{}; // list radius per type pair (0: none)
    double cell_h_min = 0.0; // smallest list radius (the cell edge the grid aims at)
    double cell_rc = 0.0;    // largest cutoff of the cell-list terms
    size_t cells_alloc = 0;  // sort keys the cell buffers hold
    NbrList nl{};          // Verlet list over the cells (cell-list LJ)
    int *d_gate = nullptr; // 1: rebuild the cell and neighbour lists at the next pass

    bool ap = false, ap_lj = false;
    int ap_idx = 0;
    int ap_per_cta = kDefaultRangesPerCta; // stream-K ranges per CTA (grouped kernels)

    // type-grouped order for the grouped kernels (built when pair sums are on)
    int *perm = nullptr;    // [n_perm] particle at each grouped position, -1 = padding
    float *qblk = nullptr;  // [n_perm / 256] charge of each 256-position block
    int *tblk = nullptr;    // [n_perm / 256] type of each 256-position block
    int *row_pos = nullptr; // [n] grouped position of particle i (-1: no pair row)
    int n_perm = 0;         // grouped length (multiple of 512)
    int grp_len = 0;        // rows and columns the grouped kernels cover
    StreamK sk{};
    StepParams sp{};

    std::map<int, cudaGraphExec_t> graphs;
    int64_t step = 0;
    int last_chunk = 0;

    // per-kernel timing: events around each kernel group of each step of a chunk
    bool profiling = false;
    cudaEvent_t ev[kChunk][4][2]{};
    // frame recorder: device staging ring, copy stream, per-slot events
    static constexpr int kRecSlots = 3;
    float4 *rec_ring = nullptr;
    cudaStream_t rec_stream = nullptr;
    cudaEvent_t rec_ready[kRecSlots]{}, rec_done[kRecSlots]{};

    // statistics (allocated on first use)
    StatsWork sw{};

    ~npsim_sim()
    {
        for (auto &g : graphs)
            cudaGraphExecDestroy(g.second);
        graphs.clear();
        for (int k = 0; k < kRecSlots; ++k) {
            if (rec_ready[k])
                cudaEventDestroy(rec_ready[k]);
            if (rec_done[k])
                cudaEventDestroy(rec_done[k]);
        }
        if (rec_stream)
            cudaStreamDestroy(rec_stream);
        dfree(rec_ring);
        for (int j = 0; j < kChunk; ++j)
            for (int k = 0; k < 4; ++k)
                for (int e = 0; e < 2; ++e)
                    if (ev[j][k][e])
                        cudaEventDestroy(ev[j][k][e]);
        dfree(x);
        dfree(stage);
        dfree(x_lo);
        dfree(v);
        dfree(F);
        dfree(F_tmp);
        dfree(xq);
        dfree(typ);
        dfree(slots);
        dfree(ap_work);
        dfree(perm);
        dfree(qblk);
        dfree(tblk);
        dfree(row_pos);
        dfree(F_lj);
        dfree(tab_full);
        dfree(tab_lj);
        dfree(tab_coul);
        dfree(d_step);
        dfree(d_spring);
        dfree(d_flags);
        dfree(d_done);
        dfree(d_gate);
        dfree(nl.nbr);
        dfree(nl.nnbr);
        dfree(nl.x_ref);
        dfree(nl.builds);
        free_cells(cb);
        free_stats(sw);
        dfree(d_rcc2);
        if (cap)
            cudaStreamDestroy(cap);
    }
};

namespace {

// List radius (largest acting cutoff + skin) of every type pair of a pair table,
// as the list kernels form it in float32 (0: the pair is never listed), for
// LJ (t.z = rc^2 where 24 eps = t.y != 0) and, with rcc2, the truncated
// Coulomb term (where C q_a q_b = t.w != 0).
void list_radii(const PairTab &tab, const float *rcc2, float skin, double *rl)
{
    for (int k = 0; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; ++k) {
        const float4 t = tab.e[k];
        const float r_lj = t.y != 0.0f ? std::sqrt(t.z) : 0.0f;
        const float r_c = (rcc2 && rcc2[k] > 0.0f && t.w != 0.0f) ? std::sqrt(rcc2[k]) : 0.0f;
        const float r = std::max(r_lj, r_c);
        rl[k] = r > 0.0f ? (double)r + (double)skin : 0.0;
    }
}

// Stencil half-widths of a grid for the list radii rl: a partner within r of an
// NP lies at most ceil(r / h) cells away along each axis (clamping coordinates
// beyond the grid into the edge cells only shortens distances); a relative
// margin of 1e-5 covers float32 rounding of the cell coordinates.
void set_extents(CellGrid &g, const double *rl)
{
    const double h = 1.0 / (double)g.inv_h;
    for (int k = 0; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; ++k) {
        const double e = rl[k] > 0.0 ? std::ceil(rl[k] * (1.0 + 1e-5) / h) : 1.0;
        g.ext[k] = (unsigned char)std::min(std::max(e, 1.0), 60.0);
    }
}

// Buffers of a cell list of n NPs over the g.tb * g.n_cells sort keys.  pos starts
// at 0 so that every slot it names is in range before the first build.
int alloc_cells(CellGrid &g, CellBufs &b, int n)
{
    const size_t m = (size_t)std::max(g.tb, 1) * (size_t)g.n_cells;
    NP_CUDA(dalloc(&b.key, n));
    NP_CUDA(dalloc(&b.rank, n));
    NP_CUDA(dalloc(&b.count, m));
    NP_CUDA(dalloc(&b.start, m + 1));
    NP_CUDA(dalloc(&b.arrived, n));
    NP_CUDA(dalloc(&b.sorted, n));
    NP_CUDA(dalloc(&b.pos, n));
    NP_CUDA(cudaMemset(b.pos, 0, sizeof(int) * (size_t)(n > 0 ? n : 1)));
    // one record past the NPs: a position far from every NP (type 0), the
    // partner that pads each neighbour list to whole blocks of four
    NP_CUDA(dalloc(&b.sxq, (size_t)n + 1));
    const float4 far = make_float4(kPairPad, kPairPad, kPairPad, 0.0f);
    NP_CUDA(cudaMemcpy(b.sxq + n, &far, sizeof(far), cudaMemcpyHostToDevice));
    NP_CUDA(dalloc(&b.tile_sum, cell_scan_tiles((int)m)));
    return NPSIM_OK;
}

// Cell grid over [-L, L)^3 with edge >= h_min, at most max_cells cells.
CellGrid make_grid(double L, double h_min, long long max_cells)
{
    CellGrid g{};
    double h = h_min * (1.0 + 1e-5);
    long long dim = (long long)std::ceil(2.0 * L / h);
    if (dim < 1)
        dim = 1;
    while (dim * dim * dim > max_cells && dim > 1) {
        h *= 1.1;
        dim = (long long)std::ceil(2.0 * L / h);
    }
    g.dim = (int)dim;
    g.n_cells = (int)(dim * dim * dim);
    g.inv_h = (float)(1.0 / h);
    g.L = (float)L;
    g.tb = 1;
    for (auto &e : g.ext)
        e = 1;
    return g;
}

// The LJ cell list's grid over [-L, L)^3: edge = the smallest list radius of
// the acting type pairs (each pair scans as many cells as its own radius
// needs), sort keys (types x cells) capped at about two per NP so that the
// cell ranges stay in L2 (the edge grows until the grid fits), cell order
// grouped by type.
CellGrid lj_grid(const npsim_sim *s, double L)
{
    CellGrid g = make_grid(L, s->cell_h_min, std::max<long long>(2LL * s->n / s->T + 4096, 1 << 16));
    g.tb = s->T; // cell order grouped by type (uniform list lengths per warp)
    set_extents(g, s->rlist);
    return g;
}

// Cell buffers large enough for grid g (reallocated only when it has more keys).
int ensure_cells(npsim_sim *s, CellGrid &g)
{
    const size_t keys = (size_t)std::max(g.tb, 1) * (size_t)g.n_cells;
    if (keys > s->cells_alloc || !s->cb.key) {
        free_cells(s->cb);
        s->cells_alloc = 0;
        int rc = alloc_cells(g, s->cb, s->n);
        if (rc)
            return rc;
        s->cells_alloc = keys;
    }
    return NPSIM_OK;
}


// Launch shapes of the all-pairs sum in one index space: [0, A) the
// identity-order kernels of allpairs.cu (scalar and packed), then [A, A + G) the
// charge-grouped Coulomb kernels and [A + G, A + G + L) the type-grouped LJ +
// Coulomb kernels of allpairs_grouped.cu.
int shape_count() { return ap_num_configs() + grp_num_configs() + ljg_num_configs(); }

bool shape_grouped(int k) { return k >= ap_num_configs(); }

bool shape_ljg(int k) { return k >= ap_num_configs() + grp_num_configs(); }

ApConfig shape_config(int k)
{
    if (shape_ljg(k))
        return ljg_config(k - ap_num_configs() - grp_num_configs());
    return shape_grouped(k) ? grp_config(k - ap_num_configs()) : ap_config(k);
}

int shape_occupancy(const npsim_sim *s, int k, bool lj)
{
    if (shape_grouped(k) && (!s->perm || s->grp_len == 0))
        return 0;
    if (shape_ljg(k))
        return ljg_occupancy(k - ap_num_configs() - grp_num_configs());
    if (shape_grouped(k))
        return lj ? 0 : grp_occupancy(k - ap_num_configs());
    return ap_occupancy(k, lj);
}

// Stream-K split of shape k on `ctas` CTAs; the grouped kernels cut the
// units into per_cta ranges per CTA and hand them out at run time.
void shape_streamk(const npsim_sim *s, int k, int ctas, int per_cta, StreamK &sk)
{
    const ApConfig c = shape_config(k);
    if (!shape_grouped(k)) {
        fill_streamk(sk, s->n, c, ctas);
        return;
    }
    // rows and columns over the grouped order (grp_len is a multiple of 512)
    sk.itile = c.block * c.ki;
    sk.jtile = c.jt;
    sk.n_it = (s->grp_len + sk.itile - 1) / sk.itile;
    sk.n_jt = s->grp_len / c.jt;
    sk.W = (long long)sk.n_it * sk.n_jt;
    ctas = std::max(ctas, 1);
    sk.grid = (int)std::min<long long>((long long)ctas * std::max(per_cta, 1), sk.W);
    sk.ctas = std::min(ctas, sk.grid);
}

// Type-pair table of a pair sum: LJ + Coulomb, LJ only or Coulomb only.
const PairTab *pair_table(const npsim_sim *s, bool lj, bool coul)
{
    return lj ? (coul ? s->tab_full : s->tab_lj) : s->tab_coul;
}

cudaError_t shape_launch(const npsim_sim *s, int k, bool lj, bool coul, const StreamK &sk,
                         float *slots, cudaStream_t st)
{
    if (shape_ljg(k))
        return launch_allpairs_ljgrp(k - ap_num_configs() - grp_num_configs(), sk, s->xq,
                                     s->perm, s->n_perm, s->tblk, pair_table(s, lj, coul),
                                     lj ? s->rc2_lim : 0.0f, coul ? s->any_charge : 0,
                                     s->ap_work, slots, st);
    if (shape_grouped(k))
        return launch_allpairs_grouped(k - ap_num_configs(), sk, s->xq, s->perm, s->n_perm,
                                       s->qblk, s->ap_work, slots, st);
    return launch_allpairs(k, lj, sk, s->xq, s->typ, s->n, lj ? pair_table(s, lj, coul) : nullptr,
                           slots, st);
}

// Queue the pair forces of the current positions and one integrator pass at
// step (device counter) + step_ofs; step_commit: this pass ends a chunk of
// steps and moves the counter on.  Kernel groups timed by npsim_kernel_times.
enum { KG_ALLPAIRS = 0, KG_CELL_BUILD = 1, KG_CELL_LJ = 2, KG_INTEGRATE = 3 };

int enqueue_pass(npsim_sim *s, int mode, bool want_lj, bool want_coul, bool ext, float *Fout,
                 cudaStream_t st, int prof_slot = -1, int step_ofs = 0, bool step_commit = false)
{
    const bool ap_lj = want_lj && s->P.lj_mode == 1;
    // with the neutral NPs left out and no type charged, the grouped Coulomb
    // sum is empty
    const bool ap_coul = want_coul && s->P.coulomb == 1 &&
                         !(shape_grouped(s->ap_idx) && s->grp_len == 0);
    // coulomb mode 2: Coulomb truncated at its cutoff, summed with LJ from the lists
    const bool cell_coul = want_coul && s->P.coulomb == 2;
    const bool lj_cell = s->cell && (want_lj || cell_coul);
    const bool ap = ap_lj || ap_coul;
    const bool ljg = shape_ljg(s->ap_idx);
    // the ungrouped kernels also serve a Coulomb-only pass of an LJ simulation
    // whose tuned shape is charge-grouped (never: LJ excludes it) or type-grouped
    const bool grouped = ap && shape_grouped(s->ap_idx) && (ljg || !ap_lj);
    const bool prof = prof_slot >= 0 && s->profiling;
    auto mark = [&](int group, int edge) -> cudaError_t {
        // inside stream capture a plain cudaEventRecord only orders the capture;
        // the External flag makes it a real event-record node of the graph
        return prof ? cudaEventRecordWithFlags(s->ev[prof_slot][group][edge], st,
                                               cudaEventRecordExternal)
                    : cudaSuccess;
    };
    if (lj_cell) {
        // the build kernels run (past their gate check) only after an NP has
        // moved more than half the skin since the last build
        NP_CUDA(mark(KG_CELL_BUILD, 0));
        NP_CUDA(launch_cell_build(s->grid, s->xq, s->typ, s->n, s->cb, s->d_gate, st));
        NP_CUDA(launch_nbr_build(s->grid, s->cb, s->n, s->tab_full, s->d_rcc2, kSkin, s->nl,
                                 s->d_flags, s->d_gate, st));
        NP_CUDA(mark(KG_CELL_BUILD, 1));
        NP_CUDA(mark(KG_CELL_LJ, 0));
        NP_CUDA(launch_lj_nbr(s->grid, s->cb, s->xq, s->typ, s->n,
                              want_lj ? s->tab_full : s->tab_coul,
                              cell_coul ? s->d_rcc2 : nullptr, s->nl, s->F_lj, s->d_gate, st));
        NP_CUDA(mark(KG_CELL_LJ, 1));
    }
    if (ap) {
        NP_CUDA(mark(KG_ALLPAIRS, 0));
        NP_CUDA(shape_launch(s, s->ap_idx, ap_lj, ap_coul, s->sk, s->slots, st));
        NP_CUDA(mark(KG_ALLPAIRS, 1));
    }
    IntArgs a{};
    a.x_lo = s->x_lo;
    a.v = s->v;
    a.F = Fout;
    a.typ = s->typ;
    a.xq = s->xq;
    a.slots = ap ? s->slots : nullptr;
    a.sk = s->sk;
    a.F_lj = lj_cell ? s->F_lj : nullptr;
    a.ext_on = ext ? 1 : 0;
    a.field_slots = (ap && !ap_lj && !ljg) ? 1 : 0; // ljg sums C q_a q_b from its table
    a.row_pos = grouped ? s->row_pos : nullptr;
    a.spring = s->d_spring;
    a.x_ref = s->cell ? s->nl.x_ref : nullptr;
    a.sxq = s->cell ? s->cb.sxq : nullptr;
    a.cell_pos = s->cell ? s->cb.pos : nullptr;
    a.nbr_gate = s->d_gate;
    a.half_skin2 = kHalfSkin2;
    a.step = s->d_step;
    a.step_ofs = step_ofs;
    a.step_commit = step_commit ? 1 : 0;
    a.flags = s->d_flags;
    a.done = s->d_done;
    NP_CUDA(mark(KG_INTEGRATE, 0));
    NP_CUDA(launch_integrate(mode, a, s->sp, st));
    NP_CUDA(mark(KG_INTEGRATE, 1));
    return NPSIM_OK;
}

// Queue k >= 1 steps from the step in the device counter: A, (pairs, BA) x
// (k - 1), pairs, B; the launches carry their offsets from the counter, and
// the last one moves it on by k.
int enqueue_chunk(npsim_sim *s, int k, cudaStream_t st)
{
    IntArgs a{};
    a.x_lo = s->x_lo;
    a.v = s->v;
    a.F = s->F;
    a.typ = s->typ;
    a.xq = s->xq;
    a.sk = s->sk;
    a.spring = s->d_spring;
    a.x_ref = s->cell ? s->nl.x_ref : nullptr;
    a.sxq = s->cell ? s->cb.sxq : nullptr;
    a.cell_pos = s->cell ? s->cb.pos : nullptr;
    a.nbr_gate = s->d_gate;
    a.half_skin2 = kHalfSkin2;
    a.step = s->d_step; // the chunk's first step; launch j + 1 below is at step + j + 1
    a.step_ofs = 0;
    a.step_commit = 0;
    a.flags = s->d_flags;
    a.done = s->d_done;
    NP_CUDA(launch_integrate(MODE_A, a, s->sp, st));
    for (int j = 0; j < k; ++j) {
        // the last pass (B at step + k) moves the counter on to step + k
        int rc = enqueue_pass(s, j + 1 < k ? MODE_BA : MODE_B, true, true, true, s->F, st, j,
                              j + 1, j + 1 == k);
        if (rc)
            return rc;
    }
    return NPSIM_OK;
}

int get_graph(npsim_sim *s, int k, cudaGraphExec_t *out)
{
    auto it = s->graphs.find(k);
    if (it != s->graphs.end()) {
        *out = it->second;
        return NPSIM_OK;
    }
    NP_CUDA(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_chunk(s, k, s->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    if (rc) {
        if (g)
            cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    s->graphs[k] = ex;
    *out = ex;
    return NPSIM_OK;
}

int set_gate(npsim_sim *s, int v)
{
    if (s->d_gate) {
        NP_CUDA(cudaMemcpyAsync(s->d_gate, &v, sizeof(int), cudaMemcpyHostToDevice, s->user));
        NP_CUDA(cudaStreamSynchronize(s->user)); // v lives on this stack frame
    }
    return NPSIM_OK;
}

// A neighbour list overflowed (those NPs were summed from the cells, so the
// forces were exact): grow the list to 1.25 x the longest count plus 8, drop
// the graphs (they hold the old buffer) and rebuild at the next pass.
int grow_neighbour_list(npsim_sim *s)
{
    std::vector<int> cnt((size_t)s->n);
    NP_CUDA(cudaMemcpy(cnt.data(), s->nl.nnbr, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost));
    const int mx = *std::max_element(cnt.begin(), cnt.end());
    if (mx <= s->nl.cap)
        return NPSIM_OK;
    const int cap = ((mx + mx / 4 + 8) + 3) & ~3; // whole blocks of four entries
    unsigned *nb = nullptr;
    cudaError_t e = dalloc(&nb, (size_t)cap * s->n);
    if (e != cudaSuccess)
        return set_err(NPSIM_ERR_OOM, "neighbour list of %d x %d entries: %s", cap, s->n,
                       cudaGetErrorString(e));
    dfree(s->nl.nbr);
    s->nl.nbr = nb;
    s->nl.cap = cap;
    for (auto &g : s->graphs)
        cudaGraphExecDestroy(g.second);
    s->graphs.clear();
    return set_gate(s, 1);
}

int read_flags(npsim_sim *s)
{
    int h = 0;
    NP_CUDA(cudaMemcpyAsync(&h, s->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s->user));
    NP_CUDA(cudaStreamSynchronize(s->user));
    if (h & FLAG_NBR_OVERFLOW) {
        const int rest = h & ~FLAG_NBR_OVERFLOW;
        NP_CUDA(cudaMemcpyAsync(s->d_flags, &rest, sizeof(int), cudaMemcpyHostToDevice, s->user));
        NP_CUDA(cudaStreamSynchronize(s->user));
        int rc = grow_neighbour_list(s);
        if (rc)
            return rc;
        h = rest;
    }
    if (h) {
        NP_CUDA(cudaMemsetAsync(s->d_flags, 0, sizeof(int), s->user));
        if (h & FLAG_NONFINITE)
            return set_err(NPSIM_ERR_NONFINITE, "a position became non-finite");
        if (h & FLAG_TIMEOUT)
            return set_err(NPSIM_ERR_TIMEOUT, "a bounded device wait expired");
        if (h & FLAG_ESCAPED)
            return set_err(NPSIM_ERR_ESCAPED,
                           "an NP was farther than 2 max(R0, R(t)) from the droplet centre");
        return set_err(NPSIM_ERR_CUDA, "device error word 0x%x", h);
    }
    return NPSIM_OK;
}

// Pick the all-pairs launch shape (and, for the grouped kernels, the ranges
// per CTA): time each candidate on the current positions, together with the
// integrator's sum over its partial slots (more ranges mean more slots per
// row: the all-pairs launch can gain less than the sum loses).
int autotune(npsim_sim *s)
{
    const bool lj = s->ap_lj;
    const int nc = shape_count();
    // NPSIM_AUTOTUNE=0 takes the first shape; NPSIM_AUTOTUNE=1:<index>[:<ranges per
    // CTA>] forces one (ignored if that shape cannot run this sum); neither
    // touches the cache.
    const char *env = getenv("NPSIM_AUTOTUNE");
    if (env && env[0] == '0') {
        s->ap_idx = 0;
        s->ap_per_cta = kDefaultRangesPerCta;
        return NPSIM_OK;
    }
    if (env && env[0] == '1' && env[1] == ':') {
        const int idx = atoi(env + 2);
        const char *m = strchr(env + 2, ':');
        if (idx >= 0 && idx < nc && shape_occupancy(s, idx, lj) > 0) {
            s->ap_idx = idx;
            s->ap_per_cta = m ? std::max(1, atoi(m + 1)) : kDefaultRangesPerCta;
            return NPSIM_OK;
        }
    }
    const std::array<long long, 4> key{s->n, lj ? 1 : 0, s->grp_len,
                                       s->P.sum_neutral ? 0 : 1};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s->ap_idx = it->second.first;
            s->ap_per_cta = it->second.second;
            return NPSIM_OK;
        }
    }
    const int n_m = (int)(sizeof(kRangesPerCta) / sizeof(kRangesPerCta[0]));
    int best = 0, best_m = kDefaultRangesPerCta;
    {
        // scratch big enough for every candidate
        size_t need = 0;
        for (int c = 0; c < nc; ++c) {
            const int occ = shape_occupancy(s, c, lj);
            if (occ <= 0)
                continue;
            StreamK sk;
            shape_streamk(s, c, occ * s->sms, kRangesPerCta[n_m - 1], sk);
            need = std::max(need, slots_floats(sk));
        }
        const size_t out_floats = 6 * (size_t)std::max(s->n, s->grp_len);
        float *tmp = nullptr;
        NP_CUDA(dalloc(&tmp, need + out_floats));
        float *sum_out = tmp + need;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best_ms = 1e30f;
        const bool coul = s->P.coulomb == 1;
        const bool log = getenv("NPSIM_AUTOTUNE_LOG") != nullptr; // per-shape times to stderr
        for (int c = 0; c < nc; ++c) {
            const int occ = shape_occupancy(s, c, lj);
            if (occ <= 0)
                continue;
            for (int mi = 0; mi < (shape_grouped(c) ? n_m : 1); ++mi) {
                const int m = shape_grouped(c) ? kRangesPerCta[mi] : 1;
                StreamK sk;
                shape_streamk(s, c, occ * s->sms, m, sk);
                if (shape_grouped(c) && mi > 0 && sk.grid == sk.ctas)
                    break; // no more ranges than CTAs: the same launch as m = 1
                const int n_pos = shape_grouped(c) ? s->grp_len : s->n;
                if (shape_launch(s, c, lj, coul, sk, tmp, s->user) != cudaSuccess ||
                    launch_slot_sum(tmp, sk, n_pos, sum_out, s->user) != cudaSuccess)
                    continue;
                const int reps = s->n > 100000 ? 2 : 5;
                cudaEventRecord(e0, s->user);
                for (int r = 0; r < reps; ++r) {
                    shape_launch(s, c, lj, coul, sk, tmp, s->user);
                    launch_slot_sum(tmp, sk, n_pos, sum_out, s->user);
                }
                cudaEventRecord(e1, s->user);
                if (cudaEventSynchronize(e1) != cudaSuccess)
                    continue;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (log) {
                    const ApConfig cf = shape_config(c);
                    fprintf(stderr,
                            "npsim autotune n=%d shape %d <%d,%d,%d> grid %d ranges %d: "
                            "%.4f ms\n",
                            s->n, c, cf.block, cf.ki, cf.jt, sk.ctas > 0 ? sk.ctas : sk.grid,
                            sk.grid, ms / reps);
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                    best_m = m;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(tmp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return set_err(NPSIM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    s->ap_idx = best;
    s->ap_per_cta = best_m;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = std::make_pair(best, best_m);
    return NPSIM_OK;
}

// 3-D Morton (Z-order) key of a point with 10 bits per axis: the bits of the
// cell indices interleaved, so that points close in the key are close in space.
uint32_t spread_bits10(uint32_t v)
{
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Order of the particles `idx` (AoS positions x) along the Z-order curve of
// their bounding box; ties keep index order.
void morton_sort(std::vector<int> &idx, const double *x)
{
    if (idx.size() < 2)
        return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i : idx)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], x[3 * (size_t)i + d]);
            hi[d] = std::max(hi[d], x[3 * (size_t)i + d]);
        }
    std::vector<std::pair<uint32_t, int>> key(idx.size());
    for (size_t k = 0; k < idx.size(); ++k) {
        const int i = idx[k];
        uint32_t c[3];
        for (int d = 0; d < 3; ++d) {
            const double ext = hi[d] - lo[d];
            const double u = ext > 0 ? (x[3 * (size_t)i + d] - lo[d]) / ext : 0.0;
            c[d] = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(u * 1024.0)));
        }
        key[k] = {spread_bits10(c[0]) | (spread_bits10(c[1]) << 1) | (spread_bits10(c[2]) << 2),
                  i};
    }
    std::sort(key.begin(), key.end());
    for (size_t k = 0; k < idx.size(); ++k)
        idx[k] = key[k].second;
}

// Type-grouped order: the charged types first (in type order), then the
// neutral ones; inside a group NPs follow the Z-order curve of their positions
// at creation when LJ is in the pair sum (tiles of nearby NPs let the LJ kernel
// skip tile pairs beyond the cutoff), else their index order; every group is
// padded with -1 to a multiple of 512, so each
// 256-position block has one type (and one charge).  Unless sum_neutral is
// set, and with no LJ in the pair sum, the grouped kernels cover only the
// charged groups and neutral NPs have no pair row (their Coulomb terms are
// exactly zero).
int build_grouping(npsim_sim *s, const int32_t *type, const double *x0, const int32_t *rank)
{
    std::vector<int> order;
    for (int t = 0; t < s->T; ++t)
        if (s->types[t].charge != 0.0)
            order.push_back(t);
    const int n_charged_types = (int)order.size();
    for (int t = 0; t < s->T; ++t)
        if (s->types[t].charge == 0.0)
            order.push_back(t);
    std::vector<std::vector<int>> members(s->T);
    for (int i = 0; i < s->n; ++i)
        members[type[i]].push_back(i);
    for (auto &m : members) {
        if (rank) // an order saved with a checkpoint: resume in the same summation order
            std::stable_sort(m.begin(), m.end(), [&](int a, int b) { return rank[a] < rank[b]; });
        else if (s->P.lj_mode == 1) // LJ in the pair sum: spatially compact tiles
            morton_sort(m, x0);
        // Coulomb only: index order keeps the integrator's partial reads coalesced
    }
    std::vector<int> perm, tb;
    std::vector<float> qb;
    std::vector<int> pos(s->n, -1);
    int charged_len = 0;
    for (int g = 0; g < (int)order.size(); ++g) {
        const int t = order[g];
        if (members[t].empty())
            continue;
        for (int i : members[t]) {
            pos[i] = (int)perm.size();
            perm.push_back(i);
        }
        while (perm.size() % 512)
            perm.push_back(-1);
        while (qb.size() < perm.size() / 256) {
            qb.push_back((float)s->types[t].charge);
            tb.push_back(t);
        }
        if (g < n_charged_types)
            charged_len = (int)perm.size();
    }
    s->n_perm = (int)perm.size();
    s->h_rank.assign(pos.begin(), pos.end());
    const bool skip = !s->P.sum_neutral && s->P.lj_mode != 1;
    if (skip) {
        s->grp_len = charged_len;
        for (int i = 0; i < s->n; ++i)
            if (s->types[type[i]].charge == 0.0)
                pos[i] = -1;
    } else {
        s->grp_len = s->n_perm;
    }
    NP_CUDA(dalloc(&s->perm, perm.size()));
    NP_CUDA(dalloc(&s->qblk, qb.size()));
    NP_CUDA(dalloc(&s->tblk, tb.size()));
    NP_CUDA(dalloc(&s->row_pos, (size_t)s->n));
    NP_CUDA(cudaMemcpy(s->perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice));
    NP_CUDA(cudaMemcpy(s->qblk, qb.data(), sizeof(float) * qb.size(), cudaMemcpyHostToDevice));
    NP_CUDA(cudaMemcpy(s->tblk, tb.data(), sizeof(int) * tb.size(), cudaMemcpyHostToDevice));
    NP_CUDA(cudaMemcpy(s->row_pos, pos.data(), sizeof(int) * pos.size(),
                       cudaMemcpyHostToDevice));
    return NPSIM_OK;
}

void to_soa(const double *aos, int n, std::vector<double> &soa)
{
    soa.resize(3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            soa[(size_t)d * n + i] = aos[3 * (size_t)i + d];
}

// Device-side AoS float64 copies of the requested parts of the state (any
// pointer NULL), then one copy each to the host arrays, on the sim's stream.
int copy_state_out(npsim_sim *s, const float *F_src, double *x, double *v, double *F)
{
    const size_t n3 = 3 * (size_t)s->n;
    if (!s->stage)
        NP_CUDA(dalloc(&s->stage, 3 * n3));
    double *dx = x ? s->stage : nullptr, *dv = v ? s->stage + n3 : nullptr,
           *dF = F ? s->stage + 2 * n3 : nullptr;
    NP_CUDA(launch_state_aos(s->xq, s->x_lo, s->v, F_src, s->n, dx, dv, dF, s->user));
    if (x)
        NP_CUDA(cudaMemcpyAsync(x, dx, sizeof(double) * n3, cudaMemcpyDeviceToHost, s->user));
    if (v)
        NP_CUDA(cudaMemcpyAsync(v, dv, sizeof(double) * n3, cudaMemcpyDeviceToHost, s->user));
    if (F)
        NP_CUDA(cudaMemcpyAsync(F, dF, sizeof(double) * n3, cudaMemcpyDeviceToHost, s->user));
    NP_CUDA(cudaStreamSynchronize(s->user));
    return NPSIM_OK;
}

// Host float64 SoA -> device float32 (rounded to nearest).
int put_f32(const std::vector<double> &src, float *d, cudaStream_t st)
{
    std::vector<float> h(src.begin(), src.end());
    NP_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st));
    NP_CUDA(cudaStreamSynchronize(st));
    return NPSIM_OK;
}

// Positions in float64 (hi + lo of every coordinate) into s->x.
int positions_f64(npsim_sim *s)
{
    NP_CUDA(launch_positions_f64(s->xq, s->x_lo, s->n, s->x, s->user));
    return NPSIM_OK;
}

// Set the step counter and recompute the forces of the current state.
int finish_upload(npsim_sim *s, int64_t step, bool rebuild = true)
{
    if (rebuild) {
        int rc = set_gate(s, 1); // new positions: rebuild the lists at the next pass
        if (rc)
            return rc;
    }
    long long st = step;
    NP_CUDA(cudaMemcpyAsync(s->d_step, &st, sizeof(long long), cudaMemcpyHostToDevice,
                            s->user));
    float4 tab[NPSIM_MAX_TYPES] = {};
    for (int t = 0; t < s->T; ++t)
        tab[t] = spring_entry(s->P.R0, s->P.k_evap, s->P.dt, st, 0.5 * s->types[t].sigma);
    NP_CUDA(cudaMemcpyAsync(s->d_spring + (st & 1) * NPSIM_MAX_TYPES, tab, sizeof(tab),
                            cudaMemcpyHostToDevice, s->user));
    NP_CUDA(cudaStreamSynchronize(s->user)); // tab lives on this stack frame
    int rc = enqueue_pass(s, MODE_FORCES, true, true, true, s->F, s->user);
    if (rc)
        return rc;
    NP_CUDA(cudaStreamSynchronize(s->user));
    s->step = step;
    return read_flags(s);
}

int upload_state(npsim_sim *s, const double *x, const double *v, int64_t step)
{
    std::vector<double> buf;
    to_soa(x, s->n, buf);
    NP_CUDA(cudaMemcpyAsync(s->x, buf.data(), sizeof(double) * buf.size(),
                            cudaMemcpyHostToDevice, s->user));
    NP_CUDA(cudaStreamSynchronize(s->user));
    if (v) {
        to_soa(v, s->n, buf);
        int rc = put_f32(buf, s->v, s->user);
        if (rc)
            return rc;
    } else {
        NP_CUDA(cudaMemsetAsync(s->v, 0, sizeof(float) * 3 * (size_t)s->n, s->user));
    }
    NP_CUDA(launch_mirror(s->x, s->typ, s->charge_f, s->n, s->xq, s->x_lo, s->user));
    return finish_upload(s, step);
}

// Replace the state by raw words (hi [3][n], lo [3][n], v [3][n], float32 SoA).
int upload_words(npsim_sim *s, const float *words, int64_t step)
{
    const size_t n = (size_t)s->n;
    std::vector<float4> xq(n);
    for (size_t i = 0; i < n; ++i)
        xq[i] = make_float4(words[i], words[n + i], words[2 * n + i],
                            s->charge_f[s->h_type[i]]);
    NP_CUDA(cudaStreamSynchronize(s->user));
    NP_CUDA(cudaMemcpy(s->xq, xq.data(), sizeof(float4) * n, cudaMemcpyHostToDevice));
    NP_CUDA(cudaMemcpy(s->x_lo, words + 3 * n, sizeof(float) * 3 * n, cudaMemcpyHostToDevice));
    NP_CUDA(cudaMemcpy(s->v, words + 6 * n, sizeof(float) * 3 * n, cudaMemcpyHostToDevice));
    return finish_upload(s, step);
}

// Per-type integrator coefficients (float64 on the host): BAOAB O-step factors
// c1 = exp(-gamma dt), sqrt((1 - c1^2) kT / m); overdamped mobility 1/(m gamma)
// and noise sqrt(2 kT dt / (m gamma)); C q for the Coulomb field.
void fill_coefs(const npsim_type_t *types, const npsim_params_t *params, TypeCoef *tc,
                float *charge_f)
{
    const double C = params->bjerrum;
    for (int t = 0; t < params->n_types; ++t) {
        const npsim_type_t &ty = types[t];
        TypeCoef &c = tc[t];
        c.mass = ty.mass;
        c.inv_mass = 1.0 / ty.mass;
        c.half_sigma = 0.5 * ty.sigma;
        c.k_wall = ty.k_wall;
        c.c1 = std::exp(-ty.gamma * params->dt);
        c.sd_o = std::sqrt((1.0 - c.c1 * c.c1) * params->kT / ty.mass);
        c.mob = ty.gamma > 0 ? 1.0 / (ty.mass * ty.gamma) : 0.0;
        c.sd_bd = std::sqrt(2.0 * params->kT * params->dt * c.mob);
        c.charge_c = C * ty.charge;
        c.hdt_m = (float)(0.5 * params->dt / ty.mass);
        c.c1f = (float)c.c1;
        c.c1lo = (float)(c.c1 - (double)c.c1f);
        c.sd_of = (float)c.sd_o;
        c.dt_mob = (float)(params->dt * c.mob);
        c.sd_bdf = (float)c.sd_bd;
        c.qc = (float)c.charge_c;
        c.mg = (float)(ty.mass * params->g);
        c.mw2 = (float)(ty.mass * params->omega * params->omega);
        c.kw = (float)ty.k_wall;
        c.hs = (float)c.half_sigma;
        c.dt_m = (float)(params->dt / ty.mass);
        c.gdt = (float)(ty.gamma * params->dt);
        c.kick = (float)params->v_kick;
        if (charge_f)
            charge_f[t] = (float)ty.charge;
    }
}

// Type-pair tables (sigma_ab^2, 24 eps_ab, rc_ab^2, C q_a q_b) with Lorentz-Berthelot
// mixing unless eps_ov (T x T) is given; tl is the same with the Coulomb column 0.
// Returns the largest cutoff.
double fill_tabs(const npsim_type_t *types, const npsim_params_t *params, const double *eps_ov,
                 PairTab *tf, PairTab *tl)
{
    const int T = params->n_types;
    const double C = params->bjerrum;
    double rc_max = 0.0;
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            const double sig = 0.5 * (types[a].sigma + types[b].sigma);
            const double eps = eps_ov ? eps_ov[a * T + b] : std::sqrt(types[a].eps * types[b].eps);
            const double rc = params->lj_cut * sig;
            rc_max = std::max(rc_max, rc);
            const float4 e = make_float4(
                (float)(sig * sig), (float)(24.0 * eps), (float)(rc * rc),
                (float)(params->coulomb ? C * types[a].charge * types[b].charge : 0.0));
            tf->e[a * NPSIM_MAX_TYPES + b] = e;
            if (tl)
                tl->e[a * NPSIM_MAX_TYPES + b] = make_float4(e.x, e.y, e.z, 0.0f);
        }
    return rc_max;
}

int validate(const npsim_type_t *types, const npsim_params_t *p, int64_t n)
{
    NP_REQUIRE(types && p, "types and params are required");
    NP_REQUIRE(n >= 1 && n <= (1ll << 29), "n = %lld out of range [1, 2^29]", (long long)n);
    NP_REQUIRE(p->n_types >= 1 && p->n_types <= NPSIM_MAX_TYPES, "n_types = %d",
               p->n_types);
    NP_REQUIRE(p->dt > 0 && std::isfinite(p->dt), "dt must be positive");
    NP_REQUIRE(p->kT >= 0, "kT must be >= 0");
    NP_REQUIRE(p->rot_mode >= 0 && p->rot_mode <= 2, "rot_mode must be 0, 1 or 2");
    NP_REQUIRE(p->lj_mode >= 0 && p->lj_mode <= 2, "lj_mode must be 0, 1 or 2");
    NP_REQUIRE(p->integrator >= 0 && p->integrator <= 2, "integrator must be 0, 1 or 2");
    NP_REQUIRE(p->wall >= 0 && p->wall <= 2, "wall must be 0, 1 or 2");
    NP_REQUIRE(p->coulomb >= 0 && p->coulomb <= 2, "coulomb must be 0, 1 or 2");
    NP_REQUIRE(p->coulomb != 2 || p->lj_mode == 2,
               "coulomb 2 (truncated, through the cell list) needs lj_mode 2");
    NP_REQUIRE(p->coulomb != 2 || (p->coulomb_cut > 0 && std::isfinite(p->coulomb_cut)),
               "coulomb 2 needs coulomb_cut > 0");
    NP_REQUIRE(p->R0 > 0 || !p->wall, "R0 must be positive when the wall is on");
    NP_REQUIRE(p->integrator != 2 || (p->v_kick >= 0 && std::isfinite(p->v_kick)),
               "v_kick must be finite and >= 0");
    NP_REQUIRE(p->lj_mode == 0 || p->lj_cut > 0, "lj_cut must be positive");
    for (int t = 0; t < p->n_types; ++t) {
        NP_REQUIRE(types[t].sigma > 0 && types[t].mass > 0, "type %d: sigma, mass > 0", t);
        NP_REQUIRE(types[t].gamma >= 0 && types[t].eps >= 0 && types[t].k_wall >= 0,
                   "type %d: gamma, eps, k_wall >= 0", t);
        NP_REQUIRE(p->integrator != 1 || types[t].gamma > 0,
                   "type %d: the overdamped integrator needs gamma > 0", t);
    }
    return NPSIM_OK;
}

} // namespace

extern "C" {

const char *npsim_last_error(void) { return g_err.c_str(); }

int npsim_device_info(int *sm_count, int *clock_khz, int *cc_major, int *cc_minor)
{
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
        return set_err(NPSIM_ERR_NO_DEVICE, "no CUDA device visible");
    int dev = 0;
    NP_CUDA(cudaGetDevice(&dev));
    if (sm_count)
        NP_CUDA(cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev));
    if (clock_khz)
        NP_CUDA(cudaDeviceGetAttribute(clock_khz, cudaDevAttrClockRate, dev));
    if (cc_major)
        NP_CUDA(cudaDeviceGetAttribute(cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    if (cc_minor)
        NP_CUDA(cudaDeviceGetAttribute(cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    return NPSIM_OK;
}

} // extern "C"

namespace {

// npsim_create with an optional saved grouping order (rank, n entries: the
// order of each NP inside its type group, from a checkpoint).
int create_impl(const npsim_type_t *types, const npsim_params_t *params, int64_t n,
                const double *x0, const double *v0, const int32_t *type, void *stream,
                const int32_t *rank, npsim_sim_t *out)
{
    if (!out)
        return set_err(NPSIM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate(types, params, n);
    if (rc)
        return rc;
    NP_REQUIRE(x0 && type, "x0 and type are required");
    int sms = 0;
    rc = check_device(&sms);
    if (rc)
        return rc;
    for (int64_t i = 0; i < n; ++i) {
        NP_REQUIRE(type[i] >= 0 && type[i] < params->n_types, "type[%lld] = %d out of range",
                   (long long)i, type[i]);
        NP_REQUIRE(std::isfinite(x0[3 * i]) && std::isfinite(x0[3 * i + 1]) &&
                       std::isfinite(x0[3 * i + 2]),
                   "x0[%lld] is not finite", (long long)i);
    }

    npsim_sim *s = new npsim_sim();
    s->n = (int)n;
    s->T = params->n_types;
    s->sms = sms;
    s->P = *params;
    for (int t = 0; t < s->T; ++t)
        s->types[t] = types[t];
    if (params->eps_override) {
        s->has_ov = true;
        for (int k = 0; k < s->T * s->T; ++k)
            s->eps_ov[k] = params->eps_override[k];
    }
    s->P.eps_override = nullptr;
    s->h_type.assign(type, type + n);
    s->user = (cudaStream_t)stream;

    auto bail = [&](int code) {
        delete s;
        return code;
    };
    cudaError_t ce = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess)
        return bail(set_err(NPSIM_ERR_CUDA, "stream create: %s", cudaGetErrorString(ce)));

    // per-type coefficients and pair tables (float64 on the host)
    std::vector<long long> tcount(s->T, 0);
    for (int64_t i = 0; i < n; ++i)
        tcount[type[i]]++;
    double dsum = 0.0;
    for (int t = 0; t < s->T; ++t)
        dsum += (double)tcount[t] * types[t].sigma;
    s->d_mean = dsum / (double)n;

    StepParams &sp = s->sp;
    sp.n = s->n;
    sp.n_types = s->T;
    sp.rot_mode = params->rot_mode;
    sp.wall = params->wall;
    sp.integrator = params->integrator;
    sp.seed = params->seed;
    sp.dt = params->dt;
    sp.R0 = params->R0;
    sp.k_evap = params->k_evap;
    sp.g = params->g;
    sp.omega2 = params->omega * params->omega;
    fill_coefs(types, params, sp.tc, s->charge_f);
    PairTab tf{}, tl{}, tc{};
    const double rc_max = fill_tabs(types, params, s->has_ov ? s->eps_ov : nullptr, &tf, &tl);
    for (int k = 0; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; ++k) { // Coulomb only: no LJ pair in range
        tc.e[k] = make_float4(0.0f, 0.0f, 0.0f, tf.e[k].w);
        if (params->lj_mode != 0 && tf.e[k].y != 0.0f)
            s->rc2_lim = std::max(s->rc2_lim, tf.e[k].z * 1.0001f);
        if (tf.e[k].w != 0.0f)
            s->any_charge = 1;
    }

#define BAIL_CUDA(call)                                                                 \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return bail(set_err(e_ == cudaErrorMemoryAllocation ? NPSIM_ERR_OOM         \
                                                                 : NPSIM_ERR_CUDA,      \
                                "%s failed: %s", #call, cudaGetErrorString(e_)));       \
    } while (0)

    const size_t n3 = 3 * (size_t)n;
    BAIL_CUDA(dalloc(&s->x, n3));
    BAIL_CUDA(dalloc(&s->x_lo, n3));
    BAIL_CUDA(dalloc(&s->v, n3));
    BAIL_CUDA(dalloc(&s->F, 2 * n3));
    BAIL_CUDA(dalloc(&s->F_tmp, 2 * n3));
    BAIL_CUDA(dalloc(&s->xq, (size_t)n));
    BAIL_CUDA(dalloc(&s->typ, (size_t)n));
    BAIL_CUDA(dalloc(&s->tab_full, 1));
    BAIL_CUDA(dalloc(&s->tab_lj, 1));
    BAIL_CUDA(dalloc(&s->tab_coul, 1));
    BAIL_CUDA(dalloc(&s->d_step, 1));
    BAIL_CUDA(dalloc(&s->d_spring, 2 * NPSIM_MAX_TYPES));
    BAIL_CUDA(cudaMemsetAsync(s->d_spring, 0, sizeof(float4) * 2 * NPSIM_MAX_TYPES, s->user));
    BAIL_CUDA(dalloc(&s->d_flags, 1));
    BAIL_CUDA(dalloc(&s->d_done, 1));
    BAIL_CUDA(cudaMemsetAsync(s->d_flags, 0, sizeof(int), s->user));
    BAIL_CUDA(cudaMemsetAsync(s->d_done, 0, sizeof(unsigned), s->user));
    BAIL_CUDA(cudaMemcpyAsync(s->tab_full, &tf, sizeof(PairTab), cudaMemcpyHostToDevice,
                              s->user));
    BAIL_CUDA(cudaMemcpyAsync(s->tab_lj, &tl, sizeof(PairTab), cudaMemcpyHostToDevice,
                              s->user));
    BAIL_CUDA(cudaMemcpyAsync(s->tab_coul, &tc, sizeof(PairTab), cudaMemcpyHostToDevice,
                              s->user));
    BAIL_CUDA(cudaMemcpyAsync(s->typ, type, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice,
                              s->user));
    BAIL_CUDA(cudaStreamSynchronize(s->user));

    s->cell = params->lj_mode == 2;
    double rc_cell = rc_max; // largest cutoff of the cell-list terms
    if (params->coulomb == 2) {
        // truncated Coulomb: cutoff coulomb_cut * sigma_ab for every charged pair
        float rcc2[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES] = {};
        const int T = params->n_types;
        for (int a = 0; a < T; ++a)
            for (int b = 0; b < T; ++b) {
                if (types[a].charge == 0.0 || types[b].charge == 0.0)
                    continue;
                const double rcc = params->coulomb_cut * 0.5 * (types[a].sigma + types[b].sigma);
                rcc2[a * NPSIM_MAX_TYPES + b] = (float)(rcc * rcc);
                rc_cell = std::max(rc_cell, rcc);
            }
        BAIL_CUDA(dalloc(&s->d_rcc2, (size_t)NPSIM_MAX_TYPES * NPSIM_MAX_TYPES));
        BAIL_CUDA(cudaMemcpy(s->d_rcc2, rcc2, sizeof(rcc2), cudaMemcpyHostToDevice));
    }
    if (s->cell) {
        double L = params->R0;
        for (int64_t i = 0; i < 3 * n; ++i)
            L = std::max(L, std::fabs(x0[i]));
        L += rc_cell + kSkin;
        // cell edge: the smallest list radius of the acting type pairs (each pair
        // scans as many cells as its own radius needs), the sort keys (types x
        // cells) capped at about two per NP, so that the cell ranges stay in L2
        // (the edge grows until the grid fits)
        float rcc2h[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES] = {};
        if (s->d_rcc2)
            BAIL_CUDA(cudaMemcpy(rcc2h, s->d_rcc2, sizeof(rcc2h), cudaMemcpyDeviceToHost));
        list_radii(tf, s->d_rcc2 ? rcc2h : nullptr, kSkin, s->rlist);
        double h_min = rc_cell + kSkin;
        for (int a = 0; a < s->T; ++a)
            for (int b = 0; b < s->T; ++b)
                if (s->rlist[a * NPSIM_MAX_TYPES + b] > 0.0)
                    h_min = std::min(h_min, s->rlist[a * NPSIM_MAX_TYPES + b]);
        s->cell_h_min = h_min;
        s->cell_rc = rc_cell;
        s->grid = lj_grid(s, L);
        rc = ensure_cells(s, s->grid);
        if (rc)
            return bail(rc);
        BAIL_CUDA(dalloc(&s->F_lj, 8 * (size_t)n)); // one 32-byte record per NP
        s->nl.cap = 32; // grown after the first build if some NP has more partners
        BAIL_CUDA(dalloc(&s->nl.nbr, (size_t)s->nl.cap * n));
        BAIL_CUDA(dalloc(&s->nl.nnbr, (size_t)n));
        BAIL_CUDA(dalloc(&s->nl.x_ref, (size_t)n));
        BAIL_CUDA(dalloc(&s->nl.builds, 1));
        BAIL_CUDA(cudaMemset(s->nl.builds, 0, sizeof(unsigned long long)));
        BAIL_CUDA(dalloc(&s->d_gate, 1));
    }
    s->ap_lj = params->lj_mode == 1;
    s->ap = params->coulomb == 1 || s->ap_lj;

    // positions for the mirror (needed before tuning)
    {
        std::vector<double> buf;
        to_soa(x0, s->n, buf);
        BAIL_CUDA(cudaMemcpy(s->x, buf.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
        BAIL_CUDA(launch_mirror(s->x, s->typ, s->charge_f, s->n, s->xq, s->x_lo, s->user));
    }
    if (s->ap) {
        rc = build_grouping(s, type, x0, rank);
        if (rc)
            return bail(rc);
        BAIL_CUDA(dalloc(&s->ap_work, 2));
        BAIL_CUDA(cudaMemset(s->ap_work, 0, 2 * sizeof(unsigned)));
        rc = autotune(s);
        if (rc)
            return bail(rc);
        const int occ = std::max(1, shape_occupancy(s, s->ap_idx, s->ap_lj));
        shape_streamk(s, s->ap_idx, occ * s->sms, s->ap_per_cta, s->sk);
        BAIL_CUDA(dalloc(&s->slots, slots_floats(s->sk)));
    } else {
        s->sk = StreamK{};
        s->sk.itile = 1;
        s->sk.n_jt = 1;
        s->sk.grid = 1;
        s->sk.W = 1;
    }
#undef BAIL_CUDA
    rc = upload_state(s, x0, v0, 0);
    if (rc)
        return bail(rc);
    *out = s;
    return NPSIM_OK;
}

} // namespace

extern "C" {

int npsim_create(const npsim_type_t *types, const npsim_params_t *params, int64_t n,
                 const double *x0, const double *v0, const int32_t *type, void *stream,
                 npsim_sim_t *out)
{
    NP_TRACE();
    return create_impl(types, params, n, x0, v0, type, stream, nullptr, out);
}

void npsim_destroy(npsim_sim_t sim)
{
    NP_TRACE();
    if (!sim)
        return;
    cudaStreamSynchronize(sim->user);
    delete sim;
}

} // extern "C"

namespace {
// Queue n_steps steps as graph chunks of at most kChunk steps (no host wait).
// The LJ cell grid follows the droplet.  With the interface spring on, the NPs
// stay within about R(t) of the centre; at every step that is a multiple of
// kRegridPeriod the grid's half-width L is compared with R(t) plus the largest
// cutoff and the skin, and when that differs from L by more than a quarter
// (the droplet has shrunk or grown) a new grid replaces the old one: the cell
// buffers are resized if needed, the lists are rebuilt at the next pass and
// the step graphs are captured again.  The decision depends on the step count
// alone, and the steps are cut at those multiples whatever the calls' sizes,
// so runs stay bit-reproducible (npsim_step(37) = 5 + 16 + 1 + 15 steps).
constexpr int64_t kRegridPeriod = 1024;

// Only the spring on every NP beyond its equilibrium point (wall 1) keeps the
// NPs inside R(t); without a spring or with the band-only one they may leave.
bool follows_droplet(const npsim_sim *s) { return s->cell && s->P.wall == 1; }

int regrid_if_needed(npsim_sim *s)
{
    if (!follows_droplet(s) || s->step % kRegridPeriod != 0)
        return NPSIM_OK;
    const double t = (double)s->step * s->P.dt;
    const double R2 = s->P.R0 * s->P.R0 - s->P.k_evap * t;
    const double R = R2 > 0.0 ? std::sqrt(R2) : 0.0;
    const double L_want = std::max(R, 1.0) + s->cell_rc + kSkin;
    const double L = (double)s->grid.L;
    if (L_want >= 0.75 * L && L_want <= L)
        return NPSIM_OK;
    NP_CUDA(cudaStreamSynchronize(s->user)); // nothing of the old grid in flight
    CellGrid g = lj_grid(s, L_want);
    int rc = ensure_cells(s, g);
    if (rc)
        return rc;
    s->grid = g;
    for (auto &e : s->graphs)
        cudaGraphExecDestroy(e.second);
    s->graphs.clear();
    return set_gate(s, 1);
}

int enqueue_steps(npsim_sim *s, int64_t n_steps)
{
    int64_t rem = n_steps;
    while (rem > 0) {
        int rc0 = regrid_if_needed(s);
        if (rc0)
            return rc0;
        int k = (int)std::min<int64_t>(rem, kChunk);
        if (follows_droplet(s)) // stop at the next multiple of kRegridPeriod
            k = (int)std::min<int64_t>(k, kRegridPeriod - s->step % kRegridPeriod);
        cudaGraphExec_t ex = nullptr;
        int rc = get_graph(s, k, &ex);
        if (rc)
            return rc;
        NP_CUDA(cudaGraphLaunch(ex, s->user));
        s->last_chunk = k;
        rem -= k;
        s->step += k;
    }
    return NPSIM_OK;
}
} // namespace

extern "C" {

int npsim_step(npsim_sim_t s, int64_t n_steps)
{
    NP_TRACE();
    NP_REQUIRE(s, "sim is NULL");
    NP_REQUIRE(n_steps >= 0, "n_steps must be >= 0");
    int rc = enqueue_steps(s, n_steps);
    if (rc)
        return rc;
    return read_flags(s);
}

int npsim_step_record(npsim_sim_t s, int64_t n_steps, int64_t every, float *frames,
                      int64_t n_frames)
{
    NP_TRACE();
    NP_REQUIRE(s && frames, "sim and frames are required");
    NP_REQUIRE(n_steps >= 0 && every >= 1, "n_steps >= 0 and every >= 1 are required");
    const int64_t nf = n_steps / every;
    NP_REQUIRE(n_frames >= nf, "frames holds %lld frames, %lld are recorded",
               (long long)n_frames, (long long)nf);
    const size_t bytes = sizeof(float4) * (size_t)s->n;
    constexpr int R = npsim_sim::kRecSlots;
    if (!s->rec_ring) {
        NP_CUDA(dalloc(&s->rec_ring, (size_t)R * s->n));
        NP_CUDA(cudaStreamCreateWithFlags(&s->rec_stream, cudaStreamNonBlocking));
        for (int k = 0; k < R; ++k) {
            NP_CUDA(cudaEventCreateWithFlags(&s->rec_ready[k], cudaEventDisableTiming));
            NP_CUDA(cudaEventCreateWithFlags(&s->rec_done[k], cudaEventDisableTiming));
        }
    }
    // copies are asynchronous only into page-locked memory: register the
    // caller's buffer for the call unless it already is
    bool registered = false;
    if (nf > 0) {
        cudaPointerAttributes at{};
        const bool locked = cudaPointerGetAttributes(&at, frames) == cudaSuccess &&
                            at.type == cudaMemoryTypeHost;
        cudaGetLastError(); // a plain host pointer may leave an error behind
        if (!locked) {
            NP_CUDA(cudaHostRegister(frames, bytes * (size_t)nf, cudaHostRegisterDefault));
            registered = true;
        }
    }
    int rc = NPSIM_OK;
    cudaError_t e = cudaSuccess;
    for (int64_t f = 0; f < nf && rc == NPSIM_OK && e == cudaSuccess; ++f) {
        rc = enqueue_steps(s, every);
        if (rc)
            break;
        const int slot = (int)(f % R);
        if (f >= R) // the slot's previous frame has reached the host
            e = cudaStreamWaitEvent(s->user, s->rec_done[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->rec_ring + (size_t)slot * s->n, s->xq, bytes,
                                cudaMemcpyDeviceToDevice, s->user);
        if (e == cudaSuccess)
            e = cudaEventRecord(s->rec_ready[slot], s->user);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s->rec_stream, s->rec_ready[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(frames + (size_t)f * 4 * s->n, s->rec_ring + (size_t)slot * s->n,
                                bytes, cudaMemcpyDeviceToHost, s->rec_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(s->rec_done[slot], s->rec_stream);
    }
    if (rc == NPSIM_OK && e == cudaSuccess)
        rc = enqueue_steps(s, n_steps - nf * every);
    const cudaError_t e2 = cudaStreamSynchronize(s->rec_stream);
    if (registered)
        cudaHostUnregister(frames);
    if (rc)
        return rc;
    if (e != cudaSuccess || e2 != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "frame recorder: %s",
                       cudaGetErrorString(e != cudaSuccess ? e : e2));
    return read_flags(s);
}

int npsim_get_state(npsim_sim_t s, double *x, double *v, double *F, int64_t *step)
{
    NP_TRACE();
    NP_REQUIRE(s, "sim is NULL");
    if (x || v || F) {
        int rc = copy_state_out(s, s->F, x, v, F);
        if (rc)
            return rc;
    }
    if (step)
        *step = s->step;
    return NPSIM_OK;
}

int npsim_set_state(npsim_sim_t s, const double *x, const double *v, int64_t step)
{
    NP_REQUIRE(s && x, "sim and x are required");
    NP_REQUIRE(step >= 0, "step must be >= 0");
    return upload_state(s, x, v, step);
}

int npsim_forces(npsim_sim_t s, int what, double *F)
{
    NP_TRACE();
    NP_REQUIRE(s && F, "sim and F are required");
    NP_REQUIRE(what >= 0 && what <= 3, "what must be 0..3");
    const bool lj = what == 0 || what == 1 || what == 2;
    const bool coul = what == 0 || what == 1 || what == 3;
    int rc = enqueue_pass(s, MODE_FORCES, lj, coul, what == 0, s->F_tmp, s->user);
    if (rc)
        return rc;
    return copy_state_out(s, s->F_tmp, nullptr, nullptr, F);
}

int npsim_positions_device(npsim_sim_t s, float *dev_xyzq)
{
    NP_REQUIRE(s && dev_xyzq, "sim and buffer are required");
    NP_CUDA(cudaMemcpyAsync(dev_xyzq, s->xq, sizeof(float4) * (size_t)s->n,
                            cudaMemcpyDeviceToDevice, s->user));
    return NPSIM_OK;
}

int npsim_allpairs_config(npsim_sim_t s, int *block, int *i_per_thread, int *j_tile,
                          int *grid, int *index, int *packed)
{
    NP_REQUIRE(s, "sim is NULL");
    const ApConfig c = shape_config(s->ap_idx);
    if (block)
        *block = s->ap ? c.block : 0;
    if (i_per_thread)
        *i_per_thread = s->ap ? c.ki : 0;
    if (j_tile)
        *j_tile = s->ap ? c.jt : 0;
    if (grid)
        *grid = !s->ap ? 0 : s->sk.ctas > 0 ? s->sk.ctas : s->sk.grid;
    if (index)
        *index = s->ap ? s->ap_idx : -1;
    if (packed)
        *packed = !s->ap                  ? 0
                  : shape_ljg(s->ap_idx)     ? 3
                  : shape_grouped(s->ap_idx) ? 2
                  : ap_packed(s->ap_idx)     ? 1
                                             : 0;
    return NPSIM_OK;
}

int npsim_allpairs_ranges(npsim_sim_t s, int *ranges)
{
    NP_REQUIRE(s && ranges, "sim and ranges are required");
    *ranges = s->ap ? s->sk.grid : 0;
    return NPSIM_OK;
}

int npsim_allpairs_num_configs(int *count)
{
    NP_REQUIRE(count, "count is NULL");
    *count = shape_count();
    return NPSIM_OK;
}

int npsim_launches_per_step(npsim_sim_t s, int *launches)
{
    NP_REQUIRE(s && launches, "sim and launches are required");
    // integrator, all-pairs, the gated cell and list builds, the list LJ forces
    *launches = 1 + (s->ap ? 1 : 0) + (s->cell ? cell_build_launches() + 2 : 0);
    return NPSIM_OK;
}

int npsim_cell_grid(npsim_sim_t s, int *dim, int64_t *n_cells)
{
    NP_REQUIRE(s, "sim is NULL");
    if (dim)
        *dim = s->cell ? s->grid.dim : 0;
    if (n_cells)
        *n_cells = s->cell ? s->grid.n_cells : 0;
    return NPSIM_OK;
}

int npsim_nbr_info(npsim_sim_t s, int *cap, double *mean_len, int64_t *builds)
{
    NP_REQUIRE(s, "sim is NULL");
    if (cap)
        *cap = s->cell ? s->nl.cap : 0;
    if (mean_len)
        *mean_len = 0.0;
    if (builds)
        *builds = 0;
    if (!s->cell)
        return NPSIM_OK;
    NP_CUDA(cudaStreamSynchronize(s->user));
    if (mean_len) {
        std::vector<int> cnt((size_t)s->n);
        NP_CUDA(cudaMemcpy(cnt.data(), s->nl.nnbr, sizeof(int) * cnt.size(),
                           cudaMemcpyDeviceToHost));
        double sum = 0.0;
        for (int c : cnt)
            sum += c;
        *mean_len = sum / (double)s->n;
    }
    if (builds) {
        unsigned long long b = 0;
        NP_CUDA(cudaMemcpy(&b, s->nl.builds, sizeof(b), cudaMemcpyDeviceToHost));
        *builds = (int64_t)b;
    }
    return NPSIM_OK;
}

int npsim_chunk_steps(npsim_sim_t s, int *chunk)
{
    NP_REQUIRE(s && chunk, "sim and chunk are required");
    *chunk = kChunk;
    return NPSIM_OK;
}

int npsim_profile(npsim_sim_t s, int enable)
{
    NP_REQUIRE(s, "sim is NULL");
    NP_CUDA(cudaStreamSynchronize(s->user));
    if (enable && !s->ev[0][0][0]) {
        for (int j = 0; j < kChunk; ++j)
            for (int k = 0; k < 4; ++k)
                for (int e = 0; e < 2; ++e)
                    NP_CUDA(cudaEventCreate(&s->ev[j][k][e]));
    }
    if ((enable != 0) != s->profiling) {
        for (auto &g : s->graphs)
            cudaGraphExecDestroy(g.second);
        s->graphs.clear();
        s->profiling = enable != 0;
        s->last_chunk = 0;
    }
    return NPSIM_OK;
}

int npsim_kernel_times(npsim_sim_t s, double *ms, int *samples)
{
    NP_REQUIRE(s && ms, "sim and ms are required");
    NP_REQUIRE(s->profiling, "profiling is not enabled (npsim_profile)");
    NP_CUDA(cudaStreamSynchronize(s->user));
    const bool used[4] = {s->ap, s->cell, s->cell, true};
    const int k = s->last_chunk;
    for (int g = 0; g < 4; ++g) {
        double tot = 0.0;
        if (used[g])
            for (int j = 0; j < k; ++j) {
                float t = 0.f;
                NP_CUDA(cudaEventElapsedTime(&t, s->ev[j][g][0], s->ev[j][g][1]));
                tot += t;
            }
        ms[g] = (k > 0 && used[g]) ? tot / k : 0.0;
    }
    if (samples)
        *samples = k;
    return NPSIM_OK;
}

// ---------------------------------------------------------------------------
// Statistics

} // extern "C"

namespace {

// One reduction of launch_block_reduce over n positions, its per-CTA partials
// copied to the host (CTA order).
int block_partials(StatsWork &w, int mode, const double *x, int n, const double *c,
                   std::vector<double> &part, cudaStream_t st)
{
    const int nblk = (n + 255) / 256;
    part.resize(3 * (size_t)nblk);
    NP_CUDA(launch_block_reduce(mode, x, n, c, w.part, st));
    NP_CUDA(cudaMemcpyAsync(part.data(), w.part, sizeof(double) * part.size(),
                            cudaMemcpyDeviceToHost, st));
    NP_CUDA(cudaStreamSynchronize(st));
    return NPSIM_OK;
}

// The statistics of Sec. 3 of one droplet of n NPs whose float64 positions
// ([3][n]) are x, float32 hi words xq and types typ (all device), at droplet
// radius R: the RDF (Sec. 3.2), the radial concentration C_NPs, N_surf, the
// centre of mass and R_g (Eqs. r0, Rg), D_f from the fractal equation (Eq. N)
// and by box counting.  Shared by npsim_stats and npsim_ens_stats.
int stats_core(StatsWork &w, const double *x, const float4 *xq, const int *typ, int n, double R,
               double d_mean, const npsim_type_t *types, int T, int *d_flags,
               const npsim_stats_cfg_t *cfg, int64_t *rdf_counts, double *rdf_g,
               int64_t *radial_counts, double *radial_c, npsim_stats_t *out, cudaStream_t st)
{
    memset(out, 0, sizeof(*out));
    out->R = R;
    out->d_mean = d_mean;
    const double pi = 3.14159265358979323846;

    const int nblk = (n + 255) / 256;
    if (!w.vec) {
        NP_CUDA(dalloc(&w.vec, 8));
        NP_CUDA(dalloc(&w.count, 1));
        NP_CUDA(dalloc(&w.surf, 1));
    }
    if (nblk > w.part_cap) {
        dfree(w.part);
        NP_CUDA(dalloc(&w.part, 3 * (size_t)nblk));
        w.part_cap = nblk;
    }
    std::vector<double> part;
    // extent of the cloud: minimum corner (box-counting origin), largest |x_d|
    int rc = block_partials(w, 2, x, n, nullptr, part, st);
    if (rc)
        return rc;
    double o[3] = {INFINITY, INFINITY, INFINITY};
    for (int b = 0; b < nblk; ++b)
        for (int d = 0; d < 3; ++d)
            o[d] = std::min(o[d], part[3 * b + d]);

    if (cfg->n_bins > 0 && rdf_counts) {
        rc = block_partials(w, 3, x, n, nullptr, part, st);
        if (rc)
            return rc;
        // cell grid with edge >= r_max over the cloud (positions are needed in
        // float32 only to choose candidates)
        double L = R;
        for (int b = 0; b < nblk; ++b)
            for (int d = 0; d < 3; ++d)
                L = std::max(L, part[3 * b + d]);
        L += cfg->r_max + 1.0;
        CellGrid g = make_grid(L, cfg->r_max * (1.0 + 1e-4) + 1e-3,
                               std::max<long long>(4 * (long long)n + 4096, 1 << 16));
        if (g.n_cells > w.cells_cap || n > w.cells_n) {
            // grow to hold both this droplet and the largest one seen so far
            CellGrid ga = g;
            ga.n_cells = std::max(g.n_cells, w.cells_cap);
            const int na = std::max(n, w.cells_n);
            free_cells(w.cb);
            w.cells_cap = w.cells_n = 0;
            rc = alloc_cells(ga, w.cb, na);
            if (rc)
                return rc;
            w.cells_cap = ga.n_cells;
            w.cells_n = na;
        }
        w.grid = g;
        if (cfg->n_bins > w.hist_cap) {
            dfree(w.hist);
            NP_CUDA(dalloc(&w.hist, cfg->n_bins));
            w.hist_cap = cfg->n_bins;
        }
        NP_CUDA(launch_cell_build(g, xq, typ, n, w.cb, nullptr, st));
        NP_CUDA(launch_pair_hist(x, n, cfg->r_max, cfg->n_bins, g, w.cb, w.hist, st));
        std::vector<unsigned long long> h(cfg->n_bins);
        NP_CUDA(cudaMemcpyAsync(h.data(), w.hist, sizeof(unsigned long long) * h.size(),
                                cudaMemcpyDeviceToHost, st));
        NP_CUDA(cudaStreamSynchronize(st));
        const double dr = cfg->r_max / (double)cfg->n_bins;
        const double V = 4.0 / 3.0 * pi * R * R * R;
        for (int b = 0; b < cfg->n_bins; ++b) {
            rdf_counts[b] = (int64_t)h[b];
            if (rdf_g) {
                const double r0 = b * dr, r1 = (b + 1) * dr;
                const double dV = 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
                rdf_g[b] = ((double)h[b] / (double)n) / ((double)(n - 1) * dV / V);
            }
        }
    }
    if (cfg->radial_bins > 0 && radial_counts) {
        if (cfg->radial_bins > w.rhist_cap) {
            dfree(w.rhist);
            NP_CUDA(dalloc(&w.rhist, cfg->radial_bins));
            w.rhist_cap = cfg->radial_bins;
        }
        NP_CUDA(launch_radial_hist(x, n, R, cfg->radial_bins, w.rhist, st));
        std::vector<unsigned long long> h(cfg->radial_bins);
        NP_CUDA(cudaMemcpyAsync(h.data(), w.rhist, sizeof(unsigned long long) * h.size(),
                                cudaMemcpyDeviceToHost, st));
        NP_CUDA(cudaStreamSynchronize(st));
        const double dr = R / (double)cfg->radial_bins;
        const double V = 4.0 / 3.0 * pi * R * R * R;
        for (int b = 0; b < cfg->radial_bins; ++b) {
            radial_counts[b] = (int64_t)h[b];
            if (radial_c) {
                const double r0 = b * dr, r1 = (b + 1) * dr;
                const double dV = 4.0 / 3.0 * pi * (r1 * r1 * r1 - r0 * r0 * r0);
                radial_c[b] = ((double)h[b] / (double)n) / (dV / V);
            }
        }
    }
    // N_surf: NPs in the band (-r_i, r_i) about the surface
    {
        SurfHalf hs{};
        for (int t = 0; t < T; ++t)
            hs.h[t] = 0.5 * types[t].sigma;
        unsigned long long cnt = 0;
        NP_CUDA(launch_surface_count(x, typ, n, R, hs, w.surf, st));
        NP_CUDA(cudaMemcpyAsync(&cnt, w.surf, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        NP_CUDA(cudaStreamSynchronize(st));
        out->n_surf = (int64_t)cnt;
    }
    // centre of mass and radius of gyration (Eqs. r0, Rg), fractal equation (Eq. N)
    rc = block_partials(w, 0, x, n, nullptr, part, st);
    if (rc)
        return rc;
    double c[3] = {0, 0, 0};
    for (int b = 0; b < nblk; ++b)
        for (int d = 0; d < 3; ++d)
            c[d] += part[3 * b + d];
    for (int d = 0; d < 3; ++d)
        c[d] /= (double)n;
    NP_CUDA(cudaMemcpyAsync(w.vec, c, sizeof(c), cudaMemcpyHostToDevice, st));
    rc = block_partials(w, 1, x, n, w.vec, part, st);
    if (rc)
        return rc;
    double ss = 0.0;
    for (int b = 0; b < nblk; ++b)
        ss += part[3 * b];
    const double Rg = std::sqrt(ss / (double)n);
    out->Rg = Rg;
    out->Df_rg = std::log((double)n / kKf) / std::log(2.0 * Rg / d_mean);
    for (int d = 0; d < 3; ++d)
        out->center[d] = c[d];

    out->Df_box = NAN;
    if (cfg->boxcount) {
        unsigned long long tsz = 1;
        while (tsz < 2ull * (unsigned long long)n)
            tsz <<= 1;
        if (tsz > w.table_size) {
            dfree(w.table);
            NP_CUDA(dalloc(&w.table, tsz));
            w.table_size = tsz;
        }
        NP_CUDA(cudaMemcpyAsync(w.vec + 3, o, sizeof(o), cudaMemcpyHostToDevice, st));
        int ns = 0;
        while (ns < cfg->max_scales && d_mean * std::ldexp(1.0, ns) <= 2.0 * Rg)
            ++ns;
        for (int k = 0; k < ns; ++k) {
            const double eps = d_mean * std::ldexp(1.0, k);
            NP_CUDA(launch_boxcount(x, n, w.vec + 3, eps, w.table, tsz, w.count, d_flags, st));
            int cnt = 0;
            NP_CUDA(cudaMemcpyAsync(&cnt, w.count, sizeof(int), cudaMemcpyDeviceToHost, st));
            NP_CUDA(cudaStreamSynchronize(st));
            out->nbox[k] = cnt;
        }
        out->n_scales = ns;
        if (ns - 1 >= 2) {
            // least squares of ln N_box on ln eps over scales k >= 1
            const int m = ns - 1;
            double mx = 0, my = 0;
            for (int k = 1; k < ns; ++k) {
                mx += std::log(d_mean * std::ldexp(1.0, k));
                my += std::log((double)out->nbox[k]);
            }
            mx /= m;
            my /= m;
            double sxy = 0, sxx = 0;
            for (int k = 1; k < ns; ++k) {
                const double ex = std::log(d_mean * std::ldexp(1.0, k)) - mx;
                sxy += ex * (std::log((double)out->nbox[k]) - my);
                sxx += ex * ex;
            }
            out->Df_box = -sxy / sxx;
        }
    }
    return NPSIM_OK;
}

int check_stats_cfg(const npsim_stats_cfg_t *cfg)
{
    NP_REQUIRE(cfg->n_bins >= 0 && cfg->radial_bins >= 0, "bins must be >= 0");
    NP_REQUIRE(cfg->n_bins == 0 || cfg->r_max > 0, "r_max must be positive");
    NP_REQUIRE(cfg->max_scales >= 0 && cfg->max_scales <= NPSIM_MAX_SCALES,
               "max_scales must be in [0, %d]", NPSIM_MAX_SCALES);
    return NPSIM_OK;
}

} // namespace

extern "C" {

int npsim_stats(npsim_sim_t s, const npsim_stats_cfg_t *cfg, int64_t *rdf_counts,
                double *rdf_g, int64_t *radial_counts, double *radial_c, npsim_stats_t *out)
{
    NP_TRACE();
    NP_REQUIRE(s && cfg && out, "sim, cfg and out are required");
    int rc = check_stats_cfg(cfg);
    if (rc)
        return rc;
    const double t = (double)s->step * s->P.dt;
    const double R2 = s->P.R0 * s->P.R0 - s->P.k_evap * t;
    const double R = R2 > 0 ? std::sqrt(R2) : 0.0;
    rc = positions_f64(s);
    if (rc)
        return rc;
    rc = stats_core(s->sw, s->x, s->xq, s->typ, s->n, R, s->d_mean, s->types, s->P.n_types,
                    s->d_flags, cfg, rdf_counts, rdf_g, radial_counts, radial_c, out, s->user);
    if (rc)
        return rc;
    return read_flags(s);
}

// ---------------------------------------------------------------------------
// Checkpoints

namespace {
// Layout: header, then the raw state words so that a resumed run is
// bit-identical: position hi words [3][n], lo words [3][n], velocities [3][n]
// (float32 SoA), the types (int32[n]) and the order of the NPs inside their
// type groups (int32[n], the pair kernels' summation order); with a cell list
// also the neighbour-list state: the cell grid and list capacity (header), the
// positions of the last build (float4[n]) and the rebuild gate (header), from
// which a resumed run rebuilds exactly the list the saved run was using.
const char kMagic[8] = {'N', 'P', 'S', 'I', 'M', 'C', 'K', '5'};

struct CkptHeader {
    char magic[8];
    int32_t version, n_types;
    int64_t n, step;
    int32_t rot_mode, lj_mode, coulomb, wall, integrator, has_ov, sum_neutral, pad_;
    uint64_t seed;
    double dt, kT, R0, k_evap, g, omega, bjerrum, lj_cut, v_kick, coulomb_cut;
    double eps_ov[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    npsim_type_t types[NPSIM_MAX_TYPES];
    int32_t cell, grid_dim, grid_cells, nbr_cap, gate, pad2_;
    float grid_inv_h, grid_L;
};

// Put the neighbour-list state of a checkpoint back: the saved grid and list
// capacity, a build from the saved build positions (which writes the same
// lists and x_ref), and the saved gate.
int restore_lists(npsim_sim *s, const CkptHeader &h, const float4 *x_ref_host)
{
    if (!s->cell || !h.cell)
        return NPSIM_OK;
    CellGrid g{};
    g.dim = h.grid_dim;
    g.n_cells = h.grid_cells;
    g.inv_h = h.grid_inv_h;
    g.L = h.grid_L;
    g.tb = s->T;
    set_extents(g, s->rlist);
    int rc0 = ensure_cells(s, g);
    if (rc0)
        return rc0;
    s->grid = g;
    if (h.nbr_cap != s->nl.cap) {
        dfree(s->nl.nbr);
        NP_CUDA(dalloc(&s->nl.nbr, (size_t)h.nbr_cap * s->n));
        s->nl.cap = h.nbr_cap;
    }
    for (auto &e : s->graphs)
        cudaGraphExecDestroy(e.second);
    s->graphs.clear();
    NP_CUDA(cudaMemcpy(s->nl.x_ref, x_ref_host, sizeof(float4) * (size_t)s->n,
                       cudaMemcpyHostToDevice));
    NP_CUDA(launch_cell_build(s->grid, s->nl.x_ref, s->typ, s->n, s->cb, nullptr, s->user));
    NP_CUDA(launch_nbr_build(s->grid, s->cb, s->n, s->tab_full, s->d_rcc2, kSkin, s->nl,
                             s->d_flags,
                             nullptr, s->user));
    // the list kernel reads the current positions from the cell-ordered records
    NP_CUDA(launch_cell_refresh(s->cb, s->xq, s->typ, s->n, s->user));
    NP_CUDA(cudaStreamSynchronize(s->user));
    return set_gate(s, h.gate);
}
} // namespace

int npsim_scattering(const double *g, int32_t n_bins, double r_max, double n_surf, double Rg,
                     double Df, const double *q, int32_t n_q, double *I, double *I_frac)
{
    NP_TRACE();
    NP_REQUIRE(g && q && I, "g, q and I are required");
    NP_REQUIRE(n_bins >= 1 && n_q >= 1, "n_bins and n_q must be >= 1");
    NP_REQUIRE(r_max > 0 && std::isfinite(r_max), "r_max must be positive");
    for (int k = 0; k < n_q; ++k)
        NP_REQUIRE(q[k] >= 0 && std::isfinite(q[k]), "q[%d] must be finite and >= 0", k);
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
        return set_err(NPSIM_ERR_NO_DEVICE, "no CUDA device visible");
    double *dg = nullptr, *dq = nullptr, *dI = nullptr, *dF = nullptr;
    auto release = [&]() {
        dfree(dg);
        dfree(dq);
        dfree(dI);
        dfree(dF);
    };
    cudaError_t e = dalloc(&dg, (size_t)n_bins);
    if (e == cudaSuccess)
        e = dalloc(&dq, (size_t)n_q);
    if (e == cudaSuccess)
        e = dalloc(&dI, (size_t)n_q);
    if (e == cudaSuccess && I_frac)
        e = dalloc(&dF, (size_t)n_q);
    if (e == cudaSuccess)
        e = cudaMemcpy(dg, g, sizeof(double) * n_bins, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dq, q, sizeof(double) * n_q, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_scattering(dg, n_bins, r_max, dq, n_q, n_surf, Rg, Df, dI, dF, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(I, dI, sizeof(double) * n_q, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && I_frac)
        e = cudaMemcpy(I_frac, dF, sizeof(double) * n_q, cudaMemcpyDeviceToHost);
    release();
    if (e != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "npsim_scattering: %s", cudaGetErrorString(e));
    return NPSIM_OK;
}

int npsim_save(npsim_sim_t s, const char *path)
{
    NP_TRACE();
    NP_REQUIRE(s && path, "sim and path are required");
    CkptHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.version = 5;
    h.n_types = s->T;
    h.n = s->n;
    h.step = s->step;
    h.rot_mode = s->P.rot_mode;
    h.lj_mode = s->P.lj_mode;
    h.coulomb = s->P.coulomb;
    h.wall = s->P.wall;
    h.integrator = s->P.integrator;
    h.has_ov = s->has_ov ? 1 : 0;
    h.sum_neutral = s->P.sum_neutral;
    h.seed = s->P.seed;
    h.dt = s->P.dt;
    h.kT = s->P.kT;
    h.R0 = s->P.R0;
    h.k_evap = s->P.k_evap;
    h.g = s->P.g;
    h.omega = s->P.omega;
    h.bjerrum = s->P.bjerrum;
    h.lj_cut = s->P.lj_cut;
    h.v_kick = s->P.v_kick;
    h.coulomb_cut = s->P.coulomb_cut;
    memcpy(h.eps_ov, s->eps_ov, sizeof(h.eps_ov));
    memcpy(h.types, s->types, sizeof(h.types));
    const size_t n = (size_t)s->n;
    NP_CUDA(cudaStreamSynchronize(s->user));
    std::vector<float4> xq(n);
    std::vector<float> words(9 * n);
    NP_CUDA(cudaMemcpy(xq.data(), s->xq, sizeof(float4) * n, cudaMemcpyDeviceToHost));
    NP_CUDA(cudaMemcpy(words.data() + 3 * n, s->x_lo, sizeof(float) * 3 * n,
                       cudaMemcpyDeviceToHost));
    NP_CUDA(cudaMemcpy(words.data() + 6 * n, s->v, sizeof(float) * 3 * n,
                       cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) {
        words[i] = xq[i].x;
        words[n + i] = xq[i].y;
        words[2 * n + i] = xq[i].z;
    }
    FILE *f = fopen(path, "wb");
    if (!f)
        return set_err(NPSIM_ERR_IO, "cannot open %s for writing", path);
    std::vector<int32_t> rank(s->h_rank);
    rank.resize(n, 0);
    std::vector<float4> xref;
    if (s->cell) {
        h.cell = 1;
        h.grid_dim = s->grid.dim;
        h.grid_cells = s->grid.n_cells;
        h.grid_inv_h = s->grid.inv_h;
        h.grid_L = s->grid.L;
        h.nbr_cap = s->nl.cap;
        NP_CUDA(cudaMemcpy(&h.gate, s->d_gate, sizeof(int), cudaMemcpyDeviceToHost));
        xref.resize(n);
        NP_CUDA(cudaMemcpy(xref.data(), s->nl.x_ref, sizeof(float4) * n, cudaMemcpyDeviceToHost));
    }
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 &&
              fwrite(words.data(), sizeof(float), words.size(), f) == words.size() &&
              fwrite(s->h_type.data(), sizeof(int32_t), s->h_type.size(), f) ==
                  s->h_type.size() &&
              fwrite(rank.data(), sizeof(int32_t), rank.size(), f) == rank.size() &&
              fwrite(xref.data(), sizeof(float4), xref.size(), f) == xref.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok)
        return set_err(NPSIM_ERR_IO, "short write to %s", path);
    return NPSIM_OK;
}

int npsim_load(const char *path, const npsim_type_t *types_override,
               const npsim_params_t *params_override, void *stream, npsim_sim_t *out)
{
    NP_TRACE();
    NP_REQUIRE(path && out, "path and out are required");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f)
        return set_err(NPSIM_ERR_IO, "cannot open %s", path);
    CkptHeader h{};
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 5 ||
        h.n < 1 || h.n > (1ll << 29) || h.n_types < 1 || h.n_types > NPSIM_MAX_TYPES) {
        fclose(f);
        return set_err(NPSIM_ERR_IO, "%s is not an npsim checkpoint", path);
    }
    const size_t n = (size_t)h.n;
    std::vector<float> words(9 * n);
    std::vector<int32_t> ty(n), rank(n);
    std::vector<float4> xref(h.cell ? n : 0);
    bool ok = fread(words.data(), sizeof(float), words.size(), f) == words.size() &&
              fread(ty.data(), sizeof(int32_t), ty.size(), f) == ty.size() &&
              fread(rank.data(), sizeof(int32_t), rank.size(), f) == rank.size() &&
              fread(xref.data(), sizeof(float4), xref.size(), f) == xref.size();
    fclose(f);
    if (!ok)
        return set_err(NPSIM_ERR_IO, "%s is truncated", path);
    // float64 values (AoS) for creation: x = hi + lo, v
    std::vector<double> x(3 * n), v(3 * n);
    for (size_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            x[3 * i + d] = (double)words[d * n + i] + (double)words[(3 + d) * n + i];
            v[3 * i + d] = (double)words[(6 + d) * n + i];
        }
    npsim_params_t p{};
    p.n_types = h.n_types;
    p.rot_mode = h.rot_mode;
    p.lj_mode = h.lj_mode;
    p.coulomb = h.coulomb;
    p.wall = h.wall;
    p.integrator = h.integrator;
    p.sum_neutral = h.sum_neutral;
    p.seed = h.seed;
    p.dt = h.dt;
    p.kT = h.kT;
    p.R0 = h.R0;
    p.k_evap = h.k_evap;
    p.g = h.g;
    p.omega = h.omega;
    p.bjerrum = h.bjerrum;
    p.lj_cut = h.lj_cut;
    p.v_kick = h.v_kick;
    p.coulomb_cut = h.coulomb_cut;
    p.eps_override = h.has_ov ? h.eps_ov : nullptr;
    if (params_override) {
        p = *params_override;
        NP_REQUIRE(p.n_types == h.n_types, "params_override changes n_types");
    }
    const npsim_type_t *tys = types_override ? types_override : h.types;
    npsim_sim_t s = nullptr;
    int rc = create_impl(tys, &p, h.n, x.data(), v.data(), ty.data(), stream, rank.data(), &s);
    if (rc)
        return rc;
    rc = upload_words(s, words.data(), h.step);
    if (!rc && h.cell) { // the saved list state, then the forces from it
        rc = restore_lists(s, h, xref.data());
        if (!rc)
            rc = finish_upload(s, h.step, false);
    }
    if (rc) {
        npsim_destroy(s);
        return rc;
    }
    *out = s;
    return NPSIM_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Ensemble of independent droplets

struct npsim_ens {
    int D = 0, n_total = 0, sms = 0;
    std::vector<int> off, cnt;
    std::vector<EnsDrop> h_drops;
    std::vector<PairTab> h_tabs;
    std::vector<npsim_params_t> P;
    std::vector<std::vector<npsim_type_t>> types;
    std::vector<std::vector<double>> eps_ov;
    std::vector<int32_t> h_type;

    cudaStream_t user = nullptr, cap = nullptr;
    // state layouts as in npsim_sim, over the concatenation of the droplets
    float *x_lo = nullptr, *v = nullptr;  // [3][n_total]
    float *F = nullptr, *F_tmp = nullptr; // [6][n_total]
    float4 *xq = nullptr;
    int *typ = nullptr, *drop_of = nullptr;
    int *perm = nullptr, *tblk = nullptr, *row_pos = nullptr; // type-grouped order
    EnsDrop *drops = nullptr;
    PairTab *tabs = nullptr;
    long long *item0 = nullptr;  // work-item prefix per droplet (n_drops + 1)
    unsigned *d_work = nullptr;  // work-item counters of the all-pairs launch
    float *slots = nullptr;      // one [6][itile] slot per work item
    long long *d_step = nullptr;
    float4 *d_spring = nullptr; // [2][D][NPSIM_MAX_TYPES]
    int *d_flags = nullptr;
    unsigned *d_done = nullptr;

    int shape = 0;
    StreamK sk{};
    int chunk = 1;          // j-tiles per work item
    long long n_items = 0;  // work items of one all-pairs launch
    std::map<int, cudaGraphExec_t> graphs;
    int64_t step = 0;
    // kernel timing (npsim_ens_profile): events around the all-pairs launch
    // (group 0) and the integrator launch (group 1) of every pass of a chunk
    bool profiling = false;
    int last_chunk = 0;
    cudaEvent_t ev[kChunk][2][2]{};

    std::vector<double> d_mean; // number-mean NP diameter of each droplet
    StatsWork sw{};             // statistics of one droplet at a time (lazy)

    ~npsim_ens()
    {
        free_stats(sw);
        for (auto &g : graphs)
            cudaGraphExecDestroy(g.second);
        for (auto &a : ev)
            for (auto &b : a)
                for (auto &x : b)
                    if (x)
                        cudaEventDestroy(x);
        dfree(x_lo);
        dfree(v);
        dfree(F);
        dfree(F_tmp);
        dfree(xq);
        dfree(typ);
        dfree(drop_of);
        dfree(perm);
        dfree(tblk);
        dfree(row_pos);
        dfree(drops);
        dfree(tabs);
        dfree(item0);
        dfree(d_work);
        dfree(slots);
        dfree(d_step);
        dfree(d_spring);
        dfree(d_flags);
        dfree(d_done);
        if (cap)
            cudaStreamDestroy(cap);
    }
};

namespace {

// Work items per CTA that the chunk size aims at: enough that the last items
// drawn (the only imbalance of dynamic scheduling) are short, few enough that
// the per-item slots stay small.
constexpr int kItemsPerCta = 32;

// Droplet geometry for launch shape `shape` on grid_target CTAs: row tiles and
// j-tiles of every droplet, the chunk size (j-tiles per work item) and the
// work items laid end to end (item0).  Returns the number of items; *chunk_out
// receives the chunk size.
long long ens_geometry(npsim_ens *e, int shape, int grid_target, std::vector<long long> &item0,
                       int *chunk_out)
{
    const ApConfig c = ens_config(shape);
    const int itile = c.block * c.ki;
    long long W = 0;
    for (int d = 0; d < e->D; ++d) {
        EnsDrop &g = e->h_drops[d];
        g.n_it = (g.npad + itile - 1) / itile;
        g.n_jt = g.npad / c.jt; // npad is a multiple of 256, jt divides 256
        W += (long long)g.n_it * g.n_jt;
    }
    const long long target = (long long)std::max(grid_target, 1) * kItemsPerCta;
    const int chunk = (int)std::max<long long>(1, (W + target - 1) / target);
    long long it = 0;
    item0.assign(e->D + 1, 0);
    for (int d = 0; d < e->D; ++d) {
        EnsDrop &g = e->h_drops[d];
        g.n_ch = (g.n_jt + chunk - 1) / chunk;
        g.item0 = it;
        item0[d] = it;
        it += (long long)g.n_it * g.n_ch;
    }
    item0[e->D] = it;
    if (chunk_out)
        *chunk_out = chunk;
    return it;
}

void ens_streamk(long long n_items, const ApConfig &c, int grid_target, StreamK &sk)
{
    sk.itile = c.block * c.ki;
    sk.jtile = c.jt;
    sk.n_it = 0;
    sk.n_jt = 0;
    sk.W = n_items;
    sk.grid = (int)std::min<long long>(std::max(grid_target, 1), n_items);
    sk.ctas = 0;
}

int ens_upload_geometry(npsim_ens *e, const std::vector<long long> &item0)
{
    NP_CUDA(cudaMemcpyAsync(e->drops, e->h_drops.data(), sizeof(EnsDrop) * e->D,
                            cudaMemcpyHostToDevice, e->user));
    NP_CUDA(cudaMemcpyAsync(e->item0, item0.data(), sizeof(long long) * item0.size(),
                            cudaMemcpyHostToDevice, e->user));
    NP_CUDA(cudaStreamSynchronize(e->user));
    return NPSIM_OK;
}

EnsAllpairsArgs ens_ap_args(npsim_ens *e, float *slots)
{
    EnsAllpairsArgs a{};
    a.xq = e->xq;
    a.perm = e->perm;
    a.tblk = e->tblk;
    a.drops = e->drops;
    a.item0 = e->item0;
    a.tabs = e->tabs;
    a.n_drops = e->D;
    a.chunk = e->chunk;
    a.n_items = e->n_items;
    a.work = e->d_work;
    a.slots = slots;
    return a;
}

int ens_pass(npsim_ens *e, int mode, bool ext, float *Fout, cudaStream_t st,
             int prof_slot = -1)
{
    const bool prof = prof_slot >= 0 && e->profiling;
    // inside stream capture the External flag makes each record a real
    // event-record node of the graph
    auto mark = [&](int group, int edge) -> cudaError_t {
        return prof ? cudaEventRecordWithFlags(e->ev[prof_slot][group][edge], st,
                                               cudaEventRecordExternal)
                    : cudaSuccess;
    };
    NP_CUDA(mark(0, 0));
    NP_CUDA(launch_ens_allpairs(e->shape, e->sk, ens_ap_args(e, e->slots), st));
    NP_CUDA(mark(0, 1));
    EnsIntArgs a{};
    a.x_lo = e->x_lo;
    a.v = e->v;
    a.F = Fout;
    a.typ = e->typ;
    a.xq = e->xq;
    a.drop_of = e->drop_of;
    a.row_pos = e->row_pos;
    a.drops = e->drops;
    a.slots = e->slots;
    a.spring = e->d_spring;
    a.ext_on = ext ? 1 : 0;
    a.step = e->d_step;
    a.flags = e->d_flags;
    a.done = e->d_done;
    NP_CUDA(mark(1, 0));
    NP_CUDA(launch_ens_integrate(mode, a, e->n_total, e->D, e->sk, st));
    NP_CUDA(mark(1, 1));
    return NPSIM_OK;
}

int ens_chunk(npsim_ens *e, int k, cudaStream_t st)
{
    EnsIntArgs a{};
    a.x_lo = e->x_lo;
    a.v = e->v;
    a.F = e->F;
    a.typ = e->typ;
    a.xq = e->xq;
    a.drop_of = e->drop_of;
    a.row_pos = e->row_pos;
    a.drops = e->drops;
    a.spring = e->d_spring;
    a.step = e->d_step;
    a.flags = e->d_flags;
    a.done = e->d_done;
    NP_CUDA(launch_ens_integrate(MODE_A, a, e->n_total, e->D, e->sk, st));
    for (int j = 0; j < k; ++j) {
        int rc = ens_pass(e, j + 1 < k ? MODE_BA : MODE_B, true, e->F, st, j);
        if (rc)
            return rc;
    }
    return NPSIM_OK;
}

int ens_graph(npsim_ens *e, int k, cudaGraphExec_t *out)
{
    auto it = e->graphs.find(k);
    if (it != e->graphs.end()) {
        *out = it->second;
        return NPSIM_OK;
    }
    NP_CUDA(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
    int rc = ens_chunk(e, k, e->cap);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->cap, &g);
    if (rc) {
        if (g)
            cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    cudaGraphExec_t ex = nullptr;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
    e->graphs[k] = ex;
    *out = ex;
    return NPSIM_OK;
}

// Time every ensemble launch shape on the current positions; keep the fastest.
int ens_autotune(npsim_ens *e)
{
    const int nc = ens_num_configs();
    const char *env = getenv("NPSIM_ENS_SHAPE");
    std::vector<long long> item0;
    int best = -1;
    if (env) {
        const int idx = atoi(env);
        if (idx >= 0 && idx < nc && ens_occupancy(idx) > 0)
            best = idx;
    }
    // the same ensemble geometry gets the same shape within a process (so
    // that repeated runs of one ensemble sum in the same order)
    std::vector<long long> key;
    for (int d = 0; d < e->D; ++d) {
        const EnsDrop &g = e->h_drops[d];
        key.push_back(((long long)g.npad << 2) | (g.rc2_lim > 0.0f ? 2 : 0) |
                      (g.has_coul ? 1 : 0));
    }
    const bool pinned = best >= 0;
    if (!pinned) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_ens_tune_cache.find(key);
        if (it != g_ens_tune_cache.end())
            best = it->second;
    }
    const bool cached = !pinned && best >= 0;
    if (best < 0) {
        size_t need = 0;
        for (int c = 0; c < nc; ++c) {
            const int occ = ens_occupancy(c);
            if (occ <= 0)
                continue;
            const long long items = ens_geometry(e, c, occ * e->sms, item0, nullptr);
            const ApConfig cc = ens_config(c);
            need = std::max(need, (size_t)items * 6 * (size_t)(cc.block * cc.ki));
        }
        float *tmp = nullptr;
        NP_CUDA(dalloc(&tmp, need));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best_ms = 1e30f;
        for (int c = 0; c < nc; ++c) {
            const int occ = ens_occupancy(c);
            if (occ <= 0)
                continue;
            e->n_items = ens_geometry(e, c, occ * e->sms, item0, &e->chunk);
            int rc = ens_upload_geometry(e, item0);
            if (rc) {
                cudaFree(tmp);
                return rc;
            }
            StreamK sk;
            ens_streamk(e->n_items, ens_config(c), occ * e->sms, sk);
            e->shape = c;
            if (launch_ens_allpairs(c, sk, ens_ap_args(e, tmp), e->user) != cudaSuccess)
                continue;
            cudaEventRecord(e0, e->user);
            for (int r = 0; r < 2; ++r)
                launch_ens_allpairs(c, sk, ens_ap_args(e, tmp), e->user);
            cudaEventRecord(e1, e->user);
            if (cudaEventSynchronize(e1) != cudaSuccess)
                continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (getenv("NPSIM_AUTOTUNE_LOG")) {
                const ApConfig cf = ens_config(c);
                fprintf(stderr, "npsim ensemble autotune shape %d <%d,%d,%d> grid %d: %.4f ms\n",
                        c, cf.block, cf.ki, cf.jt, sk.grid, ms / 2);
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(tmp);
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess)
            return set_err(NPSIM_ERR_CUDA, "ensemble autotune: %s", cudaGetErrorString(ce));
        if (best < 0)
            best = 0;
    }
    if (!pinned && !cached) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_ens_tune_cache[key] = best;
    }
    e->shape = best;
    const int grid_target = std::max(1, ens_occupancy(best)) * e->sms;
    e->n_items = ens_geometry(e, best, grid_target, item0, &e->chunk);
    ens_streamk(e->n_items, ens_config(best), grid_target, e->sk);
    int rc = ens_upload_geometry(e, item0);
    if (rc)
        return rc;
    NP_CUDA(dalloc(&e->slots, (size_t)e->n_items * 6 * (size_t)e->sk.itile));
    return NPSIM_OK;
}

} // namespace

extern "C" {

int npsim_ens_create(const npsim_droplet_t *drops, int32_t n_drops, void *stream,
                     npsim_ens_t *out)
{
    NP_TRACE();
    NP_REQUIRE(out, "out is NULL");
    *out = nullptr;
    NP_REQUIRE(drops && n_drops >= 1, "need at least one droplet");
    long long total = 0;
    for (int d = 0; d < n_drops; ++d) {
        const npsim_droplet_t &dr = drops[d];
        int rc = validate(dr.types, &dr.params, dr.n);
        if (rc)
            return set_err(rc, "droplet %d: %s", d, g_err.c_str());
        NP_REQUIRE(dr.params.lj_mode != 2, "droplet %d: the ensemble sums LJ inside the all-pairs "
                                           "kernel (lj_mode 0 or 1)", d);
        NP_REQUIRE(dr.x0 && dr.type, "droplet %d: x0 and type are required", d);
        for (int64_t i = 0; i < dr.n; ++i)
            NP_REQUIRE(dr.type[i] >= 0 && dr.type[i] < dr.params.n_types,
                       "droplet %d: type[%lld] out of range", d, (long long)i);
        total += dr.n;
    }
    NP_REQUIRE(total <= (1ll << 29), "too many particles in the ensemble");
    int sms = 0;
    int rc = check_device(&sms);
    if (rc)
        return rc;

    npsim_ens *e = new npsim_ens();
    auto bail = [&](int code) {
        delete e;
        return code;
    };
    e->D = n_drops;
    e->n_total = (int)total;
    e->sms = sms;
    e->user = (cudaStream_t)stream;
    e->off.resize(n_drops);
    e->cnt.resize(n_drops);
    e->h_drops.assign(n_drops, EnsDrop{});
    e->h_tabs.assign(n_drops, PairTab{});
    e->P.resize(n_drops);
    e->types.resize(n_drops);
    e->eps_ov.resize(n_drops);
    e->d_mean.assign(n_drops, 1.0);
    std::vector<double> xs(3 * (size_t)total), vs(3 * (size_t)total, 0.0);
    std::vector<int> dof((size_t)total);
    std::vector<float4> xq0((size_t)total);
    e->h_type.resize((size_t)total);
    int off = 0;
    for (int d = 0; d < n_drops; ++d) {
        const npsim_droplet_t &dr = drops[d];
        const int n = (int)dr.n;
        e->off[d] = off;
        e->cnt[d] = n;
        e->P[d] = dr.params;
        e->types[d].assign(dr.types, dr.types + dr.params.n_types);
        if (dr.params.eps_override)
            e->eps_ov[d].assign(dr.params.eps_override,
                                dr.params.eps_override + dr.params.n_types * dr.params.n_types);
        e->P[d].eps_override = nullptr;
        EnsDrop &g = e->h_drops[d];
        g.offset = off;
        g.n = n;
        g.rot_mode = dr.params.rot_mode;
        g.wall = dr.params.wall;
        g.integrator = dr.params.integrator;
        g.seed = dr.params.seed;
        g.dt = dr.params.dt;
        g.R0 = dr.params.R0;
        g.k_evap = dr.params.k_evap;
        g.g = dr.params.g;
        g.omega2 = dr.params.omega * dr.params.omega;
        float qf[NPSIM_MAX_TYPES] = {};
        fill_coefs(dr.types, &dr.params, g.tc, qf);
        npsim_params_t pc = dr.params;
        if (pc.lj_mode == 0) { // no LJ: zero the LJ columns of the table
            pc.lj_cut = 0.0;
        }
        fill_tabs(dr.types, &pc, e->eps_ov[d].empty() ? nullptr : e->eps_ov[d].data(),
                  &e->h_tabs[d], nullptr);
        if (pc.lj_mode == 0)
            for (int k = 0; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; ++k) {
                e->h_tabs[d].e[k].y = 0.0f;
                e->h_tabs[d].e[k].z = 0.0f;
            }
        g.rc2_lim = 0.0f;
        g.has_coul = 0;
        for (int k = 0; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; ++k) {
            const float4 t = e->h_tabs[d].e[k];
            if (t.y != 0.0f)
                g.rc2_lim = std::max(g.rc2_lim, t.z * 1.0001f);
            if (t.w != 0.0f)
                g.has_coul = 1;
        }
        double dsum = 0.0;
        for (int i = 0; i < n; ++i)
            dsum += dr.types[dr.type[i]].sigma;
        e->d_mean[d] = dsum / (double)n;
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < 3; ++k) {
                xs[(size_t)k * total + off + i] = dr.x0[3 * (size_t)i + k];
                if (dr.v0)
                    vs[(size_t)k * total + off + i] = dr.v0[3 * (size_t)i + k];
            }
            dof[off + i] = d;
            e->h_type[off + i] = dr.type[i];
        }
        off += n;
    }
    // type-grouped order of every droplet: its types in order, each group in
    // Z-order of the initial positions and padded with -1 to a multiple of 256
    std::vector<int> gperm, gtblk, gpos((size_t)total, -1);
    for (int d = 0; d < n_drops; ++d) {
        EnsDrop &g = e->h_drops[d];
        g.gpos0 = (int)gperm.size();
        for (int t = 0; t < drops[d].params.n_types; ++t) {
            std::vector<int> mem;
            for (int i = 0; i < e->cnt[d]; ++i)
                if (drops[d].type[i] == t)
                    mem.push_back(i);
            if (mem.empty())
                continue;
            morton_sort(mem, drops[d].x0);
            for (int i : mem) {
                gpos[(size_t)e->off[d] + i] = (int)gperm.size();
                gperm.push_back(e->off[d] + i);
            }
            while (gperm.size() % 256)
                gperm.push_back(-1);
            while (gtblk.size() < gperm.size() / 256)
                gtblk.push_back(t);
        }
        g.npad = (int)gperm.size() - g.gpos0;
    }
#define EBAIL(call)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return bail(set_err(e_ == cudaErrorMemoryAllocation ? NPSIM_ERR_OOM         \
                                                                 : NPSIM_ERR_CUDA,      \
                                "%s failed: %s", #call, cudaGetErrorString(e_)));       \
    } while (0)
    EBAIL(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking));
    const size_t n3 = 3 * (size_t)total;
    EBAIL(dalloc(&e->x_lo, n3));
    EBAIL(dalloc(&e->v, n3));
    EBAIL(dalloc(&e->F, 2 * n3));
    EBAIL(dalloc(&e->F_tmp, 2 * n3));
    EBAIL(dalloc(&e->xq, (size_t)total));
    EBAIL(dalloc(&e->typ, (size_t)total));
    EBAIL(dalloc(&e->drop_of, (size_t)total));
    EBAIL(dalloc(&e->drops, (size_t)n_drops));
    EBAIL(dalloc(&e->tabs, (size_t)n_drops));
    EBAIL(dalloc(&e->item0, (size_t)n_drops + 1));
    EBAIL(dalloc(&e->d_work, 2));
    EBAIL(cudaMemset(e->d_work, 0, 2 * sizeof(unsigned)));
    EBAIL(dalloc(&e->d_step, 1));
    EBAIL(dalloc(&e->d_spring, (size_t)2 * n_drops * NPSIM_MAX_TYPES));
    EBAIL(dalloc(&e->d_flags, 1));
    EBAIL(dalloc(&e->d_done, 1));
    {
        // position = hi (nearest float, in xq) + lo (the float nearest the rest)
        std::vector<float> lo(n3), vf(vs.begin(), vs.end());
        for (size_t k = 0; k < n3; ++k)
            lo[k] = (float)(xs[k] - (double)(float)xs[k]);
        EBAIL(cudaMemcpy(e->x_lo, lo.data(), sizeof(float) * n3, cudaMemcpyHostToDevice));
        EBAIL(cudaMemcpy(e->v, vf.data(), sizeof(float) * n3, cudaMemcpyHostToDevice));
    }
    EBAIL(cudaMemcpy(e->typ, e->h_type.data(), sizeof(int) * (size_t)total,
                     cudaMemcpyHostToDevice));
    EBAIL(cudaMemcpy(e->drop_of, dof.data(), sizeof(int) * (size_t)total,
                     cudaMemcpyHostToDevice));
    EBAIL(dalloc(&e->perm, gperm.size()));
    EBAIL(dalloc(&e->tblk, gtblk.size()));
    EBAIL(dalloc(&e->row_pos, (size_t)total));
    EBAIL(cudaMemcpy(e->perm, gperm.data(), sizeof(int) * gperm.size(), cudaMemcpyHostToDevice));
    EBAIL(cudaMemcpy(e->tblk, gtblk.data(), sizeof(int) * gtblk.size(), cudaMemcpyHostToDevice));
    EBAIL(cudaMemcpy(e->row_pos, gpos.data(), sizeof(int) * (size_t)total,
                     cudaMemcpyHostToDevice));
    EBAIL(cudaMemcpy(e->tabs, e->h_tabs.data(), sizeof(PairTab) * (size_t)n_drops,
                     cudaMemcpyHostToDevice));
    for (int i = 0; i < (int)total; ++i) {
        const int d = dof[i];
        const float q = (float)e->types[d][e->h_type[i]].charge;
        xq0[i] = make_float4((float)xs[i], (float)xs[total + i], (float)xs[2 * total + i], q);
    }
    EBAIL(cudaMemcpy(e->xq, xq0.data(), sizeof(float4) * (size_t)total, cudaMemcpyHostToDevice));
    EBAIL(cudaMemset(e->d_step, 0, sizeof(long long)));
    {
        // spring radii of step 0 (buffer 0)
        std::vector<float4> sp((size_t)2 * n_drops * NPSIM_MAX_TYPES, make_float4(0, 0, 0, 0));
        for (int d = 0; d < n_drops; ++d)
            for (int t = 0; t < drops[d].params.n_types; ++t)
                sp[(size_t)d * NPSIM_MAX_TYPES + t] =
                    spring_entry(drops[d].params.R0, drops[d].params.k_evap, drops[d].params.dt,
                                 0, 0.5 * drops[d].types[t].sigma);
        EBAIL(cudaMemcpy(e->d_spring, sp.data(), sizeof(float4) * sp.size(),
                         cudaMemcpyHostToDevice));
    }
    EBAIL(cudaMemset(e->d_flags, 0, sizeof(int)));
    EBAIL(cudaMemset(e->d_done, 0, sizeof(unsigned)));
#undef EBAIL
    rc = ens_autotune(e);
    if (rc)
        return bail(rc);
    rc = ens_pass(e, MODE_FORCES, true, e->F, e->user);
    if (rc)
        return bail(rc);
    if (cudaStreamSynchronize(e->user) != cudaSuccess)
        return bail(set_err(NPSIM_ERR_CUDA, "initial forces failed"));
    *out = e;
    return NPSIM_OK;
}

void npsim_ens_destroy(npsim_ens_t e)
{
    NP_TRACE();
    if (!e)
        return;
    cudaStreamSynchronize(e->user);
    delete e;
}

int npsim_ens_step(npsim_ens_t e, int64_t n_steps)
{
    NP_TRACE();
    NP_REQUIRE(e, "ensemble is NULL");
    NP_REQUIRE(n_steps >= 0, "n_steps must be >= 0");
    int64_t rem = n_steps;
    while (rem > 0) {
        const int k = (int)std::min<int64_t>(rem, kChunk);
        cudaGraphExec_t ex = nullptr;
        int rc = ens_graph(e, k, &ex);
        if (rc)
            return rc;
        NP_CUDA(cudaGraphLaunch(ex, e->user));
        rem -= k;
        e->step += k;
        e->last_chunk = k;
    }
    int h = 0;
    NP_CUDA(cudaMemcpyAsync(&h, e->d_flags, sizeof(int), cudaMemcpyDeviceToHost, e->user));
    NP_CUDA(cudaStreamSynchronize(e->user));
    if (h) {
        NP_CUDA(cudaMemsetAsync(e->d_flags, 0, sizeof(int), e->user));
        if (!(h & FLAG_NONFINITE) && (h & FLAG_ESCAPED))
            return set_err(NPSIM_ERR_ESCAPED,
                           "an NP was farther than 2 max(R0, R(t)) from its droplet's centre");
        return set_err(NPSIM_ERR_NONFINITE, "a position became non-finite");
    }
    return NPSIM_OK;
}

int npsim_ens_profile(npsim_ens_t e, int enable)
{
    NP_REQUIRE(e, "ensemble is NULL");
    NP_CUDA(cudaStreamSynchronize(e->user));
    if (enable && !e->ev[0][0][0]) {
        for (auto &a : e->ev)
            for (auto &b : a)
                for (auto &x : b)
                    NP_CUDA(cudaEventCreate(&x));
    }
    if ((enable != 0) != e->profiling) {
        for (auto &g : e->graphs)
            cudaGraphExecDestroy(g.second);
        e->graphs.clear();
        e->profiling = enable != 0;
        e->last_chunk = 0;
    }
    return NPSIM_OK;
}

int npsim_ens_kernel_times(npsim_ens_t e, double *ms, int *samples)
{
    NP_REQUIRE(e && ms, "ensemble and ms are required");
    NP_REQUIRE(e->profiling, "profiling is not enabled (npsim_ens_profile)");
    NP_CUDA(cudaStreamSynchronize(e->user));
    const int k = e->last_chunk;
    for (int g = 0; g < 2; ++g) {
        double tot = 0.0;
        for (int j = 0; j < k; ++j) {
            float t = 0.f;
            NP_CUDA(cudaEventElapsedTime(&t, e->ev[j][g][0], e->ev[j][g][1]));
            tot += t;
        }
        ms[g] = k > 0 ? tot / k : 0.0;
    }
    if (samples)
        *samples = k;
    return NPSIM_OK;
}

int npsim_ens_get_state(npsim_ens_t e, int32_t d, double *x, double *v, double *F,
                        int64_t *step)
{
    NP_TRACE();
    NP_REQUIRE(e && d >= 0 && d < e->D, "bad ensemble or droplet index");
    NP_CUDA(cudaStreamSynchronize(e->user));
    const int n = e->cnt[d], off = e->off[d];
    const size_t N = (size_t)e->n_total;
    std::vector<float> a((size_t)n), b((size_t)n);
    // component c of droplet d's rows of a [k][N] float array
    auto rows = [&](const float *src, int c, std::vector<float> &dst) -> cudaError_t {
        return cudaMemcpy(dst.data(), src + c * N + off, sizeof(float) * (size_t)n,
                          cudaMemcpyDeviceToHost);
    };
    if (x) {
        std::vector<float4> h((size_t)n);
        NP_CUDA(cudaMemcpy(h.data(), e->xq + off, sizeof(float4) * (size_t)n,
                           cudaMemcpyDeviceToHost));
        for (int c = 0; c < 3; ++c) {
            NP_CUDA(rows(e->x_lo, c, a));
            for (int i = 0; i < n; ++i) {
                const float hi = c == 0 ? h[i].x : c == 1 ? h[i].y : h[i].z;
                x[3 * (size_t)i + c] = (double)hi + (double)a[i];
            }
        }
    }
    for (int c = 0; v && c < 3; ++c) {
        NP_CUDA(rows(e->v, c, a));
        for (int i = 0; i < n; ++i)
            v[3 * (size_t)i + c] = (double)a[i];
    }
    for (int c = 0; F && c < 3; ++c) {
        NP_CUDA(rows(e->F, c, a));
        NP_CUDA(rows(e->F, 3 + c, b));
        for (int i = 0; i < n; ++i)
            F[3 * (size_t)i + c] = (double)a[i] + (double)b[i];
    }
    if (step)
        *step = e->step;
    return NPSIM_OK;
}

int npsim_ens_forces(npsim_ens_t e, int32_t d, double *F)
{
    NP_TRACE();
    NP_REQUIRE(e && F && d >= 0 && d < e->D, "bad ensemble, droplet index or F");
    int rc = ens_pass(e, MODE_FORCES, true, e->F_tmp, e->user);
    if (rc)
        return rc;
    NP_CUDA(cudaStreamSynchronize(e->user));
    const int n = e->cnt[d], off = e->off[d];
    const size_t N = (size_t)e->n_total;
    std::vector<float> a((size_t)n), b((size_t)n);
    for (int c = 0; c < 3; ++c) {
        NP_CUDA(cudaMemcpy(a.data(), e->F_tmp + c * N + off, sizeof(float) * (size_t)n,
                           cudaMemcpyDeviceToHost));
        NP_CUDA(cudaMemcpy(b.data(), e->F_tmp + (3 + c) * N + off, sizeof(float) * (size_t)n,
                           cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i)
            F[3 * (size_t)i + c] = (double)a[i] + (double)b[i];
    }
    return NPSIM_OK;
}

int npsim_ens_stats(npsim_ens_t e, int32_t d, const npsim_stats_cfg_t *cfg, int64_t *rdf_counts,
                    double *rdf_g, int64_t *radial_counts, double *radial_c, npsim_stats_t *out)
{
    NP_TRACE();
    NP_REQUIRE(e && cfg && out && d >= 0 && d < e->D,
               "bad ensemble, droplet index, cfg or out");
    int rc = check_stats_cfg(cfg);
    if (rc)
        return rc;
    const int n = e->cnt[d], off = e->off[d];
    if (n > e->sw.x_cap) {
        dfree(e->sw.x);
        e->sw.x_cap = 0;
        NP_CUDA(dalloc(&e->sw.x, 3 * (size_t)n));
        e->sw.x_cap = n;
    }
    const npsim_params_t &p = e->P[d];
    const double t = (double)e->step * p.dt;
    const double R2 = p.R0 * p.R0 - p.k_evap * t;
    const double R = R2 > 0 ? std::sqrt(R2) : 0.0;
    // droplet d's positions (hi + lo) from the ensemble's state, on the device
    NP_CUDA(launch_positions_f64_ld(e->xq + off, e->x_lo + off, n, e->n_total, e->sw.x,
                                    e->user));
    rc = stats_core(e->sw, e->sw.x, e->xq + off, e->typ + off, n, R, e->d_mean[d],
                    e->types[d].data(), p.n_types, e->d_flags, cfg, rdf_counts, rdf_g,
                    radial_counts, radial_c, out, e->user);
    if (rc)
        return rc;
    int h = 0;
    NP_CUDA(cudaMemcpyAsync(&h, e->d_flags, sizeof(int), cudaMemcpyDeviceToHost, e->user));
    NP_CUDA(cudaStreamSynchronize(e->user));
    if (h) {
        NP_CUDA(cudaMemsetAsync(e->d_flags, 0, sizeof(int), e->user));
        return set_err(NPSIM_ERR_CUDA, "device error word 0x%x", h);
    }
    return NPSIM_OK;
}

int npsim_ens_config(npsim_ens_t e, int *block, int *i_per_thread, int *j_tile, int *grid,
                     int *index)
{
    NP_REQUIRE(e, "ensemble is NULL");
    const ApConfig c = ens_config(e->shape);
    if (block)
        *block = c.block;
    if (i_per_thread)
        *i_per_thread = c.ki;
    if (j_tile)
        *j_tile = c.jt;
    if (grid)
        *grid = e->sk.grid;
    if (index)
        *index = e->shape;
    return NPSIM_OK;
}

int npsim_ens_work(npsim_ens_t e, int64_t *n_items, int32_t *itile)
{
    NP_REQUIRE(e, "ensemble is NULL");
    if (n_items)
        *n_items = e->n_items;
    if (itile)
        *itile = e->sk.itile;
    return NPSIM_OK;
}

int npsim_ens_info(npsim_ens_t e, int64_t *n_total, double *pairs_per_step)
{
    NP_REQUIRE(e, "ensemble is NULL");
    if (n_total)
        *n_total = e->n_total;
    if (pairs_per_step) {
        double p = 0.0;
        for (int d = 0; d < e->D; ++d)
            p += (double)e->cnt[d] * (double)(e->cnt[d] - 1);
        *pairs_per_step = p;
    }
    return NPSIM_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------
// Test hooks

namespace {

__global__ void k_philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         long long n_blocks, uint32_t *out)
{
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= n_blocks)
        return;
    const unsigned long long lo = (unsigned long long)c0 + (unsigned long long)b;
    const U4 r = philox10(U4{(uint32_t)lo, c1 + (uint32_t)(lo >> 32), c2, c3}, (uint32_t)seed,
                          (uint32_t)(seed >> 32));
    out[4 * b + 0] = r.x;
    out[4 * b + 1] = r.y;
    out[4 * b + 2] = r.z;
    out[4 * b + 3] = r.w;
}

__global__ void k_normals(uint64_t seed, long long step, int n, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float a, b, c;
    normals3(seed, (uint32_t)i, step, 0u, a, b, c);
    out[3 * i + 0] = a;
    out[3 * i + 1] = b;
    out[3 * i + 2] = c;
}

} // namespace

extern "C" int npsim_philox(uint64_t seed, const uint32_t ctr[4], int64_t n_blocks,
                            uint32_t *out)
{
    NP_REQUIRE(ctr && out, "ctr and out are required");
    NP_REQUIRE(n_blocks >= 0 && n_blocks <= (1ll << 28), "n_blocks out of range");
    int rc = check_device(nullptr);
    if (rc)
        return rc;
    if (n_blocks == 0)
        return NPSIM_OK;
    uint32_t *d = nullptr;
    NP_CUDA(dalloc(&d, 4 * (size_t)n_blocks));
    k_philox<<<(unsigned)((n_blocks + 255) / 256), 256>>>(seed, ctr[0], ctr[1], ctr[2], ctr[3],
                                                          n_blocks, d);
    cudaError_t e = cudaMemcpy(out, d, sizeof(uint32_t) * 4 * (size_t)n_blocks,
                               cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "philox: %s", cudaGetErrorString(e));
    return NPSIM_OK;
}

extern "C" int npsim_normals(uint64_t seed, int64_t step, int64_t n, double *out)
{
    NP_REQUIRE(out, "out is required");
    NP_REQUIRE(n >= 0 && n <= (1ll << 29), "n out of range");
    int rc = check_device(nullptr);
    if (rc)
        return rc;
    if (n == 0)
        return NPSIM_OK;
    double *d = nullptr;
    NP_CUDA(dalloc(&d, 3 * (size_t)n));
    k_normals<<<(unsigned)((n + 255) / 256), 256>>>(seed, step, (int)n, d);
    cudaError_t e = cudaMemcpy(out, d, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess)
        return set_err(NPSIM_ERR_CUDA, "normals: %s", cudaGetErrorString(e));
    return NPSIM_OK;
}
