// celllist.cu -- cell binning (step (i) of the loop in arXiv 2501.04456 Sec. 2.2:
// NPs are sorted into spatial cells so that near neighbours are found quickly)
// and the truncated, unshifted Lennard-Jones force over the 27 neighbouring
// cells (step (ii)):
//   F_i = sum_{j != i, r < rc_ij} 24 eps_ij (2 (s_ij/r)^12 - (s_ij/r)^6) r_ij / r^2.
//
// Binning is a counting sort: hash (sort key of each NP, its arrival rank from
// an atomic counter), exclusive scan of the per-key counts, scatter, then every
// NP is placed at its rank by index inside its key (one thread per NP counts
// the members of its key with a smaller index) so that the order inside a
// cell -- and therefore the float summation order of the LJ kernel -- does not
// depend on the atomic arrival order (runs are bit-reproducible).  For the LJ
// lists the key is type * n_cells + cell: the cell order lists the NPs of one
// type cell by cell, then the next type, so that consecutive threads of the
// list kernels hold NPs of one type (lists of similar length, read coalesced)
// in nearby cells (their partners lie in the same few cells).  A gather writes
// the NP records (position, type in the fourth word) in cell order so the
// kernels read neighbours from contiguous memory; with a neighbour list the
// integrator keeps these records current, so the per-step list kernel reads
// every position in cell order and never gathers by particle index.
//
// The simulation keeps a Verlet neighbour list on top of the cells: the cell
// edge is the largest cutoff plus a skin, a build lists for every NP the
// partners within its pair cutoff plus the skin and records the positions it
// saw; the integrator raises a gate when some NP has moved more than half the
// skin since then, and only then do the (gated) build kernels run again.  A
// pair within its cutoff now was within cutoff + skin at the build, so the
// list (or, for an NP whose list overflowed, the cells of the build) holds
// every pair that can interact: the forces are those of a rebuild every step.  The
// cell edge is at least the largest cutoff (times 1 + 1e-5, so float rounding
// of the cell index can never separate two NPs within the cutoff by more than
// one cell); coordinates beyond the grid are clamped into the edge cells,
// which keeps every pair within the cutoff in neighbouring cells.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

__device__ __forceinline__ int cell_coord(float x, const CellGrid &g)
{
    int c = (int)floorf((x + g.L) * g.inv_h);
    return min(max(c, 0), g.dim - 1);
}

// Build kernels return at once when a gate is given and reads 0 (no rebuild).
__device__ __forceinline__ bool gate_closed(const int *gate) { return gate && *gate == 0; }

__global__ void k_cell_zero(int *__restrict__ count, int m, const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x)
        count[c] = 0;
}

__global__ void k_cell_hash(CellGrid g, const float4 *__restrict__ xq,
                            const int *__restrict__ typ, int n, int *__restrict__ key,
                            int *__restrict__ rank, int *__restrict__ count,
                            const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = xq[i];
        int c = (cell_coord(p.z, g) * g.dim + cell_coord(p.y, g)) * g.dim + cell_coord(p.x, g);
        if (g.tb > 1)
            c += typ[i] * g.n_cells;
        key[i] = c;
        rank[i] = atomicAdd(&count[c], 1);
    }
}

// Exclusive scan of count[0..m) into start[0..m], start[m] = total, in three
// passes: each CTA scans a tile of kScanTile counts and records the tile total;
// one CTA scans the tile totals; every CTA then adds its tile's offset.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one value per thread over a CTA of kScanThreads threads;
// *total receives the sum of all values.
__device__ __forceinline__ int cta_exclusive_scan(int v, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += u;
    }
    if (lane == 31)
        s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        int ix = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, ix, o);
            if (lane >= o)
                ix += u;
        }
        if (lane < kScanThreads / 32)
            s_warp[lane] = ix - x;
        if (lane == kScanThreads / 32 - 1)
            s_warp[kScanThreads / 32] = ix;
    }
    __syncthreads();
    const int r = s_warp[w] + incl - v;
    *total = s_warp[kScanThreads / 32];
    __syncthreads(); // s_warp may be reused by the caller
    return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int *__restrict__ count, int *__restrict__ start, int *__restrict__ tile_sum,
             int m, const int *__restrict__ gate)
{
    __shared__ int s_warp[kScanThreads / 32 + 1];
    if (gate_closed(gate)) // uniform over the block
        return;
    const int n_tiles = (m + kScanTile - 1) / kScanTile;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int base = t * kScanTile + threadIdx.x * kScanItems;
        int a[kScanItems];
        int s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            a[k] = base + k < m ? count[base + k] : 0;
            s += a[k];
        }
        int total;
        int run = cta_exclusive_scan(s, s_warp, &total);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < m)
                start[base + k] = run;
            run += a[k];
        }
        if (threadIdx.x == 0)
            tile_sum[t] = total;
    }
}

// One CTA: exclusive scan of the tile totals in place; start[m] = grand total.
__global__ void __launch_bounds__(kScanThreads)
k_scan_totals(int *__restrict__ tile_sum, int n_tiles, int *__restrict__ start, int m,
              const int *__restrict__ gate)
{
    __shared__ int s_warp[kScanThreads / 32 + 1];
    if (gate_closed(gate))
        return;
    int carry = 0;
    for (int b0 = 0; b0 < n_tiles; b0 += kScanTile) {
        const int base = b0 + threadIdx.x * kScanItems;
        int a[kScanItems];
        int s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            a[k] = base + k < n_tiles ? tile_sum[base + k] : 0;
            s += a[k];
        }
        int total;
        int run = carry + cta_exclusive_scan(s, s_warp, &total);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < n_tiles)
                tile_sum[base + k] = run;
            run += a[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0)
        start[m] = carry;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_add(int *__restrict__ start, const int *__restrict__ tile_sum, int m,
           const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    const int n_tiles = (m + kScanTile - 1) / kScanTile;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int off = tile_sum[t];
        const int base = t * kScanTile + threadIdx.x;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int i = base + k * kScanThreads;
            if (i < m)
                start[i] += off;
        }
    }
}

__global__ void k_cell_scatter(const int *__restrict__ key, const int *__restrict__ rank,
                               const int *__restrict__ start, int *__restrict__ arrived,
                               int n, const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        arrived[start[key[i]] + rank[i]] = i;
}

// Members of every cell in index order: the NP at arrival slot q goes to its
// cell's start plus the number of members with a smaller index (O(m) per NP for
// a cell of m members, all NPs in parallel).
__global__ void k_cell_order(const int *__restrict__ arrived, const int *__restrict__ key,
                             const int *__restrict__ start, int *__restrict__ sorted,
                             int *__restrict__ pos, int n, const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = arrived[q];
        const int c = key[i];
        const int b = start[c], e = start[c + 1];
        int rank = 0;
        for (int k = b; k < e; ++k)
            rank += arrived[k] < i;
        sorted[b + rank] = i;
        pos[i] = b + rank;
    }
}

// Cell-ordered records: (x, y, z, type as int bits).
__global__ void k_cell_gather(const int *__restrict__ sorted, const float4 *__restrict__ xq,
                              const int *__restrict__ typ, float4 *__restrict__ sxq, int n,
                              const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int i = sorted[p];
        const float4 q = xq[i];
        sxq[p] = make_float4(q.x, q.y, q.z, __int_as_float(typ[i]));
    }
}

// Per-row-type tables in shared memory: the pair table and, per row type, its
// largest squared cutoff (force kernels) or cutoff-plus-skin (list build).
// rcc2 (or NULL): squared cutoffs of the truncated Coulomb term per type pair
// (coulomb mode 2); a pair is listed within max(LJ cutoff, Coulomb cutoff) +
// skin, counting only the terms that act (eps_ab != 0, C q_a q_b != 0).
__device__ __forceinline__ void load_tables(const PairTab *__restrict__ tab,
                                            const float *__restrict__ rcc2, float skin,
                                            float4 *s_tab, float *s_rl2, float *s_rmax,
                                            float *s_rcc2 = nullptr)
{
    for (int k = threadIdx.x; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; k += blockDim.x) {
        const float4 t = tab->e[k];
        s_tab[k] = t;
        const float rcc = rcc2 ? rcc2[k] : 0.0f;
        if (s_rcc2)
            s_rcc2[k] = rcc;
        const float r_lj = t.y != 0.0f ? sqrtf(t.z) : 0.0f;
        const float r_c = (rcc > 0.0f && t.w != 0.0f) ? sqrtf(rcc) : 0.0f;
        const float r = fmaxf(r_lj, r_c);
        s_rl2[k] = r > 0.0f ? (r + skin) * (r + skin) : 0.0f; // 0: never listed
    }
    __syncthreads();
    if (threadIdx.x < NPSIM_MAX_TYPES) {
        float m = 0.0f;
        for (int b = 0; b < NPSIM_MAX_TYPES; ++b)
            m = fmaxf(m, skin > 0.0f ? s_rl2[threadIdx.x * NPSIM_MAX_TYPES + b]
                                     : s_tab[threadIdx.x * NPSIM_MAX_TYPES + b].z);
        s_rmax[threadIdx.x] = m;
    }
    __syncthreads();
}

// Neighbour lists (gated): for the NP at cell-order slot p (threads in the cell
// order, so that a warp scans the same cells), the partners within
// (rc_ab + skin) in the 27 cells, type block by type block in scan order, as
// their cell-order slots (the partner's type is the fourth word of its
// record), in blocks of four at nbr[nbr_index(k, p, n)] for k < cap;
// nnbr[p] = the full count (an NP with more than cap partners is summed from
// the cells instead).  Lists are written by slot
// so that the per-step force kernel, which runs in the same order, reads them
// coalesced.  Records the positions of this build in x_ref (by particle).
__global__ void __launch_bounds__(128, 8)
k_nbr_build(const __grid_constant__ CellGrid g, const int *__restrict__ start, const int *__restrict__ sorted,
            const float4 *__restrict__ sxq, int n, const PairTab *__restrict__ tab,
            const float *__restrict__ rcc2, float skin,
            int cap, unsigned *__restrict__ nbr, int *__restrict__ nnbr,
            float4 *__restrict__ x_ref,
            unsigned long long *__restrict__ builds, int *__restrict__ flags,
            const int *__restrict__ gate)
{
    if (gate_closed(gate))
        return;
    if (builds && blockIdx.x == 0 && threadIdx.x == 0)
        ++*builds;
    __shared__ float4 s_tab[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ float s_rl2[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ float s_rmax[NPSIM_MAX_TYPES];
    load_tables(tab, rcc2, skin, s_tab, s_rl2, s_rmax);
    const int tb = g.tb > 1 ? g.tb : 1;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 pi = sxq[p];
        const int i = sorted[p];
        const int ti = __float_as_int(pi.w);
        const int row = ti * NPSIM_MAX_TYPES;
        const float rmax = s_rmax[ti];
        const int cx = cell_coord(pi.x, g), cy = cell_coord(pi.y, g), cz = cell_coord(pi.z, g);
        int cnt = 0;
        for (int t = 0; t < tb; ++t) {
            if (tb > 1 && s_rl2[row + t] == 0.0f)
                continue; // no term acts between these types
            const int kofs = t * g.n_cells;
            // the cells this type pair's list radius can reach (with tb == 1, the
            // widest stencil of the row type); with type blocks every candidate
            // of block t has type t, so its squared list radius is fixed
            int w = g.ext[row + t];
            if (tb == 1)
                for (int b = 1; b < NPSIM_MAX_TYPES; ++b)
                    w = max(w, (int)g.ext[row + b]);
            const float rl2_t = tb > 1 ? s_rl2[row + t] : rmax;
            for (int dz = -w; dz <= w; ++dz) {
                const int z = cz + dz;
                if (z < 0 || z >= g.dim)
                    continue;
                for (int dy = -w; dy <= w; ++dy) {
                    const int y = cy + dy;
                    if (y < 0 || y >= g.dim)
                        continue;
                    const int base = kofs + (z * g.dim + y) * g.dim;
                    const int b = start[base + max(cx - w, 0)];
                    const int e = start[base + min(cx + w, g.dim - 1) + 1];
                    for (int q = b; q < e; ++q) {
                        const float4 pj = sxq[q];
                        const float dx = pi.x - pj.x, dy2 = pi.y - pj.y, dz2 = pi.z - pj.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy2, dy2, dz2 * dz2));
                        if (r2 >= rl2_t || q == p)
                            continue;
                        const int tj = __float_as_int(pj.w);
                        if (tb > 1 || r2 < s_rl2[row + tj]) {
                            if (cnt < cap)
                                nbr[nbr_index(cnt, p, n)] = (unsigned)q;
                            ++cnt;
                        }
                    }
                }
            }
        }
        // pad the last block with the far record (whole blocks of four
        // partners); an empty list gets one block of it, so that the first
        // block, which the force kernel reads before the count, always names
        // valid records
        for (int k = cnt; k < cap && (k < 4 || (k & 3)); ++k)
            nbr[nbr_index(k, p, n)] = (unsigned)n;
        nnbr[p] = cnt;
        if (cnt > cap)
            atomicOr(flags, FLAG_NBR_OVERFLOW);
        x_ref[i] = make_float4(pi.x, pi.y, pi.z, 0.0f);
    }
}

// The forces of the NP at slot p whose list overflowed: every NP of the cells of
// its build (the NP's sort key holds its build cell; a superset of its list),
// summed pair by pair into the compensated totals.  Kept out of line so that
// it takes no registers from the list loops.
template <bool COUL>
__device__ __noinline__ void cell_slot_forces(int p, const CellGrid g, const int *__restrict__ start,
                                              const int *__restrict__ sorted,
                                              const int *__restrict__ key,
                                              const float4 *__restrict__ sxq,
                                              float *__restrict__ F_lj, const float4 *s_tab,
                                              const float *s_rcc2)
{
    const float4 pi = sxq[p];
    const int i = sorted[p];
    const int ti = __float_as_int(pi.w);
    const int row = ti * NPSIM_MAX_TYPES;
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    const int tb = g.tb > 1 ? g.tb : 1;
    const int c = key[i] - (g.tb > 1 ? ti * g.n_cells : 0);
    const int cx = c % g.dim, cy = (c / g.dim) % g.dim, cz = c / (g.dim * g.dim);
    for (int t = 0; t < tb; ++t) {
        const int kofs = t * g.n_cells;
        int w = g.ext[row + t];
        if (tb == 1)
            for (int b = 1; b < NPSIM_MAX_TYPES; ++b)
                w = max(w, (int)g.ext[row + b]);
        for (int dz = -w; dz <= w; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.dim)
                continue;
            for (int dy = -w; dy <= w; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.dim)
                    continue;
                const int base = kofs + (z * g.dim + y) * g.dim;
                const int b = start[base + max(cx - w, 0)];
                const int e = start[base + min(cx + w, g.dim - 1) + 1];
                for (int q = b; q < e; ++q)
                    if (q != p) {
                        const float4 pj = sxq[q];
                        const float dx = pi.x - pj.x, dy2 = pi.y - pj.y, dz2 = pi.z - pj.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy2, dy2, dz2 * dz2));
                        const int tj = __float_as_int(pj.w);
                        const float4 tt = s_tab[row + tj];
                        const float ri = rsqrtf(r2);
                        const float rinv2 = ri * ri;
                        const float s2 = tt.x * rinv2;
                        const float s6 = s2 * s2 * s2;
                        float f = r2 < tt.z ? tt.y * rinv2 * s6 * fmaf(2.0f, s6, -1.0f) : 0.0f;
                        if (COUL && r2 < s_rcc2[row + tj])
                            f = fmaf(tt.w * ri, rinv2, f);
                        two_sum_acc(hx, lx, f * dx);
                        two_sum_acc(hy, ly, f * dy2);
                        two_sum_acc(hz, lz, f * dz2);
                    }
            }
        }
    }
    float4 *o = reinterpret_cast<float4 *>(F_lj + 8 * (size_t)i);
    o[0] = make_float4(hx, hy, hz, lx);
    o[1] = make_float4(ly, lz, 0.0f, 0.0f);
}

// LJ forces (and, with rcc2, the truncated Coulomb term) from the neighbour
// lists at the current positions for the NP at cell-order slot p: its own
// record sxq[p] (kept current by the integrator), its list column and its
// partners' records are read in cell order -- coalesced over consecutive
// slots, and for the partners from the nearby cells -- and the 32-byte force
// record goes to the NP's index i = sorted[p], where the integrator reads it.
// An NP whose list overflowed sums over the cells of that build instead (a
// superset of its list).  Writes one (hi x, y, z, lo x, y, z, 0, 0) record.
template <bool COUL>
__device__ __forceinline__ void slot_forces(int p, const CellGrid &g, const int *__restrict__ start,
                                            const int *__restrict__ sorted,
                                            const int *__restrict__ key,
                                            const float4 *__restrict__ sxq, int n, int cap,
                                            const unsigned *__restrict__ nbr,
                                            const int *__restrict__ nnbr,
                                            float *__restrict__ F_lj, const float4 *s_tab,
                                            const float *s_rcc2)
{
    const float4 pi = sxq[p];
    const int i = sorted[p];
    const int ti = __float_as_int(pi.w);
    const int row = ti * NPSIM_MAX_TYPES;
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    // One pair's force added into (sx, sy, sz); 1/r^2 as rsqrt(r^2)^2, as in
    // the all-pairs kernels.  The block sums go into the compensated (hi, lo)
    // totals by flush(), once per block of up to four partners.
    auto pair = [&](const float4 pj, float &sx, float &sy, float &sz) {
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const int tj = __float_as_int(pj.w);
        const float4 t = s_tab[row + tj];
        const float ri = rsqrtf(r2);
        const float rinv2 = ri * ri;
        const float s2 = t.x * rinv2;
        const float s6 = s2 * s2 * s2;
        // LJ (r < rc_ab) plus, with COUL, Coulomb truncated at its own cutoff
        float f = r2 < t.z ? t.y * rinv2 * s6 * fmaf(2.0f, s6, -1.0f) : 0.0f;
        if (COUL && r2 < s_rcc2[row + tj])
            f = fmaf(t.w * ri, rinv2, f); // C q_a q_b / r^3
        sx = fmaf(f, dx, sx);
        sy = fmaf(f, dy, sy);
        sz = fmaf(f, dz, sz);
    };
    auto flush = [&](float sx, float sy, float sz) {
        two_sum_acc(hx, lx, sx);
        two_sum_acc(hy, ly, sy);
        two_sum_acc(hz, lz, sz);
    };
    // List entries arrive four at a time (one 16-byte load per block of four,
    // contiguous over consecutive slots), two blocks ahead of their use, and a
    // block's partner records are gathered one block ahead, so that each thread
    // keeps the next block's gathers and the entries after it in flight while
    // it computes.  A list's last block is padded with the far record, whose
    // terms are exactly zero, so every block is four whole pairs.  Pairs are
    // summed in list order, each block of four in float32 and then into the
    // compensated (hi, lo) total.  The first block is read before the count is
    // known (cap >= 4 entries exist for every slot).  Entries are the
    // partners' slots; a partner's type is the fourth word of its record.
    // The lists stream through once per step: they are read with the
    // evict-first (streaming) policy so that they do not push the partner
    // records out of L1 and L2.
    const uint4 *nb4 = reinterpret_cast<const uint4 *>(nbr);
    const uint4 far4 = make_uint4((unsigned)n, (unsigned)n, (unsigned)n, (unsigned)n);
    uint4 cur = __ldcs(nb4 + p);
    const int cnt = nnbr[p];
    if (cnt > cap) {
        cell_slot_forces<COUL>(p, g, start, sorted, key, sxq, F_lj, s_tab, s_rcc2);
        return;
    }
    {
        const int nblk = (cnt + 3) >> 2;
        uint4 nxt = nblk > 1 ? __ldcs(nb4 + (size_t)n + p) : far4;
        float4 pj[4];
        pj[0] = sxq[cur.x];
        pj[1] = sxq[cur.y];
        pj[2] = sxq[cur.z];
        pj[3] = sxq[cur.w];
        for (int j = 0; j < nblk; ++j) {
            const uint4 nn = j + 2 < nblk ? __ldcs(nb4 + (size_t)(j + 2) * n + p) : far4;
            float4 pn[4];
            if (j + 1 < nblk) {
                pn[0] = sxq[nxt.x];
                pn[1] = sxq[nxt.y];
                pn[2] = sxq[nxt.z];
                pn[3] = sxq[nxt.w];
            }
            float sx = 0.f, sy = 0.f, sz = 0.f;
            pair(pj[0], sx, sy, sz);
            pair(pj[1], sx, sy, sz);
            pair(pj[2], sx, sy, sz);
            pair(pj[3], sx, sy, sz);
            flush(sx, sy, sz);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                pj[u] = pn[u];
            cur = nxt;
            nxt = nn;
        }
    }
    // one 32-byte record per NP, a whole DRAM sector: (hi x, y, z, lo x), (lo y, z)
    float4 *o = reinterpret_cast<float4 *>(F_lj + 8 * (size_t)i);
    o[0] = make_float4(hx, hy, hz, lx);
    o[1] = make_float4(ly, lz, 0.0f, 0.0f);
}

// List forces, one thread per cell-order slot (slot_forces), and closes the
// rebuild gate.  The CTAs take the 128-slot tiles from the last one back: the
// cell order lists the types one after another, so the last tiles hold the
// largest NPs, whose lists are the longest (several times the mean in a
// polydisperse aggregate); started first, they no longer run alone at the end
// of the launch while the short ones fill the tail.  8 CTAs of 128 per SM (64
// registers: each thread keeps two blocks of partner records and entries in
// flight).
template <bool COUL>
__global__ void __launch_bounds__(128, 8)
k_lj_nbr(const __grid_constant__ CellGrid g, const int *__restrict__ start, const int *__restrict__ sorted,
         const int *__restrict__ key, const float4 *__restrict__ sxq, int n,
         const PairTab *__restrict__ tab, const float *__restrict__ rcc2, int cap,
         const unsigned *__restrict__ nbr, const int *__restrict__ nnbr,
         float *__restrict__ F_lj, int *__restrict__ gate)
{
    __shared__ float4 s_tab[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ float s_rl2[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ float s_rcc2[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ float s_rmax[NPSIM_MAX_TYPES];
    load_tables(tab, COUL ? rcc2 : nullptr, 0.0f, s_tab, s_rl2, s_rmax, s_rcc2);
    if (gate && blockIdx.x == 0 && threadIdx.x == 0)
        *gate = 0; // every build kernel of this step has run; the integrator may reopen it
    const int p = (int)(gridDim.x - 1 - blockIdx.x) * (int)blockDim.x + (int)threadIdx.x;
    if (p < n)
        slot_forces<COUL>(p, g, start, sorted, key, sxq, n, cap, nbr, nnbr, F_lj, s_tab, s_rcc2);
}

} // namespace

// kernels per build: zero, hash, three scan passes, scatter, order, gather
int cell_build_launches() { return 8; }

int cell_scan_tiles(int n_cells) { return (n_cells + kScanTile - 1) / kScanTile; }

namespace {
constexpr int kMaxGrid = 1216; // 8 CTAs on each of 152 SMs
int grid_for(int n, int block)
{
    const int g = (n + block - 1) / block;
    return g < 1 ? 1 : (g < kMaxGrid ? g : kMaxGrid);
}
} // namespace

cudaError_t launch_cell_build(const CellGrid &g, const float4 *xq, const int *typ, int n,
                              CellBufs &b, const int *gate, cudaStream_t st)
{
    // grid-stride kernels on at most kMaxGrid CTAs: when the gate is closed a
    // launch costs little more than its CTAs' start
    const int B = 256;
    const int m = (g.tb > 1 ? g.tb : 1) * g.n_cells; // sort keys
    const int gn = grid_for(n, B), gc = grid_for(m, B);
    k_cell_zero<<<gc, B, 0, st>>>(b.count, m, gate);
    k_cell_hash<<<gn, B, 0, st>>>(g, xq, typ, n, b.key, b.rank, b.count, gate);
    const int nt = cell_scan_tiles(m);
    const int gt = nt < kMaxGrid ? nt : kMaxGrid;
    k_scan_tiles<<<gt, kScanThreads, 0, st>>>(b.count, b.start, b.tile_sum, m, gate);
    k_scan_totals<<<1, kScanThreads, 0, st>>>(b.tile_sum, nt, b.start, m, gate);
    k_scan_add<<<gt, kScanThreads, 0, st>>>(b.start, b.tile_sum, m, gate);
    k_cell_scatter<<<gn, B, 0, st>>>(b.key, b.rank, b.start, b.arrived, n, gate);
    k_cell_order<<<gn, B, 0, st>>>(b.arrived, b.key, b.start, b.sorted, b.pos, n, gate);
    k_cell_gather<<<gn, B, 0, st>>>(b.sorted, xq, typ, b.sxq, n, gate);
    return cudaGetLastError();
}

cudaError_t launch_cell_refresh(const CellBufs &b, const float4 *xq, const int *typ, int n,
                                cudaStream_t st)
{
    k_cell_gather<<<grid_for(n, 256), 256, 0, st>>>(b.sorted, xq, typ, b.sxq, n, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_nbr_build(const CellGrid &g, const CellBufs &b, int n, const PairTab *tab,
                             const float *rcc2, float skin, const NbrList &l, int *flags,
                             const int *gate, cudaStream_t st)
{
    // heavy per-NP work (every candidate of 27 cells): up to four CTAs of
    // kMaxGrid, so that a compact droplet's build still has one NP per thread
    const int B = 128;
    const int gb = (n + B - 1) / B < 4 * kMaxGrid ? (n + B - 1) / B : 4 * kMaxGrid;
    k_nbr_build<<<gb > 0 ? gb : 1, B, 0, st>>>(g, b.start, b.sorted, b.sxq, n, tab, rcc2, skin,
                                               l.cap, l.nbr, l.nnbr, l.x_ref, l.builds, flags,
                                               gate);
    return cudaGetLastError();
}

cudaError_t launch_lj_nbr(const CellGrid &g, const CellBufs &b, const float4 *xq,
                          const int *typ, int n, const PairTab *tab, const float *rcc2,
                          const NbrList &l, float *F_lj, int *gate, cudaStream_t st)
{
    (void)xq; // the current positions are the cell-ordered records b.sxq
    (void)typ;
    const int B = 128;
    const int grid = (n + B - 1) / B;
    if (rcc2)
        k_lj_nbr<true><<<grid, B, 0, st>>>(g, b.start, b.sorted, b.key, b.sxq, n, tab, rcc2,
                                           l.cap, l.nbr, l.nnbr, F_lj, gate);
    else
        k_lj_nbr<false><<<grid, B, 0, st>>>(g, b.start, b.sorted, b.key, b.sxq, n, tab, nullptr,
                                            l.cap, l.nbr, l.nnbr, F_lj, gate);
    return cudaGetLastError();
}

} // namespace npsim
