// celllist.cu -- cell binning (step (i) of the loop in arXiv 2501.04456 Sec. 2.2:
// NPs are sorted into spatial cells so that near neighbours are found quickly)
// and the truncated, unshifted Lennard-Jones force over the 27 neighbouring
// cells (step (ii)):
//   F_i = sum_{j != i, r < rc_ij} 24 eps_ij (2 (s_ij/r)^12 - (s_ij/r)^6) r_ij / r^2.
//
// Binning is a counting sort: hash (cell of each NP, its arrival rank from an
// atomic counter), exclusive scan of the per-cell counts, scatter, then every
// NP is placed at its rank by index inside its cell (one thread per NP counts
// the members of its cell with a smaller index) so that the order inside a
// cell -- and therefore the float summation order of the LJ kernel -- does not
// depend on the atomic arrival order (runs are bit-reproducible).  A gather
// writes the NP records (position, type in the fourth word) in cell order so
// the LJ kernel reads neighbours from contiguous memory.  The
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

__global__ void k_cell_hash(CellGrid g, const float4 *__restrict__ xq, int n,
                            int *__restrict__ key, int *__restrict__ rank,
                            int *__restrict__ count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 p = xq[i];
    const int c = (cell_coord(p.z, g) * g.dim + cell_coord(p.y, g)) * g.dim +
                  cell_coord(p.x, g);
    key[i] = c;
    rank[i] = atomicAdd(&count[c], 1);
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
             int m)
{
    __shared__ int s_warp[kScanThreads / 32 + 1];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
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
        tile_sum[blockIdx.x] = total;
}

// One CTA: exclusive scan of the tile totals in place; start[m] = grand total.
__global__ void __launch_bounds__(kScanThreads)
k_scan_totals(int *__restrict__ tile_sum, int n_tiles, int *__restrict__ start, int m)
{
    __shared__ int s_warp[kScanThreads / 32 + 1];
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
k_scan_add(int *__restrict__ start, const int *__restrict__ tile_sum, int m)
{
    const int off = tile_sum[blockIdx.x];
    const int base = blockIdx.x * kScanTile + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = base + k * kScanThreads;
        if (i < m)
            start[i] += off;
    }
}

__global__ void k_cell_scatter(const int *__restrict__ key, const int *__restrict__ rank,
                               const int *__restrict__ start, int *__restrict__ arrived,
                               int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    arrived[start[key[i]] + rank[i]] = i;
}

// Members of every cell in index order: the NP at arrival slot q goes to its
// cell's start plus the number of members with a smaller index (O(m) per NP for
// a cell of m members, all NPs in parallel).
__global__ void k_cell_order(const int *__restrict__ arrived, const int *__restrict__ key,
                             const int *__restrict__ start, int *__restrict__ sorted, int n)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n)
        return;
    const int i = arrived[q];
    const int c = key[i];
    const int b = start[c], e = start[c + 1];
    int rank = 0;
    for (int k = b; k < e; ++k)
        rank += arrived[k] < i;
    sorted[b + rank] = i;
}

// Cell-ordered records: (x, y, z, type as int bits).
__global__ void k_cell_gather(const int *__restrict__ sorted, const float4 *__restrict__ xq,
                              const int *__restrict__ typ, float4 *__restrict__ sxq, int n)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const int i = sorted[p];
    const float4 q = xq[i];
    sxq[p] = make_float4(q.x, q.y, q.z, __int_as_float(typ[i]));
}

__global__ void __launch_bounds__(128)
k_cell_lj(CellGrid g, const int *__restrict__ start, const int *__restrict__ sorted,
          const float4 *__restrict__ sxq, int n, const PairTab *__restrict__ tab,
          float *__restrict__ F_lj)
{
    __shared__ float4 s_tab[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ float s_rcmax[NPSIM_MAX_TYPES]; // largest rc^2 of a row type
    for (int k = threadIdx.x; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; k += blockDim.x)
        s_tab[k] = tab->e[k];
    __syncthreads();
    if (threadIdx.x < NPSIM_MAX_TYPES) {
        float m = 0.0f;
        for (int b = 0; b < NPSIM_MAX_TYPES; ++b)
            m = fmaxf(m, s_tab[threadIdx.x * NPSIM_MAX_TYPES + b].z);
        s_rcmax[threadIdx.x] = m;
    }
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const float4 pi = sxq[p];
    const int ti = __float_as_int(pi.w);
    const int row = ti * NPSIM_MAX_TYPES;
    const float rcmax = s_rcmax[ti];
    const int cx = cell_coord(pi.x, g), cy = cell_coord(pi.y, g), cz = cell_coord(pi.z, g);
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = cz + dz;
        if (z < 0 || z >= g.dim)
            continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = cy + dy;
            if (y < 0 || y >= g.dim)
                continue;
            const int base = (z * g.dim + y) * g.dim;
            const int x0 = max(cx - 1, 0), x1 = min(cx + 1, g.dim - 1);
            // cells x0..x1 of this row are contiguous in the sorted order
            const int b = start[base + x0], e = start[base + x1 + 1];
#pragma unroll 2
            for (int q = b; q < e; ++q) {
                const float4 pj = sxq[q];
                const float dx = pi.x - pj.x, dy2 = pi.y - pj.y, dz2 = pi.z - pj.z;
                const float r2 = fmaf(dx, dx, fmaf(dy2, dy2, dz2 * dz2));
                // the row type's largest cutoff first (most candidates stop here);
                // the NP itself has r2 = 0 and is skipped by q != p
                if (r2 >= rcmax || q == p)
                    continue;
                const float4 t = s_tab[row + __float_as_int(pj.w)];
                if (r2 < t.z) {
                    const float rinv2 = 1.0f / r2;
                    const float s2 = t.x * rinv2;
                    const float s6 = s2 * s2 * s2;
                    const float f = t.y * rinv2 * s6 * fmaf(2.0f, s6, -1.0f);
                    two_sum_acc(hx, lx, f * dx);
                    two_sum_acc(hy, ly, f * dy2);
                    two_sum_acc(hz, lz, f * dz2);
                }
            }
        }
    }
    // one 24-byte record per NP: (hi x, y, z, lo x, y, z)
    float2 *o = reinterpret_cast<float2 *>(F_lj + 6 * (size_t)sorted[p]);
    o[0] = make_float2(hx, hy);
    o[1] = make_float2(hz, lx);
    o[2] = make_float2(ly, lz);
}

} // namespace

// kernels per build: hash, three scan passes, scatter, order, gather
int cell_build_launches() { return 7; }

int cell_scan_tiles(int n_cells) { return (n_cells + kScanTile - 1) / kScanTile; }

cudaError_t launch_cell_build(const CellGrid &g, const float4 *xq, const int *typ, int n,
                              CellBufs &b, int * /*flags*/, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(int) * (size_t)g.n_cells, st);
    if (e != cudaSuccess)
        return e;
    const int B = 256;
    k_cell_hash<<<(n + B - 1) / B, B, 0, st>>>(g, xq, n, b.key, b.rank, b.count);
    const int nt = cell_scan_tiles(g.n_cells);
    k_scan_tiles<<<nt, kScanThreads, 0, st>>>(b.count, b.start, b.tile_sum, g.n_cells);
    k_scan_totals<<<1, kScanThreads, 0, st>>>(b.tile_sum, nt, b.start, g.n_cells);
    k_scan_add<<<nt, kScanThreads, 0, st>>>(b.start, b.tile_sum, g.n_cells);
    k_cell_scatter<<<(n + B - 1) / B, B, 0, st>>>(b.key, b.rank, b.start, b.arrived, n);
    k_cell_order<<<(n + B - 1) / B, B, 0, st>>>(b.arrived, b.key, b.start, b.sorted, n);
    k_cell_gather<<<(n + B - 1) / B, B, 0, st>>>(b.sorted, xq, typ, b.sxq, n);
    return cudaGetLastError();
}

cudaError_t launch_cell_lj(const CellGrid &g, const CellBufs &b, int n, const PairTab *tab,
                           float *F_lj, cudaStream_t st)
{
    const int B = 128;
    k_cell_lj<<<(n + B - 1) / B, B, 0, st>>>(g, b.start, b.sorted, b.sxq, n, tab, F_lj);
    return cudaGetLastError();
}

} // namespace npsim
