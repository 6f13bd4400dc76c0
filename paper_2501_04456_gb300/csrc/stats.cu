// stats.cu -- post-processing statistics of arXiv 2501.04456 Sec. 3 on the GPU:
//  * pair-distance histogram for the RDF of Sec. 3.2 (ordered pairs, bins of
//    width r_max/n_bins over [0, r_max)); candidates come from a cell grid of
//    edge >= r_max, a float32 distance test discards far pairs, and the bin is
//    decided in float64 from the float64 positions with the operations
//    sqrt(dx*dx + dy*dy + dz*dz) and floor(r / dr) rounded one by one (no fused
//    multiply-add), so integer counts are exact;
//  * radial histogram of |x| for the concentration C_NPs(r) of Sec. 3.2;
//  * the scattered intensity I(q) of Sec. 3.3 as the transform of g(r);
//  * N_surf, the number of NPs at the droplet surface (Sec. 1: the scattered
//    intensity grows with N_surf^2), counted as the NPs whose centre lies in
//    the band (-r_i, r_i) about the surface, | |x_i| - R(t) | < r_i, the band
//    in which Sec. 2.2 step (iv) applies the interface force;
//  * per-CTA partial sums (centre of mass, squared deviations) and minima,
//    finished on the host in CTA order (deterministic);
//  * box counting: the number of distinct integer triples floor((x - o)/eps)
//    via an open-addressing hash set in device memory (the count does not
//    depend on insertion order).
#include "npsim_internal.cuh"

namespace npsim {

namespace {

__device__ __forceinline__ int cell_coord_s(float x, const CellGrid &g)
{
    int c = (int)floorf((x + g.L) * g.inv_h);
    return min(max(c, 0), g.dim - 1);
}

__device__ __forceinline__ double dist_rn(double ax, double ay, double az, double bx,
                                          double by, double bz)
{
    const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                __dmul_rn(dz, dz)));
}

constexpr int kMaxSmemBins = 4096;

__global__ void __launch_bounds__(256)
k_pair_hist(const double *__restrict__ x, int n, double r_max, double dr, int n_bins,
            float r_cut32, CellGrid g, const int *__restrict__ start,
            const int *__restrict__ sorted, const float4 *__restrict__ sxq,
            unsigned long long *__restrict__ hist)
{
    __shared__ unsigned int s_h[kMaxSmemBins];
    const bool smem = n_bins <= kMaxSmemBins;
    if (smem)
        for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
            s_h[b] = 0u;
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        const int i = sorted[p];
        const float4 pi = sxq[p];
        const double xi = x[i], yi = x[n + i], zi = x[2 * n + i];
        const int cx = cell_coord_s(pi.x, g), cy = cell_coord_s(pi.y, g),
                  cz = cell_coord_s(pi.z, g);
        const float rc2 = r_cut32 * r_cut32;
        for (int dz = -1; dz <= 1; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.dim)
                continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.dim)
                    continue;
                const int base = (z * g.dim + y) * g.dim;
                const int b0 = start[base + max(cx - 1, 0)];
                const int b1 = start[base + min(cx + 1, g.dim - 1) + 1];
                for (int q = b0; q < b1; ++q) {
                    if (q == p)
                        continue;
                    const float4 pj = sxq[q];
                    const float ex = pi.x - pj.x, ey = pi.y - pj.y, ez = pi.z - pj.z;
                    if (ex * ex + ey * ey + ez * ez > rc2)
                        continue;
                    const int j = sorted[q];
                    const double r = dist_rn(xi, yi, zi, x[j], x[n + j], x[2 * n + j]);
                    const double bb = floor(__ddiv_rn(r, dr));
                    if (bb < (double)n_bins) {
                        if (smem)
                            atomicAdd(&s_h[(int)bb], 1u);
                        else
                            atomicAdd(&hist[(int)bb], 1ull);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (smem)
        for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
            if (s_h[b])
                atomicAdd(&hist[b], (unsigned long long)s_h[b]);
}

__global__ void __launch_bounds__(256)
k_radial_hist(const double *__restrict__ x, int n, double dr, int n_bins,
              unsigned long long *__restrict__ hist)
{
    __shared__ unsigned int s_h[kMaxSmemBins];
    const bool smem = n_bins <= kMaxSmemBins;
    if (smem)
        for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
            s_h[b] = 0u;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double r = dist_rn(x[i], x[n + i], x[2 * n + i], 0.0, 0.0, 0.0);
        const double bb = floor(__ddiv_rn(r, dr));
        if (bb < (double)n_bins) {
            if (smem)
                atomicAdd(&s_h[(int)bb], 1u);
            else
                atomicAdd(&hist[(int)bb], 1ull);
        }
    }
    __syncthreads();
    if (smem)
        for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
            if (s_h[b])
                atomicAdd(&hist[b], (unsigned long long)s_h[b]);
}

// NPs with | |x_i| - R | < half_sigma[type_i] (|x| and the difference in
// float64, rounded operation by operation as in the radial histogram).
__global__ void __launch_bounds__(256)
k_surface_count(const double *__restrict__ x, const int *__restrict__ typ, int n, double R,
                SurfHalf hs, unsigned long long *__restrict__ count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int in = 0;
    if (i < n) {
        const double r = dist_rn(x[i], x[n + i], x[2 * n + i], 0.0, 0.0, 0.0);
        in = fabs(__dsub_rn(r, R)) < hs.h[typ[i]];
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0 && m)
        atomicAdd(count, (unsigned long long)__popc(m));
}

// G(u) = sin u - u cos u (the antiderivative of u sin u): by its series below
// u = 0.5, where the difference of the two terms would cancel.
__device__ __forceinline__ double scat_G(double u)
{
    if (u < 0.5) {
        const double u2 = u * u;
        // u^3/3 - u^5/30 + u^7/840 - u^9/45360 + u^11/3991680 - u^13/518918400
        double s = -1.0 / 518918400.0;
        s = s * u2 + 1.0 / 3991680.0;
        s = s * u2 - 1.0 / 45360.0;
        s = s * u2 + 1.0 / 840.0;
        s = s * u2 - 1.0 / 30.0;
        s = s * u2 + 1.0 / 3.0;
        return s * u2 * u;
    }
    return sin(u) - u * cos(u);
}

// One warp per q: I(q) = N_surf^2 4 pi sum_b g_b [G(q r_{b+1}) - G(q r_b)] / q^3
// (q = 0: N_surf^2 4 pi sum_b g_b (r_{b+1}^3 - r_b^3) / 3); lane l sums bins l,
// l + 32, ... and the lanes are combined in a fixed butterfly order.  out_frac
// (or NULL): the fractal form N_surf^2 (q R_g)^(-D_f).
__global__ void k_scattering(const double *__restrict__ g, int n_bins, double dr,
                             const double *__restrict__ q, int n_q, double n_surf, double Rg,
                             double Df, double *__restrict__ out, double *__restrict__ out_frac)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_q)
        return;
    const double qq = q[w];
    double acc = 0.0;
    for (int b = lane; b < n_bins; b += 32) {
        const double r0 = b * dr, r1 = (b + 1) * dr;
        const double t = qq > 0.0 ? scat_G(qq * r1) - scat_G(qq * r0)
                                  : (r1 * r1 * r1 - r0 * r0 * r0) / 3.0;
        acc += g[b] * t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const double four_pi = 12.566370614359172953850573533118;
        const double n2 = n_surf * n_surf;
        out[w] = n2 * (qq > 0.0 ? four_pi * acc / (qq * qq * qq) : four_pi * acc);
        if (out_frac)
            out_frac[w] = n2 * pow(qq * Rg, -Df);
    }
}

// Per-CTA partials: mode 0 -> sum of x (3 values), 1 -> sum of |x - c|^2
// (1 value), 2 -> componentwise minimum (3 values), 3 -> componentwise maximum
// of |x_d| (3 values).  Tree reduction in a fixed order inside the CTA.
template <int MODE>
__global__ void __launch_bounds__(256)
k_block_reduce(const double *__restrict__ x, int n, const double *__restrict__ c,
               double *__restrict__ part)
{
    __shared__ double s[3][256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a0, a1, a2;
    if (MODE == 2) {
        a0 = a1 = a2 = INFINITY;
        if (i < n) {
            a0 = x[i];
            a1 = x[n + i];
            a2 = x[2 * n + i];
        }
    } else if (MODE == 3) {
        a0 = a1 = a2 = 0.0;
        if (i < n) {
            a0 = fabs(x[i]);
            a1 = fabs(x[n + i]);
            a2 = fabs(x[2 * n + i]);
        }
    } else if (MODE == 0) {
        a0 = a1 = a2 = 0.0;
        if (i < n) {
            a0 = x[i];
            a1 = x[n + i];
            a2 = x[2 * n + i];
        }
    } else {
        a0 = a1 = a2 = 0.0;
        if (i < n) {
            const double e0 = __dsub_rn(c[0], x[i]), e1 = __dsub_rn(c[1], x[n + i]),
                         e2 = __dsub_rn(c[2], x[2 * n + i]);
            a0 = __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)),
                           __dmul_rn(e2, e2));
        }
    }
    s[0][threadIdx.x] = a0;
    s[1][threadIdx.x] = a1;
    s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            for (int d = 0; d < 3; ++d) {
                const double u = s[d][threadIdx.x], w = s[d][threadIdx.x + o];
                s[d][threadIdx.x] = (MODE == 2) ? fmin(u, w)
                                    : (MODE == 3) ? fmax(u, w) : __dadd_rn(u, w);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = s[0][0];
        part[3 * blockIdx.x + 1] = s[1][0];
        part[3 * blockIdx.x + 2] = s[2][0];
    }
}

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long mix64(unsigned long long k)
{
    // SplitMix64 finaliser (S. Vigna): spreads keys over the table.
    k ^= k >> 30;
    k *= 0xBF58476D1CE4E5B9ull;
    k ^= k >> 27;
    k *= 0x94D049BB133111EBull;
    k ^= k >> 31;
    return k;
}

__global__ void k_box_insert(const double *__restrict__ x, int n, const double *__restrict__ o,
                             double eps, unsigned long long *__restrict__ table,
                             unsigned long long mask, int *__restrict__ count,
                             int *__restrict__ flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    long long b[3];
    for (int k = 0; k < 3; ++k)
        b[k] = (long long)floor(__ddiv_rn(__dsub_rn(x[k * n + i], o[k]), eps));
    // triples are non-negative (o is the minimum corner); 21 bits per axis
    if (b[0] >= (1 << 21) || b[1] >= (1 << 21) || b[2] >= (1 << 21)) {
        atomicOr(flags, FLAG_BAD_CELL);
        return;
    }
    const unsigned long long key = ((unsigned long long)b[2] << 42) |
                                   ((unsigned long long)b[1] << 21) | (unsigned long long)b[0];
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&table[h], kEmpty, key);
        if (prev == kEmpty) {
            atomicAdd(count, 1);
            return;
        }
        if (prev == key)
            return;
        h = (h + 1) & mask;
    }
    atomicOr(flags, FLAG_BAD_CELL); // table full (cannot happen: size >= 2n)
}

} // namespace

cudaError_t launch_pair_hist(const double *x, int n, double r_max, int n_bins,
                             const CellGrid &g, const CellBufs &b,
                             unsigned long long *hist, cudaStream_t st)
{
    const double dr = r_max / (double)n_bins;
    // float32 prefilter radius: r_max plus a margin far above float32 rounding of
    // positions of magnitude <= g.L
    const float r_cut32 = (float)(r_max * (1.0 + 1e-4) + 1e-5 * (double)g.L + 1e-6);
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * n_bins, st);
    if (e != cudaSuccess)
        return e;
    k_pair_hist<<<(n + 255) / 256, 256, 0, st>>>(x, n, r_max, dr, n_bins, r_cut32, g,
                                                  b.start, b.sorted, b.sxq, hist);
    return cudaGetLastError();
}

cudaError_t launch_radial_hist(const double *x, int n, double r_max, int n_bins,
                               unsigned long long *hist, cudaStream_t st)
{
    const double dr = r_max / (double)n_bins;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * n_bins, st);
    if (e != cudaSuccess)
        return e;
    k_radial_hist<<<(n + 255) / 256, 256, 0, st>>>(x, n, dr, n_bins, hist);
    return cudaGetLastError();
}

cudaError_t launch_scattering(const double *g, int n_bins, double r_max, const double *q, int n_q,
                              double n_surf, double Rg, double Df, double *out,
                              double *out_frac, cudaStream_t st)
{
    const int threads = 128;
    const int grid = (n_q * 32 + threads - 1) / threads;
    k_scattering<<<grid, threads, 0, st>>>(g, n_bins, r_max / (double)n_bins, q, n_q, n_surf, Rg,
                                           Df, out, out_frac);
    return cudaGetLastError();
}

cudaError_t launch_surface_count(const double *x, const int *typ, int n, double R,
                                 const SurfHalf &hs, unsigned long long *count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess)
        return e;
    k_surface_count<<<(n + 255) / 256, 256, 0, st>>>(x, typ, n, R, hs, count);
    return cudaGetLastError();
}

cudaError_t launch_block_reduce(int mode, const double *x, int n, const double *c,
                                double *part, cudaStream_t st)
{
    const int grid = (n + 255) / 256;
    if (mode == 0)
        k_block_reduce<0><<<grid, 256, 0, st>>>(x, n, c, part);
    else if (mode == 1)
        k_block_reduce<1><<<grid, 256, 0, st>>>(x, n, c, part);
    else if (mode == 2)
        k_block_reduce<2><<<grid, 256, 0, st>>>(x, n, c, part);
    else
        k_block_reduce<3><<<grid, 256, 0, st>>>(x, n, c, part);
    return cudaGetLastError();
}

cudaError_t launch_boxcount(const double *x, int n, const double *origin, double eps,
                            unsigned long long *table, unsigned long long table_size,
                            int *count, int *flags, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(table, 0xFF, sizeof(unsigned long long) * table_size, st);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    k_box_insert<<<(n + 255) / 256, 256, 0, st>>>(x, n, origin, eps, table, table_size - 1,
                                                   count, flags);
    return cudaGetLastError();
}

} // namespace npsim
