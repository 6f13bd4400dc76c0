// allpairs_grouped.cu -- all-pairs forces (step (ii) of the loop in arXiv
// 2501.04456 Sec. 2.2) with the particles listed in a grouped order.
//
// Charge, size and LJ depth are properties of the NP type (Sec. 2.1: NPs of
// several types with their own radius, mass and charge), so the particles can
// be listed once, at creation, grouped by type (charged types first), each
// group padded to a whole number of 512-position blocks.  Every j-tile then
// holds partners of one type, and the per-pair parameters become per-tile
// constants:
//  * k_coulomb_grp (Coulomb only): the tile sum factors as
//      sum_{j in tile} q_j r_ij / r^3 = q_t sum_{j in tile} r_ij / r^3,
//    which removes the per-pair multiply by q_j: 11 FP32 operations per pair
//    on the packed float32x2 instructions (FADD2 / FMUL2 / FFMA2), two
//    partners per register pair, plus one MUFU.RSQ per pair; the tile sum is
//    multiplied by q_t once and added into a compensated (TwoSum) accumulator.
//    With two or more rows per thread the partner loop is unrolled four
//    times (8 to 16 independent pair chains per thread): at N = 250000 this
//    took <256,4,256> from 22.2 to 20.3 ms; with one row per thread the
//    registers of a fourfold unroll would halve the CTAs per SM.
//    The result is the field sum_j q_j r_ij / r^3 (the integrator multiplies
//    by C q_i).  Neutral types form the last groups; unless the caller asks
//    for the sum over all pairs (sum_neutral), it limits rows and columns to
//    the charged groups, since every Coulomb term with a neutral particle is
//    exactly zero.
//  * k_ljc_grp (LJ + Coulomb): the type-pair constants of a row and a tile are
//    loaded once per tile (ljc_tile_sweep); the result is the force.
//
// Rows (particles i) and columns (partners j) both follow the grouped order:
// perm[k] is the particle at position k (-1 for padding, placed far away).
// The (row tile x column tile) units are cut into equal ranges as in the other
// all-pairs kernels (stream-K), one compensated (hi, lo) float32 partial per
// (row, range) written to slot row + range.  The ranges are handed out at run
// time: CTA c starts on range c and then takes the next free range from a
// device counter.  Two CTAs sharing an SM do not advance at the same rate (the
// warp schedulers favour one), so with a fixed split the favoured CTA finishes
// early and leaves its SM half occupied; with several ranges per CTA it takes
// more of them instead.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

constexpr float kSelfEps = kPairSelfEps;
constexpr float kPad = kPairPad;

// The range after the current one: drawn by thread 0 from work[0] (offset by
// the CTA count: ranges below it are the CTAs' first ones) and shared through
// *s_range.  Called by every thread of the CTA.
__device__ __forceinline__ int next_range(unsigned *work, int *s_range)
{
    __syncthreads(); // every thread is done with the last range and with *s_range
    if (threadIdx.x == 0)
        *s_range = (int)gridDim.x + (int)atomicAdd(work, 1u);
    __syncthreads();
    return *s_range;
}

// The last CTA out resets both counters for the next launch: every CTA has
// drawn its last range before it counts itself out.
__device__ __forceinline__ void count_out(unsigned *work)
{
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
            work[0] = 0u;
            work[1] = 0u;
            __threadfence();
        }
    }
}

template <int BLOCK, int KI, int JT>
__global__ void __launch_bounds__(BLOCK)
k_coulomb_grp(const float4 *__restrict__ xq, const int *__restrict__ perm, int n_perm,
              const float *__restrict__ qblk, StreamK sk, unsigned *__restrict__ work,
              float *__restrict__ slots)
{
    constexpr int ITILE = BLOCK * KI;
    constexpr int JP = JT / 2;
    __shared__ float4 s_a[JP]; // (-x0, -x1, -y0, -y1)
    __shared__ float2 s_b[JP]; // (-z0, -z1)
    __shared__ int s_range;
    const float2 eps2 = make_float2(kSelfEps, kSelfEps);

    for (int c = blockIdx.x; c < sk.grid; c = next_range(work, &s_range)) {
        const long long p_end = sk_begin(sk, c + 1);
        long long p = sk_begin(sk, c);
        while (p < p_end) {
            const int r = (int)(p / sk.n_jt);
            const int jt0 = (int)(p - (long long)r * sk.n_jt);
            const int jt1 = (int)min((long long)sk.n_jt, (long long)jt0 + (p_end - p));

            float2 xi[KI], yi[KI], zi[KI];
            float hx[KI], hy[KI], hz[KI], lx[KI], ly[KI], lz[KI];
#pragma unroll
            for (int k = 0; k < KI; ++k) {
                const int pos = r * ITILE + k * BLOCK + threadIdx.x;
                const int i = pos < n_perm ? perm[pos] : -1;
                float4 q = make_float4(kPad, kPad, kPad, 0.0f);
                if (i >= 0)
                    q = xq[i];
                xi[k] = make_float2(q.x, q.x);
                yi[k] = make_float2(q.y, q.y);
                zi[k] = make_float2(q.z, q.z);
                hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.0f;
            }

            for (int jt = jt0; jt < jt1; ++jt) {
                __syncthreads(); // the previous tile has been consumed
                for (int m = threadIdx.x; m < JP; m += BLOCK) {
                    const int k0 = jt * JT + 2 * m;
                    const int j0 = perm[k0], j1 = perm[k0 + 1]; // n_perm is a multiple of JT
                    const float4 pad = make_float4(-kPad, -kPad, -kPad, 0.0f);
                    const float4 a = j0 >= 0 ? xq[j0] : pad;
                    const float4 b = j1 >= 0 ? xq[j1] : pad;
                    s_a[m] = make_float4(-a.x, -b.x, -a.y, -b.y);
                    s_b[m] = make_float2(-a.z, -b.z);
                }
                __syncthreads();

                float2 ax[KI], ay[KI], az[KI];
#pragma unroll
                for (int k = 0; k < KI; ++k)
                    ax[k] = ay[k] = az[k] = make_float2(0.0f, 0.0f);

#pragma unroll(KI >= 2 ? 4 : 2)
                for (int m = 0; m < JP; ++m) {
                    const float4 a = s_a[m];
                    const float2 nz = s_b[m];
                    const float2 nx = make_float2(a.x, a.y), ny = make_float2(a.z, a.w);
#pragma unroll
                    for (int k = 0; k < KI; ++k) {
                        const float2 dx = __fadd2_rn(xi[k], nx);
                        const float2 dy = __fadd2_rn(yi[k], ny);
                        const float2 dz = __fadd2_rn(zi[k], nz);
                        float2 r2 = __ffma2_rn(dz, dz, eps2);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dx, dx, r2);
                        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        const float2 f = __fmul2_rn(__fmul2_rn(ri, ri), ri);
                        ax[k] = __ffma2_rn(f, dx, ax[k]);
                        ay[k] = __ffma2_rn(f, dy, ay[k]);
                        az[k] = __ffma2_rn(f, dz, az[k]);
                    }
                }
                const float qt = qblk[jt * (JT / 256)];
#pragma unroll
                for (int k = 0; k < KI; ++k) { // the two partner lanes, then the charge
                    two_sum_acc(hx[k], lx[k], qt * (ax[k].x + ax[k].y));
                    two_sum_acc(hy[k], ly[k], qt * (ay[k].x + ay[k].y));
                    two_sum_acc(hz[k], lz[k], qt * (az[k].x + az[k].y));
                }
            }

            float *slot = slots + (size_t)(r + c) * 6 * ITILE; // (hi x, y, z, lo x, y, z)
#pragma unroll
            for (int k = 0; k < KI; ++k) {
                const int idx = k * BLOCK + threadIdx.x;
                slot[idx] = hx[k];
                slot[ITILE + idx] = hy[k];
                slot[2 * ITILE + idx] = hz[k];
                slot[3 * ITILE + idx] = lx[k];
                slot[4 * ITILE + idx] = ly[k];
                slot[5 * ITILE + idx] = lz[k];
            }
            p += jt1 - jt0;
        }
    }
    count_out(work);
}

// LJ + Coulomb over the type-grouped order: the constants of row k and tile
// jt come from the table passed in (full, LJ only or Coulomb only).
template <int BLOCK, int KI, int JT>
__global__ void __launch_bounds__(BLOCK)
k_ljc_grp(const float4 *__restrict__ xq, const int *__restrict__ perm, int n_perm,
          const int *__restrict__ tblk, const PairTab *__restrict__ tab, float rc2_lim,
          int has_coul, StreamK sk, unsigned *__restrict__ work, float *__restrict__ slots)
{
    constexpr int ITILE = BLOCK * KI;
    __shared__ LjcSmem<JT> sm;
    __shared__ float4 s_tab[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ int s_range;
    for (int k = threadIdx.x; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; k += BLOCK)
        s_tab[k] = tab->e[k]; // ordered before use by the first tile's barrier

    for (int c = blockIdx.x; c < sk.grid; c = next_range(work, &s_range)) {
        const long long p_end = sk_begin(sk, c + 1);
        long long p = sk_begin(sk, c);
        while (p < p_end) {
            const int r = (int)(p / sk.n_jt);
            const int jt0 = (int)(p - (long long)r * sk.n_jt);
            const int jt1 = (int)min((long long)sk.n_jt, (long long)jt0 + (p_end - p));
            ljc_row_segment<BLOCK, KI, JT>(xq, perm, tblk, 0, n_perm, s_tab, rc2_lim, has_coul,
                                           r, jt0, jt1, sm, slots + (size_t)(r + c) * 6 * ITILE);
            p += jt1 - jt0;
        }
    }
    count_out(work);
}

struct GEntry {
    ApConfig cfg;
    const void *fn;
};

#define NPSIM_GRP(B, K, J) GEntry{ApConfig{B, K, J, 0}, (const void *)k_coulomb_grp<B, K, J>}

const GEntry kGrp[] = {
    NPSIM_GRP(512, 2, 512), NPSIM_GRP(256, 2, 512), NPSIM_GRP(256, 4, 256),
    NPSIM_GRP(256, 2, 256), NPSIM_GRP(128, 4, 256), NPSIM_GRP(512, 1, 512),
    NPSIM_GRP(1024, 1, 512),
    NPSIM_GRP(256, 4, 512), NPSIM_GRP(128, 4, 512),
};

// CTAs of a dynamic launch (a static StreamK runs one CTA per range)
int dyn_ctas(const StreamK &sk) { return sk.ctas > 0 ? min(sk.ctas, sk.grid) : sk.grid; }

template <int B, int K, int J>
cudaError_t launch_g(const StreamK &sk, const float4 *xq, const int *perm, int n_perm,
                     const float *qblk, unsigned *work, float *slots, cudaStream_t st)
{
    k_coulomb_grp<B, K, J><<<dyn_ctas(sk), B, 0, st>>>(xq, perm, n_perm, qblk, sk, work, slots);
    return cudaGetLastError();
}

#define NPSIM_LJG(B, K, J) GEntry{ApConfig{B, K, J, 0}, (const void *)k_ljc_grp<B, K, J>}

const GEntry kLjg[] = {
    NPSIM_LJG(256, 1, 512), NPSIM_LJG(256, 2, 512), NPSIM_LJG(512, 1, 512),
    NPSIM_LJG(128, 2, 256), NPSIM_LJG(256, 2, 256), NPSIM_LJG(128, 4, 256),
};

template <int B, int K, int J>
cudaError_t launch_l(const StreamK &sk, const float4 *xq, const int *perm, int n_perm,
                     const int *tblk, const PairTab *tab, float rc2_lim, int has_coul,
                     unsigned *work, float *slots, cudaStream_t st)
{
    k_ljc_grp<B, K, J><<<dyn_ctas(sk), B, 0, st>>>(xq, perm, n_perm, tblk, tab, rc2_lim,
                                                    has_coul, sk, work, slots);
    return cudaGetLastError();
}

} // namespace

int grp_num_configs() { return (int)(sizeof(kGrp) / sizeof(kGrp[0])); }

ApConfig grp_config(int idx) { return kGrp[idx].cfg; }

int grp_occupancy(int idx)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kGrp[idx].fn, kGrp[idx].cfg.block,
                                                      0) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_allpairs_grouped(int idx, const StreamK &sk, const float4 *xq,
                                    const int *perm, int n_perm, const float *qblk,
                                    unsigned *work, float *slots, cudaStream_t st)
{
    switch (idx) {
    case 0: return launch_g<512, 2, 512>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 1: return launch_g<256, 2, 512>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 2: return launch_g<256, 4, 256>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 3: return launch_g<256, 2, 256>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 4: return launch_g<128, 4, 256>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 5: return launch_g<512, 1, 512>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 6: return launch_g<1024, 1, 512>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 7: return launch_g<256, 4, 512>(sk, xq, perm, n_perm, qblk, work, slots, st);
    case 8: return launch_g<128, 4, 512>(sk, xq, perm, n_perm, qblk, work, slots, st);
    default: return cudaErrorInvalidValue;
    }
}

int ljg_num_configs() { return (int)(sizeof(kLjg) / sizeof(kLjg[0])); }

ApConfig ljg_config(int idx) { return kLjg[idx].cfg; }

int ljg_occupancy(int idx)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kLjg[idx].fn, kLjg[idx].cfg.block,
                                                      0) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_allpairs_ljgrp(int idx, const StreamK &sk, const float4 *xq,
                                  const int *perm, int n_perm, const int *tblk,
                                  const PairTab *tab, float rc2_lim, int has_coul,
                                  unsigned *work, float *slots, cudaStream_t st)
{
    switch (idx) {
    case 0: return launch_l<256, 1, 512>(sk, xq, perm, n_perm, tblk, tab, rc2_lim, has_coul, work, slots, st);
    case 1: return launch_l<256, 2, 512>(sk, xq, perm, n_perm, tblk, tab, rc2_lim, has_coul, work, slots, st);
    case 2: return launch_l<512, 1, 512>(sk, xq, perm, n_perm, tblk, tab, rc2_lim, has_coul, work, slots, st);
    case 3: return launch_l<128, 2, 256>(sk, xq, perm, n_perm, tblk, tab, rc2_lim, has_coul, work, slots, st);
    case 4: return launch_l<256, 2, 256>(sk, xq, perm, n_perm, tblk, tab, rc2_lim, has_coul, work, slots, st);
    case 5: return launch_l<128, 4, 256>(sk, xq, perm, n_perm, tblk, tab, rc2_lim, has_coul, work, slots, st);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace npsim
