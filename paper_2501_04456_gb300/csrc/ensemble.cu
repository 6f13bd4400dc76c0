// ensemble.cu -- many independent droplets of uneven size advanced together:
// one all-pairs launch and one integrator launch per step cover every droplet.
//
// Each droplet d is the system of arXiv 2501.04456 Sec. 2 (its own NP types,
// charges, LJ table, radius law, seed).  Particles of all droplets are stored
// back to back (structure of arrays over the concatenation).  The all-pairs
// work of droplet d is a rectangle of n_it(d) x n_jt(d) (i-tile x j-tile)
// units; every row tile is cut into work items of at most `chunk` j-tiles,
// the items of all droplets are numbered end to end, and the CTAs of one
// launch draw items from a device counter until none are left, so a 512-NP
// and a 32768-NP droplet share the GPU in proportion to their work within one
// launch and items rich in LJ segments (which cost more than Coulomb-only
// ones) are balanced as they run.  An item writes one compensated (hi, lo)
// float32 partial per row into its own slot; the integrator sums a row's items
// in item order, so the result does not depend on which CTA ran which item.
//
// Inside the ensemble each droplet's particles are listed in a type-grouped
// order (each type's group padded to 256 positions), so every j-tile holds
// partners of one type and the pair body is the packed LJ + Coulomb sweep
// (ljc_tile_sweep) with the droplet's own type-pair table (sigma_ab^2,
// 24 eps_ab, rc_ab^2, C q_a q_b) read once per tile;
// the integrator is the fused BAOAB / overdamped pass of integrate.cu with the
// droplet's own coefficients.  Noise is keyed by the droplet's seed and counted
// by the particle's index inside its droplet, so a droplet draws the same
// normals here as in a single-droplet run.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

// Droplet whose item range contains item u (item0 has n_drops + 1 entries).
__device__ __forceinline__ int drop_of_item(const long long *__restrict__ item0, int n_drops,
                                            long long u)
{
    int lo = 0, hi = n_drops - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item0[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// At least 1024 (one row per thread) or 512 (two rows per thread) threads
// resident per SM: the register caps this implies (64, 128) hold the sweeps
// without spills.
template <int BLOCK, int KI, int JT>
__global__ void __launch_bounds__(BLOCK, KI == 1 ? 1024 / BLOCK : 512 / BLOCK)
k_ens_ljc(EnsAllpairsArgs a)
{
    constexpr int ITILE = BLOCK * KI;
    __shared__ LjcSmem<JT> sm;
    __shared__ float4 s_tab[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
    __shared__ long long s_item;
    int cur = -1;

    for (;;) {
        __syncthreads(); // every thread has read s_item and finished the last item
        if (threadIdx.x == 0)
            s_item = (long long)atomicAdd(a.work, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= a.n_items)
            break;
        const int d = drop_of_item(a.item0, a.n_drops, item);
        const EnsDrop &D = a.drops[d];
        if (d != cur) { // ordered before use by the staging barrier
            for (int k = threadIdx.x; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; k += BLOCK)
                s_tab[k] = a.tabs[d].e[k];
            cur = d;
        }
        const int li = (int)(item - D.item0);
        const int r = li / D.n_ch;
        const int jt0 = (li - r * D.n_ch) * a.chunk;
        const int jt1 = min(D.n_jt, jt0 + a.chunk);
        ljc_row_segment<BLOCK, KI, JT>(a.xq, a.perm, a.tblk, D.gpos0, D.npad, s_tab, D.rc2_lim,
                                       D.has_coul, r, jt0, jt1, sm,
                                       a.slots + (size_t)item * 6 * ITILE);
    }
    // the last CTA out resets the counters for the next launch (every CTA has
    // drawn its last item by the time it counts itself out)
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.work + 1, 1u) == gridDim.x - 1) {
            a.work[0] = 0u;
            a.work[1] = 0u;
            __threadfence();
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(256)
k_ens_integrate(EnsIntArgs a, int n_total, int n_drops, StreamK sk)
{
    constexpr bool ASSEMBLE = (MODE != MODE_A);
    constexpr bool DO_A = (MODE == MODE_A || MODE == MODE_BA);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // this thread's state first (in flight during the barrier below)
    int d = 0, ti = 0;
    float4 xh = make_float4(0.f, 0.f, 0.f, 0.f);
    float lx = 0.f, ly = 0.f, lz = 0.f;
    float v[3] = {0.f, 0.f, 0.f};
    if (i < n_total) {
        d = a.drop_of[i];
        ti = a.typ[i];
        xh = a.xq[i];
        lx = a.x_lo[i];
        ly = a.x_lo[n_total + i];
        lz = a.x_lo[2 * n_total + i];
        if (MODE != MODE_FORCES) {
            v[0] = a.v[i];
            v[1] = a.v[n_total + i];
            v[2] = a.v[2 * n_total + i];
        }
    }
    // the device step counter: read by thread 0 before the CTA's one barrier,
    // the CTA counted in right after, and the last CTA to count advances it
    __shared__ long long s_step;
    if (threadIdx.x == 0)
        s_step = *a.step;
    __syncthreads();
    const long long step = s_step;
    if (DO_A && threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(a.done, 1u);
        if (prev == gridDim.x - 1) {
            *a.step = step + 1;
            *a.done = 0u;
            __threadfence();
        }
    }
    if (DO_A) {
        // spring radii of step + 1 for every (droplet, type), spread over the
        // first CTAs of the launch (one entry per thread)
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_drops * NPSIM_MAX_TYPES;
             e += gridDim.x * blockDim.x) {
            const EnsDrop &D = a.drops[e / NPSIM_MAX_TYPES];
            a.spring[(size_t)((step + 1) & 1) * n_drops * NPSIM_MAX_TYPES + e] =
                spring_entry(D.R0, D.k_evap, D.dt, step + 1,
                             D.tc[e % NPSIM_MAX_TYPES].half_sigma);
        }
    }
    const float4 *spring = a.spring + (size_t)(step & 1) * n_drops * NPSIM_MAX_TYPES;

    if (i < n_total) {
        const int n = n_total;
        const EnsDrop &D = a.drops[d];
        const int li = i - D.offset;
        const TypeCoef tc = D.tc[ti];
        float Fh[3] = {0.f, 0.f, 0.f}, Fl[3] = {0.f, 0.f, 0.f};
        if (ASSEMBLE) {
            if (a.slots) {
                const int lpos = a.row_pos[i] - D.gpos0; // row in the droplet's grouped order
                const int r = lpos / sk.itile;
                const int idx = lpos - r * sk.itile;
                const long long it0 = D.item0 + (long long)r * D.n_ch; // the row's items
                for (int c = 0; c < D.n_ch; ++c) {
                    const float *slot = a.slots + (size_t)(it0 + c) * 6 * sk.itile + idx;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        df_add_df(Fh[k], Fl[k], slot[k * sk.itile], slot[(3 + k) * sk.itile]);
                }
            }
            if (a.ext_on) {
                float ex, ey, ez;
                external_force(xh, lx, ly, lz, tc.kw, tc.mg, tc.mw2,
                               spring[d * NPSIM_MAX_TYPES + ti], D.wall, D.rot_mode, ex, ey,
                               ez, (float)D.R0,
                               MODE == MODE_FORCES ? nullptr : a.flags); // steps only
                df_add(Fh[0], Fl[0], ex);
                df_add(Fh[1], Fl[1], ey);
                df_add(Fh[2], Fl[2], ez);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Fh[k] = a.F[k * n + i];
                Fl[k] = a.F[(3 + k) * n + i];
            }
        }
        advance_particle<MODE>(i, n, (uint32_t)li, tc, D.integrator, 0.5f * (float)D.dt, D.seed,
                               step, xh, lx, ly, lz, Fh, Fl, v, a.x_lo, a.v, a.F, a.xq, a.flags);
    }
}

struct EEntry {
    ApConfig cfg;
    const void *fn;
};

#define NPSIM_ENS(B, K, J) EEntry{ApConfig{B, K, J, 0}, (const void *)k_ens_ljc<B, K, J>}

// j-tiles of at most 256 partners: the droplets' type groups are padded to 256
const EEntry kEns[] = {
    NPSIM_ENS(128, 2, 256), NPSIM_ENS(256, 1, 256), NPSIM_ENS(256, 2, 256),
    NPSIM_ENS(1024, 1, 256), NPSIM_ENS(256, 1, 128), NPSIM_ENS(512, 1, 256),
    NPSIM_ENS(128, 1, 256), NPSIM_ENS(128, 1, 128),
};

template <int B, int K, int J>
cudaError_t launch_e(const StreamK &sk, const EnsAllpairsArgs &a, cudaStream_t st)
{
    k_ens_ljc<B, K, J><<<sk.grid, B, 0, st>>>(a);
    return cudaGetLastError();
}

} // namespace

int ens_num_configs() { return (int)(sizeof(kEns) / sizeof(kEns[0])); }

ApConfig ens_config(int idx) { return kEns[idx].cfg; }

int ens_occupancy(int idx)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kEns[idx].fn, kEns[idx].cfg.block,
                                                      0) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_ens_allpairs(int idx, const StreamK &sk, const EnsAllpairsArgs &a,
                                cudaStream_t st)
{
    switch (idx) {
    case 0: return launch_e<128, 2, 256>(sk, a, st);
    case 1: return launch_e<256, 1, 256>(sk, a, st);
    case 2: return launch_e<256, 2, 256>(sk, a, st);
    case 3: return launch_e<1024, 1, 256>(sk, a, st);
    case 4: return launch_e<256, 1, 128>(sk, a, st);
    case 5: return launch_e<512, 1, 256>(sk, a, st);
    case 6: return launch_e<128, 1, 256>(sk, a, st);
    case 7: return launch_e<128, 1, 128>(sk, a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ens_integrate(int mode, const EnsIntArgs &a, int n_total, int n_drops,
                                 const StreamK &sk, cudaStream_t st)
{
    const int grid = (n_total + 255) / 256;
    switch (mode) {
    case MODE_FORCES: k_ens_integrate<MODE_FORCES><<<grid, 256, 0, st>>>(a, n_total, n_drops, sk); break;
    case MODE_A: k_ens_integrate<MODE_A><<<grid, 256, 0, st>>>(a, n_total, n_drops, sk); break;
    case MODE_BA: k_ens_integrate<MODE_BA><<<grid, 256, 0, st>>>(a, n_total, n_drops, sk); break;
    case MODE_B: k_ens_integrate<MODE_B><<<grid, 256, 0, st>>>(a, n_total, n_drops, sk); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace npsim
