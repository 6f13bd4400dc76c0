// ensemble.cu -- many independent droplets of uneven size advanced together:
// one all-pairs launch and one integrator launch per step cover every droplet.
//
// Each droplet d is the system of arXiv 2501.04456 Sec. 2 (its own NP types,
// charges, LJ table, radius law, seed).  Particles of all droplets are stored
// back to back (structure of arrays over the concatenation).  The all-pairs
// work of droplet d is a rectangle of n_it(d) x n_jt(d) (i-tile x j-tile)
// units; the rectangles are laid end to end and the resulting unit sequence is
// split evenly over the CTAs (stream-K), so a 512-NP droplet and a 32768-NP
// droplet share the GPU in proportion to their N^2 work within one launch.
// A CTA writes one compensated (hi, lo) float32 partial per (global row, CTA)
// segment into slot row + CTA; the integrator sums a row's partials in CTA order.
//
// The pair body is the scalar Coulomb + truncated-LJ body of allpairs.cu with
// the droplet's own type-pair table (sigma_ab^2, 24 eps_ab, rc_ab^2, C q_a q_b);
// the integrator is the fused BAOAB / overdamped pass of integrate.cu with the
// droplet's own coefficients.  Noise is keyed by the droplet's seed and counted
// by the particle's index inside its droplet, so a droplet draws the same
// normals here as in a single-droplet run.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

constexpr float kSelfEps = 1e-20f;
constexpr float kSelfMin = 1e-12f;
constexpr float kFar = 1.0e15f;

// Droplet whose unit range contains global unit u (unit0 has n_drops + 1 entries).
__device__ __forceinline__ int drop_of_unit(const long long *__restrict__ unit0, int n_drops,
                                            long long u)
{
    int lo = 0, hi = n_drops - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (unit0[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int BLOCK, int KI, int JT>
__global__ void __launch_bounds__(BLOCK)
k_ens_allpairs(const float4 *__restrict__ xq, const int *__restrict__ typ,
               const EnsDrop *__restrict__ drops, const long long *__restrict__ unit0,
               const PairTab *__restrict__ tabs, int n_drops, StreamK sk,
               float *__restrict__ slots)
{
    constexpr int ITILE = BLOCK * KI;
    __shared__ float4 s_x[JT];
    __shared__ int s_t[JT];
    __shared__ float4 s_tab[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];

    const int c = blockIdx.x;
    const long long p_end = sk_begin(sk, c + 1);
    long long p = sk_begin(sk, c);
    int cur = -1;

    while (p < p_end) {
        const int d = drop_of_unit(unit0, n_drops, p);
        const EnsDrop &D = drops[d];
        if (d != cur) {
            __syncthreads(); // every thread is done with the previous table
            for (int k = threadIdx.x; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; k += BLOCK)
                s_tab[k] = tabs[d].e[k];
            cur = d;
        }
        const long long lu = p - D.unit0;
        const int r = (int)(lu / D.n_jt);
        const int jt0 = (int)(lu - (long long)r * D.n_jt);
        const long long left = min(p_end, D.unit0 + (long long)D.n_it * D.n_jt) - p;
        const int jt1 = (int)min((long long)D.n_jt, (long long)jt0 + left);

        float xi[KI], yi[KI], zi[KI];
        int trow[KI];
        float hx[KI], hy[KI], hz[KI], lx[KI], ly[KI], lz[KI];
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            const int li = r * ITILE + k * BLOCK + threadIdx.x;
            if (li < D.n) {
                const float4 q = xq[D.offset + li];
                xi[k] = q.x;
                yi[k] = q.y;
                zi[k] = q.z;
                trow[k] = typ[D.offset + li] * NPSIM_MAX_TYPES;
            } else {
                xi[k] = yi[k] = zi[k] = kFar;
                trow[k] = 0;
            }
            hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.0f;
        }

        for (int jt = jt0; jt < jt1; ++jt) {
            __syncthreads();
            for (int m = threadIdx.x; m < JT; m += BLOCK) {
                const int lj = jt * JT + m;
                if (lj < D.n) {
                    s_x[m] = xq[D.offset + lj];
                    s_t[m] = typ[D.offset + lj];
                } else {
                    s_x[m] = make_float4(-kFar, -kFar, -kFar, 0.0f);
                    s_t[m] = 0;
                }
            }
            __syncthreads();

            float ax[KI], ay[KI], az[KI];
#pragma unroll
            for (int k = 0; k < KI; ++k)
                ax[k] = ay[k] = az[k] = 0.0f;
#pragma unroll 4
            for (int m = 0; m < JT; ++m) {
                const float4 pj = s_x[m];
                const int tj = s_t[m];
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const float dx = xi[k] - pj.x;
                    const float dy = yi[k] - pj.y;
                    const float dz = zi[k] - pj.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kSelfEps)));
                    const float rinv = rsqrtf(r2);
                    const float rinv2 = rinv * rinv;
                    const float4 t = s_tab[trow[k] + tj];
                    const float s2 = t.x * rinv2;
                    const float s6 = s2 * s2 * s2;
                    float flj = t.y * rinv2 * s6 * fmaf(2.0f, s6, -1.0f);
                    flj = (r2 < t.z && r2 > kSelfMin) ? flj : 0.0f;
                    const float f = fmaf(t.w * rinv, rinv2, flj);
                    ax[k] = fmaf(f, dx, ax[k]);
                    ay[k] = fmaf(f, dy, ay[k]);
                    az[k] = fmaf(f, dz, az[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < KI; ++k) {
                two_sum_acc(hx[k], lx[k], ax[k]);
                two_sum_acc(hy[k], ly[k], ay[k]);
                two_sum_acc(hz[k], lz[k], az[k]);
            }
        }

        float *slot = slots + (size_t)(D.row0 + r + c) * 6 * ITILE; // hi x,y,z, lo x,y,z
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

template <int MODE>
__global__ void __launch_bounds__(256)
k_ens_integrate(EnsIntArgs a, int n_total, int n_drops, StreamK sk)
{
    // A CTA of 256 consecutive particles spans at most 256 droplets; the
    // spring radius of every (droplet, type) it touches is evaluated once.
    constexpr int kSpan = 256;
    __shared__ float2 s_reff2[kSpan * NPSIM_MAX_TYPES];
    __shared__ float s_reff[kSpan * NPSIM_MAX_TYPES];
    constexpr bool ASSEMBLE = (MODE != MODE_A);
    constexpr bool DO_A = (MODE == MODE_A || MODE == MODE_BA);
    const long long step = *a.step;
    const int i0 = blockIdx.x * blockDim.x;
    const int d0 = a.drop_of[i0]; // i0 < n_total: the grid is ceil(n_total / 256)
    if (ASSEMBLE && a.ext_on) {
        const int i_last = min(i0 + (int)blockDim.x, n_total) - 1;
        const int span = a.drop_of[i_last] - d0 + 1;
        for (int k = threadIdx.x; k < span * NPSIM_MAX_TYPES; k += blockDim.x) {
            const EnsDrop &D = a.drops[d0 + k / NPSIM_MAX_TYPES];
            spring_radius(D.R0, D.k_evap, D.dt, step, D.tc[k % NPSIM_MAX_TYPES].half_sigma,
                          s_reff2[k], s_reff[k]);
        }
        __syncthreads();
    }

    const int i = i0 + threadIdx.x;
    if (i < n_total) {
        const int n = n_total;
        const int d = a.drop_of[i];
        const EnsDrop &D = a.drops[d];
        const int li = i - D.offset;
        const int ti = a.typ[i];
        const TypeCoef tc = D.tc[ti];
        const float4 xh = a.xq[i];
        const float lx = a.x_lo[i], ly = a.x_lo[n + i], lz = a.x_lo[2 * n + i];
        float Fh[3] = {0.f, 0.f, 0.f}, Fl[3] = {0.f, 0.f, 0.f};
        if (ASSEMBLE) {
            if (a.slots) {
                const int r = li / sk.itile;
                const int idx = li - r * sk.itile;
                const long long u0 = D.unit0 + (long long)r * D.n_jt;
                const int c0 = sk_cta_of(sk, u0);
                const int c1 = sk_cta_of(sk, u0 + D.n_jt - 1);
                for (int c = c0; c <= c1; ++c) {
                    const float *slot = a.slots + (size_t)(D.row0 + r + c) * 6 * sk.itile + idx;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        df_add_df(Fh[k], Fl[k], slot[k * sk.itile], slot[(3 + k) * sk.itile]);
                }
            }
            if (a.ext_on) {
                const int e = (d - d0) * NPSIM_MAX_TYPES + ti;
                float ex, ey, ez;
                external_force(xh, lx, ly, lz, tc.kw, tc.mg, tc.mw2, s_reff2[e], s_reff[e],
                               D.wall, D.rot_mode, ex, ey, ez);
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
                               step, xh, lx, ly, lz, Fh, Fl, a.x_lo, a.v, a.F, a.xq, a.flags);
    }
    if (DO_A) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(a.done, 1u);
            if (prev == gridDim.x - 1) {
                *a.step = step + 1;
                *a.done = 0u;
                __threadfence();
            }
        }
    }
}

struct EEntry {
    ApConfig cfg;
    const void *fn;
};

#define NPSIM_ENS(B, K, J) EEntry{ApConfig{B, K, J, 0}, (const void *)k_ens_allpairs<B, K, J>}

const EEntry kEns[] = {
    NPSIM_ENS(128, 2, 256), NPSIM_ENS(128, 4, 256), NPSIM_ENS(256, 2, 256),
    NPSIM_ENS(256, 4, 256), NPSIM_ENS(64, 4, 128),  NPSIM_ENS(256, 1, 256),
};

template <int B, int K, int J>
cudaError_t launch_e(const StreamK &sk, const EnsAllpairsArgs &a, cudaStream_t st)
{
    k_ens_allpairs<B, K, J><<<sk.grid, B, 0, st>>>(a.xq, a.typ, a.drops, a.unit0, a.tabs,
                                                    a.n_drops, sk, a.slots);
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
    case 1: return launch_e<128, 4, 256>(sk, a, st);
    case 2: return launch_e<256, 2, 256>(sk, a, st);
    case 3: return launch_e<256, 4, 256>(sk, a, st);
    case 4: return launch_e<64, 4, 128>(sk, a, st);
    case 5: return launch_e<256, 1, 256>(sk, a, st);
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
