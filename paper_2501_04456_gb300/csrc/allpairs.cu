// allpairs.cu -- all-pairs Coulomb (+ optional Lennard-Jones) forces, step (ii)
// of the loop in arXiv 2501.04456 Sec. 2.2, for every NP i:
//   F_i = sum_{j != i} [ C q_i q_j r_ij / r^3
//                       + 24 eps_ij (2 (s_ij/r)^12 - (s_ij/r)^6) r_ij / r^2 [r < rc_ij] ]
// with r_ij = x_i - x_j.  Coulomb is not truncated; LJ is truncated, not
// shifted (Sec. 2.2 step ii).
//
// Design (GB300, FP32 CUDA cores -- the pair body is not a dense contraction):
//  * positions come from a float32 mirror (x, y, z, q) written by the integrator;
//  * each thread holds KI particles i in registers; the CTA stages a tile of JT
//    particles j in shared memory and every thread sweeps it with broadcast
//    loads, so one LDS.128 feeds KI pair evaluations;
//  * the Coulomb-only body is 12 FP32 instructions + 1 MUFU.RSQ per pair: the
//    self pair is made harmless by adding 1e-20 to r^2 (its r_ij is exactly 0),
//    and q_i C is applied once per particle at the end;
//  * each j-tile's float32 partial is added into a (hi, lo) TwoSum pair, so the
//    per-particle accumulation is compensated (FP32 pair math, ~FP64 sum);
//  * the (i-tile x j-tile) work is split evenly over exactly `grid` CTAs
//    (stream-K); each CTA writes one compensated (hi, lo) float32 partial per i-tile row it
//    touches, and the integrator sums the (at most a few) partials of a row in
//    CTA order -- deterministic, and balanced to one tile for any N.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

constexpr float kSelfEps = 1e-20f;   // added to r^2: keeps the self term finite and zero
constexpr float kSelfMin = 1e-12f;   // LJ only: r^2 below this is the self pair
constexpr float kFar = 1.0e15f;      // padding position for ragged tiles

template <int BLOCK, int KI, int JT, bool LJ>
__global__ void __launch_bounds__(BLOCK)
k_allpairs(const float4 *__restrict__ xq, const int *__restrict__ typ, int n,
           StreamK sk, const PairTab *__restrict__ tab, float *__restrict__ slots)
{
    constexpr int ITILE = BLOCK * KI;
    __shared__ float4 s_x[JT];
    __shared__ int s_t[LJ ? JT : 1];
    __shared__ float4 s_tab[LJ ? NPSIM_MAX_TYPES * NPSIM_MAX_TYPES : 1];

    if (LJ) {
        for (int k = threadIdx.x; k < NPSIM_MAX_TYPES * NPSIM_MAX_TYPES; k += BLOCK)
            s_tab[k] = tab->e[k];
    }
    const int c = blockIdx.x;
    const long long p_end = sk_begin(sk, c + 1);
    long long p = sk_begin(sk, c);

    while (p < p_end) {
        const int r = (int)(p / sk.n_jt);
        const int jt0 = (int)(p - (long long)r * sk.n_jt);
        const int jt1 = (int)min((long long)sk.n_jt, (long long)jt0 + (p_end - p));

        float xi[KI], yi[KI], zi[KI];
        int trow[KI];
        float hx[KI], hy[KI], hz[KI], lx[KI], ly[KI], lz[KI];
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            const int i = r * ITILE + k * BLOCK + threadIdx.x;
            if (i < n) {
                const float4 q = xq[i];
                xi[k] = q.x;
                yi[k] = q.y;
                zi[k] = q.z;
                trow[k] = LJ ? typ[i] * NPSIM_MAX_TYPES : 0;
            } else {
                xi[k] = yi[k] = zi[k] = kFar;
                trow[k] = 0;
            }
            hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.0f;
        }

        for (int jt = jt0; jt < jt1; ++jt) {
            __syncthreads(); // the previous tile has been consumed
            for (int m = threadIdx.x; m < JT; m += BLOCK) {
                const int j = jt * JT + m;
                if (j < n) {
                    s_x[m] = xq[j];
                    if (LJ)
                        s_t[m] = typ[j];
                } else {
                    s_x[m] = make_float4(-kFar, -kFar, -kFar, 0.0f);
                    if (LJ)
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
                int tj = 0;
                if (LJ)
                    tj = s_t[m];
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const float dx = xi[k] - pj.x;
                    const float dy = yi[k] - pj.y;
                    const float dz = zi[k] - pj.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kSelfEps)));
                    const float rinv = rsqrtf(r2);
                    const float rinv2 = rinv * rinv;
                    float f;
                    if (LJ) {
                        const float4 t = s_tab[trow[k] + tj];
                        const float s2 = t.x * rinv2;
                        const float s6 = s2 * s2 * s2;
                        float flj = t.y * rinv2 * s6 * fmaf(2.0f, s6, -1.0f);
                        flj = (r2 < t.z && r2 > kSelfMin) ? flj : 0.0f;
                        f = fmaf(t.w * rinv, rinv2, flj);
                    } else {
                        f = pj.w * rinv * rinv2;
                    }
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

// Coulomb-only variant on the packed float32x2 instructions of sm_100+
// (FADD2 / FMUL2 / FFMA2: two float32 lanes per thread per instruction).  Two
// partners j0, j1 share every register pair, so a pair costs 6 packed FP32
// instructions + 1 MUFU.RSQ instead of 12 + 1: the kernel becomes bound by the
// FP32 pipes rather than by instruction issue.  Shared memory holds, per
// j-pair, (-x0, -x1, -y0, -y1) and (-z0, -z1, q0, q1), so dx = x_i + (-x_j) is
// one FADD2 with the i coordinate duplicated in both lanes.
template <int BLOCK, int KI, int JT>
__global__ void __launch_bounds__(BLOCK)
k_coulomb_x2(const float4 *__restrict__ xq, int n, StreamK sk, float *__restrict__ slots)
{
    constexpr int ITILE = BLOCK * KI;
    constexpr int JP = JT / 2;
    __shared__ float4 s_a[JP];
    __shared__ float4 s_b[JP];

    const int c = blockIdx.x;
    const long long p_end = sk_begin(sk, c + 1);
    long long p = sk_begin(sk, c);
    const float2 eps2 = make_float2(kSelfEps, kSelfEps);

    while (p < p_end) {
        const int r = (int)(p / sk.n_jt);
        const int jt0 = (int)(p - (long long)r * sk.n_jt);
        const int jt1 = (int)min((long long)sk.n_jt, (long long)jt0 + (p_end - p));

        float2 xi[KI], yi[KI], zi[KI];
        float hx[KI], hy[KI], hz[KI], lx[KI], ly[KI], lz[KI];
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            const int i = r * ITILE + k * BLOCK + threadIdx.x;
            float4 q = make_float4(kFar, kFar, kFar, 0.0f);
            if (i < n)
                q = xq[i];
            xi[k] = make_float2(q.x, q.x);
            yi[k] = make_float2(q.y, q.y);
            zi[k] = make_float2(q.z, q.z);
            hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.0f;
        }

        for (int jt = jt0; jt < jt1; ++jt) {
            __syncthreads(); // the previous tile has been consumed
            for (int m = threadIdx.x; m < JP; m += BLOCK) {
                const int j0 = jt * JT + 2 * m;
                const float4 pad = make_float4(-kFar, -kFar, -kFar, 0.0f);
                const float4 a = j0 < n ? xq[j0] : pad;
                const float4 b = j0 + 1 < n ? xq[j0 + 1] : pad;
                s_a[m] = make_float4(-a.x, -b.x, -a.y, -b.y);
                s_b[m] = make_float4(-a.z, -b.z, a.w, b.w);
            }
            __syncthreads();

            float2 ax[KI], ay[KI], az[KI];
#pragma unroll
            for (int k = 0; k < KI; ++k)
                ax[k] = ay[k] = az[k] = make_float2(0.0f, 0.0f);

#pragma unroll 2
            for (int m = 0; m < JP; ++m) {
                const float4 a = s_a[m];
                const float4 b = s_b[m];
                const float2 nx = make_float2(a.x, a.y), ny = make_float2(a.z, a.w);
                const float2 nz = make_float2(b.x, b.y), qj = make_float2(b.z, b.w);
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const float2 dx = __fadd2_rn(xi[k], nx);
                    const float2 dy = __fadd2_rn(yi[k], ny);
                    const float2 dz = __fadd2_rn(zi[k], nz);
                    float2 r2 = __ffma2_rn(dz, dz, eps2);
                    r2 = __ffma2_rn(dy, dy, r2);
                    r2 = __ffma2_rn(dx, dx, r2);
                    const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                    const float2 ri2 = __fmul2_rn(ri, ri);
                    const float2 f = __fmul2_rn(__fmul2_rn(qj, ri), ri2);
                    ax[k] = __ffma2_rn(f, dx, ax[k]);
                    ay[k] = __ffma2_rn(f, dy, ay[k]);
                    az[k] = __ffma2_rn(f, dz, az[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < KI; ++k) {
                two_sum_acc(hx[k], lx[k], ax[k].x);
                two_sum_acc(hx[k], lx[k], ax[k].y);
                two_sum_acc(hy[k], ly[k], ay[k].x);
                two_sum_acc(hy[k], ly[k], ay[k].y);
                two_sum_acc(hz[k], lz[k], az[k].x);
                two_sum_acc(hz[k], lz[k], az[k].y);
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

// Launch-shape table of the autotuner.  Scalar entries serve both the
// Coulomb-only and the Coulomb+LJ sums; packed entries only the Coulomb sum.
struct Entry {
    ApConfig cfg;
    bool packed;
    const void *fn_coul;
    const void *fn_lj;
};

#define NPSIM_AP(B, K, J)                                                               \
    Entry{ApConfig{B, K, J, 0}, false, (const void *)k_allpairs<B, K, J, false>,      \
          (const void *)k_allpairs<B, K, J, true>}
#define NPSIM_AP2(B, K, J)                                                              \
    Entry{ApConfig{B, K, J, 0}, true, (const void *)k_coulomb_x2<B, K, J>, nullptr}

const Entry kEntries[] = {
    NPSIM_AP(128, 4, 256),  NPSIM_AP(256, 4, 256),  NPSIM_AP(128, 8, 256),
    NPSIM_AP(256, 2, 512),  NPSIM_AP(64, 8, 128),   NPSIM_AP(128, 2, 256),
    NPSIM_AP(256, 8, 256),  NPSIM_AP(512, 2, 512),  NPSIM_AP2(256, 4, 256),
    NPSIM_AP2(256, 2, 256), NPSIM_AP2(128, 4, 256), NPSIM_AP2(128, 8, 256),
    NPSIM_AP2(512, 2, 512), NPSIM_AP2(256, 2, 512),
};

template <int B, int K, int J>
cudaError_t launch_one(bool lj, const StreamK &sk, const float4 *xq, const int *typ, int n,
                       const PairTab *tab, float *slots, cudaStream_t st)
{
    if (lj)
        k_allpairs<B, K, J, true><<<sk.grid, B, 0, st>>>(xq, typ, n, sk, tab, slots);
    else
        k_allpairs<B, K, J, false><<<sk.grid, B, 0, st>>>(xq, typ, n, sk, tab, slots);
    return cudaGetLastError();
}

template <int B, int K, int J>
cudaError_t launch_x2(bool lj, const StreamK &sk, const float4 *xq, int n, float *slots,
                      cudaStream_t st)
{
    if (lj)
        return cudaErrorInvalidValue;
    k_coulomb_x2<B, K, J><<<sk.grid, B, 0, st>>>(xq, n, sk, slots);
    return cudaGetLastError();
}

} // namespace

int ap_num_configs() { return (int)(sizeof(kEntries) / sizeof(kEntries[0])); }

ApConfig ap_config(int idx) { return kEntries[idx].cfg; }

bool ap_packed(int idx) { return kEntries[idx].packed; }

int ap_occupancy(int idx, bool lj)
{
    int occ = 0;
    const Entry &e = kEntries[idx];
    const void *fn = lj ? e.fn_lj : e.fn_coul;
    if (!fn)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, e.cfg.block, 0) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_allpairs(int idx, bool lj, const StreamK &sk, const float4 *xq,
                            const int *typ, int n, const PairTab *tab, float *slots,
                            cudaStream_t st)
{
    switch (idx) {
    case 0: return launch_one<128, 4, 256>(lj, sk, xq, typ, n, tab, slots, st);
    case 1: return launch_one<256, 4, 256>(lj, sk, xq, typ, n, tab, slots, st);
    case 2: return launch_one<128, 8, 256>(lj, sk, xq, typ, n, tab, slots, st);
    case 3: return launch_one<256, 2, 512>(lj, sk, xq, typ, n, tab, slots, st);
    case 4: return launch_one<64, 8, 128>(lj, sk, xq, typ, n, tab, slots, st);
    case 5: return launch_one<128, 2, 256>(lj, sk, xq, typ, n, tab, slots, st);
    case 6: return launch_one<256, 8, 256>(lj, sk, xq, typ, n, tab, slots, st);
    case 7: return launch_one<512, 2, 512>(lj, sk, xq, typ, n, tab, slots, st);
    case 8: return launch_x2<256, 4, 256>(lj, sk, xq, n, slots, st);
    case 9: return launch_x2<256, 2, 256>(lj, sk, xq, n, slots, st);
    case 10: return launch_x2<128, 4, 256>(lj, sk, xq, n, slots, st);
    case 11: return launch_x2<128, 8, 256>(lj, sk, xq, n, slots, st);
    case 12: return launch_x2<512, 2, 512>(lj, sk, xq, n, slots, st);
    case 13: return launch_x2<256, 2, 512>(lj, sk, xq, n, slots, st);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace npsim
