// integrate.cu -- steps (iii)-(vi) of the loop in arXiv 2501.04456 Sec. 2.2,
// fused into one pass over the particles:
//   (iii) droplet radius by the radius-square law R(t)^2 = R0^2 - k t;
//   (iv)  interface spring: s = |x| - (R(t) - sigma/2), F += -k_wall s x/|x| if s > 0
//         (wall mode 2, as printed: only while s < sigma, the band (-r, r));
//   (v)   gravity -m g z^, centrifugal m w^2 (x, y, 0) (about z) or m w^2 x
//         (isotropic tumbling), viscous drag inside the Langevin O step;
//   (vi)  velocity and position update with Brownian noise:
//         BAOAB  v += dt/2 F/m; x += dt/2 v; v = c1 v + sqrt((1-c1^2) kT/m) xi;
//                x += dt/2 v; [forces at x_{n+1}]; v += dt/2 F/m,  c1 = exp(-gamma dt)
//         or overdamped  x += F dt/(m gamma) + sqrt(2 kT dt/(m gamma)) xi,
//         or as printed  v += dt (F/m - gamma v); v += v_kick xi/|xi|; x += dt v.
// The paper adds a fixed-magnitude random vector and has no temperature; the
// thermostat (BAOAB, overdamped) is the fluctuation-dissipation-consistent
// reading of it, integrator mode 2 the step as printed.
//
// Precision without float64 arithmetic (GB300's FP64 rate is ~1/64 of FP32):
// the position is the unevaluated sum of two floats, hi (the float32 word the
// pair kernels read) + lo, updated with TwoSum (about 48 significant bits, so
// increments far below one float ulp of |x| accumulate); forces are summed as
// hi/lo pairs; velocities and the per-step increments are float32.  The
// interface distance |x| - (R - sigma/2), a difference of two nearly equal
// numbers, is formed from |x|^2 - R_eff^2 (see external_force); R(t) and
// R_eff^2 come from a per-type table evaluated once per step in float64 (by
// the first CTA of each launch that takes the A part, for the next step).
//
// One kernel serves four modes (see IntMode): it sums the stream-K partials of
// the all-pairs kernel (and the list forces: LJ, and the truncated Coulomb term
// in coulomb mode 2) into the total force, adds the external forces at
// t = step*dt, and applies the B half kick and/or the BAOA part of the next
// step (or the overdamped step, or step (vi) as printed).  The step counter
// lives in device memory so that a captured CUDA graph replays without
// parameter updates.  It holds the first step of the current chunk of steps
// and no launch of the chunk changes it but the last: a launch's step is the
// counter plus its offset within the chunk (a launch parameter), read by every
// thread together with its state, with no barrier in between.  The chunk's
// last launch counts its CTAs in once each has finished with the step, and
// the CTA that counts last moves the counter on to the next chunk.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

// Add the all-pairs partial slots of position `pos` (row pos / itile of the
// stream-K order) into (Fh, Fl): the ranges that met the row, in range order.
// Four ranges per pass, their twelve loads issued before the adds.
__device__ __forceinline__ void sum_row_slots(const float *__restrict__ slots,
                                              const StreamK &sk, int pos, float Fh[3],
                                              float Fl[3])
{
    const int r = pos / sk.itile;
    const int idx = pos - r * sk.itile;
    const long long u0 = (long long)r * sk.n_jt;
    const int c0 = sk_cta_of(sk, u0);
    const int c1 = sk_cta_of(sk, u0 + sk.n_jt - 1);
    const size_t stride = 6 * (size_t)sk.itile; // floats per slot
    const float *slot = slots + (size_t)(r + c0) * stride + idx;
    int c = c0;
    for (; c + 3 <= c1; c += 4, slot += 4 * stride) {
        float w[4][6];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int e = 0; e < 6; ++e)
                w[k][e] = __ldcs(slot + k * stride + e * sk.itile);
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                df_add_df(Fh[d], Fl[d], w[k][d], w[k][3 + d]);
    }
    for (; c <= c1; ++c, slot += stride)
#pragma unroll
        for (int d = 0; d < 3; ++d)
            df_add_df(Fh[d], Fl[d], __ldcs(slot + d * sk.itile), __ldcs(slot + (3 + d) * sk.itile));
}

// The state one particle's update reads: type, position (hi + lo), velocity
// and the list force record.
struct PartState {
    int ti;
    float4 xh;
    float lx, ly, lz;
    float v[3];
    float4 flj0, flj1;
};

template <int MODE>
__device__ __forceinline__ void load_state(const IntArgs &a, int n, int i, PartState &s)
{
    constexpr bool ASSEMBLE = (MODE != MODE_A);
    s.ti = a.typ[i];
    s.xh = a.xq[i];
    s.lx = a.x_lo[i];
    s.ly = a.x_lo[n + i];
    s.lz = a.x_lo[2 * n + i];
    if (MODE != MODE_FORCES) {
        s.v[0] = a.v[i];
        s.v[1] = a.v[n + i];
        s.v[2] = a.v[2 * n + i];
    } else {
        s.v[0] = s.v[1] = s.v[2] = 0.f;
    }
    if (ASSEMBLE && a.F_lj) {
        const float4 *r = reinterpret_cast<const float4 *>(a.F_lj + 8 * (size_t)i);
        s.flj0 = r[0]; // (hx, hy, hz, lx)
        s.flj1 = r[1]; // (ly, lz, -, -)
    } else {
        s.flj0 = s.flj1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Assemble particle i's force (partials, list forces, external forces) and
// apply the mode's part of the step.
template <int MODE>
__device__ __forceinline__ void update_particle(const IntArgs &a, const StepParams &p,
                                                const TypeCoef *s_tc, const float4 *spring,
                                                float R0f, long long step, int i,
                                                const PartState &st)
{
    constexpr bool ASSEMBLE = (MODE != MODE_A);
    const int n = p.n;
    const int ti = st.ti;
    const TypeCoef &tc = s_tc[ti];
    float Fh[3] = {0.f, 0.f, 0.f}, Fl[3] = {0.f, 0.f, 0.f};
    if (ASSEMBLE) {
        bool any = false; // some force term is in (Fh, Fl) already
        const int pos = a.row_pos ? a.row_pos[i] : i;
        if (a.slots && pos >= 0) {
            any = true;
            sum_row_slots(a.slots, a.sk, pos, Fh, Fl);
            if (a.field_slots) { // the Coulomb-only kernels return sum_j q_j r_ij / r^3
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    df_mul(Fh[d], Fl[d], tc.qc);
            }
        }
        if (a.F_lj) {
            any = true;
            df_add_df(Fh[0], Fl[0], st.flj0.x, st.flj0.w);
            df_add_df(Fh[1], Fl[1], st.flj0.y, st.flj1.x);
            df_add_df(Fh[2], Fl[2], st.flj0.z, st.flj1.y);
        }
        if (a.ext_on) {
            float ex, ey, ez;
            external_force(st.xh, st.lx, st.ly, st.lz, tc.kw, tc.mg, tc.mw2, spring[ti], p.wall,
                           p.rot_mode, ex, ey, ez, R0f,
                           MODE == MODE_FORCES ? nullptr : a.flags); // steps only
            if (any) {
                df_add(Fh[0], Fl[0], ex);
                df_add(Fh[1], Fl[1], ey);
                df_add(Fh[2], Fl[2], ez);
            } else { // the first term: (x, 0), as the compensated add into zero gives
                Fh[0] = ex;
                Fh[1] = ey;
                Fh[2] = ez;
            }
        }
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Fh[d] = a.F[d * n + i];
            Fl[d] = a.F[(3 + d) * n + i];
        }
    }
    advance_particle<MODE>(i, n, (uint32_t)i, tc, p.integrator, 0.5f * (float)p.dt, p.seed,
                           step, st.xh, st.lx, st.ly, st.lz, Fh, Fl, st.v, a.x_lo, a.v, a.F,
                           a.xq, a.flags, a.x_ref, a.nbr_gate, a.half_skin2, a.sxq, a.cell_pos,
                           ti);
}

// The per-type coefficients in shared memory and, by the first CTA of a launch
// that takes the A part, the spring radius of step + 1.
template <int MODE>
__device__ __forceinline__ void integrate_prologue(const IntArgs &a, const StepParams &p,
                                                   TypeCoef *s_tc, long long step)
{
    constexpr bool DO_A = (MODE == MODE_A || MODE == MODE_BA);
    if (threadIdx.x < NPSIM_MAX_TYPES)
        s_tc[threadIdx.x] = p.tc[threadIdx.x];
    __syncthreads();
    if (DO_A && blockIdx.x == 0 && threadIdx.x < p.n_types) // spring radius of step + 1
        a.spring[((step + 1) & 1) * NPSIM_MAX_TYPES + threadIdx.x] =
            spring_entry(p.R0, p.k_evap, p.dt, step + 1, p.tc[threadIdx.x].half_sigma);
}

// The chunk's last launch: once every thread of the CTA is past its use of the
// step, count the CTA in; the last one sets the counter to the first step of
// the next chunk.
template <int MODE>
__device__ __forceinline__ void integrate_commit(const IntArgs &a, long long step)
{
    constexpr bool DO_A = (MODE == MODE_A || MODE == MODE_BA);
    if (a.step_commit) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(a.done, 1u) == gridDim.x - 1) {
                *a.step = DO_A ? step + 1 : step;
                *a.done = 0u;
                __threadfence();
            }
        }
    }
}

// A grid of resident CTAs (at most SMs x 4 of 256 threads) striding over the
// particles: each thread has the next particle's state in flight while it
// updates the current one, and reads the step counter and the per-type
// coefficients once for all of its particles.  (One particle per thread, one
// CTA per 256, measured 1.4 % slower on 8.4 M free NPs.)
template <int MODE>
__global__ void __launch_bounds__(256, 4)
k_integrate(IntArgs a, StepParams p)
{
    __shared__ TypeCoef s_tc[NPSIM_MAX_TYPES];
    const int n = p.n;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = *a.step + a.step_ofs;
    PartState st{};
    if (i < n)
        load_state<MODE>(a, n, i, st);
    integrate_prologue<MODE>(a, p, s_tc, step);
    const float4 *spring = a.spring + (step & 1) * NPSIM_MAX_TYPES;
    const float R0f = (float)p.R0; // bound of the escape check
    while (i < n) {
        const int inext = i + stride;
        PartState nx{};
        if (inext < n)
            load_state<MODE>(a, n, inext, nx);
        update_particle<MODE>(a, p, s_tc, spring, R0f, step, i, st);
        st = nx;
        i = inext;
    }
    integrate_commit<MODE>(a, step);
}

// hi = float(x), lo = float(x - hi): the nearest float and the remainder.
__global__ void k_mirror(const double *__restrict__ x, const int *__restrict__ typ,
                         PairTab charges, int n, float4 *__restrict__ xq,
                         float *__restrict__ x_lo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float h[3];
    for (int d = 0; d < 3; ++d) {
        const double v = x[d * n + i];
        h[d] = (float)v;
        x_lo[d * n + i] = (float)(v - (double)h[d]);
    }
    xq[i] = make_float4(h[0], h[1], h[2], charges.e[typ[i]].x);
}

// x = hi + lo in float64; lo words are rows of a [3][ld] array, x is [3][n].
__global__ void k_positions_f64(const float4 *__restrict__ xq, const float *__restrict__ x_lo,
                                int n, int ld, double *__restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 h = xq[i];
    x[i] = (double)h.x + (double)x_lo[i];
    x[n + i] = (double)h.y + (double)x_lo[(size_t)ld + i];
    x[2 * n + i] = (double)h.z + (double)x_lo[2 * (size_t)ld + i];
}

// Host-facing copy of the state: AoS float64 n x 3 of the position (hi + lo),
// the velocity and the force (hi + lo); any output may be NULL.
__global__ void k_state_aos(const float4 *__restrict__ xq, const float *__restrict__ x_lo,
                            const float *__restrict__ v, const float *__restrict__ F, int n,
                            double *__restrict__ xo, double *__restrict__ vo,
                            double *__restrict__ Fo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    if (xo) {
        const float4 h = xq[i];
        xo[3 * (size_t)i + 0] = (double)h.x + (double)x_lo[i];
        xo[3 * (size_t)i + 1] = (double)h.y + (double)x_lo[n + i];
        xo[3 * (size_t)i + 2] = (double)h.z + (double)x_lo[2 * n + i];
    }
    if (vo) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            vo[3 * (size_t)i + d] = (double)v[d * n + i];
    }
    if (Fo) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            Fo[3 * (size_t)i + d] = (double)F[d * n + i] + (double)F[(3 + d) * n + i];
    }
}

// The integrator's read of the all-pairs partial slots on its own (the
// autotuner charges it to each launch shape): position p's sum to
// out[d * n_pos + p] (hi) and out[(3 + d) * n_pos + p] (lo).
__global__ void k_slot_sum(const float *__restrict__ slots, StreamK sk, int n_pos,
                           float *__restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pos)
        return;
    float Fh[3] = {0.f, 0.f, 0.f}, Fl[3] = {0.f, 0.f, 0.f};
    sum_row_slots(slots, sk, p, Fh, Fl);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        out[d * (size_t)n_pos + p] = Fh[d];
        out[(3 + d) * (size_t)n_pos + p] = Fl[d];
    }
}

} // namespace

cudaError_t launch_state_aos(const float4 *xq, const float *x_lo, const float *v, const float *F,
                             int n, double *xo, double *vo, double *Fo, cudaStream_t st)
{
    k_state_aos<<<(n + 255) / 256, 256, 0, st>>>(xq, x_lo, v, F, n, xo, vo, Fo);
    return cudaGetLastError();
}

cudaError_t launch_mirror(const double *x, const int *typ, const float *charge_by_type,
                          int n, float4 *xq, float *x_lo, cudaStream_t st)
{
    PairTab q{};
    for (int t = 0; t < NPSIM_MAX_TYPES; ++t)
        q.e[t].x = charge_by_type[t];
    k_mirror<<<(n + 255) / 256, 256, 0, st>>>(x, typ, q, n, xq, x_lo);
    return cudaGetLastError();
}

cudaError_t launch_positions_f64(const float4 *xq, const float *x_lo, int n, double *x,
                                 cudaStream_t st)
{
    k_positions_f64<<<(n + 255) / 256, 256, 0, st>>>(xq, x_lo, n, n, x);
    return cudaGetLastError();
}

cudaError_t launch_positions_f64_ld(const float4 *xq, const float *x_lo, int n, int ld,
                                    double *x, cudaStream_t st)
{
    k_positions_f64<<<(n + 255) / 256, 256, 0, st>>>(xq, x_lo, n, ld, x);
    return cudaGetLastError();
}

cudaError_t launch_slot_sum(const float *slots, const StreamK &sk, int n_pos, float *out,
                            cudaStream_t st)
{
    if (n_pos <= 0)
        return cudaSuccess;
    k_slot_sum<<<(n_pos + 255) / 256, 256, 0, st>>>(slots, sk, n_pos, out);
    return cudaGetLastError();
}

cudaError_t launch_integrate(int mode, const IntArgs &a, const StepParams &p,
                             cudaStream_t st)
{
    const int block = 256;
    // resident CTAs per device (every mode has the same register bound)
    constexpr int kMaxDev = 64;
    static int resident[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    int gmax = dev < kMaxDev ? resident[dev] : 0;
    if (gmax == 0) {
        int sms = 0, occ = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_integrate<MODE_BA>, block, 0);
        if (e != cudaSuccess)
            return e;
        gmax = sms * (occ > 0 ? occ : 1);
        if (dev < kMaxDev)
            resident[dev] = gmax;
    }
    int grid = (p.n + block - 1) / block;
    if (grid > gmax)
        grid = gmax;
    if (grid < 1)
        grid = 1;
    switch (mode) {
    case MODE_FORCES: k_integrate<MODE_FORCES><<<grid, block, 0, st>>>(a, p); break;
    case MODE_A: k_integrate<MODE_A><<<grid, block, 0, st>>>(a, p); break;
    case MODE_BA: k_integrate<MODE_BA><<<grid, block, 0, st>>>(a, p); break;
    case MODE_B: k_integrate<MODE_B><<<grid, block, 0, st>>>(a, p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

} // namespace npsim
