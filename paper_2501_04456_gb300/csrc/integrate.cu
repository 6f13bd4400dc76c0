// integrate.cu -- steps (iii)-(vi) of the loop in arXiv 2501.04456 Sec. 2.2,
// fused into one pass over the particles:
//   (iii) droplet radius by the radius-square law R(t)^2 = R0^2 - k t;
//   (iv)  interface spring: s = |x| - (R(t) - sigma/2), F += -k_wall s x/|x| if s > 0;
//   (v)   gravity -m g z^, centrifugal m w^2 (x, y, 0) (about z) or m w^2 x
//         (isotropic tumbling), viscous drag inside the Langevin O step;
//   (vi)  velocity and position update with Brownian noise:
//         BAOAB  v += dt/2 F/m; x += dt/2 v; v = c1 v + sqrt((1-c1^2) kT/m) xi;
//                x += dt/2 v; [forces at x_{n+1}]; v += dt/2 F/m,  c1 = exp(-gamma dt)
//         or overdamped  x += F dt/(m gamma) + sqrt(2 kT dt/(m gamma)) xi.
// The paper adds a fixed-magnitude random vector and has no temperature; the
// thermostat here is the fluctuation-dissipation-consistent reading of it.
//
// One kernel serves four modes (see IntMode): it sums the stream-K partials
// of the all-pairs kernel (and the cell-list LJ forces) into the total force,
// adds the external forces at t = step*dt, and applies the B half kick and/or
// the BAOA part of the next step.  Positions and velocities are float64
// (structure of arrays, coalesced); the float32 mirror (x, y, z, q) the pair
// kernels read is written whenever positions move.  The step counter lives in
// device memory and is advanced by the last CTA to finish, so a captured CUDA
// graph replays without parameter updates.
#include "npsim_internal.cuh"

namespace npsim {

namespace {

template <int MODE>
__global__ void __launch_bounds__(256)
k_integrate(IntArgs a, StepParams p)
{
    __shared__ TypeCoef s_tc[NPSIM_MAX_TYPES];
    if (threadIdx.x < NPSIM_MAX_TYPES)
        s_tc[threadIdx.x] = p.tc[threadIdx.x];
    __syncthreads();

    const int n = p.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = *a.step; // positions are x_step at t = step * dt
    constexpr bool ASSEMBLE = (MODE != MODE_A);
    constexpr bool DO_B = (MODE == MODE_BA || MODE == MODE_B);
    constexpr bool DO_A = (MODE == MODE_A || MODE == MODE_BA);

    if (i < n) {
        const int ti = a.typ[i];
        const TypeCoef tc = s_tc[ti];
        double xx = a.x[i], xy = a.x[n + i], xz = a.x[2 * n + i];
        double fx, fy, fz;
        if (ASSEMBLE) {
            fx = fy = fz = 0.0;
            const int pos = a.row_pos ? a.row_pos[i] : i;
            if (a.slots && pos >= 0) {
                const StreamK &sk = a.sk;
                const int r = pos / sk.itile;
                const int idx = pos - r * sk.itile;
                const long long u0 = (long long)r * sk.n_jt;
                const int c0 = sk_cta_of(sk, u0);
                const int c1 = sk_cta_of(sk, u0 + sk.n_jt - 1);
                for (int c = c0; c <= c1; ++c) {
                    const double *slot = a.slots + (size_t)(r + c) * 3 * sk.itile;
                    fx += slot[idx];
                    fy += slot[sk.itile + idx];
                    fz += slot[2 * sk.itile + idx];
                }
                if (a.field_slots) { // the Coulomb-only kernel returns sum_j q_j r_ij / r^3
                    fx *= tc.charge_c;
                    fy *= tc.charge_c;
                    fz *= tc.charge_c;
                }
            }
            if (a.F_lj) {
                fx += a.F_lj[i];
                fy += a.F_lj[n + i];
                fz += a.F_lj[2 * n + i];
            }
            if (a.ext_on) {
                const double t = (double)step * p.dt;
                const double R2 = p.R0 * p.R0 - p.k_evap * t;
                const double R = R2 > 0.0 ? sqrt(R2) : 0.0;
                if (p.wall) {
                    const double rr = sqrt(xx * xx + xy * xy + xz * xz);
                    const double s = rr - (R - tc.half_sigma);
                    if (s > 0.0 && rr > 0.0) {
                        const double f = -tc.k_wall * s / rr;
                        fx += f * xx;
                        fy += f * xy;
                        fz += f * xz;
                    }
                }
                fz += -tc.mass * p.g;
                if (p.rot_mode == 1) {
                    fx += tc.mass * p.omega2 * xx;
                    fy += tc.mass * p.omega2 * xy;
                } else if (p.rot_mode == 2) {
                    fx += tc.mass * p.omega2 * xx;
                    fy += tc.mass * p.omega2 * xy;
                    fz += tc.mass * p.omega2 * xz;
                }
            }
        } else {
            fx = a.F[i];
            fy = a.F[n + i];
            fz = a.F[2 * n + i];
        }

        if (MODE == MODE_FORCES) {
            a.F[i] = fx;
            a.F[n + i] = fy;
            a.F[2 * n + i] = fz;
        } else {
            double vx = a.v[i], vy = a.v[n + i], vz = a.v[2 * n + i];
            const double hdt = 0.5 * p.dt;
            if (DO_B && p.integrator == 0) {
                vx += hdt * fx * tc.inv_mass;
                vy += hdt * fy * tc.inv_mass;
                vz += hdt * fz * tc.inv_mass;
            }
            if (MODE == MODE_B) {
                a.F[i] = fx;
                a.F[n + i] = fy;
                a.F[2 * n + i] = fz;
            }
            if (DO_A) {
                double n0, n1, n2;
                normals3(p.seed, (uint32_t)i, step, 0u, n0, n1, n2);
                if (p.integrator == 0) {
                    vx += hdt * fx * tc.inv_mass;
                    vy += hdt * fy * tc.inv_mass;
                    vz += hdt * fz * tc.inv_mass;
                    xx += hdt * vx;
                    xy += hdt * vy;
                    xz += hdt * vz;
                    vx = tc.c1 * vx + tc.sd_o * n0;
                    vy = tc.c1 * vy + tc.sd_o * n1;
                    vz = tc.c1 * vz + tc.sd_o * n2;
                    xx += hdt * vx;
                    xy += hdt * vy;
                    xz += hdt * vz;
                } else {
                    xx += fx * p.dt * tc.mob + tc.sd_bd * n0;
                    xy += fy * p.dt * tc.mob + tc.sd_bd * n1;
                    xz += fz * p.dt * tc.mob + tc.sd_bd * n2;
                }
                a.x[i] = xx;
                a.x[n + i] = xy;
                a.x[2 * n + i] = xz;
                const float4 old = a.xq[i];
                a.xq[i] = make_float4((float)xx, (float)xy, (float)xz, old.w);
                if (!(isfinite(xx) && isfinite(xy) && isfinite(xz)))
                    atomicOr(a.flags, FLAG_NONFINITE);
            }
            a.v[i] = vx;
            a.v[n + i] = vy;
            a.v[2 * n + i] = vz;
        }
    }

    if (DO_A) {
        // The last CTA to finish advances the step counter: every CTA has read
        // it by the time it counts itself done.
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

__global__ void k_mirror(const double *__restrict__ x, const int *__restrict__ typ,
                         PairTab charges, int n, float4 *__restrict__ xq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    xq[i] = make_float4((float)x[i], (float)x[n + i], (float)x[2 * n + i],
                        charges.e[typ[i]].x);
}

} // namespace

// Float32 mirror (x, y, z, q) of the float64 positions.
cudaError_t launch_mirror(const double *x, const int *typ, const float *charge_by_type,
                          int n, float4 *xq, cudaStream_t st)
{
    PairTab q{};
    for (int t = 0; t < NPSIM_MAX_TYPES; ++t)
        q.e[t].x = charge_by_type[t];
    k_mirror<<<(n + 255) / 256, 256, 0, st>>>(x, typ, q, n, xq);
    return cudaGetLastError();
}

cudaError_t launch_integrate(int mode, const IntArgs &a, const StepParams &p,
                             cudaStream_t st)
{
    const int block = 256;
    const int grid = (p.n + block - 1) / block;
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
