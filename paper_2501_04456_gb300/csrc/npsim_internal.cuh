// npsim_internal.cuh -- device-side types and helpers shared by the library's
// CUDA translation units (never by the CPU oracle).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/npsim.h"

namespace npsim {

// ---------------------------------------------------------------------------
// Error word bits (device int, read once per npsim_step).
enum : int {
    FLAG_NONFINITE = 1,
    FLAG_TIMEOUT = 2,
    FLAG_BAD_CELL = 4,
    FLAG_NBR_OVERFLOW = 8, // some NP had more list partners than the list holds (not an error)
    FLAG_ESCAPED = 16,     // an NP farther than 2 max(R0, R(t)) from the centre, full spring on
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (J. K. Salmon et al., "Parallel random numbers: as easy as
// 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies mixing the counter,
// with the key advanced by the two Weyl increments between rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t lo0 = c.x * m0, hi0 = __umulhi(c.x, m0);
        uint32_t lo1 = c.z * m1, hi1 = __umulhi(c.z, m1);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Three standard normals of particle i at step `step` (counter (i, step_lo,
// step_hi, purpose), key = seed).  Uniforms u = (k + 1/2) 2^-32, rounded to
// float; Box-Muller in float32 with the accurate logf, sincospif and cospif.
__device__ __forceinline__ void normals3(uint64_t seed, uint32_t i, int64_t step,
                                         uint32_t purpose, float &n0, float &n1, float &n2)
{
    const uint64_t s = (uint64_t)step;
    U4 r = philox10(U4{i, (uint32_t)s, (uint32_t)(s >> 32), purpose}, (uint32_t)seed,
                    (uint32_t)(seed >> 32));
    const float sc = 2.3283064365386963e-10f; // 2^-32
    float u0 = fmaf(__uint2float_rn(r.x), sc, 0.5f * sc);
    float u1 = fmaf(__uint2float_rn(r.y), sc, 0.5f * sc);
    float u2 = fmaf(__uint2float_rn(r.z), sc, 0.5f * sc);
    float u3 = fmaf(__uint2float_rn(r.w), sc, 0.5f * sc);
    // the radii sqrt(-2 ln u) as x rsqrt(x) (within two ulp of sqrt; 0 at u = 1)
    const float x1 = -2.0f * logf(u0), x2 = -2.0f * logf(u2);
    const float rho1 = x1 > 0.0f ? x1 * rsqrtf(x1) : 0.0f;
    const float rho2 = x2 > 0.0f ? x2 * rsqrtf(x2) : 0.0f;
    float s1, c1;
    sincospif(2.0f * u1, &s1, &c1);
    const float c3 = cospif(2.0f * u3); // the sine of this angle is not used
    n0 = rho1 * c1;
    n1 = rho1 * s1;
    n2 = rho2 * c3;
}

// Knuth's TwoSum: hi + lo accumulates a with the rounding error of hi + a
// carried in lo (compensated float32 accumulation).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float a)
{
    float s = __fadd_rn(hi, a);
    float bp = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(a, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// ---------------------------------------------------------------------------
// Pair sums over grouped (padded) orders.
constexpr float kPairSelfEps = 1e-20f; // added to r^2; the self pair has r_ij = 0 exactly
constexpr float kPairSelfMin = 1e-12f; // LJ: r^2 below this is the self pair
constexpr float kPairPad = 1.0e18f;    // padding position: every term with it underflows to 0

// One j-tile of the packed LJ + Coulomb pair sum: KI rows per thread, JP
// partner pairs staged in shared memory as negated coordinates, s_a = (-x0,
// -x1, -y0, -y1), s_b = (-z0, -z1); cst[k] = (sigma_ab^2, 24 eps_ab, rc_ab^2,
// C q_a q_b) of row k and the tile's type.  Per pair:
//   d = x_i - x_j; r^2 = d.d (+ kPairSelfEps); 1/r = rsqrt(r^2); s^6 = (sigma_ab^2/r^2)^3;
//   f = [C q_a q_b / r + [r^2 < rc_ab^2] s^6 (48 eps_ab s^6 - 24 eps_ab)] / r^2,
//   a += f d
// (the bracket is 24 eps_ab (2 s^12 - s^6) r^2 / r^2, the LJ force over r),
// on the packed float32x2 instructions, two partners per register pair: 17
// packed instructions per two pairs, two MUFU.RSQ, two cutoff selects.  DIAG
// (a tile that holds a row's own column) also masks the self pair out of the
// LJ term, whose r^-14 would overflow there.
template <int KI, bool DIAG>
__device__ __forceinline__ void ljc_tile_sweep(const float4 *__restrict__ s_a,
                                               const float2 *__restrict__ s_b, int JP,
                                               const float2 (&xi)[KI], const float2 (&yi)[KI],
                                               const float2 (&zi)[KI], const float4 (&cst)[KI],
                                               float2 (&ax)[KI], float2 (&ay)[KI],
                                               float2 (&az)[KI])
{
    const float2 eps2 = make_float2(kPairSelfEps, kPairSelfEps);
    float2 sig2[KI], e48[KI], em24[KI], cqq[KI];
#pragma unroll
    for (int k = 0; k < KI; ++k) {
        sig2[k] = make_float2(cst[k].x, cst[k].x);
        e48[k] = make_float2(2.0f * cst[k].y, 2.0f * cst[k].y);
        em24[k] = make_float2(-cst[k].y, -cst[k].y);
        cqq[k] = make_float2(cst[k].w, cst[k].w);
    }
#pragma unroll 2
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
            const float2 ri2 = __fmul2_rn(ri, ri);
            const float2 s2 = __fmul2_rn(sig2[k], ri2);
            const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
            float2 t = __fmul2_rn(s6, __ffma2_rn(e48[k], s6, em24[k]));
            if (DIAG) {
                t.x = (r2.x < cst[k].z && r2.x > kPairSelfMin) ? t.x : 0.0f;
                t.y = (r2.y < cst[k].z && r2.y > kPairSelfMin) ? t.y : 0.0f;
            } else {
                t.x = r2.x < cst[k].z ? t.x : 0.0f;
                t.y = r2.y < cst[k].z ? t.y : 0.0f;
            }
            const float2 f = __fmul2_rn(__ffma2_rn(cqq[k], ri, t), ri2);
            ax[k] = __ffma2_rn(f, dx, ax[k]);
            ay[k] = __ffma2_rn(f, dy, ay[k]);
            az[k] = __ffma2_rn(f, dz, az[k]);
        }
    }
}

// One j-tile of the Coulomb-only sum with the charge factored out: a += sum_j
// d / r^3 (the caller multiplies by the tile's C q_a q_b or q_t): 11 packed
// lanes per pair (3 sub, 3 for r^2, 2 for 1/r^3, 3 accumulate), one MUFU.RSQ.
// The self pair contributes exactly 0 (d = 0, r^2 = kPairSelfEps).
template <int KI>
__device__ __forceinline__ void coul_tile_sweep(const float4 *__restrict__ s_a,
                                                const float2 *__restrict__ s_b, int JP,
                                                const float2 (&xi)[KI], const float2 (&yi)[KI],
                                                const float2 (&zi)[KI], float2 (&ax)[KI],
                                                float2 (&ay)[KI], float2 (&az)[KI])
{
    const float2 eps2 = make_float2(kPairSelfEps, kPairSelfEps);
#pragma unroll 2
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
}

// Axis-aligned box of points: lo = +inf, hi = -inf when empty.
struct Box3 {
    float lx, ly, lz, hx, hy, hz;
};

__device__ __forceinline__ Box3 box_empty()
{
    return Box3{INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
}

__device__ __forceinline__ void box_add(Box3 &b, float x, float y, float z)
{
    b.lx = fminf(b.lx, x);
    b.ly = fminf(b.ly, y);
    b.lz = fminf(b.lz, z);
    b.hx = fmaxf(b.hx, x);
    b.hy = fmaxf(b.hy, y);
    b.hz = fmaxf(b.hz, z);
}

// Box of the points of the whole warp, in every lane.
__device__ __forceinline__ Box3 box_warp_reduce(Box3 b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b.lx = fminf(b.lx, __shfl_xor_sync(0xffffffffu, b.lx, o));
        b.ly = fminf(b.ly, __shfl_xor_sync(0xffffffffu, b.ly, o));
        b.lz = fminf(b.lz, __shfl_xor_sync(0xffffffffu, b.lz, o));
        b.hx = fmaxf(b.hx, __shfl_xor_sync(0xffffffffu, b.hx, o));
        b.hy = fmaxf(b.hy, __shfl_xor_sync(0xffffffffu, b.hy, o));
        b.hz = fmaxf(b.hz, __shfl_xor_sync(0xffffffffu, b.hz, o));
    }
    return b;
}

// Warp-reduce b and store lane 0's result as 6 floats at s_red[6 * warp]; the
// caller synchronises the block and then calls box_gather.
__device__ __forceinline__ void box_warp_store(Box3 b, float *s_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b.lx = fminf(b.lx, __shfl_xor_sync(0xffffffffu, b.lx, o));
        b.ly = fminf(b.ly, __shfl_xor_sync(0xffffffffu, b.ly, o));
        b.lz = fminf(b.lz, __shfl_xor_sync(0xffffffffu, b.lz, o));
        b.hx = fmaxf(b.hx, __shfl_xor_sync(0xffffffffu, b.hx, o));
        b.hy = fmaxf(b.hy, __shfl_xor_sync(0xffffffffu, b.hy, o));
        b.hz = fmaxf(b.hz, __shfl_xor_sync(0xffffffffu, b.hz, o));
    }
    if ((threadIdx.x & 31) == 0) {
        float *r = s_red + 6 * (threadIdx.x >> 5);
        r[0] = b.lx;
        r[1] = b.ly;
        r[2] = b.lz;
        r[3] = b.hx;
        r[4] = b.hy;
        r[5] = b.hz;
    }
}

__device__ __forceinline__ Box3 box_gather(const float *s_red, int n_warps)
{
    Box3 b = box_empty();
    for (int w = 0; w < n_warps; ++w) {
        const float *r = s_red + 6 * w;
        b.lx = fminf(b.lx, r[0]);
        b.ly = fminf(b.ly, r[1]);
        b.lz = fminf(b.lz, r[2]);
        b.hx = fmaxf(b.hx, r[3]);
        b.hy = fmaxf(b.hy, r[4]);
        b.hz = fmaxf(b.hz, r[5]);
    }
    return b;
}

// Squared distance between two boxes (0 if they overlap; +inf if one is empty).
__device__ __forceinline__ float box_gap2(const Box3 &a, const Box3 &b)
{
    if (a.lx > a.hx || b.lx > b.hx)
        return INFINITY;
    const float gx = fmaxf(0.0f, fmaxf(b.lx - a.hx, a.lx - b.hx));
    const float gy = fmaxf(0.0f, fmaxf(b.ly - a.hy, a.ly - b.hy));
    const float gz = fmaxf(0.0f, fmaxf(b.lz - a.hz, a.lz - b.hz));
    return gx * gx + gy * gy + gz * gz;
}

// 16-byte asynchronous copy global -> shared (cp.async, L2 only), and its
// completion by the issuing thread.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_own()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Shared memory of ljc_row_segment: two staged j-tiles (negated coordinates,
// two partners per entry, and the box of each 64-partner segment) -- one
// swept while the next is filled -- and the raw partner records of the next
// tile as gathered by cp.async.
template <int JT>
struct LjcSmem {
    float4 raw[JT];      // (x, y, z, q) of the next tile's partners, grouped order
    float4 a[2][JT / 2]; // (-x0, -x1, -y0, -y1)
    float2 b[2][JT / 2]; // (-z0, -z1)
    Box3 seg[2][JT / 64];
};

// Staging of entry m (partners 2m, 2m + 1) of a j-tile from its raw records:
// negated, paired coordinates and, by a warp reduction (whole warps stage), the
// box of the warp's 64 partners.  vmask bit k: partner 2m + k is a particle
// (not padding).
template <int JT>
__device__ __forceinline__ void ljc_stage_entry(LjcSmem<JT> &sm, int buf, int m, float4 a,
                                                float4 b, int vmask)
{
    sm.a[buf][m] = make_float4(-a.x, -b.x, -a.y, -b.y);
    sm.b[buf][m] = make_float2(-a.z, -b.z);
    Box3 pb = box_empty();
    if (vmask & 1)
        box_add(pb, a.x, a.y, a.z);
    if (vmask & 2)
        box_add(pb, b.x, b.y, b.z);
    pb = box_warp_reduce(pb); // the 32 entries m of this warp = one segment
    if ((threadIdx.x & 31) == 0)
        sm.seg[buf][m >> 5] = pb;
}

// Row tile r (rows r*ITILE .. of a grouped order occupying positions [gbase,
// gbase + glen) of perm / tblk) against its j-tiles jt0 .. jt1-1 of the same
// order; writes the row partials, as compensated (hi, lo) pairs, to slot
// [6][ITILE].  For every (warp, 64-partner segment) pair the LJ term is
// evaluated only when the box of the warp's rows and the box of the segment
// come within sqrt(rc2_lim); elsewhere the Coulomb-only sweep runs (the charge
// product applied once per tile), or nothing when has_coul is 0.  s_tab: the
// 8 x 8 type-pair table (sigma^2, 24 eps, rc^2, C q q) in shared memory.
//
// Staging is software-pipelined: while tile jt is swept, the first JT/2
// threads have the partner records of tile jt + 1 in flight (cp.async into
// sm.raw, the partner indices read one tile earlier still) and turn them into
// the other staged buffer after the sweep, so one barrier per tile remains and
// the gather's latency hides behind the sweep.
template <int BLOCK, int KI, int JT>
__device__ __forceinline__ void ljc_row_segment(const float4 *__restrict__ xq,
                                                const int *__restrict__ perm,
                                                const int *__restrict__ tblk, int gbase,
                                                int glen, const float4 *__restrict__ s_tab,
                                                float rc2_lim, int has_coul, int r, int jt0,
                                                int jt1, LjcSmem<JT> &sm, float *__restrict__ slot)
{
    constexpr int ITILE = BLOCK * KI;
    constexpr int JP = JT / 2;
    constexpr int NSEG = JT / 64;
    static_assert(JP <= BLOCK && JP % 32 == 0, "one staged entry per thread of whole warps");
    float2 xi[KI], yi[KI], zi[KI];
    int trow[KI];
    float hx[KI], hy[KI], hz[KI], lx[KI], ly[KI], lz[KI];
    Box3 wb = box_empty();
#pragma unroll
    for (int k = 0; k < KI; ++k) {
        const int lpos = r * ITILE + k * BLOCK + threadIdx.x;
        const bool in = lpos < glen;
        const int i = in ? perm[gbase + lpos] : -1;
        float4 q = make_float4(kPairPad, kPairPad, kPairPad, 0.0f);
        if (i >= 0) {
            q = xq[i];
            box_add(wb, q.x, q.y, q.z);
        }
        xi[k] = make_float2(q.x, q.x);
        yi[k] = make_float2(q.y, q.y);
        zi[k] = make_float2(q.z, q.z);
        trow[k] = (in ? tblk[(gbase + lpos) >> 8] : 0) * NPSIM_MAX_TYPES;
        hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.0f;
    }
    wb = box_warp_reduce(wb); // the box of this warp's rows

    const bool stager = threadIdx.x < JP;
    const int m = threadIdx.x;
    const float4 pad = make_float4(-kPairPad, -kPairPad, -kPairPad, 0.0f);
    int pn0 = -1, pn1 = -1; // partner indices of the tile after the one staged next
    if (stager) {           // tile jt0 staged synchronously (glen is a multiple of JT)
        const int k0 = gbase + jt0 * JT + 2 * m;
        const int j0 = perm[k0], j1 = perm[k0 + 1];
        if (jt0 + 1 < jt1) {
            pn0 = perm[k0 + JT];
            pn1 = perm[k0 + JT + 1];
        }
        ljc_stage_entry<JT>(sm, 0, m, j0 >= 0 ? xq[j0] : pad, j1 >= 0 ? xq[j1] : pad,
                            (j0 >= 0) | ((j1 >= 0) << 1));
    }
    __syncthreads();

    for (int jt = jt0; jt < jt1; ++jt) {
        const int cur = (jt - jt0) & 1;
        const bool next = jt + 1 < jt1; // uniform over the block
        int vmask = 0;
        if (stager && next) { // gather tile jt + 1 while this one is swept
            vmask = (pn0 >= 0) | ((pn1 >= 0) << 1);
            if (pn0 >= 0)
                cp_async16(&sm.raw[2 * m], xq + pn0);
            else
                sm.raw[2 * m] = pad;
            if (pn1 >= 0)
                cp_async16(&sm.raw[2 * m + 1], xq + pn1);
            else
                sm.raw[2 * m + 1] = pad;
            cp_async_commit();
            if (jt + 2 < jt1) {
                const int k2 = gbase + (jt + 2) * JT + 2 * m;
                pn0 = perm[k2];
                pn1 = perm[k2 + 1];
            }
        }

        const int tt = tblk[(gbase + jt * JT) >> 8]; // one type per tile
        float4 cst[KI];
        float2 ax[KI], ay[KI], az[KI], cx[KI], cy[KI], cz[KI];
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            cst[k] = s_tab[trow[k] + tt];
            ax[k] = ay[k] = az[k] = cx[k] = cy[k] = cz[k] = make_float2(0.0f, 0.0f);
        }
        const bool diag = jt * JT < (r + 1) * ITILE && (jt + 1) * JT > r * ITILE;
        for (int sg = 0; sg < NSEG; ++sg) { // warp-uniform choice per segment
            const bool lj = rc2_lim > 0.0f && box_gap2(wb, sm.seg[cur][sg]) <= rc2_lim;
            const float4 *sa = sm.a[cur] + 32 * sg;
            const float2 *sb = sm.b[cur] + 32 * sg;
            if (lj && diag)
                ljc_tile_sweep<KI, true>(sa, sb, 32, xi, yi, zi, cst, ax, ay, az);
            else if (lj)
                ljc_tile_sweep<KI, false>(sa, sb, 32, xi, yi, zi, cst, ax, ay, az);
            else if (has_coul)
                coul_tile_sweep<KI>(sa, sb, 32, xi, yi, zi, cx, cy, cz);
        }
#pragma unroll
        for (int k = 0; k < KI; ++k) {
            const float qq = cst[k].w; // C q_a q_b of the Coulomb-only segments
            two_sum_acc(hx[k], lx[k], fmaf(qq, cx[k].x + cx[k].y, ax[k].x + ax[k].y));
            two_sum_acc(hy[k], ly[k], fmaf(qq, cy[k].x + cy[k].y, ay[k].x + ay[k].y));
            two_sum_acc(hz[k], lz[k], fmaf(qq, cz[k].x + cz[k].y, az[k].x + az[k].y));
        }

        if (stager && next) { // this thread's copies have landed: stage tile jt + 1
            cp_async_wait_own();
            ljc_stage_entry<JT>(sm, cur ^ 1, m, sm.raw[2 * m], sm.raw[2 * m + 1], vmask);
        }
        __syncthreads(); // tile jt + 1 staged; tile jt's buffer free again
    }

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
}

// ---------------------------------------------------------------------------
// Per-type coefficients used by the integrator (computed on the host in
// float64 from npsim_type_t and the scenario).
struct TypeCoef {
    double mass, inv_mass, half_sigma, k_wall;
    double c1, sd_o;    // BAOAB O step: v <- c1 v + sd_o xi
    double mob, sd_bd;  // overdamped: x += F dt mob + sd_bd xi
    double charge_c;    // C * q (Coulomb-only all-pairs kernel returns the field)
    // float32 copies used by the integrator (all of its arithmetic is float32 or
    // compensated float32): dt/(2m), c1 as hi + lo (its rounding error would
    // otherwise compound over the 1/(gamma dt) steps a velocity remembers),
    // sd_o, dt*mob, sd_bd, C q, m g, m w^2, k_wall, sigma/2; for the printed
    // step (vi) dt/m, gamma dt and the kick magnitude
    float hdt_m, c1f, c1lo, sd_of, dt_mob, sd_bdf, qc, mg, mw2, kw, hs;
    float dt_m, gdt, kick;
};

// ---------------------------------------------------------------------------
// Compensated float32 ("double-float") arithmetic: a value is an unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
// Every operation is rounded separately (no fused multiply-add contraction).

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ float2 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return make_float2(s, e);
}

// Dekker's Fast2Sum (|a| >= |b| or a == 0): s + e == a + b exactly.
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// (h, l) += b, renormalised.
__device__ __forceinline__ void df_add(float &h, float &l, float b)
{
    const float2 t = df_two_sum(h, b);
    const float2 u = df_fast_two_sum(t.x, __fadd_rn(t.y, l));
    h = u.x;
    l = u.y;
}

// (h, l) += (bh, bl), renormalised.
__device__ __forceinline__ void df_add_df(float &h, float &l, float bh, float bl)
{
    const float2 t = df_two_sum(h, bh);
    const float2 u = df_fast_two_sum(t.x, __fadd_rn(__fadd_rn(t.y, l), bl));
    h = u.x;
    l = u.y;
}

// (h, l) *= b (float), renormalised; the product of h and b is exact via FMA.
__device__ __forceinline__ void df_mul(float &h, float &l, float b)
{
    const float p = __fmul_rn(h, b);
    const float e = __fmaf_rn(h, b, -p);
    const float2 u = df_fast_two_sum(p, __fmaf_rn(l, b, e));
    h = u.x;
    l = u.y;
}

// Equilibrium radius of the interface spring for a particle of half-diameter
// hs at t = step dt: R_eff = R(t) - hs with R(t)^2 = R0^2 - k t (radius-square
// law, 0 once the droplet has gone).  Returned as (R_eff^2 hi, R_eff^2 lo,
// R_eff, 2 hs = the width of the band (-r, r) about the surface) from one
// float64 evaluation.  Host and device both call this (the
// explicit fma fixes the rounding), so a table set by the host equals the one
// the integrator writes for the same step bit for bit.
__host__ __device__ inline float4 spring_entry(double R0, double k_evap, double dt,
                                               long long step, double hs)
{
    const double t = (double)step * dt;
    const double R2 = fma(-k_evap, t, R0 * R0);
    const double R = R2 > 0.0 ? sqrt(R2) : 0.0;
    const double re = R - hs;
    const double re2 = re * re;
    const float h = (float)re2;
    return make_float4(h, (float)(re2 - (double)h), (float)re, (float)(2.0 * hs));
}

// External forces (interface spring, gravity, centrifugal) on a particle at
// x = xh + xl (float hi / lo words).  The spring needs s = |x| - R_eff, the
// difference of two nearly equal numbers; it is formed as
// (|x|^2 - R_eff^2) / (|x| + R_eff) with |x|^2 from exact products and sums
// (the lo^2 terms lie below the precision kept), so s keeps float32 relative
// precision however large |x| is.  wall = 2 limits the spring to the band
// (-r, r) about the surface, 0 < s < 2 r (spring.w = 2 r).
//
// With flags given, the failure check of the interface (no counterpart in the
// paper, whose runs rely on strong damping for stability) runs on the NPs near
// or beyond the surface: with the full spring on (wall 1) no NP gets farther
// than twice the larger of R0 and R(t) from the centre unless a step went
// unstable (twice R(t) alone is not a bound: under a fast compression a heavy
// NP can lag the moving interface by more than R(t) itself); R(t) = R_eff +
// sigma/2 from the spring entry.  Sets FLAG_ESCAPED.
__device__ __forceinline__ void external_force(const float4 &xh, float lx, float ly, float lz,
                                               float kw, float mg, float mw2, float4 spring,
                                               int wall, int rot_mode, float &fx,
                                               float &fy, float &fz, float R0 = 0.0f,
                                               int *flags = nullptr)
{
    fx = fy = fz = 0.0f;
    // the spring acts only beyond R_eff (s > 0): an NP whose float32 |x|^2 from
    // the hi words lies below (R_eff - 0.01)^2 is certainly inside (the lo words
    // and the rounding of that sum move |x| by far less than 0.01), so the
    // exact distance is formed only near the surface
    const float reff_in = spring.z - 0.01f;
    const float r2_cheap = __fmaf_rn(xh.x, xh.x, __fmaf_rn(xh.y, xh.y, __fmul_rn(xh.z, xh.z)));
    if (wall && !(reff_in > 0.0f && r2_cheap < reff_in * reff_in)) {
        if (flags && wall == 1) {
            const float R = fmaxf(__fmaf_rn(0.5f, spring.w, spring.z), R0);
            if (r2_cheap > __fmul_rn(4.0f, __fmul_rn(R, R)))
                atomicOr(flags, FLAG_ESCAPED);
        }
        float r2h = 0.0f, r2l = 0.0f;
        const float hh[3] = {xh.x, xh.y, xh.z}, ll[3] = {lx, ly, lz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float p = __fmul_rn(hh[d], hh[d]);
            const float e = __fmaf_rn(hh[d], hh[d], -p);
            df_add_df(r2h, r2l, p, __fmaf_rn(2.0f * hh[d], ll[d], e));
        }
        // |x| and 1/|x| from one rsqrt (a few ulp: far below the force tolerance);
        // every operation below is rounded explicitly, so the force does not
        // depend on how the compiler fuses operations in each kernel that
        // inlines this (the integrator's modes must agree bit for bit)
        const float rinv = rsqrtf(r2h);
        const float reff = spring.z;
        float s;
        if (reff > 0.0f) {
            float dh = r2h, dl = r2l;
            df_add_df(dh, dl, -spring.x, -spring.y);
            s = __fdividef(dh, __fmaf_rn(r2h, rinv, reff)); // (|x|^2 - R_eff^2) / (|x| + R_eff)
        } else {
            s = __fmaf_rn(r2h, rinv, -reff);
        }
        if (s > 0.0f && r2h > 0.0f && (wall != 2 || s < spring.w)) {
            const float f = __fmul_rn(__fmul_rn(-kw, s), rinv);
            fx = __fmul_rn(f, xh.x);
            fy = __fmul_rn(f, xh.y);
            fz = __fmul_rn(f, xh.z);
        }
    }
    fz = __fsub_rn(fz, mg);
    if (rot_mode == 1) {
        fx = __fmaf_rn(mw2, xh.x, fx);
        fy = __fmaf_rn(mw2, xh.y, fy);
    } else if (rot_mode == 2) {
        fx = __fmaf_rn(mw2, xh.x, fx);
        fy = __fmaf_rn(mw2, xh.y, fy);
        fz = __fmaf_rn(mw2, xh.z, fz);
    }
}

struct StepParams {
    int n;
    int n_types;
    int rot_mode;
    int wall;
    int integrator;
    int pad_;
    uint64_t seed;
    double dt, R0, k_evap, g, omega2;
    TypeCoef tc[NPSIM_MAX_TYPES];
};

// Stream-K decomposition of the all-pairs sum: W = n_it * n_jt work units
// (i-tile x j-tile) split evenly into `grid` ranges; range c covers units
// [W c / grid, W (c+1) / grid).  The part of i-tile row r computed in range c
// is written to partial slot r + c (unique: rows and ranges both advance
// along the unit order).  A static launch runs range c on CTA c; a dynamic
// launch (the grouped kernels) starts `ctas` CTAs on ranges 0 .. ctas - 1 and
// hands out the rest from a device counter, so a CTA that runs ahead of the
// others on its SM takes more ranges.  Slots depend only on the range, so the
// sums do not depend on which CTA ran which range.
struct StreamK {
    int itile;   // i per CTA tile = block * ki
    int jtile;   // j per shared-memory tile
    int n_it;    // number of i tiles
    int n_jt;    // number of j tiles
    int grid;    // ranges (= CTAs of a static launch)
    int ctas;    // CTAs of a dynamic launch (<= grid; 0 for static launches)
    long long W; // n_it * n_jt
};

__host__ __device__ __forceinline__ long long sk_begin(const StreamK &s, int c)
{
    return s.W * (long long)c / s.grid;
}

// First CTA whose range contains unit p.
__host__ __device__ __forceinline__ int sk_cta_of(const StreamK &s, long long p)
{
    int c = (int)(p * s.grid / s.W);
    while (c + 1 < s.grid && sk_begin(s, c + 1) <= p)
        ++c;
    while (c > 0 && sk_begin(s, c) > p)
        --c;
    return c;
}

// LJ / Coulomb type-pair table entry: (sigma_ab^2, 24 eps_ab, rc_ab^2, C q_a q_b).
// Stored 8 x 8 (row a, column b).
struct PairTab {
    float4 e[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
};

// Cell grid for the LJ cutoff path.
struct CellGrid {
    int dim;        // cells per axis
    int n_cells;    // dim^3
    float inv_h;    // 1 / cell edge
    float L;        // grid covers [-L, L)^3; coordinates outside are clamped
    int tb;         // type blocks of the sort key: key = type * n_cells + cell when
                    // tb > 1 (cell order grouped by type first), key = cell when tb == 1
    // stencil half-width (in cells) per type pair: partners of type b of an NP of
    // type a within its list radius lie within ext[a * 8 + b] cells along each
    // axis (1 when the edge is at least every radius)
    unsigned char ext[NPSIM_MAX_TYPES * NPSIM_MAX_TYPES];
};

// Record a message for npsim_last_error() on this thread and return `code`
// (defined in capi.cu).
int report_error(int code, const char *fmt, ...);

// An NVTX range named after the C-ABI entry point it is declared in, for the
// length of the call: the calls show on Nsight Systems timelines above the
// kernels they launch (the NVTX calls do nothing when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define NP_TRACE() ::npsim::TraceRange np_trace_range_(__func__)

// ---------------------------------------------------------------------------
// Launchers (host functions defined in the .cu files).

struct ApConfig {
    int block, ki, jt, occ;
};

// All-pairs kernels (allpairs.cu)
int ap_num_configs();
ApConfig ap_config(int idx);
int ap_occupancy(int idx, bool lj);
bool ap_packed(int idx); // float32x2 Coulomb-only kernel
// Charge-grouped packed Coulomb kernel (allpairs_grouped.cu): rows and columns
// follow perm (grouped by charge, groups padded to 512), qblk = charge of each
// 256-position block.
int grp_num_configs();
ApConfig grp_config(int idx);
int grp_occupancy(int idx);
// work: two zeroed device counters (ranges handed out, CTAs done), reset to 0
// by the last CTA of each launch; launches sharing one pair must not overlap.
cudaError_t launch_allpairs_grouped(int idx, const StreamK &sk, const float4 *xq,
                                    const int *perm, int n_perm, const float *qblk,
                                    unsigned *work, float *slots, cudaStream_t st);
// Type-grouped packed LJ + Coulomb kernel (allpairs_grouped.cu): rows and
// columns follow perm (grouped by type, groups padded to 512), tblk = type of
// each 256-position block; the table selects LJ + Coulomb, LJ or Coulomb.
int ljg_num_configs();
ApConfig ljg_config(int idx);
int ljg_occupancy(int idx);
// rc2_lim: LJ is evaluated only between tiles whose boxes come within
// sqrt(rc2_lim) (0: no LJ); has_coul = 0 skips the other tiles entirely.
cudaError_t launch_allpairs_ljgrp(int idx, const StreamK &sk, const float4 *xq,
                                  const int *perm, int n_perm, const int *tblk,
                                  const PairTab *tab, float rc2_lim, int has_coul,
                                  unsigned *work, float *slots, cudaStream_t st);
cudaError_t launch_allpairs(int cfg_idx, bool lj, const StreamK &sk, const float4 *xq,
                            const int *typ, int n, const PairTab *tab, float *slots,
                            cudaStream_t st);

// Integrator (integrate.cu)
enum IntMode : int {
    MODE_FORCES = 0, // assemble F from partials + external, write F
    MODE_A = 1,      // BAOA (or overdamped update) from the stored F; step += 1
    MODE_BA = 2,     // assemble F, finish the step (B), then BAOA of the next; step += 1
    MODE_B = 3,      // assemble F, finish the step (B), write F and v
};

// State of the integrator: position = xq.xyz (float32, the word the pair kernels
// read) + x_lo (float32 SoA [3][n]); velocity float32 SoA [3][n]; force as
// float32 hi/lo SoA [6][n] (hi x, y, z, then lo x, y, z).  Stream-K partial
// slots use the same hi/lo split; the cell-list LJ forces are one 32-byte
// (hi x, y, z, lo x, y, z, 0, 0) record per NP, indexed by particle.
struct IntArgs {
    float *x_lo, *v, *F;     // see above
    const int *typ;
    float4 *xq;              // (x hi, y hi, z hi, q)
    const float *slots;      // stream-K partials [slot][6][itile] (or NULL)
    StreamK sk;
    const float *F_lj;       // cell-list LJ forces [n][8] (hi x, y, z, lo x, y, z, 0, 0) (or NULL)
    const int *row_pos;      // grouped layout: position of particle i in the rows (-1:
                             // no Coulomb partial); NULL: row position = i
    const float4 *x_ref;     // positions at the last neighbour-list build (or NULL)
    float4 *sxq;             // cell-ordered current positions of the neighbour-list
    const int *cell_pos;     // kernel, and the slot of NP i (both NULL without one)
    int *nbr_gate;           // set to 1 when an NP has moved more than half the skin
    float half_skin2;        // (skin / 2)^2, with margin
    float4 *spring;          // spring radius per type (spring_entry), two buffers
                             // [2][NPSIM_MAX_TYPES]: buffer (step & 1) holds the
                             // current step's; modes that advance the step write
                             // the other one for step + 1
    int ext_on;              // add external forces
    int field_slots;         // slots hold sum_j q_j r_ij/r^3 (Coulomb-only kernel): scale by C q_i
    long long *step;         // device step counter: the first step of the current chunk
    int step_ofs;            // this launch's step = *step + step_ofs
    int step_commit;         // last launch of a chunk: set *step to this launch's step
                             // (+ 1 in the modes that take the A part) once every CTA
                             // has read it
    int *flags;
    unsigned *done;          // CTAs counted in by the committing launch (zero between)
};

// One particle's update after its force (Fh + Fl) has been assembled: store F
// (MODE_FORCES, MODE_B), the closing half kick B (MODE_BA, MODE_B) and the
// B-A-O-A part of the next step, or the overdamped update (MODE_A, MODE_BA).
// Arrays are SoA over n particles: x_lo [3][n], v_ [3][n], F [6][n]; xq holds
// the hi words of the position.  Noise is drawn for particle noise_idx.
template <int MODE>
__device__ __forceinline__ void advance_particle(int i, int n, uint32_t noise_idx,
                                                 const TypeCoef &tc, int integrator, float hdt,
                                                 uint64_t seed, long long step, const float4 &xh,
                                                 float lx, float ly, float lz, const float Fh[3],
                                                 const float Fl[3], const float (&v0)[3],
                                                 float *x_lo, float *v_, float *F, float4 *xq,
                                                 int *flags,
                                                 const float4 *x_ref = nullptr,
                                                 int *nbr_gate = nullptr, float half_skin2 = 0.f,
                                                 float4 *sxq = nullptr,
                                                 const int *cell_pos = nullptr, int ti = 0)
{
    constexpr bool DO_B = (MODE == MODE_BA || MODE == MODE_B);
    constexpr bool DO_A = (MODE == MODE_A || MODE == MODE_BA);
    if (MODE == MODE_FORCES || MODE == MODE_B) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            F[d * n + i] = Fh[d];
            F[(3 + d) * n + i] = Fl[d];
        }
    }
    if (MODE == MODE_FORCES)
        return;
    const float f[3] = {__fadd_rn(Fh[0], Fl[0]), __fadd_rn(Fh[1], Fl[1]),
                        __fadd_rn(Fh[2], Fl[2])};
    float v[3] = {v0[0], v0[1], v0[2]}; // v_ at i, read by the caller
    const bool baoab = integrator == 0;
    if (DO_B && baoab) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            v[d] = __fmaf_rn(tc.hdt_m, f[d], v[d]);
    }
    if (DO_A) {
        float nz[3];
        normals3(seed, noise_idx, step, 0u, nz[0], nz[1], nz[2]);
        float xhi[3] = {xh.x, xh.y, xh.z}, xlo[3] = {lx, ly, lz};
        if (baoab) {
            // the two A half steps around the O step add dt/2 (v' + v'') to the
            // position (the O step does not depend on x): one compensated add
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = __fmaf_rn(tc.hdt_m, f[d], v[d]);               // B
                const float va = v[d];                                // A (first half)
                v[d] = __fmaf_rn(tc.c1f, v[d],
                                 __fmaf_rn(tc.c1lo, v[d], __fmul_rn(tc.sd_of, nz[d]))); // O
                df_add(xhi[d], xlo[d], __fmul_rn(hdt, __fadd_rn(va, v[d]))); // A + A
            }
        } else if (integrator == 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
                df_add(xhi[d], xlo[d], __fmaf_rn(f[d], tc.dt_mob, __fmul_rn(tc.sd_bdf, nz[d])));
        } else { // step (vi) as printed: drag and force, a kick of fixed size, drift
            const float nn = sqrtf(__fmaf_rn(nz[0], nz[0], __fmaf_rn(nz[1], nz[1],
                                                                     __fmul_rn(nz[2], nz[2]))));
            const float a = nn > 0.0f ? __fdiv_rn(tc.kick, nn) : 0.0f; // kick / |n|
            const float dt = 2.0f * hdt;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = __fmaf_rn(tc.dt_m, f[d], __fmaf_rn(-tc.gdt, v[d], v[d]));
                v[d] = __fmaf_rn(a, nz[d], v[d]);
                df_add(xhi[d], xlo[d], __fmul_rn(dt, v[d]));
            }
        }
        xq[i] = make_float4(xhi[0], xhi[1], xhi[2], xh.w);
        if (sxq) // the neighbour-list kernel's cell-ordered copy
            sxq[cell_pos[i]] = make_float4(xhi[0], xhi[1], xhi[2], __int_as_float(ti));
        x_lo[i] = xlo[0];
        x_lo[n + i] = xlo[1];
        x_lo[2 * n + i] = xlo[2];
        if (!(isfinite(xhi[0]) && isfinite(xhi[1]) && isfinite(xhi[2])))
            atomicOr(flags, FLAG_NONFINITE);
        if (x_ref) { // moved more than half the skin since the list was built: rebuild
            const float4 r = x_ref[i];
            const float ex = xhi[0] - r.x, ey = xhi[1] - r.y, ez = xhi[2] - r.z;
            if (!(fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= half_skin2))
                *nbr_gate = 1;
        }
    }
    v_[i] = v[0];
    v_[n + i] = v[1];
    v_[2 * n + i] = v[2];
}

cudaError_t launch_integrate(int mode, const IntArgs &a, const StepParams &p,
                             cudaStream_t st);
// The integrator's sum of the all-pairs partial slots alone, for positions
// 0 .. n_pos - 1 of the stream-K order, to out (6 n_pos floats: hi x, y, z,
// lo x, y, z planes).
cudaError_t launch_slot_sum(const float *slots, const StreamK &sk, int n_pos, float *out,
                            cudaStream_t st);

// Ensemble of droplets (ensemble.cu).  Each droplet's particles are listed in a
// type-grouped order (groups padded to 256 positions) at positions [gpos0,
// gpos0 + npad) of the ensemble's grouped order.  Geometry depends on the
// launch shape: n_it = ceil(npad / itile) row tiles, n_jt = npad / jtile
// j-tiles, each row tile cut into n_ch = ceil(n_jt / chunk) work items of at
// most `chunk` consecutive j-tiles; item0 is the prefix sum of n_it * n_ch
// over the droplets (item = item0 + row * n_ch + chunk index).
struct EnsDrop {
    int offset, n, n_it, n_jt, n_ch, rot_mode, wall, integrator;
    int gpos0, npad;
    float rc2_lim;  // LJ only between tiles within this squared distance (0: no LJ)
    int has_coul;   // 0: tiles out of LJ range add nothing
    long long item0;
    uint64_t seed;
    double dt, R0, k_evap, g, omega2;
    TypeCoef tc[NPSIM_MAX_TYPES];
};

struct EnsAllpairsArgs {
    const float4 *xq;
    const int *perm;        // grouped position -> particle (-1: padding)
    const int *tblk;        // type of each 256-position block
    const EnsDrop *drops;
    const long long *item0; // n_drops + 1 entries
    const PairTab *tabs;    // one table per droplet
    int n_drops;
    int chunk;              // j-tiles per work item
    long long n_items;
    unsigned *work;         // [0] next item, [1] CTAs done (both 0 between launches)
    float *slots;           // one [6][itile] slot per work item
};

struct EnsIntArgs {
    float *x_lo, *v, *F;     // layouts as in IntArgs, over the concatenation
    const int *typ;
    float4 *xq;
    const int *drop_of;
    const int *row_pos;      // grouped position of particle i
    const EnsDrop *drops;
    const float *slots;
    float4 *spring;          // [2][n_drops][NPSIM_MAX_TYPES], as in IntArgs
    int ext_on;
    int pad_;
    long long *step;
    int *flags;
    unsigned *done;
};

int ens_num_configs();
ApConfig ens_config(int idx);
int ens_occupancy(int idx);
cudaError_t launch_ens_allpairs(int idx, const StreamK &sk, const EnsAllpairsArgs &a,
                                cudaStream_t st);
cudaError_t launch_ens_integrate(int mode, const EnsIntArgs &a, int n_total, int n_drops,
                                 const StreamK &sk, cudaStream_t st);

// BF16 tensor-core MLP kernels (mlp.cu).
enum : int {
    GEMM_F32 = 0,  // C (FP32) = A B^T (+ bias)
    GEMM_ACT = 1,  // z = A B^T + bias -> Z (FP32, optional); C (BF16) = SiLU(z) or z
    GEMM_DACT = 2, // C (BF16, and FP32 if Cf) = (A B^T) * SiLU'(Z)
};

struct GemmArgs {
    const __nv_bfloat16 *A; // M x K, row-major, lda
    const __nv_bfloat16 *B; // N x K, row-major, ldb
    int M, N, K, lda, ldb, ldc;
    int n_tile;    // columns per CTA (multiple of 16, <= 256)
    int tmem_cols; // power of two >= max(32, n_tile)
    int mode, act;
    const float *bias;      // N or NULL
    float *Cf;              // FP32 output (M x N, ldc) or NULL
    __nv_bfloat16 *Cb;      // BF16 output or NULL
    float *Z;               // pre-activation (GEMM_ACT writes, GEMM_DACT reads), ldc
    int *flags;             // FLAG_TIMEOUT on a bounded wait that expired
    long long wait_cycles;  // bound of the main loop's waits in SM cycles (0: 2^32)
};

struct AdamArgs {
    float lr, b1, b2, eps, wd, bc1, bc2; // bc = 1 - beta^t
};

int gemm_smem_bytes(int n_tile);
cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t st);

// Fused inference of a whole MLP (mlp.cu): every layer of every network in one
// launch, activations kept in shared memory, one CTA per (128 rows, network).
// W[l] / b[l]: layer l's BF16 weights (N_l x K_l, K-major) and FP32 biases of
// all networks stacked (network k at rows k N_l); y: [n_nets][bp][out_p].
constexpr int kMaxMlpLayers = 6; // hidden layers the fused kernel takes
struct MlpInferArgs {
    const __nv_bfloat16 *X;                    // bp x in_p
    const __nv_bfloat16 *W[kMaxMlpLayers + 1]; // layer l: n_nets * N_l x K_l
    const float *b[kMaxMlpLayers + 1];         // layer l: n_nets * N_l
    int NL, in_p, H, out_p, bp, n_nets;
    float *y;
    int *flags;
};
bool mlp_infer_supported(int NL, int in_p, int H, int out_p);
cudaError_t launch_mlp_infer(const MlpInferArgs &a, cudaStream_t st);
cudaError_t launch_transpose_bf16(const void *in, int R, int C, int ldi, void *out, int ldo,
                                  cudaStream_t st);
cudaError_t launch_mse_grad(const float *y, const float *t, const float *w, int M, int m_valid,
                            int n_valid, int ldy, float *gf, void *gb, float *loss,
                            cudaStream_t st);
cudaError_t launch_colsum(const float *G, int M, int N, int ld, float *out, cudaStream_t st);
cudaError_t launch_adamw(float *w, const float *g, float *m, float *v, int rows, int cols,
                         const AdamArgs &a, void *wb, void *wt, const unsigned char *mask,
                         cudaStream_t st);
cudaError_t launch_f32_to_bf16(const float *x, int n, void *y, cudaStream_t st);
cudaError_t launch_weights_bf16(const float *w, int rows, int cols, void *wb, void *wt,
                                cudaStream_t st);

// Cell list (celllist.cu).  The sort key of NP i is its cell (tb == 1) or
// type * n_cells + cell (tb = the number of types): the cell order lists all NPs
// of type 0 cell by cell, then those of type 1, and so on.  count and start
// cover the tb * n_cells keys.
struct CellBufs {
    int *key, *rank, *count, *start, *arrived, *sorted, *tile_sum;
    int *pos;    // cell-ordered position of NP i (the inverse of sorted)
    float4 *sxq; // cell-ordered (x, y, z, type as int bits): the positions of the
                 // build, and with a neighbour list the current positions (the
                 // integrator writes each new position to its NP's slot);
                 // sxq[n] is a record far from every NP (type 0) that pads the
                 // neighbour lists
};
// Build the cell list of positions xq (gate: NULL = always, else only when *gate != 0).
cudaError_t launch_cell_build(const CellGrid &g, const float4 *xq, const int *typ, int n,
                              CellBufs &b, const int *gate, cudaStream_t st);
// Rewrite the cell-ordered records from positions xq in the order of the last build.
cudaError_t launch_cell_refresh(const CellBufs &b, const float4 *xq, const int *typ, int n,
                                cudaStream_t st);
// Verlet neighbour list over the cells (celllist.cu): entries are cell-order
// slots; entry k of the NP at cell-order slot p at nbr[nbr_index(k, p, n)]
// -- blocks of four entries, block j of all slots contiguous, so that a thread
// reads its next four entries with one 16-byte load and a warp reads 512
// contiguous bytes; cap (a multiple of 4) entries per slot; a list's last block
// is padded with entries n naming the far record sxq[n].  nnbr [n] the full
// counts by slot; x_ref [n] the positions of the last build by particle index.
__host__ __device__ __forceinline__ size_t nbr_index(int k, int p, int n)
{
    return ((size_t)(k >> 2) * (size_t)n + (size_t)p) * 4 + (size_t)(k & 3);
}
struct NbrList {
    unsigned *nbr; // partner slots
    int *nnbr;
    float4 *x_ref;
    unsigned long long *builds; // number of builds run (device counter)
    int cap;
};
// rcc2 (or NULL): squared cutoffs of the truncated Coulomb term per type pair
// (8 x 8); with it the lists cover both cutoffs and the list force kernel adds
// C q_a q_b r_ij / r^3 within the Coulomb cutoff to the LJ term.
cudaError_t launch_nbr_build(const CellGrid &g, const CellBufs &b, int n, const PairTab *tab,
                             const float *rcc2, float skin, const NbrList &l, int *flags,
                             const int *gate, cudaStream_t st);
cudaError_t launch_lj_nbr(const CellGrid &g, const CellBufs &b, const float4 *xq,
                          const int *typ, int n, const PairTab *tab, const float *rcc2,
                          const NbrList &l, float *F_lj, int *gate, cudaStream_t st);
int cell_build_launches();
int cell_scan_tiles(int n_cells);

// Stats (stats.cu)
cudaError_t launch_pair_hist(const double *x, int n, double r_max, int n_bins,
                             const CellGrid &g, const CellBufs &b,
                             unsigned long long *hist, cudaStream_t st);
cudaError_t launch_radial_hist(const double *x, int n, double r_max, int n_bins,
                               unsigned long long *hist, cudaStream_t st);
// mode 0: per-CTA sums of x; 1: sums of |x - c|^2; 2: componentwise minima;
// 3: componentwise maxima of |x_d|.  part holds 3 doubles per CTA of 256 threads.
// I(q) of Sec. 3.3 for a piecewise-constant g on [0, r_max), and its fractal form
// N_surf^2 (q R_g)^(-D_f) into out_frac (or NULL); device arrays.
cudaError_t launch_scattering(const double *g, int n_bins, double r_max, const double *q, int n_q,
                              double n_surf, double Rg, double Df, double *out,
                              double *out_frac, cudaStream_t st);
// Half diameter of every type (surface band of N_surf).
struct SurfHalf {
    double h[NPSIM_MAX_TYPES];
};
cudaError_t launch_surface_count(const double *x, const int *typ, int n, double R,
                                 const SurfHalf &hs, unsigned long long *count, cudaStream_t st);
cudaError_t launch_block_reduce(int mode, const double *x, int n, const double *c,
                                double *part, cudaStream_t st);
cudaError_t launch_boxcount(const double *x, int n, const double *origin, double eps,
                            unsigned long long *table, unsigned long long table_size,
                            int *count, int *flags, cudaStream_t st);
// Split float64 positions (SoA) into the integrator's hi (mirror) / lo words,
// and back (x = hi + lo in float64, for statistics).
cudaError_t launch_mirror(const double *x, const int *typ, const float *charge_by_type,
                          int n, float4 *xq, float *x_lo, cudaStream_t st);
cudaError_t launch_positions_f64(const float4 *xq, const float *x_lo, int n, double *x,
                                 cudaStream_t st);
// The same for n NPs whose lo words are rows of a [3][ld] array (one droplet of
// an ensemble); x is [3][n].
cudaError_t launch_positions_f64_ld(const float4 *xq, const float *x_lo, int n, int ld,
                                    double *x, cudaStream_t st);
// The state as host-facing AoS float64 (n x 3 each; NULL outputs are skipped):
// position hi + lo, velocity, force hi + lo (F: [6][n] hi/lo SoA).
cudaError_t launch_state_aos(const float4 *xq, const float *x_lo, const float *v, const float *F,
                             int n, double *xo, double *vo, double *Fo, cudaStream_t st);

// Test hooks (capi.cu)
cudaError_t launch_philox(uint64_t seed, const uint32_t ctr[4], long long n_blocks,
                          uint32_t *out, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, long long step, int n, double *out,
                           cudaStream_t st);

} // namespace npsim
