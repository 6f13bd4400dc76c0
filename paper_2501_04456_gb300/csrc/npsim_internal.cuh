// npsim_internal.cuh -- device-side types and helpers shared by the library's
// CUDA translation units (never by the CPU oracle).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/npsim.h"

namespace npsim {

// ---------------------------------------------------------------------------
// Error word bits (device int, read once per npsim_step).
enum : int {
    FLAG_NONFINITE = 1,
    FLAG_TIMEOUT = 2,
    FLAG_BAD_CELL = 4,
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
// float; Box-Muller in float32 with the accurate logf / sincospif.
__device__ __forceinline__ void normals3(uint64_t seed, uint32_t i, int64_t step,
                                         uint32_t purpose, double &n0, double &n1,
                                         double &n2)
{
    const uint64_t s = (uint64_t)step;
    U4 r = philox10(U4{i, (uint32_t)s, (uint32_t)(s >> 32), purpose}, (uint32_t)seed,
                    (uint32_t)(seed >> 32));
    const float sc = 2.3283064365386963e-10f; // 2^-32
    float u0 = fmaf(__uint2float_rn(r.x), sc, 0.5f * sc);
    float u1 = fmaf(__uint2float_rn(r.y), sc, 0.5f * sc);
    float u2 = fmaf(__uint2float_rn(r.z), sc, 0.5f * sc);
    float u3 = fmaf(__uint2float_rn(r.w), sc, 0.5f * sc);
    float rho1 = sqrtf(-2.0f * logf(u0));
    float rho2 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    n0 = (double)(rho1 * c1);
    n1 = (double)(rho1 * s1);
    n2 = (double)(rho2 * c3);
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
// Per-type coefficients used by the integrator (computed on the host in
// float64 from npsim_type_t and the scenario).
struct TypeCoef {
    double mass, inv_mass, half_sigma, k_wall;
    double c1, sd_o;    // BAOAB O step: v <- c1 v + sd_o xi
    double mob, sd_bd;  // overdamped: x += F dt mob + sd_bd xi
    double charge_c;    // C * q (Coulomb-only all-pairs kernel returns the field)
};

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
// (i-tile x j-tile) split evenly over `grid` CTAs; CTA c covers units
// [W c / grid, W (c+1) / grid).  The part of i-tile row r computed by CTA c is
// written to partial slot r + c (unique: rows and CTAs both advance along
// the unit order).
struct StreamK {
    int itile;   // i per CTA tile = block * ki
    int jtile;   // j per shared-memory tile
    int n_it;    // number of i tiles
    int n_jt;    // number of j tiles
    int grid;    // CTAs
    int pad_;
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
};

// Record a message for npsim_last_error() on this thread and return `code`
// (defined in capi.cu).
int report_error(int code, const char *fmt, ...);

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
cudaError_t launch_allpairs_grouped(int idx, const StreamK &sk, const float4 *xq,
                                    const int *perm, int n_perm, const float *qblk,
                                    double *slots, cudaStream_t st);
cudaError_t launch_allpairs(int cfg_idx, bool lj, const StreamK &sk, const float4 *xq,
                            const int *typ, int n, const PairTab *tab, double *slots,
                            cudaStream_t st);

// Integrator (integrate.cu)
enum IntMode : int {
    MODE_FORCES = 0, // assemble F from partials + external, write F
    MODE_A = 1,      // BAOA (or overdamped update) from the stored F; step += 1
    MODE_BA = 2,     // assemble F, finish the step (B), then BAOA of the next; step += 1
    MODE_B = 3,      // assemble F, finish the step (B), write F and v
};

struct IntArgs {
    double *x, *v, *F;       // SoA [3][n]
    const int *typ;
    float4 *xq;              // float32 mirror (x, y, z, q), written when positions move
    const double *slots;     // stream-K partials (or NULL)
    StreamK sk;
    const double *F_lj;      // cell-list LJ forces SoA [3][n] (or NULL)
    const int *row_pos;      // grouped layout: position of particle i in the rows (-1:
                             // no Coulomb partial); NULL: row position = i
    int ext_on;              // add external forces
    int field_slots;         // slots hold sum_j q_j r_ij/r^3 (Coulomb-only kernel): scale by C q_i
    long long *step;         // device step counter
    int *flags;
    unsigned *done;          // last-block counter
};

cudaError_t launch_integrate(int mode, const IntArgs &a, const StepParams &p,
                             cudaStream_t st);

// Ensemble of droplets (ensemble.cu).  Geometry depends on the launch shape:
// n_it = ceil(n / itile), n_jt = ceil(n / jtile); row0 and unit0 are prefix sums
// of n_it and n_it * n_jt over the droplets.
struct EnsDrop {
    int offset, n, n_it, n_jt, row0, rot_mode, wall, integrator;
    long long unit0;
    uint64_t seed;
    double dt, R0, k_evap, g, omega2;
    TypeCoef tc[NPSIM_MAX_TYPES];
};

struct EnsAllpairsArgs {
    const float4 *xq;
    const int *typ;
    const EnsDrop *drops;
    const long long *unit0; // n_drops + 1 entries
    const PairTab *tabs;    // one table per droplet
    int n_drops;
    int pad_;
    double *slots;
};

struct EnsIntArgs {
    double *x, *v, *F;
    const int *typ;
    float4 *xq;
    const int *drop_of;
    const EnsDrop *drops;
    const double *slots;
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
};

struct AdamArgs {
    float lr, b1, b2, eps, wd, bc1, bc2; // bc = 1 - beta^t
};

int gemm_smem_bytes(int n_tile);
cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t st);
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

// Cell list (celllist.cu)
struct CellBufs {
    int *key, *rank, *count, *start, *sorted, *tile_sum;
    float4 *sxq;
    int *styp;
};
cudaError_t launch_cell_build(const CellGrid &g, const float4 *xq, const int *typ, int n,
                              CellBufs &b, int *flags, cudaStream_t st);
cudaError_t launch_cell_lj(const CellGrid &g, const CellBufs &b, int n, const PairTab *tab,
                           double *F_lj, cudaStream_t st);
int cell_build_launches();
int cell_scan_tiles(int n_cells);

// Stats (stats.cu)
cudaError_t launch_pair_hist(const double *x, int n, double r_max, int n_bins,
                             const CellGrid &g, const CellBufs &b,
                             unsigned long long *hist, cudaStream_t st);
cudaError_t launch_radial_hist(const double *x, int n, double r_max, int n_bins,
                               unsigned long long *hist, cudaStream_t st);
// mode 0: per-CTA sums of x; 1: sums of |x - c|^2; 2: componentwise minima.
// part holds 3 doubles per CTA of 256 threads.
cudaError_t launch_block_reduce(int mode, const double *x, int n, const double *c,
                                double *part, cudaStream_t st);
cudaError_t launch_boxcount(const double *x, int n, const double *origin, double eps,
                            unsigned long long *table, unsigned long long table_size,
                            int *count, int *flags, cudaStream_t st);
cudaError_t launch_mirror(const double *x, const int *typ, const float *charge_by_type,
                          int n, float4 *xq, cudaStream_t st);

// Test hooks (capi.cu)
cudaError_t launch_philox(uint64_t seed, const uint32_t ctr[4], long long n_blocks,
                          uint32_t *out, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, long long step, int n, double *out,
                           cudaStream_t st);

} // namespace npsim
