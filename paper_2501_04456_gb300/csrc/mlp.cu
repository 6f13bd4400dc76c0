// mlp.cu -- BF16 tensor-core kernels of the learned surrogate: a multilayer
// perceptron (SiLU hidden layers) trained with AdamW and evaluated in batches.
// The paper has no learned component; this is the surrogate that maps scenario
// parameters to the aggregate's fractal dimension and RDF.
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T, A and B row-major BF16 (both
// "K-major"), FP32 accumulation in tensor memory, on the 5th-generation
// tensor cores of sm_100+ (tcgen05):
//  * one CTA of 256 threads computes a 128 x n_tile block (n_tile <= 256,
//    multiple of 16); the FP32 accumulator lives in TMEM (allocated per CTA);
//  * operands arrive by TMA (cp.async.bulk.tensor, 2-D tensor maps, boxes of
//    8 K-columns x rows) into a ring of up to four stages of 64 K-columns each,
//    in the canonical no-swizzle K-major layout of the tcgen05 matrix
//    descriptors: 8-row x 16-byte core matrices, adjacent along M/N at 128 B
//    (stride-dimension byte offset) and along K at rows x 16 B (leading-
//    dimension byte offset).  Rows beyond M or N are zero-filled by the TMA;
//  * one thread issues the loads (mbarrier expect_tx per stage), one thread
//    issues tcgen05.mma (M = 128, N = n_tile, K = 16 per instruction) and
//    releases each stage with tcgen05.commit; every wait is bounded (clock64
//    budget) and reports FLAG_TIMEOUT instead of hanging;
//  * the epilogue (8 warps) reads the accumulator with tcgen05.ld (32 lanes x
//    32 bit, 16 columns per load; warps w and w + 4 share TMEM lanes
//    32(w mod 4) .. +31 and split the 16-column groups), stages the tile in
//    shared memory and writes it row by row (one warp per row, lanes along the
//    columns), applying bias, SiLU, the SiLU derivative for back-propagation,
//    or a plain FP32 store.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "npsim_internal.cuh"

namespace npsim {

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets, each encoded >> 4;
// bits 46-47 carry the descriptor version (1) required by tcgen05.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D = F32 (bits 4-5 = 1),
// A = B = BF16 (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Default bound of every mbarrier wait: 2^32 SM cycles, ~2 s at 2 GHz.
constexpr long long kWaitCycles = 1ll << 32;

// Bounded wait for the completion of the mbarrier phase with the given parity:
// false once `budget` SM cycles have passed without it.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  long long budget = kWaitCycles)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > budget)
            return false;
    }
    return true;
}

// SiLU and its derivative with the fast exponential and division intrinsics:
// their ~1e-6 relative error lies far below the BF16 rounding (2^-9) applied to
// every activation and gradient.  A huge exp(-z) gives a quotient of exactly 0.
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

__device__ __forceinline__ float dsilu(float z)
{
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

constexpr int kChunkK = 64;    // K columns per pipeline stage
constexpr int kTileM = 128;    // rows per CTA
constexpr int kMaxTileN = 256;
constexpr int kMaxStages = 4;
constexpr int kStageBudget = 200 * 1024; // shared memory for the operand ring

__host__ __device__ __forceinline__ int stage_bytes(int n_tile)
{
    return (kTileM + n_tile) * kChunkK * 2;
}

// Shared memory of one CTA: the operand ring, reused by the epilogue for the
// FP32 output tile (row pitch n_tile + 1 floats: conflict-free both ways).
__host__ __device__ __forceinline__ int dyn_smem_bytes(int n_tile, int stages)
{
    const int ring = stages * stage_bytes(n_tile);
    const int tile = kTileM * (n_tile + 1) * 4;
    return ring > tile ? ring : tile;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// 2-D TMA load of the box at (x = K column, y = row) into shared memory,
// completing `bytes` of the barrier's transaction count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

constexpr int kGemmThreads = 256;

__global__ void __launch_bounds__(kGemmThreads, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            GemmArgs g, int stages)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_issued;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int n0 = blockIdx.y * g.n_tile;
    const int nt = min(g.n_tile, g.N - n0); // multiple of 16 (N and n_tile are)
    const int nchunks = (g.K + kChunkK - 1) / kChunkK;
    const uint32_t base = smem_addr(smem);
    const uint32_t sbytes = (uint32_t)stage_bytes(g.n_tile);
    const uint32_t a_bytes = kTileM * kChunkK * 2;
    const uint32_t done_bar = smem_addr(&done);
    // bound of the main loop's waits (a test may shorten it); the drain after an
    // abort always waits with the default bound, so copies and MMAs in flight
    // land before the CTA frees its tensor memory and leaves
    const long long wb = g.wait_cycles > 0 ? g.wait_cycles : kWaitCycles;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&s_tmem)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), 1);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
        s_issued = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) { // TMA producer
            int c = 0;
            for (; c < nchunks; ++c) {
                const int s = c % stages, u = c / stages;
                if (u > 0 &&
                    !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)((u - 1) & 1), wb)) {
                    atomicExch(&s_abort, 1);
                    break;
                }
                const int k0 = c * kChunkK, kc = min(kChunkK, g.K - k0);
                const uint32_t sa = base + (uint32_t)s * sbytes, sb = sa + a_bytes;
                const uint32_t fb = smem_addr(&full[s]);
                mbar_expect_tx(fb, (uint32_t)((kTileM + g.n_tile) * kc * 2));
                for (int kg = 0; kg < kc / 8; ++kg) {
                    tma_load_2d(sa + (uint32_t)(kg * kTileM * 16), &tmA, k0 + kg * 8, m0, fb);
                    tma_load_2d(sb + (uint32_t)(kg * g.n_tile * 16), &tmB, k0 + kg * 8, n0, fb);
                }
            }
            s_issued = c;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) { // MMA issuer
            const uint32_t idesc = idesc_bf16(kTileM, nt);
            for (int c = 0; c < nchunks; ++c) {
                const int s = c % stages, u = c / stages;
                if (!mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)(u & 1), wb)) {
                    atomicExch(&s_abort, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int kc = min(kChunkK, g.K - c * kChunkK);
                const uint32_t sa = base + (uint32_t)s * sbytes, sb = sa + a_bytes;
                for (int ks = 0; ks < kc; ks += 16) {
                    const uint64_t ad = smem_desc(sa + (uint32_t)((ks / 8) * kTileM * 16),
                                                  kTileM * 16, 128);
                    const uint64_t bd = smem_desc(sb + (uint32_t)((ks / 8) * g.n_tile * 16),
                                                  (uint32_t)(g.n_tile * 16), 128);
                    const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                     tmem),
                                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
                mma_commit(smem_addr(&empty[s])); // stage s may be refilled
            }
            // fires once every MMA issued so far has completed (also after an abort)
            mma_commit(done_bar);
        }
        __syncwarp();
    }

    // wait for the accumulator (bounded), then the epilogue
    if (!mbar_wait_bounded(done_bar, 0, wb))
        atomicExch(&s_abort, 1);
    __syncthreads();
    const bool abort = s_abort != 0;
    if (abort) {
        if (tid == 0) {
            atomicOr(g.flags, FLAG_TIMEOUT);
            // let the copies still in flight land before the CTA leaves: at most
            // one outstanding load per stage (the last one issued)
            const int issued = s_issued;
            for (int s = 0; s < stages && s < issued; ++s) {
                const int u_last = (issued - 1 - s) / stages;
                mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)(u_last & 1));
            }
            mbar_wait_bounded(done_bar, 0);
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        float *S = reinterpret_cast<float *>(smem);
        const int pitch = g.n_tile + 1;
        const int quad = warp & 3, half = warp >> 2;
        const int rl = quad * 32 + lane;
        for (int j = half * 16; j < nt; j += 32) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)j;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                           "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),
                           "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q)
                S[rl * pitch + j + q] = __uint_as_float(r[q]);
        }
        __syncthreads();
        // one warp per output row, lanes along the columns (coalesced)
        const int rows = min(kTileM, g.M - m0);
        constexpr int kWarps = kGemmThreads / 32;
        for (int rr = warp; rr < rows; rr += kWarps) {
            const size_t ro = (size_t)(m0 + rr) * g.ldc + n0;
            const float *Sr = S + rr * pitch;
            for (int cc = lane; cc < nt; cc += 32) {
                const size_t o = ro + cc;
                float v = Sr[cc];
                if (g.mode == GEMM_F32) {
                    if (g.bias)
                        v += g.bias[n0 + cc];
                    g.Cf[o] = v;
                } else if (g.mode == GEMM_ACT) {
                    if (g.bias)
                        v += g.bias[n0 + cc];
                    if (g.Z)
                        g.Z[o] = v;
                    const float act = g.act ? silu(v) : v;
                    g.Cb[o] = __float2bfloat16_rn(act);
                    if (g.Cf)
                        g.Cf[o] = act;
                } else { // GEMM_DACT: gradient through the SiLU of the previous layer
                    const float d = v * dsilu(g.Z[o]);
                    g.Cb[o] = __float2bfloat16_rn(d);
                    if (g.Cf)
                        g.Cf[o] = d;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(g.tmem_cols));
}

// ---------------------------------------------------------------------------
// Fused inference of the whole network: one CTA runs every layer of one
// network on 128 rows of the batch, so activations never leave the SM.
//  * the A operand of every layer lives in shared memory (`abuf`, canonical
//    no-swizzle K-major layout): layer 0's input arrives by TMA, the epilogue
//    of layer l writes the BF16 activations of layer l + 1 into the same
//    buffer once layer l's MMAs have completed;
//  * weights stream by TMA through a ring of kInferStages stages of up to
//    N x 64 BF16 (one producer thread, running ahead across layers);
//  * one thread issues tcgen05.mma (M = 128, N = layer width, K = 16) into
//    one TMEM accumulator that every layer reuses;
//  * 8 epilogue warps read the accumulator (tcgen05.ld), add the bias, apply
//    SiLU and write BF16 activations (hidden layers) or FP32 outputs (last
//    layer, to the network's slice of y); they release the next layer with
//    an mbarrier after a proxy fence (generic writes -> tensor-core reads).
// The arithmetic is that of the layer-by-layer GEMM path (same MMA sequence,
// same epilogue operations), so both give the same bits.
constexpr int kInferThreads = 320; // warp 0 producer, warp 1 MMA, warps 2-9 epilogue
constexpr int kInferStages = 3;

// Tensor maps of the fused inference: the batch input (rows x in_p) and, per
// layer, the weights of every network stacked along the rows (n_nets * N x K).
struct MlpMaps {
    CUtensorMap x;
    CUtensorMap w[kMaxMlpLayers + 1];
};

struct MlpDev {
    int NL, in_p, H, out_p, bp, tmem_cols, abuf_bytes, stage_bytes;
    const float *bias[kMaxMlpLayers + 1]; // per layer, n_nets * N stacked
    float *y;                              // [n_nets][bp][out_p]
    int *flags;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ int infer_k(const MlpDev &d, int l) { return l == 0 ? d.in_p : d.H; }
__device__ __forceinline__ int infer_n(const MlpDev &d, int l) { return l == d.NL ? d.out_p : d.H; }

__global__ void __launch_bounds__(kInferThreads, 1)
k_mlp_infer(const __grid_constant__ MlpMaps maps, MlpDev d)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kInferStages], empty[kInferStages], x_full, acc_full,
        act_ready, drain, bias_ready;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_issued, s_x_issued;
    __shared__ float s_bias[2][256]; // the epilogue's bias, by layer parity

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int net = blockIdx.y;
    const int m0 = blockIdx.x * kTileM;
    const uint32_t abuf = smem_addr(smem);
    const uint32_t ring = abuf + (uint32_t)d.abuf_bytes;
    const uint32_t sbytes = (uint32_t)d.stage_bytes;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&s_tmem)),
                     "r"(d.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kInferStages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), 1);
        }
        mbar_init(smem_addr(&x_full), 1);
        mbar_init(smem_addr(&acc_full), 1);
        mbar_init(smem_addr(&act_ready), 8); // one arrival per epilogue warp
        mbar_init(smem_addr(&drain), 1);
        mbar_init(smem_addr(&bias_ready), kInferThreads - 64); // every epilogue thread
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
        s_issued = 0;
        s_x_issued = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) { // TMA producer: the input tile, then every layer's weights
            const uint32_t xb = smem_addr(&x_full);
            mbar_expect_tx(xb, (uint32_t)(kTileM * d.in_p * 2));
            for (int kg = 0; kg < d.in_p / 8; ++kg)
                tma_load_2d(abuf + (uint32_t)(kg * kTileM * 16), &maps.x, kg * 8, m0, xb);
            s_x_issued = 1;
            int c = 0;
            bool ok = true;
            for (int l = 0; l <= d.NL && ok; ++l) {
                const int K = infer_k(d, l), N = infer_n(d, l);
                const int row0 = net * N;
                for (int k0 = 0; k0 < K; k0 += kChunkK, ++c) {
                    const int s = c % kInferStages, u = c / kInferStages;
                    if (u > 0 && !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)((u - 1) & 1))) {
                        atomicExch(&s_abort, 1);
                        ok = false;
                        break;
                    }
                    const int kc = min(kChunkK, K - k0);
                    const uint32_t sb = ring + (uint32_t)s * sbytes, fb = smem_addr(&full[s]);
                    mbar_expect_tx(fb, (uint32_t)(N * kc * 2));
                    for (int kg = 0; kg < kc / 8; ++kg)
                        tma_load_2d(sb + (uint32_t)(kg * N * 16), &maps.w[l], k0 + kg * 8, row0, fb);
                }
            }
            s_issued = c;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) { // MMA issuer
            int c = 0;
            bool ok = true;
            for (int l = 0; l <= d.NL && ok; ++l) {
                const uint32_t gate = l == 0 ? smem_addr(&x_full) : smem_addr(&act_ready);
                const uint32_t par = l == 0 ? 0u : (uint32_t)((l - 1) & 1);
                if (!mbar_wait_bounded(gate, par)) {
                    atomicExch(&s_abort, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int K = infer_k(d, l), N = infer_n(d, l);
                const uint32_t idesc = idesc_bf16(kTileM, N);
                for (int k0 = 0; k0 < K; k0 += kChunkK, ++c) {
                    const int s = c % kInferStages, u = c / kInferStages;
                    if (!mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)(u & 1))) {
                        atomicExch(&s_abort, 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const int kc = min(kChunkK, K - k0);
                    const uint32_t sb = ring + (uint32_t)s * sbytes;
                    for (int ks = 0; ks < kc; ks += 16) {
                        const int k = k0 + ks;
                        const uint64_t ad = smem_desc(abuf + (uint32_t)((k / 8) * kTileM * 16),
                                                      kTileM * 16, 128);
                        const uint64_t bd = smem_desc(sb + (uint32_t)((ks / 8) * N * 16),
                                                      (uint32_t)(N * 16), 128);
                        const uint32_t acc = k > 0 ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                         tmem),
                                     "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                    mma_commit(smem_addr(&empty[s]));
                }
                mma_commit(smem_addr(&acc_full)); // this layer's accumulator is complete
            }
            mma_commit(smem_addr(&drain)); // every MMA issued has completed (also after an abort)
        }
        __syncwarp();
    } else { // epilogue warps 2..9: TMEM lanes 32 (warp mod 4) .. +31, alternate 16-column groups
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const int r = quad * 32 + lane; // row inside the tile
        for (int l = 0; l <= d.NL; ++l) {
            const int N = infer_n(d, l);
            // this layer's bias into shared memory while its MMAs run.  Every
            // epilogue thread arrives after its store and waits for all 256
            // (bounded): the completed phase also shows that every thread has
            // left the previous layer, so the other parity's buffer is free
            float *bias = s_bias[l & 1];
            if (tid - 64 < N)
                bias[tid - 64] = d.bias[l][(size_t)net * N + (tid - 64)];
            mbar_arrive(smem_addr(&bias_ready));
            if (!mbar_wait_bounded(smem_addr(&bias_ready), (uint32_t)(l & 1)) ||
                !mbar_wait_bounded(smem_addr(&acc_full), (uint32_t)(l & 1))) {
                atomicExch(&s_abort, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const bool last = l == d.NL;
            float *yrow = last ? d.y + ((size_t)net * d.bp + m0 + r) * d.out_p : nullptr;
            for (int j = half * 16; j < N; j += 32) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)j;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
                               "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]),
                               "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                               "=r"(v[15])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (last) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(yrow + j + q) = make_float4(
                            __uint_as_float(v[q]) + bias[j + q],
                            __uint_as_float(v[q + 1]) + bias[j + q + 1],
                            __uint_as_float(v[q + 2]) + bias[j + q + 2],
                            __uint_as_float(v[q + 3]) + bias[j + q + 3]);
                } else {
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) { // two 8-column core-matrix rows
                        uint32_t p[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int q = h8 * 8 + 2 * e;
                            const float a0 = silu(__uint_as_float(v[q]) + bias[j + q]);
                            const float a1 = silu(__uint_as_float(v[q + 1]) + bias[j + q + 1]);
                            const __nv_bfloat162 b2 = __floats2bfloat162_rn(a0, a1);
                            p[e] = *reinterpret_cast<const uint32_t *>(&b2);
                        }
                        const int col = j + h8 * 8;
                        uint8_t *dst = smem + (size_t)(col / 8) * kTileM * 16 + (size_t)r * 16;
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(p[0], p[1], p[2], p[3]);
                    }
                }
            }
            if (!last) { // the activations are the next layer's A operand
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(smem_addr(&act_ready));
            }
        }
    }

    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            atomicOr(d.flags, FLAG_TIMEOUT);
            // copies still in flight land before the CTA leaves (at most the
            // last one issued per stage, and the input tile)
            const int issued = s_issued;
            for (int s = 0; s < kInferStages && s < issued; ++s) {
                const int u_last = (issued - 1 - s) / kInferStages;
                mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)(u_last & 1));
            }
            if (s_x_issued)
                mbar_wait_bounded(smem_addr(&x_full), 0);
            mbar_wait_bounded(smem_addr(&drain), 0);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(d.tmem_cols));
}

// out[c][r] = in[r][c] for an R x C BF16 matrix (32 x 32 tiles in shared memory).
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, int R, int C, int ldi,
                                 __nv_bfloat16 *__restrict__ out, int ldo)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * ldi + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < C && r < R)
            out[(size_t)c * ldo + r] = t[threadIdx.x][k];
    }
}

// Mean-squared error over rows < m_valid and the first n_valid columns of a
// padded M x ldy output: dL/dy = 2 w_c (y - t) / (m_valid * n_valid) (FP32 and
// BF16); loss accumulated (sum of w_c (y - t)^2 / (m_valid n_valid)).
__global__ void k_mse_grad(const float *__restrict__ y, const float *__restrict__ t,
                           const float *__restrict__ w, int M, int m_valid, int n_valid,
                           int ldy, float *__restrict__ gf, __nv_bfloat16 *__restrict__ gb,
                           float *__restrict__ loss)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = idx / ldy, c = idx - r * ldy;
    float g = 0.f, l = 0.f;
    if (r < M) {
        if (r < m_valid && c < n_valid) {
            const float e = y[idx] - t[(size_t)r * ldy + c];
            const float wc = w ? w[c] : 1.f;
            const float s = 1.0f / ((float)m_valid * (float)n_valid);
            g = 2.f * wc * e * s;
            l = wc * e * e * s;
        }
        gf[idx] = g;
        gb[idx] = __float2bfloat16_rn(g);
    }
    // warp reduction of the loss, one atomic per warp
    for (int o = 16; o > 0; o >>= 1)
        l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f)
        atomicAdd(loss, l);
}

// Column sums of an M x N FP32 matrix (bias gradients), one thread per column,
// rows in fixed order (deterministic).
__global__ void k_colsum(const float *__restrict__ G, int M, int N, int ld, float *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N)
        return;
    float s = 0.f;
    for (int r = 0; r < M; ++r)
        s += G[(size_t)r * ld + c];
    out[c] = s;
}

// AdamW (I. Loshchilov, F. Hutter, "Decoupled weight decay regularization"):
// m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; w -= lr (m_hat / (sqrt(v_hat) + eps) + wd w),
// with m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t).  Writes the BF16 copy of w,
// and (if wt) its transpose for back-propagation.  mask (optional) keeps padded
// entries at zero.
__global__ void k_adamw(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, int rows, int cols, AdamArgs a,
                        __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ wt,
                        const unsigned char *__restrict__ mask)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols)
        return;
    float wi = w[idx];
    if (!mask || mask[idx]) {
        const float gi = g[idx];
        const float mi = a.b1 * m[idx] + (1.f - a.b1) * gi;
        const float vi = a.b2 * v[idx] + (1.f - a.b2) * gi * gi;
        m[idx] = mi;
        v[idx] = vi;
        const float mh = mi / a.bc1, vh = vi / a.bc2;
        wi -= a.lr * (mh / (sqrtf(vh) + a.eps) + a.wd * wi);
        w[idx] = wi;
    }
    if (wb) {
        const __nv_bfloat16 b = __float2bfloat16_rn(wi);
        wb[idx] = b;
        if (wt) {
            const int r = idx / cols, c = idx - r * cols;
            wt[(size_t)c * rows + r] = b;
        }
    }
}

// BF16 copy of an FP32 weight matrix (rows x cols) and its transpose.
__global__ void k_weights_bf16(const float *__restrict__ w, int rows, int cols,
                               __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ wt)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols)
        return;
    const __nv_bfloat16 b = __float2bfloat16_rn(w[idx]);
    wb[idx] = b;
    const int r = idx / cols, c = idx - r * cols;
    wt[(size_t)c * rows + r] = b;
}

__global__ void k_f32_to_bf16(const float *__restrict__ x, int n, __nv_bfloat16 *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        y[i] = __float2bfloat16_rn(x[i]);
}

} // namespace

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of a row-major BF16 matrix (rows x K, leading dimension ld
// elements) read in boxes of 8 K-columns x box_rows rows; out-of-range rows
// read as zero.
bool encode_operand(CUtensorMap *m, const __nv_bfloat16 *ptr, int rows, int K, int ld,
                    int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

} // namespace

int gemm_smem_bytes(int n_tile) { return dyn_smem_bytes(n_tile, kMaxStages); }

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || (g.N % 16) || (g.K % 16) || (g.n_tile % 16) ||
        g.n_tile < 16 || g.n_tile > kMaxTileN || (g.lda % 8) || (g.ldb % 8) || g.lda < g.K ||
        g.ldb < g.K || ((uintptr_t)g.A % 16) || ((uintptr_t)g.B % 16))
        return cudaErrorInvalidValue;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dyn_smem_bytes(kMaxTileN, kMaxStages));
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    CUtensorMap ta, tb;
    if (!encode_operand(&ta, g.A, g.M, g.K, g.lda, kTileM) ||
        !encode_operand(&tb, g.B, g.N, g.K, g.ldb, g.n_tile))
        return cudaErrorInvalidValue;
    const int nchunks = (g.K + kChunkK - 1) / kChunkK;
    int stages = kStageBudget / stage_bytes(g.n_tile);
    stages = stages < kMaxStages ? stages : kMaxStages;
    stages = stages < nchunks ? stages : nchunks;
    dim3 grid((g.M + kTileM - 1) / kTileM, (g.N + g.n_tile - 1) / g.n_tile);
    k_gemm_bf16<<<grid, kGemmThreads, dyn_smem_bytes(g.n_tile, stages), st>>>(ta, tb, g, stages);
    return cudaGetLastError();
}

bool mlp_infer_supported(int NL, int in_p, int H, int out_p)
{
    return NL >= 1 && NL <= kMaxMlpLayers && H >= 16 && H <= 256 && H % 16 == 0 &&
           out_p >= 16 && out_p <= 256 && out_p % 16 == 0 && in_p >= 16 && in_p <= 256 &&
           in_p % 16 == 0;
}

cudaError_t launch_mlp_infer(const MlpInferArgs &a, cudaStream_t st)
{
    if (!mlp_infer_supported(a.NL, a.in_p, a.H, a.out_p) || a.bp < kTileM || a.bp % kTileM ||
        a.n_nets < 1 || !a.X || !a.y)
        return cudaErrorInvalidValue;
    const int kmax = a.in_p > a.H ? a.in_p : a.H;
    const int nmax = a.H > a.out_p ? a.H : a.out_p;
    MlpDev d{};
    d.NL = a.NL;
    d.in_p = a.in_p;
    d.H = a.H;
    d.out_p = a.out_p;
    d.bp = a.bp;
    d.tmem_cols = 32;
    while (d.tmem_cols < nmax) // TMEM columns: a power of two >= 32
        d.tmem_cols *= 2;
    d.abuf_bytes = (kTileM * kmax * 2 + 1023) / 1024 * 1024;
    d.stage_bytes = nmax * kChunkK * 2;
    d.y = a.y;
    d.flags = a.flags;
    MlpMaps maps{};
    if (!encode_operand(&maps.x, a.X, a.bp, a.in_p, a.in_p, kTileM))
        return cudaErrorInvalidValue;
    for (int l = 0; l <= a.NL; ++l) {
        const int K = l == 0 ? a.in_p : a.H, N = l == a.NL ? a.out_p : a.H;
        if (!a.W[l] || !a.b[l] || ((uintptr_t)a.W[l] % 16) ||
            !encode_operand(&maps.w[l], a.W[l], a.n_nets * N, K, K, N))
            return cudaErrorInvalidValue;
        d.bias[l] = a.b[l];
    }
    const int smem = d.abuf_bytes + kInferStages * d.stage_bytes;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kTileM * 256 * 2 + kInferStages * 256 * kChunkK * 2);
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    dim3 grid(a.bp / kTileM, a.n_nets);
    k_mlp_infer<<<grid, kInferThreads, smem, st>>>(maps, d);
    return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const void *in, int R, int C, int ldi, void *out, int ldo,
                                  cudaStream_t st)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>((const __nv_bfloat16 *)in, R, C, ldi,
                                                   (__nv_bfloat16 *)out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_mse_grad(const float *y, const float *t, const float *w, int M, int m_valid,
                            int n_valid, int ldy, float *gf, void *gb, float *loss,
                            cudaStream_t st)
{
    const int n = M * ldy;
    k_mse_grad<<<(n + 255) / 256, 256, 0, st>>>(y, t, w, M, m_valid, n_valid, ldy, gf,
                                                (__nv_bfloat16 *)gb, loss);
    return cudaGetLastError();
}

cudaError_t launch_colsum(const float *G, int M, int N, int ld, float *out, cudaStream_t st)
{
    k_colsum<<<(N + 127) / 128, 128, 0, st>>>(G, M, N, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_adamw(float *w, const float *g, float *m, float *v, int rows, int cols,
                         const AdamArgs &a, void *wb, void *wt, const unsigned char *mask,
                         cudaStream_t st)
{
    const int n = rows * cols;
    k_adamw<<<(n + 255) / 256, 256, 0, st>>>(w, g, m, v, rows, cols, a, (__nv_bfloat16 *)wb,
                                             (__nv_bfloat16 *)wt, mask);
    return cudaGetLastError();
}

cudaError_t launch_weights_bf16(const float *w, int rows, int cols, void *wb, void *wt,
                                cudaStream_t st)
{
    const int n = rows * cols;
    k_weights_bf16<<<(n + 255) / 256, 256, 0, st>>>(w, rows, cols, (__nv_bfloat16 *)wb,
                                                    (__nv_bfloat16 *)wt);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float *x, int n, void *y, cudaStream_t st)
{
    k_f32_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(x, n, (__nv_bfloat16 *)y);
    return cudaGetLastError();
}

} // namespace npsim
