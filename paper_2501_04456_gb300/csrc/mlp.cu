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

// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > (1ll << 32)) // ~2 s at 2 GHz
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
                if (u > 0 && !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)((u - 1) & 1))) {
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
                if (!mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)(u & 1))) {
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
    if (!mbar_wait_bounded(done_bar, 0))
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
