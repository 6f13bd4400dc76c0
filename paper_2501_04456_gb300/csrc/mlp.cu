// mlp.cu -- BF16 tensor-core kernels of the learned surrogate: a multilayer
// perceptron (SiLU hidden layers) trained with AdamW and evaluated in batches.
// The paper has no learned component; this is the surrogate that maps scenario
// parameters to the aggregate's fractal dimension and RDF.
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T, A and B row-major BF16 (both
// "K-major"), FP32 accumulation in tensor memory, on the 5th-generation
// tensor cores of sm_100+ (tcgen05):
//  * one CTA of 128 threads computes a 128 x n_tile block (n_tile <= 256,
//    multiple of 16); the FP32 accumulator lives in TMEM (allocated per CTA);
//  * operands are staged in shared memory in the canonical no-swizzle K-major
//    layout of the tcgen05 matrix descriptors: 8-row x 16-byte core matrices,
//    adjacent along K at 128 B (leading-dimension byte offset) and along M/N at
//    1024 B (stride-dimension byte offset) for 64-column chunks;
//  * one elected thread issues tcgen05.mma (M = 128, N = n_tile, K = 16 per
//    instruction) and commits to an mbarrier; every wait on it is bounded
//    (clock64 budget) and reports FLAG_TIMEOUT instead of hanging;
//  * the epilogue reads the accumulator with tcgen05.ld (32 lanes x 32 bit,
//    16 columns per load; warp w owns rows 32w..32w+31) and applies bias,
//    SiLU, the SiLU derivative for back-propagation, or a plain FP32 store.
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

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

constexpr int kChunkK = 64;   // K columns staged per round
constexpr int kTileM = 128;   // rows per CTA
constexpr int kMaxTileN = 256;

__global__ void __launch_bounds__(128, 1)
k_gemm_bf16(GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;                          // 128 x 64 bf16 = 16 KB
    uint8_t *sB = smem + kTileM * kChunkK * 2;   // n_tile x 64 bf16 <= 32 KB
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int n0 = blockIdx.y * g.n_tile;
    const int nt = min(g.n_tile, g.N - n0); // multiple of 16 (N and n_tile are)
    const uint32_t bar_a = smem_addr(&bar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&s_tmem)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    const int nchunks = (g.K + kChunkK - 1) / kChunkK;
    const uint32_t idesc = idesc_bf16(kTileM, nt);
    const uint32_t a_base = smem_addr(sA), b_base = smem_addr(sB);
    for (int c = 0; c < nchunks; ++c) {
        const int k0 = c * kChunkK;
        const int kc = min(kChunkK, g.K - k0); // multiple of 16
        if (c > 0) {
            // the MMAs of the previous round must be done reading shared memory
            if (tid == 0 && !mbar_wait_bounded(bar_a, (uint32_t)((c - 1) & 1)))
                s_abort = 1;
            __syncthreads();
            if (s_abort)
                break;
        }
        // stage A (128 x kc) and B (nt x kc): 16-byte pieces = core-matrix rows
        const int kg_n = kc / 8;
        for (int p = tid; p < kTileM * kg_n; p += 128) {
            const int r = p / kg_n, kg = p - r * kg_n;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (m0 + r < g.M)
                v = *reinterpret_cast<const uint4 *>(g.A + (size_t)(m0 + r) * g.lda + k0 + kg * 8);
            *reinterpret_cast<uint4 *>(sA + ((r >> 3) * 8 + kg) * 128 + (r & 7) * 16) = v;
        }
        for (int p = tid; p < nt * kg_n; p += 128) {
            const int r = p / kg_n, kg = p - r * kg_n;
            const uint4 v =
                *reinterpret_cast<const uint4 *>(g.B + (size_t)(n0 + r) * g.ldb + k0 + kg * 8);
            *reinterpret_cast<uint4 *>(sB + ((r >> 3) * 8 + kg) * 128 + (r & 7) * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int ks = 0; ks < kc; ks += 16) {
                const uint64_t ad = smem_desc(a_base + (ks / 8) * 128, 128, 1024);
                const uint64_t bd = smem_desc(b_base + (ks / 8) * 128, 128, 1024);
                const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar_a));
        }
    }
    if (!s_abort) {
        if (tid == 0 && !mbar_wait_bounded(bar_a, (uint32_t)((nchunks - 1) & 1)))
            s_abort = 1;
        __syncthreads();
    }
    if (s_abort) {
        if (tid == 0)
            atomicOr(g.flags, FLAG_TIMEOUT);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int row = m0 + warp * 32 + lane;
        for (int j = 0; j < nt; j += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                           "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),
                           "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.M) {
                for (int q = 0; q < 16; ++q) {
                    const int col = n0 + j + q;
                    float v = __uint_as_float(r[q]);
                    if (g.mode == GEMM_F32) {
                        if (g.bias)
                            v += g.bias[col];
                        g.Cf[(size_t)row * g.ldc + col] = v;
                    } else if (g.mode == GEMM_ACT) {
                        if (g.bias)
                            v += g.bias[col];
                        if (g.Z)
                            g.Z[(size_t)row * g.ldc + col] = v;
                        const float a = g.act ? silu(v) : v;
                        g.Cb[(size_t)row * g.ldc + col] = __float2bfloat16_rn(a);
                        if (g.Cf)
                            g.Cf[(size_t)row * g.ldc + col] = a;
                    } else { // GEMM_DACT: gradient through the SiLU of the previous layer
                        const float d = v * dsilu(g.Z[(size_t)row * g.ldc + col]);
                        g.Cb[(size_t)row * g.ldc + col] = __float2bfloat16_rn(d);
                        if (g.Cf)
                            g.Cf[(size_t)row * g.ldc + col] = d;
                    }
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

int gemm_smem_bytes(int n_tile) { return (kTileM + n_tile) * kChunkK * 2; }

cudaError_t launch_gemm(const GemmArgs &g, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || (g.N % 16) || (g.K % 16) || (g.n_tile % 16) ||
        g.n_tile > kMaxTileN || (g.lda % 8) || (g.ldb % 8))
        return cudaErrorInvalidValue;
    const int smem = gemm_smem_bytes(g.n_tile);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             gemm_smem_bytes(kMaxTileN));
        if (e != cudaSuccess)
            return e;
        attr_done = true;
    }
    dim3 grid((g.M + kTileM - 1) / kTileM, (g.N + g.n_tile - 1) / g.n_tile);
    k_gemm_bf16<<<grid, 128, smem, st>>>(g);
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
