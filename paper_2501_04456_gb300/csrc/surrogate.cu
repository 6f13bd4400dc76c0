// surrogate.cu -- deep ensemble of multilayer perceptrons that map scenario
// parameters to the statistics of the final aggregate (fractal dimension and
// RDF), trained and evaluated on the GPU by the BF16 tcgen05 kernels of
// mlp.cu.  The paper has no learned component; the plain simulation is the
// surrogate's fallback and the measure of its error.
//
// Network: n_in inputs (padded to 16) -> n_layers hidden layers of width H
// with SiLU -> n_out outputs (padded to a multiple of 16).  Weights and
// activations are BF16, accumulation and the pre-activations FP32, master
// weights and the AdamW moments FP32.  Padded weight rows and columns are
// masked and stay zero.  Inputs and targets are standardised with the
// (mean, std) vectors set by npsim_surr_set_norm.
//
// Parameter layout of one network (npsim_surr_get_params): for each layer l
// in order, W_l (out_pad x in_pad, row-major) then b_l (out_pad).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "npsim_internal.cuh"

using namespace npsim;

namespace {

int round16(int x) { return (x + 15) / 16 * 16; }

int pow2_at_least(int x)
{
    int p = 32;
    while (p < x)
        p <<= 1;
    return p;
}

struct Layer {
    int out = 0, in = 0, out_p = 0, in_p = 0;
    float *W = nullptr, *b = nullptr;          // FP32 master weights
    __nv_bfloat16 *Wb = nullptr, *Wt = nullptr; // BF16 copy and its transpose
    float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    float *gW = nullptr, *gb = nullptr;
    unsigned char *mask = nullptr, *bmask = nullptr;
};

template <class T> cudaError_t dmalloc(T **p, size_t n)
{
    *p = nullptr;
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

template <class T> void dfree2(T *&p)
{
    if (p)
        cudaFree((void *)p);
    p = nullptr;
}

} // namespace

struct npsim_surr {
    int n_in = 0, n_in_p = 0, H = 0, NL = 0, n_out = 0, n_out_p = 0, n_nets = 0;
    int bcap = 0; // batch capacity (multiple of 128)
    std::vector<std::vector<Layer>> nets;
    // per layer, the BF16 weights and FP32 biases of all networks in one block
    // (network k at rows k out_p): Layer::Wb and Layer::b point into these
    std::vector<__nv_bfloat16 *> Wb_stack;
    std::vector<float *> b_stack;
    std::vector<float> xm, xs, ym, ys; // normalisation
    cudaStream_t st = nullptr;
    // activations and gradients for one batch
    std::vector<__nv_bfloat16 *> a; // NL + 1 (a[0] = input)
    std::vector<float *> z;         // NL pre-activations
    float *y = nullptr, *yt = nullptr, *dyf = nullptr;
    __nv_bfloat16 *dyb = nullptr;
    __nv_bfloat16 *dz[2] = {nullptr, nullptr};
    float *dzf[2] = {nullptr, nullptr};
    __nv_bfloat16 *tA = nullptr, *tB = nullptr; // transposes
    float *loss = nullptr, *outw = nullptr;
    float *xin = nullptr;          // normalised FP32 inputs of a batch (staging)
    float *y_all = nullptr;        // outputs of every network [n_nets][bcap][n_out_p]
    float *ystat = nullptr;        // ensemble mean and spread [2][bcap][n_out]
    float *d_ym = nullptr, *d_ys = nullptr; // output de-normalisation (n_out)
    int *flags = nullptr;
    long long adam_t = 0;
    // dataset on the device
    __nv_bfloat16 *dsx = nullptr;
    float *dsy = nullptr;
    int ds_n = 0;

    ~npsim_surr()
    {
        for (auto &net : nets)
            for (auto &L : net) {
                L.b = nullptr; // inside b_stack / Wb_stack
                L.Wb = nullptr;
                dfree2(L.W);
                dfree2(L.Wt);
                dfree2(L.mW);
                dfree2(L.vW);
                dfree2(L.mb);
                dfree2(L.vb);
                dfree2(L.gW);
                dfree2(L.gb);
                dfree2(L.mask);
                dfree2(L.bmask);
            }
        for (auto *p : a)
            dfree2(p);
        for (auto *p : z)
            dfree2(p);
        dfree2(y);
        dfree2(yt);
        dfree2(dyf);
        dfree2(dyb);
        for (int k = 0; k < 2; ++k) {
            dfree2(dz[k]);
            dfree2(dzf[k]);
        }
        dfree2(tA);
        dfree2(tB);
        dfree2(loss);
        dfree2(outw);
        dfree2(xin);
        dfree2(y_all);
        dfree2(ystat);
        dfree2(d_ym);
        dfree2(d_ys);
        dfree2(flags);
        dfree2(dsx);
        dfree2(dsy);
        for (auto *p : Wb_stack)
            dfree2(p);
        for (auto *p : b_stack)
            dfree2(p);
        if (st)
            cudaStreamDestroy(st);
    }
};

namespace {

#define SR_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return report_error(e_ == cudaErrorMemoryAllocation ? NPSIM_ERR_OOM         \
                                                                 : NPSIM_ERR_CUDA,      \
                                "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                __FILE__, __LINE__);                                    \
    } while (0)

int n_tile_for(int N) { return (N % 64 == 0) ? 64 : N; }

// Bound of the GEMM kernel's main-loop waits set by npsim_test_wait_cycles
// (0: the kernel's default).
std::atomic<long long> g_wait_cycles{0};

cudaError_t gemm(npsim_surr *s, int mode, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
                 int ldb, int M, int N, int K, const float *bias, float *Cf, __nv_bfloat16 *Cb,
                 int ldc, float *Z, int act)
{
    GemmArgs g{};
    g.A = A;
    g.B = B;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.n_tile = n_tile_for(N);
    g.tmem_cols = pow2_at_least(g.n_tile);
    g.mode = mode;
    g.act = act;
    g.bias = bias;
    g.Cf = Cf;
    g.Cb = Cb;
    g.Z = Z;
    g.flags = s->flags;
    g.wait_cycles = g_wait_cycles.load();
    return launch_gemm(g, s->st);
}

int alloc_batch(npsim_surr *s, int bcap)
{
    if (bcap <= s->bcap)
        return NPSIM_OK;
    for (auto *&p : s->a)
        dfree2(p);
    for (auto *&p : s->z)
        dfree2(p);
    dfree2(s->y);
    dfree2(s->yt);
    dfree2(s->dyf);
    dfree2(s->dyb);
    for (int k = 0; k < 2; ++k) {
        dfree2(s->dz[k]);
        dfree2(s->dzf[k]);
    }
    dfree2(s->tA);
    dfree2(s->tB);
    dfree2(s->xin);
    dfree2(s->y_all);
    dfree2(s->ystat);
    s->a.assign(s->NL + 1, nullptr);
    s->z.assign(s->NL, nullptr);
    SR_CUDA(dmalloc(&s->a[0], (size_t)bcap * s->n_in_p));
    for (int l = 1; l <= s->NL; ++l)
        SR_CUDA(dmalloc(&s->a[l], (size_t)bcap * s->H));
    for (int l = 0; l < s->NL; ++l)
        SR_CUDA(dmalloc(&s->z[l], (size_t)bcap * s->H));
    SR_CUDA(dmalloc(&s->y, (size_t)bcap * s->n_out_p));
    SR_CUDA(dmalloc(&s->yt, (size_t)bcap * s->n_out_p));
    SR_CUDA(dmalloc(&s->dyf, (size_t)bcap * s->n_out_p));
    SR_CUDA(dmalloc(&s->dyb, (size_t)bcap * s->n_out_p));
    for (int k = 0; k < 2; ++k) {
        SR_CUDA(dmalloc(&s->dz[k], (size_t)bcap * s->H));
        SR_CUDA(dmalloc(&s->dzf[k], (size_t)bcap * s->H));
    }
    const int wmax = std::max(s->H, s->n_out_p);
    SR_CUDA(dmalloc(&s->tA, (size_t)bcap * wmax));
    SR_CUDA(dmalloc(&s->tB, (size_t)bcap * wmax));
    SR_CUDA(dmalloc(&s->xin, (size_t)bcap * s->n_in_p));
    SR_CUDA(dmalloc(&s->y_all, (size_t)s->n_nets * bcap * s->n_out_p));
    SR_CUDA(dmalloc(&s->ystat, (size_t)2 * bcap * s->n_out));
    s->bcap = bcap;
    return NPSIM_OK;
}

// Forward pass of network k on the batch in a[0] (bp rows, a multiple of 128):
// hidden layers write z (FP32) and a (BF16); the output layer writes y_out
// (FP32; s->y when NULL).
int forward(npsim_surr *s, int k, int bp, float *y_out = nullptr)
{
    auto &net = s->nets[k];
    for (int l = 0; l < s->NL; ++l) {
        Layer &L = net[l];
        SR_CUDA(gemm(s, GEMM_ACT, s->a[l], L.in_p, L.Wb, L.in_p, bp, L.out_p, L.in_p, L.b,
                     nullptr, s->a[l + 1], L.out_p, s->z[l], 1));
    }
    Layer &O = net[s->NL];
    SR_CUDA(gemm(s, GEMM_F32, s->a[s->NL], O.in_p, O.Wb, O.in_p, bp, O.out_p, O.in_p, O.b,
                 y_out ? y_out : s->y, nullptr, O.out_p, nullptr, 0));
    return NPSIM_OK;
}

// Back-propagation of the mean-squared error on rows < m_valid of the batch:
// weight gradients gW = dZ^T A_prev (via transposes), bias gradients = column
// sums of dZ, dZ_prev = (dZ W) * SiLU'(Z_prev).
int backward(npsim_surr *s, int k, int bp, int m_valid)
{
    auto &net = s->nets[k];
    SR_CUDA(cudaMemsetAsync(s->loss, 0, sizeof(float), s->st));
    SR_CUDA(launch_mse_grad(s->y, s->yt, s->outw, bp, m_valid, s->n_out, s->n_out_p, s->dyf,
                            s->dyb, s->loss, s->st));
    // current gradient wrt the pre-activation of layer l: (bf16, fp32, width)
    const __nv_bfloat16 *g_b = s->dyb;
    const float *g_f = s->dyf;
    int g_w = s->n_out_p;
    int ping = 0;
    for (int l = s->NL; l >= 0; --l) {
        Layer &L = net[l];
        // gW = dZ^T (out_p x bp) * A_prev^T^T: A = dZ^T (out_p x bp), B = A_prev^T (in_p x bp)
        SR_CUDA(launch_transpose_bf16(g_b, bp, g_w, g_w, s->tA, bp, s->st));
        SR_CUDA(launch_transpose_bf16(s->a[l], bp, L.in_p, L.in_p, s->tB, bp, s->st));
        SR_CUDA(gemm(s, GEMM_F32, s->tA, bp, s->tB, bp, L.out_p, L.in_p, bp, nullptr, L.gW,
                     nullptr, L.in_p, nullptr, 0));
        SR_CUDA(launch_colsum(g_f, bp, L.out_p, g_w, L.gb, s->st));
        if (l > 0) {
            // dZ_prev = (dZ W) * SiLU'(Z_prev): A = dZ (bp x out_p), B = W^T (in_p x out_p)
            SR_CUDA(gemm(s, GEMM_DACT, g_b, g_w, L.Wt, L.out_p, bp, L.in_p, L.out_p, nullptr,
                         s->dzf[ping], s->dz[ping], L.in_p, s->z[l - 1], 0));
            g_b = s->dz[ping];
            g_f = s->dzf[ping];
            g_w = L.in_p;
            ping ^= 1;
        }
    }
    return NPSIM_OK;
}

int adamw_step(npsim_surr *s, int k, float lr, float wd)
{
    AdamArgs a{};
    a.lr = lr;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    a.wd = wd;
    const double t = (double)s->adam_t;
    a.bc1 = (float)(1.0 - std::pow(0.9, t));
    a.bc2 = (float)(1.0 - std::pow(0.999, t));
    for (auto &L : s->nets[k]) {
        SR_CUDA(launch_adamw(L.W, L.gW, L.mW, L.vW, L.out_p, L.in_p, a, L.Wb, L.Wt, L.mask, s->st));
        AdamArgs ab = a;
        ab.wd = 0.f; // no decay on biases
        SR_CUDA(launch_adamw(L.b, L.gb, L.mb, L.vb, 1, L.out_p, ab, nullptr, nullptr, L.bmask,
                             s->st));
    }
    return NPSIM_OK;
}

// Upload (normalised, padded, BF16) inputs of `rows` samples into a[0] and the
// (normalised, padded) targets into yt; rows beyond are zero.
int upload_batch(npsim_surr *s, const float *X, const float *Y, int rows, int bp)
{
    std::vector<float> xf((size_t)bp * s->n_in_p, 0.f);
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < s->n_in; ++c)
            xf[(size_t)r * s->n_in_p + c] = (X[(size_t)r * s->n_in + c] - s->xm[c]) / s->xs[c];
    SR_CUDA(cudaMemcpyAsync(s->xin, xf.data(), sizeof(float) * xf.size(), cudaMemcpyHostToDevice,
                            s->st));
    SR_CUDA(launch_f32_to_bf16(s->xin, (int)xf.size(), s->a[0], s->st));
    if (Y) {
        std::vector<float> yf((size_t)bp * s->n_out_p, 0.f);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < s->n_out; ++c)
                yf[(size_t)r * s->n_out_p + c] =
                    (Y[(size_t)r * s->n_out + c] - s->ym[c]) / s->ys[c];
        SR_CUDA(cudaMemcpyAsync(s->yt, yf.data(), sizeof(float) * yf.size(),
                                cudaMemcpyHostToDevice, s->st));
        SR_CUDA(cudaStreamSynchronize(s->st));
    }
    return NPSIM_OK;
}

int check_flags(npsim_surr *s)
{
    int h = 0;
    SR_CUDA(cudaMemcpyAsync(&h, s->flags, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    SR_CUDA(cudaStreamSynchronize(s->st));
    if (h) {
        SR_CUDA(cudaMemsetAsync(s->flags, 0, sizeof(int), s->st));
        return report_error(NPSIM_ERR_TIMEOUT, "a tensor-core wait expired (flags 0x%x)", h);
    }
    return NPSIM_OK;
}

__global__ void k_gather_rows(const __nv_bfloat16 *__restrict__ sx, const float *__restrict__ sy,
                              const int *__restrict__ idx, int rows, int bp, int nx, int ny,
                              __nv_bfloat16 *__restrict__ x, float *__restrict__ y)
{
    const int r = blockIdx.x;
    const bool ok = r < rows;
    const int src = ok ? idx[r] : 0;
    for (int c = threadIdx.x; c < nx; c += blockDim.x)
        x[(size_t)r * nx + c] = ok ? sx[(size_t)src * nx + c] : __float2bfloat16_rn(0.f);
    for (int c = threadIdx.x; c < ny; c += blockDim.x)
        y[(size_t)r * ny + c] = ok ? sy[(size_t)src * ny + c] : 0.f;
}

// Mean and spread (population standard deviation) over the networks of the
// de-normalised outputs y * ys + ym, for rows < B and the n_out valid columns.
__global__ void k_ens_stats(const float *__restrict__ y_all, int n_nets, int bp, int ldy, int B,
                            int n_out, const float *__restrict__ ym, const float *__restrict__ ys,
                            float *__restrict__ mean, float *__restrict__ spread)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * n_out)
        return;
    const int r = idx / n_out, c = idx - r * n_out;
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < n_nets; ++k) {
        const double v = (double)y_all[((size_t)k * bp + r) * ldy + c] * ys[c] + ym[c];
        s1 += v;
        s2 += v * v;
    }
    const double m = s1 / n_nets;
    mean[idx] = (float)m;
    spread[idx] = (float)sqrt(fmax(0.0, s2 / n_nets - m * m));
}

} // namespace

extern "C" {

int npsim_surr_create(int32_t n_in, int32_t n_hidden, int32_t n_layers, int32_t n_out,
                      int32_t n_nets, uint64_t seed, npsim_surr_t *out)
{
    NP_TRACE();
    if (!out)
        return report_error(NPSIM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > 64 || n_hidden < 16 || n_hidden > 256 || n_hidden % 16 ||
        n_layers < 1 || n_layers > 8 || n_out < 1 || n_out > 256 || n_nets < 1 || n_nets > 64)
        return report_error(NPSIM_ERR_INVALID_ARG,
                            "surrogate shape out of range (n_in <= 64, hidden 16..256 step 16, "
                            "1..8 layers, n_out <= 256, 1..64 nets)");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
        return report_error(NPSIM_ERR_NO_DEVICE, "no CUDA device visible");
    npsim_surr *s = new npsim_surr();
    auto bail = [&](int rc) {
        delete s;
        return rc;
    };
    s->n_in = n_in;
    s->n_in_p = round16(n_in);
    s->H = n_hidden;
    s->NL = n_layers;
    s->n_out = n_out;
    s->n_out_p = round16(n_out);
    s->n_nets = n_nets;
    s->xm.assign(n_in, 0.f);
    s->xs.assign(n_in, 1.f);
    s->ym.assign(n_out, 0.f);
    s->ys.assign(n_out, 1.f);
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess)
        return bail(report_error(NPSIM_ERR_CUDA, "stream create failed"));
    std::mt19937_64 rng(seed);
    s->Wb_stack.assign(n_layers + 1, nullptr);
    s->b_stack.assign(n_layers + 1, nullptr);
    for (int l = 0; l <= n_layers; ++l) {
        const size_t in_p = l == 0 ? s->n_in_p : n_hidden;
        const size_t out_p = l == n_layers ? s->n_out_p : n_hidden;
        if (dmalloc(&s->Wb_stack[l], (size_t)n_nets * out_p * in_p) != cudaSuccess ||
            dmalloc(&s->b_stack[l], (size_t)n_nets * out_p) != cudaSuccess)
            return bail(report_error(NPSIM_ERR_OOM, "surrogate weights"));
    }
    s->nets.resize(n_nets);
    for (int k = 0; k < n_nets; ++k) {
        s->nets[k].resize(n_layers + 1);
        for (int l = 0; l <= n_layers; ++l) {
            Layer &L = s->nets[k][l];
            L.in = l == 0 ? n_in : n_hidden;
            L.in_p = l == 0 ? s->n_in_p : n_hidden;
            L.out = l == n_layers ? n_out : n_hidden;
            L.out_p = l == n_layers ? s->n_out_p : n_hidden;
            const size_t nw = (size_t)L.out_p * L.in_p;
            // He-uniform initialisation on the valid block, zero padding
            std::vector<float> w(nw, 0.f), b(L.out_p, 0.f);
            std::vector<unsigned char> m(nw, 0), bm(L.out_p, 0);
            const float lim = std::sqrt(6.0f / (float)L.in);
            std::uniform_real_distribution<float> U(-lim, lim);
            for (int r = 0; r < L.out; ++r) {
                bm[r] = 1;
                for (int c = 0; c < L.in; ++c) {
                    w[(size_t)r * L.in_p + c] = U(rng);
                    m[(size_t)r * L.in_p + c] = 1;
                }
            }
            int rc = 0;
#define SRB(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            rc = report_error(NPSIM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
            SRB(dmalloc(&L.W, nw));
            L.b = s->b_stack[l] + (size_t)k * L.out_p;
            L.Wb = s->Wb_stack[l] + (size_t)k * nw;
            SRB(dmalloc(&L.Wt, nw));
            SRB(dmalloc(&L.mW, nw));
            SRB(dmalloc(&L.vW, nw));
            SRB(dmalloc(&L.mb, L.out_p));
            SRB(dmalloc(&L.vb, L.out_p));
            SRB(dmalloc(&L.gW, nw));
            SRB(dmalloc(&L.gb, L.out_p));
            SRB(dmalloc(&L.mask, nw));
            SRB(dmalloc(&L.bmask, L.out_p));
            if (rc)
                return bail(rc);
            SRB(cudaMemcpy(L.W, w.data(), sizeof(float) * nw, cudaMemcpyHostToDevice));
            SRB(cudaMemcpy(L.b, b.data(), sizeof(float) * L.out_p, cudaMemcpyHostToDevice));
            SRB(cudaMemcpy(L.mask, m.data(), nw, cudaMemcpyHostToDevice));
            SRB(cudaMemcpy(L.bmask, bm.data(), L.out_p, cudaMemcpyHostToDevice));
            SRB(cudaMemset(L.mW, 0, sizeof(float) * nw));
            SRB(cudaMemset(L.vW, 0, sizeof(float) * nw));
            SRB(cudaMemset(L.mb, 0, sizeof(float) * L.out_p));
            SRB(cudaMemset(L.vb, 0, sizeof(float) * L.out_p));
            if (rc)
                return bail(rc);
            SRB(cudaMemset(L.gW, 0, sizeof(float) * nw));
            SRB(cudaMemset(L.gb, 0, sizeof(float) * L.out_p));
            SRB(launch_weights_bf16(L.W, L.out_p, L.in_p, L.Wb, L.Wt, s->st));
#undef SRB
            if (rc)
                return bail(rc);
        }
    }
    if (dmalloc(&s->loss, 1) != cudaSuccess || dmalloc(&s->flags, 1) != cudaSuccess ||
        dmalloc(&s->outw, (size_t)s->n_out_p) != cudaSuccess ||
        dmalloc(&s->d_ym, (size_t)n_out) != cudaSuccess ||
        dmalloc(&s->d_ys, (size_t)n_out) != cudaSuccess)
        return bail(report_error(NPSIM_ERR_OOM, "surrogate scratch"));
    cudaMemcpy(s->d_ym, s->ym.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
    cudaMemcpy(s->d_ys, s->ys.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
    std::vector<float> ow(s->n_out_p, 0.f);
    for (int c = 0; c < n_out; ++c)
        ow[c] = 1.f;
    cudaMemcpy(s->outw, ow.data(), sizeof(float) * ow.size(), cudaMemcpyHostToDevice);
    cudaMemset(s->flags, 0, sizeof(int));
    int rc = alloc_batch(s, 512);
    if (rc)
        return bail(rc);
    if (cudaStreamSynchronize(s->st) != cudaSuccess)
        return bail(report_error(NPSIM_ERR_CUDA, "surrogate init failed"));
    *out = s;
    return NPSIM_OK;
}

void npsim_surr_destroy(npsim_surr_t s)
{
    if (!s)
        return;
    cudaStreamSynchronize(s->st);
    delete s;
}

int npsim_surr_set_norm(npsim_surr_t s, const float *x_mean, const float *x_std,
                        const float *y_mean, const float *y_std)
{
    if (!s)
        return report_error(NPSIM_ERR_INVALID_ARG, "surrogate is NULL");
    for (int c = 0; c < s->n_in; ++c) {
        s->xm[c] = x_mean ? x_mean[c] : 0.f;
        s->xs[c] = x_std ? x_std[c] : 1.f;
        if (!(s->xs[c] > 0.f))
            return report_error(NPSIM_ERR_INVALID_ARG, "x_std[%d] must be positive", c);
    }
    for (int c = 0; c < s->n_out; ++c) {
        s->ym[c] = y_mean ? y_mean[c] : 0.f;
        s->ys[c] = y_std ? y_std[c] : 1.f;
        if (!(s->ys[c] > 0.f))
            return report_error(NPSIM_ERR_INVALID_ARG, "y_std[%d] must be positive", c);
    }
    SR_CUDA(cudaMemcpyAsync(s->d_ym, s->ym.data(), sizeof(float) * s->n_out,
                            cudaMemcpyHostToDevice, s->st));
    SR_CUDA(cudaMemcpyAsync(s->d_ys, s->ys.data(), sizeof(float) * s->n_out,
                            cudaMemcpyHostToDevice, s->st));
    SR_CUDA(cudaStreamSynchronize(s->st));
    return NPSIM_OK;
}

int npsim_surr_param_count(npsim_surr_t s, int64_t *count)
{
    if (!s || !count)
        return report_error(NPSIM_ERR_INVALID_ARG, "surrogate and count are required");
    int64_t n = 0;
    for (auto &L : s->nets[0])
        n += (int64_t)L.out_p * L.in_p + L.out_p;
    *count = n;
    return NPSIM_OK;
}

int npsim_surr_get_params(npsim_surr_t s, int32_t net, float *flat, float *grads)
{
    if (!s || net < 0 || net >= s->n_nets)
        return report_error(NPSIM_ERR_INVALID_ARG, "bad surrogate or net index");
    SR_CUDA(cudaStreamSynchronize(s->st));
    size_t off = 0;
    for (auto &L : s->nets[net]) {
        const size_t nw = (size_t)L.out_p * L.in_p;
        if (flat) {
            SR_CUDA(cudaMemcpy(flat + off, L.W, sizeof(float) * nw, cudaMemcpyDeviceToHost));
            SR_CUDA(cudaMemcpy(flat + off + nw, L.b, sizeof(float) * L.out_p,
                               cudaMemcpyDeviceToHost));
        }
        if (grads) {
            SR_CUDA(cudaMemcpy(grads + off, L.gW, sizeof(float) * nw, cudaMemcpyDeviceToHost));
            SR_CUDA(cudaMemcpy(grads + off + nw, L.gb, sizeof(float) * L.out_p,
                               cudaMemcpyDeviceToHost));
        }
        off += nw + L.out_p;
    }
    return NPSIM_OK;
}

int npsim_surr_set_params(npsim_surr_t s, int32_t net, const float *flat)
{
    if (!s || !flat || net < 0 || net >= s->n_nets)
        return report_error(NPSIM_ERR_INVALID_ARG, "bad surrogate, net index or params");
    size_t off = 0;
    for (auto &L : s->nets[net]) {
        const size_t nw = (size_t)L.out_p * L.in_p;
        SR_CUDA(cudaMemcpy(L.W, flat + off, sizeof(float) * nw, cudaMemcpyHostToDevice));
        SR_CUDA(cudaMemcpy(L.b, flat + off + nw, sizeof(float) * L.out_p, cudaMemcpyHostToDevice));
        SR_CUDA(launch_weights_bf16(L.W, L.out_p, L.in_p, L.Wb, L.Wt, s->st));
        off += nw + L.out_p;
    }
    SR_CUDA(cudaStreamSynchronize(s->st));
    return NPSIM_OK;
}

int npsim_surr_grads(npsim_surr_t s, int32_t net, const float *X, const float *Y, int32_t B,
                     float *grads, float *loss, float *Yhat)
{
    if (!s || !X || !Y || B < 1 || net < 0 || net >= s->n_nets)
        return report_error(NPSIM_ERR_INVALID_ARG, "bad surrogate, net, inputs or batch");
    const int bp = (B + 127) / 128 * 128;
    int rc = alloc_batch(s, bp);
    if (rc)
        return rc;
    rc = upload_batch(s, X, Y, B, bp);
    if (rc)
        return rc;
    rc = forward(s, net, bp);
    if (rc)
        return rc;
    rc = backward(s, net, bp, B);
    if (rc)
        return rc;
    rc = check_flags(s);
    if (rc)
        return rc;
    if (loss)
        SR_CUDA(cudaMemcpy(loss, s->loss, sizeof(float), cudaMemcpyDeviceToHost));
    if (Yhat) {
        std::vector<float> yy((size_t)bp * s->n_out_p);
        SR_CUDA(cudaMemcpy(yy.data(), s->y, sizeof(float) * yy.size(), cudaMemcpyDeviceToHost));
        for (int r = 0; r < B; ++r)
            for (int c = 0; c < s->n_out; ++c)
                Yhat[(size_t)r * s->n_out + c] = yy[(size_t)r * s->n_out_p + c];
    }
    return npsim_surr_get_params(s, net, nullptr, grads);
}

int npsim_surr_train(npsim_surr_t s, const float *X, const float *Y, int32_t n_samples,
                     int32_t epochs, int32_t batch, float lr, float wd, uint64_t shuffle_seed,
                     float *final_loss)
{
    NP_TRACE();
    if (!s || !X || !Y || n_samples < 1 || epochs < 0 || batch < 1 || batch > 8192)
        return report_error(NPSIM_ERR_INVALID_ARG, "bad training arguments");
    const int bp = (batch + 127) / 128 * 128;
    int rc = alloc_batch(s, bp);
    if (rc)
        return rc;
    // dataset on the device, normalised and padded
    dfree2(s->dsx);
    dfree2(s->dsy);
    {
        std::vector<float> xf((size_t)n_samples * s->n_in_p, 0.f);
        std::vector<float> yf((size_t)n_samples * s->n_out_p, 0.f);
        for (int r = 0; r < n_samples; ++r) {
            for (int c = 0; c < s->n_in; ++c)
                xf[(size_t)r * s->n_in_p + c] = (X[(size_t)r * s->n_in + c] - s->xm[c]) / s->xs[c];
            for (int c = 0; c < s->n_out; ++c)
                yf[(size_t)r * s->n_out_p + c] = (Y[(size_t)r * s->n_out + c] - s->ym[c]) / s->ys[c];
        }
        float *tmp = nullptr;
        SR_CUDA(dmalloc(&tmp, xf.size()));
        SR_CUDA(dmalloc(&s->dsx, xf.size()));
        SR_CUDA(dmalloc(&s->dsy, yf.size()));
        SR_CUDA(cudaMemcpy(tmp, xf.data(), sizeof(float) * xf.size(), cudaMemcpyHostToDevice));
        SR_CUDA(launch_f32_to_bf16(tmp, (int)xf.size(), s->dsx, s->st));
        SR_CUDA(cudaMemcpy(s->dsy, yf.data(), sizeof(float) * yf.size(), cudaMemcpyHostToDevice));
        SR_CUDA(cudaStreamSynchronize(s->st));
        cudaFree(tmp);
        s->ds_n = n_samples;
    }
    int *d_idx = nullptr;
    SR_CUDA(dmalloc(&d_idx, (size_t)n_samples));
    std::vector<std::vector<int>> order(s->n_nets, std::vector<int>(n_samples));
    std::mt19937_64 rng(shuffle_seed);
    float last = 0.f;
    const int nb = (n_samples + batch - 1) / batch;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int k = 0; k < s->n_nets; ++k) {
            for (int i = 0; i < n_samples; ++i)
                order[k][i] = i;
            std::shuffle(order[k].begin(), order[k].end(), rng);
        }
        for (int b = 0; b < nb; ++b) {
            const int r0 = b * batch, rows = std::min(batch, n_samples - r0);
            ++s->adam_t;
            for (int k = 0; k < s->n_nets; ++k) {
                cudaError_t e = cudaMemcpyAsync(d_idx, order[k].data() + r0, sizeof(int) * rows,
                                                cudaMemcpyHostToDevice, s->st);
                if (e != cudaSuccess) {
                    cudaFree(d_idx);
                    return report_error(NPSIM_ERR_CUDA, "index upload: %s", cudaGetErrorString(e));
                }
                k_gather_rows<<<bp, 128, 0, s->st>>>(s->dsx, s->dsy, d_idx, rows, bp, s->n_in_p,
                                                     s->n_out_p, s->a[0], s->yt);
                rc = forward(s, k, bp);
                if (!rc)
                    rc = backward(s, k, bp, rows);
                if (!rc)
                    rc = adamw_step(s, k, lr, wd);
                if (rc) {
                    cudaFree(d_idx);
                    return rc;
                }
            }
            if (b + 1 == nb) {
                cudaStreamSynchronize(s->st);
                cudaMemcpy(&last, s->loss, sizeof(float), cudaMemcpyDeviceToHost);
            }
        }
        rc = check_flags(s);
        if (rc) {
            cudaFree(d_idx);
            return rc;
        }
    }
    cudaFree(d_idx);
    SR_CUDA(cudaStreamSynchronize(s->st));
    if (final_loss)
        *final_loss = last;
    return NPSIM_OK;
}

int npsim_surr_predict(npsim_surr_t s, const float *X, int32_t B, float *Y_mean, float *Y_spread)
{
    NP_TRACE();
    if (!s || !X || !Y_mean || B < 1 || B > 65536)
        return report_error(NPSIM_ERR_INVALID_ARG, "bad prediction arguments");
    const int bp = (B + 127) / 128 * 128;
    int rc = alloc_batch(s, bp);
    if (rc)
        return rc;
    rc = upload_batch(s, X, nullptr, B, bp);
    if (rc)
        return rc;
    // NPSIM_SURR_LAYERED selects the layer-by-layer GEMM path (same arithmetic)
    const bool layered = getenv("NPSIM_SURR_LAYERED") != nullptr;
    if (!layered && mlp_infer_supported(s->NL, s->n_in_p, s->H, s->n_out_p)) {
        // every layer of every network in one launch
        MlpInferArgs f{};
        f.X = s->a[0];
        for (int l = 0; l <= s->NL; ++l) {
            f.W[l] = s->Wb_stack[l];
            f.b[l] = s->b_stack[l];
        }
        f.NL = s->NL;
        f.in_p = s->n_in_p;
        f.H = s->H;
        f.out_p = s->n_out_p;
        f.bp = bp;
        f.n_nets = s->n_nets;
        f.y = s->y_all;
        f.flags = s->flags;
        SR_CUDA(launch_mlp_infer(f, s->st));
    } else {
        for (int k = 0; k < s->n_nets; ++k) {
            rc = forward(s, k, bp, s->y_all + (size_t)k * bp * s->n_out_p);
            if (rc)
                return rc;
        }
    }
    float *d_mean = s->ystat, *d_spread = s->ystat + (size_t)B * s->n_out;
    const int ne = B * s->n_out;
    k_ens_stats<<<(ne + 255) / 256, 256, 0, s->st>>>(s->y_all, s->n_nets, bp, s->n_out_p, B,
                                                     s->n_out, s->d_ym, s->d_ys, d_mean,
                                                     d_spread);
    SR_CUDA(cudaGetLastError());
    SR_CUDA(cudaMemcpyAsync(Y_mean, d_mean, sizeof(float) * ne, cudaMemcpyDeviceToHost, s->st));
    if (Y_spread)
        SR_CUDA(cudaMemcpyAsync(Y_spread, d_spread, sizeof(float) * ne, cudaMemcpyDeviceToHost,
                                s->st));
    SR_CUDA(cudaStreamSynchronize(s->st));
    return check_flags(s);
}

int npsim_test_wait_cycles(int64_t cycles)
{
    if (cycles < 0)
        return report_error(NPSIM_ERR_INVALID_ARG, "cycles must be >= 0");
    g_wait_cycles.store((long long)cycles);
    return NPSIM_OK;
}

// Test hook: C = A B^T for host BF16 matrices (bit patterns), C in FP32.
int npsim_gemm_bf16(const uint16_t *A, const uint16_t *B, int32_t M, int32_t N, int32_t K,
                    int32_t n_tile, float *C)
{
    NP_TRACE();
    if (!A || !B || !C || M < 1 || N < 16 || K < 16 || N % 16 || K % 16 || n_tile % 16 ||
        n_tile < 16 || n_tile > 256)
        return report_error(NPSIM_ERR_INVALID_ARG, "gemm shape: N, K, n_tile multiples of 16");
    __nv_bfloat16 *dA = nullptr, *dB = nullptr;
    float *dC = nullptr;
    int *dflag = nullptr;
    SR_CUDA(dmalloc(&dA, (size_t)M * K));
    SR_CUDA(dmalloc(&dB, (size_t)N * K));
    SR_CUDA(dmalloc(&dC, (size_t)M * N));
    SR_CUDA(dmalloc(&dflag, 1));
    SR_CUDA(cudaMemcpy(dA, A, sizeof(uint16_t) * (size_t)M * K, cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemcpy(dB, B, sizeof(uint16_t) * (size_t)N * K, cudaMemcpyHostToDevice));
    SR_CUDA(cudaMemset(dflag, 0, sizeof(int)));
    GemmArgs g{};
    g.A = dA;
    g.B = dB;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = K;
    g.ldb = K;
    g.ldc = N;
    g.n_tile = n_tile;
    g.tmem_cols = pow2_at_least(n_tile);
    g.mode = GEMM_F32;
    g.Cf = dC;
    g.flags = dflag;
    g.wait_cycles = g_wait_cycles.load();
    cudaError_t e = launch_gemm(g, 0);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    int flag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(C, dC, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(dflag);
    if (e != cudaSuccess)
        return report_error(NPSIM_ERR_CUDA, "gemm: %s", cudaGetErrorString(e));
    if (flag)
        return report_error(NPSIM_ERR_TIMEOUT, "gemm: a tensor-core wait expired");
    return NPSIM_OK;
}

} // extern "C"
