// noalloc.cu -- all-pairs Coulomb forces for callers that must not allocate
// device memory.
//
// The regular path keeps the all-pairs partial sums (one slot of compensated
// float32 (hi, lo) pairs per i-tile row and CTA of the stream-K split) in memory that npsim_create
// allocates.  Some callers cannot allocate at the moment they need forces:
// code running under a framework that owns all device memory through its own
// pool and forbids raw allocations, or a real-time loop that cannot afford an
// allocation's latency or its failure in the middle of a run.  For them, this
// file holds the partial sums in one file-scope __device__ array of fixed size,
// present on every GPU that loads the library until the process exits, and the
// entry point npsim_coulomb_forces_noalloc allocates nothing.
//
// The computation is the same Coulomb sum as npsim_forces(sim, 3, ...):
//   F_i = C q_i sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3,
// using the packed float32x2 all-pairs kernel of allpairs.cu, followed by a
// reduction of each row's partials in CTA order (deterministic).
#include <cuda.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "npsim_internal.cuh"

namespace npsim {

namespace {

// Largest number of NPs one call accepts, and the fixed scratch it needs: with a
// launch shape of i-tile 512 and at most kMaxGrid CTAs, a call writes at most
// (ceil(n / 512) + kMaxGrid) slots of 6 x 512 floats.
constexpr int kMaxN = 32768;
constexpr int kMaxGrid = 256;
constexpr int kMaxItile = 512;
constexpr size_t kScratchFloats =
    (size_t)((kMaxN + kMaxItile - 1) / kMaxItile + kMaxGrid) * 6 * kMaxItile; // 3.75 MiB

__device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool done = false;
    CUcontext ctx = nullptr;   // the context the set-up was done in
    float *scratch = nullptr;  // device address of g_scratch on this device
    int shape = -1;            // all-pairs launch shape (index in the autotuner table)
    int grid_cap = 0;          // CTAs: min(kMaxGrid, resident CTAs of the shape)
};

std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

// The calling thread's current driver context (NULL if none yet, or if the
// driver entry point is unavailable), through the runtime's driver entry point
// lookup so that the library does not link the driver library.
CUcontext current_context()
{
    using Fn = CUresult (*)(CUcontext *);
    static const Fn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<Fn>(p);
        return static_cast<Fn>(nullptr);
    }();
    CUcontext c = nullptr;
    if (fn && fn(&c) != CUDA_SUCCESS)
        c = nullptr;
    return c;
}

// Once per device and context, with that device current: the device address
// of g_scratch (in host code the array's name is only a host-side stand-in)
// and the launch shape.  The first call on a device runs this; the result is
// kept and reused while the calling thread's current context is the one it was
// made in, and made again when that changes (after a cudaDeviceReset the
// module is loaded again in a new primary context, at a new address).
int setup_device(int dev, DeviceSetup &out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup &s = g_setup[dev];
    const CUcontext ctx = current_context();
    if (!s.done || ctx == nullptr || ctx != s.ctx) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess)
            return report_error(NPSIM_ERR_CUDA, "cudaGetSymbolAddress(g_scratch) failed: %s",
                                cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return report_error(NPSIM_ERR_CUDA, "cudaDeviceGetAttribute failed: %s",
                                cudaGetErrorString(e));
        int shape = -1, cap = 0;
        for (int k = 0; k < ap_num_configs() && shape < 0; ++k) {
            const ApConfig c = ap_config(k);
            const int occ = ap_occupancy(k, false);
            if (ap_packed(k) && occ > 0 && c.block * c.ki == kMaxItile) {
                shape = k;
                cap = occ * sms < kMaxGrid ? occ * sms : kMaxGrid;
            }
        }
        if (shape < 0)
            return report_error(NPSIM_ERR_CUDA, "no packed all-pairs shape with i-tile %d",
                                kMaxItile);
        s.scratch = (float *)ptr;
        s.shape = shape;
        s.grid_cap = cap;
        s.ctx = current_context(); // made current by the symbol lookup if it was not
        s.done = true;
    }
    out = s;
    return NPSIM_OK;
}

__global__ void k_noalloc_reduce(const float4 *__restrict__ xq, int n, StreamK sk, double C,
                                 double *__restrict__ F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int r = i / sk.itile;
    const int idx = i - r * sk.itile;
    const long long u0 = (long long)r * sk.n_jt;
    const int c0 = sk_cta_of(sk, u0);
    const int c1 = sk_cta_of(sk, u0 + sk.n_jt - 1);
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int c = c0; c <= c1; ++c) {
        // slots hold (hi x, y, z, lo x, y, z) float words
        const float *slot = g_scratch + (size_t)(r + c) * 6 * sk.itile;
        fx += (double)slot[idx] + (double)slot[3 * sk.itile + idx];
        fy += (double)slot[sk.itile + idx] + (double)slot[4 * sk.itile + idx];
        fz += (double)slot[2 * sk.itile + idx] + (double)slot[5 * sk.itile + idx];
    }
    const double qc = C * (double)xq[i].w;
    F[3 * (size_t)i + 0] = qc * fx;
    F[3 * (size_t)i + 1] = qc * fy;
    F[3 * (size_t)i + 2] = qc * fz;
}

} // namespace

} // namespace npsim

using namespace npsim;

extern "C" int npsim_coulomb_forces_noalloc(const float *dev_xyzq, int64_t n, double bjerrum,
                                            double *dev_F, void *stream)
{
    if (!dev_xyzq || !dev_F)
        return report_error(NPSIM_ERR_INVALID_ARG, "dev_xyzq and dev_F are required");
    if (n < 1 || n > kMaxN)
        return report_error(NPSIM_ERR_INVALID_ARG,
                            "n = %lld is outside [1, %d], the size the fixed scratch holds",
                            (long long)n, kMaxN);
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1)
        return report_error(NPSIM_ERR_NO_DEVICE, "no CUDA device visible");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report_error(NPSIM_ERR_CUDA, "cudaGetDevice failed or device index too large");
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (!(major == 10 && minor == 3))
        return report_error(NPSIM_ERR_NO_DEVICE, "device %d is sm_%d%d, not sm_103", dev,
                            major, minor);
    DeviceSetup su;
    int rc = setup_device(dev, su);
    if (rc)
        return rc;

    const ApConfig c = ap_config(su.shape);
    StreamK sk{};
    sk.itile = c.block * c.ki;
    sk.jtile = c.jt;
    sk.n_it = (int)((n + sk.itile - 1) / sk.itile);
    sk.n_jt = (int)((n + c.jt - 1) / c.jt);
    sk.W = (long long)sk.n_it * sk.n_jt;
    sk.grid = (int)(sk.W < su.grid_cap ? sk.W : su.grid_cap);
    if ((size_t)(sk.n_it + sk.grid) * 6 * (size_t)sk.itile > kScratchFloats)
        return report_error(NPSIM_ERR_INVALID_ARG, "n = %lld needs more scratch than %zu floats",
                            (long long)n, kScratchFloats);

    cudaStream_t st = (cudaStream_t)stream;
    const float4 *xq = (const float4 *)dev_xyzq;
    e = launch_allpairs(su.shape, false, sk, xq, nullptr, (int)n, nullptr, su.scratch, st);
    if (e != cudaSuccess)
        return report_error(NPSIM_ERR_CUDA, "all-pairs launch failed: %s", cudaGetErrorString(e));
    k_noalloc_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xq, (int)n, sk, bjerrum, dev_F);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return report_error(NPSIM_ERR_CUDA, "reduction launch failed: %s", cudaGetErrorString(e));
    return NPSIM_OK;
}
