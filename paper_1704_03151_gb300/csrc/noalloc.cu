// noalloc.cu -- residual-norm reduction that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need the
// convergence measure: host frameworks that hand out only their own pre-sized
// pools and forbid the CUDA allocator, and long-running loops that must not
// touch the allocator for latency reasons.
// miugks_residual_rms_noalloc serves them: it reduces caller-owned device
// arrays into a caller-owned output using a scratch area that lives in this
// file, in a static __device__ array that every GPU loading the library keeps
// until the process exits.
//
// The scratch holds one row of partial sums per 256-cell block, at most
// kNoAllocMaxBlocks rows, so a call accepts at most 1,048,576 cells.  Cells
// marked solid (inside a body) are left out of the sums and of the count the
// mean divides by, as in the solver's own residual.  Every
// row a call reads is written by the same call first, so nothing needs
// clearing between calls; the array keeps the last call's partial sums.  All
// calls share this one array: calls whose kernels overlap on the GPU (on
// different streams, or different host threads) race on it and must be
// serialised by the caller.
#include <mutex>

#include "../../include/miugks.h"
#include "common.cuh"

namespace {

constexpr int kNoAllocBlock = 256;                  // cells per partial row
constexpr int kNoAllocMaxBlocks = 4096;             // rows of scratch
constexpr int kNoAllocRow = 6;                      // 4 squared sums, unphysical cells, fluid cells
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_rms_scratch[kNoAllocMaxBlocks * kNoAllocRow];

// per-device address of g_rms_scratch (host code only sees a stand-in for the symbol)
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__global__ void k_rms_rows(const double* __restrict__ R, const double* __restrict__ W,
                           const unsigned char* __restrict__ solid, int nc, double* __restrict__ rows)
{
    __shared__ double red[32 * kNoAllocRow];
    double s[kNoAllocRow] = {0, 0, 0, 0, 0, 0};
    int c = blockIdx.x * kNoAllocBlock + threadIdx.x;
    if (c < nc && !(solid && solid[c])) {
        for (int m = 0; m < 4; ++m) s[m] = R[4 * (size_t)c + m] * R[4 * (size_t)c + m];
        const double* w = W + 4 * (size_t)c;
        // rho > 0 and rho * (internal energy) = rho E - |m|^2 / 2 > 0 (false for NaN), without a division
        const double e2 = w[3] * w[0] - 0.5 * (w[1] * w[1] + w[2] * w[2]);
        if (!(w[0] > 0.0) || !(e2 > 0.0)) s[4] = 1.0;
        s[5] = 1.0;
    }
    miugks::block_sum<kNoAllocRow>(s, red);
    if (threadIdx.x == 0)
        for (int m = 0; m < kNoAllocRow; ++m) rows[kNoAllocRow * (size_t)blockIdx.x + m] = s[m];
}

__global__ void k_rms_rows_final(const double* __restrict__ rows, int nrows, double* __restrict__ out)
{
    __shared__ double red[32 * kNoAllocRow];
    double s[kNoAllocRow] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nrows; b += blockDim.x)
        for (int m = 0; m < kNoAllocRow; ++m) s[m] += rows[kNoAllocRow * (size_t)b + m];
    miugks::block_sum<kNoAllocRow>(s, red);
    if (threadIdx.x == 0) {
        const double n = s[5] > 0.0 ? s[5] : 1.0;     // every cell solid: zero sums, reported as 0
        for (int m = 0; m < 4; ++m) out[m] = sqrt(s[m] / n);
        out[4] = s[4];
    }
}

} // namespace

extern "C" void miugks_set_thread_error(const char* msg);

extern "C" miugks_status miugks_residual_rms_noalloc(const double* R_dev, const double* W_dev,
                                                     const unsigned char* solid_dev, int nc, double* out_dev,
                                                     void* cuda_stream)
{
    if (!R_dev || !W_dev || !out_dev || nc < 1) {
        miugks_set_thread_error("miugks_residual_rms_noalloc: null pointer or nc < 1");
        return MIUGKS_EINVAL;
    }
    const int nrows = (nc + kNoAllocBlock - 1) / kNoAllocBlock;
    if (nrows > kNoAllocMaxBlocks) {
        miugks_set_thread_error("miugks_residual_rms_noalloc: nc exceeds the fixed scratch capacity of 1048576 cells");
        return MIUGKS_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        miugks_set_thread_error("miugks_residual_rms_noalloc: no usable current CUDA device");
        return MIUGKS_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* rows;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            // first call on this device: resolve the scratch symbol with this device current.
            // The address is kept for the life of the process; a device reset reloads the
            // module elsewhere, so the library must not be used across cudaDeviceReset.
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_rms_scratch) != cudaSuccess || !p) {
                (void)cudaGetLastError();
                miugks_set_thread_error("miugks_residual_rms_noalloc: cudaGetSymbolAddress failed");
                return MIUGKS_ECUDA;
            }
            g_scratch_addr[dev] = (double*)p;
        }
        rows = g_scratch_addr[dev];
    }
    k_rms_rows<<<nrows, kNoAllocBlock, 0, st>>>(R_dev, W_dev, solid_dev, nc, rows);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_rms_rows_final<<<1, 256, 0, st>>>(rows, nrows, out_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        miugks_set_thread_error(cudaGetErrorString(e));
        return MIUGKS_ECUDA;
    }
    return MIUGKS_OK;
}
