// noalloc.cu -- one plain ST-BIEM step from caller-provided buffers, without any allocation.
//
// Some callers cannot allocate device memory at all: code that runs inside another runtime's
// memory pool, inside a stream-ordered region where a cudaMalloc would synchronise the device,
// or in a process whose allocator is owned and budgeted by someone else.  For them,
// fdph_plain_step_noalloc evaluates T_n = sum_{k <= min(n, W-1)} K_k D_{n-k} (Eq. 4) from a
// kernel tensor and a slip-rate history they already hold, and keeps its split-k partial sums
// in the file-scope array below instead of in allocated scratch.  The array lives on every GPU
// that loads the library until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/fdph.h"
#include "internal.h"

namespace {

const int kTile = 32;          // receivers per work item
const int kSteps = 64;         // kernel steps per work item
const int kThreads = 128;

// Shared by every call on a device; each call overwrites the slots it uses.
static __device__ __align__(256) double g_noalloc_partials[FDPH_NOALLOC_MAX_PARTIALS];

std::mutex g_mu;
double* g_addr[64] = {nullptr};   // device address of the array, per device ordinal

__device__ __forceinline__ int ring_slot(long long t, int L) {
    long long r = t % L;
    return (int)(r < 0 ? r + L : r);
}

// Work item = (receiver tile, chunk of kernel steps); lane = receiver, warps split the steps.
__global__ void __launch_bounds__(kThreads) noalloc_partial_kernel(const double* __restrict__ K, int n, int kmax,
                                                                   const double* __restrict__ D, int hist_len,
                                                                   int step, int nchunks, double* partial) {
    __shared__ double red[kThreads / 32][32];
    const int tile = blockIdx.x / nchunks, chunk = blockIdx.x % nchunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = tile * kTile + lane;
    const int k0 = chunk * kSteps, k1 = min(kmax, k0 + kSteps);
    double acc = 0.0;
    for (int k = k0 + warp; k < k1; k += kThreads / 32) {
        const double* Dk = D + (size_t)ring_slot((long long)step - k, hist_len) * n;
        const double* Kk = K + (size_t)k * n * n;
        if (i < n)
            for (int j = 0; j < n; ++j) acc += Kk[(size_t)j * n + i] * Dk[j];
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][lane];
        partial[(size_t)blockIdx.x * kTile + lane] = s;   // every slot of the item is written
    }
}

__global__ void noalloc_reduce_kernel(const double* partial, int n, int nchunks, double* T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int tile = i / kTile, lane = i % kTile;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += partial[((size_t)tile * nchunks + c) * kTile + lane];
    T[i] = s;
}

}  // namespace

extern "C" int fdph_plain_step_noalloc(const double* K, int32_t n, int32_t W, const double* D_hist,
                                       int32_t hist_len, int32_t step, double* T, void* stream) {
    if (!K || !D_hist || !T || n <= 0 || W <= 0 || hist_len <= 0 || step < 0) {
        fdph::set_error("fdph_plain_step_noalloc: null pointer or non-positive size");
        return FDPH_E_ARG;
    }
    const int kmax = step + 1 < W ? step + 1 : W;
    if (hist_len < kmax) {
        fdph::set_error("fdph_plain_step_noalloc: hist_len must cover min(step + 1, W) steps");
        return FDPH_E_ARG;
    }
    // sizes in 64-bit arithmetic: n + kTile - 1 would overflow int32 for n near INT32_MAX
    const long long tiles = ((long long)n + kTile - 1) / kTile;
    const long long nchunks = ((long long)kmax + kSteps - 1) / kSteps;
    if (tiles * nchunks * kTile > FDPH_NOALLOC_MAX_PARTIALS) {
        fdph::set_error("fdph_plain_step_noalloc: ceil(n/32) * ceil(min(step+1, W)/64) * 32 = " +
                        std::to_string(tiles * nchunks * kTile) + " exceeds FDPH_NOALLOC_MAX_PARTIALS = " +
                        std::to_string(FDPH_NOALLOC_MAX_PARTIALS));
        return FDPH_E_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        fdph::set_error("fdph_plain_step_noalloc: no current CUDA device");
        return FDPH_E_CUDA;
    }
    double* partial = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            // first call on this device: host code must ask the runtime for the array's device
            // address (its host-side name is only a stand-in)
            cudaError_t e = cudaGetSymbolAddress((void**)&g_addr[dev], g_noalloc_partials);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                fdph::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return FDPH_E_CUDA;
            }
        }
        partial = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    noalloc_partial_kernel<<<(unsigned)(tiles * nchunks), kThreads, 0, s>>>(K, n, kmax, D_hist, hist_len, step,
                                                                             (int)nchunks, partial);
    noalloc_reduce_kernel<<<(unsigned)(((long long)n + 127) / 128), 128, 0, s>>>(partial, n, (int)nchunks, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fdph::set_error(std::string("fdph_plain_step_noalloc launch: ") + cudaGetErrorString(e));
        return FDPH_E_CUDA;
    }
    return FDPH_OK;
}
