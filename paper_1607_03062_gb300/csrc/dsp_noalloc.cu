// dsp_noalloc.cu -- a pair-density reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a host application or framework may
// already own all of the device memory through its own allocator (so a raw
// cudaMalloc would fail or fragment its pool), or the caller may run in a
// latency-critical loop where cudaMalloc/cudaFree, which can synchronise the
// device, are not allowed.  For them, dsp_density_noalloc reduces a |c+|^2
// map they already hold in device memory to the pair density using only a
// fixed scratch array that lives in this library's static device memory.
//
// The scratch is a file-scope __device__ array of kStaticMaxParts + 1 doubles
// (about 2 MB); every GPU that loads the library holds it until the process
// exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current and
// cached for the rest of the process (a cudaDeviceReset afterwards is not
// supported); the kernels are given that address (in host code the array's
// name is only a host-side stand-in, never a device address).
//
// The arithmetic is the same as the reduction behind dsp_reduce_density: the
// same granules of 256 points, the same double-float pairwise tree per granule
// (granule_sums), the same fixed-order final sum and the same 4/(2 pi)^2 hx hy
// prefactor.  Each point's term is its map value: a double of an FP64 map split
// into a pair exactly as the projection splits it, a float of an FP32_MIXED
// map as (value, 0).

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "dsp.h"
#include "dsp_df.cuh"
#include "dsp_internal.h"

namespace {

// Up to 262144 granules of 256 points: DSP_NOALLOC_MAX_POINTS = 67,108,864 points.
constexpr int kStaticMaxParts = DSP_NOALLOC_MAX_POINTS / dsp::kGranule;
static_assert(static_cast<long long>(kStaticMaxParts) * dsp::kGranule == DSP_NOALLOC_MAX_POINTS,
              "the static scratch must hold one partial sum per granule");
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;
constexpr int kPoints = dsp::kTilePoints / kThreads;  // points per thread

// [0, kStaticMaxParts): per-granule partial sums; [kStaticMaxParts]: the density.
static __device__ __align__(256) double g_noalloc_scratch[kStaticMaxParts + 1];

std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Granule partial sums of the map, one CTA per 1024 points (4 granules).
__global__ void __launch_bounds__(kThreads)
    noalloc_granule_sums(const void *map, int precision, int64_t n_points, double *partials)
{
    __shared__ float2 red[dsp::kTilePoints];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * dsp::kTilePoints;
#pragma unroll
    for (int s = 0; s < kPoints; ++s) {
        const int64_t idx = base + s * kThreads + threadIdx.x;
        float2 v = make_float2(0.0f, 0.0f);
        if (idx < n_points) {
            if (precision == DSP_FP64)
                dsp::split_f64(static_cast<const double *>(map)[idx], v.x, v.y);
            else
                v.x = static_cast<const float *>(map)[idx];
        }
        red[s * kThreads + threadIdx.x] = v;
    }
    dsp::granule_sums(red, dsp::kTilePoints / dsp::kGranule, partials,
                      (n_points + dsp::kGranule - 1) / dsp::kGranule,
                      [&](int g) { return base / dsp::kGranule + g; });
}

// Fixed-order sum of the partials (per-thread strided sums, then a tree).
__global__ void __launch_bounds__(1024)
    noalloc_finalize(const double *partials, int64_t n_parts, double scale, double *out)
{
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n_parts; i += blockDim.x)
        acc += partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out = red[0] * scale;
}

// Device address of the static scratch on the current device (set up once).
dsp_status scratch_on_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DSP_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DSP_E_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return DSP_OK;
}

}  // namespace

extern "C" dsp_status dsp_density_noalloc(const void *map_dev, int32_t precision, int32_t nx,
                                          int32_t ny, double px_min, double px_max, double py_min,
                                          double py_max, void *cuda_stream, double *n_host)
{
    if (!map_dev || !n_host || nx < 1 || ny < 1)
        return DSP_E_INVALID;
    if (precision != DSP_FP64 && precision != DSP_FP32_MIXED)
        return DSP_E_INVALID;
    if (!(px_min < px_max) || !(py_min < py_max) || !std::isfinite(px_max - px_min) ||
        !std::isfinite(py_max - py_min))
        return DSP_E_INVALID;
    const int64_t n_points = static_cast<int64_t>(nx) * ny;
    if (n_points > DSP_NOALLOC_MAX_POINTS)
        return DSP_E_INVALID;  // more points than the static scratch holds tile sums for
    double *scratch = nullptr;
    dsp_status s = scratch_on_current_device(&scratch);
    if (s != DSP_OK)
        return s;
    const int n_tiles = static_cast<int>((n_points + dsp::kTilePoints - 1) / dsp::kTilePoints);
    const int64_t n_parts = (n_points + dsp::kGranule - 1) / dsp::kGranule;
    const double hx = (px_max - px_min) / nx, hy = (py_max - py_min) / ny;
    const double scale = 4.0 / ((2.0 * 3.14159265358979323846) * (2.0 * 3.14159265358979323846)) *
                         hx * hy;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // a non-sticky error left by the caller's earlier launches is cleared here,
    // so the check after the launches reports this call's own
    (void)cudaGetLastError();
    // Every partial and the result slot are overwritten, so nothing left over
    // from an earlier call is read.
    noalloc_granule_sums<<<n_tiles, kThreads, 0, stream>>>(map_dev, precision, n_points, scratch);
    noalloc_finalize<<<1, 1024, 0, stream>>>(scratch, n_parts, scale, scratch + kStaticMaxParts);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n_host, scratch + kStaticMaxParts, sizeof(double),
                            cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    return e == cudaSuccess ? DSP_OK : DSP_E_CUDA;
}
