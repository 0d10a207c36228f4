// noalloc.cu -- stored water volume sum(h) dx^2 of a caller-owned depth array,
// computed without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need
// this number: code running inside a CUDA-graph capture region (where
// cudaMalloc is not allowed), callers that hand all device memory to their
// own allocator or pool, and embedded or real-time hosts that forbid
// allocation after start-up.  For them this entry point keeps its scratch (one
// partial sum per grid row) in a fixed, file-scope device array instead of
// memory from cudaMalloc or the PyTorch caching allocator.
//
// Limits and sharing: the scratch holds kMaxRows = 65536 row sums (512 KiB),
// so grids with more than 65536 rows are rejected with FLOOD_ERR_ARG.  Every
// GPU that loads the library holds that array until the process exits.  All
// calls on a device share the one array and it keeps the last call's row
// sums; each call overwrites every entry it reads, so nothing needs clearing,
// but two calls whose kernels overlap on the GPU (different streams, or host
// threads without ordering) race on it.
//
// Set-up: host code cannot use the array's name as a device address, so the
// first call on each device (with that device current) looks the address up
// with cudaGetSymbolAddress and caches it.  Make that first call outside any
// stream capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "device_common.cuh"
#include "flood.h"
#include "flood_runtime.h"

namespace flood {

namespace {

constexpr int kMaxRows = 65536;
constexpr int kMaxDevices = 64;
constexpr int kRowThreads = 256;

__device__ __align__(256) double g_row_sums[kMaxRows];

double *g_scratch[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Row j's sum into rows[j] (fixed reduction order for a fixed launch shape).
template <typename T>
__global__ void row_sums_kernel(const T *h, int nx, int ny, long long pitch, double *rows)
{
    __shared__ double red[32];
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) s += (double)h[(size_t)j * pitch + i];
        s = block_reduce<false>(s, red);
        if (threadIdx.x == 0) rows[j] = s;
        __syncthreads();
    }
}

__global__ void rows_total_kernel(const double *rows, int ny, double area, double *out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) s += rows[j];
    s = block_reduce<false>(s, red);
    if (threadIdx.x == 0) *out = s * area;
}

}  // namespace

}  // namespace flood

using namespace flood;

extern "C" flood_status flood_volume_noalloc(const void *depth, int32_t nx, int32_t ny, int64_t row_pitch,
                                             int32_t precision, double dx, double *out_device, void *stream)
{
    if (!depth || !out_device) return fail(nullptr, FLOOD_ERR_ARG, "flood_volume_noalloc: NULL pointer");
    if (nx < 1 || ny < 1 || row_pitch < nx) return fail(nullptr, FLOOD_ERR_ARG, "flood_volume_noalloc: bad sizes");
    if (ny > kMaxRows)
        return fail(nullptr, FLOOD_ERR_ARG,
                    "flood_volume_noalloc: ny = " + std::to_string(ny) + " exceeds the fixed scratch of " +
                        std::to_string(kMaxRows) + " rows");
    if (precision != FLOOD_F32 && precision != FLOOD_F64)
        return fail(nullptr, FLOOD_ERR_ARG, "flood_volume_noalloc: bad precision");
    if (!(dx > 0.0)) return fail(nullptr, FLOOD_ERR_ARG, "flood_volume_noalloc: dx must be > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, FLOOD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, FLOOD_ERR_UNSUPPORTED, "flood_volume_noalloc: device index");
    double *rows = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_row_sums);
            if (e != cudaSuccess)
                return fail(nullptr, FLOOD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch[dev] = (double *)p;
        }
        rows = g_scratch[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int blocks = ny < 152 * 8 ? ny : 152 * 8;
    if (precision == FLOOD_F32)
        row_sums_kernel<float><<<blocks, kRowThreads, 0, st>>>((const float *)depth, nx, ny, (long long)row_pitch, rows);
    else
        row_sums_kernel<double><<<blocks, kRowThreads, 0, st>>>((const double *)depth, nx, ny, (long long)row_pitch, rows);
    rows_total_kernel<<<1, 1024, 0, st>>>(rows, ny, dx * dx, out_device);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, FLOOD_ERR_CUDA, std::string("flood_volume_noalloc launch: ") + cudaGetErrorString(e));
    return FLOOD_OK;
}
