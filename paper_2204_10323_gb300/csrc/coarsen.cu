// coarsen.cu -- block average of a cell field, the coarsening by which the
// paper builds its 2, 4 and 8 m grids from the 1 m DEM (Methods, "Data").
//
// Output cell (J, I) is the mean of the input cells (j, i) with
// j in [J f, min((J + 1) f, ny)) and i in [I f, min((I + 1) f, nx)): an exact
// f x f block mean where f divides the grid, the mean of the cells present in
// the partial blocks along the far (x = nx, y = ny) edges otherwise.  Sums
// are taken in double and rounded once to the field's precision.
#include <cuda_runtime.h>

#include "flood_internal.h"

namespace flood {

namespace {

template <typename T>
__global__ void coarsen_kernel(const T *src, int nx, int ny, int f, T *dst, int mx, int my)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= mx) return;
    const int i0 = I * f, i1 = min(i0 + f, nx);
    for (int J = blockIdx.y; J < my; J += gridDim.y) {
        const int j0 = J * f, j1 = min(j0 + f, ny);
        double s = 0.0;
        for (int j = j0; j < j1; j++) {
            const T *row = src + (size_t)j * nx;
            for (int i = i0; i < i1; i++) s += (double)row[i];
        }
        dst[(size_t)J * mx + I] = (T)(s / (double)((j1 - j0) * (i1 - i0)));
    }
}

}  // namespace

template <typename T>
cudaError_t launch_coarsen(const T *src, int nx, int ny, int f, T *dst, cudaStream_t st)
{
    const int mx = (nx + f - 1) / f, my = (ny + f - 1) / f;
    dim3 grid((mx + 127) / 128, my < 65535 ? my : 65535);
    coarsen_kernel<T><<<grid, 128, 0, st>>>(src, nx, ny, f, dst, mx, my);
    return cudaGetLastError();
}

template cudaError_t launch_coarsen<float>(const float *, int, int, int, float *, cudaStream_t);
template cudaError_t launch_coarsen<double>(const double *, int, int, int, double *, cudaStream_t);

}  // namespace flood
