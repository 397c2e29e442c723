// Double-float instantiations of the Burgers sweeps (burgers_impl.cuh with
// T = dfloat): FP64-class accuracy from FP32-pipe arithmetic, used for the
// defect-correction residuals of PCG and for SC4DVAR_DF64 block products.
#include "dfloat.cuh"
#include "burgers_impl.cuh"

namespace sc4 {
template int burgers_tlm<dfloat>(const ModelGeom&, const dfloat*, const dfloat*, int, int, dfloat*, int,
                                 cudaStream_t);
template int burgers_adj<dfloat>(const ModelGeom&, const dfloat*, const dfloat*, int, int, dfloat*, int,
                                 cudaStream_t);

namespace {
__global__ void d2df_kernel(int rows, int cols, const double* __restrict__ x, int ldx, dfloat* y, int ldy) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    y[(size_t)c * ldy + i] = dfloat(x[(size_t)c * ldx + i]);
  }
}
__global__ void df2d_kernel(int rows, int cols, const dfloat* __restrict__ x, int ldx, double* y, int ldy) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    y[(size_t)c * ldy + i] = (double)x[(size_t)c * ldx + i];
  }
}
int grid_for(size_t total) { return (int)std::min<size_t>((total + 255) / 256, 8 * 152); }
}  // namespace

int to_dfloat(int rows, int cols, const double* x, int ldx, dfloat* y, int ldy, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SC4DVAR_OK;
  d2df_kernel<<<grid_for((size_t)rows * cols), 256, 0, st>>>(rows, cols, x, ldx, y, ldy);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}
int from_dfloat(int rows, int cols, const dfloat* x, int ldx, double* y, int ldy, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return SC4DVAR_OK;
  df2d_kernel<<<grid_for((size_t)rows * cols), 256, 0, st>>>(rows, cols, x, ldx, y, ldy);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}
}  // namespace sc4
