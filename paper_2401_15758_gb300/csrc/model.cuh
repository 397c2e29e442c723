#pragma once
#include <cuda_runtime.h>

namespace sc4 {

// Geometry of the assimilation window shared by the model sweeps.
struct ModelGeom {
  int n;                    // state size
  int N;                    // RK steps
  double h;                 // RK step
  double nu;                // viscosity
  double sigma;             // observation standard deviation (R = sigma^2 I)
  int n_t, n_o;             // observation times, sites per time
  const int* obs_of_step;   // device [N+1]: observation index at step t, or -1
  const int* obs_idx;       // device [n_t * n_o]
  int fold32 = 0;           // FP32 trajectory copy stored folded (pairs x_i, x_{i+n/2})
  int pairs_tuned = 0;      // packed FP32 sweeps: pairs per thread chosen by sc4dvar_autotune (0: default)
};

// FP32 sweeps on grids of at least this many points use packed FP32x2 kernels
// over the folded trajectory copy.
constexpr int kPackedMinN = 1024;
bool packed_f32_supported(int n);
int burgers_tlm_f32x2(const ModelGeom& m, const float* traj_folded, const float* U0, int ldu, int k,
                      float* W, int ldw, cudaStream_t st);
int burgers_adj_f32x2(const ModelGeom& m, const float* traj_folded, const float* Win, int ldw, int k,
                      float* Out, int ldo, cudaStream_t st);

template <typename T>
int burgers_fwd(const ModelGeom& g, const T* x0, T* traj, float* traj32, const double* y,
                double* d_out, double* obs_out, T* xN, cudaStream_t st);
template <typename T>
int burgers_tlm(const ModelGeom& g, const T* traj, const T* U0, int ldu, int k, T* W, int ldw,
                cudaStream_t st);
struct dfloat;
// column-major block conversions between double and double-float
int to_dfloat(int rows, int cols, const double* x, int ldx, dfloat* y, int ldy, cudaStream_t st);
int from_dfloat(int rows, int cols, const dfloat* x, int ldx, double* y, int ldy, cudaStream_t st);
template <typename T>
int burgers_adj(const ModelGeom& g, const T* traj, const T* W, int ldw, int k, T* Out, int ldo,
                cudaStream_t st);

}  // namespace sc4
