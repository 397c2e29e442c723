// Dirichlet-boundary Burgers (the Burgers set-up of Sec. 5.1): geometry and the
// host entry points of burgers_dirichlet.cu.
#pragma once
#include <cuda_runtime.h>

namespace sc4 {

struct DirGeom {
  int n;                   // interior points (<= 1024), dx = 1/(n+1)
  int N;                   // RK steps
  int S;                   // RK stages (3: RK3-TVD, 4: classic RK4)
  int n_o;                 // sites per observation time
  double h, nu, sigma;
  double a[4][4], b[4];    // Butcher tableau
  const int* obs_of_step;  // device [N+1]
  const int* obs_idx;      // device [n_t * n_o]
  // prior (a I - b Delta*)^{-1}: elimination of the constant tridiagonal matrix
  double bcoef;
  double* cp;              // device [n] c'_i
  double* den;             // device [n] pivots
  double* work;            // device [n * work_cols] FP64 work columns
  int work_cols;
};

int dir_setup(DirGeom& g, double a, double b, cudaStream_t st);
int dir_fwd(const DirGeom& g, const double* x0, double* traj, float* traj32, const double* y, double* d_out,
            double* obs_out, double* xN, cudaStream_t st);
template <typename T>
int dir_tlm(const DirGeom& g, const T* traj, const T* U0, int ldu, int k, T* W, int ldw, cudaStream_t st);
template <typename T>
int dir_adj(const DirGeom& g, const T* traj, const T* W, int ldw, int k, T* Out, int ldo, cudaStream_t st);
template <typename TI, typename TO, typename TZ>
int dir_prior_apply(const DirGeom& g, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz,
                    cudaStream_t st);

}  // namespace sc4
