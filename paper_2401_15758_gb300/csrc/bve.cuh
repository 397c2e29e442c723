#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace sc4 {

// Geometry and device tables of a barotropic vorticity problem.
struct BveGeom {
  int N;                     // grid points per side (power of two)
  int Nsteps;                // RK4 steps
  int n_t, n_o;
  double h, nu, sigma, famp, prior_c, prior_ell;
  int fk;
  const int* obs_of_step_h;  // host [Nsteps+1]
  const int* obs_idx;        // device [n_t * n_o]
  double2* tw64;             // device [N/2] twiddles
  float2* tw32;
  double* poisson;           // device [N*N] symbol -1/|kappa|^2
  double* prior;             // device [N*N] symbol of Gamma^{1/2}
  // column-pass copies of both symbols (both wavenumbers bit-reversed), FP64 / FP32
  double* poisson_c64;
  float* poisson_c32;
  double* prior_c64;
  float* prior_c32;
  // Stored stage states q_s(t), psi_s(t) at row 4 t + s. With checkpointing
  // (ckpt_every = L > 0) they hold one segment of L steps at row 4 (t - t0) + s,
  // recomputed from the FP64 checkpoint of the segment by every sweep.
  double* q64;
  double* p64;
  float* q32;
  float* p32;
  int ckpt_every;            // L: steps per checkpoint segment, 0 = store every stage state
  double* ckpt;              // device [ceil(Nsteps / L) * N*N] FP64 states at steps 0, L, 2L, ...
  void* rws;                 // device recompute workspace (bve_fwd_ws_bytes)
};

int bve_setup(BveGeom& g, cudaStream_t st);
template <typename R, typename RI, typename RO, typename RZ>
int fft2_apply(const BveGeom& g, int k, const RI* X, int ldx, RO* Y, int ldy, const RZ* Z, int ldz,
               const double* table, void* cbuf, cudaStream_t st);
int bve_fwd(const BveGeom& g, const double* x0, bool store, const double* y, double* d_out,
            double* obs_out, double* xN, void* ws, cudaStream_t st);
template <typename T>
int bve_tlm(const BveGeom& g, const T* U0, int ldu, int k, T* W, int ldw, void* ws, cudaStream_t st);
template <typename T>
int bve_adj(const BveGeom& g, const T* W, int ldw, int k, T* Out, int ldo, void* ws, cudaStream_t st);
size_t bve_sweep_ws_bytes(const BveGeom& g, int k, size_t tb);
size_t bve_fwd_ws_bytes(const BveGeom& g);

}  // namespace sc4
