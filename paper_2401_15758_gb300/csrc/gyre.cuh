// Wind-driven barotropic vorticity in a closed basin (the double-gyre set-up of
// Sec. 5.2): geometry and the host entry points of gyre.cu.
//
//   omega_t = -J(psi, omega) + Ro^{-1} psi_x + Re^{-1} Lap omega + Ro^{-1} sin(pi y),
//   Lap psi = -omega,  psi = omega = 0 on the boundary of (0, 1) x (-1, 1),
//
// second-order central differences on nx x ny interior points (h = 1/(nx+1),
// ny = 2 nx + 1), fields row-major (y slow). Elliptic solves (the Poisson solve
// of every RK stage and the prior (a I - b Delta*)^{-1}) diagonalise the x
// direction with the orthonormal sine transform S (S_ip = sqrt(2/(nx+1))
// sin(pi i p/(nx+1)), S = S^T = S^{-1}) and solve one tridiagonal system along y
// per x-mode p: (alpha + beta (mu_p + 2)) on the diagonal, -beta off it,
// mu_p = 4 sin^2(pi p / (2 (nx+1))).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

namespace sc4 {

struct GyreGeom {
  int nx, ny, n;               // interior grid (nx a power of two in [8, 128]), n = nx ny
  int N, S, n_t, n_o;          // RK steps, stages, observation times and sites
  double dt, h, re_inv, ro_inv, sigma;
  double a[4][4], b[4];        // Butcher tableau
  const int* obs_of_step;      // device [N+1]: observation time of a step or -1
  const int* obs_of_step_h;    // host copy
  const int* obs_idx;          // device [n_t * n_o]
  // transform and tridiagonal factors (device): S [nx*nx]; per factor set
  // [2][ny][nx]: inverse pivots, then c'_j = off * pivot^{-1}
  double* S64;
  float* S32;
  void* S_tc;                  // nx = 128: S packed for the tensor-core row transform (else null)
  double* pois64;
  float* pois32;
  double pois_off;             // off-diagonal of the Poisson systems (-1/h^2)
  double* prior64;
  float* prior32;
  double prior_off;            // off-diagonal of the prior systems (-b)
  double* Fy;                  // device [ny] sin(pi y_j)
  // FWD stage states [N * S][n]: omega_s(t) and psi_s(t), FP64 and FP32 copies
  double* om64;
  double* ps64;
  float* om32;
  float* ps32;
};

// Device bytes of the set-up arrays (transform, factors, forcing) and of the
// stage states.
size_t gyre_setup_bytes(int nx);
// offset of the packed transform (S_tc) in the set-up block (nx = 128)
size_t gyre_tc_offset(int nx);
size_t gyre_stage_bytes(int nx, int N, int S);
// Fills S, the factors and the forcing; the pointers must already be set.
int gyre_setup(GyreGeom& g, double prior_a, double prior_b, cudaStream_t st);

// Work bytes of a TLM or ADJ sweep of k columns in element size tb (also covers
// the FWD with k = 1, tb = 8) and of a prior apply.
size_t gyre_sweep_ws_bytes(const GyreGeom& g, int k, size_t tb);
size_t gyre_prior_ws_bytes(const GyreGeom& g, int k, size_t tb);

// FWD from x0 (FP64). store: keep the stage states; y/d_out: innovations
// d = (O x - y)/sigma at the observation steps; obs_out: O x; xN: final state.
int gyre_fwd(const GyreGeom& g, const double* x0, bool store, const double* y, double* d_out,
             double* obs_out, double* xN, void* ws, cudaStream_t st);
template <typename T>
int gyre_tlm(const GyreGeom& g, const T* U0, int ldu, int k, T* W, int ldw, void* ws, cudaStream_t st);
template <typename T>
int gyre_adj(const GyreGeom& g, const T* W, int ldw, int k, T* Out, int ldo, void* ws, cudaStream_t st);
// Y = (a I - b Delta*)^{-1} X (+ Z), arithmetic in FP32 when X and Y are FP32,
// else FP64.
template <typename TI, typename TO, typename TZ>
int gyre_prior_apply(const GyreGeom& g, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz,
                     void* ws, cudaStream_t st);

}  // namespace sc4
