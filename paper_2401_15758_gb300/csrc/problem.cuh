// Handle layouts shared by the C ABI sources (api.cu, noalloc.cu).
#pragma once
#include <cuda_runtime.h>
#include <string>
#include "common.cuh"
#include "model.cuh"
#include "bve.cuh"
#include "dirichlet.cuh"
#include "gyre.cuh"
#include <vector>

namespace sc4 {

// Growable device buffer (freed explicitly by its owner).
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t b) {
    if (b <= bytes) return SC4DVAR_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of " + std::to_string(b) + " bytes failed");
      return SC4DVAR_ERR_OOM;
    }
    bytes = b;
    return SC4DVAR_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

enum CountMode { kOnline = 0, kOffline = 1, kKappa = 2 };

}  // namespace sc4

struct sc4dvar_problem_s {
  int model = 0, n = 0, N = 0, n_t = 0, n_o = 0, m = 0;
  double nu = 0, h = 0, sigma = 1;
  sc4::ModelGeom geom;
  int* obs_of_step = nullptr;
  int* obs_idx = nullptr;
  double* sym = nullptr;
  double2* tw = nullptr;
  double *xb = nullptr, *y = nullptr, *v = nullptr, *x0 = nullptr, *d = nullptr;
  double* traj64 = nullptr;
  float* traj32 = nullptr;
  void* traj_df = nullptr;     // double-float copy of traj64 (periodic Burgers, on demand)
  bool traj_df_valid = false;  // the copy matches the current trajectory
  sc4::Buf wDF;                // double-float work blocks of the DF64 products
  bool have_traj = false;
  // barotropic vorticity problems: geometry, tables and stored stage states
  sc4::BveGeom bve{};
  std::vector<int> obs_of_step_h;
  double2* bve_tw64 = nullptr;
  float2* bve_tw32 = nullptr;
  double *bve_poisson = nullptr, *bve_prior = nullptr;
  double* bve_tabc64 = nullptr;
  float* bve_tabc32 = nullptr;
  double *bve_q64 = nullptr, *bve_p64 = nullptr;
  float *bve_q32 = nullptr, *bve_p32 = nullptr;
  // Dirichlet Burgers problems: geometry, prior elimination tables, prior work columns
  sc4::DirGeom dir{};
  double* dir_cp = nullptr;
  sc4::Buf wDir;
  // double-gyre vorticity problems: geometry, set-up arrays, stage states, work
  sc4::GyreGeom gy{};
  void* gy_setup = nullptr;
  void* gy_stages = nullptr;
  sc4::Buf wGy, wGyPrior;
  double* bve_ckpt = nullptr;  // checkpoint states (checkpointing only)
  void* bve_rws = nullptr;     // segment recompute workspace (checkpointing only)
  sc4::Buf wBve, wCplx;
  // scratch: block operator work arrays, reductions, small host-visible scalars
  sc4::Buf wU, wW, wL, part, scal, vec;
  int count_mode = sc4::kOnline;
  sc4dvar_counters_t counters{};
  // single-vector Hessian products recorded as CUDA graphs (vorticity problems):
  // key (p, q, precision) plus the work-array addresses the recording used
  struct HvpGraph {
    const double* p;
    double* q;
    int prec;
    void* bufs[7];
    cudaGraphExec_t exec;
    bool eager_only;
  };
  std::vector<HvpGraph> hvp_graphs;
  cudaStream_t graph_stream = nullptr;
};

struct sc4dvar_precond_s {
  int n = 0, l = 0;
  double* V = nullptr;    // n x l
  double* lam = nullptr;  // l
  double* dsc = nullptr;  // lam / (1 + lam)
  sc4::Buf T;             // l x k workspace
};

