#pragma once
// Burgers FWD / TLM / ADJ sweeps (periodic grid, central differences, RK4).
// Templates; instantiated for FP32 in burgers_f32.cu and FP64 in burgers_f64.cu.
//
// Model (Sec. 5.1, periodic reading): f_j(u) = -u_j (u_{j+1}-u_{j-1})/(2dx)
//   + nu (u_{j+1} - 2u_j + u_{j-1})/dx^2, classic RK4 (a21 = a32 = 1/2, a43 = 1,
//   b = 1/6, 1/3, 1/3, 1/6).
// TLM (Sandu's discrete RK tangent-linear model, Sec. 2.1): dk_i = F_i dX_i with
//   F(U) d = -(D1 U) d - U (D1 d) + nu D2 d.
// ADJ (the exact transpose of the TLM step): kappa_i = h b_i lam' + h a_{i+1,i}
//   theta_{i+1}, theta_i = F_i^T kappa_i, lam = lam' + sum theta_i, with
//   F(U)^T w = -(D1 U) w + D1 (U w) + nu D2 w.
// Observations (Eq. Rhalf): at RK step t_i the TLM writes R^{-1/2} O x_{t_i};
//   the ADJ adds O^T R^{-1/2} w_i to lam_{t_i} before stepping back.
//
// GB300 mapping. One column (one direction of the block) belongs to one CTA, or
// to a thread-block cluster of CL CTAs that split the periodic grid into CL
// segments. The whole time loop runs inside the kernel: nothing crosses HBM per
// step except the stored base state x_t (read once per step per column, shared
// through L2 by all columns marching in step). Stage vectors that need
// neighbours live in shared memory with one halo cell on each side; a CTA writes
// its first / last point into its neighbours' halo cells (DSMEM when clustered)
// and one barrier per RK stage publishes them. Thread t owns the points
// t + p*NT (p < P), so shared-memory accesses are conflict-free and global
// accesses coalesced.
#include <cooperative_groups.h>
#include <algorithm>
#include <cstdlib>
#include "common.cuh"
#include "cluster.cuh"
#include "model.cuh"

namespace cg = cooperative_groups;

namespace sc4 {

template <typename T>
struct BurgersParams {
  int n, seg, N, n_o;
  T h, inv2dx, nudx2, inv_sigma;
  const int* obs_of_step;  // [N+1]: observation-time index at that step or -1
  const int* obs_idx;      // [n_t * n_o]
  int fold32;              // write the FP32 trajectory copy folded (x_i, x_{i+n/2})
};

// Position of point j of a row in the folded FP32 layout (pairs x_i, x_{i+n/2}).
__device__ __forceinline__ size_t fold_pos(int j, int n) {
  int H = n >> 1;
  return j < H ? (size_t)(2 * j) : (size_t)(2 * (j - H) + 1);
}

__constant__ double kRkA[3] = {0.5, 0.5, 1.0};  // a21, a32, a43
__constant__ double kRkB[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

template <bool CL>
__device__ __forceinline__ void bar() {
  if constexpr (CL) cg::this_cluster().sync();
  else __syncthreads();
}

// Store v at local point jl of a halo-padded segment array, and into the
// neighbour segments' halo cells when jl is a segment end.
template <bool CL, typename T>
__device__ __forceinline__ void put(T* arr, int jl, int seg, T v, int crank, int csize) {
  arr[jl + 1] = v;
  if (jl == 0) {
    if constexpr (CL) {
      T* r = cg::this_cluster().map_shared_rank(arr, (crank + csize - 1) % csize);
      r[seg + 1] = v;
    } else {
      arr[seg + 1] = v;
    }
  }
  if (jl == seg - 1) {
    if constexpr (CL) {
      T* r = cg::this_cluster().map_shared_rank(arr, (crank + 1) % csize);
      r[0] = v;
    } else {
      arr[0] = v;
    }
  }
}


// f(U) at local index i (halo-padded array)
template <typename T>
__device__ __forceinline__ T rhs_at(const T* U, int i, T inv2dx, T nudx2, T& d1u) {
  T u = U[i], ul = U[i - 1], ur = U[i + 1];
  d1u = (ur - ul) * inv2dx;
  return -u * d1u + nudx2 * (ur - (T)2 * u + ul);
}

// ---------------------------------------------------------------- FWD
// x_{t+1} = RK4(x_t). Stores the trajectory (optional FP32 copy), and at each
// observation step writes O x (obs_out) and/or d = (O x - y)/sigma (d_out).
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(1024) burgers_fwd_kernel(
    BurgersParams<T> pr, const T* __restrict__ x0, T* __restrict__ traj, float* __restrict__ traj32,
    const double* __restrict__ y, double* __restrict__ d_out, double* __restrict__ obs_out,
    T* __restrict__ xN) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, S = seg + 2, NT = blockDim.x;
  T* Ub[2] = {sm, sm + S};
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const int j0 = crank * seg;
  T x[P], acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) x[p] = x0[j0 + threadIdx.x + p * NT];
  for (int t = 0;; ++t) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      int jl = threadIdx.x + p * NT;
      size_t g = (size_t)t * pr.n + j0 + jl;
      if (traj) traj[g] = x[p];
      if (traj32) traj32[(size_t)t * pr.n + (pr.fold32 ? fold_pos(j0 + jl, pr.n) : (size_t)(j0 + jl))] = (float)x[p];
      put<CL>(Ub[0], jl, seg, x[p], crank, csize);
    }
    bar<CL>();
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      for (int o = threadIdx.x; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) {
          double v = (double)Ub[0][gj + 1];
          int r = oi * pr.n_o + o;
          if (obs_out) obs_out[r] = v;
          if (d_out) d_out[r] = (v - y[r]) * (double)pr.inv_sigma;
        }
      }
    }
    if (t == pr.N) break;
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = (T)0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const T* Uc = Ub[s & 1];
      T* Un = Ub[(s + 1) & 1];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        int jl = threadIdx.x + p * NT;
        T d1u;
        T k = rhs_at(Uc, jl + 1, pr.inv2dx, pr.nudx2, d1u);
        acc[p] += (T)kRkB[s] * k;
        if (s < 3) put<CL>(Un, jl, seg, x[p] + pr.h * (T)kRkA[s] * k, crank, csize);
      }
      if (s < 3) bar<CL>();
    }
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] += pr.h * acc[p];
  }
  if (xN) {
#pragma unroll
    for (int p = 0; p < P; ++p) xN[j0 + threadIdx.x + p * NT] = x[p];
  }
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

// ---------------------------------------------------------------- TLM
// W[:, col] = R^{-1/2} O_i dx_{t_i} for all i, dx_0 = U0[:, col].
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(1024) burgers_tlm_kernel(
    BurgersParams<T> pr, const T* __restrict__ traj, const T* __restrict__ U0, int ldu,
    T* __restrict__ W, int ldw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, S = seg + 2, NT = blockDim.x;
  T* Ub[2] = {sm, sm + S};
  T* Db[2] = {sm + 2 * S, sm + 3 * S};
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const int col = blockIdx.x / csize;
  const int j0 = crank * seg;
  const T* u0 = U0 + (size_t)col * ldu;
  T* w = W + (size_t)col * ldw;
  T x[P], dx[P], acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) dx[p] = u0[j0 + threadIdx.x + p * NT];
  for (int t = 0;; ++t) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      int jl = threadIdx.x + p * NT;
      if (t < pr.N) {
        x[p] = traj[(size_t)t * pr.n + j0 + jl];
        put<CL>(Ub[0], jl, seg, x[p], crank, csize);
      }
      put<CL>(Db[0], jl, seg, dx[p], crank, csize);
    }
    bar<CL>();
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      for (int o = threadIdx.x; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) w[oi * pr.n_o + o] = Db[0][gj + 1] * pr.inv_sigma;
      }
    }
    if (t == pr.N) break;
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = (T)0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const T* Uc = Ub[s & 1];
      const T* Dc = Db[s & 1];
      T* Un = Ub[(s + 1) & 1];
      T* Dn = Db[(s + 1) & 1];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        int jl = threadIdx.x + p * NT;
        int i = jl + 1;
        T d1u;
        T k = rhs_at(Uc, i, pr.inv2dx, pr.nudx2, d1u);
        T d = Dc[i], dl = Dc[i - 1], dr = Dc[i + 1];
        T dk = -d1u * d - Uc[i] * (dr - dl) * pr.inv2dx + pr.nudx2 * (dr - (T)2 * d + dl);
        acc[p] += (T)kRkB[s] * dk;
        if (s < 3) {
          T ha = pr.h * (T)kRkA[s];
          put<CL>(Un, jl, seg, x[p] + ha * k, crank, csize);
          put<CL>(Dn, jl, seg, dx[p] + ha * dk, crank, csize);
        }
      }
      if (s < 3) bar<CL>();
    }
#pragma unroll
    for (int p = 0; p < P; ++p) dx[p] += pr.h * acc[p];
  }
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

// ---------------------------------------------------------------- ADJ
// Out[:, col] = lam_0 of the adjoint sweep forced by W[:, col].
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(1024) burgers_adj_kernel(
    BurgersParams<T> pr, const T* __restrict__ traj, const T* __restrict__ Win, int ldw,
    T* __restrict__ Out, int ldo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, S = seg + 2, NT = blockDim.x;
  T* U[4] = {sm, sm + S, sm + 2 * S, sm + 3 * S};
  T* K[2] = {sm + 4 * S, sm + 5 * S};
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const int col = blockIdx.x / csize;
  const int j0 = crank * seg;
  const T* win = Win + (size_t)col * ldw;
  const T h = pr.h;
  T lam[P], x[P], th[P];
#pragma unroll
  for (int p = 0; p < P; ++p) lam[p] = (T)0;
  for (int t = pr.N; t >= 1; --t) {
    bar<CL>();  // every reader of the previous step is done
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
#pragma unroll
      for (int p = 0; p < P; ++p) K[0][threadIdx.x + p * NT + 1] = lam[p];
      __syncthreads();
      for (int o = threadIdx.x; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) atomicAdd(&K[0][gj + 1], win[oi * pr.n_o + o] * pr.inv_sigma);
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < P; ++p) lam[p] = K[0][threadIdx.x + p * NT + 1];
    }
    // base stage states X_1..X_4 of the step t-1 -> t
#pragma unroll
    for (int p = 0; p < P; ++p) {
      int jl = threadIdx.x + p * NT;
      x[p] = traj[(size_t)(t - 1) * pr.n + j0 + jl];
      put<CL>(U[0], jl, seg, x[p], crank, csize);
    }
    bar<CL>();
#pragma unroll
    for (int s = 0; s < 3; ++s) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        int jl = threadIdx.x + p * NT;
        T d1u;
        T k = rhs_at(U[s], jl + 1, pr.inv2dx, pr.nudx2, d1u);
        put<CL>(U[s + 1], jl, seg, x[p] + h * (T)kRkA[s] * k, crank, csize);
        if (s == 2) put<CL>(K[0], jl, seg, h * (T)kRkB[3] * lam[p], crank, csize);
      }
      bar<CL>();
    }
    // adjoint stages 4, 3, 2, 1
#pragma unroll
    for (int p = 0; p < P; ++p) th[p] = (T)0;
#pragma unroll
    for (int s = 3; s >= 0; --s) {
      const T* Us = U[s];
      const T* Kc = K[(3 - s) & 1];
      T* Kn = K[(4 - s) & 1];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        int jl = threadIdx.x + p * NT;
        int i = jl + 1;
        T u = Us[i], ul = Us[i - 1], ur = Us[i + 1];
        T kc = Kc[i], kl = Kc[i - 1], kr = Kc[i + 1];
        T d1u = (ur - ul) * pr.inv2dx;
        T theta = -d1u * kc + (ur * kr - ul * kl) * pr.inv2dx + pr.nudx2 * (kr - (T)2 * kc + kl);
        th[p] += theta;
        if (s > 0) {
          T kn = h * (T)kRkB[s - 1] * lam[p] + h * (T)kRkA[s - 1] * theta;
          put<CL>(Kn, jl, seg, kn, crank, csize);
        }
      }
      if (s > 0) bar<CL>();
    }
#pragma unroll
    for (int p = 0; p < P; ++p) lam[p] += th[p];
  }
  T* out = Out + (size_t)col * ldo;
#pragma unroll
  for (int p = 0; p < P; ++p) out[j0 + threadIdx.x + p * NT] = lam[p];
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

}  // namespace sc4

#include "burgers_v2.cuh"

namespace sc4 {

// ---------------------------------------------------------------- host side
static const size_t kMaxSmem = 227 * 1024;

enum SweepKind { kFwd = 0, kTlm = 1, kAdj = 2 };

// The register-resident (v2) kernels need whole warps of contiguous points.
static bool use_v2(int seg) { return seg >= 256 && seg % 32 == 0; }

static size_t sweep_smem(int kind, int seg, size_t tb) {
  if (use_v2(seg)) {
    size_t S = (size_t)seg + 2 * kPad;
    if (kind == kAdj) return (4 * S + 4 * 32) * tb;
    if (kind == kTlm) return (2 * (size_t)seg + S + 8 * 32) * tb;
    return (S + 4 * 32) * tb;
  }
  int arrays = kind == kAdj ? 6 : (kind == kTlm ? 4 : 2);
  return (size_t)arrays * (seg + 2) * tb;
}

template <typename T>
static BurgersParams<T> make_params(const ModelGeom& g, int seg) {
  BurgersParams<T> pr;
  pr.n = g.n;
  pr.seg = seg;
  pr.N = g.N;
  pr.n_o = g.n_o;
  pr.h = (T)g.h;
  double dx = 1.0 / g.n;
  pr.inv2dx = (T)(1.0 / (2.0 * dx));
  pr.nudx2 = (T)(g.nu / (dx * dx));
  pr.inv_sigma = (T)(1.0 / g.sigma);
  pr.obs_of_step = g.obs_of_step;
  pr.obs_idx = g.obs_idx;
  pr.fold32 = g.fold32;
  return pr;
}

// Points per thread for a segment: NT = seg / P <= 1024 threads. The
// register-resident kernels take more points per thread where the segment is
// long enough (fewer threads, per-thread overhead spread over more points);
// SC4DVAR_SWEEP_P overrides that choice (a tuning knob: 8, 16 or 32).
static int pick_P(int seg) {
  int P = 1;
  while (seg / P > 1024) P *= 2;
  return P;
}

// Largest points per thread of the register-resident kernels: FP32 rows up to
// 32 values (128 B), FP64 rows up to 4 values (32 B; longer FP64 segments are
// split over a cluster instead).
static int max_P_v2(size_t tb) { return tb == 4 ? 32 : 4; }
static int threads_bound(int P, size_t tb) {
  int bytes = P * (int)tb;
  return bytes >= 128 ? 256 : (bytes >= 64 ? 512 : 1024);
}
static bool v2_fits(int seg, size_t tb) {
  return seg / max_P_v2(tb) <= threads_bound(max_P_v2(tb), tb);
}

static int pick_P_v2(int seg, size_t tb) {
  static int forced = [] {
    const char* e = getenv("SC4DVAR_SWEEP_P");
    return e ? atoi(e) : 0;
  }();
  static int forced8 = [] {
    const char* e = getenv("SC4DVAR_SWEEP_P8");
    return e ? atoi(e) : 0;
  }();
  int want = tb == 4 ? (forced > 0 ? std::min(forced, 32) : 16) : (forced8 > 0 ? std::min(forced8, 4) : 4);
  int P = 1;
  while (P < want && seg / (2 * P) >= 256) P *= 2;
  while (seg / P > threads_bound(P, tb) && P < max_P_v2(tb)) P *= 2;
  return P;
}

// Cluster size: the smallest power of two whose per-CTA shared memory fits,
// raised for small blocks (few columns) so that one direction is spread over
// more SMs.
static int pick_cluster(int n, int k, size_t tb, int kind) {
  int cl = 1;
  while ((sweep_smem(kind, n / cl, tb) > kMaxSmem || (use_v2(n / cl) && !v2_fits(n / cl, tb))) &&
         cl < 16)
    cl *= 2;
  if (k <= 4) {
    // few directions: spread each over up to 16 CTAs (non-portable cluster size)
    // while a CTA keeps at least 512 points; SC4DVAR_FEW_CLUSTER8 caps the
    // spread for 8-byte types (a tuning knob: 1, 2, 4, 8 or 16)
    static int cap8 = [] {
      const char* e = getenv("SC4DVAR_FEW_CLUSTER8");
      int c = e ? atoi(e) : 16;
      return (c == 1 || c == 2 || c == 4 || c == 8) ? c : 16;
    }();
    const int cap = tb == 8 ? cap8 : 16;
    while (cl < cap && n / (cl * 2) >= 512) cl *= 2;
  }
  return cl;
}

template <typename Kern, typename... Args>
static int launch(Kern kern, int grid, int threads, size_t smem, int cl, cudaStream_t st,
                  Args... args) {
  SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cl > 1) {
    if (cl > 8) SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  SC4_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
  note_launch();
  return SC4DVAR_OK;
}

// The strided kernels only run on segments below 256 points (one point per
// thread); the register-resident ones take 1..32 (FP32) or 1..4 (FP64) points.
#define SC4_DISPATCH_V1(P, BODY)                                        \
  switch (P) {                                                          \
    case 1: { constexpr int PP = 1; BODY; } break;                      \
    default: set_error("unsupported points per thread"); return SC4DVAR_ERR_INVALID_ARG; \
  }

#define SC4_DISPATCH_V2(T, P, BODY)                                     \
  switch (P) {                                                          \
    case 1: { constexpr int PP = 1; BODY; } break;                      \
    case 2: { constexpr int PP = 2; BODY; } break;                      \
    case 4: { constexpr int PP = 4; BODY; } break;                      \
    case 8: { if constexpr (sizeof(T) == 4) { constexpr int PP = 8; BODY; } } break;   \
    case 16: { if constexpr (sizeof(T) == 4) { constexpr int PP = 16; BODY; } } break; \
    case 32: { if constexpr (sizeof(T) == 4) { constexpr int PP = 32; BODY; } } break; \
    default: set_error("unsupported points per thread"); return SC4DVAR_ERR_INVALID_ARG; \
  }

template <typename T>
int burgers_fwd(const ModelGeom& g, const T* x0, T* traj, float* traj32, const double* y,
                double* d_out, double* obs_out, T* xN, cudaStream_t st) {
  int cl = pick_cluster(g.n, 1, sizeof(T), kFwd);
  int seg = g.n / cl, P = use_v2(seg) ? pick_P_v2(seg, sizeof(T)) : pick_P(seg), NT = seg / P;
  size_t smem = sweep_smem(kFwd, seg, sizeof(T));
  auto pr = make_params<T>(g, seg);
  if (use_v2(seg)) {
    if (cl > 1) {
      SC4_DISPATCH_V2(T, P, SC4_TRY(launch(burgers_fwd_v2_kernel<T, PP, true>, cl, NT, smem, cl, st, pr,
                                       x0, traj, traj32, y, d_out, obs_out, xN)));
    } else {
      SC4_DISPATCH_V2(T, P, SC4_TRY(launch(burgers_fwd_v2_kernel<T, PP, false>, 1, NT, smem, 1, st, pr,
                                       x0, traj, traj32, y, d_out, obs_out, xN)));
    }
    return SC4DVAR_OK;
  }
  if (cl > 1) {
    SC4_DISPATCH_V1(P, SC4_TRY(launch(burgers_fwd_kernel<T, PP, true>, cl, NT, smem, cl, st, pr, x0,
                                     traj, traj32, y, d_out, obs_out, xN)));
  } else {
    SC4_DISPATCH_V1(P, SC4_TRY(launch(burgers_fwd_kernel<T, PP, false>, 1, NT, smem, 1, st, pr, x0,
                                     traj, traj32, y, d_out, obs_out, xN)));
  }
  return SC4DVAR_OK;
}

template <typename T>
int burgers_tlm(const ModelGeom& g, const T* traj, const T* U0, int ldu, int k, T* W, int ldw,
                cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  if constexpr (sizeof(T) == 4) {
    if (g.fold32) return burgers_tlm_f32x2(g, traj, U0, ldu, k, W, ldw, st);
  }
  int cl = pick_cluster(g.n, k, sizeof(T), kTlm);
  int seg = g.n / cl, P = use_v2(seg) ? pick_P_v2(seg, sizeof(T)) : pick_P(seg), NT = seg / P;
  size_t smem = sweep_smem(kTlm, seg, sizeof(T));
  auto pr = make_params<T>(g, seg);
  if (use_v2(seg)) {
    if (cl > 1) {
      SC4_DISPATCH_V2(T, P, SC4_TRY(launch(burgers_tlm_v2_kernel<T, PP, true>, k * cl, NT, smem, cl, st,
                                       pr, traj, U0, ldu, W, ldw)));
    } else {
      SC4_DISPATCH_V2(T, P, SC4_TRY(launch(burgers_tlm_v2_kernel<T, PP, false>, k, NT, smem, 1, st, pr,
                                       traj, U0, ldu, W, ldw)));
    }
    return SC4DVAR_OK;
  }
  if (cl > 1) {
    SC4_DISPATCH_V1(P, SC4_TRY(launch(burgers_tlm_kernel<T, PP, true>, k * cl, NT, smem, cl, st, pr,
                                     traj, U0, ldu, W, ldw)));
  } else {
    SC4_DISPATCH_V1(P, SC4_TRY(launch(burgers_tlm_kernel<T, PP, false>, k, NT, smem, 1, st, pr, traj,
                                     U0, ldu, W, ldw)));
  }
  return SC4DVAR_OK;
}

template <typename T>
int burgers_adj(const ModelGeom& g, const T* traj, const T* W, int ldw, int k, T* Out, int ldo,
                cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  if constexpr (sizeof(T) == 4) {
    if (g.fold32) return burgers_adj_f32x2(g, traj, W, ldw, k, Out, ldo, st);
  }
  int cl = pick_cluster(g.n, k, sizeof(T), kAdj);
  int seg = g.n / cl, P = use_v2(seg) ? pick_P_v2(seg, sizeof(T)) : pick_P(seg), NT = seg / P;
  size_t smem = sweep_smem(kAdj, seg, sizeof(T));
  auto pr = make_params<T>(g, seg);
  if (use_v2(seg)) {
    if (cl > 1) {
      SC4_DISPATCH_V2(T, P, SC4_TRY(launch(burgers_adj_v2_kernel<T, PP, true>, k * cl, NT, smem, cl, st,
                                       pr, traj, W, ldw, Out, ldo)));
    } else {
      SC4_DISPATCH_V2(T, P, SC4_TRY(launch(burgers_adj_v2_kernel<T, PP, false>, k, NT, smem, 1, st, pr,
                                       traj, W, ldw, Out, ldo)));
    }
    return SC4DVAR_OK;
  }
  if (cl > 1) {
    SC4_DISPATCH_V1(P, SC4_TRY(launch(burgers_adj_kernel<T, PP, true>, k * cl, NT, smem, cl, st, pr,
                                     traj, W, ldw, Out, ldo)));
  } else {
    SC4_DISPATCH_V1(P, SC4_TRY(launch(burgers_adj_kernel<T, PP, false>, k, NT, smem, 1, st, pr, traj,
                                     W, ldw, Out, ldo)));
  }
  return SC4DVAR_OK;
}


}  // namespace sc4
