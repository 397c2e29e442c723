// Viscous Burgers with homogeneous Dirichlet boundaries (the Burgers set-up of
// Sec. 5.1): u_t + u u_x = nu u_xx on (0, 1), u(0) = u(1) = 0, central
// differences on n interior points x_j = j dx, dx = 1/(n+1), an explicit
// Runge-Kutta method given by its tableau (classic RK4 or the third-order
// TVD scheme RK3 the paper's experiments use), its tangent-linear model and its
// discrete adjoint (the same construction as the periodic sweeps):
//   TLM  dX_i = dx + h sum_{j<i} a_ij dk_j,  dk_i = F_i dX_i,  dx' = dx + h sum b_i dk_i
//   ADJ  kappa_i = h b_i lam' + h sum_{j>i} a_ji theta_j,  theta_i = F_i^T kappa_i,
//        lam = lam' + sum theta_i
// with F(u) d = -(d D1u + u D1d) + nu D2 d and, D1 being skew and D2 symmetric
// under zero boundary values, F(u)^T w = -(D1u) w + D1(u w) + nu D2 w.
//
// Grids of up to 1024 points: one CTA per direction, one point per thread, the
// whole window inside one launch; neighbour values travel through a
// zero-padded shared row (index 0 and n+1 hold the boundary values).
// The prior Gamma^{1/2} = (a I - b Delta*)^{-1}, Delta* = tridiag(1, -2, 1), is
// applied per column by the Thomas algorithm with a precomputed elimination.
#include <vector>
#include "common.cuh"
#include "dirichlet.cuh"

namespace sc4 {
namespace {

template <typename T>
struct DirParams {
  int n, N, n_o, S;
  T h, c1, c2, inv_sigma;  // c1 = 1/(2 dx), c2 = nu / dx^2
  T a[4][4], b[4];
  const int* obs_of_step;
  const int* obs_idx;
};

template <typename T>
DirParams<T> make_params(const DirGeom& g) {
  DirParams<T> p{};
  p.n = g.n;
  p.N = g.N;
  p.n_o = g.n_o;
  p.S = g.S;
  p.h = (T)g.h;
  const double dx = 1.0 / (g.n + 1);
  p.c1 = (T)(1.0 / (2.0 * dx));
  p.c2 = (T)(g.nu / (dx * dx));
  p.inv_sigma = (T)(1.0 / g.sigma);
  for (int i = 0; i < 4; ++i) {
    p.b[i] = (T)g.b[i];
    for (int j = 0; j < 4; ++j) p.a[i][j] = (T)g.a[i][j];
  }
  p.obs_of_step = g.obs_of_step;
  p.obs_idx = g.obs_idx;
  return p;
}

// row arrays hold n + 2 values: [0] and [n+1] are the zero boundary values
template <typename T>
__device__ __forceinline__ T rhs_at(const T* u, int j, T c1, T c2) {
  const T ul = u[j - 1], uc = u[j], ur = u[j + 1];
  return -uc * ((ur - ul) * c1) + c2 * (ur - (T)2 * uc + ul);
}
template <typename T>
__device__ __forceinline__ T jvp_at(const T* u, const T* d, int j, T c1, T c2) {
  const T dl = d[j - 1], dc = d[j], dr = d[j + 1];
  return -(dc * ((u[j + 1] - u[j - 1]) * c1) + u[j] * ((dr - dl) * c1)) + c2 * (dr - (T)2 * dc + dl);
}
template <typename T>
__device__ __forceinline__ T vjp_at(const T* u, const T* w, int j, T c1, T c2) {
  const T wl = w[j - 1], wc = w[j], wr = w[j + 1];
  return -((u[j + 1] - u[j - 1]) * c1) * wc + (u[j + 1] * wr - u[j - 1] * wl) * c1 +
         c2 * (wr - (T)2 * wc + wl);
}

template <typename T>
__device__ __forceinline__ void zero_ends(T* row, int n) {
  if (threadIdx.x == 0) {
    row[0] = (T)0;
    row[n + 1] = (T)0;
  }
}

// FWD from x0 (FP64 arithmetic for T = double); trajectory rows x_t (optional
// FP32 copy), observation outputs d = (O x - y)/sigma and/or O x, final state.
template <typename T>
__global__ void __launch_bounds__(1024) dir_fwd_kernel(DirParams<T> p, const T* __restrict__ x0, T* traj,
                                                      float* traj32, const double* __restrict__ y,
                                                      double* d_out, double* obs_out, T* xN) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* u = reinterpret_cast<T*>(smraw);  // [n + 2]
  const int j = threadIdx.x, n = p.n;
  const bool act = j < n;
  zero_ends(u, n);
  T x = act ? x0[j] : (T)0;
  T k[4];
  for (int t = 0;; ++t) {
    if (act) {
      if (traj) traj[(size_t)t * n + j] = x;
      if (traj32) traj32[(size_t)t * n + j] = (float)x;
      u[j + 1] = x;
    }
    __syncthreads();
    const int oi = p.obs_of_step[t];
    if (oi >= 0 && (d_out || obs_out)) {
      for (int o = j; o < p.n_o; o += blockDim.x) {
        const int r = oi * p.n_o + o;
        const double v = (double)u[p.obs_idx[r] + 1];
        if (obs_out) obs_out[r] = v;
        if (d_out) d_out[r] = (v - y[r]) * (double)p.inv_sigma;
      }
    }
    if (t == p.N) break;
    for (int s = 0; s < p.S; ++s) {
      T Xs = x;
      for (int q = 0; q < s; ++q) Xs += p.h * p.a[s][q] * k[q];
      __syncthreads();
      if (act) u[j + 1] = Xs;
      __syncthreads();
      k[s] = act ? rhs_at(u, j + 1, p.c1, p.c2) : (T)0;
    }
    T acc = (T)0;
    for (int s = 0; s < p.S; ++s) acc += p.b[s] * k[s];
    x += p.h * acc;
    __syncthreads();
  }
  if (xN && act) xN[j] = x;
}

// TLM of one direction per CTA: W[:, col] = R^{-1/2} O_i dx_{t_i}.
template <typename T>
__global__ void __launch_bounds__(1024) dir_tlm_kernel(DirParams<T> p, const T* __restrict__ traj,
                                                      const T* __restrict__ U0, int ldu, T* W, int ldw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* u = reinterpret_cast<T*>(smraw);  // base stage state [n + 2]
  T* d = u + p.n + 2;                   // direction stage state [n + 2]
  const int j = threadIdx.x, n = p.n, col = blockIdx.x;
  const bool act = j < n;
  zero_ends(u, n);
  zero_ends(d, n);
  T dx = act ? U0[(size_t)col * ldu + j] : (T)0;
  T k[4], dk[4];
  for (int t = 0;; ++t) {
    const int oi = p.obs_of_step[t];
    if (oi >= 0) {
      if (act) d[j + 1] = dx;
      __syncthreads();
      for (int o = j; o < p.n_o; o += blockDim.x) {
        const int r = oi * p.n_o + o;
        W[(size_t)col * ldw + r] = d[p.obs_idx[r] + 1] * p.inv_sigma;
      }
    }
    if (t == p.N) break;
    const T x = act ? traj[(size_t)t * n + j] : (T)0;
    for (int s = 0; s < p.S; ++s) {
      T Xs = x, Ds = dx;
      for (int q = 0; q < s; ++q) {
        Xs += p.h * p.a[s][q] * k[q];
        Ds += p.h * p.a[s][q] * dk[q];
      }
      __syncthreads();
      if (act) {
        u[j + 1] = Xs;
        d[j + 1] = Ds;
      }
      __syncthreads();
      if (act) {
        k[s] = rhs_at(u, j + 1, p.c1, p.c2);
        dk[s] = jvp_at(u, d, j + 1, p.c1, p.c2);
      } else {
        k[s] = dk[s] = (T)0;
      }
    }
    T acc = (T)0;
    for (int s = 0; s < p.S; ++s) acc += p.b[s] * dk[s];
    dx += p.h * acc;
    __syncthreads();
  }
}

// ADJ of one direction per CTA: Out[:, col] = lam_0 forced by W.
template <typename T>
__global__ void __launch_bounds__(1024) dir_adj_kernel(DirParams<T> p, const T* __restrict__ traj,
                                                      const T* __restrict__ Win, int ldw, T* Out, int ldo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = p.n, R = n + 2;
  T* X = reinterpret_cast<T*>(smraw);  // base stage states [S][n + 2]
  T* w = X + 4 * R;                     // kappa / lambda staging [n + 2]
  const int j = threadIdx.x, col = blockIdx.x;
  const bool act = j < n;
  for (int s = 0; s < 4; ++s) zero_ends(X + s * R, n);
  zero_ends(w, n);
  T lam = (T)0;
  T k[4], th[4];
  for (int t = p.N; t >= 1; --t) {
    const int oi = p.obs_of_step[t];
    if (oi >= 0) {
      __syncthreads();
      if (act) w[j + 1] = lam;
      __syncthreads();
      for (int o = j; o < p.n_o; o += blockDim.x) {
        const int r = oi * p.n_o + o;
        atomicAdd(&w[p.obs_idx[r] + 1], Win[(size_t)col * ldw + r] * p.inv_sigma);
      }
      __syncthreads();
      if (act) lam = w[j + 1];
    }
    // base stages of step t - 1
    const T x = act ? traj[(size_t)(t - 1) * n + j] : (T)0;
    for (int s = 0; s < p.S; ++s) {
      T Xs = x;
      for (int q = 0; q < s; ++q) Xs += p.h * p.a[s][q] * k[q];
      __syncthreads();
      if (act) X[s * R + j + 1] = Xs;
      __syncthreads();
      k[s] = act ? rhs_at(X + s * R, j + 1, p.c1, p.c2) : (T)0;
    }
    for (int i = p.S - 1; i >= 0; --i) {
      T kap = p.h * p.b[i] * lam;
      for (int q = i + 1; q < p.S; ++q) kap += p.h * p.a[q][i] * th[q];
      __syncthreads();
      if (act) w[j + 1] = kap;
      __syncthreads();
      th[i] = act ? vjp_at(X + i * R, w, j + 1, p.c1, p.c2) : (T)0;
    }
    T sum = (T)0;
    for (int i = 0; i < p.S; ++i) sum += th[i];
    lam += sum;
  }
  if (act) Out[(size_t)col * ldo + j] = lam;
}

// Y = (a I - b Delta*)^{-1} X (+ Z), one column per thread: forward
// elimination with the precomputed multipliers into an FP64 work column, back
// substitution in FP64, one rounding to the output type.
template <typename TI, typename TO, typename TZ>
__global__ void dir_prior_kernel(int n, int k, double bcoef, const double* __restrict__ cp,
                                 const double* __restrict__ den, const TI* __restrict__ X, int ldx, TO* Y,
                                 int ldy, const TZ* __restrict__ Z, int ldz, double* work) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= k) return;
  const TI* x = X + (size_t)col * ldx;
  double* dw = work + (size_t)col * n;
  // d'_i = (r_i + b d'_{i-1}) / den_i   (den_i = a + 2b + b c'_{i-1})
  double dprev = 0.0;
  for (int i = 0; i < n; ++i) {
    dprev = ((double)x[i] + bcoef * dprev) / den[i];
    dw[i] = dprev;
  }
  // x_i = d'_i - c'_i x_{i+1}, c'_i = -b / den_i
  TO* y = Y + (size_t)col * ldy;
  const TZ* z = Z ? Z + (size_t)col * ldz : nullptr;
  double xn = dprev;
  y[n - 1] = (TO)(z ? xn + (double)z[n - 1] : xn);
  for (int i = n - 2; i >= 0; --i) {
    xn = dw[i] - cp[i] * xn;
    y[i] = (TO)(z ? xn + (double)z[i] : xn);
  }
}

int threads_for(int n) { return ((n + 31) / 32) * 32; }

template <typename Kern, typename... Args>
int launch_dir(Kern kern, int grid, int threads, size_t smem, cudaStream_t st, Args... args) {
  if (smem > 48 * 1024) SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, threads, smem, st>>>(args...);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

}  // namespace

int dir_setup(DirGeom& g, double a, double b, cudaStream_t st) {
  // elimination of the constant tridiagonal matrix (a + 2b) on the diagonal, -b off it
  const int n = g.n;
  std::vector<double> cp(n), den(n);
  const double diag = a + 2.0 * b;
  double cprev = 0.0;
  for (int i = 0; i < n; ++i) {
    den[i] = diag + b * cprev;  // = diag - (-b) c'_{i-1}
    cp[i] = -b / den[i];
    cprev = cp[i];
  }
  g.bcoef = b;
  SC4_CUDA(cudaMemcpyAsync(g.cp, cp.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.den, den.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  return SC4DVAR_OK;
}

template <typename TI, typename TO, typename TZ>
int dir_prior_apply(const DirGeom& g, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz,
                    cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  if (k > g.work_cols) {
    set_error("Dirichlet prior: more columns than the handle's work array holds");
    return SC4DVAR_ERR_INVALID_ARG;
  }
  dir_prior_kernel<TI, TO, TZ><<<div_up(k, 64), 64, 0, st>>>(g.n, k, g.bcoef, g.cp, g.den, X, ldx, Y, ldy, Z,
                                                             ldz, g.work);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int dir_fwd(const DirGeom& g, const double* x0, double* traj, float* traj32, const double* y, double* d_out,
            double* obs_out, double* xN, cudaStream_t st) {
  auto p = make_params<double>(g);
  return launch_dir(dir_fwd_kernel<double>, 1, threads_for(g.n), (size_t)(g.n + 2) * sizeof(double), st, p,
                    x0, traj, traj32, y, d_out, obs_out, xN);
}

template <typename T>
int dir_tlm(const DirGeom& g, const T* traj, const T* U0, int ldu, int k, T* W, int ldw, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  auto p = make_params<T>(g);
  return launch_dir(dir_tlm_kernel<T>, k, threads_for(g.n), (size_t)2 * (g.n + 2) * sizeof(T), st, p, traj,
                    U0, ldu, W, ldw);
}

template <typename T>
int dir_adj(const DirGeom& g, const T* traj, const T* W, int ldw, int k, T* Out, int ldo, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  auto p = make_params<T>(g);
  return launch_dir(dir_adj_kernel<T>, k, threads_for(g.n), (size_t)5 * (g.n + 2) * sizeof(T), st, p, traj,
                    W, ldw, Out, ldo);
}

template int dir_tlm<double>(const DirGeom&, const double*, const double*, int, int, double*, int, cudaStream_t);
template int dir_tlm<float>(const DirGeom&, const float*, const float*, int, int, float*, int, cudaStream_t);
template int dir_adj<double>(const DirGeom&, const double*, const double*, int, int, double*, int, cudaStream_t);
template int dir_adj<float>(const DirGeom&, const float*, const float*, int, int, float*, int, cudaStream_t);
template int dir_prior_apply<double, double, double>(const DirGeom&, int, const double*, int, double*, int,
                                                     const double*, int, cudaStream_t);
template int dir_prior_apply<float, float, float>(const DirGeom&, int, const float*, int, float*, int,
                                                  const float*, int, cudaStream_t);
template int dir_prior_apply<double, float, float>(const DirGeom&, int, const double*, int, float*, int,
                                                   const float*, int, cudaStream_t);
template int dir_prior_apply<float, double, double>(const DirGeom&, int, const float*, int, double*, int,
                                                    const double*, int, cudaStream_t);

}  // namespace sc4
