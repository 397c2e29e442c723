// C ABI of the sc4dvar library: problem handles, the model operators of
// Eq. Rhalf, the sketches of Algs. 1-5, PCG (Eq. pcgsystem) and the GN loop with
// the reuse rule of Sec. 3.2. Host code here only orchestrates: every arithmetic
// step runs in the kernels of burgers.cu, fft.cu and dense.cu.
#include <atomic>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "common.cuh"
#include "dense.cuh"
#include "tall_tc.cuh"
#include "dfloat.cuh"
#include "fft.cuh"
#include "model.cuh"
#include "problem.cuh"
#include "dirichlet.cuh"

namespace sc4 {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static const double kClampRel = 1e-10;  // SE prior: eigenvalues below this x max -> 0

}  // namespace sc4

namespace sc4 {

using Prob = sc4dvar_problem_s;
using Prec = sc4dvar_precond_s;

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------ small kernels
__global__ void gaussian_kernel(uint64_t seed, uint64_t stream, int rows, int cols, int64_t col0,
                                double* out) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t tot = (size_t)rows * cols;
  if (idx < tot) {
    uint64_t i = idx % rows, j = idx / rows;
    uint64_t e = i + (uint64_t)rows * (uint64_t)(col0 + (int64_t)j);
    out[idx] = philox_normal(seed, stream, e);
  }
}

__global__ void fill_kernel(size_t n, double v, double* x) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

template <typename TI, typename TO>
__global__ void convert_kernel(size_t n, const TI* x, TO* y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = (TO)x[i];
}

// copy an r x c block (ld in) into a dense r x c (ld r) or back
template <typename TI, typename TO>
__global__ void copy_block_kernel(int r, int c, const TI* A, int lda, TO* B, int ldb) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)r * c) {
    int i = (int)(idx % r), j = (int)(idx / r);
    B[(size_t)j * ldb + i] = (TO)A[(size_t)j * lda + i];
  }
}

// A = (A + A^T)/2 (+ shift I), l x l
__global__ void symmetrize_kernel(int l, double* A, int lda, double shift) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * l) {
    int i = idx % l, j = idx / l;
    if (i < j) {
      double a = 0.5 * (A[(size_t)j * lda + i] + A[(size_t)i * lda + j]);
      A[(size_t)j * lda + i] = a;
      A[(size_t)i * lda + j] = a;
    } else if (i == j) {
      A[(size_t)j * lda + i] += shift;
    }
  }
}

// A[:r, :c] = 0 (ld lda)
__global__ void zero_block_kernel(int r, int c, double* A, int lda) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)r * c) A[(idx / r) * lda + idx % r] = 0.0;
}

// B = the upper triangle of A (zeros below the diagonal), or its transpose
// (a lower triangle) when trans; l x l
__global__ void triu_copy_kernel(int l, const double* A, int lda, double* B, int ldb, int trans) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * l) {
    int i = idx % l, j = idx / l;
    if (trans) B[(size_t)j * ldb + i] = (i >= j) ? A[(size_t)i * lda + j] : 0.0;
    else B[(size_t)j * ldb + i] = (i <= j) ? A[(size_t)j * lda + i] : 0.0;
  }
}

// B (l x r) = U[:, :r] * diag(1/sqrt(w)), and lam = max(0, w - nu) (first r)
__global__ void svd_scale_kernel(int l, int r, const double* U, int ldu, const double* w,
                                 double nu, double* B, double* lam, double* dsc) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * r) {
    int i = idx % l, j = idx / l;
    B[(size_t)j * l + i] = U[(size_t)j * ldu + i] / sqrt(w[j]);
  }
  if (idx < r) {
    double lm = fmax(0.0, w[idx] - nu);
    lam[idx] = lm;
    dsc[idx] = lm / (1.0 + lm);
  }
}

template <typename TI, typename TO>
static int convert(size_t n, const TI* x, TO* y, cudaStream_t st) {
  if (n == 0) return SC4DVAR_OK;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 8 * 152);
  convert_kernel<TI, TO><<<blocks, 256, 0, st>>>(n, x, y);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template <typename TI, typename TO>
static int copy_block(int r, int c, const TI* A, int lda, TO* B, int ldb, cudaStream_t st) {
  if ((size_t)r * c == 0) return SC4DVAR_OK;
  copy_block_kernel<TI, TO><<<(unsigned)(((size_t)r * c + 255) / 256), 256, 0, st>>>(r, c, A, lda,
                                                                                   B, ldb);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

static int gaussian(uint64_t seed, uint64_t stream, int rows, int cols, int64_t col0, double* out,
                    cudaStream_t st) {
  size_t tot = (size_t)rows * cols;
  if (tot == 0) return SC4DVAR_OK;
  gaussian_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(seed, stream, rows, cols, col0, out);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

static int d2h(double* host, const double* dev, size_t n, cudaStream_t st) {
  SC4_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  return SC4DVAR_OK;
}

static void count(Prob* P, int64_t tlm, int64_t adj) {
  switch (P->count_mode) {
    case kOffline: P->counters.tlm_offline += tlm; P->counters.adj_offline += adj; break;
    case kKappa: P->counters.tlm_kappa += tlm; P->counters.adj_kappa += adj; break;
    default: P->counters.tlm_online += tlm; P->counters.adj_online += adj; break;
  }
}

template <typename T> static const T* traj_of(Prob* P);
template <> const double* traj_of<double>(Prob* P) { return P->traj64; }
template <> const float* traj_of<float>(Prob* P) { return P->traj32; }

static bool is_bve(const Prob* P) { return P->model == SC4DVAR_MODEL_BVE2D; }
static bool is_dir(const Prob* P) { return P->model == SC4DVAR_MODEL_BURGERS1D_DIRICHLET; }
static bool is_gyre(const Prob* P) { return P->model == SC4DVAR_MODEL_BVE_GYRE; }

// Y = Gamma^{1/2} X (+ Z) for k columns: the 1D circulant (FFT), the 2D
// spectral multiplier of the model's grid, or the tridiagonal inverse of the
// Dirichlet prior.
template <typename TI, typename TO, typename TZ>
static int prior_any(Prob* P, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz,
                     cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  if (is_gyre(P)) {
    SC4_TRY(P->wGyPrior.ensure(gyre_prior_ws_bytes(P->gy, k, sizeof(double))));
    return gyre_prior_apply<TI, TO, TZ>(P->gy, k, X, ldx, Y, ldy, Z, ldz, P->wGyPrior.p, st);
  }
  if (is_dir(P)) {
    SC4_TRY(P->wDir.ensure((size_t)P->n * k * sizeof(double)));
    P->dir.work = P->wDir.as<double>();
    P->dir.work_cols = (int)(P->wDir.bytes / ((size_t)P->n * sizeof(double)));
    return dir_prior_apply<TI, TO, TZ>(P->dir, k, X, ldx, Y, ldy, Z, ldz, st);
  }
  if (!is_bve(P)) return prior_apply<TI, TO, TZ>(P->n, k, X, ldx, Y, ldy, Z, ldz, P->sym, P->tw, st);
  constexpr bool f32 = sizeof(TI) == 4 && sizeof(TO) == 4;
  using R = typename std::conditional<f32, float, double>::type;
  SC4_TRY(P->wCplx.ensure((size_t)((k + 1) / 2) * P->n * 2 * sizeof(R) + 256));
  return fft2_apply<R, TI, TO, TZ>(P->bve, k, X, ldx, Y, ldy, Z, ldz, P->bve.prior, P->wCplx.p, st);
}

// W = R^{-1/2} O_i M_i U for all i (TLM sweep of k columns)
template <typename T>
static int model_tlm(Prob* P, const T* U, int ldu, int k, T* W, int ldw, cudaStream_t st) {
  if (is_dir(P)) return dir_tlm<T>(P->dir, traj_of<T>(P), U, ldu, k, W, ldw, st);
  if (is_gyre(P)) {
    SC4_TRY(P->wGy.ensure(gyre_sweep_ws_bytes(P->gy, k, sizeof(T))));
    return gyre_tlm<T>(P->gy, U, ldu, k, W, ldw, P->wGy.p, st);
  }
  if (!is_bve(P)) return burgers_tlm<T>(P->geom, traj_of<T>(P), U, ldu, k, W, ldw, st);
  SC4_TRY(P->wBve.ensure(bve_sweep_ws_bytes(P->bve, k, sizeof(T))));
  return bve_tlm<T>(P->bve, U, ldu, k, W, ldw, P->wBve.p, st);
}

// L = sum_i M_i^T O_i^T R^{-1/2} W_i (ADJ sweep of k columns)
template <typename T>
static int model_adj(Prob* P, const T* W, int ldw, int k, T* L, int ldl, cudaStream_t st) {
  if (is_dir(P)) return dir_adj<T>(P->dir, traj_of<T>(P), W, ldw, k, L, ldl, st);
  if (is_gyre(P)) {
    SC4_TRY(P->wGy.ensure(gyre_sweep_ws_bytes(P->gy, k, sizeof(T))));
    return gyre_adj<T>(P->gy, W, ldw, k, L, ldl, P->wGy.p, st);
  }
  if (!is_bve(P)) return burgers_adj<T>(P->geom, traj_of<T>(P), W, ldw, k, L, ldl, st);
  SC4_TRY(P->wBve.ensure(bve_sweep_ws_bytes(P->bve, k, sizeof(T))));
  return bve_adj<T>(P->bve, W, ldw, k, L, ldl, P->wBve.p, st);
}

// ------------------------------------------------------------------ operators
template <typename T>
static int tlm_block(Prob* P, const T* X, int ldx, int k, T* W, int ldw, cudaStream_t st) {
  NvtxRange r("sc4dvar TLM block sweep");
  SC4_TRY(P->wU.ensure((size_t)P->n * k * sizeof(T)));
  T* U = P->wU.as<T>();
  SC4_TRY(prior_any<T, T, T>(P, k, X, ldx, U, P->n, (const T*)nullptr, 0, st));
  SC4_TRY(model_tlm<T>(P, U, P->n, k, W, ldw, st));
  count(P, k, 0);
  return SC4DVAR_OK;
}

template <typename T>
static int adj_block(Prob* P, const T* W, int ldw, int k, T* X, int ldx, const T* addZ, int ldz,
                     cudaStream_t st) {
  NvtxRange r("sc4dvar ADJ block sweep");
  SC4_TRY(P->wL.ensure((size_t)P->n * k * sizeof(T)));
  T* L = P->wL.as<T>();
  SC4_TRY(model_adj<T>(P, W, ldw, k, L, P->n, st));
  SC4_TRY(prior_any<T, T, T>(P, k, L, P->n, X, ldx, addZ, ldz, st));
  count(P, 0, k);
  return SC4DVAR_OK;
}

// Y = (I + A^T A) X or A^T A X, k columns, arithmetic in T.
template <typename T>
static int hvp_block(Prob* P, const T* X, int ldx, int k, T* Y, int ldy, int misfit_only,
                     cudaStream_t st) {
  SC4_TRY(P->wW.ensure((size_t)P->m * k * sizeof(T)));
  T* W = P->wW.as<T>();
  SC4_TRY(tlm_block<T>(P, X, ldx, k, W, P->m, st));
  SC4_TRY(adj_block<T>(P, W, P->m, k, Y, ldy, misfit_only ? (const T*)nullptr : X, ldx, st));
  return SC4DVAR_OK;
}

// Y = (I + A^T A) X (or A^T A X) for double blocks with double-float sweeps
// (periodic Burgers): the prior square root in FP64, the TLM / ADJ sweeps on
// (hi, lo) float pairs over a double-float copy of the FP64 trajectory.
static int hvp_block_df64(Prob* P, const double* X, int ldx, int k, double* Y, int ldy, int misfit_only,
                          cudaStream_t st) {
  const int n = P->n, m = P->m;
  if (k <= 0) return SC4DVAR_OK;
  if (!P->traj_df) {
    if (cudaMalloc(&P->traj_df, (size_t)(P->N + 1) * n * sizeof(dfloat)) != cudaSuccess) {
      cudaGetLastError();
      P->traj_df = nullptr;
      set_error("DF64: allocation of the double-float trajectory failed");
      return SC4DVAR_ERR_OOM;
    }
    P->traj_df_valid = false;
  }
  dfloat* traj = reinterpret_cast<dfloat*>(P->traj_df);
  if (!P->traj_df_valid) {
    SC4_TRY(to_dfloat(n, P->N + 1, P->traj64, n, traj, n, st));
    P->traj_df_valid = true;
  }
  SC4_TRY(P->wU.ensure((size_t)n * k * sizeof(double)));
  SC4_TRY(P->wL.ensure((size_t)n * k * sizeof(double)));
  SC4_TRY(P->wDF.ensure((size_t)(2 * n + m) * k * sizeof(dfloat)));
  double* U = P->wU.as<double>();
  double* L = P->wL.as<double>();
  dfloat* Ud = P->wDF.as<dfloat>();
  dfloat* Wd = Ud + (size_t)n * k;
  dfloat* Ld = Wd + (size_t)m * k;
  SC4_TRY(prior_any<double, double, double>(P, k, X, ldx, U, n, (const double*)nullptr, 0, st));
  SC4_TRY(to_dfloat(n, k, U, n, Ud, n, st));
  SC4_TRY(burgers_tlm<dfloat>(P->geom, traj, Ud, n, k, Wd, m, st));
  SC4_TRY(burgers_adj<dfloat>(P->geom, traj, Wd, m, k, Ld, n, st));
  SC4_TRY(from_dfloat(n, k, Ld, n, L, n, st));
  SC4_TRY(prior_any<double, double, double>(P, k, L, n, Y, ldy, misfit_only ? (const double*)nullptr : X, ldx,
                                            st));
  count(P, k, k);
  return SC4DVAR_OK;
}

// q = (I + H) p for one FP64 vector, operator arithmetic in prec (launches only).
static int hvp_vec_launch(Prob* P, const double* p, double* q, int prec, cudaStream_t st) {
  if (prec == SC4DVAR_DF64) return hvp_block_df64(P, p, P->n, 1, q, P->n, 0, st);
  if (prec == SC4DVAR_FP64) return hvp_block<double>(P, p, P->n, 1, q, P->n, 0, st);
  int n = P->n, m = P->m;
  SC4_TRY(P->wU.ensure((size_t)n * sizeof(float)));
  SC4_TRY(P->wW.ensure((size_t)m * sizeof(float)));
  SC4_TRY(P->wL.ensure((size_t)n * sizeof(float)));
  float* U = P->wU.as<float>();
  float* W = P->wW.as<float>();
  float* L = P->wL.as<float>();
  SC4_TRY(prior_any<double, float, float>(P, 1, p, n, U, n, (const float*)nullptr, 0, st));
  SC4_TRY(model_tlm<float>(P, U, n, 1, W, m, st));
  SC4_TRY(model_adj<float>(P, W, m, 1, L, n, st));
  SC4_TRY(prior_any<float, double, double>(P, 1, L, n, q, n, p, n, st));
  count(P, 1, 1);
  return SC4DVAR_OK;
}

// Vorticity problems run a single-vector product as thousands of small
// launches (every RK stage of both sweeps is a 2D transform and a stencil
// kernel), so it is recorded once per (p, q, precision) as a CUDA graph on the
// handle's private stream and replayed on the caller's stream. The first call
// of a key runs eagerly (it sizes the work arrays, so nothing allocates during
// recording); a recording is discarded when a work array has moved since.
static void hvp_bufs(Prob* P, void* (&b)[7]) {
  b[0] = P->wBve.p; b[1] = P->wCplx.p; b[2] = P->wU.p; b[3] = P->wW.p; b[4] = P->wL.p;
  b[5] = P->wGy.p; b[6] = P->wGyPrior.p;
}

static int hvp_vec(Prob* P, const double* p, double* q, int prec, cudaStream_t st) {
  if (!is_bve(P) && !is_gyre(P)) return hvp_vec_launch(P, p, q, prec, st);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return hvp_vec_launch(P, p, q, prec, st);
  }
  Prob::HvpGraph* e = nullptr;
  for (auto& g : P->hvp_graphs)
    if (g.p == p && g.q == q && g.prec == prec) e = &g;
  if (!e) {
    SC4_TRY(hvp_vec_launch(P, p, q, prec, st));
    if (P->hvp_graphs.size() >= 8) {
      if (P->hvp_graphs.front().exec) cudaGraphExecDestroy(P->hvp_graphs.front().exec);
      P->hvp_graphs.erase(P->hvp_graphs.begin());
    }
    Prob::HvpGraph g{p, q, prec, {}, nullptr, false};
    hvp_bufs(P, g.bufs);
    P->hvp_graphs.push_back(g);
    return SC4DVAR_OK;
  }
  void* now[7];
  hvp_bufs(P, now);
  bool same = true;
  for (int i = 0; i < 7; ++i) same = same && now[i] == e->bufs[i];
  if (e->exec && !same) {
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
  }
  if (!e->exec && !e->eager_only) {
    if (!P->graph_stream) SC4_CUDA(cudaStreamCreateWithFlags(&P->graph_stream, cudaStreamNonBlocking));
    SC4_CUDA(cudaStreamSynchronize(st));
    const sc4dvar_counters_t saved = P->counters;
    cudaGraph_t graph = nullptr;
    int rc = SC4DVAR_OK;
    if (cudaStreamBeginCapture(P->graph_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = SC4DVAR_ERR_CUDA;
    } else {
      rc = hvp_vec_launch(P, p, q, prec, P->graph_stream);
      if (cudaStreamEndCapture(P->graph_stream, &graph) != cudaSuccess) rc = SC4DVAR_ERR_CUDA;
    }
    P->counters = saved;  // recording executes nothing
    if (rc == SC4DVAR_OK && graph && cudaGraphInstantiate(&e->exec, graph, 0) != cudaSuccess) {
      e->exec = nullptr;
      rc = SC4DVAR_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc != SC4DVAR_OK) {
      cudaGetLastError();
      e->eager_only = true;  // the same kernels, launched one by one
    } else {
      hvp_bufs(P, e->bufs);
    }
  }
  if (!e->exec) return hvp_vec_launch(P, p, q, prec, st);
  SC4_CUDA(cudaGraphLaunch(e->exec, st));
  count(P, 1, 1);
  return SC4DVAR_OK;
}

// Entry points of the batch module (batch.cu): the same operators, by problem.
int batch_hvp_one(Prob* P, const void* X, int k, void* Y, int misfit_only, int prec, cudaStream_t st) {
  if (prec == SC4DVAR_FP64)
    return hvp_block<double>(P, (const double*)X, P->n, k, (double*)Y, P->n, misfit_only, st);
  return hvp_block<float>(P, (const float*)X, P->n, k, (float*)Y, P->n, misfit_only, st);
}

int batch_hvp_vec(Prob* P, const double* p, double* q, int prec, cudaStream_t st) {
  return hvp_vec(P, p, q, prec, st);
}

int batch_precond(Prec* pc, const double* r, double* z, int n, cudaStream_t st) {
  if (pc && pc->l > 0) {
    SC4_TRY(pc->T.ensure((size_t)pc->l * sizeof(double)));
    return woodbury_apply(n, pc->l, 1, pc->V, n, pc->dsc, r, n, z, n, pc->T.as<double>(), st);
  }
  SC4_CUDA(cudaMemcpyAsync(z, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SC4DVAR_OK;
}

static int host_scalar(Prob* P, double* out, cudaStream_t st) {
  return d2h(out, P->scal.as<double>(), 1, st);
}

// ------------------------------------------------------------------ sketch helpers
// Workspace for the dense steps of one sketch.
struct SketchWS {
  Buf a, b, c, g, g2, u, w, info, jw, tc;
  int64_t* shifted = nullptr;  // problem counter of shifted CholeskyQR retries
  int tall = kTall3xTF32;      // arithmetic of the FP32 tall products (sketch_opts.gemm)
  void release() {
    a.release(); b.release(); c.release(); g.release(); g2.release(); u.release(); w.release();
    info.release(); jw.release(); tc.release();
  }
};

// A tall product with an l x l factor: FP32 sketch matrices with several
// columns go to the tensor cores in the sketch's mode (or the CUDA-core kernel
// when asked); FP64 operands and single vectors keep the FP64 / CUDA-core path.
template <typename T, typename TC>
static int tall_nn(SketchWS& ws, int rows, int kk, int c, double alpha, const T* A, int lda,
                   const double* B, int ldb, int transB, double beta, TC* C, int ldc, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (c > 1 && kk > 0 && ws.tall != kTallSIMT) {
      SC4_TRY(ws.tc.ensure(tall_pack_bytes(ws.tall, kk, c)));
      return tall_gemm_tc<TC>(ws.tall, rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C, ldc, ws.tc.p, st);
    }
  }
  return gemm_nn<T, TC>(rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C, ldc, st);
}

static int check_info(Buf& info, const char* what, cudaStream_t st) {
  int h = 0;
  SC4_CUDA(cudaMemcpyAsync(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  if (h != 0) {
    set_error(std::string(what) + ": matrix not positive definite at pivot " + std::to_string(h));
    return SC4DVAR_ERR_NOT_SPD;
  }
  return SC4DVAR_OK;
}

// One CholeskyQR pass: G = src^T src (FP64), L = chol(G), dst = src L^{-T}.
// When allowed, a failed factorization is retried with the diagonal shift
// 11 (rows l + l(l+1)) u tr(G) (shifted CholeskyQR, Fukaya et al. 2020;
// tr(G) >= |G|_2), u = 2^-53.
template <typename T>
static int cholqr_pass(int rows, int l, const T* src, int lds, T* dst, int ldd, bool allow_shift,
                       bool* shifted, SketchWS& ws, cudaStream_t st) {
  SC4_TRY(ws.g.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.g2.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.info.ensure(64));
  double* G = ws.g.as<double>();
  double* Li = ws.g2.as<double>();
  SC4_TRY(gemm_tn<T, T>(rows, l, l, 1.0, src, lds, src, lds, 0.0, G, l, st));
  SC4_TRY(chol_lower(l, G, l, ws.info.as<int>(), st));
  int s = check_info(ws.info, "CholeskyQR", st);
  if (s == SC4DVAR_ERR_NOT_SPD && allow_shift) {
    SC4_TRY(gemm_tn<T, T>(rows, l, l, 1.0, src, lds, src, lds, 0.0, G, l, st));
    std::vector<double> hg((size_t)l * l);
    SC4_CUDA(cudaMemcpyAsync(hg.data(), G, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    SC4_CUDA(cudaStreamSynchronize(st));
    double tr = 0;
    for (int i = 0; i < l; ++i) tr += hg[(size_t)i * l + i];
    // u is the unit roundoff of the Gram matrix, which is FP64-accurate for FP32
    // data as well (products accumulated exactly in double-float): with the FP32
    // roundoff the shift would exceed tr(G) at rows l ~ 10^7 and wipe out the
    // factorization.
    const double u = std::ldexp(1.0, -53);
    double shift = 11.0 * ((double)rows * l + (double)l * (l + 1)) * u * tr;
    symmetrize_kernel<<<div_up(l * l, 256), 256, 0, st>>>(l, G, l, shift);
    SC4_LAUNCH_CHECK();
    SC4_TRY(chol_lower(l, G, l, ws.info.as<int>(), st));
    s = check_info(ws.info, "shifted CholeskyQR", st);
    if (s == SC4DVAR_OK && shifted) *shifted = true;
    if (s == SC4DVAR_OK && ws.shifted) ++*ws.shifted;
  }
  if (s != SC4DVAR_OK) return s;
  SC4_TRY(trtri_lower(l, G, l, Li, l, 0.0, st));
  return tall_nn<T, T>(ws, rows, l, l, 1.0, src, lds, Li, l, 1, 0.0, dst, ldd, st);
}

// Thin QR Y = Q R by CholeskyQR2 (Q separate from Y; a third pass when the
// first one needed a shift: shifted CholeskyQR3). When Y is rank deficient
// (a sketch wider than the operator's numerical rank) the columns of the first
// pass beyond that rank are tiny and the later Gram matrices are singular too:
// every pass may then take the shift, those columns stay tiny (their A^T q is
// negligible and the thin SVD that follows drops them) and the others come out
// orthonormal.
template <typename T>
static int cholqr2(int rows, int l, const T* Y, int ldy, T* Q, int ldq, SketchWS& ws, cudaStream_t st) {
  bool shifted = false;
  SC4_TRY(cholqr_pass<T>(rows, l, Y, ldy, Q, ldq, true, &shifted, ws, st));
  SC4_TRY(ws.c.ensure((size_t)rows * l * sizeof(T)));
  T* C = ws.c.as<T>();
  int passes = shifted ? 2 : 1;
  for (int p = 0; p < passes; ++p) {
    SC4_TRY(copy_block<T, T>(rows, l, Q, ldq, C, rows, st));
    SC4_TRY(cholqr_pass<T>(rows, l, C, rows, Q, ldq, true, nullptr, ws, st));
  }
  return SC4DVAR_OK;
}

// Thin SVD of W = Wt^T through the eigen-decomposition of the l x l Gram
// Wt^T Wt (FP64 Jacobi): V = Wt U Sigma^{-1}, lam = max(0, Sigma^2 - nu).
// Singular values below sqrt(drop) sigma_1 are dropped (their lam <= drop lam_1).
template <typename T>
static int finalize_svd(Prob* P, int l, const T* Wt, int ldw, double nu, double drop, Prec* out,
                        SketchWS& ws, cudaStream_t st) {
  int n = P->n;
  SC4_TRY(ws.g.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.g2.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.u.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.w.ensure((size_t)4 * l * sizeof(double)));
  double* G = ws.g.as<double>();
  double* U = ws.g2.as<double>();
  double* Us = ws.u.as<double>();
  double* w = ws.w.as<double>();
  double* ws_ = w + l;
  SC4_TRY(gemm_tn<T, T>(n, l, l, 1.0, Wt, ldw, Wt, ldw, 0.0, G, l, st));
  SC4_TRY(ws.jw.ensure(jacobi_work_bytes(l)));
  SC4_TRY(jacobi_eig(l, G, l, U, l, w, 60, 1e-15, ws.jw.p, nullptr, st));
  SC4_TRY(sort_desc(l, w, U, l, ws_, Us, l, st));
  std::vector<double> hw(l);
  SC4_CUDA(cudaMemcpyAsync(hw.data(), ws_, l * sizeof(double), cudaMemcpyDeviceToHost, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  int r = 0;
  while (r < l && hw[r] > drop * hw[0] && hw[r] > 0.0) ++r;
  out->n = n;
  out->l = r;
  if (out->V) cudaFree(out->V);
  if (out->lam) cudaFree(out->lam);
  out->V = out->lam = out->dsc = nullptr;
  if (r == 0) return SC4DVAR_OK;
  SC4_CUDA(cudaMalloc(&out->V, (size_t)n * r * sizeof(double)));
  SC4_CUDA(cudaMalloc(&out->lam, 2 * (size_t)r * sizeof(double)));
  out->dsc = out->lam + r;
  double* B = G;  // reuse: l x r
  svd_scale_kernel<<<div_up(l * r, 256), 256, 0, st>>>(l, r, Us, l, ws_, nu, B, out->lam, out->dsc);
  SC4_LAUNCH_CHECK();
  SC4_TRY(tall_nn<T, double>(ws, n, l, r, 1.0, Wt, ldw, B, l, 0, 0.0, out->V, n, st));
  return SC4DVAR_OK;
}

// z = (I + Wt Wt^T)^{-1} r for one vector, with L = chol(I + Wt^T Wt) given
// as Linv = L^{-1} (Remark 1, Eq. randsvdsv): z = r - Wt Linv^T Linv Wt^T r.
template <typename T>
static int remark1_apply(int n, int l, const T* Wt, int ldw, const double* Linv, const double* r,
                         double* z, double* t1, double* t2, cudaStream_t st) {
  SC4_TRY(gemm_tn<T, double>(n, l, 1, 1.0, Wt, ldw, r, n, 0.0, t1, l, st));         // Wt^T r
  SC4_TRY(gemm_nn<double, double>(l, l, 1, 1.0, Linv, l, t1, l, 0, 0.0, t2, l, st)); // Linv t1
  SC4_TRY(gemm_tn<double, double>(l, l, 1, 1.0, Linv, l, t2, l, 0.0, t1, l, st));   // Linv^T t2
  if (z != r) SC4_TRY(copy_block<double, double>(n, 1, r, n, z, n, st));
  SC4_TRY(gemm_nn<T, double>(n, l, 1, -1.0, Wt, ldw, t1, l, 0, 1.0, z, n, st));
  return SC4DVAR_OK;
}

// kappa = |(I + H) z| with z = P v, v the unit Philox test vector (seed, stream, col).
static int unit_test_vector(Prob* P, uint64_t seed, uint64_t stream, int col, double* v,
                            cudaStream_t st) {
  SC4_TRY(gaussian(seed, stream, P->n, 1, col, v, st));
  SC4_TRY(vnrm2<double>(P->n, v, P->scal.as<double>(), P->part.as<double>(), st));
  double nrm;
  SC4_TRY(host_scalar(P, &nrm, st));
  SC4_TRY(axpby<double, double>(P->n, 0.0, v, 1.0 / nrm, v, st));
  return SC4DVAR_OK;
}

// vec workspace: 3 n doubles (v, z, q) + 4 * lmax doubles
static int ensure_vec(Prob* P, int lmax) {
  return P->vec.ensure(((size_t)3 * P->n + 4 * (size_t)lmax + 64) * sizeof(double));
}

template <typename T>
static int kappa_remark1(Prob* P, int l, const T* Wt, int ldw, uint64_t seed, uint64_t stream,
                         int col, int prec, SketchWS& ws, double* kappa, cudaStream_t st) {
  int n = P->n;
  SC4_TRY(ensure_vec(P, l));
  double* v = P->vec.as<double>();
  double* z = v + n;
  double* q = z + n;
  double* t1 = q + n;
  double* t2 = t1 + l;
  SC4_TRY(ws.g.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.g2.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.info.ensure(64));
  double* G = ws.g.as<double>();
  double* Li = ws.g2.as<double>();
  SC4_TRY(gemm_tn<T, T>(n, l, l, 1.0, Wt, ldw, Wt, ldw, 0.0, G, l, st));
  symmetrize_kernel<<<div_up(l * l, 256), 256, 0, st>>>(l, G, l, 1.0);
  SC4_LAUNCH_CHECK();
  SC4_TRY(chol_lower(l, G, l, ws.info.as<int>(), st));
  SC4_TRY(check_info(ws.info, "Remark 1 Cholesky", st));
  SC4_TRY(trtri_lower(l, G, l, Li, l, 0.0, st));
  SC4_TRY(unit_test_vector(P, seed, stream, col, v, st));
  SC4_TRY(remark1_apply<T>(n, l, Wt, ldw, Li, v, z, t1, t2, st));
  int saved = P->count_mode;
  P->count_mode = kKappa;
  int s = hvp_vec(P, z, q, prec, st);
  P->count_mode = saved;
  SC4_TRY(s);
  SC4_TRY(vnrm2<double>(n, q, P->scal.as<double>(), P->part.as<double>(), st));
  return host_scalar(P, kappa, st);
}

static int kappa_precond(Prob* P, Prec* pc, uint64_t seed, uint64_t stream, int col, int prec,
                         double* kappa, cudaStream_t st) {
  int n = P->n;
  int l = pc ? pc->l : 0;
  SC4_TRY(ensure_vec(P, l));
  double* v = P->vec.as<double>();
  double* z = v + n;
  double* q = z + n;
  SC4_TRY(unit_test_vector(P, seed, stream, col, v, st));
  if (pc && l > 0) {
    SC4_TRY(pc->T.ensure((size_t)l * sizeof(double)));
    SC4_TRY(woodbury_apply(n, l, 1, pc->V, n, pc->dsc, v, n, z, n, pc->T.as<double>(), st));
  } else {
    SC4_TRY(copy_block<double, double>(n, 1, v, n, z, n, st));
  }
  int saved = P->count_mode;
  P->count_mode = kKappa;
  int s = hvp_vec(P, z, q, prec, st);
  P->count_mode = saved;
  SC4_TRY(s);
  SC4_TRY(vnrm2<double>(n, q, P->scal.as<double>(), P->part.as<double>(), st));
  return host_scalar(P, kappa, st);
}

// Draw (or copy) an rows x cols double block into a T buffer.
template <typename T>
static int draw_block(Prob* P, const double* given, uint64_t seed, uint64_t stream, int rows,
                      int cols, int64_t col0, T* out, int ldo, Buf& tmp, cudaStream_t st) {
  const double* src = given;
  if (!src) {
    SC4_TRY(tmp.ensure((size_t)rows * cols * sizeof(double)));
    SC4_TRY(gaussian(seed, stream, rows, cols, col0, tmp.as<double>(), st));
    src = tmp.as<double>();
  }
  return copy_block<double, T>(rows, cols, src, rows, out, ldo, st);
}

// ------------------------------------------------------------------ sketches
template <typename T>
static int build_randsvd(Prob* P, const sc4dvar_sketch_opts& o, const double* Om_in, Prec* out,
                         cudaStream_t st) {
  const int n = P->n, m = P->m;
  const int l0 = o.l;
  const bool adapt = o.adaptive != 0;
  const int lh = adapt ? (o.l_hat > 0 ? o.l_hat : std::max(1, l0 / 2)) : 0;
  const int lmax = adapt ? (o.l_max > 0 ? o.l_max : std::min(8 * l0, n)) : l0;
  const uint64_t s_om = SC4DVAR_STREAM_SKETCH + (uint64_t)o.gn_iter;
  const uint64_t s_ka = SC4DVAR_STREAM_KAPPA + (uint64_t)o.gn_iter;
  SketchWS ws;
  ws.shifted = &P->counters.qr_shifted;
  ws.tall = o.gemm;
  Buf Om, Y, Qall, Wt, tmp;
  int rc = SC4DVAR_OK;
  auto body = [&]() -> int {
    SC4_TRY(Om.ensure((size_t)n * lmax * sizeof(T)));
    SC4_TRY(Y.ensure((size_t)m * lmax * sizeof(T)));
    SC4_TRY(Qall.ensure((size_t)m * lmax * sizeof(T)));
    SC4_TRY(Wt.ensure((size_t)n * lmax * sizeof(T)));
    T* om = Om.as<T>();
    T* y = Y.as<T>();
    T* Q = Qall.as<T>();   // columns 0..l-1: the accumulated orthonormal basis
    T* wt = Wt.as<T>();
    // Alg. 1 / Alg. 4 steps 1-4
    SC4_TRY(draw_block<T>(P, Om_in, o.seed, s_om, n, l0, 0, om, n, tmp, st));
    SC4_TRY(tlm_block<T>(P, om, n, l0, y, m, st));
    SC4_TRY(cholqr2<T>(m, l0, y, m, Q, m, ws, st));
    SC4_TRY(adj_block<T>(P, Q, m, l0, wt, n, (const T*)nullptr, 0, st));
    int l = l0;
    if (adapt) {
      double kap;
      int t = 1;
      SC4_TRY(kappa_remark1<T>(P, l, wt, n, o.seed, s_ka, t++, o.prec, ws, &kap, st));
      while (kap > o.eps_sk && l + lh <= lmax) {
        // Alg. 4 steps 8-14: new block, two Gram-Schmidt passes against Q, QR, ADJ
        T* yh = y + (size_t)m * l;
        SC4_TRY(draw_block<T>(P, nullptr, o.seed, s_om, n, lh, l, om + (size_t)n * l, n, tmp, st));
        SC4_TRY(tlm_block<T>(P, om + (size_t)n * l, n, lh, yh, m, st));
        SC4_TRY(ws.b.ensure((size_t)l * lh * sizeof(double)));
        for (int pass = 0; pass < 2; ++pass) {
          SC4_TRY(gemm_tn<T, T>(m, l, lh, 1.0, Q, m, yh, m, 0.0, ws.b.as<double>(), l, st));
          SC4_TRY(tall_nn<T, T>(ws, m, l, lh, -1.0, Q, m, ws.b.as<double>(), l, 0, 1.0, yh, m, st));
        }
        SC4_TRY(cholqr2<T>(m, lh, yh, m, Q + (size_t)m * l, m, ws, st));
        SC4_TRY(adj_block<T>(P, Q + (size_t)m * l, m, lh, wt + (size_t)n * l, n, (const T*)nullptr, 0, st));
        l += lh;
        SC4_TRY(kappa_remark1<T>(P, l, wt, n, o.seed, s_ka, t++, o.prec, ws, &kap, st));
      }
    }
    double drop = (sizeof(T) == 4) ? 1e-12 : 1e-15;
    SC4_TRY(finalize_svd<T>(P, l, wt, n, 0.0, drop, out, ws, st));
    return SC4DVAR_OK;
  };
  rc = body();
  cudaStreamSynchronize(st);
  ws.release(); Om.release(); Y.release(); Qall.release(); Wt.release(); tmp.release();
  return rc;
}

// Alg. 2 steps 3-7 on the sketch (Om, Y) with l columns; result into out.
template <typename T>
static int nystrom_core(Prob* P, int l, const T* om, T* y, double eps, Prec* out, SketchWS& ws,
                        cudaStream_t st) {
  const int n = P->n;
  SC4_TRY(ws.g.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.g2.ensure((size_t)l * l * sizeof(double)));
  SC4_TRY(ws.info.ensure(64));
  double* G = ws.g.as<double>();
  double* Li = ws.g2.as<double>();
  // nu = sqrt(n) eps |Y|_2, |Y|_2^2 = lambda_max(Y^T Y)
  SC4_TRY(gemm_tn<T, T>(n, l, l, 1.0, y, n, y, n, 0.0, G, l, st));
  SC4_TRY(power_lmax(l, G, l, P->scal.as<double>(), st));
  double lmax;
  SC4_TRY(host_scalar(P, &lmax, st));
  double nu = std::sqrt((double)n) * eps * std::sqrt(std::max(lmax, 0.0));
  // Y <- Y + nu Omega; C = Omega^T Y; L = chol((C + C^T)/2); W^T = Y L^{-T}
  SC4_TRY(axpby<T, T>((size_t)n * l, nu, om, 1.0, y, st));
  SC4_TRY(gemm_tn<T, T>(n, l, l, 1.0, om, n, y, n, 0.0, G, l, st));
  symmetrize_kernel<<<div_up(l * l, 256), 256, 0, st>>>(l, G, l, 0.0);
  SC4_LAUNCH_CHECK();
  SC4_TRY(chol_lower(l, G, l, ws.info.as<int>(), st));
  SC4_TRY(check_info(ws.info, "Nystrom Cholesky", st));
  SC4_TRY(trtri_lower(l, G, l, Li, l, 0.0, st));
  SC4_TRY(ws.a.ensure((size_t)n * l * sizeof(T)));
  T* wt = ws.a.as<T>();
  SC4_TRY(tall_nn<T, T>(ws, n, l, l, 1.0, y, n, Li, l, 1, 0.0, wt, n, st));
  double drop = (sizeof(T) == 4) ? 1e-12 : 1e-15;
  return finalize_svd<T>(P, l, wt, n, nu, drop, out, ws, st);
}

template <typename T>
static int build_nystrom(Prob* P, const sc4dvar_sketch_opts& o, const double* Om_in, Prec* out,
                         cudaStream_t st) {
  const int n = P->n;
  const int l0 = o.l;
  const bool adapt = o.adaptive != 0;
  const int lh = adapt ? (o.l_hat > 0 ? o.l_hat : std::max(1, l0 / 2)) : 0;
  const int lmax = adapt ? (o.l_max > 0 ? o.l_max : std::min(8 * l0, n)) : l0;
  const uint64_t s_om = SC4DVAR_STREAM_SKETCH + (uint64_t)o.gn_iter;
  const uint64_t s_ka = SC4DVAR_STREAM_KAPPA + (uint64_t)o.gn_iter;
  const double eps = (sizeof(T) == 4) ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
  SketchWS ws;
  ws.shifted = &P->counters.qr_shifted;
  ws.tall = o.gemm;
  Buf Om, Y, Yc, tmp;
  auto body = [&]() -> int {
    SC4_TRY(Om.ensure((size_t)n * lmax * sizeof(T)));
    SC4_TRY(Y.ensure((size_t)n * lmax * sizeof(T)));
    SC4_TRY(Yc.ensure((size_t)n * lmax * sizeof(T)));
    T* om = Om.as<T>();
    T* y = Y.as<T>();
    T* yc = Yc.as<T>();
    SC4_TRY(draw_block<T>(P, Om_in, o.seed, s_om, n, l0, 0, om, n, tmp, st));
    SC4_TRY(hvp_block<T>(P, om, n, l0, y, n, 1, st));
    int l = l0;
    int t = 1;
    for (;;) {
      // the Nystrom steps shift Y in place: keep the raw sketch for growth
      SC4_TRY(copy_block<T, T>(n, l, y, n, yc, n, st));
      SC4_TRY(nystrom_core<T>(P, l, om, yc, eps, out, ws, st));
      if (!adapt) break;
      double kap;
      SC4_TRY(kappa_precond(P, out, o.seed, s_ka, t++, o.prec, &kap, st));
      if (!(kap > o.eps_sk) || l + lh > lmax) break;
      SC4_TRY(draw_block<T>(P, nullptr, o.seed, s_om, n, lh, l, om + (size_t)n * l, n, tmp, st));
      SC4_TRY(hvp_block<T>(P, om + (size_t)n * l, n, lh, y + (size_t)n * l, n, 1, st));
      l += lh;
    }
    return SC4DVAR_OK;
  };
  int rc = body();
  cudaStreamSynchronize(st);
  ws.release(); Om.release(); Y.release(); Yc.release(); tmp.release();
  return rc;
}

// Thin QR of an FP64 matrix A (rows x c, rows >= c): Q by CholeskyQR2, then
// R = Q^T A with its lower triangle set to zero.
static int qr_f64(int rows, int c, const double* A, int lda, double* Q, int ldq, double* R, int ldr,
                  cudaStream_t st) {
  if (c == 0) return SC4DVAR_OK;
  SketchWS w;
  Buf rt;
  auto body = [&]() -> int {
    SC4_TRY(cholqr2<double>(rows, c, A, lda, Q, ldq, w, st));
    SC4_TRY(rt.ensure((size_t)c * c * sizeof(double)));
    SC4_TRY(gemm_tn<double, double>(rows, c, c, 1.0, Q, ldq, A, lda, 0.0, rt.as<double>(), c, st));
    triu_copy_kernel<<<div_up(c * c, 256), 256, 0, st>>>(c, rt.as<double>(), c, R, ldr, 0);
    SC4_LAUNCH_CHECK();
    return SC4DVAR_OK;
  };
  int rc = body();
  cudaStreamSynchronize(st);
  w.release();
  rt.release();
  return rc;
}

// Alg. 6 (QR update for adaptive SingleView). With A1 = P[:, :r1]^T,
// A2 = P[:, r1:r1+r2]^T (P is m x (r1 + r2), ld ldp) and B1 = B[:, :k1],
// B2 = B[:, k1:k1+k2] (orthonormal columns, ld ldb): on entry the leading
// r1 x k1 block of Qm and k1 x k1 block of Rm hold Q1 R1 = A1 B1; on exit
// Qm ((r1 + r2) x (k1 + k2)) and Rm ((k1 + k2) x (k1 + k2), upper triangular)
// hold the thin QR of [A1; A2][B1 B2]. Steps 1-3 are taken together as the QR
// of [R1; A2 B1] followed by blockdiag(Q1, I): when A2 B1 = Q2 R2,
// [R1; A2 B1] = blockdiag(I, Q2) [R1; R2], so this is the QR of step 2 carried
// through step 3, without the thin QR of A2 B1 (a wide r2 x k1 matrix once the
// sketch has grown past r2 columns).
template <typename T>
static int qr_update(int m, int r1, int r2, int k1, int k2, const T* P, int ldp, const T* B, int ldb,
                     double* Qm, int ldq, double* Rm, int ldr, cudaStream_t st) {
  const int ra = r1 + r2, rs = k1 + r2;
  Buf bS, bQ3s, bQ3, bP1;
  auto body = [&]() -> int {
    SC4_TRY(bS.ensure((size_t)rs * std::max(k1, 1) * sizeof(double)));
    SC4_TRY(bQ3s.ensure((size_t)rs * std::max(k1, 1) * sizeof(double)));
    SC4_TRY(bQ3.ensure((size_t)ra * std::max(k1, 1) * sizeof(double)));
    SC4_TRY(bP1.ensure((size_t)ra * std::max(k2, 1) * sizeof(double)));
    double *S = bS.as<double>(), *Q3s = bQ3s.as<double>(), *Q3 = bQ3.as<double>(), *P1 = bP1.as<double>();
    if (k1 > 0) {
      // steps 1-2: S = [R1; A2 B1], S = Q3s R3 (R3 into Rm's leading block)
      SC4_TRY(copy_block<double, double>(k1, k1, Rm, ldr, S, rs, st));
      SC4_TRY(gemm_tn<T, T>(m, r2, k1, 1.0, P + (size_t)ldp * r1, ldp, B, ldb, 0.0, S + k1, rs, st));
      SC4_TRY(qr_f64(rs, k1, S, rs, Q3s, rs, Rm, ldr, st));
      // step 3: Q3 = blockdiag(Q1, I) Q3s
      SC4_TRY(gemm_nn<double, double>(r1, k1, k1, 1.0, Qm, ldq, Q3s, rs, 0, 0.0, Q3, ra, st));
      SC4_TRY(copy_block<double, double>(r2, k1, Q3s + k1, rs, Q3 + r1, ra, st));
    }
    if (k2 > 0) {
      // step 4: P1 = [A1; A2] B2
      SC4_TRY(gemm_tn<T, T>(m, ra, k2, 1.0, P, ldp, B + (size_t)ldb * k1, ldb, 0.0, P1, ra, st));
      if (k1 > 0) {
        // step 5: Q3^T P1 (the upper-right block of R5), P2 = P1 - Q3 (Q3^T P1)
        double* Rtr = Rm + (size_t)ldr * k1;
        SC4_TRY(gemm_tn<double, double>(ra, k1, k2, 1.0, Q3, ra, P1, ra, 0.0, Rtr, ldr, st));
        SC4_TRY(gemm_nn<double, double>(ra, k1, k2, -1.0, Q3, ra, Rtr, ldr, 0, 1.0, P1, ra, st));
      }
      // step 6: P2 = Q4 R4 into the new columns of Qm and the lower-right block of Rm
      SC4_TRY(qr_f64(ra, k2, P1, ra, Qm + (size_t)ldq * k1, ldq, Rm + (size_t)ldr * k1 + k1, ldr, st));
    }
    if (k1 > 0) {
      // step 7: Q5 = [Q3 Q4], R5 = [R3 Q3^T P1; 0 R4]
      SC4_TRY(copy_block<double, double>(ra, k1, Q3, ra, Qm, ldq, st));
      if (k2 > 0) {
        zero_block_kernel<<<div_up(k2 * k1, 256), 256, 0, st>>>(k2, k1, Rm + k1, ldr);
        SC4_LAUNCH_CHECK();
      }
    }
    return SC4DVAR_OK;
  };
  int rc = body();
  cudaStreamSynchronize(st);
  bS.release(); bQ3s.release(); bQ3.release(); bP1.release();
  return rc;
}

// Alg. 3 / Alg. 5: W = R_M^dagger (Z Q_M)^T with M = Psi^T Q_Y = Q_M R_M, formed
// as W^T = Z (Q_M R_M^{-T}) (full column rank: R_M^dagger = R_M^{-1}).
template <typename T>
static int singleview_W(Prob* P, int l1, int l2, const double* Qm, int ldq, const double* Rm, int ldr,
                        const T* Z, T* wt, SketchWS& ws, cudaStream_t st) {
  const int n = P->n;
  SC4_TRY(ws.g.ensure((size_t)l1 * l1 * sizeof(double)));
  SC4_TRY(ws.g2.ensure((size_t)l1 * l1 * sizeof(double)));
  SC4_TRY(ws.u.ensure((size_t)l2 * l1 * sizeof(double)));
  double* Lt = ws.g.as<double>();
  double* Li = ws.g2.as<double>();
  double* Bm = ws.u.as<double>();
  triu_copy_kernel<<<div_up(l1 * l1, 256), 256, 0, st>>>(l1, Rm, ldr, Lt, l1, 1);  // R_M^T
  SC4_LAUNCH_CHECK();
  SC4_TRY(trtri_lower(l1, Lt, l1, Li, l1, 0.0, st));                                 // R_M^{-T}
  SC4_TRY(gemm_nn<double, double>(l2, l1, l1, 1.0, Qm, ldq, Li, l1, 0, 0.0, Bm, l2, st));
  // W^T = Z Bm  (n x l1)
  SC4_TRY(tall_nn<T, T>(ws, n, l2, l1, 1.0, Z, n, Bm, l2, 0, 0.0, wt, n, st));
  return SC4DVAR_OK;
}

template <typename T>
static int build_singleview(Prob* P, const sc4dvar_sketch_opts& o, const double* Om_in,
                            const double* Psi_in, Prec* out, cudaStream_t st) {
  const int n = P->n, m = P->m;
  const int l1_0 = o.l;
  const int l2_0 = o.l2 > 0 ? o.l2 : 2 * l1_0 + 1;
  const bool adapt = o.adaptive != 0;
  const int lh1 = adapt ? (o.l_hat > 0 ? o.l_hat : std::max(1, l1_0 / 2)) : 0;
  const int lh2 = 2 * lh1;
  const int lmax = adapt ? (o.l_max > 0 ? o.l_max : std::min(8 * l1_0, n)) : l1_0;
  const int l2max = l2_0 + (lmax - l1_0) / std::max(1, lh1) * lh2;
  const uint64_t s_om = SC4DVAR_STREAM_SKETCH + (uint64_t)o.gn_iter;
  const uint64_t s_ps = s_om + SC4DVAR_STREAM_PSI;
  const uint64_t s_ka = SC4DVAR_STREAM_KAPPA + (uint64_t)o.gn_iter;
  SketchWS ws;
  ws.shifted = &P->counters.qr_shifted;
  ws.tall = o.gemm;
  Buf Om, Ps, Y, QY, Z, Wt, tmp, Mq, Mr, Mb;
  const int ldq = l2max, ldr = lmax;  // Q_M (l2 x l1) and R_M (l1 x l1) at their largest
  auto body = [&]() -> int {
    SC4_ARG(l2_0 >= l1_0, "SingleView needs l2 >= l1");
    SC4_TRY(Mq.ensure((size_t)ldq * lmax * sizeof(double)));
    SC4_TRY(Mr.ensure((size_t)ldr * lmax * sizeof(double)));
    SC4_TRY(Mb.ensure((size_t)l2_0 * l1_0 * sizeof(double)));
    SC4_CUDA(cudaMemsetAsync(Mr.p, 0, (size_t)ldr * lmax * sizeof(double), st));
    double *qm = Mq.as<double>(), *rm = Mr.as<double>();
    SC4_TRY(Om.ensure((size_t)n * lmax * sizeof(T)));
    SC4_TRY(Ps.ensure((size_t)m * l2max * sizeof(T)));
    SC4_TRY(Y.ensure((size_t)m * lmax * sizeof(T)));
    SC4_TRY(QY.ensure((size_t)m * lmax * sizeof(T)));
    SC4_TRY(Z.ensure((size_t)n * l2max * sizeof(T)));
    SC4_TRY(Wt.ensure((size_t)n * lmax * sizeof(T)));
    T *om = Om.as<T>(), *ps = Ps.as<T>(), *y = Y.as<T>(), *qy = QY.as<T>(), *z = Z.as<T>(),
      *wt = Wt.as<T>();
    SC4_TRY(draw_block<T>(P, Om_in, o.seed, s_om, n, l1_0, 0, om, n, tmp, st));
    SC4_TRY(draw_block<T>(P, Psi_in, o.seed, s_ps, m, l2_0, 0, ps, m, tmp, st));
    // Alg. 3 step 2: Y = A Omega and Z = A^T Psi (independent sweeps)
    SC4_TRY(tlm_block<T>(P, om, n, l1_0, y, m, st));
    SC4_TRY(adj_block<T>(P, ps, m, l2_0, z, n, (const T*)nullptr, 0, st));
    SC4_TRY(cholqr2<T>(m, l1_0, y, m, qy, m, ws, st));
    int l1 = l1_0, l2 = l2_0;
    // M = Psi^T Q_Y = Q_M R_M (Alg. 3 step 4)
    SC4_TRY(gemm_tn<T, T>(m, l2, l1, 1.0, ps, m, qy, m, 0.0, Mb.as<double>(), l2, st));
    SC4_TRY(qr_f64(l2, l1, Mb.as<double>(), l2, qm, ldq, rm, ldr, st));
    SC4_TRY(singleview_W<T>(P, l1, l2, qm, ldq, rm, ldr, z, wt, ws, st));
    if (adapt) {
      double kap;
      int t = 1;
      SC4_TRY(kappa_remark1<T>(P, l1, wt, n, o.seed, s_ka, t++, o.prec, ws, &kap, st));
      while (kap > o.eps_sk && l1 + lh1 <= lmax) {
        T* yh = y + (size_t)m * l1;
        SC4_TRY(draw_block<T>(P, nullptr, o.seed, s_om, n, lh1, l1, om + (size_t)n * l1, n, tmp, st));
        SC4_TRY(draw_block<T>(P, nullptr, o.seed, s_ps, m, lh2, l2, ps + (size_t)m * l2, m, tmp, st));
        SC4_TRY(tlm_block<T>(P, om + (size_t)n * l1, n, lh1, yh, m, st));
        SC4_TRY(adj_block<T>(P, ps + (size_t)m * l2, m, lh2, z + (size_t)n * l2, n, (const T*)nullptr, 0, st));
        SC4_TRY(ws.c.ensure((size_t)l1 * lh1 * sizeof(double)));
        for (int pass = 0; pass < 2; ++pass) {
          SC4_TRY(gemm_tn<T, T>(m, l1, lh1, 1.0, qy, m, yh, m, 0.0, ws.c.as<double>(), l1, st));
          SC4_TRY(tall_nn<T, T>(ws, m, l1, lh1, -1.0, qy, m, ws.c.as<double>(), l1, 0, 1.0, yh, m, st));
        }
        {
          // QR of the new block into Q_Y's next columns (cholqr2 needs its own c buffer)
          SketchWS ws2;
          ws2.shifted = &P->counters.qr_shifted;
          ws2.tall = o.gemm;
          int s2 = cholqr2<T>(m, lh1, yh, m, qy + (size_t)m * l1, m, ws2, st);
          cudaStreamSynchronize(st);
          ws2.release();
          SC4_TRY(s2);
        }
        // Alg. 6: QR of [Psi Psi_hat]^T [Q_Y Q_Y_hat] from the QR of Psi^T Q_Y
        SC4_TRY(qr_update<T>(m, l2, lh2, l1, lh1, ps, m, qy, m, qm, ldq, rm, ldr, st));
        l1 += lh1;
        l2 += lh2;
        SC4_TRY(singleview_W<T>(P, l1, l2, qm, ldq, rm, ldr, z, wt, ws, st));
        SC4_TRY(kappa_remark1<T>(P, l1, wt, n, o.seed, s_ka, t++, o.prec, ws, &kap, st));
      }
    }
    double drop = (sizeof(T) == 4) ? 1e-12 : 1e-15;
    SC4_TRY(finalize_svd<T>(P, l1, wt, n, 0.0, drop, out, ws, st));
    return SC4DVAR_OK;
  };
  int rc = body();
  cudaStreamSynchronize(st);
  ws.release(); Om.release(); Ps.release(); Y.release(); QY.release(); Z.release(); Wt.release();
  tmp.release(); Mq.release(); Mr.release(); Mb.release();
  return rc;
}

// ------------------------------------------------------------------ PCG
static int pcg_run(Prob* P, Prec* pc, const double* b, double* x, const sc4dvar_pcg_opts& o,
                   sc4dvar_pcg_info* info, cudaStream_t st) {
  const int n = P->n;
  const int maxit = o.maxit > 0 ? o.maxit : n;
  Buf wb;
  SC4_TRY(wb.ensure((size_t)6 * n * sizeof(double)));
  double* r = wb.as<double>();
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* e = q + n;
  double* rhs = e + n;
  double* sc = P->scal.as<double>();
  double* part = P->part.as<double>();
  if (pc && pc->l > 0) SC4_TRY(pc->T.ensure((size_t)pc->l * sizeof(double)));
  auto precond = [&](const double* src, double* dst) -> int {
    if (pc && pc->l > 0)
      return woodbury_apply(n, pc->l, 1, pc->V, n, pc->dsc, src, n, dst, n, pc->T.as<double>(), st);
    return copy_block<double, double>(n, 1, src, n, dst, n, st);
  };
  int total_its = 0, restarts = 0, status = SC4DVAR_OK;
  double bnorm;
  SC4_TRY(vnrm2<double>(n, b, sc, part, st));
  SC4_TRY(host_scalar(P, &bnorm, st));
  fill_kernel<<<div_up(n, 256), 256, 0, st>>>(n, 0.0, x);
  SC4_LAUNCH_CHECK();
  double relres = 0.0;
  if (bnorm == 0.0 || !std::isfinite(bnorm)) {
    // b = 0: x = 0 solves it; a non-finite b: a breakdown before the first iteration
    const bool ok = bnorm == 0.0;
    if (info) {
      info->iterations = 0;
      info->restarts = 0;
      info->relres = ok ? 0.0 : bnorm;
      info->status = ok ? SC4DVAR_OK : SC4DVAR_ERR_BREAKDOWN;
    }
    cudaStreamSynchronize(st);
    wb.release();
    return SC4DVAR_OK;
  }
  const int max_restarts = (o.prec == SC4DVAR_FP32) ? std::max(0, o.refine) : 0;
  // outer defect-correction loop: rhs = b - (I + H)_64 x; inner PCG solves for e
  SC4_TRY(copy_block<double, double>(n, 1, b, n, rhs, n, st));
  double rhs_norm = bnorm;
  for (int outer = 0;; ++outer) {
    fill_kernel<<<div_up(n, 256), 256, 0, st>>>(n, 0.0, e);
    SC4_LAUNCH_CHECK();
    SC4_TRY(copy_block<double, double>(n, 1, rhs, n, r, n, st));
    SC4_TRY(precond(r, z));
    SC4_TRY(copy_block<double, double>(n, 1, z, n, p, n, st));
    double rz;
    SC4_TRY(vdot<double, double>(n, r, z, sc, part, st));
    SC4_TRY(host_scalar(P, &rz, st));
    // inner tolerance relative to the current right-hand side
    double tol_in = o.tol * bnorm / rhs_norm;
    // an FP32 operator: solve a decade below the target so that one FP64 check
    // usually suffices; the recurrence residual itself is not limited by FP32
    if (o.prec == SC4DVAR_FP32) tol_in = std::max(0.1 * tol_in, 1e-7);
    status = SC4DVAR_ERR_NOT_CONVERGED;
    double rel_in = 1.0;
    int it = 0;
    while (it < maxit && total_its < maxit * (max_restarts + 1)) {
      ++it;
      ++total_its;
      NvtxRange r_it("sc4dvar PCG iteration");
      SC4_TRY(hvp_vec(P, p, q, o.prec, st));
      double pq;
      SC4_TRY(vdot<double, double>(n, p, q, sc, part, st));
      SC4_TRY(host_scalar(P, &pq, st));
      if (!(pq > 0.0) || !std::isfinite(pq)) { status = SC4DVAR_ERR_BREAKDOWN; break; }
      double alpha = rz / pq;
      SC4_TRY(axpby<double, double>(n, alpha, p, 1.0, e, st));
      SC4_TRY(axpby<double, double>(n, -alpha, q, 1.0, r, st));
      double rn;
      SC4_TRY(vnrm2<double>(n, r, sc, part, st));
      SC4_TRY(host_scalar(P, &rn, st));
      rel_in = rn / rhs_norm;
      if (rel_in <= tol_in) { status = SC4DVAR_OK; break; }
      SC4_TRY(precond(r, z));
      double rz_new;
      SC4_TRY(vdot<double, double>(n, r, z, sc, part, st));
      SC4_TRY(host_scalar(P, &rz_new, st));
      double beta = rz_new / rz;
      rz = rz_new;
      SC4_TRY(axpby<double, double>(n, 1.0, z, beta, p, st));
    }
    SC4_TRY(axpby<double, double>(n, 1.0, e, 1.0, x, st));
    if (o.prec != SC4DVAR_FP32) {
      relres = rel_in * rhs_norm / bnorm;
      break;
    }
    // FP64-class residual of the accumulated solution (counted as one online
    // HVP): double-float sweeps for periodic Burgers, FP64 otherwise
    SC4_TRY(hvp_vec(P, x, q, P->model == SC4DVAR_MODEL_BURGERS1D ? SC4DVAR_DF64 : SC4DVAR_FP64, st));
    SC4_TRY(copy_block<double, double>(n, 1, b, n, rhs, n, st));
    SC4_TRY(axpby<double, double>(n, -1.0, q, 1.0, rhs, st));
    SC4_TRY(vnrm2<double>(n, rhs, sc, part, st));
    SC4_TRY(host_scalar(P, &rhs_norm, st));
    relres = rhs_norm / bnorm;
    if (relres <= o.tol) { status = SC4DVAR_OK; break; }
    if (status == SC4DVAR_ERR_BREAKDOWN || outer >= max_restarts) {
      if (status == SC4DVAR_OK) status = SC4DVAR_ERR_NOT_CONVERGED;
      break;
    }
    ++restarts;
  }
  if (info) {
    info->iterations = total_its;
    info->restarts = restarts;
    info->relres = relres;
    info->status = status;
  }
  cudaStreamSynchronize(st);
  wb.release();
  return SC4DVAR_OK;
}

// ------------------------------------------------------------------ model runs
static int fwd_run(Prob* P, const double* v, double* J_host, double* d_out, cudaStream_t st) {
  NvtxRange r("sc4dvar FWD");
  const int n = P->n, m = P->m;
  if (v != P->v) SC4_CUDA(cudaMemcpyAsync(P->v, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SC4_TRY(prior_any<double, double, double>(P, 1, P->v, n, P->x0, n, P->xb, n, st));
  if (is_dir(P)) {
    SC4_TRY(dir_fwd(P->dir, P->x0, P->traj64, P->traj32, P->y, P->d, nullptr, nullptr, st));
  } else if (is_gyre(P)) {
    SC4_TRY(P->wGy.ensure(gyre_sweep_ws_bytes(P->gy, 1, 8)));
    SC4_TRY(gyre_fwd(P->gy, P->x0, true, P->y, P->d, nullptr, nullptr, P->wGy.p, st));
  } else if (is_bve(P)) {
    SC4_TRY(P->wBve.ensure(std::max(bve_fwd_ws_bytes(P->bve), bve_sweep_ws_bytes(P->bve, 1, 8))));
    SC4_TRY(bve_fwd(P->bve, P->x0, true, P->y, P->d, nullptr, nullptr, P->wBve.p, st));
  } else {
    SC4_TRY(burgers_fwd<double>(P->geom, P->x0, P->traj64, P->traj32, P->y, P->d, nullptr, nullptr, st));
  }
  P->have_traj = true;
  P->traj_df_valid = false;
  P->counters.fwd += 1;
  if (d_out) SC4_CUDA(cudaMemcpyAsync(d_out, P->d, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (J_host) {
    double a, b;
    SC4_TRY(vdot<double, double>(n, P->v, P->v, P->scal.as<double>(), P->part.as<double>(), st));
    SC4_TRY(host_scalar(P, &a, st));
    SC4_TRY(vdot<double, double>(m, P->d, P->d, P->scal.as<double>(), P->part.as<double>(), st));
    SC4_TRY(host_scalar(P, &b, st));
    *J_host = 0.5 * a + 0.5 * b;
  }
  return SC4DVAR_OK;
}

static int gradient_run(Prob* P, double* g, cudaStream_t st) {
  NvtxRange r("sc4dvar gradient (ADJ)");
  if (!P->have_traj) {
    set_error("gradient: no forward trajectory (call sc4dvar_fwd first)");
    return SC4DVAR_ERR_STATE;
  }
  const int n = P->n, m = P->m;
  SC4_TRY(P->wL.ensure((size_t)n * sizeof(double)));
  double* lam = P->wL.as<double>();
  SC4_TRY(model_adj<double>(P, P->d, m, 1, lam, n, st));
  SC4_TRY(prior_any<double, double, double>(P, 1, lam, n, g, n, P->v, n, st));
  P->counters.adj_online += 1;
  return SC4DVAR_OK;
}

static int build_precond_impl(Prob* P, const sc4dvar_sketch_opts& o, const double* Om,
                              const double* Ps, Prec** out, cudaStream_t st) {
  NvtxRange r("sc4dvar sketch");
  if (!P->have_traj) {
    set_error("build_precond: no forward trajectory (call sc4dvar_fwd first)");
    return SC4DVAR_ERR_STATE;
  }
  SC4_ARG(o.l >= 1 && o.l <= P->n, "sketch size l must be in [1, n]");
  SC4_ARG(o.prec == SC4DVAR_FP64 || o.prec == SC4DVAR_FP32, "prec");
  SC4_ARG(o.gemm >= SC4DVAR_GEMM_3XTF32 && o.gemm <= SC4DVAR_GEMM_BF16, "gemm mode");
  Prec* pc = new Prec();
  int saved = P->count_mode;
  P->count_mode = kOffline;
  int rc;
  bool f32 = o.prec == SC4DVAR_FP32;
  switch (o.method) {
    case SC4DVAR_SKETCH_RANDSVD:
      rc = f32 ? build_randsvd<float>(P, o, Om, pc, st) : build_randsvd<double>(P, o, Om, pc, st);
      break;
    case SC4DVAR_SKETCH_NYSTROM:
      rc = f32 ? build_nystrom<float>(P, o, Om, pc, st) : build_nystrom<double>(P, o, Om, pc, st);
      break;
    case SC4DVAR_SKETCH_SINGLEVIEW:
      rc = f32 ? build_singleview<float>(P, o, Om, Ps, pc, st)
               : build_singleview<double>(P, o, Om, Ps, pc, st);
      break;
    default:
      set_error("unknown sketch method");
      rc = SC4DVAR_ERR_INVALID_ARG;
  }
  P->count_mode = saved;
  if (rc == SC4DVAR_OK && f32) rc = tall_tc_take_error();
  if (rc != SC4DVAR_OK) {
    if (pc->V) cudaFree(pc->V);
    if (pc->lam) cudaFree(pc->lam);
    pc->T.release();
    delete pc;
    return rc;
  }
  *out = pc;
  return SC4DVAR_OK;
}

static void precond_free(Prec* pc) {
  if (!pc) return;
  if (pc->V) cudaFree(pc->V);
  if (pc->lam) cudaFree(pc->lam);
  pc->T.release();
  delete pc;
}

}  // namespace sc4

// =================================================================== C ABI
using namespace sc4;

extern "C" {

const char* sc4dvar_last_error(void) { return g_err.c_str(); }
int sc4dvar_version(void) { return 100; }
long long sc4dvar_launch_count(void) { return g_launches.load(); }

int sc4dvar_problem_create(const sc4dvar_problem_desc* d, sc4dvar_problem_t* out) {
  SC4_ARG(d && out, "null descriptor or output");
  SC4_ARG(d->model == SC4DVAR_MODEL_BURGERS1D || d->model == SC4DVAR_MODEL_BVE2D ||
              d->model == SC4DVAR_MODEL_BURGERS1D_DIRICHLET || d->model == SC4DVAR_MODEL_BVE_GYRE,
          "unknown model");
  const bool bve = d->model == SC4DVAR_MODEL_BVE2D;
  const bool dirm = d->model == SC4DVAR_MODEL_BURGERS1D_DIRICHLET;
  const bool gym = d->model == SC4DVAR_MODEL_BVE_GYRE;
  SC4_ARG(d->integrator == SC4DVAR_RK4 || ((dirm || gym) && d->integrator == SC4DVAR_RK3_TVD),
          "integrator: RK4, or RK3-TVD for the Dirichlet Burgers and double-gyre models");
  if (gym) {
    SC4_ARG(d->nx >= 8 && d->nx <= 128 && (d->nx & (d->nx - 1)) == 0 && d->ny == 2 * d->nx + 1,
            "double gyre: nx a power of two in [8, 128] and ny = 2 nx + 1");
    SC4_ARG(d->prior_kind == SC4DVAR_PRIOR_DIRICHLET_INV_HELMHOLTZ && d->prior_sigma >= 0 &&
                d->prior_length > 0,
            "double-gyre prior: SC4DVAR_PRIOR_DIRICHLET_INV_HELMHOLTZ with a = prior_sigma >= 0, "
            "b = prior_length > 0");
    SC4_ARG(d->forcing_amp > 0, "double gyre: forcing_amp = 1/Ro must be positive");
    SC4_ARG(d->n_checkpoints == 0, "checkpointing covers the doubly periodic BVE model (n_checkpoints must be 0)");
  } else if (dirm) {
    SC4_ARG(d->nx >= 3 && d->nx <= 1024 && d->ny == 1, "Dirichlet Burgers: n interior points in [3, 1024]");
    SC4_ARG(d->prior_kind == SC4DVAR_PRIOR_DIRICHLET_INV_HELMHOLTZ && d->prior_sigma > 0 &&
                d->prior_length >= 0,
            "Dirichlet Burgers prior: SC4DVAR_PRIOR_DIRICHLET_INV_HELMHOLTZ with a = prior_sigma > 0, "
            "b = prior_length >= 0");
    SC4_ARG(d->n_checkpoints == 0, "checkpointing covers the BVE model (n_checkpoints must be 0)");
  } else if (bve) {
    SC4_ARG(d->nx == d->ny && d->nx >= 16 && d->nx <= 1024 && (d->nx & (d->nx - 1)) == 0,
            "BVE grid must be N x N with N a power of two in [16, 1024]");
    SC4_ARG(d->prior_kind == SC4DVAR_PRIOR_INV_HELMHOLTZ && d->prior_sigma > 0 && d->prior_length >= 0,
            "BVE prior: SC4DVAR_PRIOR_INV_HELMHOLTZ with prior_sigma > 0, prior_length >= 0");
    SC4_ARG(d->n_checkpoints >= 0 && d->n_checkpoints <= d->n_steps,
            "n_checkpoints must lie in [0, n_steps]");
  } else {
    SC4_ARG(d->nx >= 8 && d->nx <= 8192 && (d->nx & (d->nx - 1)) == 0,
            "Burgers n must be a power of two in [8, 8192]");
    SC4_ARG(d->n_checkpoints == 0, "checkpointing covers the BVE model (n_checkpoints must be 0)");
  }
  int n = (bve || gym) ? d->nx * d->ny : d->nx;
  SC4_ARG(d->n_steps >= 1 && d->dt > 0 && d->nu >= 0, "time window");
  SC4_ARG(d->n_obs_times >= 1 && d->n_obs >= 1 && d->obs_steps && d->obs_idx, "observations");
  SC4_ARG(d->sigma_obs > 0, "sigma_obs must be positive");
  for (int i = 0; i < d->n_obs_times; ++i) {
    SC4_ARG(d->obs_steps[i] >= 1 && d->obs_steps[i] <= d->n_steps, "obs_steps must lie in [1, N]");
    SC4_ARG(i == 0 || d->obs_steps[i] > d->obs_steps[i - 1], "obs_steps must increase");
  }
  for (long i = 0; i < (long)d->n_obs_times * d->n_obs; ++i)
    SC4_ARG(d->obs_idx[i] >= 0 && d->obs_idx[i] < n, "obs_idx out of range");
  SC4_ARG(bve || dirm || gym || d->prior_kind == SC4DVAR_PRIOR_SE ||
              (d->prior_kind == SC4DVAR_PRIOR_SYMBOL && d->prior_symbol),
          "prior");
  SC4_ARG(d->prior_kind != SC4DVAR_PRIOR_SE || (d->prior_sigma > 0 && d->prior_length > 0),
          "SE prior parameters must be positive");
  Prob* P = new Prob();
  P->model = d->model;
  P->n = n;
  P->N = d->n_steps;
  P->n_t = d->n_obs_times;
  P->n_o = d->n_obs;
  P->m = P->n_t * P->n_o;
  P->nu = d->nu;
  P->h = d->dt;
  P->sigma = d->sigma_obs;
  auto fail = [&](int code) {
    sc4dvar_problem_destroy(P);
    return code;
  };
  std::vector<int> oos(P->N + 1, -1);
  for (int i = 0; i < P->n_t; ++i) oos[d->obs_steps[i]] = i;
  P->obs_of_step_h = oos;
  size_t traj_pts = (bve || gym) ? 0 : (size_t)(P->N + 1) * n;
  if (bve) {
    const int Ng = d->nx;
    // Checkpointing: L = ceil(N / c) steps per segment; the stage-state buffers
    // hold one segment, the FP64 checkpoints one state per segment.
    const int L = d->n_checkpoints > 0 ? (P->N + d->n_checkpoints - 1) / d->n_checkpoints : 0;
    const int n_seg = L > 0 ? (P->N + L - 1) / L : 0;
    P->bve.ckpt_every = L;
    size_t stages = (size_t)4 * (L > 0 ? L : P->N) * n;
    if (L > 0) {
      BveGeom tmp{};
      tmp.N = Ng;
      if (cudaMalloc(&P->bve_ckpt, (size_t)n_seg * n * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&P->bve_rws, bve_fwd_ws_bytes(tmp)) != cudaSuccess) {
        cudaGetLastError();
        set_error("problem_create: device allocation of the BVE checkpoints failed");
        return fail(SC4DVAR_ERR_OOM);
      }
    }
    if (cudaMalloc(&P->bve_tw64, (Ng / 2) * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&P->bve_tw32, (Ng / 2) * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&P->bve_poisson, (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->bve_prior, (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->bve_tabc64, 2 * (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->bve_tabc32, 2 * (size_t)n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&P->bve_q64, stages * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->bve_p64, stages * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&P->bve_q32, stages * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&P->bve_p32, stages * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      set_error("problem_create: device allocation of the BVE stage states failed");
      return fail(SC4DVAR_ERR_OOM);
    }
  }
  if (cudaMalloc(&P->obs_of_step, oos.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&P->obs_idx, (size_t)P->m * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&P->sym, (bve || dirm || gym ? 1 : n) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&P->tw, (bve || dirm || gym ? 1 : n / 2) * sizeof(double2)) != cudaSuccess ||
      (dirm && cudaMalloc(&P->dir_cp, 2 * (size_t)n * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&P->xb, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&P->y, P->m * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&P->v, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&P->x0, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&P->d, P->m * sizeof(double)) != cudaSuccess ||
      (traj_pts && cudaMalloc(&P->traj64, traj_pts * sizeof(double)) != cudaSuccess) ||
      (traj_pts && cudaMalloc(&P->traj32, traj_pts * sizeof(float)) != cudaSuccess)) {
    cudaGetLastError();
    set_error("problem_create: device allocation failed");
    return fail(SC4DVAR_ERR_OOM);
  }
  int rc;
  if ((rc = P->part.ensure(1024 * sizeof(double))) || (rc = P->scal.ensure(64 * sizeof(double))))
    return fail(rc);
  if (cudaMemcpy(P->obs_of_step, oos.data(), oos.size() * sizeof(int), cudaMemcpyHostToDevice) ||
      cudaMemcpy(P->obs_idx, d->obs_idx, (size_t)P->m * sizeof(int), cudaMemcpyHostToDevice) ||
      cudaMemset(P->xb, 0, n * sizeof(double)) || cudaMemset(P->y, 0, P->m * sizeof(double)) ||
      cudaMemset(P->v, 0, n * sizeof(double))) {
    set_error("problem_create: copy failed");
    return fail(SC4DVAR_ERR_CUDA);
  }
  P->geom.n = n;
  P->geom.N = P->N;
  P->geom.h = P->h;
  P->geom.nu = P->nu;
  P->geom.sigma = P->sigma;
  P->geom.n_t = P->n_t;
  P->geom.n_o = P->n_o;
  P->geom.obs_of_step = P->obs_of_step;
  P->geom.obs_idx = P->obs_idx;
  P->geom.fold32 = (!bve && !dirm && !gym && packed_f32_supported(n)) ? 1 : 0;
  if (bve) {
    BveGeom& b = P->bve;
    b.N = d->nx;
    b.Nsteps = P->N;
    b.n_t = P->n_t;
    b.n_o = P->n_o;
    b.h = P->h;
    b.nu = P->nu;
    b.sigma = P->sigma;
    b.famp = d->forcing_amp;
    b.fk = d->forcing_k;
    b.prior_c = d->prior_sigma;
    b.prior_ell = d->prior_length;
    b.obs_of_step_h = P->obs_of_step_h.data();
    b.obs_idx = P->obs_idx;
    b.tw64 = P->bve_tw64;
    b.tw32 = P->bve_tw32;
    b.poisson = P->bve_poisson;
    b.prior = P->bve_prior;
    b.poisson_c64 = P->bve_tabc64;
    b.prior_c64 = P->bve_tabc64 + n;
    b.poisson_c32 = P->bve_tabc32;
    b.prior_c32 = P->bve_tabc32 + n;
    b.q64 = P->bve_q64;
    b.p64 = P->bve_p64;
    b.q32 = P->bve_q32;
    b.p32 = P->bve_p32;
    b.ckpt = P->bve_ckpt;
    b.rws = P->bve_rws;
    if ((rc = bve_setup(b, 0))) return fail(rc);
  } else if (gym) {
    GyreGeom& g = P->gy;
    g.nx = d->nx;
    g.ny = d->ny;
    g.n = n;
    g.N = P->N;
    g.n_t = P->n_t;
    g.n_o = P->n_o;
    g.dt = P->h;
    g.h = 1.0 / (d->nx + 1);
    g.re_inv = d->nu;
    g.ro_inv = d->forcing_amp;
    g.sigma = P->sigma;
    for (int i = 0; i < 4; ++i) {
      g.b[i] = 0.0;
      for (int j = 0; j < 4; ++j) g.a[i][j] = 0.0;
    }
    if (d->integrator == SC4DVAR_RK3_TVD) {
      g.S = 3;
      g.a[1][0] = 1.0;
      g.a[2][0] = 0.25;
      g.a[2][1] = 0.25;
      g.b[0] = 1.0 / 6.0;
      g.b[1] = 1.0 / 6.0;
      g.b[2] = 2.0 / 3.0;
    } else {
      g.S = 4;
      g.a[1][0] = 0.5;
      g.a[2][1] = 0.5;
      g.a[3][2] = 1.0;
      g.b[0] = g.b[3] = 1.0 / 6.0;
      g.b[1] = g.b[2] = 1.0 / 3.0;
    }
    g.obs_of_step = P->obs_of_step;
    g.obs_of_step_h = P->obs_of_step_h.data();
    g.obs_idx = P->obs_idx;
    const size_t nn = (size_t)g.nx * g.nx, f = 2 * (size_t)g.nx * g.ny;
    const size_t st_pts = (size_t)g.N * g.S * n;
    if (cudaMalloc(&P->gy_setup, gyre_setup_bytes(g.nx)) != cudaSuccess ||
        cudaMalloc(&P->gy_stages, gyre_stage_bytes(g.nx, g.N, g.S)) != cudaSuccess) {
      cudaGetLastError();
      set_error("problem_create: device allocation of the double-gyre arrays failed");
      return fail(SC4DVAR_ERR_OOM);
    }
    char* b = static_cast<char*>(P->gy_setup);
    g.S64 = reinterpret_cast<double*>(b);
    g.pois64 = reinterpret_cast<double*>(b + nn * 8);
    g.prior64 = reinterpret_cast<double*>(b + nn * 8 + f * 8);
    g.Fy = reinterpret_cast<double*>(b + nn * 8 + 2 * f * 8);
    char* b4 = b + nn * 8 + 2 * f * 8 + (size_t)g.ny * 8;
    g.S32 = reinterpret_cast<float*>(b4);
    g.S_tc = g.nx == 128 ? static_cast<void*>(b + gyre_tc_offset(g.nx)) : nullptr;
    g.pois32 = reinterpret_cast<float*>(b4 + nn * 4);
    g.prior32 = reinterpret_cast<float*>(b4 + nn * 4 + f * 4);
    char* sb = static_cast<char*>(P->gy_stages);
    g.om64 = reinterpret_cast<double*>(sb);
    g.ps64 = reinterpret_cast<double*>(sb + st_pts * 8);
    g.om32 = reinterpret_cast<float*>(sb + 2 * st_pts * 8);
    g.ps32 = reinterpret_cast<float*>(sb + 2 * st_pts * 8 + st_pts * 4);
    if ((rc = gyre_setup(g, d->prior_sigma, d->prior_length, 0))) return fail(rc);
  } else if ((rc = fft_make_twiddles(n, P->tw, 0))) {
    return fail(rc);
  }
  if (dirm) {
    DirGeom& g = P->dir;
    g.n = n;
    g.N = P->N;
    g.n_o = P->n_o;
    g.h = P->h;
    g.nu = P->nu;
    g.sigma = P->sigma;
    g.obs_of_step = P->obs_of_step;
    g.obs_idx = P->obs_idx;
    for (int i = 0; i < 4; ++i) {
      g.b[i] = 0.0;
      for (int j = 0; j < 4; ++j) g.a[i][j] = 0.0;
    }
    if (d->integrator == SC4DVAR_RK3_TVD) {  // Butcher form of the TVD scheme
      g.S = 3;
      g.a[1][0] = 1.0;
      g.a[2][0] = 0.25;
      g.a[2][1] = 0.25;
      g.b[0] = 1.0 / 6.0;
      g.b[1] = 1.0 / 6.0;
      g.b[2] = 2.0 / 3.0;
    } else {
      g.S = 4;
      g.a[1][0] = 0.5;
      g.a[2][1] = 0.5;
      g.a[3][2] = 1.0;
      g.b[0] = g.b[3] = 1.0 / 6.0;
      g.b[1] = g.b[2] = 1.0 / 3.0;
    }
    g.cp = P->dir_cp;
    g.den = P->dir_cp + n;
    g.work = nullptr;
    g.work_cols = 0;
    if ((rc = dir_setup(g, d->prior_sigma, d->prior_length, 0))) return fail(rc);
  } else if (bve || gym) {
    // prior handled by the 2D multiplier / the sine-transform solve
  } else if (d->prior_kind == SC4DVAR_PRIOR_SE) {
    if ((rc = fft_se_symbol(n, d->prior_sigma, d->prior_length, kClampRel, P->tw, P->sym, 0)))
      return fail(rc);
  } else {
    if (cudaMemcpy(P->sym, d->prior_symbol, n * sizeof(double), cudaMemcpyHostToDevice)) {
      set_error("problem_create: symbol copy failed");
      return fail(SC4DVAR_ERR_CUDA);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error(std::string("problem_create: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(SC4DVAR_ERR_CUDA);
  }
  *out = P;
  return SC4DVAR_OK;
}

int sc4dvar_problem_destroy(sc4dvar_problem_t P) {
  if (!P) return SC4DVAR_OK;
  cudaFree(P->obs_of_step); cudaFree(P->obs_idx); cudaFree(P->sym); cudaFree(P->tw);
  cudaFree(P->xb); cudaFree(P->y); cudaFree(P->v); cudaFree(P->x0); cudaFree(P->d);
  cudaFree(P->traj64); cudaFree(P->traj32); cudaFree(P->dir_cp); cudaFree(P->traj_df);
  P->wDF.release();
  P->wDir.release();
  cudaFree(P->gy_setup);
  cudaFree(P->gy_stages);
  P->wGy.release();
  P->wGyPrior.release();
  cudaFree(P->bve_tw64); cudaFree(P->bve_tw32); cudaFree(P->bve_poisson); cudaFree(P->bve_prior);
  cudaFree(P->bve_tabc64); cudaFree(P->bve_tabc32);
  cudaFree(P->bve_q64); cudaFree(P->bve_p64); cudaFree(P->bve_q32); cudaFree(P->bve_p32);
  cudaFree(P->bve_ckpt); cudaFree(P->bve_rws);
  for (auto& g : P->hvp_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (P->graph_stream) cudaStreamDestroy(P->graph_stream);
  P->wBve.release(); P->wCplx.release();
  P->wU.release(); P->wW.release(); P->wL.release(); P->part.release(); P->scal.release();
  P->vec.release();
  delete P;
  return SC4DVAR_OK;
}

int sc4dvar_problem_dims(sc4dvar_problem_t P, int* n, int* m) {
  SC4_ARG(P, "null problem");
  if (n) *n = P->n;
  if (m) *m = P->m;
  return SC4DVAR_OK;
}

int sc4dvar_set_background(sc4dvar_problem_t P, const double* xb, void* stream) {
  SC4_ARG(P && xb, "null argument");
  SC4_CUDA(cudaMemcpyAsync(P->xb, xb, P->n * sizeof(double), cudaMemcpyDeviceToDevice, S(stream)));
  P->have_traj = false;
  return SC4DVAR_OK;
}

int sc4dvar_set_observations(sc4dvar_problem_t P, const double* y, void* stream) {
  SC4_ARG(P && y, "null argument");
  SC4_CUDA(cudaMemcpyAsync(P->y, y, P->m * sizeof(double), cudaMemcpyDeviceToDevice, S(stream)));
  P->have_traj = false;
  return SC4DVAR_OK;
}

int sc4dvar_prior_sqrt_apply(sc4dvar_problem_t P, const double* X, int ldx, int k, double* Y,
                             int ldy, void* stream) {
  SC4_ARG(P && k >= 0 && (k == 0 || (X && Y)) && ldx >= P->n && ldy >= P->n, "prior_sqrt_apply arguments");
  return prior_any<double, double, double>(P, k, X, ldx, Y, ldy, (const double*)nullptr, 0, S(stream));
}

int sc4dvar_prior_symbol(sc4dvar_problem_t P, double* symbol_host) {
  SC4_ARG(P && symbol_host, "null argument");
  SC4_ARG(!is_dir(P) && !is_gyre(P), "the Dirichlet prior has no Fourier symbol");
  if (is_bve(P)) {
    SC4_CUDA(cudaMemcpy(symbol_host, P->bve.prior, P->n * sizeof(double), cudaMemcpyDeviceToHost));
    return SC4DVAR_OK;
  }
  SC4_CUDA(cudaMemcpy(symbol_host, P->sym, P->n * sizeof(double), cudaMemcpyDeviceToHost));
  return SC4DVAR_OK;
}

int sc4dvar_forecast(sc4dvar_problem_t P, const double* x0, double* obs, double* xN, void* stream) {
  SC4_ARG(P && x0 && obs, "null argument");
  if (is_dir(P)) return dir_fwd(P->dir, x0, nullptr, nullptr, nullptr, nullptr, obs, xN, S(stream));
  if (is_gyre(P)) {
    SC4_TRY(P->wGy.ensure(gyre_sweep_ws_bytes(P->gy, 1, 8)));
    return gyre_fwd(P->gy, x0, false, nullptr, nullptr, obs, xN, P->wGy.p, S(stream));
  }
  if (is_bve(P)) {
    SC4_TRY(P->wBve.ensure(std::max(bve_fwd_ws_bytes(P->bve), P->wBve.bytes)));
    return bve_fwd(P->bve, x0, false, nullptr, nullptr, obs, xN, P->wBve.p, S(stream));
  }
  return burgers_fwd<double>(P->geom, x0, nullptr, nullptr, nullptr, nullptr, obs, xN, S(stream));
}

int sc4dvar_fwd(sc4dvar_problem_t P, const double* v, double* J_host, double* d_dev, void* stream) {
  SC4_ARG(P && v, "null argument");
  return fwd_run(P, v, J_host, d_dev, S(stream));
}

int sc4dvar_gradient(sc4dvar_problem_t P, double* g, void* stream) {
  SC4_ARG(P && g, "null argument");
  return gradient_run(P, g, S(stream));
}

static int check_block(sc4dvar_problem_t P, int k, int prec) {
  SC4_ARG(P, "null problem");
  SC4_ARG(k >= 0, "k must be >= 0");
  SC4_ARG(prec == SC4DVAR_FP64 || prec == SC4DVAR_FP32, "prec must be SC4DVAR_FP64 or SC4DVAR_FP32");
  if (!P->have_traj) {
    set_error("no forward trajectory (call sc4dvar_fwd first)");
    return SC4DVAR_ERR_STATE;
  }
  return SC4DVAR_OK;
}

int sc4dvar_tlm_block(sc4dvar_problem_t P, const void* X, int ldx, int k, void* W, int ldw, int prec,
                      void* stream) {
  SC4_TRY(check_block(P, k, prec));
  SC4_ARG(ldx >= P->n && ldw >= P->m && (k == 0 || (X && W)), "leading dimensions / pointers");
  if (prec == SC4DVAR_FP64)
    return tlm_block<double>(P, (const double*)X, ldx, k, (double*)W, ldw, S(stream));
  return tlm_block<float>(P, (const float*)X, ldx, k, (float*)W, ldw, S(stream));
}

int sc4dvar_adj_block(sc4dvar_problem_t P, const void* W, int ldw, int k, void* X, int ldx, int prec,
                      void* stream) {
  SC4_TRY(check_block(P, k, prec));
  SC4_ARG(ldx >= P->n && ldw >= P->m && (k == 0 || (X && W)), "leading dimensions / pointers");
  if (prec == SC4DVAR_FP64)
    return adj_block<double>(P, (const double*)W, ldw, k, (double*)X, ldx, (const double*)nullptr, 0,
                             S(stream));
  return adj_block<float>(P, (const float*)W, ldw, k, (float*)X, ldx, (const float*)nullptr, 0,
                          S(stream));
}

int sc4dvar_gn_hessian_apply_block(sc4dvar_problem_t P, const void* X, int ldx, int k, void* Y,
                                   int ldy, int misfit_only, int prec, void* stream) {
  if (P && prec == SC4DVAR_DF64) {
    SC4_ARG(P->model == SC4DVAR_MODEL_BURGERS1D, "SC4DVAR_DF64 needs the periodic Burgers model");
    SC4_TRY(check_block(P, k, SC4DVAR_FP64));
    SC4_ARG(ldx >= P->n && ldy >= P->n && (k == 0 || (X && Y)), "leading dimensions / pointers");
    return hvp_block_df64(P, (const double*)X, ldx, k, (double*)Y, ldy, misfit_only, S(stream));
  }
  SC4_TRY(check_block(P, k, prec));
  SC4_ARG(ldx >= P->n && ldy >= P->n && (k == 0 || (X && Y)), "leading dimensions / pointers");
  if (prec == SC4DVAR_FP64)
    return hvp_block<double>(P, (const double*)X, ldx, k, (double*)Y, ldy, misfit_only, S(stream));
  return hvp_block<float>(P, (const float*)X, ldx, k, (float*)Y, ldy, misfit_only, S(stream));
}

int sc4dvar_build_precond(sc4dvar_problem_t P, const sc4dvar_sketch_opts* o, const double* Om,
                          const double* Ps, sc4dvar_precond_t* out, void* stream) {
  SC4_ARG(P && o && out, "null argument");
  return build_precond_impl(P, *o, Om, Ps, out, S(stream));
}

int sc4dvar_tall_gemm(int mode, int rows, int kk, int c, double alpha, const float* A, int lda, const double* B,
                      int ldb, int transB, double beta, void* C, int c_double, int ldc, void* stream) {
  SC4_ARG(mode >= SC4DVAR_GEMM_3XTF32 && mode <= SC4DVAR_GEMM_BF16, "gemm mode");
  SC4_ARG(rows >= 0 && kk >= 0 && c >= 0, "sizes");
  SC4_ARG(rows == 0 || c == 0 || (A && B && C), "pointers");
  SC4_ARG(lda >= std::max(rows, 1) && ldc >= std::max(rows, 1) && ldb >= std::max(transB ? c : kk, 1),
          "leading dimensions");
  cudaStream_t st = S(stream);
  SketchWS ws;
  ws.tall = mode;
  if (c_double)
    SC4_TRY(tall_nn<float, double>(ws, rows, kk, c, alpha, A, lda, B, ldb, transB, beta, (double*)C, ldc, st));
  else
    SC4_TRY(tall_nn<float, float>(ws, rows, kk, c, alpha, A, lda, B, ldb, transB, beta, (float*)C, ldc, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  ws.release();
  return tall_tc_take_error();
}

int sc4dvar_precond_destroy(sc4dvar_precond_t pc) {
  precond_free(pc);
  return SC4DVAR_OK;
}

int sc4dvar_precond_info(sc4dvar_precond_t pc, int* rank, double* lam_host, double* V_host) {
  SC4_ARG(pc, "null preconditioner");
  if (rank) *rank = pc->l;
  if (pc->l > 0) {
    if (lam_host) SC4_CUDA(cudaMemcpy(lam_host, pc->lam, pc->l * sizeof(double), cudaMemcpyDeviceToHost));
    if (V_host)
      SC4_CUDA(cudaMemcpy(V_host, pc->V, (size_t)pc->n * pc->l * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return SC4DVAR_OK;
}

int sc4dvar_precond_apply(sc4dvar_precond_t pc, const double* R, int ldr, int k, double* Z, int ldz,
                          void* stream) {
  SC4_ARG(pc && k >= 0 && (k == 0 || (R && Z)) && ldr >= pc->n && ldz >= pc->n, "precond_apply arguments");
  if (k == 0) return SC4DVAR_OK;
  SC4_TRY(pc->T.ensure((size_t)std::max(pc->l, 1) * std::max(k, 1) * sizeof(double)));
  return woodbury_apply(pc->n, pc->l, k, pc->V, pc->n, pc->dsc, R, ldr, Z, ldz, pc->T.as<double>(),
                        S(stream));
}

int sc4dvar_kappa_estimate(sc4dvar_problem_t P, sc4dvar_precond_t pc, uint64_t seed,
                           uint64_t stream_id, int column, double* kappa, void* stream) {
  SC4_ARG(P && kappa, "null argument");
  SC4_TRY(check_block(P, 1, SC4DVAR_FP64));
  return kappa_precond(P, pc, seed, stream_id, column, SC4DVAR_FP64, kappa, S(stream));
}

int sc4dvar_pcg(sc4dvar_problem_t P, sc4dvar_precond_t pc, const double* b, double* x,
                const sc4dvar_pcg_opts* o, sc4dvar_pcg_info* info, void* stream) {
  SC4_ARG(P && b && x && o, "null argument");
  SC4_TRY(check_block(P, 1, o->prec));
  SC4_ARG(o->tol > 0, "tol must be positive");
  SC4_ARG(!pc || pc->n == P->n, "preconditioner size");
  return pcg_run(P, pc, b, x, *o, info, S(stream));
}

int sc4dvar_sketchsolv(sc4dvar_precond_t pc, const double* g, double* dv, void* stream) {
  SC4_ARG(pc && g && dv, "null argument");
  SC4_TRY(pc->T.ensure((size_t)std::max(pc->l, 1) * sizeof(double)));
  SC4_TRY(woodbury_apply(pc->n, pc->l, 1, pc->V, pc->n, pc->dsc, g, pc->n, dv, pc->n,
                         pc->T.as<double>(), S(stream)));
  return axpby<double, double>(pc->n, 0.0, dv, -1.0, dv, S(stream));
}

int sc4dvar_qr_update(int m, int r1, int r2, int k1, int k2, const double* Pm, int ldp, const double* B,
                      int ldb, double* Q, int ldq, double* R, int ldr, void* stream) {
  SC4_ARG(m >= 0 && r1 >= 0 && r2 >= 0 && k1 >= 0 && k2 >= 0, "qr_update: negative size");
  SC4_ARG(r1 >= k1 && r1 + r2 >= k1 + k2, "qr_update: needs r1 >= k1 and r1 + r2 >= k1 + k2 (thin QR)");
  SC4_ARG(Pm && B && Q && R, "qr_update: null argument");
  SC4_ARG(ldp >= std::max(m, 1) && ldb >= std::max(m, 1) && ldq >= std::max(r1 + r2, 1) &&
              ldr >= std::max(k1 + k2, 1),
          "qr_update: leading dimensions");
  return qr_update<double>(m, r1, r2, k1, k2, Pm, ldp, B, ldb, Q, ldq, R, ldr, S(stream));
}

// ------------------------------------------------------------------ line search
// Strong-Wolfe step length along dv from v (bracketing and zoom of Nocedal &
// Wright, Algs. 3.5 / 3.6, cubic interpolation kept 10 % inside the bracket,
// else bisection; values equal to within rounding leave the decision to the
// derivative). phi(a) = J(v + a dv) by a FWD, phi'(a) = g(v + a dv)^T dv by the
// gradient. On return, g holds the gradient at the last trial point and
// `last` says whether that point is the accepted step.
namespace {
constexpr int kLsOk = 0, kLsNotDescent = 1, kLsMaxEvals = 2;

bool cubic_min(double a, double fa, double da, double b, double fb, double db, double* out) {
  if (a == b) return false;
  const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
  const double disc = d1 * d1 - da * db;
  if (disc < 0.0) return false;
  const double d2 = std::copysign(std::sqrt(disc), b - a);
  const double den = db - da + 2.0 * d2;
  if (den == 0.0) return false;
  *out = b - (b - a) * (db + d2 - d1) / den;
  return true;
}

struct LsResult {
  double alpha = 1.0, phi = 0.0;
  int evals = 0, status = kLsOk;
  bool last = false;
};
}  // namespace

static int line_search(Prob* P, const double* v, const double* dv, double* vt, double* g, double phi0,
                       double dphi0, double alpha1, double c1, double c2, LsResult* out, cudaStream_t st) {
  const int n = P->n;
  const double alpha_max = 10.0, eps = std::ldexp(1.0, -52);
  const int max_evals = 30;
  LsResult r;
  if (!(dphi0 < 0.0)) {
    r.alpha = alpha1;
    r.status = kLsNotDescent;
    *out = r;
    return SC4DVAR_OK;
  }
  auto ev = [&](double a, double* f, double* d) -> int {
    ++r.evals;
    SC4_TRY(copy_block<double, double>(n, 1, v, n, vt, n, st));
    SC4_TRY(axpby<double, double>(n, a, dv, 1.0, vt, st));
    SC4_TRY(fwd_run(P, vt, f, nullptr, st));
    SC4_TRY(gradient_run(P, g, st));
    SC4_TRY(vdot<double, double>(n, g, dv, P->scal.as<double>(), P->part.as<double>(), st));
    return host_scalar(P, d, st);
  };
  auto finish = [&](double a, double f, int status, bool last) {
    r.alpha = a;
    r.phi = f;
    r.status = status;
    r.last = last;
    *out = r;
    return SC4DVAR_OK;
  };
  auto zoom = [&](double lo, double flo, double dlo, double hi, double fhi, double dhi) -> int {
    while (r.evals < max_evals) {
      const double width = hi - lo;
      double a;
      const double lo_b = std::min(lo, hi), hi_b = std::max(lo, hi), pad = 0.1 * std::fabs(width);
      if (!cubic_min(lo, flo, dlo, hi, fhi, dhi, &a) || !(lo_b + pad <= a && a <= hi_b - pad))
        a = 0.5 * (lo + hi);
      double f, d;
      SC4_TRY(ev(a, &f, &d));
      const bool flat = std::fabs(f - flo) <= 16.0 * eps * std::max(std::fabs(f), std::fabs(flo));
      if (f > phi0 + c1 * a * dphi0 || (f >= flo && !flat)) {
        hi = a; fhi = f; dhi = d;
      } else {
        if (std::fabs(d) <= -c2 * dphi0) return finish(a, f, kLsOk, true);
        if (d * (hi - lo) >= 0.0) { hi = lo; fhi = flo; dhi = dlo; }
        lo = a; flo = f; dlo = d;
      }
    }
    return finish(lo, flo, kLsMaxEvals, false);
  };
  double a_prev = 0.0, f_prev = phi0, d_prev = dphi0, a = alpha1;
  bool first = true;
  while (r.evals < max_evals) {
    double f, d;
    SC4_TRY(ev(a, &f, &d));
    if (f > phi0 + c1 * a * dphi0 || (!first && f >= f_prev)) return zoom(a_prev, f_prev, d_prev, a, f, d);
    if (std::fabs(d) <= -c2 * dphi0) return finish(a, f, kLsOk, true);
    if (d >= 0.0) return zoom(a, f, d, a_prev, f_prev, d_prev);
    a_prev = a; f_prev = f; d_prev = d;
    a = std::min(2.0 * a, alpha_max);
    if (a == a_prev) return finish(a, f, kLsMaxEvals, true);
    first = false;
  }
  return finish(a_prev, f_prev, kLsMaxEvals, false);
}

int sc4dvar_gauss_newton_resume(sc4dvar_problem_t P, const sc4dvar_gn_opts* o, double* v_io,
                                sc4dvar_gn_state* state, sc4dvar_precond_t* held, sc4dvar_gn_info* info,
                                void* stream) {
  SC4_ARG(P && o && v_io && state && held, "null argument");
  SC4_ARG(o->iters >= 1 && o->iters <= SC4DVAR_GN_MAX_ITERS, "iters");
  SC4_ARG(state->next_iter >= 0 && state->next_iter <= o->iters, "state->next_iter in [0, iters]");
  SC4_ARG(state->next_iter > 0 || *held == nullptr, "a new run (next_iter = 0) holds no preconditioner");
  SC4_ARG(*held == nullptr || (*held)->n == P->n, "held preconditioner of another size");
  SC4_ARG(*held == nullptr || o->sketch.method != SC4DVAR_SKETCH_NONE,
          "a held preconditioner needs a sketch method (method NONE runs Prec_Gamma)");
  SC4_ARG(!o->line_search || (o->ls_c1 > 0 && o->ls_c1 < o->ls_c2 && o->ls_c2 < 1 && o->ls_alpha1 > 0),
          "line search constants: 0 < c1 < c2 < 1, alpha1 > 0");
  SC4_ARG(o->solve == 0 || (o->solve == 1 && o->sketch.method != SC4DVAR_SKETCH_NONE),
          "solve: 0 (PCG) or 1 (SketchSolv, needs a sketch method)");
  cudaStream_t st = S(stream);
  const int n = P->n;
  const int k0 = state->next_iter;
  if (info && k0 == 0) std::memset(info, 0, sizeof(*info));
  if (info && k0 > 0) {
    // the entries of this call start clean; those of earlier calls are kept
    for (int i = k0; i < SC4DVAR_GN_MAX_ITERS; ++i) {
      info->J[i] = info->g_inf[i] = info->relres[i] = info->kappa_re[i] = info->alpha[i] = 0.0;
      info->pcg_its[i] = info->sketched[i] = info->rank[i] = info->ls_evals[i] = info->ls_status[i] = 0;
    }
  }
  Buf gb;
  SC4_TRY(gb.ensure((size_t)3 * n * sizeof(double)));
  double* g = gb.as<double>();
  double* dv = g + n;
  double* vt = dv + n;
  Prec* pc = *held;
  *held = nullptr;
  double g0 = k0 > 0 ? state->g0_inf : 0.0;
  int sketch_iter = pc ? state->sketch_iter : -1;
  int rc = SC4DVAR_OK;
  bool carry = false;  // J and g at v_io come from the last line-search trial
  double J = 0.0;
  int k = k0;
  char label[48];
  for (; k < o->iters; ++k) {
    std::snprintf(label, sizeof(label), "sc4dvar GN iteration %d", k);
    NvtxRange r_it(label);
    if (!carry) {
      if ((rc = fwd_run(P, v_io, &J, nullptr, st))) break;
      if ((rc = gradient_run(P, g, st))) break;
    }
    carry = false;
    double ginf;
    if ((rc = vamax(n, g, P->scal.as<double>(), P->part.as<double>(), st))) break;
    if ((rc = host_scalar(P, &ginf, st))) break;
    if (k == 0) g0 = ginf;
    if (info) {
      info->J[k] = J;
      info->g_inf[k] = ginf;
      info->iters_done = k + 1;
    }
    if (k > 0 && o->gtol > 0 && ginf / g0 < o->gtol) break;
    if (o->sketch.method != SC4DVAR_SKETCH_NONE) {
      NvtxRange r_sk("sc4dvar sketch or reuse");
      bool need = (pc == nullptr) || !o->sketch.adaptive;
      if (!need) {
        double kre;
        if ((rc = kappa_precond(P, pc, o->sketch.seed, SC4DVAR_STREAM_KAPPA + k, 0, o->sketch.prec,
                                &kre, st)))
          break;
        if (info) info->kappa_re[k] = kre;
        need = !(kre < o->eps_re);
      }
      if (need) {
        precond_free(pc);
        pc = nullptr;
        sketch_iter = -1;
        sc4dvar_sketch_opts so = o->sketch;
        so.gn_iter = k;
        if ((rc = build_precond_impl(P, so, nullptr, nullptr, &pc, st))) break;
        sketch_iter = k;
        if (info) info->sketched[k] = 1;
      }
      if (info) info->rank[k] = pc->l;
    }
    // b = -g
    if ((rc = axpby<double, double>(n, -1.0, g, 0.0, g, st))) break;
    if (o->solve == 1) {
      // SketchSolv (Eq. dxsol): dv = (I + H_hat)^{-1} b, b = -g
      if ((rc = pc->T.ensure((size_t)std::max(pc->l, 1) * sizeof(double)))) break;
      if ((rc = woodbury_apply(n, pc->l, 1, pc->V, n, pc->dsc, g, n, dv, n, pc->T.as<double>(), st))) break;
    } else {
      sc4dvar_pcg_info pi{};
      if ((rc = pcg_run(P, pc, g, dv, o->pcg, &pi, st))) break;
      if (info) {
        info->pcg_its[k] = pi.iterations;
        info->relres[k] = pi.relres;
      }
    }
    double alpha = 1.0;
    if (o->line_search) {
      NvtxRange r_ls("sc4dvar line search");
      // phi'(0) = g^T dv with g = -b
      double gdv;
      if ((rc = vdot<double, double>(n, g, dv, P->scal.as<double>(), P->part.as<double>(), st))) break;
      if ((rc = host_scalar(P, &gdv, st))) break;
      LsResult ls;
      if ((rc = line_search(P, v_io, dv, vt, g, J, -gdv, o->ls_alpha1, o->ls_c1, o->ls_c2, &ls, st))) break;
      if (ls.status != kLsNotDescent) alpha = ls.alpha;
      if (info) {
        info->ls_evals[k] = ls.evals;
        info->ls_status[k] = ls.status;
      }
      if (ls.last && ls.status != kLsNotDescent) {
        carry = true;
        J = ls.phi;
      }
    }
    if (info) info->alpha[k] = alpha;
    if ((rc = axpby<double, double>(n, alpha, dv, 1.0, v_io, st))) break;
  }
  cudaStreamSynchronize(st);
  gb.release();
  state->next_iter = k;
  state->g0_inf = g0;
  state->sketch_iter = pc ? sketch_iter : -1;
  *held = pc;
  return rc;
}

int sc4dvar_gauss_newton(sc4dvar_problem_t P, const sc4dvar_gn_opts* o, double* v_io,
                         sc4dvar_gn_info* info, void* stream) {
  sc4dvar_gn_state state{0, 0.0, -1};
  sc4dvar_precond_t held = nullptr;
  const int rc = sc4dvar_gauss_newton_resume(P, o, v_io, &state, &held, info, stream);
  precond_free(held);
  return rc;
}

int sc4dvar_precond_import(sc4dvar_problem_t P, int l, const double* lam_host, const double* V_host,
                           sc4dvar_precond_t* out) {
  SC4_ARG(P && out, "null argument");
  SC4_ARG(l >= 0 && l <= P->n, "precond_import: 0 <= l <= n");
  SC4_ARG(l == 0 || (lam_host && V_host), "precond_import: lam and V needed for l > 0");
  std::vector<double> lam_dsc(2 * (size_t)l);
  for (int i = 0; i < l; ++i) {
    const double lm = lam_host[i];
    SC4_ARG(std::isfinite(lm) && lm >= 0.0, "precond_import: lam finite and >= 0");
    lam_dsc[i] = lm;
    lam_dsc[l + i] = lm / (1.0 + lm);  // as the sketches form it on the device (IEEE division)
  }
  Prec* pc = new Prec();
  pc->n = P->n;
  pc->l = l;
  if (l > 0) {
    if (cudaMalloc(&pc->V, (size_t)P->n * l * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&pc->lam, 2 * (size_t)l * sizeof(double)) != cudaSuccess ||
        cudaMemcpy(pc->V, V_host, (size_t)P->n * l * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pc->lam, lam_dsc.data(), 2 * (size_t)l * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      precond_free(pc);
      sc4::set_error("precond_import: device allocation or copy failed");
      return SC4DVAR_ERR_CUDA;
    }
    pc->dsc = pc->lam + l;
  }
  *out = pc;
  return SC4DVAR_OK;
}

int sc4dvar_counters(sc4dvar_problem_t P, sc4dvar_counters_t* out) {
  SC4_ARG(P && out, "null argument");
  *out = P->counters;
  return SC4DVAR_OK;
}

int sc4dvar_counters_reset(sc4dvar_problem_t P) {
  SC4_ARG(P, "null argument");
  P->counters = sc4dvar_counters_t{};
  return SC4DVAR_OK;
}

int sc4dvar_counters_set(sc4dvar_problem_t P, const sc4dvar_counters_t* c) {
  SC4_ARG(P && c, "null argument");
  P->counters = *c;
  return SC4DVAR_OK;
}

int sc4dvar_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, int64_t col0,
                     double* out, void* stream) {
  SC4_ARG(out && rows >= 0 && cols >= 0 && col0 >= 0, "gaussian arguments");
  return gaussian(seed, stream_id, rows, cols, col0, out, S(stream));
}

}  // extern "C"
