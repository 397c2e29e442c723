// Batched serving: many independent assimilation problems of uneven size.
//
// A batch groups problem handles (each with its own grid, window, observations
// and block width). The block Gauss-Newton Hessian products of all problems are
// recorded once into one CUDA graph -- every problem's kernels on its own branch
// (forked streams), so problems of different sizes run side by side -- and each
// later call with the same buffers replays it with a single graph launch.
// Likewise a PCG iteration for every problem (Hessian product, two reductions,
// the updates and the preconditioner, all with scalars kept on the device) is
// one graph launch; residuals come back to the host only when asked.
//
// Also here: sc4dvar_autotune, which times the packed FP32 sweep of a problem
// for each valid number of point pairs per thread and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include "common.cuh"
#include "dense.cuh"
#include "problem.cuh"

namespace sc4 {
// defined in api.cu
int batch_hvp_one(sc4dvar_problem_s* P, const void* X, int k, void* Y, int misfit_only, int prec,
                  cudaStream_t st);
int batch_hvp_vec(sc4dvar_problem_s* P, const double* p, double* q, int prec, cudaStream_t st);
int batch_precond(sc4dvar_precond_s* pc, const double* r, double* z, int n, cudaStream_t st);
}  // namespace sc4

namespace {

using namespace sc4;

// Device scalars of one PCG run (doubles): 0 rz, 1 pq, 2 alpha, 3 beta, 4 rz_new,
// 5 |r|, 6 |b|, 7 tol, 8 iterations, 9 status (0 ok, -4 breakdown).
enum { S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RZN, S_RN, S_BN, S_TOL, S_ITS, S_STATUS, S_N = 16 };

__global__ void pcg_alpha_kernel(double* sc) {
  if (threadIdx.x == 0) {
    bool active = sc[S_STATUS] == 0.0 && sc[S_RN] > sc[S_TOL] * sc[S_BN];
    double pq = sc[S_PQ];
    if (active && !(pq > 0.0 && isfinite(pq))) {
      sc[S_STATUS] = (double)SC4DVAR_ERR_BREAKDOWN;
      active = false;
    }
    sc[S_ALPHA] = active ? sc[S_RZ] / pq : 0.0;
    if (active) sc[S_ITS] += 1.0;
  }
}

__global__ void pcg_beta_kernel(double* sc) {
  if (threadIdx.x == 0) {
    bool moved = sc[S_ALPHA] != 0.0;
    sc[S_BETA] = moved && sc[S_RZ] != 0.0 ? sc[S_RZN] / sc[S_RZ] : 0.0;
    if (moved) sc[S_RZ] = sc[S_RZN];
  }
}

// x += alpha p; r -= alpha q   (alpha on the device)
__global__ void pcg_xr_kernel(int n, const double* __restrict__ sc, const double* __restrict__ p,
                              const double* __restrict__ q, double* x, double* r) {
  const double a = sc[S_ALPHA];
  if (a == 0.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    r[i] -= a * q[i];
  }
}

// p = z + beta p (only while iterating)
__global__ void pcg_p_kernel(int n, const double* __restrict__ sc, const double* __restrict__ z, double* p) {
  if (sc[S_ALPHA] == 0.0) return;
  const double b = sc[S_BETA];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = z[i] + b * p[i];
}

__global__ void fill0_kernel(int n, double* x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

__global__ void pcg_init_scalars(double* sc, double tol) {
  if (threadIdx.x == 0) {
    sc[S_TOL] = tol;
    sc[S_ITS] = 0.0;
    sc[S_STATUS] = 0.0;
    sc[S_ALPHA] = 0.0;
    sc[S_RN] = sc[S_BN];
  }
}

int blocks_for(int n) { return std::max(1, std::min((n + 255) / 256, 4 * 152)); }

struct PcgSlot {
  Buf buf;  // x, r, z, p, q (n each) + scalars
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *sc = nullptr;
  sc4dvar_precond_s* pc = nullptr;
};

}  // namespace

struct sc4dvar_batch_s {
  std::vector<sc4dvar_problem_s*> probs;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> evs;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // private stream that records (the caller's may be the legacy stream)
  // recorded Hessian-product graph and the arguments it was recorded with
  cudaGraphExec_t hvp_exec = nullptr;
  std::vector<const void*> hvp_X;
  std::vector<void*> hvp_Y;
  std::vector<int> hvp_k;
  int hvp_misfit = -1, hvp_prec = -1;
  // PCG
  std::vector<PcgSlot> pcg;
  int pcg_prec = SC4DVAR_FP64;
  cudaGraphExec_t pcg_exec = nullptr;
};

namespace {

using Batch = sc4dvar_batch_s;

int ensure_streams(Batch* b) {
  if (!b->side.empty()) return SC4DVAR_OK;
  const int S = std::min<int>((int)b->probs.size(), 16);
  b->side.resize(S);
  b->evs.resize(S);
  for (int i = 0; i < S; ++i) {
    SC4_CUDA(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking));
    SC4_CUDA(cudaEventCreateWithFlags(&b->evs[i], cudaEventDisableTiming));
  }
  SC4_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  SC4_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  return SC4DVAR_OK;
}

// Record `body(problem index, stream)` for every problem into a graph, problems
// spread over the side streams. Recording happens on the batch's private stream
// after `st` has drained; the graph is later launched on the caller's stream.
template <typename F>
int record(Batch* b, cudaStream_t st_user, F body, cudaGraphExec_t* exec) {
  SC4_TRY(ensure_streams(b));
  SC4_CUDA(cudaStreamSynchronize(st_user));
  cudaStream_t st = b->cap;
  cudaGraph_t graph = nullptr;
  SC4_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = SC4DVAR_OK;
  const int S = (int)b->side.size();
  if (cudaEventRecord(b->fork, st) != cudaSuccess) rc = SC4DVAR_ERR_CUDA;
  for (int i = 0; i < S && rc == SC4DVAR_OK; ++i)
    if (cudaStreamWaitEvent(b->side[i], b->fork, 0) != cudaSuccess) rc = SC4DVAR_ERR_CUDA;
  for (size_t p = 0; p < b->probs.size() && rc == SC4DVAR_OK; ++p) rc = body((int)p, b->side[p % S]);
  for (int i = 0; i < S && rc == SC4DVAR_OK; ++i) {
    if (cudaEventRecord(b->evs[i], b->side[i]) != cudaSuccess ||
        cudaStreamWaitEvent(st, b->evs[i], 0) != cudaSuccess)
      rc = SC4DVAR_ERR_CUDA;
  }
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc != SC4DVAR_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (rc == SC4DVAR_OK) {
      set_error(std::string("graph capture failed: ") + cudaGetErrorString(e));
      rc = SC4DVAR_ERR_CUDA;
    }
    return rc;
  }
  if (*exec) cudaGraphExecDestroy(*exec);
  *exec = nullptr;
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    set_error(std::string("graph instantiation failed: ") + cudaGetErrorString(e));
    *exec = nullptr;
    return SC4DVAR_ERR_CUDA;
  }
  return SC4DVAR_OK;
}

}  // namespace

extern "C" {

int sc4dvar_batch_create(const sc4dvar_problem_t* problems, int B, sc4dvar_batch_t* out) {
  SC4_ARG(problems && out && B >= 1, "batch_create arguments");
  for (int i = 0; i < B; ++i) SC4_ARG(problems[i] != nullptr, "null problem in batch");
  Batch* b = new Batch();
  b->probs.assign(problems, problems + B);
  *out = b;
  return SC4DVAR_OK;
}

int sc4dvar_batch_destroy(sc4dvar_batch_t b) {
  if (!b) return SC4DVAR_OK;
  if (b->hvp_exec) cudaGraphExecDestroy(b->hvp_exec);
  if (b->pcg_exec) cudaGraphExecDestroy(b->pcg_exec);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->evs) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto& s : b->pcg) s.buf.release();
  delete b;
  return SC4DVAR_OK;
}

int sc4dvar_batch_hessian_apply(sc4dvar_batch_t b, const void* const* X, void* const* Y, const int* k,
                                int misfit_only, int prec, void* stream) {
  SC4_ARG(b && X && Y && k, "batch_hessian_apply arguments");
  SC4_ARG(prec == SC4DVAR_FP64 || prec == SC4DVAR_FP32, "prec");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int B = (int)b->probs.size();
  for (int i = 0; i < B; ++i) {
    SC4_ARG(k[i] >= 1 && X[i] && Y[i], "every problem needs k >= 1 and buffers");
    if (!b->probs[i]->have_traj) {
      set_error("batch: a problem has no forward trajectory (call sc4dvar_fwd first)");
      return SC4DVAR_ERR_STATE;
    }
  }
  bool same = b->hvp_exec && b->hvp_misfit == misfit_only && b->hvp_prec == prec;
  for (int i = 0; same && i < B; ++i)
    same = b->hvp_X[i] == X[i] && b->hvp_Y[i] == Y[i] && b->hvp_k[i] == k[i];
  if (!same) {
    // one eager pass sizes every workspace (no allocation may happen while recording)
    for (int i = 0; i < B; ++i)
      SC4_TRY(batch_hvp_one(b->probs[i], X[i], k[i], Y[i], misfit_only, prec, st));
    SC4_CUDA(cudaStreamSynchronize(st));
    SC4_TRY(record(b, st, [&](int i, cudaStream_t s) {
      return batch_hvp_one(b->probs[i], X[i], k[i], Y[i], misfit_only, prec, s);
    }, &b->hvp_exec));
    b->hvp_X.assign(X, X + B);
    b->hvp_Y.assign(Y, Y + B);
    b->hvp_k.assign(k, k + B);
    b->hvp_misfit = misfit_only;
    b->hvp_prec = prec;
  }
  SC4_CUDA(cudaGraphLaunch(b->hvp_exec, st));
  note_launch();
  return SC4DVAR_OK;
}

int sc4dvar_batch_pcg_start(sc4dvar_batch_t b, const sc4dvar_precond_t* pcs, const double* const* rhs,
                            double tol, int prec, void* stream) {
  SC4_ARG(b && rhs && tol > 0, "batch_pcg_start arguments");
  SC4_ARG(prec == SC4DVAR_FP64 || prec == SC4DVAR_FP32, "prec");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int B = (int)b->probs.size();
  b->pcg.resize(B);
  b->pcg_prec = prec;
  for (int i = 0; i < B; ++i) {
    sc4dvar_problem_s* P = b->probs[i];
    if (!P->have_traj) {
      set_error("batch: a problem has no forward trajectory (call sc4dvar_fwd first)");
      return SC4DVAR_ERR_STATE;
    }
    PcgSlot& s = b->pcg[i];
    const int n = P->n;
    SC4_TRY(s.buf.ensure((size_t)(5 * n + S_N) * sizeof(double)));
    s.x = s.buf.as<double>();
    s.r = s.x + n;
    s.z = s.r + n;
    s.p = s.z + n;
    s.q = s.p + n;
    s.sc = s.q + n;
    s.pc = pcs ? pcs[i] : nullptr;
    SC4_ARG(!s.pc || s.pc->n == n, "preconditioner size");
    fill0_kernel<<<blocks_for(n), 256, 0, st>>>(n, s.x);
    SC4_LAUNCH_CHECK();
    SC4_CUDA(cudaMemcpyAsync(s.r, rhs[i], n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SC4_TRY(batch_precond(s.pc, s.r, s.z, n, st));
    SC4_CUDA(cudaMemcpyAsync(s.p, s.z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SC4_TRY(vdot<double, double>(n, s.r, s.z, s.sc + S_RZ, P->part.as<double>(), st));
    SC4_TRY(vnrm2<double>(n, s.r, s.sc + S_BN, P->part.as<double>(), st));
    pcg_init_scalars<<<1, 32, 0, st>>>(s.sc, tol);
    SC4_LAUNCH_CHECK();
    // size the operator's workspaces before any recording
    SC4_TRY(batch_hvp_vec(P, s.p, s.q, prec, st));
  }
  SC4_CUDA(cudaStreamSynchronize(st));
  // one PCG iteration of every problem, recorded once
  auto step = [&](int i, cudaStream_t s) -> int {
    sc4dvar_problem_s* P = b->probs[i];
    PcgSlot& sl = b->pcg[i];
    const int n = P->n;
    double* part = P->part.as<double>();
    SC4_TRY(batch_hvp_vec(P, sl.p, sl.q, b->pcg_prec, s));
    SC4_TRY(vdot<double, double>(n, sl.p, sl.q, sl.sc + S_PQ, part, s));
    pcg_alpha_kernel<<<1, 32, 0, s>>>(sl.sc);
    SC4_LAUNCH_CHECK();
    pcg_xr_kernel<<<blocks_for(n), 256, 0, s>>>(n, sl.sc, sl.p, sl.q, sl.x, sl.r);
    SC4_LAUNCH_CHECK();
    SC4_TRY(vnrm2<double>(n, sl.r, sl.sc + S_RN, part, s));
    SC4_TRY(batch_precond(sl.pc, sl.r, sl.z, n, s));
    SC4_TRY(vdot<double, double>(n, sl.r, sl.z, sl.sc + S_RZN, part, s));
    pcg_beta_kernel<<<1, 32, 0, s>>>(sl.sc);
    SC4_LAUNCH_CHECK();
    pcg_p_kernel<<<blocks_for(n), 256, 0, s>>>(n, sl.sc, sl.z, sl.p);
    SC4_LAUNCH_CHECK();
    return SC4DVAR_OK;
  };
  return record(b, st, step, &b->pcg_exec);
}

int sc4dvar_batch_pcg_step(sc4dvar_batch_t b, int nsteps, void* stream) {
  SC4_ARG(b && b->pcg_exec && nsteps >= 0, "batch_pcg_step: call sc4dvar_batch_pcg_start first");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < nsteps; ++i) {
    SC4_CUDA(cudaGraphLaunch(b->pcg_exec, st));
    note_launch();
  }
  for (auto* P : b->probs) {
    P->counters.tlm_online += nsteps;
    P->counters.adj_online += nsteps;
  }
  return SC4DVAR_OK;
}

int sc4dvar_batch_pcg_status(sc4dvar_batch_t b, double* relres, int* its, int* status, void* stream) {
  SC4_ARG(b && !b->pcg.empty(), "batch_pcg_status: no PCG started");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int B = (int)b->probs.size();
  std::vector<double> h((size_t)B * S_N);
  for (int i = 0; i < B; ++i)
    SC4_CUDA(cudaMemcpyAsync(h.data() + (size_t)i * S_N, b->pcg[i].sc, S_N * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < B; ++i) {
    const double* s = h.data() + (size_t)i * S_N;
    if (relres) relres[i] = s[S_BN] > 0 ? s[S_RN] / s[S_BN] : 0.0;
    if (its) its[i] = (int)s[S_ITS];
    if (status) status[i] = (int)s[S_STATUS];
  }
  return SC4DVAR_OK;
}

int sc4dvar_batch_pcg_solution(sc4dvar_batch_t b, double* const* x, void* stream) {
  SC4_ARG(b && x && !b->pcg.empty(), "batch_pcg_solution arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (size_t i = 0; i < b->probs.size(); ++i)
    SC4_CUDA(cudaMemcpyAsync(x[i], b->pcg[i].x, b->probs[i]->n * sizeof(double), cudaMemcpyDeviceToDevice,
                             st));
  return SC4DVAR_OK;
}

int sc4dvar_autotune(sc4dvar_problem_t P, int k, int* chosen) {
  SC4_ARG(P && k >= 1, "autotune arguments");
  if (!P->have_traj) {
    set_error("autotune: no forward trajectory (call sc4dvar_fwd first)");
    return SC4DVAR_ERR_STATE;
  }
  if (P->model != SC4DVAR_MODEL_BURGERS1D || !P->geom.fold32) {
    if (chosen) *chosen = 0;  // only the packed FP32 sweeps have a choice to make
    return SC4DVAR_OK;
  }
  const int n = P->n;
  Buf xb, yb;
  SC4_TRY(xb.ensure((size_t)n * k * sizeof(float)));
  SC4_TRY(yb.ensure((size_t)P->m * k * sizeof(float)));
  SC4_CUDA(cudaMemset(xb.p, 0, (size_t)n * k * sizeof(float)));
  cudaEvent_t e0, e1;
  SC4_CUDA(cudaEventCreate(&e0));
  SC4_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 1e30f;
  const int saved = P->geom.pairs_tuned;
  const int H = n / 2;
  for (int pp = 1; pp <= 8; pp *= 2) {
    if (H / pp < 32 || H / pp > (pp >= 8 ? 512 : 1024)) continue;
    P->geom.pairs_tuned = pp;
    int rc = burgers_tlm<float>(P->geom, P->traj32, xb.as<float>(), n, k, yb.as<float>(), P->m, 0);
    if (rc != SC4DVAR_OK) continue;
    cudaEventRecord(e0, 0);
    rc = burgers_tlm<float>(P->geom, P->traj32, xb.as<float>(), n, k, yb.as<float>(), P->m, 0);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess || rc != SC4DVAR_OK) continue;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = pp;
    }
  }
  P->geom.pairs_tuned = best > 0 ? best : saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  xb.release();
  yb.release();
  if (chosen) *chosen = P->geom.pairs_tuned;
  return SC4DVAR_OK;
}

}  // extern "C"
