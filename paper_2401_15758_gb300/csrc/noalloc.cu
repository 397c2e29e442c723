// Block Gauss-Newton Hessian product that allocates no device memory.
//
// sc4dvar_gn_hessian_apply_block needs three n x k / m x k work arrays between
// its four kernels (Gamma^{1/2} X, A X, and the adjoint state), and the handle
// grows them with cudaMalloc on first use or when k grows. Some callers cannot
// allow that: a host that hands every byte of device memory to its own pool
// allocator, or a real-time loop that must never enter the driver's allocator
// (cudaMalloc can synchronize the device). This file gives them the same
// product with the work arrays carved from one file-scope device array of fixed
// size. The caller still passes X and Y; the library allocates nothing in this
// call.
//
// The array is a static __device__ object: every GPU that loads the library
// holds SC4_NOALLOC_SCRATCH_BYTES of it until the process exits. Host code may
// not use the symbol as a device pointer (on the host it names a host-side
// stand-in), so the device address is looked up with cudaGetSymbolAddress once
// per device, with that device current, on the first call made on it. Make that
// first call before any stream capture begins. A cudaDeviceReset releases the
// array (and every problem's memory); the cached address is not valid after it.
#include <mutex>
#include <string>
#include "common.cuh"
#include "fft.cuh"
#include "model.cuh"
#include "problem.cuh"

#define SC4_NOALLOC_SCRATCH_BYTES (32u << 20)  // 32 MiB per device

namespace sc4 {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SC4_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(void** out) {
  int dev = 0;
  SC4_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("noalloc: device index out of range");
    return SC4DVAR_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error(std::string("noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return SC4DVAR_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SC4DVAR_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
const T* trajectory(sc4dvar_problem_s* P);
template <>
const double* trajectory<double>(sc4dvar_problem_s* P) { return P->traj64; }
template <>
const float* trajectory<float>(sc4dvar_problem_s* P) { return P->traj32; }

template <typename T>
int hvp_noalloc(sc4dvar_problem_s* P, const T* X, int ldx, int k, T* Y, int ldy, int misfit_only,
                cudaStream_t st) {
  const int n = P->n, m = P->m;
  const size_t bu = round256((size_t)n * k * sizeof(T));
  const size_t bw = round256((size_t)m * k * sizeof(T));
  const size_t need = 2 * bu + bw;
  if (need > SC4_NOALLOC_SCRATCH_BYTES) {
    set_error("noalloc: k = " + std::to_string(k) + " needs " + std::to_string(need) +
              " bytes of scratch; the fixed scratch holds " +
              std::to_string((size_t)SC4_NOALLOC_SCRATCH_BYTES) +
              " bytes ((2 n + m) k elements at most); use sc4dvar_gn_hessian_apply_block");
    return SC4DVAR_ERR_INVALID_ARG;
  }
  if (k == 0) return SC4DVAR_OK;
  void* base = nullptr;
  SC4_TRY(scratch_address(&base));
  // Every entry of the three work arrays is written before it is read, so no
  // clearing is needed between calls.
  T* U = reinterpret_cast<T*>(base);
  T* W = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(base) + bu);
  T* L = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(base) + bu + bw);
  const T* traj = trajectory<T>(P);
  SC4_TRY(prior_apply<T, T, T>(n, k, X, ldx, U, n, (const T*)nullptr, 0, P->sym, P->tw, st));
  SC4_TRY(burgers_tlm<T>(P->geom, traj, U, n, k, W, m, st));
  SC4_TRY(burgers_adj<T>(P->geom, traj, W, m, k, L, n, st));
  SC4_TRY(prior_apply<T, T, T>(n, k, L, n, Y, ldy, misfit_only ? (const T*)nullptr : X, ldx, P->sym,
                               P->tw, st));
  switch (P->count_mode) {
    case kOffline: P->counters.tlm_offline += k; P->counters.adj_offline += k; break;
    case kKappa: P->counters.tlm_kappa += k; P->counters.adj_kappa += k; break;
    default: P->counters.tlm_online += k; P->counters.adj_online += k; break;
  }
  return SC4DVAR_OK;
}

}  // namespace
}  // namespace sc4

extern "C" int sc4dvar_gn_hessian_apply_block_noalloc(sc4dvar_problem_t P, const void* X, int ldx,
                                                      int k, void* Y, int ldy, int misfit_only,
                                                      int prec, void* stream) {
  using namespace sc4;
  SC4_ARG(P, "null problem");
  SC4_ARG(k >= 0, "k must be >= 0");
  SC4_ARG(prec == SC4DVAR_FP64 || prec == SC4DVAR_FP32, "prec must be SC4DVAR_FP64 or SC4DVAR_FP32");
  SC4_ARG(ldx >= P->n && ldy >= P->n && (k == 0 || (X && Y)), "leading dimensions / pointers");
  if (!P->have_traj) {
    set_error("no forward trajectory (call sc4dvar_fwd first)");
    return SC4DVAR_ERR_STATE;
  }
  SC4_ARG(P->model == SC4DVAR_MODEL_BURGERS1D, "the allocation-free product covers the Burgers model");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (prec == SC4DVAR_FP64)
    return hvp_noalloc<double>(P, (const double*)X, ldx, k, (double*)Y, ldy, misfit_only, st);
  return hvp_noalloc<float>(P, (const float*)X, ldx, k, (float*)Y, ldy, misfit_only, st);
}
