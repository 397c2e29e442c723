// Shared device/host helpers of the sc4dvar CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string>
#include "../../include/sc4dvar.h"

namespace sc4 {

// ---- tracing ------------------------------------------------------------------
// An NVTX range for the lifetime of the object (GN iterations, sketches, sweeps,
// PCG iterations); a no-op unless a profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- error plumbing ---------------------------------------------------------
void set_error(const std::string& msg);
struct Status {
  int code = SC4DVAR_OK;
};

#define SC4_CUDA(call)                                                            \
  do {                                                                            \
    cudaError_t _e = (call);                                                      \
    if (_e != cudaSuccess) {                                                      \
      sc4::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));         \
      return SC4DVAR_ERR_CUDA;                                                    \
    }                                                                             \
  } while (0)

// Kernels launched by this library since load (diagnostics: sc4dvar_launch_count).
void note_launch();

#define SC4_LAUNCH_CHECK()                                                        \
  do {                                                                            \
    sc4::note_launch();                                                           \
    cudaError_t _e = cudaGetLastError();                                          \
    if (_e != cudaSuccess) {                                                      \
      sc4::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e));    \
      return SC4DVAR_ERR_CUDA;                                                    \
    }                                                                             \
  } while (0)

#define SC4_TRY(...)                                                              \
  do {                                                                            \
    int _s = (__VA_ARGS__);                                                       \
    if (_s != SC4DVAR_OK) return _s;                                              \
  } while (0)

#define SC4_ARG(cond, msg)                                                        \
  do {                                                                            \
    if (!(cond)) {                                                                \
      sc4::set_error(std::string("invalid argument: ") + (msg));                  \
      return SC4DVAR_ERR_INVALID_ARG;                                             \
    }                                                                             \
  } while (0)

inline int div_up(int a, int b) { return (a + b - 1) / b; }

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------------
// 10 rounds; each multiplies words 0 and 2 by M0 / M1, recombines the high and
// low halves with words 1, 3 and the key; the key advances by the Weyl
// constants between rounds.
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * c.x;
    uint64_t p1 = (uint64_t)M1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 o;
    o.x = hi1 ^ c.y ^ k0;
    o.y = lo1;
    o.z = hi0 ^ c.w ^ k1;
    o.w = lo0;
    c = o;
  }
  return c;
}

// 53-bit uniform in (0, 1) from two 32-bit words.
__device__ inline double uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// Normal number e of stream (seed, stream): the library's Box-Muller convention.
__device__ inline double philox_normal(uint64_t seed, uint64_t stream, uint64_t e) {
  uint64_t p = e >> 1;
  U4 c{(uint32_t)p, (uint32_t)(p >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
  U4 w = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  double u1 = uniform53(w.x, w.y);
  double u2 = uniform53(w.z, w.w);
  double r = sqrt(-2.0 * log(u1));
  double s, co;
  sincospi(2.0 * u2, &s, &co);
  return (e & 1) ? r * s : r * co;
}

// ---- reductions ---------------------------------------------------------------
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ inline T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; every thread gets the result. `red` holds >= 32 values.
template <typename T>
__device__ inline T block_sum(T v, T* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T out = red[0];
  __syncthreads();
  return out;
}

template <typename T>
__device__ inline T block_max(T v, T* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(-1e300);
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T out = red[0];
  __syncthreads();
  return out;
}

}  // namespace sc4
