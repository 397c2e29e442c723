// Double-gyre barotropic vorticity (Sec. 5.2): FWD, TLM and discrete RK adjoint
// sweeps, and the elliptic solves they need.
//
// Every RK stage needs psi = P omega, P = h^2 (-Delta*)^{-1}. The solve is
//   1. a sine transform of every grid row (a dense product with the nx x nx
//      matrix S; nx <= 128, so one CTA tile holds all output modes; FP32 fields
//      at nx = 128 run it on the tensor cores in the 3xTF32 split),
//   2. one tridiagonal (Thomas) solve along y per x-mode, one thread per
//      (field, mode) running down the rows,
//   3. the inverse transform (S again).
// The stage kernels are pointwise with a one-point halo (central differences,
// zero boundary values) and fuse the RK combinations, so one stage of k
// directions is three transform/solve launches and one stencil launch (two for
// the adjoint, which needs a Poisson solve between its two halves).
//
// Adjoint of one stage (omega_b, psi_b the stored base stage, kappa the stage
// adjoint input):
//   theta = D_x(psi_b,y kappa) - D_y(psi_b,x kappa) + Re^{-1} Lap kappa
//           + P [ D_y(omega_b,x kappa) - D_x(omega_b,y kappa) - Ro^{-1} D_x kappa ],
// the transpose of the TLM stage -(J(P d, omega_b) + J(psi_b, d)) +
// Ro^{-1} D_x P d + Re^{-1} Lap d (D_x, D_y skew, Lap and P symmetric with zero
// boundary values). kappa_s = h b_s lambda' + h sum_{j>s} a_js theta_j is never
// stored: both halves rebuild it at each point they read from lambda' and the
// stored theta_j.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>
#include <vector>
#include "common.cuh"
#include "gyre.cuh"
#include "tall_tc.cuh"

namespace sc4 {
namespace {

constexpr int kBK = 16;        // reduction chunk of the tiled transform
constexpr int kTileThreads = 256;

template <typename T>
struct GyP {
  int nx, ny, n, lnx;  // nx = 2^lnx
  T inv2h, invh2, re_inv, ro_inv;
};

template <typename T>
GyP<T> make_p(const GyreGeom& g) {
  GyP<T> p;
  p.nx = g.nx;
  p.ny = g.ny;
  p.n = g.n;
  p.lnx = 0;
  while ((1 << p.lnx) < g.nx) ++p.lnx;
  p.inv2h = (T)(1.0 / (2.0 * g.h));
  p.invh2 = (T)(1.0 / (g.h * g.h));
  p.re_inv = (T)g.re_inv;
  p.ro_inv = (T)g.ro_inv;
  return p;
}

// value of a field at (i, j); zero outside the interior (boundary values)
template <typename T>
__device__ __forceinline__ T at(const T* f, int i, int j, const GyP<T>& p) {
  return (i >= 0 && i < p.nx && j >= 0 && j < p.ny) ? f[j * p.nx + i] : T(0);
}

// sum_q c_q src_q at (i, j), zero outside: the rebuilt adjoint stage input
template <typename T>
struct Comb {
  const T* src[4];
  T c[4];
  int m;
};

template <typename T>
__device__ __forceinline__ T comb_at(const Comb<T>& cb, size_t off, int i, int j, const GyP<T>& p) {
  if (i < 0 || i >= p.nx || j < 0 || j >= p.ny) return T(0);
  const size_t e = off + (size_t)j * p.nx + i;
  T v = cb.c[0] * cb.src[0][e];
#pragma unroll
  for (int q = 1; q < 4; ++q)
    if (q < cb.m) v += cb.c[q] * cb.src[q][e];
  return v;
}

// ---------------------------------------------------------------- transforms
// out[r][p] = sum_i in[r][i] S[i][p] (+ Z[r][p]) for the rows r = c ny + j of k
// fields (field strides ldi / ldo / ldz). One thread per output element: used
// for few rows, where a tile per CTA would leave most SMs idle.
template <typename TI, typename TC, typename TO, typename TZ>
__global__ void gy_dst_simple_kernel(int nx, int ny, int rows, const TI* __restrict__ in, int ldi,
                                     const TC* __restrict__ Sm, TO* __restrict__ out, int ldo,
                                     const TZ* __restrict__ Z, int ldz) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)rows * nx) return;
  const int r = (int)(e / nx), p = (int)(e % nx);
  const int c = r / ny, j = r - c * ny;
  const TI* row = in + (size_t)c * ldi + (size_t)j * nx;
  // four partial sums: a quarter of the dependent FMA chain (this form runs for
  // few rows, where the chain latency, not throughput, sets the time)
  TC a0 = TC(0), a1 = TC(0), a2 = TC(0), a3 = TC(0);
  int i = 0;
  for (; i + 3 < nx; i += 4) {
    a0 += (TC)row[i] * Sm[(size_t)i * nx + p];
    a1 += (TC)row[i + 1] * Sm[(size_t)(i + 1) * nx + p];
    a2 += (TC)row[i + 2] * Sm[(size_t)(i + 2) * nx + p];
    a3 += (TC)row[i + 3] * Sm[(size_t)(i + 3) * nx + p];
  }
  for (; i < nx; ++i) a0 += (TC)row[i] * Sm[(size_t)i * nx + p];
  TC acc = (a0 + a1) + (a2 + a3);
  const size_t o = (size_t)j * nx + p;
  if (Z) acc += (TC)Z[(size_t)c * ldz + o];
  out[(size_t)c * ldo + o] = (TO)acc;
}

// Tiled form: CG = nx/8 column groups of 8 modes x RG = 256/CG row groups of 4
// rows per CTA (BR = 4 RG rows); the reduction runs over chunks of kBK inputs
// staged in shared memory (inputs transposed, padded by 4 against bank
// conflicts). nx in {16, 32, 64, 128}.
template <typename TI, typename TC, typename TO, typename TZ>
__global__ void __launch_bounds__(kTileThreads) gy_dst_tiled_kernel(int nx, int ny, int rows,
                                                                    const TI* __restrict__ in, int ldi,
                                                                    const TC* __restrict__ Sm,
                                                                    TO* __restrict__ out, int ldo,
                                                                    const TZ* __restrict__ Z, int ldz) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int CG = nx / 8, RG = kTileThreads / CG, BR = 4 * RG, BRP = BR + 4;
  TC* sIn = reinterpret_cast<TC*>(smraw);  // [kBK][BRP]
  TC* sS = sIn + kBK * BRP;                // [kBK][nx]
  const int tid = threadIdx.x, cgi = tid % CG, rgi = tid / CG;
  const int r0 = blockIdx.x * BR;
  TC acc[4][8];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) acc[x][y] = TC(0);
  for (int i0 = 0; i0 < nx; i0 += kBK) {
    for (int e = tid; e < BR * kBK; e += kTileThreads) {
      const int rr = e / kBK, ii = e - rr * kBK, r = r0 + rr;
      TC v = TC(0);
      if (r < rows) {
        const int c = r / ny, j = r - c * ny;
        v = (TC)in[(size_t)c * ldi + (size_t)j * nx + i0 + ii];
      }
      sIn[ii * BRP + rr] = v;
    }
    for (int e = tid; e < kBK * nx; e += kTileThreads) sS[e] = Sm[(size_t)i0 * nx + e];
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < kBK; ++ii) {
      TC a[4], b[8];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = sIn[ii * BRP + rgi * 4 + x];
#pragma unroll
      for (int y = 0; y < 8; ++y) b[y] = sS[ii * nx + cgi * 8 + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int r = r0 + rgi * 4 + x;
    if (r >= rows) continue;
    const int c = r / ny, j = r - c * ny;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const size_t o = (size_t)j * nx + cgi * 8 + y;
      TC v = acc[x][y];
      if (Z) v += (TC)Z[(size_t)c * ldz + o];
      out[(size_t)c * ldo + o] = (TO)v;
    }
  }
}

// Tensor-core form for FP32 fields with nx = 128 (the row transform is a dense
// rows x 128 by 128 x 128 product): rows128_tc in tall_tc.cu, tcgen05 MMAs in
// the 3xTF32 split with the accumulators in tensor memory and S packed once at
// set-up (GyreGeom::S_tc).

size_t tiled_smem(int nx, size_t tb) {
  const int CG = nx / 8, BR = 4 * (kTileThreads / CG);
  return ((size_t)kBK * (BR + 4) + (size_t)kBK * nx) * tb;
}

template <typename TI, typename TC, typename TO, typename TZ>
int dst_rows(const GyreGeom& g, int k, const TI* in, int ldi, const TC* Sm, TO* out, int ldo, const TZ* Z,
             int ldz, cudaStream_t st) {
  const int nx = g.nx, rows = k * g.ny;
  if (rows <= 0) return SC4DVAR_OK;
  if constexpr (std::is_same<TI, float>::value && std::is_same<TC, float>::value &&
                std::is_same<TO, float>::value) {
    // tensor-core form: nx = 128, no added term, input fields back to back from
    // a 16-byte aligned start (one 2D tensor map over all rows), 16-byte aligned
    // output rows, at least 16 tiles of 128 rows
    const int tiles = div_up(rows, 128);
    if (nx == 128 && g.S_tc && Z == nullptr && ((uintptr_t)in % 16) == 0 && ldi == g.ny * nx &&
        ((uintptr_t)out % 16) == 0 && ldo % 4 == 0 && tiles >= 16)
      return rows128_tc(g.ny, rows, in, g.S_tc, out, ldo, st);
  }
  const int BR = 4 * (kTileThreads / std::max(1, nx / 8));
  if (nx >= 16 && div_up(rows, BR) >= 152) {
    const size_t smem = tiled_smem(nx, sizeof(TC));
    auto kern = gy_dst_tiled_kernel<TI, TC, TO, TZ>;
    SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<div_up(rows, BR), kTileThreads, smem, st>>>(nx, g.ny, rows, in, ldi, Sm, out, ldo, Z, ldz);
  } else {
    const size_t total = (size_t)rows * nx;
    gy_dst_simple_kernel<TI, TC, TO, TZ><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        nx, g.ny, rows, in, ldi, Sm, out, ldo, Z, ldz);
  }
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// In place, for each field and x-mode p: solve the tridiagonal system along y
// (diagonal 1/piv_j after elimination, off-diagonal off). One thread per
// (field, mode): the recurrences run down the rows in global memory, a warp's
// 32 modes reading and writing 32 consecutive words of a row. Rows (and their
// factors) are loaded kTh at a time into registers one chunk ahead of the
// recurrence, so the dependent chain is only the arithmetic and the loads of
// the next chunk overlap it: forward z_j = (r_j - off z_{j-1}) / piv_j, back
// x_j = z_j - c'_j x_{j+1}.
constexpr int kTh = 16;

template <typename T>
__global__ void __launch_bounds__(128) gy_thomas_kernel(int nx, int ny, int k, T* F, int ldf,
                                                        const T* __restrict__ fac, T off) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= k * nx) return;
  const int c = gid / nx, p = gid - c * nx;
  T* f = F + (size_t)c * ldf + p;
  const T* ipv = fac + p;
  const T* cpr = fac + (size_t)nx * ny + p;
  T r[kTh], q[kTh], rn[kTh], qn[kTh];
#pragma unroll
  for (int u = 0; u < kTh; ++u) {
    r[u] = (u < ny) ? f[(size_t)u * nx] : T(0);
    q[u] = (u < ny) ? ipv[(size_t)u * nx] : T(0);
  }
  T z = T(0);
  for (int j0 = 0; j0 < ny; j0 += kTh) {
#pragma unroll
    for (int u = 0; u < kTh; ++u) {
      const int j = j0 + kTh + u;
      rn[u] = (j < ny) ? f[(size_t)j * nx] : T(0);
      qn[u] = (j < ny) ? ipv[(size_t)j * nx] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kTh; ++u)
      if (j0 + u < ny) {
        z = (r[u] - off * z) * q[u];
        r[u] = z;
      }
#pragma unroll
    for (int u = 0; u < kTh; ++u)
      if (j0 + u < ny) f[(size_t)(j0 + u) * nx] = r[u];
#pragma unroll
    for (int u = 0; u < kTh; ++u) {
      r[u] = rn[u];
      q[u] = qn[u];
    }
  }
  T x = z;  // x_{ny-1} = z_{ny-1}
  const int jt = ny - 2;
#pragma unroll
  for (int u = 0; u < kTh; ++u) {
    r[u] = (jt - u >= 0) ? f[(size_t)(jt - u) * nx] : T(0);
    q[u] = (jt - u >= 0) ? cpr[(size_t)(jt - u) * nx] : T(0);
  }
  for (int j0 = jt; j0 >= 0; j0 -= kTh) {
#pragma unroll
    for (int u = 0; u < kTh; ++u) {
      const int j = j0 - kTh - u;
      rn[u] = (j >= 0) ? f[(size_t)j * nx] : T(0);
      qn[u] = (j >= 0) ? cpr[(size_t)j * nx] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kTh; ++u)
      if (j0 - u >= 0) {
        x = r[u] - q[u] * x;
        r[u] = x;
      }
#pragma unroll
    for (int u = 0; u < kTh; ++u)
      if (j0 - u >= 0) f[(size_t)(j0 - u) * nx] = r[u];
#pragma unroll
    for (int u = 0; u < kTh; ++u) {
      r[u] = rn[u];
      q[u] = qn[u];
    }
  }
}

template <typename T>
int thomas(const GyreGeom& g, int k, T* F, int ldf, const T* fac, double off, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  gy_thomas_kernel<T><<<div_up(k * g.nx, 128), 128, 0, st>>>(g.nx, g.ny, k, F, ldf, fac, (T)off);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template <typename T> const T* S_of(const GyreGeom& g);
template <> const double* S_of<double>(const GyreGeom& g) { return g.S64; }
template <> const float* S_of<float>(const GyreGeom& g) { return g.S32; }
template <typename T> const T* pois_of(const GyreGeom& g);
template <> const double* pois_of<double>(const GyreGeom& g) { return g.pois64; }
template <> const float* pois_of<float>(const GyreGeom& g) { return g.pois32; }
template <typename T> const T* prior_of(const GyreGeom& g);
template <> const double* prior_of<double>(const GyreGeom& g) { return g.prior64; }
template <> const float* prior_of<float>(const GyreGeom& g) { return g.prior32; }
template <typename T> const T* om_of(const GyreGeom& g);
template <> const double* om_of<double>(const GyreGeom& g) { return g.om64; }
template <> const float* om_of<float>(const GyreGeom& g) { return g.om32; }
template <typename T> const T* ps_of(const GyreGeom& g);
template <> const double* ps_of<double>(const GyreGeom& g) { return g.ps64; }
template <> const float* ps_of<float>(const GyreGeom& g) { return g.ps32; }

// psi = P omega for k fields (ld n), tmp: k n work
template <typename T>
int poisson(const GyreGeom& g, int k, const T* om, T* psi, T* tmp, cudaStream_t st) {
  const T* Sm = S_of<T>(g);
  SC4_TRY((dst_rows<T, T, T, T>(g, k, om, g.n, Sm, tmp, g.n, (const T*)nullptr, 0, st)));
  SC4_TRY(thomas<T>(g, k, tmp, g.n, pois_of<T>(g), g.pois_off, st));
  SC4_TRY((dst_rows<T, T, T, T>(g, k, tmp, g.n, Sm, psi, g.n, (const T*)nullptr, 0, st)));
  return SC4DVAR_OK;
}

// ---------------------------------------------------------------- FWD stage
struct FwdStage {
  const double* X;       // stage input
  const double* psi;     // P X
  const double* x;       // state at the step start
  double* next;          // next stage input, or the new state (last stage)
  double* K[4];          // slopes of the step
  double cK[4];          // next = x + sum_{j<=s} cK[j] K_j
  int s;
  bool last;
  double* om_st;         // stage-state stores (null: do not store)
  double* ps_st;
  float* om_st32;
  float* ps_st32;
};

__global__ void gy_fwd_stage_kernel(GyP<double> p, FwdStage a, const double* __restrict__ Fy) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.n) return;
  const int j = q / p.nx, i = q - j * p.nx;
  const double* X = a.X;
  const double* ps = a.psi;
  const double Xc = X[q];
  const double ox = (at(X, i + 1, j, p) - at(X, i - 1, j, p)) * p.inv2h;
  const double oy = (at(X, i, j + 1, p) - at(X, i, j - 1, p)) * p.inv2h;
  const double lap = (at(X, i + 1, j, p) + at(X, i - 1, j, p) + at(X, i, j + 1, p) + at(X, i, j - 1, p) -
                      4.0 * Xc) * p.invh2;
  const double px = (at(ps, i + 1, j, p) - at(ps, i - 1, j, p)) * p.inv2h;
  const double py = (at(ps, i, j + 1, p) - at(ps, i, j - 1, p)) * p.inv2h;
  const double K = -(py * ox - px * oy) + p.ro_inv * px + p.re_inv * lap + p.ro_inv * Fy[j];
  if (a.om_st) {
    a.om_st[q] = Xc;
    a.ps_st[q] = ps[q];
    a.om_st32[q] = (float)Xc;
    a.ps_st32[q] = (float)ps[q];
  }
  if (!a.last) a.K[a.s][q] = K;
  double v = a.x[q];
  for (int jj = 0; jj < a.s; ++jj) v += a.cK[jj] * a.K[jj][q];
  a.next[q] = v + a.cK[a.s] * K;
}

// ---------------------------------------------------------------- TLM stage
template <typename T>
struct TlmStage {
  const T* dX;     // stage input (k fields)
  const T* dpsi;   // P dX
  const T* dom;    // state at the step start
  T* next;         // next stage input, or the new state (last stage, in place)
  T* K[4];
  T cK[4];
  int s;
  bool last;
};

// Fields per thread of the stage kernels: the derivatives of the stored
// trajectory (the same for every field) are formed once and reused, which cuts
// the L1/L2 traffic of the neighbour loads that bound these kernels.
constexpr int kGyFields = 4;

template <typename T>
__global__ void gy_tlm_stage_kernel(GyP<T> p, int k, const T* __restrict__ om_b, const T* __restrict__ ps_b,
                                    TlmStage<T> a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // grid point; blockIdx.y = group of fields
  const int c0 = (int)blockIdx.y * kGyFields;
  if (q >= p.n || c0 >= k) return;
  const int j = q >> p.lnx, i = q & (p.nx - 1);
  const T obx = (at(om_b, i + 1, j, p) - at(om_b, i - 1, j, p)) * p.inv2h;
  const T oby = (at(om_b, i, j + 1, p) - at(om_b, i, j - 1, p)) * p.inv2h;
  const T pbx = (at(ps_b, i + 1, j, p) - at(ps_b, i - 1, j, p)) * p.inv2h;
  const T pby = (at(ps_b, i, j + 1, p) - at(ps_b, i, j - 1, p)) * p.inv2h;
#pragma unroll 1
  for (int f = 0; f < kGyFields && c0 + f < k; ++f) {
    const size_t off = (size_t)(c0 + f) * p.n;
    const T* X = a.dX + off;
    const T* dp = a.dpsi + off;
    const T Xc = X[q];
    const T dxx = (at(X, i + 1, j, p) - at(X, i - 1, j, p)) * p.inv2h;
    const T dxy = (at(X, i, j + 1, p) - at(X, i, j - 1, p)) * p.inv2h;
    const T lap = (at(X, i + 1, j, p) + at(X, i - 1, j, p) + at(X, i, j + 1, p) + at(X, i, j - 1, p) -
                   T(4) * Xc) * p.invh2;
    const T dpx = (at(dp, i + 1, j, p) - at(dp, i - 1, j, p)) * p.inv2h;
    const T dpy = (at(dp, i, j + 1, p) - at(dp, i, j - 1, p)) * p.inv2h;
    // -(J(dpsi, omega_b) + J(psi_b, dX)) + Ro^{-1} dpsi_x + Re^{-1} Lap dX
    const T K = -((dpy * obx - dpx * oby) + (pby * dxx - pbx * dxy)) + p.ro_inv * dpx + p.re_inv * lap;
    if (!a.last) a.K[a.s][off + q] = K;
    T v = a.dom[off + q];
    for (int jj = 0; jj < a.s; ++jj) v += a.cK[jj] * a.K[jj][off + q];
    a.next[off + q] = v + a.cK[a.s] * K;
  }
}

// ---------------------------------------------------------------- ADJ stage
// first half: g = D_y(omega_b,x kappa) - D_x(omega_b,y kappa) - Ro^{-1} D_x kappa
template <typename T>
__global__ void gy_adj_pre_kernel(GyP<T> p, int k, const T* __restrict__ om_b, Comb<T> kap, T* __restrict__ gout) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // grid point; blockIdx.y = group of fields
  const int c0 = (int)blockIdx.y * kGyFields;
  if (q >= p.n || c0 >= k) return;
  const int j = q >> p.lnx, i = q & (p.nx - 1);
  auto obx = [&](int ii, int jj) { return (at(om_b, ii + 1, jj, p) - at(om_b, ii - 1, jj, p)) * p.inv2h; };
  auto oby = [&](int ii, int jj) { return (at(om_b, ii, jj + 1, p) - at(om_b, ii, jj - 1, p)) * p.inv2h; };
  const T obxN = obx(i, j + 1), obxS = obx(i, j - 1), obyE = oby(i + 1, j), obyW = oby(i - 1, j);
#pragma unroll 1
  for (int f = 0; f < kGyFields && c0 + f < k; ++f) {
    const size_t off = (size_t)(c0 + f) * p.n;
    const T kE = comb_at(kap, off, i + 1, j, p), kW = comb_at(kap, off, i - 1, j, p);
    const T kN = comb_at(kap, off, i, j + 1, p), kS = comb_at(kap, off, i, j - 1, p);
    const T gy = (obxN * kN - obxS * kS) * p.inv2h;
    const T gx = (obyE * kE - obyW * kW) * p.inv2h;
    gout[off + q] = gy - gx - p.ro_inv * (kE - kW) * p.inv2h;
  }
}

template <typename T>
struct AdjPost {
  const T* phi;    // P g
  const T* lam;    // lambda' (step end)
  T* lam_out;      // lambda at the step start (stage 0 only)
  T* Th[4];        // theta_j of the step
  int s;
};

// second half: theta = D_x(psi_b,y kappa) - D_y(psi_b,x kappa) + Re^{-1} Lap kappa + phi
template <typename T>
__global__ void gy_adj_post_kernel(GyP<T> p, int k, const T* __restrict__ ps_b, Comb<T> kap, AdjPost<T> a,
                                   int S) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // grid point; blockIdx.y = group of fields
  const int c0 = (int)blockIdx.y * kGyFields;
  if (q >= p.n || c0 >= k) return;
  const int j = q >> p.lnx, i = q & (p.nx - 1);
  auto pbx = [&](int ii, int jj) { return (at(ps_b, ii + 1, jj, p) - at(ps_b, ii - 1, jj, p)) * p.inv2h; };
  auto pby = [&](int ii, int jj) { return (at(ps_b, ii, jj + 1, p) - at(ps_b, ii, jj - 1, p)) * p.inv2h; };
  const T pbyE = pby(i + 1, j), pbyW = pby(i - 1, j), pbxN = pbx(i, j + 1), pbxS = pbx(i, j - 1);
#pragma unroll 1
  for (int f = 0; f < kGyFields && c0 + f < k; ++f) {
    const size_t off = (size_t)(c0 + f) * p.n;
    const T kC = comb_at(kap, off, i, j, p);
    const T kE = comb_at(kap, off, i + 1, j, p), kW = comb_at(kap, off, i - 1, j, p);
    const T kN = comb_at(kap, off, i, j + 1, p), kS = comb_at(kap, off, i, j - 1, p);
    const T tx = (pbyE * kE - pbyW * kW) * p.inv2h;
    const T ty = (pbxN * kN - pbxS * kS) * p.inv2h;
    const T lap = (kE + kW + kN + kS - T(4) * kC) * p.invh2;
    const T th = tx - ty + p.re_inv * lap + a.phi[off + q];
    if (a.s > 0) {
      a.Th[a.s][off + q] = th;
    } else {
      T v = a.lam[off + q] + th;
      for (int jj = 1; jj < S; ++jj) v += a.Th[jj][off + q];
      a.lam_out[off + q] = v;
    }
  }
}

// ---------------------------------------------------------------- observations
template <typename T>
__global__ void gy_tlm_obs_kernel(int n, int n_o, int k, const T* __restrict__ dom, const int* __restrict__ idx,
                                  T inv_sigma, T* W, int ldw, int row0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * n_o) return;
  const int c = e / n_o, o = e - c * n_o;
  W[(size_t)c * ldw + row0 + o] = dom[(size_t)c * n + idx[o]] * inv_sigma;
}

template <typename T>
__global__ void gy_adj_obs_kernel(int n, int n_o, int k, T* lam, const int* __restrict__ idx, T inv_sigma,
                                  const T* __restrict__ W, int ldw, int row0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * n_o) return;
  const int c = e / n_o, o = e - c * n_o;
  atomicAdd(&lam[(size_t)c * n + idx[o]], W[(size_t)c * ldw + row0 + o] * inv_sigma);
}

__global__ void gy_fwd_obs_kernel(int n_o, const double* __restrict__ x, const int* __restrict__ idx,
                                  const double* __restrict__ y, double* d_out, double* obs_out, double inv_sigma,
                                  int row0) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_o) return;
  const double v = x[idx[o]];
  if (obs_out) obs_out[row0 + o] = v;
  if (d_out) d_out[row0 + o] = (v - y[row0 + o]) * inv_sigma;
}

// copy k fields between strided layouts
template <typename TA, typename TB>
__global__ void gy_copy_kernel(int n, int k, const TA* __restrict__ a, int lda, TB* __restrict__ b, int ldb) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)k * n) return;
  const int c = (int)(e / n), q = (int)(e - (size_t)c * n);
  b[(size_t)c * ldb + q] = (TB)a[(size_t)c * lda + q];
}

template <typename TA, typename TB>
int copy_fields(int n, int k, const TA* a, int lda, TB* b, int ldb, cudaStream_t st) {
  const size_t total = (size_t)k * n;
  if (!total) return SC4DVAR_OK;
  gy_copy_kernel<TA, TB><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, k, a, lda, b, ldb);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

unsigned blocks_of(size_t total) { return (unsigned)((total + 255) / 256); }

size_t field_bytes(const GyreGeom& g, int k, size_t tb) {
  return (((size_t)k * g.n * tb) + 255) / 256 * 256;
}

// Thomas factors of tridiag(off, alpha + beta (mu_p + 2), off) per x-mode, laid
// out [inverse pivots | c'] x [ny][nx]
void thomas_factors(int nx, int ny, double alpha, double beta, std::vector<double>& out) {
  out.assign(2 * (size_t)nx * ny, 0.0);
  const double off = -beta;
  for (int p = 0; p < nx; ++p) {
    const double s = std::sin(M_PI * (p + 1) / (2.0 * (nx + 1)));
    const double d = alpha + beta * (4.0 * s * s + 2.0);
    double cprev = 0.0;
    for (int j = 0; j < ny; ++j) {
      const double piv = d - (j > 0 ? off * cprev : 0.0);
      const double ip = 1.0 / piv;
      const double cp = off * ip;
      out[(size_t)j * nx + p] = ip;
      out[(size_t)nx * ny + (size_t)j * nx + p] = cp;
      cprev = cp;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host API
size_t gyre_setup_bytes(int nx) {
  const int ny = 2 * nx + 1;
  const size_t nn = (size_t)nx * nx, f = 2 * (size_t)nx * ny;
  const size_t base = nn * (8 + 4) + 2 * f * (8 + 4) + (size_t)ny * 8;
  return nx == 128 ? gyre_tc_offset(nx) + rows128_pack_bytes() : base;
}

size_t gyre_tc_offset(int nx) {
  const int ny = 2 * nx + 1;
  const size_t nn = (size_t)nx * nx, f = 2 * (size_t)nx * ny;
  return (nn * (8 + 4) + 2 * f * (8 + 4) + (size_t)ny * 8 + 255) & ~(size_t)255;
}

size_t gyre_stage_bytes(int nx, int N, int S) {
  const size_t n = (size_t)nx * (2 * nx + 1);
  return (size_t)N * S * n * (2 * 8 + 2 * 4);
}

int gyre_setup(GyreGeom& g, double prior_a, double prior_b, cudaStream_t st) {
  const int nx = g.nx, ny = g.ny;
  std::vector<double> S((size_t)nx * nx);
  const double sc = std::sqrt(2.0 / (nx + 1));
  for (int i = 0; i < nx; ++i)
    for (int p = 0; p < nx; ++p) S[(size_t)i * nx + p] = sc * std::sin(M_PI * (double)(i + 1) * (p + 1) / (nx + 1));
  std::vector<double> pois, prior;
  const double ih2 = 1.0 / (g.h * g.h);
  thomas_factors(nx, ny, 0.0, ih2, pois);
  thomas_factors(nx, ny, prior_a, prior_b, prior);
  g.pois_off = -ih2;
  g.prior_off = -prior_b;
  std::vector<double> Fy(ny);
  for (int j = 0; j < ny; ++j) Fy[j] = std::sin(M_PI * (-1.0 + (j + 1) * g.h));
  auto to32 = [](const std::vector<double>& v) {
    std::vector<float> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
    return f;
  };
  const std::vector<float> S32 = to32(S), pois32 = to32(pois), prior32 = to32(prior);
  SC4_CUDA(cudaMemcpyAsync(g.S64, S.data(), S.size() * 8, cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.S32, S32.data(), S32.size() * 4, cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.pois64, pois.data(), pois.size() * 8, cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.pois32, pois32.data(), pois32.size() * 4, cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.prior64, prior.data(), prior.size() * 8, cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.prior32, prior32.data(), prior32.size() * 4, cudaMemcpyHostToDevice, st));
  SC4_CUDA(cudaMemcpyAsync(g.Fy, Fy.data(), Fy.size() * 8, cudaMemcpyHostToDevice, st));
  if (g.S_tc) SC4_TRY(rows128_pack(g.S32, g.S_tc, st));
  SC4_CUDA(cudaStreamSynchronize(st));
  return SC4DVAR_OK;
}

size_t gyre_sweep_ws_bytes(const GyreGeom& g, int k, size_t tb) {
  return (size_t)(5 + g.S) * field_bytes(g, k, tb);
}

size_t gyre_prior_ws_bytes(const GyreGeom& g, int k, size_t tb) { return field_bytes(g, k, tb); }

int gyre_fwd(const GyreGeom& g, const double* x0, bool store, const double* y, double* d_out, double* obs_out,
             double* xN, void* ws, cudaStream_t st) {
  const int n = g.n;
  const size_t fb = field_bytes(g, 1, 8);
  char* w = static_cast<char*>(ws);
  double* x = reinterpret_cast<double*>(w);
  double* bufA = reinterpret_cast<double*>(w + fb);
  double* bufB = reinterpret_cast<double*>(w + 2 * fb);
  double* psi = reinterpret_cast<double*>(w + 3 * fb);
  double* tmp = reinterpret_cast<double*>(w + 4 * fb);
  double* K[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int s = 0; s < g.S; ++s) K[s] = reinterpret_cast<double*>(w + (5 + s) * fb);
  SC4_CUDA(cudaMemcpyAsync(x, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const GyP<double> p = make_p<double>(g);
  const double isg = 1.0 / g.sigma;
  for (int t = 0; t < g.N; ++t) {
    for (int s = 0; s < g.S; ++s) {
      const double* X = s == 0 ? x : (s % 2 == 1 ? bufA : bufB);
      SC4_TRY(poisson<double>(g, 1, X, psi, tmp, st));
      FwdStage a{};
      a.X = X;
      a.psi = psi;
      a.x = x;
      a.last = s == g.S - 1;
      a.next = a.last ? x : ((s + 1) % 2 == 1 ? bufA : bufB);
      for (int q = 0; q < 4; ++q) {
        a.K[q] = K[q];
        a.cK[q] = a.last ? g.dt * g.b[q] : (s + 1 < 4 ? g.dt * g.a[s + 1][q] : 0.0);
      }
      a.s = s;
      if (store) {
        const size_t row = ((size_t)t * g.S + s) * n;
        a.om_st = g.om64 + row;
        a.ps_st = g.ps64 + row;
        a.om_st32 = g.om32 + row;
        a.ps_st32 = g.ps32 + row;
      }
      gy_fwd_stage_kernel<<<blocks_of(n), 256, 0, st>>>(p, a, g.Fy);
      SC4_LAUNCH_CHECK();
    }
    const int oi = g.obs_of_step_h[t + 1];
    if (oi >= 0 && (d_out || obs_out)) {
      gy_fwd_obs_kernel<<<div_up(g.n_o, 128), 128, 0, st>>>(g.n_o, x, g.obs_idx + (size_t)oi * g.n_o, y, d_out,
                                                            obs_out, isg, oi * g.n_o);
      SC4_LAUNCH_CHECK();
    }
  }
  if (xN) SC4_CUDA(cudaMemcpyAsync(xN, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SC4DVAR_OK;
}

template <typename T>
int gyre_tlm(const GyreGeom& g, const T* U0, int ldu, int k, T* W, int ldw, void* ws, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  SC4_ARG(k <= 65535, "double gyre: at most 65535 directions per sweep (one grid row per direction)");
  const int n = g.n;
  const size_t fb = field_bytes(g, k, sizeof(T));
  char* w = static_cast<char*>(ws);
  T* dom = reinterpret_cast<T*>(w);
  T* bufA = reinterpret_cast<T*>(w + fb);
  T* bufB = reinterpret_cast<T*>(w + 2 * fb);
  T* dpsi = reinterpret_cast<T*>(w + 3 * fb);
  T* tmp = reinterpret_cast<T*>(w + 4 * fb);
  T* K[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int s = 0; s < g.S; ++s) K[s] = reinterpret_cast<T*>(w + (5 + s) * fb);
  SC4_TRY((copy_fields<T, T>(n, k, U0, ldu, dom, n, st)));
  const GyP<T> p = make_p<T>(g);
  const T* om = om_of<T>(g);
  const T* ps = ps_of<T>(g);
  const T isg = (T)(1.0 / g.sigma);
  for (int t = 0; t < g.N; ++t) {
    for (int s = 0; s < g.S; ++s) {
      const T* X = s == 0 ? dom : (s % 2 == 1 ? bufA : bufB);
      SC4_TRY(poisson<T>(g, k, X, dpsi, tmp, st));
      TlmStage<T> a{};
      a.dX = X;
      a.dpsi = dpsi;
      a.dom = dom;
      a.last = s == g.S - 1;
      a.next = a.last ? dom : ((s + 1) % 2 == 1 ? bufA : bufB);
      for (int q = 0; q < 4; ++q) {
        a.K[q] = K[q];
        a.cK[q] = (T)(a.last ? g.dt * g.b[q] : (s + 1 < 4 ? g.dt * g.a[s + 1][q] : 0.0));
      }
      a.s = s;
      const size_t row = ((size_t)t * g.S + s) * n;
      gy_tlm_stage_kernel<T><<<dim3(blocks_of(n), div_up(k, kGyFields)), 256, 0, st>>>(p, k, om + row, ps + row, a);
      SC4_LAUNCH_CHECK();
    }
    const int oi = g.obs_of_step_h[t + 1];
    if (oi >= 0) {
      gy_tlm_obs_kernel<T><<<div_up(k * g.n_o, 256), 256, 0, st>>>(n, g.n_o, k, dom, g.obs_idx + (size_t)oi * g.n_o,
                                                                   isg, W, ldw, oi * g.n_o);
      SC4_LAUNCH_CHECK();
    }
  }
  return SC4DVAR_OK;
}

template <typename T>
int gyre_adj(const GyreGeom& g, const T* W, int ldw, int k, T* Out, int ldo, void* ws, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  SC4_ARG(k <= 65535, "double gyre: at most 65535 directions per sweep (one grid row per direction)");
  const int n = g.n;
  const size_t fb = field_bytes(g, k, sizeof(T));
  char* w = static_cast<char*>(ws);
  T* lam[2] = {reinterpret_cast<T*>(w), reinterpret_cast<T*>(w + fb)};
  T* gb = reinterpret_cast<T*>(w + 2 * fb);
  T* phi = reinterpret_cast<T*>(w + 3 * fb);
  T* tmp = reinterpret_cast<T*>(w + 4 * fb);
  T* Th[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int s = 0; s < g.S; ++s) Th[s] = reinterpret_cast<T*>(w + (5 + s) * fb);
  SC4_CUDA(cudaMemsetAsync(lam[0], 0, (size_t)k * n * sizeof(T), st));
  const GyP<T> p = make_p<T>(g);
  const T* om = om_of<T>(g);
  const T* ps = ps_of<T>(g);
  const T isg = (T)(1.0 / g.sigma);
  int cur = 0;
  for (int t = g.N; t >= 1; --t) {
    const int oi = g.obs_of_step_h[t];
    if (oi >= 0) {
      gy_adj_obs_kernel<T><<<div_up(k * g.n_o, 256), 256, 0, st>>>(n, g.n_o, k, lam[cur],
                                                                   g.obs_idx + (size_t)oi * g.n_o, isg, W, ldw,
                                                                   oi * g.n_o);
      SC4_LAUNCH_CHECK();
    }
    for (int s = g.S - 1; s >= 0; --s) {
      // kappa_s = h b_s lambda' + h sum_{j>s} a_js theta_j
      Comb<T> kap{};
      kap.src[0] = lam[cur];
      kap.c[0] = (T)(g.dt * g.b[s]);
      kap.m = 1;
      for (int jj = s + 1; jj < g.S; ++jj)
        if (g.a[jj][s] != 0.0) {
          kap.src[kap.m] = Th[jj];
          kap.c[kap.m] = (T)(g.dt * g.a[jj][s]);
          ++kap.m;
        }
      for (int q = kap.m; q < 4; ++q) {
        kap.src[q] = lam[cur];
        kap.c[q] = T(0);
      }
      const size_t row = ((size_t)(t - 1) * g.S + s) * n;
      gy_adj_pre_kernel<T><<<dim3(blocks_of(n), div_up(k, kGyFields)), 256, 0, st>>>(p, k, om + row, kap, gb);
      SC4_LAUNCH_CHECK();
      SC4_TRY(poisson<T>(g, k, gb, phi, tmp, st));
      AdjPost<T> a{};
      a.phi = phi;
      a.lam = lam[cur];
      a.lam_out = lam[cur ^ 1];
      for (int q = 0; q < 4; ++q) a.Th[q] = Th[q];
      a.s = s;
      gy_adj_post_kernel<T><<<dim3(blocks_of(n), div_up(k, kGyFields)), 256, 0, st>>>(p, k, ps + row, kap, a, g.S);
      SC4_LAUNCH_CHECK();
    }
    cur ^= 1;
  }
  return copy_fields<T, T>(n, k, lam[cur], n, Out, ldo, st);
}

template <typename TI, typename TO, typename TZ>
int gyre_prior_apply(const GyreGeom& g, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz, void* ws,
                     cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  constexpr bool f32 = sizeof(TI) == 4 && sizeof(TO) == 4;
  using TC = typename std::conditional<f32, float, double>::type;
  TC* tmp = static_cast<TC*>(ws);
  const TC* Sm = S_of<TC>(g);
  SC4_TRY((dst_rows<TI, TC, TC, TC>(g, k, X, ldx, Sm, tmp, g.n, (const TC*)nullptr, 0, st)));
  SC4_TRY(thomas<TC>(g, k, tmp, g.n, prior_of<TC>(g), g.prior_off, st));
  SC4_TRY((dst_rows<TC, TC, TO, TZ>(g, k, tmp, g.n, Sm, Y, ldy, Z, ldz, st)));
  return SC4DVAR_OK;
}

template int gyre_tlm<double>(const GyreGeom&, const double*, int, int, double*, int, void*, cudaStream_t);
template int gyre_tlm<float>(const GyreGeom&, const float*, int, int, float*, int, void*, cudaStream_t);
template int gyre_adj<double>(const GyreGeom&, const double*, int, int, double*, int, void*, cudaStream_t);
template int gyre_adj<float>(const GyreGeom&, const float*, int, int, float*, int, void*, cudaStream_t);
#define SC4_GY_PRIOR(TI, TO, TZ)                                                                      \
  template int gyre_prior_apply<TI, TO, TZ>(const GyreGeom&, int, const TI*, int, TO*, int, const TZ*, int, \
                                             void*, cudaStream_t);
SC4_GY_PRIOR(double, double, double)
SC4_GY_PRIOR(float, float, float)
SC4_GY_PRIOR(double, float, float)
SC4_GY_PRIOR(float, double, double)
#undef SC4_GY_PRIOR

}  // namespace sc4
