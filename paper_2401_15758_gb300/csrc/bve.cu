// Barotropic vorticity model: FWD / TLM / ADJ sweeps and the 2D FFT multiplier.
//
// Model (doubly periodic [0, 2 pi)^2, N x N points, d = 2 pi / N; the workload
// form of the paper's Sec. 5.2 equation):
//   q_t = -J_A(psi, q) + nu Lap_h q + a sin(k_f y),   psi = Lap^{-1} q (spectral)
// with J_A Arakawa's nine-point Jacobian and Lap_h the five-point Laplacian.
// TLM stage:  dk = -J_A(Lap^{-1} dq, q) - J_A(psi, dq) + nu Lap_h dq
// ADJ stage:  theta = -Lap^{-1} J_A(q, kappa) + J_A(psi, kappa) + nu Lap_h kappa
// (exact transposes: Lap^{-1}, Lap_h symmetric; J_A antisymmetric in its two
// arguments and skew-symmetric in the second), inside the same discrete RK4
// adjoint as the Burgers sweeps.
//
// GB300 mapping. The field of one direction (N^2 up to 1M points) does not fit
// one SM, so the sweeps stream: per RK stage, batched kernels over all k
// directions -- a 2D FFT multiplier (Poisson solve) and one stencil kernel --
// with the base stage states q_s, psi_s stored by the FWD and shared by all
// directions through L2. Fields are row-major (y slow, x fast).
//
// 2D FFT multiplier Y = IFFT2(S . FFT2(X)) with a real, even symbol S: two real
// fields are transformed together as one complex field (the multiplier maps
// real fields to real fields). Three kernels: row FFTs; column FFT, symbol,
// inverse column FFT (one pass); inverse row FFTs. Radix-2 in shared memory with
// a per-problem twiddle table.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include "bve.cuh"
#include "common.cuh"

namespace sc4 {

template <typename C> struct CplxOf;
template <> struct CplxOf<float2> { using R = float; };
template <> struct CplxOf<double2> { using R = double; };
template <typename R> struct CplxT;
template <> struct CplxT<float> { using C = float2; };
template <> struct CplxT<double> { using C = double2; };

template <typename C>
__device__ __forceinline__ C cmk(typename CplxOf<C>::R x, typename CplxOf<C>::R y) { C c; c.x = x; c.y = y; return c; }
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__device__ __forceinline__ unsigned brev_n(unsigned j, int logn) { return __brev(j) >> (32 - logn); }

// Radix-2 transforms of `nb` sequences of length N in shared memory; element
// (b, i) at s[b * sb + i * si]. DIT: bit-reversed in, natural out. DIF: natural
// in, bit-reversed out. dir = -1 forward, +1 inverse (unscaled). Work items are
// ordered so that consecutive threads touch consecutive addresses.
template <typename C, bool DIT>
__device__ void fft_batch(C* s, int N, int nb, int sb, int si, bool b_fast, const C* __restrict__ tw,
                          int dir) {
  const int nbf = N / 2;
  for (int step = 0, half = DIT ? 1 : N / 2; step < 32 && half >= 1 && half < N;
       ++step, half = DIT ? half * 2 : half / 2) {
    const int stride = N / (2 * half);
    __syncthreads();
    for (int it = threadIdx.x; it < nb * nbf; it += blockDim.x) {
      int b, bf;
      if (b_fast) { b = it % nb; bf = it / nb; }
      else { bf = it % nbf; b = it / nbf; }
      int grp = bf / half, kk = bf - grp * half;
      int i0 = grp * 2 * half + kk, i1 = i0 + half;
      C w = tw[kk * stride];
      if (dir > 0) w.y = -w.y;
      C* p0 = s + b * sb + i0 * si;
      C* p1 = s + b * sb + i1 * si;
      C u = *p0, v = *p1;
      if (DIT) {
        C t = cmulc(w, v);
        *p0 = cmk<C>(u.x + t.x, u.y + t.y);
        *p1 = cmk<C>(u.x - t.x, u.y - t.y);
      } else {
        *p0 = cmk<C>(u.x + v.x, u.y + v.y);
        *p1 = cmulc(w, cmk<C>(u.x - v.x, u.y - v.y));
      }
    }
  }
  __syncthreads();
}

// rows, forward: fields (2p, 2p+1) -> complex rows (natural kx), RB rows per CTA
template <typename C, typename RI>
__global__ void fft2_rows_fwd(int N, int logN, int k, const RI* __restrict__ X, int ldx, C* cbuf,
                              const C* __restrict__ tw, int RB) {
  using R = typename CplxOf<C>::R;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tile = reinterpret_cast<C*>(smraw);  // [RB][N]
  const int p = blockIdx.y, fa = 2 * p, fb = 2 * p + 1;
  const int j0 = blockIdx.x * RB;
  const RI* xa = X + (size_t)fa * ldx;
  const RI* xb = X + (size_t)fb * ldx;
  const bool hasb = fb < k;
  for (int it = threadIdx.x; it < RB * N; it += blockDim.x) {
    int r = it / N, i = it - r * N;
    size_t g = (size_t)(j0 + r) * N + i;
    tile[r * N + brev_n(i, logN)] = cmk<C>((R)xa[g], hasb ? (R)xb[g] : (R)0);
  }
  fft_batch<C, true>(tile, N, RB, N, 1, false, tw, -1);
  C* out = cbuf + (size_t)p * N * N;
  for (int it = threadIdx.x; it < RB * N; it += blockDim.x) {
    int r = it / N, i = it - r * N;
    out[(size_t)(j0 + r) * N + i] = tile[r * N + i];
  }
}

// columns: forward FFT along y, multiply by the symbol, inverse FFT along y
template <typename C>
__global__ void fft2_cols(int N, int logN, C* cbuf, const double* __restrict__ table,
                          const C* __restrict__ tw, int CB) {
  using R = typename CplxOf<C>::R;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tile = reinterpret_cast<C*>(smraw);  // [N][CB+1]
  const int ld = CB + 1;
  const int p = blockIdx.y;
  const int i0 = blockIdx.x * CB;
  C* g = cbuf + (size_t)p * N * N;
  for (int it = threadIdx.x; it < N * CB; it += blockDim.x) {
    int j = it / CB, c = it - j * CB;
    tile[brev_n(j, logN) * ld + c] = g[(size_t)j * N + i0 + c];
  }
  fft_batch<C, true>(tile, N, CB, 1, ld, true, tw, -1);
  for (int it = threadIdx.x; it < N * CB; it += blockDim.x) {
    int j = it / CB, c = it - j * CB;
    R s = (R)table[(size_t)j * N + i0 + c];
    C v = tile[j * ld + c];
    tile[j * ld + c] = cmk<C>(v.x * s, v.y * s);
  }
  fft_batch<C, false>(tile, N, CB, 1, ld, true, tw, +1);
  for (int it = threadIdx.x; it < N * CB; it += blockDim.x) {
    int j = it / CB, c = it - j * CB;
    g[(size_t)j * N + i0 + c] = tile[brev_n(j, logN) * ld + c];
  }
}

// rows, inverse: complex rows -> fields (2p, 2p+1), scaled by 1/N^2 (+ Z)
template <typename C, typename RO, typename RZ>
__global__ void fft2_rows_inv(int N, int logN, int k, const C* cbuf, RO* __restrict__ Y, int ldy,
                              const RZ* __restrict__ Z, int ldz, const C* __restrict__ tw, int RB) {
  using R = typename CplxOf<C>::R;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tile = reinterpret_cast<C*>(smraw);
  const int p = blockIdx.y, fa = 2 * p, fb = 2 * p + 1;
  const int j0 = blockIdx.x * RB;
  const bool hasb = fb < k;
  const C* in = cbuf + (size_t)p * N * N;
  for (int it = threadIdx.x; it < RB * N; it += blockDim.x) {
    int r = it / N, i = it - r * N;
    tile[r * N + i] = in[(size_t)(j0 + r) * N + i];
  }
  fft_batch<C, false>(tile, N, RB, N, 1, false, tw, +1);
  const R scale = (R)1 / ((R)N * (R)N);
  for (int it = threadIdx.x; it < RB * N; it += blockDim.x) {
    int r = it / N, i = it - r * N;
    size_t gi = (size_t)(j0 + r) * N + i;
    C v = tile[r * N + brev_n(i, logN)];
    R a = v.x * scale, b = v.y * scale;
    if (Z) {
      a += (R)Z[(size_t)fa * ldz + gi];
      if (hasb) b += (R)Z[(size_t)fb * ldz + gi];
    }
    Y[(size_t)fa * ldy + gi] = (RO)a;
    if (hasb) Y[(size_t)fb * ldy + gi] = (RO)b;
  }
}

// ---- warp-resident FFTs (N >= 32): lane l holds elements i = r * 32 + l ----
// Stages whose butterfly span is below 32 exchange values across lanes with
// shfl_xor; longer spans pair registers of the same lane. DIF: natural order in,
// bit-reversed out. DIT: bit-reversed in, natural out. No shared memory and no
// barriers; twiddles w_j = exp(-2 pi i j / N) from the table (conjugated for the
// inverse).
template <typename C>
__device__ __forceinline__ C shfl_xor_c(C v, int m) {
  C o;
  o.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  o.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return o;
}

template <typename C>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int j, int dir) {
  C w = __ldg(tw + j);
  if (dir > 0) w.y = -w.y;
  return w;
}

template <typename C, int R>
__device__ __forceinline__ void warp_fft_dif(C (&v)[R], int lane, const C* __restrict__ tw, int N, int dir) {
#pragma unroll
  for (int hr = R / 2; hr >= 1; hr >>= 1) {
    const int stride = N / (64 * hr);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & hr) continue;
      C u = v[r], x = v[r + hr];
      C w = twid(tw, ((r % hr) * 32 + lane) * stride, dir);
      v[r] = cmk<C>(u.x + x.x, u.y + x.y);
      v[r + hr] = cmulc(w, cmk<C>(u.x - x.x, u.y - x.y));
    }
  }
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool upper = (lane & half) == 0;
    C w = twid(tw, (lane & (half - 1)) * (N / (2 * half)), dir);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C o = shfl_xor_c(v[r], half);
      if (upper) v[r] = cmk<C>(v[r].x + o.x, v[r].y + o.y);
      else v[r] = cmulc(w, cmk<C>(o.x - v[r].x, o.y - v[r].y));
    }
  }
}

template <typename C, int R>
__device__ __forceinline__ void warp_fft_dit(C (&v)[R], int lane, const C* __restrict__ tw, int N, int dir) {
#pragma unroll
  for (int half = 1; half <= 16; half <<= 1) {
    const bool upper = (lane & half) == 0;
    C w = twid(tw, (lane & (half - 1)) * (N / (2 * half)), dir);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C o = shfl_xor_c(v[r], half);
      if (upper) {
        C t = cmulc(w, o);
        v[r] = cmk<C>(v[r].x + t.x, v[r].y + t.y);
      } else {
        C t = cmulc(w, v[r]);
        v[r] = cmk<C>(o.x - t.x, o.y - t.y);
      }
    }
  }
#pragma unroll
  for (int hr = 1; hr < R; hr <<= 1) {
    const int stride = N / (64 * hr);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & hr) continue;
      C w = twid(tw, ((r % hr) * 32 + lane) * stride, dir);
      C t = cmulc(w, v[r + hr]);
      v[r + hr] = cmk<C>(v[r].x - t.x, v[r].y - t.y);
      v[r] = cmk<C>(v[r].x + t.x, v[r].y + t.y);
    }
  }
}

// rows forward: one warp per row of a field pair; complex output in bit-reversed kx order
template <typename C, typename RI, int R>
__global__ void __launch_bounds__(256) wfft_rows_fwd(int N, int k, const RI* __restrict__ X, int ldx,
                                                     C* cbuf, const C* __restrict__ tw) {
  using Rl = typename CplxOf<C>::R;
  const int lane = threadIdx.x & 31, j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int p = blockIdx.y, fa = 2 * p, fb = 2 * p + 1;
  if (j >= N) return;
  const bool hasb = fb < k;
  const RI* xa = X + (size_t)fa * ldx + (size_t)j * N;
  const RI* xb = X + (size_t)fb * ldx + (size_t)j * N;
  C v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = cmk<C>((Rl)xa[r * 32 + lane], hasb ? (Rl)xb[r * 32 + lane] : (Rl)0);
  warp_fft_dif<C, R>(v, lane, tw, N, -1);
  C* out = cbuf + (size_t)p * N * N + (size_t)j * N;
#pragma unroll
  for (int r = 0; r < R; ++r) out[r * 32 + lane] = v[r];
}

// Column pass of the 2D multiplier (forward transform along y, symbol,
// inverse transform along y) with lanes mapped to columns: a block owns CB
// adjacent columns of one complex field and all N rows, thread (g, c) =
// (tid / CB, tid % CB), so every load and store is a full row segment of the
// block and no butterfly crosses lanes. A thread holds R = N / G values of its
// column: rows g + G r (interleaved layout) or rows g R + r (blocked layout;
// G^2 <= N keeps spans below G inside a thread there). Forward DIF: spans
// N/2 .. G interleaved, one shared-memory transpose, spans G/2 .. 1 blocked;
// multiply by the symbol at the bit-reversed (ky, kx) that the DIF leaves;
// inverse DIT: spans 1 .. G/2 blocked, transpose back, G .. N/2 interleaved.
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }

// w^idx v with the two trivial twiddles (idx 0: 1; idx N/4: -i forward, +i
// inverse) applied without a multiply; where idx is a compile-time constant
// after unrolling the branches fold away. tw[0] = 1 and tw[N/4] = -i exactly,
// so the result equals the general product.
template <typename C, int N>
__device__ __forceinline__ C twmul(const C* __restrict__ tw, int idx, int dir, C v) {
  if (idx == 0) return v;
  if (idx == N / 4) return dir < 0 ? cmk<C>(v.y, -v.x) : cmk<C>(-v.y, v.x);
  return cmulc(twid(tw, idx, dir), v);
}

template <typename C, int N, int CB, int G, int MINB>
__global__ void __launch_bounds__(G * CB, MINB) wfft_cols2(C* cbuf, const typename CplxOf<C>::R* __restrict__ tab,
                                                           const C* __restrict__ tw) {
  constexpr int R = N / G;
  static_assert(G * G <= N && R >= 2, "two-phase column split needs G^2 <= N");
  using Rl = typename CplxOf<C>::R;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tile = reinterpret_cast<C*>(smraw);  // [N][CB]
  const int c = threadIdx.x % CB, gi = threadIdx.x / CB;
  const int col = blockIdx.x * CB + c;
  C* gcol = cbuf + (size_t)blockIdx.y * N * N + col;
  C v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = gcol[(size_t)(gi + G * r) * N];
  // forward DIF, interleaved rows j = gi + G r: span h = hr G
#pragma unroll
  for (int hr = R / 2; hr >= 1; hr >>= 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & hr) continue;
      const int jm = gi + G * (r & (hr - 1));  // j mod h
      C w = twid(tw, jm * (N / (2 * hr * G)), -1);
      C u = v[r], x = v[r + hr];
      v[r] = cadd(u, x);
      v[r + hr] = cmulc(w, csub(u, x));
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) tile[(gi + G * r) * CB + c] = v[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = tile[(gi * R + r) * CB + c];
  // forward DIF, blocked rows j = gi R + r: span h < G, j mod h = r mod h
#pragma unroll
  for (int h = G / 2; h >= 1; h >>= 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      C u = v[r], x = v[r + h];
      v[r] = cadd(u, x);
      v[r + h] = twmul<C, N>(tw, (r & (h - 1)) * (N / (2 * h)), -1, csub(u, x));
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const Rl sv = __ldg(tab + (size_t)(gi * R + r) * N + col);
    v[r] = cmk<C>(v[r].x * sv, v[r].y * sv);
  }
  // inverse DIT, blocked rows: spans 1 .. G/2
#pragma unroll
  for (int h = 1; h < G; h <<= 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      C t = twmul<C, N>(tw, (r & (h - 1)) * (N / (2 * h)), +1, v[r + h]);
      v[r + h] = csub(v[r], t);
      v[r] = cadd(v[r], t);
    }
  }
  // each thread rewrites exactly the slots it read, so no barrier is needed here
#pragma unroll
  for (int r = 0; r < R; ++r) tile[(gi * R + r) * CB + c] = v[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = tile[(gi + G * r) * CB + c];
  // inverse DIT, interleaved rows: spans G .. N/2
#pragma unroll
  for (int hr = 1; hr < R; hr <<= 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & hr) continue;
      const int jm = gi + G * (r & (hr - 1));
      C w = twid(tw, jm * (N / (2 * hr * G)), +1);
      C t = cmulc(w, v[r + hr]);
      v[r + hr] = csub(v[r], t);
      v[r] = cadd(v[r], t);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) gcol[(size_t)(gi + G * r) * N] = v[r];
}

// rows inverse: bit-reversed kx in (DIT), natural x out, scaled 1/N^2 (+ Z)
template <typename C, typename RO, typename RZ, int R>
__global__ void __launch_bounds__(256) wfft_rows_inv(int N, int k, const C* cbuf, RO* __restrict__ Y,
                                                     int ldy, const RZ* __restrict__ Z, int ldz,
                                                     const C* __restrict__ tw) {
  using Rl = typename CplxOf<C>::R;
  const int lane = threadIdx.x & 31, j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int p = blockIdx.y, fa = 2 * p, fb = 2 * p + 1;
  if (j >= N) return;
  const bool hasb = fb < k;
  const C* in = cbuf + (size_t)p * N * N + (size_t)j * N;
  C v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[r * 32 + lane];
  warp_fft_dit<C, R>(v, lane, tw, N, +1);
  const Rl scale = (Rl)1 / ((Rl)N * (Rl)N);
  const size_t ra = (size_t)fa * ldy + (size_t)j * N, rb = (size_t)fb * ldy + (size_t)j * N;
  const size_t za = (size_t)fa * ldz + (size_t)j * N, zb = (size_t)fb * ldz + (size_t)j * N;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = r * 32 + lane;
    Rl a = v[r].x * scale, b = v[r].y * scale;
    if (Z) {
      a += (Rl)Z[za + i];
      if (hasb) b += (Rl)Z[zb + i];
    }
    Y[ra + i] = (RO)a;
    if (hasb) Y[rb + i] = (RO)b;
  }
}

__global__ void bve_twiddle_kernel(int N, double2* tw64, float2* tw32) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N / 2) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)N, &s, &c);
    tw64[j] = make_double2(c, s);
    tw32[j] = make_float2((float)c, (float)s);
  }
}

// Column-pass copy of a symbol table: entry (j, i) = S(ky = bitrev(j), kx =
// bitrev(i)) at j * N + i, in the real type of the transform (the row and
// column DIFs leave both wavenumbers in bit-reversed order), so the lanes of a
// row segment read adjacent entries.
template <typename R>
__global__ void bve_table_brev_kernel(int N, int logN, const double* __restrict__ table, R* out) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)N * N) {
    int j = (int)(idx / N), i = (int)(idx % N);
    out[idx] = (R)table[(size_t)brev_n(j, logN) * N + brev_n(i, logN)];
  }
}

// kind 0: Poisson -1/|kappa|^2 (0 at kappa = 0); kind 1: c / (1 + ell^2 |kappa|^2)
__global__ void bve_table_kernel(int N, int kind, double c, double ell, double* table) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)N * N) {
    int j = (int)(idx / N), i = (int)(idx % N);
    double kx = (i < N / 2) ? i : i - N;
    double ky = (j < N / 2) ? j : j - N;
    double k2 = kx * kx + ky * ky;
    table[idx] = (kind == 0) ? (k2 > 0 ? -1.0 / k2 : 0.0) : c / (1.0 + ell * ell * k2);
  }
}

// ------------------------------------------------------------------ stencils
template <typename T>
struct St9 {
  T c, e, w, n, s, ne, nw, se, sw;
};

// Arakawa J_A(a, b) times 12 d^2 (the mean of J++, J+x, Jx+ without its scale)
template <typename T>
__device__ __forceinline__ T arakawa12(const St9<T>& a, const St9<T>& b) {
  T jpp = (a.e - a.w) * (b.n - b.s) - (a.n - a.s) * (b.e - b.w);
  T jpx = a.e * (b.ne - b.se) - a.w * (b.nw - b.sw) - a.n * (b.ne - b.nw) + a.s * (b.se - b.sw);
  T jxp = b.n * (a.ne - a.nw) - b.s * (a.se - a.sw) - b.e * (a.ne - a.se) + b.w * (a.nw - a.sw);
  return jpp + jpx + jxp;
}

template <typename T>
__device__ __forceinline__ T lap5(const St9<T>& a) {
  return a.e + a.w + a.n + a.s - (T)4 * a.c;
}

__constant__ double kBveA[3] = {0.5, 0.5, 1.0};
__constant__ double kBveB[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

struct StencilConsts {
  double c12;    // 1 / (12 d^2)
  double nudd;   // nu / d^2
  double famp;   // forcing amplitude
  double fk_d;   // forcing wavenumber * d
};

// Stencil kernels: a block of 256 threads owns a tile of TX x TY points of
// one field (TX = min(N, 64); TY = min(N, 32) for FP32, min(N, 16) for FP64);
// every field read through the nine-point stencil is staged with its one-point
// periodic halo in shared memory by asynchronous copies (16-byte vectors for
// the tile interior), and the pointwise operands are loaded into registers
// before the wait, so all of a block's global loads are in flight at once.
constexpr int kTileThreads = 256;

template <typename T, int TX>
struct TileGeom {
  static constexpr int V = 16 / (int)sizeof(T);              // elements per 16-byte vector
  static constexpr int TY = sizeof(T) == 4 ? (TX < 32 ? TX : 32) : (TX < 16 ? TX : 16);
  static constexpr int O = V;                                // column of the first interior point
  static constexpr int W = TX + 2 * V;                       // row stride (16-byte multiple)
  static constexpr int SIZE = W * (TY + 2);
  static constexpr int P = TX * TY / kTileThreads;           // points per thread
  static constexpr int BANDS = kTileThreads / TX;            // row bands per tile (P rows each)
  static constexpr int UPR = TX / V + 2;                     // copies per row: vectors + two halos
};

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

// tile row jj <- f row (j0 - 1 + jj) mod N: interior columns i0 .. i0 + TX - 1
// at O .. O + TX - 1 (16-byte copies; i0 and N are multiples of TX, so both
// sides are 16-byte aligned), halos (i0 - 1) mod N at O - 1 and (i0 + TX) mod N
// at O + TX. tile_wait() completes the copies and synchronizes the block.
template <typename T, int TX>
__device__ __forceinline__ void tile_load(T* sm, const T* __restrict__ f, int N, int i0, int j0) {
  using TG = TileGeom<T, TX>;
  constexpr int UNITS = TG::UPR * (TG::TY + 2);
  constexpr int IT = (UNITS + kTileThreads - 1) / kTileThreads;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int u = it * kTileThreads + threadIdx.x;
    if (u < UNITS) {
      const int jj = u / TG::UPR, c = u - jj * TG::UPR;
      const T* row = f + (size_t)((j0 - 1 + jj) & (N - 1)) * N;
      T* srow = sm + jj * TG::W;
      if (c < TX / TG::V) cp_async16(srow + TG::O + c * TG::V, row + i0 + c * TG::V);
      else if (c == TX / TG::V) cp_async_elem(srow + TG::O - 1, row + ((i0 - 1) & (N - 1)));
      else cp_async_elem(srow + TG::O + TX, row + ((i0 + TX) & (N - 1)));
    }
  }
}
__device__ __forceinline__ void tile_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

// Three-row register window over a staged tile: a thread owns P consecutive
// interior rows of one column and slides down them, reading three values of
// the new row per step. n = row j + 1, e = column i + 1.
template <typename T, int TX>
struct TileWin {
  const T* col;     // the thread's column in tile row 0
  T sw, sc, se, mw, mc, me, nw, nc, ne;
  __device__ __forceinline__ void init(const T* sm, int tx, int ty) {  // ty: first interior row
    col = sm + TileGeom<T, TX>::O + tx;
    ld(ty, sw, sc, se);
    ld(ty + 1, mw, mc, me);
    ld(ty + 2, nw, nc, ne);
  }
  __device__ __forceinline__ void ld(int trow, T& w, T& c, T& e) const {
    const T* p = col + trow * TileGeom<T, TX>::W;
    w = p[-1]; c = p[0]; e = p[1];
  }
  __device__ __forceinline__ void advance(int ty) {  // ty: the new centre interior row
    sw = mw; sc = mc; se = me;
    mw = nw; mc = nc; me = ne;
    ld(ty + 2, nw, nc, ne);
  }
  __device__ __forceinline__ St9<T> st() const {
    St9<T> v;
    v.c = mc; v.e = me; v.w = mw;
    v.n = nc; v.s = sc; v.ne = ne; v.nw = nw; v.se = se; v.sw = sw;
    return v;
  }
};

// FWD stage: f = -J_A(psi, X_s) + nu Lap X_s + F; acc += b_s f; next = x + h a_s f
// (s = 3: x += h acc). Single field.
template <typename T, int TX>
__global__ void __launch_bounds__(kTileThreads) bve_fwd_stage_kernel(int N, StencilConsts sc, int s, T h,
                                                                     const T* __restrict__ X,
                                                                     const T* __restrict__ psi, T* acc,
                                                                     T* x, T* next) {
  using TG = TileGeom<T, TX>;
  __shared__ __align__(16) T sq[TG::SIZE], sp[TG::SIZE];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TG::TY;
  const int tx = threadIdx.x % TX, ty0 = (threadIdx.x / TX) * TG::P;
  T a_r[TG::P], x_r[TG::P];
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    const size_t g = (size_t)(j0 + ty0 + r) * N + i0 + tx;
    a_r[r] = s == 0 ? (T)0 : acc[g];
    x_r[r] = x[g];
  }
  tile_load<T, TX>(sq, X, N, i0, j0);
  tile_load<T, TX>(sp, psi, N, i0, j0);
  tile_wait();
  TileWin<T, TX> q, ps;
  q.init(sq, tx, ty0);
  ps.init(sp, tx, ty0);
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    const int j = j0 + ty0 + r;
    if (r) { q.advance(ty0 + r); ps.advance(ty0 + r); }
    St9<T> qq = q.st(), pp = ps.st();
    T f = -(T)sc.c12 * arakawa12(pp, qq) + (T)sc.nudd * lap5(qq) + (T)(sc.famp * sin(sc.fk_d * j));
    const size_t g = (size_t)j * N + i0 + tx;
    T a = a_r[r] + (T)kBveB[s] * f;
    if (s < 3) {
      acc[g] = a;
      next[g] = x_r[r] + h * (T)kBveA[s] * f;
    } else {
      x[g] = x_r[r] + h * a;
    }
  }
}

// TLM stage over k directions (base q_s, psi_s shared; direction = blockIdx.z):
// dk = -J_A(dpsi, q_s) - J_A(psi_s, dq) + nu Lap dq; acc += b_s dk;
// next = dx + h a_s dk (s = 3: dx += h acc).
template <typename T, int TX>
__global__ void __launch_bounds__(kTileThreads) bve_tlm_stage_kernel(int N, StencilConsts sc, int s, T h,
                                                                     const T* __restrict__ qb,
                                                                     const T* __restrict__ pb,
                                                                     const T* __restrict__ cur,
                                                                     const T* __restrict__ dpsi, T* acc,
                                                                     T* dx, T* next, size_t ld) {
  using TG = TileGeom<T, TX>;
  __shared__ __align__(16) T sq[TG::SIZE], sp[TG::SIZE], sd[TG::SIZE], sdp[TG::SIZE];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TG::TY;
  const int tx = threadIdx.x % TX, ty0 = (threadIdx.x / TX) * TG::P;
  const size_t off = (size_t)blockIdx.z * ld;
  T a_r[TG::P], x_r[TG::P];
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    const size_t g = off + (size_t)(j0 + ty0 + r) * N + i0 + tx;
    a_r[r] = s == 0 ? (T)0 : acc[g];
    x_r[r] = dx[g];
  }
  tile_load<T, TX>(sd, cur + off, N, i0, j0);
  tile_load<T, TX>(sdp, dpsi + off, N, i0, j0);
  tile_load<T, TX>(sq, qb, N, i0, j0);
  tile_load<T, TX>(sp, pb, N, i0, j0);
  tile_wait();
  const T bs = (T)kBveB[s];
  const T ha = (s < 3) ? h * (T)kBveA[s] : (T)0;
  TileWin<T, TX> q, ps, d, dp;
  q.init(sq, tx, ty0);
  ps.init(sp, tx, ty0);
  d.init(sd, tx, ty0);
  dp.init(sdp, tx, ty0);
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    if (r) { q.advance(ty0 + r); ps.advance(ty0 + r); d.advance(ty0 + r); dp.advance(ty0 + r); }
    St9<T> qq = q.st(), pp = ps.st(), dd = d.st(), ddp = dp.st();
    T dk = -(T)sc.c12 * (arakawa12(ddp, qq) + arakawa12(pp, dd)) + (T)sc.nudd * lap5(dd);
    const size_t g = off + (size_t)(j0 + ty0 + r) * N + i0 + tx;
    T a = a_r[r] + bs * dk;
    if (s < 3) {
      acc[g] = a;
      next[g] = x_r[r] + ha * dk;
    } else {
      dx[g] = x_r[r] + h * a;
    }
  }
}

// ADJ: T1 = J_A(q_s, kappa)
template <typename T, int TX>
__global__ void __launch_bounds__(kTileThreads) bve_adj_jac_kernel(int N, StencilConsts sc,
                                                                   const T* __restrict__ qb,
                                                                   const T* __restrict__ kap, T* t1,
                                                                   size_t ld) {
  using TG = TileGeom<T, TX>;
  __shared__ __align__(16) T sq[TG::SIZE], sk[TG::SIZE];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TG::TY;
  const int tx = threadIdx.x % TX, ty0 = (threadIdx.x / TX) * TG::P;
  const size_t off = (size_t)blockIdx.z * ld;
  tile_load<T, TX>(sk, kap + off, N, i0, j0);
  tile_load<T, TX>(sq, qb, N, i0, j0);
  tile_wait();
  TileWin<T, TX> q, kk;
  q.init(sq, tx, ty0);
  kk.init(sk, tx, ty0);
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    if (r) { q.advance(ty0 + r); kk.advance(ty0 + r); }
    t1[off + (size_t)(j0 + ty0 + r) * N + i0 + tx] = (T)sc.c12 * arakawa12(q.st(), kk.st());
  }
}

// ADJ stage: theta = -T2 + J_A(psi_s, kappa) + nu Lap kappa; th += theta;
// s > 0: kappa_{s-1} = h b_{s-1} lam + h a_{s-1} theta; s = 0: lam += th
template <typename T, int TX>
__global__ void __launch_bounds__(kTileThreads) bve_adj_stage_kernel(int N, StencilConsts sc, int s, T h,
                                                                     const T* __restrict__ pb,
                                                                     const T* __restrict__ kap,
                                                                     const T* __restrict__ t2, T* th,
                                                                     T* lam, T* knext, size_t ld) {
  using TG = TileGeom<T, TX>;
  __shared__ __align__(16) T sp[TG::SIZE], sk[TG::SIZE];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TG::TY;
  const int tx = threadIdx.x % TX, ty0 = (threadIdx.x / TX) * TG::P;
  const size_t off = (size_t)blockIdx.z * ld;
  T t2_r[TG::P], th_r[TG::P], l_r[TG::P];
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    const size_t g = off + (size_t)(j0 + ty0 + r) * N + i0 + tx;
    t2_r[r] = t2[g];
    th_r[r] = s == 3 ? (T)0 : th[g];
    l_r[r] = lam[g];
  }
  tile_load<T, TX>(sk, kap + off, N, i0, j0);
  tile_load<T, TX>(sp, pb, N, i0, j0);
  tile_wait();
  const T hb = (s > 0) ? h * (T)kBveB[s - 1] : (T)0;
  const T ha = (s > 0) ? h * (T)kBveA[s - 1] : (T)0;
  TileWin<T, TX> ps, kk;
  ps.init(sp, tx, ty0);
  kk.init(sk, tx, ty0);
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    if (r) { ps.advance(ty0 + r); kk.advance(ty0 + r); }
    St9<T> k9 = kk.st();
    const size_t g = off + (size_t)(j0 + ty0 + r) * N + i0 + tx;
    T theta = -t2_r[r] + (T)sc.c12 * arakawa12(ps.st(), k9) + (T)sc.nudd * lap5(k9);
    T a = th_r[r] + theta;
    if (s > 0) {
      th[g] = a;
      knext[g] = hb * l_r[r] + ha * theta;
    } else {
      lam[g] = l_r[r] + a;
    }
  }
}

// ---- two directions per thread in packed FP32x2 (FP32 blocks, N >= 64) ----
// Thread (tx, band) of block (x, y, zp) computes directions z = 2 zp and
// 2 zp + 1 at the same points: their values travel as float2 pairs (one
// 4-byte shared load per direction, no reshuffling), the base stencils (q_s,
// psi_s) are read once and broadcast to both lanes, and the stencil arithmetic
// runs on packed FP32x2 instructions. For odd k the last pair repeats
// direction z in its second lane and does not store it. Used for the TLM stage
// and the ADJ Jacobian (the ADJ stage kernel measured faster in scalar form,
// at higher occupancy).
using pf2 = float2;
__device__ __forceinline__ pf2 pmk(float a) { return make_float2(a, a); }
__device__ __forceinline__ pf2 padd(pf2 a, pf2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ pf2 pmul(pf2 a, pf2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ pf2 pfma(pf2 a, pf2 b, pf2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ pf2 psub(pf2 a, pf2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

struct St9p {
  pf2 c, e, w, n, s, ne, nw, se, sw;
};

__device__ __forceinline__ St9p bcast9(const St9<float>& v) {
  St9p o;
  o.c = pmk(v.c); o.e = pmk(v.e); o.w = pmk(v.w); o.n = pmk(v.n); o.s = pmk(v.s);
  o.ne = pmk(v.ne); o.nw = pmk(v.nw); o.se = pmk(v.se); o.sw = pmk(v.sw);
  return o;
}

// 12 d^2 J_A(a, b) on packed pairs (the three Jacobians of arakawa12)
__device__ __forceinline__ pf2 arakawa12p(const St9p& a, const St9p& b) {
  pf2 jpp = pfma(psub(a.e, a.w), psub(b.n, b.s), pmul(psub(a.s, a.n), psub(b.e, b.w)));
  pf2 jpx = pfma(a.e, psub(b.ne, b.se),
                 pfma(a.w, psub(b.sw, b.nw), pfma(a.n, psub(b.nw, b.ne), pmul(a.s, psub(b.se, b.sw)))));
  pf2 jxp = pfma(b.n, psub(a.ne, a.nw),
                 pfma(b.s, psub(a.sw, a.se), pfma(b.e, psub(a.se, a.ne), pmul(b.w, psub(a.nw, a.sw)))));
  return padd(padd(jpp, jpx), jxp);
}

__device__ __forceinline__ pf2 lap5p(const St9p& a) {
  return pfma(a.c, pmk(-4.f), padd(padd(a.e, a.w), padd(a.n, a.s)));
}

// three-row window over the same column of two staged tiles (two directions)
struct TileWin2 {
  const float* a;
  const float* b;
  pf2 sw, sc, se, mw, mc, me, nw, nc, ne;
  __device__ __forceinline__ void ld(int trow, pf2& w, pf2& c, pf2& e) const {
    const float* pa = a + trow * TileGeom<float, 64>::W;
    const float* pb = b + trow * TileGeom<float, 64>::W;
    w = make_float2(pa[-1], pb[-1]);
    c = make_float2(pa[0], pb[0]);
    e = make_float2(pa[1], pb[1]);
  }
  __device__ __forceinline__ void init(const float* ta, const float* tb, int tx, int ty) {
    a = ta + TileGeom<float, 64>::O + tx;
    b = tb + TileGeom<float, 64>::O + tx;
    ld(ty, sw, sc, se);
    ld(ty + 1, mw, mc, me);
    ld(ty + 2, nw, nc, ne);
  }
  __device__ __forceinline__ void advance(int ty) {
    sw = mw; sc = mc; se = me;
    mw = nw; mc = nc; me = ne;
    ld(ty + 2, nw, nc, ne);
  }
  __device__ __forceinline__ St9p st() const {
    St9p v;
    v.c = mc; v.e = me; v.w = mw;
    v.n = nc; v.s = sc; v.ne = ne; v.nw = nw; v.se = se; v.sw = sw;
    return v;
  }
};

__device__ __forceinline__ pf2 ld2(const float* f, size_t o0, size_t o1) { return make_float2(f[o0], f[o1]); }
__device__ __forceinline__ void st2(float* f, size_t o0, size_t o1, bool has1, pf2 v) {
  f[o0] = v.x;
  if (has1) f[o1] = v.y;
}

constexpr int kD2TlmTiles = 6;

__global__ void __launch_bounds__(kTileThreads) bve_tlm_stage_d2_kernel(int N, StencilConsts sc, int s, float h,
                                                                        const float* __restrict__ qb,
                                                                        const float* __restrict__ pb,
                                                                        const float* __restrict__ cur,
                                                                        const float* __restrict__ dpsi,
                                                                        float* acc, float* dx, float* next,
                                                                        size_t ld, int k) {
  using TG = TileGeom<float, 64>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* sq = reinterpret_cast<float*>(smraw);
  float* sp = sq + TG::SIZE;
  float* sd0 = sp + TG::SIZE;
  float* sd1 = sd0 + TG::SIZE;
  float* sg0 = sd1 + TG::SIZE;
  float* sg1 = sg0 + TG::SIZE;
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * TG::TY;
  const int tx = threadIdx.x % 64, ty0 = (threadIdx.x / 64) * TG::P;
  const int z0 = 2 * blockIdx.z;
  const bool has1 = z0 + 1 < k;
  const size_t off0 = (size_t)z0 * ld, off1 = has1 ? off0 + ld : off0;
  pf2 a_r[TG::P], x_r[TG::P];
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    const size_t g = (size_t)(j0 + ty0 + r) * N + i0 + tx;
    a_r[r] = s == 0 ? pmk(0.f) : ld2(acc, off0 + g, off1 + g);
    x_r[r] = ld2(dx, off0 + g, off1 + g);
  }
  tile_load<float, 64>(sd0, cur + off0, N, i0, j0);
  tile_load<float, 64>(sd1, cur + off1, N, i0, j0);
  tile_load<float, 64>(sg0, dpsi + off0, N, i0, j0);
  tile_load<float, 64>(sg1, dpsi + off1, N, i0, j0);
  tile_load<float, 64>(sq, qb, N, i0, j0);
  tile_load<float, 64>(sp, pb, N, i0, j0);
  tile_wait();
  const pf2 bs = pmk((float)kBveB[s]);
  const pf2 ha = pmk((s < 3) ? h * (float)kBveA[s] : 0.f);
  const pf2 mc12 = pmk(-(float)sc.c12), nudd = pmk((float)sc.nudd), h2 = pmk(h);
  TileWin<float, 64> q, ps;
  TileWin2 d, dp;
  q.init(sq, tx, ty0);
  ps.init(sp, tx, ty0);
  d.init(sd0, sd1, tx, ty0);
  dp.init(sg0, sg1, tx, ty0);
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    if (r) { q.advance(ty0 + r); ps.advance(ty0 + r); d.advance(ty0 + r); dp.advance(ty0 + r); }
    const St9p qq = bcast9(q.st()), pp = bcast9(ps.st()), dd = d.st(), ddp = dp.st();
    const pf2 dk = pfma(mc12, padd(arakawa12p(ddp, qq), arakawa12p(pp, dd)), pmul(nudd, lap5p(dd)));
    const size_t g = (size_t)(j0 + ty0 + r) * N + i0 + tx;
    const pf2 a = pfma(bs, dk, a_r[r]);
    if (s < 3) {
      st2(acc, off0 + g, off1 + g, has1, a);
      st2(next, off0 + g, off1 + g, has1, pfma(ha, dk, x_r[r]));
    } else {
      st2(dx, off0 + g, off1 + g, has1, pfma(h2, a, x_r[r]));
    }
  }
}

__global__ void __launch_bounds__(kTileThreads) bve_adj_jac_d2_kernel(int N, StencilConsts sc,
                                                                      const float* __restrict__ qb,
                                                                      const float* __restrict__ kap, float* t1,
                                                                      size_t ld, int k) {
  using TG = TileGeom<float, 64>;
  __shared__ __align__(16) float sq[TG::SIZE], sk0[TG::SIZE], sk1[TG::SIZE];
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * TG::TY;
  const int tx = threadIdx.x % 64, ty0 = (threadIdx.x / 64) * TG::P;
  const int z0 = 2 * blockIdx.z;
  const bool has1 = z0 + 1 < k;
  const size_t off0 = (size_t)z0 * ld, off1 = has1 ? off0 + ld : off0;
  tile_load<float, 64>(sk0, kap + off0, N, i0, j0);
  tile_load<float, 64>(sk1, kap + off1, N, i0, j0);
  tile_load<float, 64>(sq, qb, N, i0, j0);
  tile_wait();
  const pf2 c12 = pmk((float)sc.c12);
  TileWin<float, 64> q;
  TileWin2 kk;
  q.init(sq, tx, ty0);
  kk.init(sk0, sk1, tx, ty0);
#pragma unroll
  for (int r = 0; r < TG::P; ++r) {
    if (r) { q.advance(ty0 + r); kk.advance(ty0 + r); }
    const size_t g = (size_t)(j0 + ty0 + r) * N + i0 + tx;
    st2(t1, off0 + g, off1 + g, has1, pmul(c12, arakawa12p(bcast9(q.st()), kk.st())));
  }
}

template <typename T>
__global__ void scale_fields_kernel(size_t total, T a, const T* __restrict__ x, T* y) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x)
    y[idx] = a * x[idx];
}

template <typename T>
__global__ void copy_fields_kernel(size_t total, const T* __restrict__ x, T* y) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x)
    y[idx] = x[idx];
}

// observation gather / scatter for k directions
template <typename T>
__global__ void bve_gather_kernel(int n_o, const int* __restrict__ sites, const T* __restrict__ X,
                                  size_t ldx, T* W, int ldw, int row0, T inv_sigma) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  int col = blockIdx.y;
  if (o < n_o) W[(size_t)col * ldw + row0 + o] = X[(size_t)col * ldx + sites[o]] * inv_sigma;
}

template <typename T>
__global__ void bve_scatter_kernel(int n_o, const int* __restrict__ sites, const T* __restrict__ W,
                                   int ldw, int row0, T* X, size_t ldx, T inv_sigma) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  int col = blockIdx.y;
  if (o < n_o) atomicAdd(&X[(size_t)col * ldx + sites[o]], W[(size_t)col * ldw + row0 + o] * inv_sigma);
}

// FWD observation: obs_out = x[sites], d = (x[sites] - y) / sigma
__global__ void bve_fwd_obs_kernel(int n_o, const int* __restrict__ sites, const double* __restrict__ x,
                                   int row0, const double* __restrict__ y, double* d_out,
                                   double* obs_out, double inv_sigma) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n_o) {
    double v = x[sites[o]];
    if (obs_out) obs_out[row0 + o] = v;
    if (d_out) d_out[row0 + o] = (v - y[row0 + o]) * inv_sigma;
  }
}

// ------------------------------------------------------------------ host
static int log2i(int n) { return 31 - __builtin_clz((unsigned)n); }

// The bit-reversed copy of `table` in the transform's real type.
static const void* table_brev(const BveGeom& g, const double* table, size_t rb) {
  if (table == g.poisson) return rb == 4 ? (const void*)g.poisson_c32 : (const void*)g.poisson_c64;
  return rb == 4 ? (const void*)g.prior_c32 : (const void*)g.prior_c64;
}

template <typename C>
static const C* tw_of(const BveGeom& g);
template <> const double2* tw_of<double2>(const BveGeom& g) { return g.tw64; }
template <> const float2* tw_of<float2>(const BveGeom& g) { return g.tw32; }



// Column-pass shape: CB adjacent columns per block (16 FP32 / 8 FP64 complex
// values: a 128-byte row segment), G row groups with G^2 <= N, and a register
// cap (MINB resident blocks). FP32 grids of 256 and more points per side take
// one of four shapes (kColsShape below; SC4DVAR_COLS_SHAPE = 0..3 overrides
// it as a tuning knob): 0 = 16 columns, no cap; 1 = 16 columns, <= 64
// registers; 2 = 8 columns, no cap; 3 = 8 columns, <= 96 registers.
constexpr int col_groups(int N) { return N >= 1024 ? 32 : N >= 256 ? 16 : N >= 64 ? 8 : 4; }
constexpr int col_minb(int threads, int cap) {
  return cap == 0 ? 1 : (65536 / (threads * cap) > 0 ? 65536 / (threads * cap) : 1);
}
static int cols_shape(int N) {
  static const int env = [] {
    const char* e = getenv("SC4DVAR_COLS_SHAPE");
    return e ? atoi(e) : -1;
  }();
  if (env >= 0 && env <= 3) return env;
  return 3;
}

template <typename C, int N, int CB, int CAP>
static void launch_cols(int pairs, C* cb, const typename CplxOf<C>::R* tab, const C* tw, cudaStream_t st,
                        int* rc) {
  constexpr int G = col_groups(N);
  auto kc = wfft_cols2<C, N, CB, G, col_minb(G * CB, CAP)>;
  const size_t smc = (size_t)N * CB * sizeof(C);
  if (cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc) != cudaSuccess) {
    *rc = SC4DVAR_ERR_CUDA;
    return;
  }
  kc<<<dim3(N / CB, pairs), G * CB, smc, st>>>(cb, tab, tw);
}

// Rows per block of the row transforms (one warp per row): 8, fewer when the
// grid would not cover the GPU twice (single fields).
static int rows_per_block(int N, int pairs) {
  int rpb = 8;
  while (rpb > 1 && (N / rpb) * pairs < 2 * 152) rpb /= 2;
  return rpb;
}

template <typename C, typename RI, typename RO, typename RZ, int RR>
static int wfft2(const BveGeom& g, int k, const RI* X, int ldx, RO* Y, int ldy, const RZ* Z, int ldz,
                 const double* table, C* cb, cudaStream_t st) {
  constexpr int N = RR * 32;
  const int pairs = (k + 1) / 2;
  const int rpb = rows_per_block(N, pairs);
  wfft_rows_fwd<C, RI, RR><<<dim3(N / rpb, pairs), 32 * rpb, 0, st>>>(N, k, X, ldx, cb, tw_of<C>(g));
  SC4_LAUNCH_CHECK();
  using Rl = typename CplxOf<C>::R;
  const Rl* tab = reinterpret_cast<const Rl*>(table_brev(g, table, sizeof(Rl)));
  int rc = SC4DVAR_OK;
  if (N >= 128 && pairs * (N / 8) < 2 * 152) {
    // single fields: two columns per block spread the transform over the GPU
    launch_cols<C, N, 2, 0>(pairs, cb, tab, tw_of<C>(g), st, &rc);
  } else if constexpr (sizeof(C) == 8 && N >= 256) {
    switch (cols_shape(N)) {
      case 0: launch_cols<C, N, 16, 0>(pairs, cb, tab, tw_of<C>(g), st, &rc); break;
      case 1: launch_cols<C, N, 16, 64>(pairs, cb, tab, tw_of<C>(g), st, &rc); break;
      case 2: launch_cols<C, N, 8, 0>(pairs, cb, tab, tw_of<C>(g), st, &rc); break;
      default: launch_cols<C, N, 8, 96>(pairs, cb, tab, tw_of<C>(g), st, &rc); break;
    }
  } else {
    launch_cols<C, N, sizeof(C) == 8 ? 16 : 8, 0>(pairs, cb, tab, tw_of<C>(g), st, &rc);
  }
  if (rc != SC4DVAR_OK) {
    set_error("column pass: cudaFuncSetAttribute failed");
    return rc;
  }
  SC4_LAUNCH_CHECK();
  wfft_rows_inv<C, RO, RZ, RR><<<dim3(N / rpb, pairs), 32 * rpb, 0, st>>>(N, k, cb, Y, ldy, Z, ldz,
                                                                          tw_of<C>(g));
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template <typename R, typename RI, typename RO, typename RZ>
int fft2_apply(const BveGeom& g, int k, const RI* X, int ldx, RO* Y, int ldy, const RZ* Z, int ldz,
               const double* table, void* cbuf, cudaStream_t st) {
  using C = typename CplxT<R>::C;
  if (k <= 0) return SC4DVAR_OK;
  const int N = g.N, logN = log2i(N);
  const int pairs = (k + 1) / 2;
  C* cb = reinterpret_cast<C*>(cbuf);
  switch (N) {
    case 32: return wfft2<C, RI, RO, RZ, 1>(g, k, X, ldx, Y, ldy, Z, ldz, table, cb, st);
    case 64: return wfft2<C, RI, RO, RZ, 2>(g, k, X, ldx, Y, ldy, Z, ldz, table, cb, st);
    case 128: return wfft2<C, RI, RO, RZ, 4>(g, k, X, ldx, Y, ldy, Z, ldz, table, cb, st);
    case 256: return wfft2<C, RI, RO, RZ, 8>(g, k, X, ldx, Y, ldy, Z, ldz, table, cb, st);
    case 512: return wfft2<C, RI, RO, RZ, 16>(g, k, X, ldx, Y, ldy, Z, ldz, table, cb, st);
    case 1024: return wfft2<C, RI, RO, RZ, 32>(g, k, X, ldx, Y, ldy, Z, ldz, table, cb, st);
    default: break;  // N = 16: shared-memory radix-2 kernels below
  }
  int RB = std::max(1, std::min(16, (int)(32768 / (N * sizeof(C)))));
  while (N % RB) RB /= 2;
  int CB = (sizeof(C) == 8 || N <= 512) ? 16 : 8;
  size_t smr = (size_t)RB * N * sizeof(C);
  size_t smc = (size_t)N * (CB + 1) * sizeof(C);
  auto kr = fft2_rows_fwd<C, RI>;
  auto kc = fft2_cols<C>;
  auto ki = fft2_rows_inv<C, RO, RZ>;
  SC4_CUDA(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
  SC4_CUDA(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc));
  SC4_CUDA(cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
  kr<<<dim3(N / RB, pairs), 256, smr, st>>>(N, logN, k, X, ldx, cb, tw_of<C>(g), RB);
  SC4_LAUNCH_CHECK();
  kc<<<dim3(N / CB, pairs), 256, smc, st>>>(N, logN, cb, table, tw_of<C>(g), CB);
  SC4_LAUNCH_CHECK();
  ki<<<dim3(N / RB, pairs), 256, smr, st>>>(N, logN, k, cb, Y, ldy, Z, ldz, tw_of<C>(g), RB);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int bve_setup(BveGeom& g, cudaStream_t st) {
  const int N = g.N;
  bve_twiddle_kernel<<<div_up(N / 2, 256), 256, 0, st>>>(N, g.tw64, g.tw32);
  SC4_LAUNCH_CHECK();
  size_t nn = (size_t)N * N;
  bve_table_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(N, 0, 0.0, 0.0, g.poisson);
  SC4_LAUNCH_CHECK();
  bve_table_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(N, 1, g.prior_c, g.prior_ell, g.prior);
  SC4_LAUNCH_CHECK();
  const int logN = log2i(N);
  const unsigned nb = (unsigned)((nn + 255) / 256);
  bve_table_brev_kernel<double><<<nb, 256, 0, st>>>(N, logN, g.poisson, g.poisson_c64);
  SC4_LAUNCH_CHECK();
  bve_table_brev_kernel<float><<<nb, 256, 0, st>>>(N, logN, g.poisson, g.poisson_c32);
  SC4_LAUNCH_CHECK();
  bve_table_brev_kernel<double><<<nb, 256, 0, st>>>(N, logN, g.prior, g.prior_c64);
  SC4_LAUNCH_CHECK();
  bve_table_brev_kernel<float><<<nb, 256, 0, st>>>(N, logN, g.prior, g.prior_c32);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

static StencilConsts consts(const BveGeom& g) {
  double d = 2.0 * M_PI / g.N;
  StencilConsts c;
  c.c12 = 1.0 / (12.0 * d * d);
  c.nudd = g.nu / (d * d);
  c.famp = g.famp;
  c.fk_d = g.fk * d;
  return c;
}

// Launch grid of the tiled stencil kernels for k fields, and the dispatch on
// the tile width: TX = min(N, 64), or 32 for one or two fields (four times the
// blocks of a single field, so it spreads over the GPU).
template <typename T, int TX>
static dim3 sgrid(int N, int k) { return dim3(N / TX, N / TileGeom<T, TX>::TY, k); }
#define SC4_STENCIL(N, KERNEL, T, ...)                                                          \
  do {                                                                                          \
    if ((N) >= 64 && kz > 2) KERNEL<T, 64><<<sgrid<T, 64>(N, kz), kTileThreads, 0, st>>>(__VA_ARGS__); \
    else if ((N) >= 32) KERNEL<T, 32><<<sgrid<T, 32>(N, kz), kTileThreads, 0, st>>>(__VA_ARGS__); \
    else KERNEL<T, 16><<<sgrid<T, 16>(N, kz), kTileThreads, 0, st>>>(__VA_ARGS__);              \
    SC4_LAUNCH_CHECK();                                                                         \
  } while (0)

template <typename T>
static int scale_fields(size_t total, T a, const T* x, T* y, cudaStream_t st) {
  int blocks = (int)std::min<size_t>((total + 255) / 256, 8 * 152);
  scale_fields_kernel<T><<<blocks, 256, 0, st>>>(total, a, x, y);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template <typename T>
static int copy_fields(size_t total, const T* x, T* y, cudaStream_t st) {
  int blocks = (int)std::min<size_t>((total + 255) / 256, 8 * 152);
  copy_fields_kernel<T><<<blocks, 256, 0, st>>>(total, x, y);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

__global__ void bve_d2f_kernel(size_t total, const double* __restrict__ x, float* y) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x)
    y[idx] = (float)x[idx];
}

static int d2f(size_t total, const double* x, float* y, cudaStream_t st) {
  int blocks = (int)std::min<size_t>((total + 255) / 256, 8 * 152);
  bve_d2f_kernel<<<blocks, 256, 0, st>>>(total, x, y);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// Observation outputs of the FP64 state x at step t (when t is an observation step).
static int fwd_obs(const BveGeom& g, int t, const double* x, const double* y, double* d_out,
                   double* obs_out, cudaStream_t st) {
  int oi = g.obs_of_step_h[t];
  if (oi < 0 || !(d_out || obs_out)) return SC4DVAR_OK;
  bve_fwd_obs_kernel<<<div_up(g.n_o, 256), 256, 0, st>>>(g.n_o, g.obs_idx + (size_t)oi * g.n_o, x,
                                                         oi * g.n_o, y, d_out, obs_out, 1.0 / g.sigma);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// FP64 RK4 steps [t0, t1) from the state x (advanced in place; ws_fwd laid out
// as x, acc, two stage buffers, psi scratch, complex FFT buffer). Stage states
// go to row 4 (t - t0) + s of q64 / p64 / q32 / p32 (each may be null);
// observation outputs at the steps in [t0, t1); with save_ckpt, the state at
// every multiple of g.ckpt_every goes to its checkpoint slot.
static int fwd_steps(const BveGeom& g, void* ws_fwd, int t0, int t1, double* q64, double* p64,
                     float* q32, float* p32, const double* y, double* d_out, double* obs_out,
                     bool save_ckpt, cudaStream_t st) {
  const int N = g.N;
  const size_t n = (size_t)N * N;
  double* x = reinterpret_cast<double*>(ws_fwd);
  double* acc = x + n;
  double* S[2] = {acc + n, acc + 2 * n};
  double* ptmp = acc + 3 * n;
  void* cbuf = ptmp + n;
  StencilConsts sc = consts(g);
  const int kz = 1;
  for (int t = t0; t < t1; ++t) {
    SC4_TRY(fwd_obs(g, t, x, y, d_out, obs_out, st));
    if (save_ckpt && g.ckpt_every > 0 && t % g.ckpt_every == 0)
      SC4_TRY(copy_fields<double>(n, x, g.ckpt + (size_t)(t / g.ckpt_every) * n, st));
    for (int s = 0; s < 4; ++s) {
      const double* Xs = (s == 0) ? x : S[(s - 1) & 1];
      double* nxt = (s < 3) ? S[s & 1] : nullptr;
      size_t row = (size_t)(4 * (t - t0) + s) * n;
      double* ps = p64 ? p64 + row : ptmp;
      SC4_TRY(fft2_apply<double, double, double, double>(g, 1, Xs, (int)n, ps, (int)n,
                                                         (const double*)nullptr, 0, g.poisson, cbuf, st));
      if (q64) SC4_TRY(copy_fields<double>(n, Xs, q64 + row, st));
      if (q32) {
        SC4_TRY(d2f(n, Xs, q32 + row, st));
        SC4_TRY(d2f(n, ps, p32 + row, st));
      }
      SC4_STENCIL(N, bve_fwd_stage_kernel, double, N, sc, s, g.h, Xs, ps, acc, x, nxt);
    }
  }
  return SC4DVAR_OK;
}

// FWD in FP64 from x0 with the observation outputs (d = R^{-1/2}(O x - y) and/or
// O x). With `store`, keeps what the sweeps need: every stage state (FP64 and
// FP32 copies), or with checkpointing only the FP64 checkpoints. ws: bve_fwd_ws_bytes.
int bve_fwd(const BveGeom& g, const double* x0, bool store, const double* y, double* d_out,
            double* obs_out, double* xN, void* ws, cudaStream_t st) {
  const size_t n = (size_t)g.N * g.N;
  double* x = reinterpret_cast<double*>(ws);
  SC4_TRY(copy_fields<double>(n, x0, x, st));
  const bool full = store && g.ckpt_every == 0;
  SC4_TRY(fwd_steps(g, ws, 0, g.Nsteps, full ? g.q64 : nullptr, full ? g.p64 : nullptr,
                    full ? g.q32 : nullptr, full ? g.p32 : nullptr, y, d_out, obs_out,
                    store && g.ckpt_every > 0, st));
  SC4_TRY(fwd_obs(g, g.Nsteps, x, y, d_out, obs_out, st));
  if (xN) SC4_TRY(copy_fields<double>(n, x, xN, st));
  return SC4DVAR_OK;
}

// Steps [t0, t1) of checkpoint segment j and the row base of its stage states.
struct Segment {
  int t0, t1;
};
static Segment segment_of(const BveGeom& g, int j) {
  const int L = g.ckpt_every > 0 ? g.ckpt_every : g.Nsteps;
  return {j * L, std::min((j + 1) * L, g.Nsteps)};
}
static int n_segments(const BveGeom& g) {
  return g.ckpt_every > 0 ? (g.Nsteps + g.ckpt_every - 1) / g.ckpt_every : 1;
}

// FP32 RK4 steps [t0, t1) of the FWD from the FP32 state at the start of ws
// (laid out as x, acc, two stage buffers, complex FFT buffer), storing the stage
// states q_s, psi_s at row 4 (t - t0) + s of q32 / p32.
static int fwd_steps_f32(const BveGeom& g, void* ws, int t0, int t1, float* q32, float* p32,
                         cudaStream_t st) {
  const int N = g.N;
  const size_t n = (size_t)N * N;
  float* x = reinterpret_cast<float*>(ws);
  float* acc = x + n;
  float* S[2] = {acc + n, acc + 2 * n};
  void* cbuf = acc + 3 * n;
  StencilConsts sc = consts(g);
  const int kz = 1;
  for (int t = t0; t < t1; ++t) {
    for (int s = 0; s < 4; ++s) {
      const float* Xs = (s == 0) ? x : S[(s - 1) & 1];
      float* nxt = (s < 3) ? S[s & 1] : nullptr;
      const size_t row = (size_t)(4 * (t - t0) + s) * n;
      SC4_TRY(fft2_apply<float, float, float, float>(g, 1, Xs, (int)n, p32 + row, (int)n,
                                                     (const float*)nullptr, 0, g.poisson, cbuf, st));
      SC4_TRY(copy_fields<float>(n, Xs, q32 + row, st));
      SC4_STENCIL(N, bve_fwd_stage_kernel, float, N, sc, s, (float)g.h, Xs, p32 + row, acc, x, nxt);
    }
  }
  return SC4DVAR_OK;
}

// With checkpointing: recompute the stage states of segment j from its FP64
// checkpoint into the segment buffers, in the precision of the sweep that reads
// them. FP64 sweeps: the FWD's own kernels in the FWD's order, so the states
// are bit-identical to stored ones. FP32 sweeps: FP32 steps from the rounded
// checkpoint (a segment spans few steps, so the states agree with the rounded
// FP64 ones to FP32 accuracy); the TLM and the ADJ recompute the same states,
// so they stay exact transposes of each other.
template <typename T>
static int recompute_segment(const BveGeom& g, int j, cudaStream_t st) {
  if (g.ckpt_every == 0) return SC4DVAR_OK;
  const size_t n = (size_t)g.N * g.N;
  const Segment sg = segment_of(g, j);
  if constexpr (sizeof(T) == 4) {
    SC4_TRY(d2f(n, g.ckpt + (size_t)j * n, reinterpret_cast<float*>(g.rws), st));
    return fwd_steps_f32(g, g.rws, sg.t0, sg.t1, g.q32, g.p32, st);
  } else {
    SC4_TRY(copy_fields<double>(n, g.ckpt + (size_t)j * n, reinterpret_cast<double*>(g.rws), st));
    return fwd_steps(g, g.rws, sg.t0, sg.t1, g.q64, g.p64, nullptr, nullptr, nullptr, nullptr, nullptr,
                     false, st);
  }
}

template <typename T>
static const T* qbase(const BveGeom& g);
template <> const double* qbase<double>(const BveGeom& g) { return g.q64; }
template <> const float* qbase<float>(const BveGeom& g) { return g.q32; }
template <typename T>
static const T* pbase(const BveGeom& g);
template <> const double* pbase<double>(const BveGeom& g) { return g.p64; }
template <> const float* pbase<float>(const BveGeom& g) { return g.p32; }

// TLM of k directions: W = R^{-1/2} O_i dx_{t_i}; U0 = initial dx (n x k, ld ldu).
// ws: bve_sweep_ws_bytes (five n k fields of T, then the complex FFT buffer).
template <typename T>
int bve_tlm(const BveGeom& g, const T* U0, int ldu, int k, T* W, int ldw, void* ws, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  const int N = g.N;
  const size_t n = (size_t)N * N, nk = n * k;
  T* dx = reinterpret_cast<T*>(ws);
  T* acc = dx + nk;
  T* S[2] = {acc + nk, acc + 2 * nk};
  T* dpsi = acc + 3 * nk;
  void* cbuf = dpsi + nk;
  StencilConsts sc = consts(g);
  const T inv_sigma = (T)(1.0 / g.sigma);
  for (int c = 0; c < k; ++c)
    SC4_CUDA(cudaMemcpyAsync(dx + (size_t)c * n, U0 + (size_t)c * ldu, n * sizeof(T),
                             cudaMemcpyDeviceToDevice, st));
  const int kz = k;
  auto gather = [&](int t) -> int {
    int oi = g.obs_of_step_h[t];
    if (oi >= 0) {
      bve_gather_kernel<T><<<dim3(div_up(g.n_o, 256), k), 256, 0, st>>>(
          g.n_o, g.obs_idx + (size_t)oi * g.n_o, dx, n, W, ldw, oi * g.n_o, inv_sigma);
      SC4_LAUNCH_CHECK();
    }
    return SC4DVAR_OK;
  };
  for (int j = 0; j < n_segments(g); ++j) {
    const Segment sg = segment_of(g, j);
    SC4_TRY(recompute_segment<T>(g, j, st));
    const int base = g.ckpt_every > 0 ? sg.t0 : 0;
    for (int t = sg.t0; t < sg.t1; ++t) {
      SC4_TRY(gather(t));
      for (int s = 0; s < 4; ++s) {
        const T* cur = (s == 0) ? dx : S[(s - 1) & 1];
        T* nxt = (s < 3) ? S[s & 1] : nullptr;
        size_t row = (size_t)(4 * (t - base) + s) * n;
        SC4_TRY(fft2_apply<T, T, T, T>(g, k, cur, (int)n, dpsi, (int)n, (const T*)nullptr, 0, g.poisson,
                                       cbuf, st));
        if (sizeof(T) == 4 && N >= 64 && k > 2) {
          const size_t smd = (size_t)kD2TlmTiles * TileGeom<float, 64>::SIZE * sizeof(float);
          SC4_CUDA(cudaFuncSetAttribute(bve_tlm_stage_d2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smd));
          bve_tlm_stage_d2_kernel<<<sgrid<float, 64>(N, (k + 1) / 2), kTileThreads, smd, st>>>(
              N, sc, s, (float)g.h, (const float*)(qbase<T>(g) + row), (const float*)(pbase<T>(g) + row),
              (const float*)cur, (const float*)dpsi, (float*)acc, (float*)dx, (float*)nxt, n, k);
          SC4_LAUNCH_CHECK();
        } else {
          SC4_STENCIL(N, bve_tlm_stage_kernel, T, N, sc, s, (T)g.h, qbase<T>(g) + row, pbase<T>(g) + row,
                      cur, dpsi, acc, dx, nxt, n);
        }
      }
    }
  }
  return gather(g.Nsteps);
}

// ADJ of k directions: Out = lam_0 forced by W. ws as for bve_tlm.
template <typename T>
int bve_adj(const BveGeom& g, const T* W, int ldw, int k, T* Out, int ldo, void* ws, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  const int N = g.N;
  const size_t n = (size_t)N * N, nk = n * k;
  T* lam = reinterpret_cast<T*>(ws);
  T* th = lam + nk;
  T* K[2] = {th + nk, th + 2 * nk};
  T* t12 = th + 3 * nk;
  void* cbuf = t12 + nk;
  StencilConsts sc = consts(g);
  const T inv_sigma = (T)(1.0 / g.sigma);
  SC4_CUDA(cudaMemsetAsync(lam, 0, nk * sizeof(T), st));
  const int kz = k;
  const T h = (T)g.h;
  for (int j = n_segments(g) - 1; j >= 0; --j) {
    const Segment sg = segment_of(g, j);
    SC4_TRY(recompute_segment<T>(g, j, st));
    const int base = g.ckpt_every > 0 ? sg.t0 : 0;
    for (int t = sg.t1; t > sg.t0; --t) {
      int oi = g.obs_of_step_h[t];
      if (oi >= 0) {
        bve_scatter_kernel<T><<<dim3(div_up(g.n_o, 256), k), 256, 0, st>>>(
            g.n_o, g.obs_idx + (size_t)oi * g.n_o, W, ldw, oi * g.n_o, lam, n, inv_sigma);
        SC4_LAUNCH_CHECK();
      }
      SC4_TRY(scale_fields<T>(nk, h * (T)(1.0 / 6.0), lam, K[0], st));  // kappa_4 = h b_4 lam
      for (int s = 3; s >= 0; --s) {
        const T* kap = K[(3 - s) & 1];
        T* knext = K[(4 - s) & 1];
        size_t row = (size_t)(4 * (t - 1 - base) + s) * n;
        if (sizeof(T) == 4 && N >= 64 && k > 2) {
          bve_adj_jac_d2_kernel<<<sgrid<float, 64>(N, (k + 1) / 2), kTileThreads, 0, st>>>(
              N, sc, (const float*)(qbase<T>(g) + row), (const float*)kap, (float*)t12, n, k);
          SC4_LAUNCH_CHECK();
        } else {
          SC4_STENCIL(N, bve_adj_jac_kernel, T, N, sc, qbase<T>(g) + row, kap, t12, n);
        }
        SC4_TRY(fft2_apply<T, T, T, T>(g, k, t12, (int)n, t12, (int)n, (const T*)nullptr, 0, g.poisson,
                                       cbuf, st));
        SC4_STENCIL(N, bve_adj_stage_kernel, T, N, sc, s, h, pbase<T>(g) + row, kap, t12, th, lam,
                    s > 0 ? knext : nullptr, n);
      }
    }
  }
  for (int c = 0; c < k; ++c)
    SC4_CUDA(cudaMemcpyAsync(Out + (size_t)c * ldo, lam + (size_t)c * n, n * sizeof(T),
                             cudaMemcpyDeviceToDevice, st));
  return SC4DVAR_OK;
}

// Workspace of bve_tlm / bve_adj: five n x k fields of T (TLM: dx, acc, two
// stage buffers, dpsi; ADJ: lam, th, two kappa buffers, T1/T2) followed by the
// complex FFT buffer of ceil(k/2) n complex values.
size_t bve_sweep_ws_bytes(const BveGeom& g, int k, size_t tb) {
  size_t n = (size_t)g.N * g.N;
  return 5 * n * k * tb + (size_t)((k + 1) / 2) * n * 2 * tb + 256;
}

size_t bve_fwd_ws_bytes(const BveGeom& g) {
  size_t n = (size_t)g.N * g.N;
  return 5 * n * sizeof(double) + n * sizeof(double2) + 256;
}

template int fft2_apply<double, double, double, double>(const BveGeom&, int, const double*, int, double*,
                                                        int, const double*, int, const double*, void*,
                                                        cudaStream_t);
template int fft2_apply<float, float, float, float>(const BveGeom&, int, const float*, int, float*, int,
                                                    const float*, int, const double*, void*,
                                                    cudaStream_t);
template int fft2_apply<double, double, float, float>(const BveGeom&, int, const double*, int, float*,
                                                      int, const float*, int, const double*, void*,
                                                      cudaStream_t);
template int fft2_apply<double, float, double, double>(const BveGeom&, int, const float*, int, double*,
                                                       int, const double*, int, const double*, void*,
                                                       cudaStream_t);
template int bve_tlm<double>(const BveGeom&, const double*, int, int, double*, int, void*, cudaStream_t);
template int bve_tlm<float>(const BveGeom&, const float*, int, int, float*, int, void*, cudaStream_t);
template int bve_adj<double>(const BveGeom&, const double*, int, int, double*, int, void*, cudaStream_t);
template int bve_adj<float>(const BveGeom&, const float*, int, int, float*, int, void*, cudaStream_t);

}  // namespace sc4
