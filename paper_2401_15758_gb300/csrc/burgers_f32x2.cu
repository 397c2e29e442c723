// FP32 Burgers TLM / ADJ sweeps in packed FP32x2 arithmetic (n >= 1024).
//
// Same discretization, TLM and discrete RK4 adjoint as burgers_impl.cuh. The
// periodic ring of n points is folded into H = n/2 pairs (x_i, x_{i+H}): pair
// i's neighbours are pairs i-1 and i+1, except at the ring ends where the left
// neighbour of pair 0 is (x_{n-1}, x_{H-1}) = swap(pair H-1) and the right
// neighbour of pair H-1 is (x_H, x_0) = swap(pair 0). Every stencil operation
// then acts on two points at once with the packed FP32 instructions of sm_100+
// (__ffma2_rn / __fadd2_rn / __fmul2_rn), halving the arithmetic instructions
// of the sweeps, which are issue-bound. The FP32 trajectory copy is stored
// folded (row t: x_0, x_H, x_1, x_{H+1}, ...) so a thread's pairs load as
// 16-byte vectors.
//
// Thread t of a CTA owns P contiguous pairs; halos travel by warp shuffles,
// per-warp edge slots and, in a cluster, DSMEM, as in the scalar kernels.
#include <cooperative_groups.h>
#include <algorithm>
#include <cstdlib>
#include "common.cuh"
#include "cluster.cuh"
#include "model.cuh"

namespace cg = cooperative_groups;

namespace sc4 {
namespace {

using f2 = float2;

__device__ __forceinline__ f2 mk(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 swp(f2 a) { return make_float2(a.y, a.x); }

__device__ __forceinline__ f2 shfl_up2(f2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ f2 shfl_dn2(f2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

constexpr int kPad2 = 2;  // pair arrays: pair j at index j + kPad2 (16-byte aligned)

template <bool CL>
__device__ __forceinline__ void bar2() {
  if constexpr (CL) cg::this_cluster().sync();
  else __syncthreads();
}

struct Geo {
  int n, H, Hs, N, n_o;  // points, pairs, pairs per CTA, steps, obs sites per time
  float h, c1, c2, inv_sigma;
  const int* obs_of_step;
  const int* obs_idx;
};

__constant__ float kA2[3] = {0.5f, 0.5f, 1.0f};
__constant__ float kB2[4] = {1.0f / 6.0f, 1.0f / 3.0f, 1.0f / 3.0f, 1.0f / 6.0f};

// Chunk-major pair rows: chunk q (2 pairs) of thread t at chunk slot q*NT + t.
template <int P>
struct PRows {
  static_assert(P % 2 == 0 || P == 1, "pairs per thread");
  __device__ static __forceinline__ int elem(int t, int p, int NT) {
    if constexpr (P % 2 == 0) return ((p >> 1) * NT + t) * 2 + (p & 1);
    else return t;
  }
  __device__ static __forceinline__ void load(const f2* base, int t, int NT, f2 (&v)[P]) {
    if constexpr (P % 2 == 0) {
      const float4* b4 = reinterpret_cast<const float4*>(base);
#pragma unroll
      for (int q = 0; q < P / 2; ++q) {
        float4 c = b4[q * NT + t];
        v[2 * q] = make_float2(c.x, c.y);
        v[2 * q + 1] = make_float2(c.z, c.w);
      }
    } else {
      v[0] = base[t];
    }
  }
  __device__ static __forceinline__ void store(f2* base, int t, int NT, const f2 (&v)[P]) {
    if constexpr (P % 2 == 0) {
      float4* b4 = reinterpret_cast<float4*>(base);
#pragma unroll
      for (int q = 0; q < P / 2; ++q)
        b4[q * NT + t] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
    } else {
      base[t] = v[0];
    }
  }
  // asynchronous copy of my P pairs of a folded global row into a chunk-major buffer
  __device__ static __forceinline__ void prefetch(f2* base, const f2* __restrict__ src, int t, int NT) {
    if constexpr (P % 2 == 0) {
#pragma unroll
      for (int q = 0; q < P / 2; ++q) {
        unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<float4*>(base) + q * NT + t);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + 2 * q));
      }
      asm volatile("cp.async.commit_group;\n" ::);
    } else {
      base[t] = __ldg(src);
    }
  }
  __device__ static __forceinline__ void wait() {
    if constexpr (P % 2 == 0) asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
};

// Edge exchange of a pair vector: slot arrays L (first pair of each warp) and R
// (last pair); the reading lanes apply the ring-end swap.
struct EdgeNb2 {
  const f2* lbase;
  const f2* rbase;
  int lw, rw;
  bool swapL, swapR;
};

template <bool CL>
__device__ __forceinline__ EdgeNb2 edge_nb2(f2* slots, int w, int nw, int crank, int csize) {
  EdgeNb2 nb;
  nb.lbase = slots;
  nb.rbase = slots;
  nb.lw = (w > 0) ? w - 1 : nw - 1;
  nb.rw = (w < nw - 1) ? w + 1 : 0;
  nb.swapL = (crank == 0 && w == 0);
  nb.swapR = (crank == csize - 1 && w == nw - 1);
  if constexpr (CL) {
    if (w == 0) nb.lbase = cg::this_cluster().map_shared_rank(slots, (crank + csize - 1) % csize);
    if (w == nw - 1) nb.rbase = cg::this_cluster().map_shared_rank(slots, (crank + 1) % csize);
  }
  return nb;
}

__device__ __forceinline__ void edge_put2(f2* L, f2* R, int lane, int w, f2 first, f2 last) {
  if (lane == 0) L[w] = first;
  if (lane == 31) R[w] = last;
}

__device__ __forceinline__ void edge_get2(const EdgeNb2& nb, int offL, int offR, int lane, f2& left,
                                          f2& right) {
  if (lane == 0) {
    f2 v = nb.lbase[offR + nb.lw];
    left = nb.swapL ? swp(v) : v;
  }
  if (lane == 31) {
    f2 v = nb.rbase[offL + nb.rw];
    right = nb.swapR ? swp(v) : v;
  }
}

// Pair neighbours of my row in a shared pair array (warp-edge lanes read it).
template <int P>
struct RowNb2 {
  int lofs, rofs;
  bool swapL, swapR;
  __device__ RowNb2(int tid, int NT, int Hs, int crank, int csize) {
    lofs = (tid == 0) ? kPad2 - 1 : kPad2 + PRows<P>::elem(tid - 1, P - 1, NT);
    rofs = (tid == NT - 1) ? kPad2 + Hs : kPad2 + PRows<P>::elem(tid + 1, 0, NT);
    swapL = (tid == 0 && crank == 0);
    swapR = (tid == NT - 1 && crank == csize - 1);
  }
};

template <int P>
__device__ __forceinline__ void row_halos2(const f2* arr, const f2 (&v)[P], const RowNb2<P>& nb, int lane,
                                           f2& left, f2& right) {
  left = shfl_up2(v[P - 1]);
  right = shfl_dn2(v[0]);
  if (lane == 0) {
    f2 a = arr[nb.lofs];
    left = nb.swapL ? swp(a) : a;
  }
  if (lane == 31) {
    f2 a = arr[nb.rofs];
    right = nb.swapR ? swp(a) : a;
  }
}

template <bool CL, int P>
__device__ __forceinline__ void row_store2(f2* arr, int tid, int NT, int Hs, const f2 (&v)[P], int crank,
                                           int csize) {
  PRows<P>::store(arr + kPad2, tid, NT, v);
  if (tid == 0) {
    if constexpr (CL) cg::this_cluster().map_shared_rank(arr, (crank + csize - 1) % csize)[kPad2 + Hs] = v[0];
    else arr[kPad2 + Hs] = v[0];
  }
  if (tid == NT - 1) {
    if constexpr (CL) cg::this_cluster().map_shared_rank(arr, (crank + 1) % csize)[kPad2 - 1] = v[P - 1];
    else arr[kPad2 - 1] = v[P - 1];
  }
}

// Shared pair index and component of global point j, for the CTA owning it.
__device__ __forceinline__ bool pair_of(int j, const Geo& g, int crank, int& il, int& half) {
  int i = j < g.H ? j : j - g.H;
  half = j < g.H ? 0 : 1;
  il = i - crank * g.Hs;
  return il >= 0 && il < g.Hs;
}

template <int P>
struct Bounds2 {
  static constexpr int kThreads = P >= 8 ? 512 : 1024;
};

// ---------------------------------------------------------------- TLM
template <int P, bool CL>
__global__ void __launch_bounds__(Bounds2<P>::kThreads, 1) tlm_f32x2_kernel(
    Geo g, const float* __restrict__ traj, const float* __restrict__ U0, int ldu,
    float* __restrict__ W, int ldw) {
  using R = PRows<P>;
  extern __shared__ __align__(16) unsigned char smraw[];
  f2* sm = reinterpret_cast<f2*>(smraw);
  const int Hs = g.Hs, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  f2* xbuf[2] = {sm, sm + Hs};
  f2* stage = sm + 2 * Hs;             // Hs + 2 kPad2
  f2* slots = stage + Hs + 2 * kPad2;  // [parity 2][array 2][L/R 2][32]
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const EdgeNb2 enb = edge_nb2<CL>(slots, w, nw, crank, csize);
  const int col = blockIdx.x / csize;
  const int i0 = crank * Hs + tid * P;  // first pair of mine
  const f2* trajp = reinterpret_cast<const f2*>(traj);
  f2 x[P], dx[P], acc[P], U[P], D[P];
  {
    const float* u0 = U0 + (size_t)col * ldu;
#pragma unroll
    for (int p = 0; p < P; ++p) dx[p] = make_float2(u0[i0 + p], u0[g.H + i0 + p]);
  }
  float* wcol = W + (size_t)col * ldw;
  const f2 h2 = mk(g.h), c1n = mk(-g.c1), c2 = mk(g.c2), m1 = mk(-1.f), m2 = mk(-2.f);
  if (g.N > 0) R::prefetch(xbuf[0], trajp + i0, tid, NT);
  for (int t = 0;; ++t) {
    int oi = g.obs_of_step[t];
    if (oi >= 0) {
      R::store(stage + kPad2, tid, NT, dx);
      bar2<CL>();
      for (int o = tid; o < g.n_o; o += NT) {
        int il, half;
        if (pair_of(g.obs_idx[oi * g.n_o + o], g, crank, il, half)) {
          f2 v = stage[kPad2 + R::elem(il / P, il % P, NT)];
          wcol[oi * g.n_o + o] = (half ? v.y : v.x) * g.inv_sigma;
        }
      }
    }
    if (t == g.N) break;
    R::wait();
    R::load(xbuf[t & 1], tid, NT, x);
    if (t + 1 < g.N) R::prefetch(xbuf[(t + 1) & 1], trajp + (size_t)(t + 1) * g.H + i0, tid, NT);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      U[p] = x[p];
      D[p] = dx[p];
      acc[p] = mk(0.f);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int q = s & 1;
      f2* su = slots + ((q * 2 + 0) * 2) * 32;
      f2* sd = slots + ((q * 2 + 1) * 2) * 32;
      edge_put2(su, su + 32, lane, w, U[0], U[P - 1]);
      edge_put2(sd, sd + 32, lane, w, D[0], D[P - 1]);
      f2 uL = shfl_up2(U[P - 1]), uR = shfl_dn2(U[0]);
      f2 dL = shfl_up2(D[P - 1]), dR = shfl_dn2(D[0]);
      bar2<CL>();
      edge_get2(enb, (int)(su - slots), (int)(su - slots) + 32, lane, uL, uR);
      edge_get2(enb, (int)(sd - slots), (int)(sd - slots) + 32, lane, dL, dR);
      const f2 bs = mk(kB2[s]);
      const f2 ha = mk(s < 3 ? g.h * kA2[s] : 0.f);
      f2 up = uL, dp = dL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        f2 u = U[p], d = D[p];
        f2 un = (p + 1 < P) ? U[p + 1] : uR;
        f2 dn = (p + 1 < P) ? D[p + 1] : dR;
        f2 nd1u = mul2(fma2(up, m1, un), c1n);               // -(D1 u)
        f2 dk = mul2(c2, fma2(d, m2, add2(dn, dp)));          // nu D2 d
        dk = fma2(u, mul2(fma2(dp, m1, dn), c1n), dk);        // - u D1 d
        dk = fma2(nd1u, d, dk);                               // - (D1 u) d
        acc[p] = fma2(bs, dk, acc[p]);
        if (s < 3) {
          f2 k = mul2(c2, fma2(u, m2, add2(un, up)));         // nu D2 u
          k = fma2(u, nd1u, k);                               // - u D1 u
          U[p] = fma2(ha, k, x[p]);
          D[p] = fma2(ha, dk, dx[p]);
        }
        up = u;
        dp = d;
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) dx[p] = fma2(h2, acc[p], dx[p]);
  }
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

// ---------------------------------------------------------------- ADJ
template <int P, bool CL>
__global__ void __launch_bounds__(Bounds2<P>::kThreads, 1) adj_f32x2_kernel(
    Geo g, const float* __restrict__ traj, const float* __restrict__ Win, int ldw,
    float* __restrict__ Out, int ldo) {
  using R = PRows<P>;
  extern __shared__ __align__(16) unsigned char smraw[];
  f2* sm = reinterpret_cast<f2*>(smraw);
  const int Hs = g.Hs, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  const int S = Hs + 2 * kPad2;
  f2* buf[4] = {sm, sm + S, sm + 2 * S, sm + 3 * S};
  f2* slots = sm + 4 * S;  // [parity 2][L/R 2][32]
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const EdgeNb2 enb = edge_nb2<CL>(slots, w, nw, crank, csize);
  const RowNb2<P> rnb(tid, NT, Hs, crank, csize);
  const int col = blockIdx.x / csize;
  const int i0 = crank * Hs + tid * P;
  const f2* trajp = reinterpret_cast<const f2*>(traj);
  const float* win = Win + (size_t)col * ldw;
  const f2 c1n = mk(-g.c1), c1 = mk(g.c1), c2 = mk(g.c2), m1 = mk(-1.f), m2 = mk(-2.f);
  f2 lam[P], x[P], th[P], K[P], u[P];
#pragma unroll
  for (int p = 0; p < P; ++p) lam[p] = mk(0.f);
  R::prefetch(buf[0] + kPad2, trajp + (size_t)(g.N - 1) * g.H + i0, tid, NT);
  for (int t = g.N, c = 0; t >= 1; --t, ++c) {
    const int r = c & 3;
    f2* B0 = buf[(4 - r) & 3];
    f2* B1 = buf[(5 - r) & 3];
    f2* B2 = buf[(6 - r) & 3];
    f2* B3 = buf[(7 - r) & 3];
    int oi = g.obs_of_step[t];
    if (oi >= 0) {
      bar2<CL>();
      R::store(B1 + kPad2, tid, NT, lam);
      __syncthreads();
      for (int o = tid; o < g.n_o; o += NT) {
        int il, half;
        if (pair_of(g.obs_idx[oi * g.n_o + o], g, crank, il, half)) {
          f2* cell = &B1[kPad2 + R::elem(il / P, il % P, NT)];
          atomicAdd(half ? &cell->y : &cell->x, win[oi * g.n_o + o] * g.inv_sigma);
        }
      }
      __syncthreads();
      R::load(B1 + kPad2, tid, NT, lam);
    }
    R::wait();
    R::load(B0 + kPad2, tid, NT, x);
    if (tid == 0) {
      if constexpr (CL) cg::this_cluster().map_shared_rank(B0, (crank + csize - 1) % csize)[kPad2 + Hs] = x[0];
      else B0[kPad2 + Hs] = x[0];
    }
    if (tid == NT - 1) {
      if constexpr (CL) cg::this_cluster().map_shared_rank(B0, (crank + 1) % csize)[kPad2 - 1] = x[P - 1];
      else B0[kPad2 - 1] = x[P - 1];
    }
    bar2<CL>();                                                   // 1
#pragma unroll
    for (int p = 0; p < P; ++p) u[p] = x[p];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const f2* Bs = (s == 0) ? B0 : (s == 1 ? B1 : B2);
      f2* Bn = (s == 0) ? B1 : (s == 1 ? B2 : B3);
      f2 uL, uR;
      row_halos2<P>(Bs, u, rnb, lane, uL, uR);
      const f2 ha = mk(g.h * kA2[s]);
      f2 up = uL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        f2 uc = u[p];
        f2 un = (p + 1 < P) ? u[p + 1] : uR;
        f2 nd1u = mul2(fma2(up, m1, un), c1n);
        f2 k = mul2(c2, fma2(uc, m2, add2(un, up)));
        k = fma2(uc, nd1u, k);
        u[p] = fma2(ha, k, x[p]);
        up = uc;
      }
      row_store2<CL, P>(Bn, tid, NT, Hs, u, crank, csize);
      if (s == 2) {
        const f2 hb = mk(g.h * kB2[3]);
#pragma unroll
        for (int p = 0; p < P; ++p) K[p] = mul2(hb, lam[p]);
        edge_put2(slots, slots + 32, lane, w, K[0], K[P - 1]);
      }
      bar2<CL>();                                                 // 2, 3, 4
    }
#pragma unroll
    for (int p = 0; p < P; ++p) th[p] = mk(0.f);
#pragma unroll
    for (int s = 3; s >= 0; --s) {
      const f2* Bs = (s == 3) ? B3 : (s == 2 ? B2 : (s == 1 ? B1 : B0));
      if (s == 2 || s == 1) R::load(Bs + kPad2, tid, NT, u);
      if (s == 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = x[p];
      }
      const int qin = ((3 - s) & 1) * 64;
      f2 kL = shfl_up2(K[P - 1]), kR = shfl_dn2(K[0]);
      edge_get2(enb, qin, qin + 32, lane, kL, kR);
      f2 uL, uR;
      row_halos2<P>(Bs, u, rnb, lane, uL, uR);
      const f2 hb = mk(s > 0 ? g.h * kB2[s - 1] : 0.f);
      const f2 ha = mk(s > 0 ? g.h * kA2[s - 1] : 0.f);
      f2 up = uL, kp = kL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        f2 uc = u[p], kc = K[p];
        f2 un = (p + 1 < P) ? u[p + 1] : uR;
        f2 kn = (p + 1 < P) ? K[p + 1] : kR;
        f2 nd1u = mul2(fma2(up, m1, un), c1n);               // -(D1 u)
        f2 theta = mul2(c2, fma2(kc, m2, add2(kn, kp)));      // nu D2 kappa
        f2 flux = fma2(up, mul2(kp, m1), mul2(un, kn));       // u_{+} k_{+} - u_{-} k_{-}
        theta = fma2(flux, c1, theta);                        // + D1 (u kappa)
        theta = fma2(nd1u, kc, theta);                        // - (D1 u) kappa
        th[p] = add2(th[p], theta);
        if (s > 0) K[p] = fma2(ha, theta, mul2(hb, lam[p]));
        up = uc;
        kp = kc;
      }
      if (s > 0) {
        f2* so = slots + ((4 - s) & 1) * 64;
        edge_put2(so, so + 32, lane, w, K[0], K[P - 1]);
        bar2<CL>();                                               // 5, 6, 7
        if (s == 3 && t > 1) R::prefetch(B3 + kPad2, trajp + (size_t)(t - 2) * g.H + i0, tid, NT);
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) lam[p] = add2(lam[p], th[p]);
  }
  float* out = Out + (size_t)col * ldo;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    out[i0 + p] = lam[p].x;
    out[g.H + i0 + p] = lam[p].y;
  }
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

// ---------------------------------------------------------------- one-CTA sweeps, factored stencils
//
// With P_j = c2 + c1 u_j and M_j = c2 - c1 u_j (c1 = 1/(2 dx), c2 = nu/dx^2) the
// semi-discrete Burgers right-hand side, its Jacobian F = f'(u) and F^T are
//   f_j       = M_j (u_{j+1} - u_j) - P_j (u_j - u_{j-1})
//   (F d)_j   = M_j (d_{j+1} - d_j) - P_j (d_j - d_{j-1}) - (P_{j+1} - P_{j-1}) d_j
//   (F^T k)_j = P_{j+1} (k_{j+1} - k_j) - M_{j-1} (k_j - k_{j-1})
// (from F_{j,j+1} = M_j, F_{j,j-1} = P_j, F_{jj} = -(P_{j+1} + M_{j-1})). The
// kernels below evaluate these factored forms, with nM = -M = c1 u - c2 so that
// every operation is one packed FMA or multiply: per point and RK4 step about 51
// packed operations for the TLM and 47 for the ADJ (its base-state
// recomputation included), against 61 and 74 for the expanded stencils.
//
// One CTA sweeps one direction over the whole window; thread t owns P contiguous
// folded pairs. In every stage a thread first computes its interior pairs, whose
// neighbours it holds, then its first and last pair with the halos loaded after
// the previous barrier, and stores those two results in the exchange rows (one
// entry per thread, so stores and loads are unconditional and conflict-free)
// before the barrier.

// Exchange rows: [parity 2][array 2][NT] first pairs, then the same for last pairs.
struct Xch {
  f2* first;
  f2* last;
  int NT, tid, tl, tr;
  bool swl, swr;
  __device__ __forceinline__ void put(int par, int a, f2 f, f2 l) const {
    first[(par * 2 + a) * NT + tid] = f;
    last[(par * 2 + a) * NT + tid] = l;
  }
  // left neighbour of my first pair, right neighbour of my last pair (ring ends swapped)
  __device__ __forceinline__ void get(int par, int a, f2& left, f2& right) const {
    const f2 l = last[(par * 2 + a) * NT + tl], r = first[(par * 2 + a) * NT + tr];
    left = swl ? swp(l) : l;
    right = swr ? swp(r) : r;
  }
};

// Neighbour pairs of my first and last pair in a chunk-major row (ring wrap and swap).
template <int P>
struct RowHalo {
  int el, er;
  bool swl, swr;
  __device__ RowHalo(int tid, int NT) {
    el = PRows<P>::elem(tid > 0 ? tid - 1 : NT - 1, P - 1, NT);
    er = PRows<P>::elem(tid < NT - 1 ? tid + 1 : 0, 0, NT);
    swl = tid == 0;
    swr = tid == NT - 1;
  }
  __device__ __forceinline__ void get(const f2* row, f2& left, f2& right) const {
    const f2 a = row[el], b = row[er];
    left = swl ? swp(a) : a;
    right = swr ? swp(b) : b;
  }
};

template <int P>
struct Bounds1 {
  static constexpr int kThreads = P >= 16 ? 256 : 512;
};

template <int P>
__global__ void __launch_bounds__(Bounds1<P>::kThreads, 1) tlm1_kernel(
    Geo g, const float* __restrict__ traj, const float* __restrict__ U0, int ldu,
    float* __restrict__ W, int ldw) {
  static_assert(P >= 4 && P % 2 == 0, "pairs per thread");
  using R = PRows<P>;
  extern __shared__ __align__(16) unsigned char smraw[];
  f2* sm = reinterpret_cast<f2*>(smraw);
  const int H = g.H, NT = blockDim.x, tid = threadIdx.x;
  f2* stage = sm + 2 * H;  // rows t (even / odd) at sm and sm + H
  f2* carry = stage + H;   // low-order part of the state (my chunks)
  Xch X;
  X.first = carry + H;
  X.last = X.first + 4 * NT;
  X.NT = NT;
  X.tid = tid;
  X.tl = tid > 0 ? tid - 1 : NT - 1;
  X.tr = tid < NT - 1 ? tid + 1 : 0;
  X.swl = tid == 0;
  X.swr = tid == NT - 1;
  const RowHalo<P> rh(tid, NT);
  const int col = blockIdx.x;
  const int i0 = tid * P;
  const f2* trajp = reinterpret_cast<const f2*>(traj);
  const f2 c1 = mk(g.c1), c2 = mk(g.c2), nc2 = mk(-g.c2), m1 = mk(-1.f), mh = mk(-g.h);
  constexpr float kA[3] = {0.5f, 0.5f, 1.0f};
  constexpr float kB[4] = {1.0f / 6.0f, 1.0f / 3.0f, 1.0f / 3.0f, 1.0f / 6.0f};
  f2 dx[P], acc[P], dL, dR;
  {
    const float* u0 = U0 + (size_t)col * ldu;
#pragma unroll
    for (int p = 0; p < P; ++p) dx[p] = make_float2(u0[i0 + p], u0[H + i0 + p]);
    const int il = X.swl ? H - 1 : i0 - 1, ir = X.swr ? 0 : i0 + P;
    const f2 a = make_float2(u0[il], u0[H + il]), b = make_float2(u0[ir], u0[H + ir]);
    dL = X.swl ? swp(a) : a;
    dR = X.swr ? swp(b) : b;
  }
  float* wcol = W + (size_t)col * ldw;
  {
    f2 z[P];
#pragma unroll
    for (int p = 0; p < P; ++p) z[p] = mk(0.f);
    R::store(carry, tid, NT, z);
  }
  if (g.N > 0) {
    R::prefetch(sm, trajp + i0, tid, NT);
    R::wait();
  }
  __syncthreads();
  int oi_next = g.obs_of_step[0];
  for (int t = 0;; ++t) {
    const int oi = oi_next;
    if (t < g.N) oi_next = g.obs_of_step[t + 1];
    if (oi >= 0) {
      R::store(stage, tid, NT, dx);
      __syncthreads();
      for (int o = tid; o < g.n_o; o += NT) {
        int il, half;
        if (pair_of(g.obs_idx[oi * g.n_o + o], g, 0, il, half)) {
          const f2 v = stage[R::elem(il / P, il % P, NT)];
          wcol[oi * g.n_o + o] = (half ? v.y : v.x) * g.inv_sigma;
        }
      }
    }
    if (t == g.N) break;
    const f2* xb = sm + (t & 1) * H;
    f2 x[P], U[P], D[P], uL, uR;
    R::load(xb, tid, NT, x);
    rh.get(xb, uL, uR);
    if (t + 1 < g.N) R::prefetch(sm + ((t + 1) & 1) * H, trajp + (size_t)(t + 1) * H + i0, tid, NT);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      U[p] = x[p];
      D[p] = dx[p];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const f2 bs = mk(kB[s]);
      const f2 mha = mk(s < 3 ? -g.h * kA[s] : 0.f);
      f2 Un[P], Dn[P], cy[P];
      if (s == 3) R::load(carry, tid, NT, cy);
      // pair p from P at p-1, p, p+1 and the forward differences at p (q = p) and p + 1
      auto pair = [&](int p, f2 Pm, f2 Pc, f2 Pn, f2 du0, f2 du1, f2 dd0, f2 dd1) {
        const f2 nM = fma2(c1, U[p], nc2);
        const f2 E = fma2(Pm, m1, Pn);
        const f2 G = fma2(E, D[p], fma2(Pc, dd0, mul2(nM, dd1)));  // -(F D)_p
        acc[p] = (s == 0) ? mul2(bs, G) : fma2(bs, G, acc[p]);
        if (s < 3) {
          const f2 gu = fma2(Pc, du0, mul2(nM, du1));               // -f(U)_p
          Un[p] = fma2(mha, gu, x[p]);
          Dn[p] = fma2(mha, G, dx[p]);
        } else {
          // dx += -h acc with the rounding error of the sum carried to the next
          // step (Fast2Sum, |dx| >= |increment|): the FP32 state then drifts by
          // far less than u per step over windows of 10^4 steps
          const f2 inc = fma2(mh, acc[p], cy[p]);
          const f2 sum = add2(dx[p], inc);
          cy[p] = add2(fma2(sum, m1, dx[p]), inc);
          dx[p] = sum;
        }
      };
      // interior pairs 1 .. P-2, streaming a window of P and differences
      const f2 P0 = fma2(c1, U[0], c2), P1 = fma2(c1, U[1], c2);
      const f2 du1 = fma2(U[0], m1, U[1]), dd1 = fma2(D[0], m1, D[1]);
      f2 Pm = P0, Pc = P1, dum = du1, ddm = dd1;
#pragma unroll
      for (int p = 1; p < P - 1; ++p) {
        const f2 Pn = fma2(c1, U[p + 1], c2);
        const f2 dun = fma2(U[p], m1, U[p + 1]), ddn = fma2(D[p], m1, D[p + 1]);
        pair(p, Pm, Pc, Pn, dum, dun, ddm, ddn);
        Pm = Pc;
        Pc = Pn;
        dum = dun;
        ddm = ddn;
      }
      // last and first pair with the halos
      pair(P - 1, Pm, Pc, fma2(c1, uR, c2), dum, fma2(U[P - 1], m1, uR), ddm, fma2(D[P - 1], m1, dR));
      pair(0, fma2(c1, uL, c2), P0, P1, fma2(uL, m1, U[0]), du1, fma2(dL, m1, D[0]), dd1);
      const int par = s & 1;
      if (s < 3) {
        X.put(par, 0, Un[0], Un[P - 1]);
        X.put(par, 1, Dn[0], Dn[P - 1]);
      } else {
        X.put(par, 1, dx[0], dx[P - 1]);
        R::store(carry, tid, NT, cy);
        R::wait();
      }
      __syncthreads();
      if (s < 3) {
        X.get(par, 0, uL, uR);
        X.get(par, 1, dL, dR);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          U[p] = Un[p];
          D[p] = Dn[p];
        }
      } else {
        X.get(par, 1, dL, dR);
      }
    }
  }
}

template <int P>
__global__ void __launch_bounds__(Bounds1<P>::kThreads, 1) adj1_kernel(
    Geo g, const float* __restrict__ traj, const float* __restrict__ Win, int ldw,
    float* __restrict__ Out, int ldo) {
  static_assert(P >= 4 && P % 2 == 0, "pairs per thread");
  using R = PRows<P>;
  extern __shared__ __align__(16) unsigned char smraw[];
  f2* sm = reinterpret_cast<f2*>(smraw);
  const int H = g.H, NT = blockDim.x, tid = threadIdx.x;
  // rows x_r (even / odd r) at sm and sm + H; stage states 1, 2 of the step at
  // ubuf[0], ubuf[1] (ubuf[0] also stages lambda for the observation forcing);
  // the low-order part of lambda's sums (my chunks)
  f2* ubuf[2] = {sm + 2 * H, sm + 3 * H};
  f2* lam_c = sm + 4 * H;
  Xch X;
  X.first = sm + 5 * H;
  X.last = X.first + 4 * NT;
  X.NT = NT;
  X.tid = tid;
  X.tl = tid > 0 ? tid - 1 : NT - 1;
  X.tr = tid < NT - 1 ? tid + 1 : 0;
  X.swl = tid == 0;
  X.swr = tid == NT - 1;
  const RowHalo<P> rh(tid, NT);
  const int col = blockIdx.x;
  const int i0 = tid * P;
  const f2* trajp = reinterpret_cast<const f2*>(traj);
  const float* win = Win + (size_t)col * ldw;
  const f2 c1 = mk(g.c1), c2 = mk(g.c2), nc2 = mk(-g.c2), m1 = mk(-1.f);
  const f2 h3 = mk(g.h / 3.f), h6 = mk(g.h / 6.f);
  constexpr float kA[3] = {0.5f, 0.5f, 1.0f};
  f2 lam[P];
#pragma unroll
  for (int p = 0; p < P; ++p) lam[p] = mk(0.f);
  R::store(lam_c, tid, NT, lam);
  if (g.N > 0) {
    R::prefetch(sm + ((g.N - 1) & 1) * H, trajp + (size_t)(g.N - 1) * H + i0, tid, NT);
    R::wait();
  }
  __syncthreads();
  int oi_next = g.obs_of_step[g.N];
  for (int t = g.N; t >= 1; --t) {
    const int oi = oi_next;
    oi_next = g.obs_of_step[t - 1];
    if (oi >= 0) {
      R::store(ubuf[0], tid, NT, lam);
      __syncthreads();
      for (int o = tid; o < g.n_o; o += NT) {
        int il, half_;
        if (pair_of(g.obs_idx[oi * g.n_o + o], g, 0, il, half_)) {
          f2* cell = &ubuf[0][R::elem(il / P, il % P, NT)];
          atomicAdd(half_ ? &cell->y : &cell->x, win[oi * g.n_o + o] * g.inv_sigma);
        }
      }
      __syncthreads();
      R::load(ubuf[0], tid, NT, lam);
    }
    const int r = t - 1;  // base state x_{t-1}
    const f2* xb = sm + (r & 1) * H;
    f2 x[P], U[P], uL, uR, kL, kR;
    R::load(xb, tid, NT, x);
    rh.get(xb, uL, uR);
#pragma unroll
    for (int p = 0; p < P; ++p) U[p] = x[p];
    // forward: stage states U1, U2 (kept in shared memory) and U3 (registers)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const float ha = g.h * kA[s];
      const f2 sc1 = mk(-ha * g.c1), sc2 = mk(ha * g.c2), nsc2 = mk(-ha * g.c2);
      f2 Un[P];
      // U_{s+1} = x - h a (nM du_{p+1} + P du_p) with du_q = U_q - U_{q-1}
      auto pair = [&](int p, f2 du0, f2 du1) {
        const f2 Ps = fma2(sc1, U[p], nsc2);   // -h a P
        const f2 Ms = fma2(sc1, U[p], sc2);    // -h a nM
        Un[p] = fma2(Ms, du1, fma2(Ps, du0, x[p]));
      };
      const f2 du1 = fma2(U[0], m1, U[1]);
      f2 dum = du1;
#pragma unroll
      for (int p = 1; p < P - 1; ++p) {
        const f2 dun = fma2(U[p], m1, U[p + 1]);
        pair(p, dum, dun);
        dum = dun;
      }
      pair(P - 1, dum, fma2(U[P - 1], m1, uR));
      pair(0, fma2(uL, m1, U[0]), du1);
      const int par = s & 1;
      X.put(par, 0, Un[0], Un[P - 1]);
      if (s == 2) X.put(par, 1, mul2(h6, lam[0]), mul2(h6, lam[P - 1]));  // kappa_3 = h/6 lambda'
      if (s < 2) R::store(ubuf[s], tid, NT, Un);
      __syncthreads();
      if (s == 0 && r >= 1) R::prefetch(sm + ((r - 1) & 1) * H, trajp + (size_t)(r - 1) * H + i0, tid, NT);
      X.get(par, 0, uL, uR);
      if (s == 2) X.get(par, 1, kL, kR);
#pragma unroll
      for (int p = 0; p < P; ++p) U[p] = Un[p];
    }
    // backward: kappa_3 = h b_3 lambda', theta_s = F_s^T kappa_s, lambda += theta_s,
    // kappa_{s-1} = h b_{s-1} lambda' + h a_{s-1} theta_s
    // (h b lambda' is formed where it is used: no register array for it)
    f2 K[P], th[P];
#pragma unroll
    for (int p = 0; p < P; ++p) K[p] = mul2(h6, lam[p]);
#pragma unroll
    for (int s = 3; s >= 0; --s) {
      if (s == 1 || s == 2) rh.get(ubuf[s - 1], uL, uR);
      else if (s == 0) rh.get(xb, uL, uR);
      const f2 hA = mk(s > 0 ? g.h * kA[s - 1] : 0.f);
      f2 Kn[P];
      // theta_p = P_{p+1} dk_{p+1} + nM_{p-1} dk_p with dk_q = K_q - K_{q-1}
      auto pair = [&](int p, f2 nMm, f2 Pn, f2 dk0, f2 dk1) {
        const f2 ts = fma2(Pn, dk1, mul2(nMm, dk0));
        th[p] = (s == 3) ? ts : add2(th[p], ts);
        if (s == 3 || s == 2) Kn[p] = fma2(hA, ts, mul2(h3, lam[p]));
        else if (s == 1) Kn[p] = fma2(hA, ts, mul2(h6, lam[p]));
      };
      const f2 nM0 = fma2(c1, U[0], nc2), dk1 = fma2(K[0], m1, K[1]);
      f2 nMm = nM0, dkm = dk1;
#pragma unroll
      for (int p = 1; p < P - 1; ++p) {
        const f2 dkn = fma2(K[p], m1, K[p + 1]);
        pair(p, nMm, fma2(c1, U[p + 1], c2), dkm, dkn);
        nMm = fma2(c1, U[p], nc2);
        dkm = dkn;
      }
      pair(P - 1, nMm, fma2(c1, uR, c2), dkm, fma2(K[P - 1], m1, kR));
      pair(0, fma2(c1, uL, nc2), fma2(c1, U[1], c2), fma2(kL, m1, K[0]), dk1);
      if (s > 0) {
        const int par = s & 1;  // exchanges 3, 4, 5 of the step alternate with 2
        X.put(par, 1, Kn[0], Kn[P - 1]);
        // the next stage state (my own chunks) is loaded before the barrier
        if (s == 1) {
          R::load(xb, tid, NT, U);
          R::wait();
        } else {
          R::load(ubuf[s - 2], tid, NT, U);
        }
        __syncthreads();
        X.get(par, 1, kL, kR);
#pragma unroll
        for (int p = 0; p < P; ++p) K[p] = Kn[p];
      }
    }
    // lambda += sum_s theta_s, the rounding error carried to the next step
    // (Fast2Sum, as for the tangent-linear state)
    {
      f2 cv[P];
      R::load(lam_c, tid, NT, cv);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const f2 inc = add2(th[p], cv[p]);
        const f2 sum = add2(lam[p], inc);
        cv[p] = add2(fma2(sum, m1, lam[p]), inc);
        lam[p] = sum;
      }
      R::store(lam_c, tid, NT, cv);
    }
  }
  f2 cv[P];
  R::load(lam_c, tid, NT, cv);
  float* out = Out + (size_t)col * ldo;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const f2 l = add2(lam[p], cv[p]);
    out[i0 + p] = l.x;
    out[H + i0 + p] = l.y;
  }
}

// ---------------------------------------------------------------- host
const size_t kMaxSmem2 = 227 * 1024;

// Pairs per thread of a sweep over Hs pairs per CTA. Default: up to 8 (512
// threads); the one-CTA adjoint sweep over 4096 pairs (n = 8192) takes 16 pairs
// per thread (256 threads), which measured faster there.
int pairs_per_thread(int Hs, int tuned, bool adj = false) {
  static int forced = [] {
    const char* e = getenv("SC4DVAR_PAIRS_P");
    return e ? atoi(e) : 0;
  }();
  const int dflt = (adj && Hs == 4096) ? 16 : std::max(1, std::min(8, Hs / 512));
  // the tuned shape is the tangent-linear sweep's; the adjoint keeps 16 at 4096 pairs
  int P = (tuned > 0 && !(adj && Hs == 4096)) ? tuned : (forced > 0 ? forced : dflt);
  if (P == 16 && Hs % 16 == 0 && Hs / 16 >= 64 && Hs / 16 <= 256) return P;  // one-CTA sweeps only
  if (P != 1 && P != 2 && P != 4 && P != 8) P = 8;
  while (P > 1 && Hs / P < 32) P /= 2;
  while (Hs / P > Bounds2<8>::kThreads * (P >= 8 ? 1 : 2) && P < 8) P *= 2;
  return P;
}

int cluster_for(int H, int k, int arrays) {
  int cl = 1;
  while ((size_t)(arrays * (H / cl + 2 * kPad2) + 256) * sizeof(f2) > kMaxSmem2 && cl < 16) cl *= 2;
  if (k <= 4) {
    // few directions: SC4DVAR_FEW_CLUSTER (2, 4 or 8) spreads each over that
    // many CTAs of a cluster. The default keeps one CTA per direction: the
    // one-CTA sweeps beat the cluster sweeps, which wait on a cluster barrier per
    // exchange (n = 8192, one direction: TLM + ADJ 79 ms on one SM, 101 ms on 8)
    static int cap = [] {
      const char* e = getenv("SC4DVAR_FEW_CLUSTER");
      int c = e ? atoi(e) : 1;
      return (c == 2 || c == 4 || c == 8) ? c : 1;
    }();
    while (cl < cap && H / (cl * 2) >= 256) cl *= 2;
  }
  return cl;
}

Geo make_geo(const ModelGeom& m, int cl) {
  Geo g;
  g.n = m.n;
  g.H = m.n / 2;
  g.Hs = g.H / cl;
  g.N = m.N;
  g.n_o = m.n_o;
  double dx = 1.0 / m.n;
  g.h = (float)m.h;
  g.c1 = (float)(1.0 / (2.0 * dx));
  g.c2 = (float)(m.nu / (dx * dx));
  g.inv_sigma = (float)(1.0 / m.sigma);
  g.obs_of_step = m.obs_of_step;
  g.obs_idx = m.obs_idx;
  return g;
}

template <typename Kern, typename... Args>
int launch2(Kern kern, int grid, int threads, size_t smem, int cl, cudaStream_t st, Args... args) {
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

#define SC4_DISPATCH_PAIRS(P, BODY)                                      \
  switch (P) {                                                           \
    case 1: { constexpr int PP = 1; BODY; } break;                       \
    case 2: { constexpr int PP = 2; BODY; } break;                       \
    case 4: { constexpr int PP = 4; BODY; } break;                       \
    case 8: { constexpr int PP = 8; BODY; } break;                       \
    default: set_error("unsupported pairs per thread"); return SC4DVAR_ERR_INVALID_ARG; \
  }

}  // namespace

bool packed_f32_supported(int n) { return n >= kPackedMinN && n % 64 == 0; }

int burgers_tlm_f32x2(const ModelGeom& m, const float* traj_folded, const float* U0, int ldu, int k,
                      float* W, int ldw, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  const int H = m.n / 2;
  int cl = cluster_for(H, k, 3);
  Geo g = make_geo(m, cl);
  int P = pairs_per_thread(g.Hs, m.pairs_tuned);
  if (cl > 1 && P > 8) P = 8;
  int NT = g.Hs / P;
  const size_t sm1 = (size_t)(4 * H + 8 * NT) * sizeof(f2);
  if (cl == 1 && P >= 4 && NT <= 512 && sm1 <= kMaxSmem2) {
    if (P == 4) SC4_TRY(launch2(tlm1_kernel<4>, k, NT, sm1, 1, st, g, traj_folded, U0, ldu, W, ldw));
    else if (P == 16) SC4_TRY(launch2(tlm1_kernel<16>, k, NT, sm1, 1, st, g, traj_folded, U0, ldu, W, ldw));
    else SC4_TRY(launch2(tlm1_kernel<8>, k, NT, sm1, 1, st, g, traj_folded, U0, ldu, W, ldw));
    return SC4DVAR_OK;
  }
  size_t smem = (size_t)(2 * g.Hs + g.Hs + 2 * kPad2 + 8 * 32) * sizeof(f2);
  if (cl > 1) {
    SC4_DISPATCH_PAIRS(P, SC4_TRY(launch2(tlm_f32x2_kernel<PP, true>, k * cl, NT, smem, cl, st, g,
                                          traj_folded, U0, ldu, W, ldw)));
  } else {
    SC4_DISPATCH_PAIRS(P, SC4_TRY(launch2(tlm_f32x2_kernel<PP, false>, k, NT, smem, 1, st, g,
                                          traj_folded, U0, ldu, W, ldw)));
  }
  return SC4DVAR_OK;
}

int burgers_adj_f32x2(const ModelGeom& m, const float* traj_folded, const float* Win, int ldw, int k,
                      float* Out, int ldo, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  const int H = m.n / 2;
  int cl = cluster_for(H, k, 4);
  Geo g = make_geo(m, cl);
  int P = pairs_per_thread(g.Hs, m.pairs_tuned, true);
  if (cl > 1 && P > 8) P = 8;
  int NT = g.Hs / P;
  const size_t sm1 = (size_t)(5 * H + 8 * NT) * sizeof(f2);
  if (cl == 1 && P >= 4 && NT <= 512 && sm1 <= kMaxSmem2) {
    if (P == 4) SC4_TRY(launch2(adj1_kernel<4>, k, NT, sm1, 1, st, g, traj_folded, Win, ldw, Out, ldo));
    else if (P == 16) SC4_TRY(launch2(adj1_kernel<16>, k, NT, sm1, 1, st, g, traj_folded, Win, ldw, Out, ldo));
    else SC4_TRY(launch2(adj1_kernel<8>, k, NT, sm1, 1, st, g, traj_folded, Win, ldw, Out, ldo));
    return SC4DVAR_OK;
  }
  size_t smem = (size_t)(4 * (g.Hs + 2 * kPad2) + 4 * 32) * sizeof(f2);
  if (cl > 1) {
    SC4_DISPATCH_PAIRS(P, SC4_TRY(launch2(adj_f32x2_kernel<PP, true>, k * cl, NT, smem, cl, st, g,
                                          traj_folded, Win, ldw, Out, ldo)));
  } else {
    SC4_DISPATCH_PAIRS(P, SC4_TRY(launch2(adj_f32x2_kernel<PP, false>, k, NT, smem, 1, st, g,
                                          traj_folded, Win, ldw, Out, ldo)));
  }
  return SC4DVAR_OK;
}

}  // namespace sc4
