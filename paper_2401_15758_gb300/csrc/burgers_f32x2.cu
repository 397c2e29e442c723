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
  if constexpr (CL) {
    crank = (int)cg::this_cluster().block_rank();
    csize = (int)cg::this_cluster().num_blocks();
  } else {
    crank = 0;
    csize = 1;
  }
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
  if constexpr (CL) {
    crank = (int)cg::this_cluster().block_rank();
    csize = (int)cg::this_cluster().num_blocks();
  } else {
    crank = 0;
    csize = 1;
  }
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
}

// ---------------------------------------------------------------- host
const size_t kMaxSmem2 = 227 * 1024;

int pairs_per_thread(int Hs, int tuned) {
  static int forced = [] {
    const char* e = getenv("SC4DVAR_PAIRS_P");
    return e ? atoi(e) : 0;
  }();
  int P = tuned > 0 ? tuned : (forced > 0 ? forced : std::max(1, std::min(8, Hs / 512)));
  if (P != 1 && P != 2 && P != 4 && P != 8) P = 8;
  while (P > 1 && Hs / P < 32) P /= 2;
  while (Hs / P > Bounds2<8>::kThreads * (P >= 8 ? 1 : 2) && P < 8) P *= 2;
  return P;
}

int cluster_for(int H, int k, int arrays) {
  int cl = 1;
  while ((size_t)(arrays * (H / cl + 2 * kPad2) + 256) * sizeof(f2) > kMaxSmem2 && cl < 16) cl *= 2;
  if (k <= 4) {
    // few directions: spread each over up to 8 CTAs; SC4DVAR_FEW_CLUSTER caps
    // the spread (a tuning knob: 1, 2, 4 or 8)
    static int cap = [] {
      const char* e = getenv("SC4DVAR_FEW_CLUSTER");
      int c = e ? atoi(e) : 8;
      return (c == 1 || c == 2 || c == 4) ? c : 8;
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
  int P = pairs_per_thread(g.Hs, m.pairs_tuned), NT = g.Hs / P;
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
  int P = pairs_per_thread(g.Hs, m.pairs_tuned), NT = g.Hs / P;
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
