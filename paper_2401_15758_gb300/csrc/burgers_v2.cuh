// Register-resident Burgers sweeps (segments of >= 256 points).
//
// Same arithmetic as the kernels in burgers.cu (see there for the model, the
// TLM and the discrete RK4 adjoint), laid out to cut instructions per point:
// thread t of a CTA owns P CONTIGUOUS points of its segment and keeps the
// tangent (or adjoint) stage vector in registers. Neighbour values inside the
// thread come from its own registers; across threads from warp shuffles; across
// warps from two edge slots per warp in shared memory (one barrier per RK
// stage publishes them); across CTAs of a cluster through DSMEM. The base stage
// states of the ADJ sweep are kept in shared memory (they are needed again, in
// reverse order, by the adjoint stages). Trajectory rows are read with 16-byte
// vector loads.
#pragma once

namespace sc4 {

constexpr int kPad = 4;  // shared-memory arrays: element j at index j + kPad (16-byte aligned)

// Row of P contiguous values from GLOBAL memory (read-only path).
template <typename T, int P>
__device__ __forceinline__ void load_row_g(const T* __restrict__ src, T (&dst)[P]) {
  if constexpr ((P * sizeof(T)) % 16 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < (int)(P * sizeof(T) / 16); ++i) d4[i] = __ldg(s4 + i);
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) dst[p] = __ldg(src + p);
  }
}

// Row of P contiguous values from SHARED memory (plain loads: the read-only
// global path must not be used on shared addresses).
template <typename T, int P>
__device__ __forceinline__ void load_row_s(const T* src, T (&dst)[P]) {
  if constexpr ((P * sizeof(T)) % 16 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < (int)(P * sizeof(T) / 16); ++i) d4[i] = s4[i];
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) dst[p] = src[p];
  }
}

template <typename T, int P>
__device__ __forceinline__ void store_row(T* dst, const T (&src)[P]) {
  if constexpr ((P * sizeof(T)) % 16 == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < (int)(P * sizeof(T) / 16); ++i) d4[i] = s4[i];
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) dst[p] = src[p];
  }
}

// Edge slots of one exchanged vector: L[w] = first value of warp w, R[w] = last.
template <typename T>
struct Edge {
  T* L;
  T* R;
};

// Publish my edge values (before the barrier).
template <typename T>
__device__ __forceinline__ void edge_put(Edge<T> e, int lane, int w, T first, T last) {
  if (lane == 0) e.L[w] = first;
  if (lane == 31) e.R[w] = last;
}

// Halo values left/right of my P points (after the barrier). `sl`/`sr` are the
// shuffled neighbour values computed before the barrier.
template <bool CL, typename T>
__device__ __forceinline__ void edge_get(Edge<T> e, int lane, int w, int nw, int crank, int csize,
                                         T& left, T& right) {
  if (lane == 0) {
    if (w > 0) {
      left = e.R[w - 1];
    } else if constexpr (CL) {
      left = cg::this_cluster().map_shared_rank(e.R, (crank + csize - 1) % csize)[nw - 1];
    } else {
      left = e.R[nw - 1];
    }
  }
  if (lane == 31) {
    if (w < nw - 1) {
      right = e.L[w + 1];
    } else if constexpr (CL) {
      right = cg::this_cluster().map_shared_rank(e.L, (crank + 1) % csize)[0];
    } else {
      right = e.L[0];
    }
  }
}

// Store my P points into a padded shared array and, for the segment ends, into
// the neighbour segment's halo cells.
template <bool CL, typename T, int P>
__device__ __forceinline__ void seg_store(T* arr, int tid, int NT, int seg, const T (&v)[P], int crank,
                                          int csize) {
  store_row<T, P>(arr + kPad + tid * P, v);
  if (tid == 0) {
    if constexpr (CL) cg::this_cluster().map_shared_rank(arr, (crank + csize - 1) % csize)[kPad + seg] = v[0];
    else arr[kPad + seg] = v[0];
  }
  if (tid == NT - 1) {
    if constexpr (CL) cg::this_cluster().map_shared_rank(arr, (crank + 1) % csize)[kPad - 1] = v[P - 1];
    else arr[kPad - 1] = v[P - 1];
  }
}

// ---------------------------------------------------------------- TLM (v2)
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(1024, 1) burgers_tlm_v2_kernel(
    BurgersParams<T> pr, const T* __restrict__ traj, const T* __restrict__ U0, int ldu,
    T* __restrict__ W, int ldw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  T* stage = sm;                       // seg + 2 kPad: dx for observation gathers
  T* slots = sm + seg + 2 * kPad;      // [parity 2][array 2][L/R 2][32]
  auto edge = [&](int q, int a) { return Edge<T>{slots + ((q * 2 + a) * 2 + 0) * 32,
                                                  slots + ((q * 2 + a) * 2 + 1) * 32}; };
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const int col = blockIdx.x / csize;
  const int j0 = crank * seg;
  const int my0 = j0 + tid * P;
  T x[P], dx[P], acc[P], U[P], D[P];
  load_row_g<T, P>(U0 + (size_t)col * ldu + my0, dx);
  T* wcol = W + (size_t)col * ldw;
  const T h = pr.h, c1 = pr.inv2dx, c2 = pr.nudx2;
  for (int t = 0;; ++t) {
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      store_row<T, P>(stage + kPad + tid * P, dx);
      bar<CL>();
      for (int o = tid; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) wcol[oi * pr.n_o + o] = stage[kPad + gj] * pr.inv_sigma;
      }
    }
    if (t == pr.N) break;
    load_row_g<T, P>(traj + (size_t)t * pr.n + my0, x);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      U[p] = x[p];
      D[p] = dx[p];
      acc[p] = (T)0;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      Edge<T> eu = edge(s & 1, 0), ed = edge(s & 1, 1);
      edge_put(eu, lane, w, U[0], U[P - 1]);
      edge_put(ed, lane, w, D[0], D[P - 1]);
      T uL = __shfl_up_sync(0xffffffffu, U[P - 1], 1), uR = __shfl_down_sync(0xffffffffu, U[0], 1);
      T dL = __shfl_up_sync(0xffffffffu, D[P - 1], 1), dR = __shfl_down_sync(0xffffffffu, D[0], 1);
      bar<CL>();
      edge_get<CL>(eu, lane, w, nw, crank, csize, uL, uR);
      edge_get<CL>(ed, lane, w, nw, crank, csize, dL, dR);
      const T bs = (T)kRkB[s];
      const T ha = (s < 3) ? h * (T)kRkA[s] : (T)0;
      T up = uL, dp = dL;  // old values at p-1
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T u = U[p], d = D[p];
        T un = (p + 1 < P) ? U[p + 1] : uR;
        T dn = (p + 1 < P) ? D[p + 1] : dR;
        T d1u = (un - up) * c1;
        T dk = -d1u * d - u * ((dn - dp) * c1) + c2 * (dn - (T)2 * d + dp);
        acc[p] += bs * dk;
        if (s < 3) {
          T k = -u * d1u + c2 * (un - (T)2 * u + up);
          U[p] = x[p] + ha * k;
          D[p] = dx[p] + ha * dk;
        }
        up = u;
        dp = d;
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) dx[p] += h * acc[p];
  }
}

// ---------------------------------------------------------------- ADJ (v2)
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(1024, 1) burgers_adj_v2_kernel(
    BurgersParams<T> pr, const T* __restrict__ traj, const T* __restrict__ Win, int ldw,
    T* __restrict__ Out, int ldo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  const int S = seg + 2 * kPad;
  T* Sx[4] = {sm, sm + S, sm + 2 * S, sm + 3 * S};  // base stage states X_1..X_4
  T* slots = sm + 4 * S;                            // [parity 2][L/R 2][32]
  auto edge = [&](int q) { return Edge<T>{slots + (q * 2 + 0) * 32, slots + (q * 2 + 1) * 32}; };
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const int col = blockIdx.x / csize;
  const int j0 = crank * seg;
  const int my0 = j0 + tid * P;
  const T* win = Win + (size_t)col * ldw;
  const T h = pr.h, c1 = pr.inv2dx, c2 = pr.nudx2;
  T lam[P], x[P], th[P], K[P];
#pragma unroll
  for (int p = 0; p < P; ++p) lam[p] = (T)0;
  for (int t = pr.N; t >= 1; --t) {
    bar<CL>();  // every reader of the previous step's stage arrays is done
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      T* st = Sx[0];
      store_row<T, P>(st + kPad + tid * P, lam);
      __syncthreads();
      for (int o = tid; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) atomicAdd(&st[kPad + gj], win[oi * pr.n_o + o] * pr.inv_sigma);
      }
      __syncthreads();
      load_row_s<T, P>(st + kPad + tid * P, lam);
      __syncthreads();
    }
    // base stage states of the step t-1 -> t
    load_row_g<T, P>(traj + (size_t)(t - 1) * pr.n + my0, x);
    seg_store<CL, T, P>(Sx[0], tid, NT, seg, x, crank, csize);
    bar<CL>();
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const T* Us = Sx[s] + kPad + tid * P;
      T u[P];
      load_row_s<T, P>(Us, u);
      T up = Us[-1], un_last = Us[P];
      const T ha = h * (T)kRkA[s];
      T nx[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T uc = u[p];
        T un = (p + 1 < P) ? u[p + 1] : un_last;
        T d1u = (un - up) * c1;
        T k = -uc * d1u + c2 * (un - (T)2 * uc + up);
        nx[p] = x[p] + ha * k;
        up = uc;
      }
      seg_store<CL, T, P>(Sx[s + 1], tid, NT, seg, nx, crank, csize);
      if (s == 2) {
        const T hb = h * (T)kRkB[3];
#pragma unroll
        for (int p = 0; p < P; ++p) K[p] = hb * lam[p];
      }
      bar<CL>();
    }
    // adjoint stages 4, 3, 2, 1
#pragma unroll
    for (int p = 0; p < P; ++p) th[p] = (T)0;
#pragma unroll
    for (int s = 3; s >= 0; --s) {
      Edge<T> ek = edge(s & 1);
      edge_put(ek, lane, w, K[0], K[P - 1]);
      T kL = __shfl_up_sync(0xffffffffu, K[P - 1], 1), kR = __shfl_down_sync(0xffffffffu, K[0], 1);
      bar<CL>();
      edge_get<CL>(ek, lane, w, nw, crank, csize, kL, kR);
      const T* Us = Sx[s] + kPad + tid * P;
      T u[P];
      load_row_s<T, P>(Us, u);
      T up = Us[-1], un_last = Us[P];
      const T hb = (s > 0) ? h * (T)kRkB[s - 1] : (T)0;
      const T ha = (s > 0) ? h * (T)kRkA[s - 1] : (T)0;
      T kp = kL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T uc = u[p], kc = K[p];
        T un = (p + 1 < P) ? u[p + 1] : un_last;
        T kn = (p + 1 < P) ? K[p + 1] : kR;
        T d1u = (un - up) * c1;
        T theta = -d1u * kc + (un * kn - up * kp) * c1 + c2 * (kn - (T)2 * kc + kp);
        th[p] += theta;
        if (s > 0) K[p] = hb * lam[p] + ha * theta;
        up = uc;
        kp = kc;
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) lam[p] += th[p];
  }
  store_row<T, P>(Out + (size_t)col * ldo + my0, lam);
}

// ---------------------------------------------------------------- FWD (v2)
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(1024, 1) burgers_fwd_v2_kernel(
    BurgersParams<T> pr, const T* __restrict__ x0, T* __restrict__ traj, float* __restrict__ traj32,
    const double* __restrict__ y, double* __restrict__ d_out, double* __restrict__ obs_out,
    T* __restrict__ xN) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  T* stage = sm;
  T* slots = sm + seg + 2 * kPad;  // [parity 2][L/R 2][32]
  auto edge = [&](int q) { return Edge<T>{slots + (q * 2 + 0) * 32, slots + (q * 2 + 1) * 32}; };
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const int j0 = crank * seg;
  const int my0 = j0 + tid * P;
  const T h = pr.h, c1 = pr.inv2dx, c2 = pr.nudx2;
  T x[P], acc[P], U[P];
  load_row_g<T, P>(x0 + my0, x);
  for (int t = 0;; ++t) {
    if (traj) store_row<T, P>(traj + (size_t)t * pr.n + my0, x);
    if (traj32) {
#pragma unroll
      for (int p = 0; p < P; ++p) traj32[(size_t)t * pr.n + my0 + p] = (float)x[p];
    }
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      store_row<T, P>(stage + kPad + tid * P, x);
      bar<CL>();
      for (int o = tid; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) {
          double v = (double)stage[kPad + gj];
          int r = oi * pr.n_o + o;
          if (obs_out) obs_out[r] = v;
          if (d_out) d_out[r] = (v - y[r]) * (double)pr.inv_sigma;
        }
      }
    }
    if (t == pr.N) break;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      U[p] = x[p];
      acc[p] = (T)0;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      Edge<T> eu = edge(s & 1);
      edge_put(eu, lane, w, U[0], U[P - 1]);
      T uL = __shfl_up_sync(0xffffffffu, U[P - 1], 1), uR = __shfl_down_sync(0xffffffffu, U[0], 1);
      bar<CL>();
      edge_get<CL>(eu, lane, w, nw, crank, csize, uL, uR);
      const T bs = (T)kRkB[s];
      const T ha = (s < 3) ? h * (T)kRkA[s] : (T)0;
      T up = uL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T u = U[p];
        T un = (p + 1 < P) ? U[p + 1] : uR;
        T k = -u * ((un - up) * c1) + c2 * (un - (T)2 * u + up);
        acc[p] += bs * k;
        if (s < 3) U[p] = x[p] + ha * k;
        up = u;
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] += h * acc[p];
  }
  if (xN) store_row<T, P>(xN + my0, x);
}

}  // namespace sc4
