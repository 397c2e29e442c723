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

// Where a warp's edge lanes find their neighbours' edge values: computed once
// per thread. `lo` / `ro` are the element offsets (from the slot base) of the
// left warp's last value and the right warp's first value; `lbase` / `rbase` are
// this CTA's slot base or, for the segment ends in a cluster, the neighbour
// CTA's (DSMEM).
template <typename T>
struct EdgeNb {
  const T* lbase;
  const T* rbase;
  int lw, rw;
};

template <bool CL, typename T>
__device__ __forceinline__ EdgeNb<T> edge_nb(T* slots, int w, int nw, int crank, int csize) {
  EdgeNb<T> nb;
  nb.lbase = slots;
  nb.rbase = slots;
  nb.lw = (w > 0) ? w - 1 : nw - 1;
  nb.rw = (w < nw - 1) ? w + 1 : 0;
  if constexpr (CL) {
    if (w == 0) nb.lbase = cg::this_cluster().map_shared_rank(slots, (crank + csize - 1) % csize);
    if (w == nw - 1) nb.rbase = cg::this_cluster().map_shared_rank(slots, (crank + 1) % csize);
  }
  return nb;
}

// Halo values left/right of my P points (after the barrier); e.L / e.R are
// offsets of that vector's slot arrays from the slot base.
template <typename T>
__device__ __forceinline__ void edge_get(const EdgeNb<T>& nb, int offL, int offR, int lane, T& left,
                                         T& right) {
  if (lane == 0) left = nb.lbase[offR + nb.lw];
  if (lane == 31) right = nb.rbase[offL + nb.rw];
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

// ---- chunk-major shared rows and asynchronous row prefetch ----------------
// A thread's P contiguous values are E-element 16-byte chunks (E = 16/sizeof(T));
// chunk q of thread t lives at chunk slot q*NT + t, so that a warp's 16-byte
// shared accesses of one chunk index hit consecutive slots (no bank conflicts).
// Rows that are not a whole number of chunks use the plain layout t*P + p.
template <typename T, int P>
struct Rows {
  static constexpr bool kVec = (P * sizeof(T)) % 16 == 0;
  static constexpr int E = 16 / sizeof(T);
  static constexpr int C = kVec ? P / E : 0;
  __device__ static __forceinline__ int elem(int t, int p, int NT) {
    if constexpr (kVec) return ((p / E) * NT + t) * E + (p % E);
    else return t * P + p;
  }
  __device__ static __forceinline__ void load(const T* base, int t, int NT, T (&v)[P]) {
    if constexpr (kVec) {
      const float4* b4 = reinterpret_cast<const float4*>(base);
      float4* v4 = reinterpret_cast<float4*>(v);
#pragma unroll
      for (int q = 0; q < C; ++q) v4[q] = b4[q * NT + t];
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) v[p] = base[t * P + p];
    }
  }
  __device__ static __forceinline__ void store(T* base, int t, int NT, const T (&v)[P]) {
    if constexpr (kVec) {
      float4* b4 = reinterpret_cast<float4*>(base);
      const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll
      for (int q = 0; q < C; ++q) b4[q * NT + t] = v4[q];
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) base[t * P + p] = v[p];
    }
  }
  // Asynchronous copy of my global row (P contiguous values at src) into base.
  // Rows that are not whole chunks fall back to plain loads and stores.
  __device__ static __forceinline__ void prefetch(T* base, const T* __restrict__ src, int t, int NT) {
    if constexpr (kVec) {
#pragma unroll
      for (int q = 0; q < C; ++q) {
        unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<float4*>(base) + q * NT + t);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + q * E));
      }
      asm volatile("cp.async.commit_group;\n" ::);
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) base[t * P + p] = __ldg(src + p);
    }
  }
  __device__ static __forceinline__ void wait_prefetch() {
    if constexpr (kVec) asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
};

// Shared-memory offsets (within a halo-padded chunk-major segment array) of
// the values left of my first point and right of my last point.
template <typename T, int P>
struct RowNb {
  int lofs, rofs;
  __device__ RowNb(int tid, int NT, int seg) {
    lofs = (tid == 0) ? kPad - 1 : kPad + Rows<T, P>::elem(tid - 1, P - 1, NT);
    rofs = (tid == NT - 1) ? kPad + seg : kPad + Rows<T, P>::elem(tid + 1, 0, NT);
  }
};

// Neighbours of my row v of the shared array arr: shuffles inside the warp, the
// shared copy for the warp's edge lanes.
template <typename T, int P>
__device__ __forceinline__ void row_halos(const T* arr, const T (&v)[P], const RowNb<T, P>& nb,
                                          int lane, T& left, T& right) {
  left = __shfl_up_sync(0xffffffffu, v[P - 1], 1);
  right = __shfl_down_sync(0xffffffffu, v[0], 1);
  if (lane == 0) left = arr[nb.lofs];
  if (lane == 31) right = arr[nb.rofs];
}

// Store my row into a chunk-major segment array and the segment-end values into
// the neighbour segments' halo cells (DSMEM in a cluster).
template <bool CL, typename T, int P>
__device__ __forceinline__ void row_store(T* arr, int tid, int NT, int seg, const T (&v)[P], int crank,
                                          int csize) {
  Rows<T, P>::store(arr + kPad, tid, NT, v);
  if (tid == 0) {
    if constexpr (CL) cg::this_cluster().map_shared_rank(arr, (crank + csize - 1) % csize)[kPad + seg] = v[0];
    else arr[kPad + seg] = v[0];
  }
  if (tid == NT - 1) {
    if constexpr (CL) cg::this_cluster().map_shared_rank(arr, (crank + 1) % csize)[kPad - 1] = v[P - 1];
    else arr[kPad - 1] = v[P - 1];
  }
}

// Threads per CTA for rows of P values of type T: the register budget per
// thread grows with the bytes of a row (32 B rows: 1024 threads, 64 B: 512,
// 128 B: 256).
template <typename T, int P>
struct Bounds {
  static constexpr int kBytes = P * (int)sizeof(T);
  static constexpr int kThreads = kBytes >= 128 ? 256 : (kBytes >= 64 ? 512 : 1024);
};

// ---------------------------------------------------------------- TLM (v2)
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(Bounds<T, P>::kThreads, 1) burgers_tlm_v2_kernel(
    BurgersParams<T> pr, const T* __restrict__ traj, const T* __restrict__ U0, int ldu,
    T* __restrict__ W, int ldw) {
  using R = Rows<T, P>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  T* xbuf[2] = {sm, sm + seg};          // prefetched base rows (chunk-major, own cells only)
  T* stage = sm + 2 * seg;              // seg + 2 kPad: dx for observation gathers
  T* slots = stage + seg + 2 * kPad;    // [parity 2][array 2][L/R 2][32]
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const EdgeNb<T> enb = edge_nb<CL, T>(slots, w, nw, crank, csize);
  const int col = blockIdx.x / csize;
  const int j0 = crank * seg;
  const int my0 = j0 + tid * P;
  T x[P], dx[P], acc[P], U[P], D[P];
  load_row_g<T, P>(U0 + (size_t)col * ldu + my0, dx);
  T* wcol = W + (size_t)col * ldw;
  const T h = pr.h, c1 = pr.inv2dx, c2 = pr.nudx2;
  const T two = (T)2;
  if (pr.N > 0) R::prefetch(xbuf[0], traj + my0, tid, NT);
  for (int t = 0;; ++t) {
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      R::store(stage + kPad, tid, NT, dx);
      bar<CL>();
      for (int o = tid; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg) wcol[oi * pr.n_o + o] = stage[kPad + R::elem(gj / P, gj % P, NT)] * pr.inv_sigma;
      }
    }
    if (t == pr.N) break;
    R::wait_prefetch();
    R::load(xbuf[t & 1], tid, NT, x);
    if (t + 1 < pr.N) R::prefetch(xbuf[(t + 1) & 1], traj + (size_t)(t + 1) * pr.n + my0, tid, NT);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      U[p] = x[p];
      D[p] = dx[p];
      acc[p] = (T)0;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int q = s & 1;
      T* su = slots + ((q * 2 + 0) * 2) * 32;
      T* sd = slots + ((q * 2 + 1) * 2) * 32;
      edge_put(Edge<T>{su, su + 32}, lane, w, U[0], U[P - 1]);
      edge_put(Edge<T>{sd, sd + 32}, lane, w, D[0], D[P - 1]);
      T uL = __shfl_up_sync(0xffffffffu, U[P - 1], 1), uR = __shfl_down_sync(0xffffffffu, U[0], 1);
      T dL = __shfl_up_sync(0xffffffffu, D[P - 1], 1), dR = __shfl_down_sync(0xffffffffu, D[0], 1);
      bar<CL>();
      edge_get(enb, (int)(su - slots), (int)(su - slots) + 32, lane, uL, uR);
      edge_get(enb, (int)(sd - slots), (int)(sd - slots) + 32, lane, dL, dR);
      const T bs = (T)kRkB[s];
      const T ha = (s < 3) ? h * (T)kRkA[s] : (T)0;
      T up = uL, dp = dL;  // old values at p-1
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T u = U[p], d = D[p];
        T un = (p + 1 < P) ? U[p + 1] : uR;
        T dn = (p + 1 < P) ? D[p + 1] : dR;
        T d1u = (un - up) * c1;
        T dk = -d1u * d - u * ((dn - dp) * c1) + c2 * (dn - two * d + dp);
        acc[p] += bs * dk;
        if (s < 3) {
          T k = -u * d1u + c2 * (un - two * u + up);
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
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

// ---------------------------------------------------------------- ADJ (v2)
// Per step (t -> t-1, base x_{t-1}): the four base stage states X_1..X_4 go to
// four shared buffers whose roles rotate from step to step (the buffer of X_4
// becomes the next step's X_1, prefetched with cp.async once X_4 is no longer
// read), so no barrier is needed between steps; seven barriers per step.
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(Bounds<T, P>::kThreads, 1) burgers_adj_v2_kernel(
    BurgersParams<T> pr, const T* __restrict__ traj, const T* __restrict__ Win, int ldw,
    T* __restrict__ Out, int ldo) {
  using R = Rows<T, P>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  const int S = seg + 2 * kPad;
  T* buf[4] = {sm, sm + S, sm + 2 * S, sm + 3 * S};
  T* slots = sm + 4 * S;  // [parity 2][L/R 2][32]
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const EdgeNb<T> enb = edge_nb<CL, T>(slots, w, nw, crank, csize);
  const RowNb<T, P> rnb(tid, NT, seg);
  const int col = blockIdx.x / csize;
  const int j0 = crank * seg;
  const int my0 = j0 + tid * P;
  const T* win = Win + (size_t)col * ldw;
  const T h = pr.h, c1 = pr.inv2dx, c2 = pr.nudx2;
  const T two = (T)2;
  T lam[P], x[P], th[P], K[P], u[P];
#pragma unroll
  for (int p = 0; p < P; ++p) lam[p] = (T)0;
  // X_1 of the first step (t = N, base x_{N-1}) into buf[0]
  R::prefetch(buf[0] + kPad, traj + (size_t)(pr.N - 1) * pr.n + my0, tid, NT);
  for (int t = pr.N, c = 0; t >= 1; --t, ++c) {
    const int r = c & 3;
    T* B0 = buf[(4 - r) & 3];        // X_1
    T* B1 = buf[(5 - r) & 3];        // X_2
    T* B2 = buf[(6 - r) & 3];        // X_3
    T* B3 = buf[(7 - r) & 3];        // X_4 (next step's X_1)
    int oi = pr.obs_of_step[t];
    if (oi >= 0) {
      // lam += O^T R^{-1/2} w_t, scattered through B1 (free: last read one step ago)
      bar<CL>();
      R::store(B1 + kPad, tid, NT, lam);
      __syncthreads();
      for (int o = tid; o < pr.n_o; o += NT) {
        int gj = pr.obs_idx[oi * pr.n_o + o] - j0;
        if (gj >= 0 && gj < seg)
          atomicAdd(&B1[kPad + R::elem(gj / P, gj % P, NT)], win[oi * pr.n_o + o] * pr.inv_sigma);
      }
      __syncthreads();
      R::load(B1 + kPad, tid, NT, lam);
    }
    R::wait_prefetch();
    R::load(B0 + kPad, tid, NT, x);
    if (tid == 0) {
      if constexpr (CL) cg::this_cluster().map_shared_rank(B0, (crank + csize - 1) % csize)[kPad + seg] = x[0];
      else B0[kPad + seg] = x[0];
    }
    if (tid == NT - 1) {
      if constexpr (CL) cg::this_cluster().map_shared_rank(B0, (crank + 1) % csize)[kPad - 1] = x[P - 1];
      else B0[kPad - 1] = x[P - 1];
    }
    bar<CL>();                                                    // 1
    // base stage states X_2..X_4 (kept in registers from one stage to the next)
#pragma unroll
    for (int p = 0; p < P; ++p) u[p] = x[p];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const T* Bs = (s == 0) ? B0 : (s == 1 ? B1 : B2);
      T* Bn = (s == 0) ? B1 : (s == 1 ? B2 : B3);
      T uL, uR;
      row_halos<T, P>(Bs, u, rnb, lane, uL, uR);
      const T ha = h * (T)kRkA[s];
      T up = uL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T uc = u[p];
        T un = (p + 1 < P) ? u[p + 1] : uR;
        T d1u = (un - up) * c1;
        T k = -uc * d1u + c2 * (un - two * uc + up);
        u[p] = x[p] + ha * k;
        up = uc;
      }
      row_store<CL, T, P>(Bn, tid, NT, seg, u, crank, csize);
      if (s == 2) {
        const T hb = h * (T)kRkB[3];
#pragma unroll
        for (int p = 0; p < P; ++p) K[p] = hb * lam[p];
        edge_put(Edge<T>{slots, slots + 32}, lane, w, K[0], K[P - 1]);
      }
      bar<CL>();                                                  // 2, 3, 4
    }
    // adjoint stages 4, 3, 2, 1 (u holds X_4 now)
#pragma unroll
    for (int p = 0; p < P; ++p) th[p] = (T)0;
#pragma unroll
    for (int s = 3; s >= 0; --s) {
      const T* Bs = (s == 3) ? B3 : (s == 2 ? B2 : (s == 1 ? B1 : B0));
      if (s == 2 || s == 1) R::load(Bs + kPad, tid, NT, u);
      if (s == 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = x[p];
      }
      const int qin = ((3 - s) & 1) * 64;   // slot offset of this phase's K edges
      T kL = __shfl_up_sync(0xffffffffu, K[P - 1], 1), kR = __shfl_down_sync(0xffffffffu, K[0], 1);
      edge_get(enb, qin, qin + 32, lane, kL, kR);
      T uL, uR;
      row_halos<T, P>(Bs, u, rnb, lane, uL, uR);
      const T hb = (s > 0) ? h * (T)kRkB[s - 1] : (T)0;
      const T ha = (s > 0) ? h * (T)kRkA[s - 1] : (T)0;
      T up = uL, kp = kL;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        T uc = u[p], kc = K[p];
        T un = (p + 1 < P) ? u[p + 1] : uR;
        T kn = (p + 1 < P) ? K[p + 1] : kR;
        T d1u = (un - up) * c1;
        T theta = -d1u * kc + (un * kn - up * kp) * c1 + c2 * (kn - two * kc + kp);
        th[p] += theta;
        if (s > 0) K[p] = hb * lam[p] + ha * theta;
        up = uc;
        kp = kc;
      }
      if (s > 0) {
        T* so = slots + ((4 - s) & 1) * 64;
        edge_put(Edge<T>{so, so + 32}, lane, w, K[0], K[P - 1]);
        bar<CL>();                                                // 5, 6, 7
        // after barrier 5 nobody reads X_4 any more: prefetch the next X_1 into it
        if (s == 3 && t > 1) R::prefetch(B3 + kPad, traj + (size_t)(t - 2) * pr.n + my0, tid, NT);
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) lam[p] += th[p];
  }
  store_row<T, P>(Out + (size_t)col * ldo + my0, lam);
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

// ---------------------------------------------------------------- FWD (v2)
template <typename T, int P, bool CL>
__global__ void __launch_bounds__(Bounds<T, P>::kThreads, 1) burgers_fwd_v2_kernel(
    BurgersParams<T> pr, const T* __restrict__ x0, T* __restrict__ traj, float* __restrict__ traj32,
    const double* __restrict__ y, double* __restrict__ d_out, double* __restrict__ obs_out,
    T* __restrict__ xN) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int seg = pr.seg, NT = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5, nw = NT >> 5;
  T* stage = sm;
  T* slots = sm + seg + 2 * kPad;  // [parity 2][L/R 2][32]
  int crank, csize;
  cluster_pos<CL>(crank, csize);
  const EdgeNb<T> enb = edge_nb<CL, T>(slots, w, nw, crank, csize);
  const int j0 = crank * seg;
  const int my0 = j0 + tid * P;
  const T h = pr.h, c1 = pr.inv2dx, c2 = pr.nudx2;
  T x[P], acc[P], U[P];
  load_row_g<T, P>(x0 + my0, x);
  for (int t = 0;; ++t) {
    if (traj) store_row<T, P>(traj + (size_t)t * pr.n + my0, x);
    if (traj32) {
#pragma unroll
      for (int p = 0; p < P; ++p)
        traj32[(size_t)t * pr.n + (pr.fold32 ? fold_pos(my0 + p, pr.n) : (size_t)(my0 + p))] = (float)x[p];
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
      T* so = slots + (s & 1) * 64;
      edge_put(Edge<T>{so, so + 32}, lane, w, U[0], U[P - 1]);
      T uL = __shfl_up_sync(0xffffffffu, U[P - 1], 1), uR = __shfl_down_sync(0xffffffffu, U[0], 1);
      bar<CL>();
      edge_get(enb, (int)(so - slots), (int)(so - slots) + 32, lane, uL, uR);
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
  cluster_leave<CL>();  // no CTA leaves while a peer may still reach its shared memory
}

}  // namespace sc4
