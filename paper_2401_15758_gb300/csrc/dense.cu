// Dense kernels of the sketching steps (Algs. 1-5) and of PCG.
//
// * gemm_tn:  C (la x lb) = alpha A^T B + beta C, A rows x la, B rows x lb
//             (tall-skinny Gram products: Y^T Y, Omega^T Y, Psi^T Q, Q^T Y).
// * gemm_nn:  C (rows x c) = alpha A B + beta C, A rows x kk, B kk x c (or B^T)
//             (Q = Y L^{-T}, V = W^T U Sigma^{-1}, reorthogonalisation updates).
// FP64 operands accumulate in FP64. FP32 operands avoid the FP64 pipe, which
// runs at 1/64 of the FP32 rate on this GPU: gemm_tn keeps every product exactly
// as a float pair (rounded product + FMA residual) and sums pairs with TwoSum
// into a (hi, lo) float accumulator, so its Gram matrices keep FP64-level
// accuracy (relative error ~1e-14) for CholeskyQR2; gemm_nn (products with a
// small factor: Y L^{-T}, W^T U Sigma^{-1}, projections) accumulates in FP32,
// the precision of its FP32 output. Symmetric Gram products (A == B) compute
// the upper tiles only and mirror them.
// * Small l x l factorizations on one CTA: Cholesky (lower), triangular inverse,
//   cyclic Jacobi eigensolver in round-robin (circle) order, descending sort.
// * Vector helpers for PCG with deterministic two-pass reductions.
#include <algorithm>
#include "common.cuh"
#include "dense.cuh"

namespace sc4 {

// ------------------------------------------------------------------ gemm_tn
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) gemm_tn_kernel(int rows, int la, int lb, int rows_per_chunk,
                                                      double alpha, const TA* __restrict__ A,
                                                      int lda, const TB* __restrict__ B, int ldb,
                                                      double* __restrict__ C, int ldc) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  int r_begin = blockIdx.z * rows_per_chunk;
  int r_end = min(rows, r_begin + rows_per_chunk);
  int ti = threadIdx.x & 31, tj = threadIdx.x >> 5;  // tj in 0..7 -> 4 columns each
  double acc[4] = {0, 0, 0, 0};
  for (int r0 = r_begin; r0 < r_end; r0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      int rr = e & 31, cc = e >> 5;
      int r = r0 + rr;
      As[rr][cc] = (r < r_end && i0 + cc < la) ? (double)A[(size_t)(i0 + cc) * lda + r] : 0.0;
      Bs[rr][cc] = (r < r_end && j0 + cc < lb) ? (double)B[(size_t)(j0 + cc) * ldb + r] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      double a = As[rr][ti];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(a, Bs[rr][tj * 4 + q], acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int i = i0 + ti, j = j0 + tj * 4 + q;
    if (i < la && j < lb) atomicAdd(&C[(size_t)j * ldc + i], alpha * acc[q]);
  }
}

__global__ void scale_matrix_kernel(int r, int c, double beta, double* C, int ldc) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < r * c) {
    int i = idx % r, j = idx / r;
    double* p = &C[(size_t)j * ldc + i];
    *p = (beta == 0.0) ? 0.0 : beta * *p;
  }
}

template <typename TA, typename TB>
int gemm_tn(int rows, int la, int lb, double alpha, const TA* A, int lda, const TB* B, int ldb,
            double beta, double* C, int ldc, cudaStream_t st) {
  if (la <= 0 || lb <= 0) return SC4DVAR_OK;
  scale_matrix_kernel<<<div_up(la * lb, 256), 256, 0, st>>>(la, lb, beta, C, ldc);
  SC4_LAUNCH_CHECK();
  if (rows <= 0) return SC4DVAR_OK;
  int tiles = div_up(la, 32) * div_up(lb, 32);
  int chunks = max(1, min(div_up(rows, 256), div_up(4 * 152, tiles)));
  int rpc = div_up(div_up(rows, chunks), 32) * 32;
  chunks = div_up(rows, rpc);
  dim3 grid(div_up(la, 32), div_up(lb, 32), chunks);
  gemm_tn_kernel<TA, TB><<<grid, 256, 0, st>>>(rows, la, lb, rpc, alpha, A, lda, B, ldb, C, ldc);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// ---- FP32 operands: double-float accumulation (gemm_tn) ----
// (s, c) += a * b with the exact product p + e (p = fl(a b), e = fma(a, b, -p))
// and TwoSum of s and p (Knuth); the explicit _rn intrinsics keep the compiler
// from fusing the product into the sum.
__device__ __forceinline__ void dfloat_acc(float a, float b, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bv = __fsub_rn(t, s);
  const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  s = t;
  c = __fadd_rn(c, __fadd_rn(er, e));
}

constexpr int kGT = 64;   // output tile (kGT x kGT) of the FP32 Gram kernel
constexpr int kGR = 32;   // rows per shared-memory stage

// C (la x lb) += alpha A^T B over one chunk of rows (grid.z); 256 threads, 4 x 4
// outputs each; sym: A == B, tiles below the diagonal skipped.
__global__ void __launch_bounds__(256) gemm_tn_f32_kernel(int rows, int la, int lb, int rows_per_chunk,
                                                          double alpha, const float* __restrict__ A, int lda,
                                                          const float* __restrict__ B, int ldb, double* C,
                                                          int ldc, int sym) {
  __shared__ __align__(16) float As[kGR][kGT];
  __shared__ __align__(16) float Bs[kGR][kGT];
  const int i0 = blockIdx.x * kGT, j0 = blockIdx.y * kGT;
  if (sym && j0 + kGT <= i0) return;
  const int r_begin = blockIdx.z * rows_per_chunk;
  const int r_end = min(rows, r_begin + rows_per_chunk);
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.f;
  for (int r0 = r_begin; r0 < r_end; r0 += kGR) {
    for (int e = threadIdx.x; e < kGR * kGT; e += 256) {
      const int rr = e % kGR, cc = e / kGR;
      const int r = r0 + rr;
      As[rr][cc] = (r < r_end && i0 + cc < la) ? A[(size_t)(i0 + cc) * lda + r] : 0.f;
      Bs[rr][cc] = (r < r_end && j0 + cc < lb) ? B[(size_t)(j0 + cc) * ldb + r] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kGR; ++rr) {
      const float4 av = *reinterpret_cast<const float4*>(&As[rr][ti * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[rr][tj * 4]);
      const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dfloat_acc(a4[a], b4[b], sh[a][b], sl[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ti * 4 + a, j = j0 + tj * 4 + b;
      if (i < la && j < lb && (!sym || j >= i))
        atomicAdd(&C[(size_t)j * ldc + i], alpha * ((double)sh[a][b] + (double)sl[a][b]));
    }
}

// lower triangle <- upper triangle
__global__ void mirror_upper_kernel(int l, double* C, int ldc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * l) {
    const int i = idx % l, j = idx / l;
    if (i > j) C[(size_t)j * ldc + i] = C[(size_t)i * ldc + j];
  }
}

template <>
int gemm_tn<float, float>(int rows, int la, int lb, double alpha, const float* A, int lda, const float* B,
                          int ldb, double beta, double* C, int ldc, cudaStream_t st) {
  if (la <= 0 || lb <= 0) return SC4DVAR_OK;
  scale_matrix_kernel<<<div_up(la * lb, 256), 256, 0, st>>>(la, lb, beta, C, ldc);
  SC4_LAUNCH_CHECK();
  if (rows <= 0) return SC4DVAR_OK;
  const int sym = (A == B && la == lb && lda == ldb && beta == 0.0) ? 1 : 0;
  const int ta = div_up(la, kGT), tb = div_up(lb, kGT);
  const int tiles = sym ? ta * (ta + 1) / 2 : ta * tb;
  int chunks = max(1, min(div_up(rows, 256), div_up(4 * 152, tiles)));
  int rpc = div_up(div_up(rows, chunks), kGR) * kGR;
  chunks = div_up(rows, rpc);
  gemm_tn_f32_kernel<<<dim3(ta, tb, chunks), 256, 0, st>>>(rows, la, lb, rpc, alpha, A, lda, B, ldb, C, ldc,
                                                           sym);
  SC4_LAUNCH_CHECK();
  if (sym) {
    mirror_upper_kernel<<<div_up(la * la, 256), 256, 0, st>>>(la, C, ldc);
    SC4_LAUNCH_CHECK();
  }
  return SC4DVAR_OK;
}

// ---- FP32 operands: FP32 accumulation (gemm_nn) ----
// C (rows x c) = alpha A op(B) + beta C; tile 128 rows x 64 columns per CTA,
// 256 threads with 8 x 4 outputs each, k in stages of 32.
template <typename TC>
__global__ void __launch_bounds__(256) gemm_nn_f32_kernel(int rows, int kk, int c, float alpha,
                                                          const float* __restrict__ A, int lda,
                                                          const double* __restrict__ B, int ldb, int transB,
                                                          double beta, TC* __restrict__ C, int ldc) {
  __shared__ __align__(16) float As[32][128];  // [k][row]
  __shared__ __align__(16) float Bs[32][64];   // [k][col]
  const int r0 = blockIdx.x * 128, c0 = blockIdx.y * 64;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;  // 16 row groups of 8, 16 column groups of 4
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < kk; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * 128; e += 256) {
      const int rr = e & 127, kc = e >> 7;
      const int r = r0 + rr, k = k0 + kc;
      As[kc][rr] = (r < rows && k < kk) ? A[(size_t)k * lda + r] : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int kc = e & 31, cc = e >> 5;
      const int k = k0 + kc, j = c0 + cc;
      float v = 0.f;
      if (k < kk && j < c) v = (float)(transB ? B[(size_t)k * ldb + j] : B[(size_t)j * ldb + k]);
      Bs[kc][cc] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kc = 0; kc < 32; ++kc) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kc][tr * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kc][tr * 8 + 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[kc][tc * 4]);
      const float a8[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(a8[a], b4[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = c0 + tc * 4 + b;
    if (j >= c) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int r = r0 + tr * 8 + a;
      if (r < rows) {
        TC* p = &C[(size_t)j * ldc + r];
        double v = (double)(alpha * acc[a][b]);
        if (beta != 0.0) v += beta * (double)*p;
        *p = (TC)v;
      }
    }
  }
}

// ------------------------------------------------------------------ gemm_nn
// C = alpha * A * op(B) + beta * C; op(B) = B (kk x c) or B^T (B stored c x kk).
template <typename TA, typename TC>
__global__ void __launch_bounds__(256) gemm_nn_kernel(int rows, int kk, int c, double alpha,
                                                      const TA* __restrict__ A, int lda,
                                                      const double* __restrict__ B, int ldb,
                                                      int transB, double beta, TC* __restrict__ C,
                                                      int ldc) {
  __shared__ double As[32][65];  // [k][row]
  __shared__ double Bs[32][33];  // [k][col]
  int r0 = blockIdx.x * 64, c0 = blockIdx.y * 32;
  int tc = threadIdx.x & 31, tr = threadIdx.x >> 5;  // 8 row groups of 8 rows
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int k0 = 0; k0 < kk; k0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int rr = e & 63, kc = e >> 6;
      int r = r0 + rr, k = k0 + kc;
      As[kc][rr] = (r < rows && k < kk) ? (double)A[(size_t)k * lda + r] : 0.0;
    }
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      int kc = e & 31, cc = e >> 5;
      int k = k0 + kc, j = c0 + cc;
      double v = 0.0;
      if (k < kk && j < c) v = transB ? B[(size_t)k * ldb + j] : B[(size_t)j * ldb + k];
      Bs[kc][cc] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kc = 0; kc < 32; ++kc) {
      double b = Bs[kc][tc];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(As[kc][tr * 8 + q], b, acc[q]);
    }
    __syncthreads();
  }
  int j = c0 + tc;
  if (j < c) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int r = r0 + tr * 8 + q;
      if (r < rows) {
        TC* p = &C[(size_t)j * ldc + r];
        double v = alpha * acc[q];
        if (beta != 0.0) v += beta * (double)*p;
        *p = (TC)v;
      }
    }
  }
}

template <typename TA, typename TC>
int gemm_nn(int rows, int kk, int c, double alpha, const TA* A, int lda, const double* B, int ldb,
            int transB, double beta, TC* C, int ldc, cudaStream_t st) {
  if (rows <= 0 || c <= 0) return SC4DVAR_OK;
  if constexpr (sizeof(TA) == 4) {
    if (c > 1) {  // single-vector products keep FP64 accumulation (Remark 1 applies inside PCG)
      gemm_nn_f32_kernel<TC><<<dim3(div_up(rows, 128), div_up(c, 64)), 256, 0, st>>>(
          rows, kk, c, (float)alpha, A, lda, B, ldb, transB, beta, C, ldc);
      SC4_LAUNCH_CHECK();
      return SC4DVAR_OK;
    }
  }
  dim3 grid(div_up(rows, 64), div_up(c, 32));
  gemm_nn_kernel<TA, TC><<<grid, 256, 0, st>>>(rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C,
                                              ldc);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// ------------------------------------------------------------------ Cholesky
// In place, lower: A = L L^T (upper part untouched). info[0] = 0 or j+1 of the
// first non-positive pivot (then L is incomplete).
__global__ void chol_kernel(int l, double* A, int lda, int* info) {
  __shared__ double red[32];
  __shared__ double piv;
  for (int j = 0; j < l; ++j) {
    double s = 0.0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) {
      double v = A[(size_t)k * lda + j];
      s = fma(v, v, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
      double d = A[(size_t)j * lda + j] - s;
      piv = (d > 0.0 && isfinite(d)) ? sqrt(d) : -1.0;
      if (piv > 0) A[(size_t)j * lda + j] = piv;
    }
    __syncthreads();
    if (piv <= 0.0) {
      if (threadIdx.x == 0) info[0] = j + 1;
      return;
    }
    double inv = 1.0 / piv;
    for (int i = j + 1 + threadIdx.x; i < l; i += blockDim.x) {
      double t = A[(size_t)j * lda + i];
      for (int k = 0; k < j; ++k) t = fma(-A[(size_t)k * lda + i], A[(size_t)k * lda + j], t);
      A[(size_t)j * lda + i] = t * inv;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) info[0] = 0;
}

// Linv = L^{-1} (lower), one thread per column; zero above the diagonal. Diagonal
// entries below tiny * max|diag| are treated as zero (their rows of the inverse
// are set to zero: the pseudo-inverse reading used for R_M^dagger of Alg. 3).
__global__ void trtri_lower_kernel(int l, const double* L, int ldl, double* X, int ldx, double tiny) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) mx = fmax(mx, fabs(L[(size_t)i * ldl + i]));
  mx = block_max(mx, red);
  double thr = tiny * mx;
  for (int c = threadIdx.x; c < l; c += blockDim.x) {
    double* x = X + (size_t)c * ldx;
    for (int i = 0; i < c; ++i) x[i] = 0.0;
    for (int i = c; i < l; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) t = fma(-L[(size_t)k * ldl + i], x[k], t);
      double d = L[(size_t)i * ldl + i];
      x[i] = (fabs(d) > thr) ? t / d : 0.0;
    }
  }
}

// ------------------------------------------------------------------ Jacobi
// Cyclic two-sided Jacobi for a symmetric l x l matrix in parallel order: a
// sweep has m - 1 rounds (m = l rounded up to even); in round r the m/2
// disjoint pairs are (m-1, r) and ((r+i) mod (m-1), (r-i) mod (m-1)),
// i = 1..m/2-1 (a pair with an index >= l is a padding no-op). One launch per
// round updates the whole matrix: the rotation of pair i zeroes A[p,q] of the
// current matrix, and the 2 x 2 block of rows (p_i, q_i) and columns (p_j, q_j)
// becomes R_i^T A R_j, so every thread transforms its own block(s) reading the
// previous buffer and writing the next (A is double-buffered; each CTA
// recomputes the rotations it needs from the previous buffer). V <- V R is
// updated in place (disjoint column pairs). The off-diagonal mass is checked
// once per sweep.
__device__ __forceinline__ void jacobi_pair(int i, int r, int m, int& p, int& q) {
  if (i == 0) {
    p = m - 1;
    q = r;
  } else {
    p = (r + i) % (m - 1);
    q = (r - i + (m - 1)) % (m - 1);
  }
  if (p > q) {
    int t = p;
    p = q;
    q = t;
  }
}

// Rotation (c, s) that zeroes A[p, q] (c = 1, s = 0 for padding or a zero entry).
__device__ __forceinline__ void jacobi_rot(const double* A, int lda, int l, int p, int q, double& c,
                                           double& s) {
  c = 1.0;
  s = 0.0;
  if (q >= l) return;
  const double apq = A[(size_t)q * lda + p];
  if (apq == 0.0 || fabs(apq) <= 1e-300) return;
  const double app = A[(size_t)p * lda + p], aqq = A[(size_t)q * lda + q];
  const double th = (aqq - app) / (2.0 * apq);
  const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

constexpr int kJT = 16;  // pair tile per CTA side

// blockIdx.z = 0: 2 x 2 blocks of A (tile of kJT x kJT pair blocks);
// blockIdx.z = 1: rows of V (kJT pairs x kJT rows per CTA).
__global__ void __launch_bounds__(kJT * kJT) jacobi_round_kernel(int l, int m, int r, const double* __restrict__ Ain,
                                                                 double* __restrict__ Aout, int lda, double* V,
                                                                 int ldv) {
  __shared__ double rc[2][kJT], rs[2][kJT];
  __shared__ int rp[2][kJT], rq[2][kJT];
  const int np = m / 2;
  const int tx = threadIdx.x % kJT, ty = threadIdx.x / kJT;
  if (blockIdx.z == 0) {
    const int bi0 = blockIdx.y * kJT, bj0 = blockIdx.x * kJT;
    if (bi0 >= np || bj0 >= np) return;
    if (threadIdx.x < 2 * kJT) {
      const int side = threadIdx.x / kJT, t = threadIdx.x % kJT;
      const int pi = (side == 0 ? bi0 : bj0) + t;
      int p = 0, q = 0;
      double c = 1.0, sn = 0.0;
      if (pi < np) {
        jacobi_pair(pi, r, m, p, q);
        jacobi_rot(Ain, lda, l, p, q, c, sn);
      }
      rp[side][t] = p; rq[side][t] = q; rc[side][t] = c; rs[side][t] = sn;
    }
    __syncthreads();
    const int bi = bi0 + ty, bj = bj0 + tx;
    if (bi >= np || bj >= np) return;
    const int p = rp[0][ty], q = rq[0][ty], p2 = rp[1][tx], q2 = rq[1][tx];
    const double c1 = rc[0][ty], s1 = rs[0][ty], c2 = rc[1][tx], s2 = rs[1][tx];
    const bool hq = q < l, hq2 = q2 < l;
    const double a = Ain[(size_t)p2 * lda + p];
    const double b = hq2 ? Ain[(size_t)q2 * lda + p] : 0.0;
    const double d = hq ? Ain[(size_t)p2 * lda + q] : 0.0;
    const double e = (hq && hq2) ? Ain[(size_t)q2 * lda + q] : 0.0;
    // rows: (p, q) <- (c1 p - s1 q, s1 p + c1 q); then columns likewise with (c2, s2)
    const double ra = c1 * a - s1 * d, rb = c1 * b - s1 * e;
    const double rd = s1 * a + c1 * d, re = s1 * b + c1 * e;
    Aout[(size_t)p2 * lda + p] = c2 * ra - s2 * rb;
    if (hq2) Aout[(size_t)q2 * lda + p] = s2 * ra + c2 * rb;
    if (hq) Aout[(size_t)p2 * lda + q] = c2 * rd - s2 * re;
    if (hq && hq2) Aout[(size_t)q2 * lda + q] = s2 * rd + c2 * re;
  } else {
    const int bj0 = blockIdx.x * kJT, row0 = blockIdx.y * kJT;
    if (bj0 >= np || row0 >= l) return;
    if (threadIdx.x < kJT) {
      const int pi = bj0 + threadIdx.x;
      int p = 0, q = 0;
      double c = 1.0, sn = 0.0;
      if (pi < np) {
        jacobi_pair(pi, r, m, p, q);
        jacobi_rot(Ain, lda, l, p, q, c, sn);
      }
      rp[0][threadIdx.x] = p; rq[0][threadIdx.x] = q; rc[0][threadIdx.x] = c; rs[0][threadIdx.x] = sn;
    }
    __syncthreads();
    const int pj = bj0 + tx, row = row0 + ty;
    if (pj >= np || row >= l) return;
    const int p = rp[0][tx], q = rq[0][tx];
    const double c = rc[0][tx], sn = rs[0][tx];
    if (q >= l || sn == 0.0) return;
    const double vp = V[(size_t)p * ldv + row], vq = V[(size_t)q * ldv + row];
    V[(size_t)p * ldv + row] = c * vp - sn * vq;
    V[(size_t)q * ldv + row] = sn * vp + c * vq;
  }
}

__global__ void jacobi_init_kernel(int l, const double* A, int lda, double* A0, double* V, int ldv) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)l * l;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % l), j = (int)(e / l);
    A0[(size_t)j * l + i] = A[(size_t)j * lda + i];
    V[(size_t)j * ldv + i] = (i == j) ? 1.0 : 0.0;
  }
}

// out[0] = sum of squared off-diagonal entries, out[1] = sum of squared diagonal entries
__global__ void jacobi_offnorm_kernel(int l, const double* A, double* out) {
  __shared__ double red[32];
  double off = 0.0, dia = 0.0;
  for (size_t e = threadIdx.x; e < (size_t)l * l; e += blockDim.x) {
    const int i = (int)(e % l), j = (int)(e / l);
    const double a = A[e];
    if (i == j) dia = fma(a, a, dia);
    else off = fma(a, a, off);
  }
  off = block_sum(off, red);
  __syncthreads();
  dia = block_sum(dia, red);
  if (threadIdx.x == 0) {
    out[0] = off;
    out[1] = dia;
  }
}

__global__ void jacobi_diag_kernel(int l, const double* A, double* w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < l; i += gridDim.x * blockDim.x)
    w[i] = A[(size_t)i * l + i];
}

// Descending order: perm[rank] = i (ties broken by index); w_out, V_out permuted.
__global__ void sort_desc_kernel(int l, const double* w, const double* V, int ldv, double* w_out,
                                 double* V_out, int ldo) {
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    double wi = w[i];
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      double wj = w[j];
      rank += (wj > wi) || (wj == wi && j < i);
    }
    w_out[rank] = wi;
    for (int r = 0; r < l; ++r) V_out[(size_t)rank * ldo + r] = V[(size_t)i * ldv + r];
  }
}

// Largest eigenvalue of a symmetric PSD l x l matrix by power iteration (used
// only for the Nystrom shift nu = sqrt(n) eps |Y|_2).
__global__ void power_lmax_kernel(int l, const double* G, int ldg, int iters, double* out) {
  extern __shared__ double pv[];
  __shared__ double red[32];
  double* x = pv;
  double* y = pv + l;
  for (int i = threadIdx.x; i < l; i += blockDim.x) x[i] = 1.0 + 0.01 * (double)(i % 7);
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < l; ++j) s = fma(G[(size_t)j * ldg + i], x[j], s);
      y[i] = s;
    }
    __syncthreads();
    double nn = 0.0, xy = 0.0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
      nn = fma(y[i], y[i], nn);
      xy = fma(x[i], y[i], xy);
    }
    nn = block_sum(nn, red);
    xy = block_sum(xy, red);
    double xx = 0.0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) xx = fma(x[i], x[i], xx);
    xx = block_sum(xx, red);
    lam = (xx > 0) ? xy / xx : 0.0;
    double inv = (nn > 0) ? 1.0 / sqrt(nn) : 0.0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) x[i] = y[i] * inv;
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = lam;
}

int chol_lower(int l, double* A, int lda, int* info_dev, cudaStream_t st) {
  chol_kernel<<<1, 512, 0, st>>>(l, A, lda, info_dev);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int trtri_lower(int l, const double* L, int ldl, double* X, int ldx, double tiny, cudaStream_t st) {
  trtri_lower_kernel<<<1, 512, 0, st>>>(l, L, ldl, X, ldx, tiny);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

size_t jacobi_work_bytes(int l) { return ((size_t)2 * l * l + 8) * sizeof(double); }

int jacobi_eig(int l, const double* A, int lda, double* V, int ldv, double* w, int max_sweeps, double tol,
               void* work, int* sweeps_out, cudaStream_t st) {
  if (l <= 0) return SC4DVAR_OK;
  const int m = (l + 1) & ~1, np = m / 2;
  double* buf[2] = {reinterpret_cast<double*>(work), reinterpret_cast<double*>(work) + (size_t)l * l};
  double* red = buf[1] + (size_t)l * l;
  const int nb = (np + kJT - 1) / kJT, nr = (l + kJT - 1) / kJT;
  const dim3 grid(nb, std::max(nb, nr), 2);
  jacobi_init_kernel<<<std::min(8 * 152, (int)(((size_t)l * l + 255) / 256)), 256, 0, st>>>(l, A, lda, buf[0],
                                                                                           V, ldv);
  SC4_LAUNCH_CHECK();
  int cur = 0, sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    jacobi_offnorm_kernel<<<1, 1024, 0, st>>>(l, buf[cur], red);
    SC4_LAUNCH_CHECK();
    double h[2];
    SC4_CUDA(cudaMemcpyAsync(h, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SC4_CUDA(cudaStreamSynchronize(st));
    if (h[0] <= tol * tol * h[1] || h[0] == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      jacobi_round_kernel<<<grid, kJT * kJT, 0, st>>>(l, m, r, buf[cur], buf[cur ^ 1], l, V, ldv);
      SC4_LAUNCH_CHECK();
      cur ^= 1;
    }
  }
  jacobi_diag_kernel<<<(l + 255) / 256, 256, 0, st>>>(l, buf[cur], w);
  SC4_LAUNCH_CHECK();
  if (sweeps_out) *sweeps_out = sweep;
  return SC4DVAR_OK;
}

int sort_desc(int l, const double* w, const double* V, int ldv, double* w_out, double* V_out,
              int ldo, cudaStream_t st) {
  sort_desc_kernel<<<1, 256, 0, st>>>(l, w, V, ldv, w_out, V_out, ldo);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int power_lmax(int l, const double* G, int ldg, double* out_dev, cudaStream_t st) {
  power_lmax_kernel<<<1, 256, 2 * l * sizeof(double), st>>>(l, G, ldg, 200, out_dev);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// ------------------------------------------------------------------ vectors
// partial sums per block, then one block finishes (deterministic order).
template <int OP, typename TX, typename TY>
__global__ void reduce_partial_kernel(size_t n, const TX* __restrict__ x, const TY* __restrict__ y,
                                      double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double a = (double)x[i];
    if (OP == 0) s = fma(a, (double)y[i], s);   // dot
    else if (OP == 1) s = fma(a, a, s);         // sum of squares
    else s = fmax(s, fabs(a));                  // max |x|
  }
  if (OP == 2) s = block_max(s, red);
  else s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <int OP>
__global__ void reduce_final_kernel(int nb, const double* part, double* out, int sqrt_out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s = (OP == 2) ? fmax(s, part[i]) : s + part[i];
  s = (OP == 2) ? block_max(s, red) : block_sum(s, red);
  if (threadIdx.x == 0) *out = sqrt_out ? sqrt(s) : s;
}

static const int kRedBlocks = 304;

template <typename TX, typename TY>
int vdot(size_t n, const TX* x, const TY* y, double* out_dev, double* part, cudaStream_t st) {
  reduce_partial_kernel<0, TX, TY><<<kRedBlocks, 256, 0, st>>>(n, x, y, part);
  note_launch();
  reduce_final_kernel<0><<<1, 256, 0, st>>>(kRedBlocks, part, out_dev, 0);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template <typename TX>
int vnrm2(size_t n, const TX* x, double* out_dev, double* part, cudaStream_t st) {
  reduce_partial_kernel<1, TX, TX><<<kRedBlocks, 256, 0, st>>>(n, x, x, part);
  note_launch();
  reduce_final_kernel<1><<<1, 256, 0, st>>>(kRedBlocks, part, out_dev, 1);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int vamax(size_t n, const double* x, double* out_dev, double* part, cudaStream_t st) {
  reduce_partial_kernel<2, double, double><<<kRedBlocks, 256, 0, st>>>(n, x, x, part);
  note_launch();
  reduce_final_kernel<2><<<1, 256, 0, st>>>(kRedBlocks, part, out_dev, 0);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// y = a x + b y (a, b host scalars)
template <typename TX, typename TY>
__global__ void axpby_kernel(size_t n, double a, const TX* __restrict__ x, double b, TY* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = a * (double)x[i];
    if (b != 0.0) v += b * (double)y[i];
    y[i] = (TY)v;
  }
}

template <typename TX, typename TY>
int axpby(size_t n, double a, const TX* x, double b, TY* y, cudaStream_t st) {
  if (n == 0) return SC4DVAR_OK;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 4 * 152);
  axpby_kernel<TX, TY><<<blocks, 256, 0, st>>>(n, a, x, b, y);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// z = r - V (d .* (V^T r)) for k columns: Woodbury (Eq. woodbury) with
// d = lam / (1 + lam). T is an l x k workspace.
int woodbury_apply(int n, int l, int k, const double* V, int ldv, const double* dscale,
                   const double* R, int ldr, double* Z, int ldz, double* T, cudaStream_t st);

__global__ void scale_rows_kernel(int l, int k, const double* d, double* T, int ldt) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * k) {
    int i = idx % l, j = idx / l;
    T[(size_t)j * ldt + i] *= d[i];
  }
}

__global__ void copy_cols_kernel(int n, int k, const double* R, int ldr, double* Z, int ldz) {
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx < (size_t)n * k) {
    int i = (int)(idx % n), j = (int)(idx / n);
    Z[(size_t)j * ldz + i] = R[(size_t)j * ldr + i];
  }
}

int woodbury_apply(int n, int l, int k, const double* V, int ldv, const double* dscale,
                   const double* R, int ldr, double* Z, int ldz, double* T, cudaStream_t st) {
  if (R != Z || ldr != ldz) {
    copy_cols_kernel<<<(unsigned)div_up(n * k, 256), 256, 0, st>>>(n, k, R, ldr, Z, ldz);
    SC4_LAUNCH_CHECK();
  }
  if (l <= 0) return SC4DVAR_OK;
  SC4_TRY(gemm_tn<double, double>(n, l, k, 1.0, V, ldv, R, ldr, 0.0, T, l, st));
  scale_rows_kernel<<<div_up(l * k, 256), 256, 0, st>>>(l, k, dscale, T, l);
  SC4_LAUNCH_CHECK();
  SC4_TRY(gemm_nn<double, double>(n, l, k, -1.0, V, ldv, T, l, 0, 1.0, Z, ldz, st));
  return SC4DVAR_OK;
}

// ---- explicit instantiations ---------------------------------------------------
template int gemm_tn<double, double>(int, int, int, double, const double*, int, const double*, int,
                                     double, double*, int, cudaStream_t);
template int gemm_tn<double, float>(int, int, int, double, const double*, int, const float*, int,
                                    double, double*, int, cudaStream_t);
template int gemm_tn<float, double>(int, int, int, double, const float*, int, const double*, int,
                                    double, double*, int, cudaStream_t);
template int gemm_nn<double, double>(int, int, int, double, const double*, int, const double*, int,
                                     int, double, double*, int, cudaStream_t);
template int gemm_nn<float, float>(int, int, int, double, const float*, int, const double*, int,
                                   int, double, float*, int, cudaStream_t);
template int gemm_nn<float, double>(int, int, int, double, const float*, int, const double*, int,
                                    int, double, double*, int, cudaStream_t);
template int gemm_nn<double, float>(int, int, int, double, const double*, int, const double*, int,
                                    int, double, float*, int, cudaStream_t);
template int vdot<double, double>(size_t, const double*, const double*, double*, double*,
                                  cudaStream_t);
template int vnrm2<double>(size_t, const double*, double*, double*, cudaStream_t);
template int vnrm2<float>(size_t, const float*, double*, double*, cudaStream_t);
template int axpby<double, double>(size_t, double, const double*, double, double*, cudaStream_t);
template int axpby<double, float>(size_t, double, const double*, double, float*, cudaStream_t);
template int axpby<float, double>(size_t, double, const float*, double, double*, cudaStream_t);
template int axpby<float, float>(size_t, double, const float*, double, float*, cudaStream_t);

}  // namespace sc4
