// Periodic prior square root Gamma^{1/2} applied through a hand-written FFT.
//
// Gamma is stationary on the periodic grid, so Gamma^{1/2} is circulant and acts
// as a real, even Fourier multiplier s_j (the first-level preconditioning of
// Eq. gniterf1 / pcgsystem: x0 = xb + Gamma^{1/2} v). Because s is real and
// even, the multiplier maps real columns to real columns, and two real columns
// x_a, x_b are transformed together as one complex column z = x_a + i x_b:
//   Gamma^{1/2} x_a = Re IFFT(s . FFT(z)),  Gamma^{1/2} x_b = Im IFFT(s . FFT(z)).
//
// The FFT is an in-place radix-2 decimation-in-time transform of length n (a power
// of two, n <= 8192) held in shared memory as double2, one CTA per column pair,
// with a per-problem twiddle table w_j = exp(-2 pi i j / n), j < n/2, in global
// memory. Everything is FP64: on GB300 the transforms cost little next to the
// model sweeps, and the same code serves the FP64 parity path.
#include "common.cuh"
#include "fft.cuh"

namespace sc4 {

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ inline unsigned bitrev(unsigned j, int logn) { return __brev(j) >> (32 - logn); }

// In-place decimation-in-time FFT of s[0..n): input in bit-reversed order, output
// in natural order. dir = -1 forward, +1 inverse (unscaled). All threads take part.
__device__ void fft_dit(double2* s, int n, const double2* __restrict__ tw, int dir) {
  for (int half = 1; half < n; half <<= 1) {
    int stride = n / (2 * half);  // twiddle index step
    __syncthreads();
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      int grp = b / half, k = b - grp * half;
      int i0 = grp * 2 * half + k, i1 = i0 + half;
      double2 w = __ldg(&tw[k * stride]);
      if (dir > 0) w.y = -w.y;
      double2 t = cmul(w, s[i1]);
      double2 u = s[i0];
      s[i0] = make_double2(u.x + t.x, u.y + t.y);
      s[i1] = make_double2(u.x - t.x, u.y - t.y);
    }
  }
  __syncthreads();
}

// In-place decimation-in-frequency FFT: input in natural order, output in
// bit-reversed order.
__device__ void fft_dif(double2* s, int n, const double2* __restrict__ tw, int dir) {
  for (int half = n / 2; half >= 1; half >>= 1) {
    int stride = n / (2 * half);
    __syncthreads();
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      int grp = b / half, k = b - grp * half;
      int i0 = grp * 2 * half + k, i1 = i0 + half;
      double2 w = __ldg(&tw[k * stride]);
      if (dir > 0) w.y = -w.y;
      double2 u = s[i0], v = s[i1];
      s[i0] = make_double2(u.x + v.x, u.y + v.y);
      s[i1] = cmul(w, make_double2(u.x - v.x, u.y - v.y));
    }
  }
  __syncthreads();
}

__global__ void twiddle_kernel(int n, double2* tw) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n / 2) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)n, &s, &c);
    tw[j] = make_double2(c, s);
  }
}

// Squared-exponential symbol: c_d = sigma^2 exp(-d^2/(2 L^2)), d the periodic
// distance in [0, 1/2]; lambda = Re FFT(c); lambda_j < CLAMP * max -> 0; s = sqrt.
__global__ void se_symbol_kernel(int n, int logn, double sigma, double length, double clamp_rel,
                                 const double2* __restrict__ tw, double* sym) {
  extern __shared__ double2 sm[];
  __shared__ double red[32];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int jj = min(j, n - j);
    double d = (double)jj / (double)n;
    double c = sigma * sigma * exp(-(d * d) / (2.0 * length * length));
    sm[bitrev(j, logn)] = make_double2(c, 0.0);
  }
  fft_dit(sm, n, tw, -1);
  double mx = -1e300;
  for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmax(mx, sm[j].x);
  mx = block_max(mx, red);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double l = sm[j].x;
    sym[j] = (l < clamp_rel * mx) ? 0.0 : sqrt(l);
  }
}

// Y[:, c] = Gamma^{1/2} X[:, c] (+ Z[:, c] when Z != nullptr), two columns per CTA.
template <typename TI, typename TO, typename TZ>
__global__ void prior_apply_kernel(int n, int logn, int k, const TI* __restrict__ X, int ldx,
                                   TO* __restrict__ Y, int ldy, const TZ* __restrict__ Z, int ldz,
                                   const double* __restrict__ sym, const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  int ca = 2 * blockIdx.x, cb = ca + 1;
  bool hasb = cb < k;
  const TI* xa = X + (size_t)ca * ldx;
  const TI* xb = X + (size_t)cb * ldx;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double a = (double)xa[j];
    double b = hasb ? (double)xb[j] : 0.0;
    sm[bitrev(j, logn)] = make_double2(a, b);
  }
  fft_dit(sm, n, tw, -1);
  double inv_n = 1.0 / (double)n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = sym[j] * inv_n;
    double2 v = sm[j];
    sm[j] = make_double2(v.x * s, v.y * s);
  }
  fft_dif(sm, n, tw, +1);
  TO* ya = Y + (size_t)ca * ldy;
  TO* yb = Y + (size_t)cb * ldy;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double2 v = sm[bitrev(j, logn)];
    double ra = v.x, rb = v.y;
    if (Z != nullptr) {
      ra += (double)Z[(size_t)ca * ldz + j];
      if (hasb) rb += (double)Z[(size_t)cb * ldz + j];
    }
    ya[j] = (TO)ra;
    if (hasb) yb[j] = (TO)rb;
  }
}

// ---- host side ---------------------------------------------------------------
static int fft_threads(int n) { return n >= 1024 ? 512 : (n >= 64 ? n / 2 : 32); }

int fft_make_twiddles(int n, double2* tw, cudaStream_t st) {
  twiddle_kernel<<<div_up(n / 2, 256), 256, 0, st>>>(n, tw);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int fft_se_symbol(int n, double sigma, double length, double clamp_rel, const double2* tw,
                  double* sym, cudaStream_t st) {
  int logn = 31 - __builtin_clz((unsigned)n);
  size_t smem = (size_t)n * sizeof(double2);
  SC4_CUDA(cudaFuncSetAttribute(se_symbol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  se_symbol_kernel<<<1, 1024, smem, st>>>(n, logn, sigma, length, clamp_rel, tw, sym);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template <typename TI, typename TO, typename TZ>
int prior_apply(int n, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz,
                const double* sym, const double2* tw, cudaStream_t st) {
  if (k <= 0) return SC4DVAR_OK;
  int logn = 31 - __builtin_clz((unsigned)n);
  size_t smem = (size_t)n * sizeof(double2);
  auto kern = prior_apply_kernel<TI, TO, TZ>;
  SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int th = fft_threads(n);
  kern<<<div_up(k, 2), th, smem, st>>>(n, logn, k, X, ldx, Y, ldy, Z, ldz, sym, tw);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

template int prior_apply<double, double, double>(int, int, const double*, int, double*, int,
                                                 const double*, int, const double*, const double2*,
                                                 cudaStream_t);
template int prior_apply<float, float, float>(int, int, const float*, int, float*, int,
                                              const float*, int, const double*, const double2*,
                                              cudaStream_t);
template int prior_apply<double, float, float>(int, int, const double*, int, float*, int,
                                               const float*, int, const double*, const double2*,
                                               cudaStream_t);
template int prior_apply<float, double, double>(int, int, const float*, int, double*, int,
                                                const double*, int, const double*, const double2*,
                                                cudaStream_t);

}  // namespace sc4
