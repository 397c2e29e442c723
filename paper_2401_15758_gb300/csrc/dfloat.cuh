// Double-float numbers: a value is the unevaluated sum hi + lo of two floats
// with |lo| <= ulp(hi) / 2, about 48 significant bits. Sums and products use
// the error-free transformations of Knuth (TwoSum) and of Dekker with a fused
// multiply-add (TwoProduct), so every operation runs on the FP32 pipe; on this
// GPU that pipe is 64 times faster than the FP64 one. Relative error per
// operation is a small multiple of 2^-48 (cancellation aside), far below what
// a defect-correction residual at the 1e-6 level needs.
#pragma once
#include <cuda_runtime.h>

namespace sc4 {

struct __align__(8) dfloat {
  float hi, lo;
  __host__ __device__ dfloat() : hi(0.f), lo(0.f) {}
  __host__ __device__ dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit dfloat(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfloat df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_norm(p, e);
}

__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// warp shuffles, read-only loads and shared-memory atomic accumulation of dfloats
__device__ __forceinline__ dfloat __shfl_up_sync(unsigned mask, dfloat v, unsigned d) {
  return dfloat(::__shfl_up_sync(mask, v.hi, d), ::__shfl_up_sync(mask, v.lo, d));
}
__device__ __forceinline__ dfloat __shfl_down_sync(unsigned mask, dfloat v, unsigned d) {
  return dfloat(::__shfl_down_sync(mask, v.hi, d), ::__shfl_down_sync(mask, v.lo, d));
}
__device__ __forceinline__ dfloat __ldg(const dfloat* p) {
  const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
  return dfloat(v.x, v.y);
}

// Atomic a += v by compare-and-swap of the 64-bit pair. Observation sites of one
// time are distinct in the workloads, so the first attempt succeeds; the loop
// is bounded all the same and falls back to a plain update.
__device__ __forceinline__ void atomicAdd(dfloat* a, dfloat v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  for (int tries = 0; tries < (1 << 16); ++tries) {
    dfloat cur = *reinterpret_cast<dfloat*>(&old);
    dfloat nw = cur + v;
    const unsigned long long want = *reinterpret_cast<unsigned long long*>(&nw);
    const unsigned long long seen = atomicCAS(p, old, want);
    if (seen == old) return;
    old = seen;
  }
  *a = *a + v;
}

}  // namespace sc4
