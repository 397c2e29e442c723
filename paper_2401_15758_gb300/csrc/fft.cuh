#pragma once
#include <cuda_runtime.h>

namespace sc4 {
int fft_make_twiddles(int n, double2* tw, cudaStream_t st);
int fft_se_symbol(int n, double sigma, double length, double clamp_rel, const double2* tw,
                  double* sym, cudaStream_t st);
// Y = Gamma^{1/2} X (+ Z), k columns of length n (power of two, 8..8192).
template <typename TI, typename TO, typename TZ>
int prior_apply(int n, int k, const TI* X, int ldx, TO* Y, int ldy, const TZ* Z, int ldz,
                const double* sym, const double2* tw, cudaStream_t st);
}  // namespace sc4
