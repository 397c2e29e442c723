#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace sc4 {
template <typename TA, typename TB>
int gemm_tn(int rows, int la, int lb, double alpha, const TA* A, int lda, const TB* B, int ldb,
            double beta, double* C, int ldc, cudaStream_t st);
template <typename TA, typename TC>
int gemm_nn(int rows, int kk, int c, double alpha, const TA* A, int lda, const double* B, int ldb,
            int transB, double beta, TC* C, int ldc, cudaStream_t st);
int chol_lower(int l, double* A, int lda, int* info_dev, cudaStream_t st);
int trtri_lower(int l, const double* L, int ldl, double* X, int ldx, double tiny, cudaStream_t st);
// Symmetric eigen-decomposition (FP64 Jacobi): A (l x l, not modified) = V diag(w) V^T,
// eigenvalues unsorted. work: jacobi_work_bytes(l) of device memory. Synchronizes
// the stream once per sweep (convergence test); sweeps_out (host, nullable).
size_t jacobi_work_bytes(int l);
int jacobi_eig(int l, const double* A, int lda, double* V, int ldv, double* w, int max_sweeps, double tol,
               void* work, int* sweeps_out, cudaStream_t st);
int sort_desc(int l, const double* w, const double* V, int ldv, double* w_out, double* V_out,
              int ldo, cudaStream_t st);
int power_lmax(int l, const double* G, int ldg, double* out_dev, cudaStream_t st);
template <typename TX, typename TY>
int vdot(size_t n, const TX* x, const TY* y, double* out_dev, double* part, cudaStream_t st);
template <typename TX>
int vnrm2(size_t n, const TX* x, double* out_dev, double* part, cudaStream_t st);
int vamax(size_t n, const double* x, double* out_dev, double* part, cudaStream_t st);
template <typename TX, typename TY>
int axpby(size_t n, double a, const TX* x, double b, TY* y, cudaStream_t st);
int woodbury_apply(int n, int l, int k, const double* V, int ldv, const double* dscale,
                   const double* R, int ldr, double* Z, int ldz, double* T, cudaStream_t st);
}  // namespace sc4
