#pragma once
#include <cuda_runtime.h>

namespace sc4 {
// Tensor-core modes of the sketches' tall products (see tall_tc.cu).
enum { kTall3xTF32 = 0, kTallSIMT = 1, kTallTF32 = 2, kTallBF16 = 3 };

// C (rows x c) = alpha A op(B) + beta C on the tensor cores; A FP32 column-major
// (rows x kk), B FP64 (kk x c, or c x kk with transB), C FP32 or FP64.
// pack: device workspace of tall_pack_bytes(mode, kk, c) bytes for the converted B.
size_t tall_pack_bytes(int mode, int kk, int c);
template <typename TC>
int tall_gemm_tc(int mode, int rows, int kk, int c, double alpha, const float* A, int lda, const double* B,
                 int ldb, int transB, double beta, TC* C, int ldc, void* pack, cudaStream_t st);
// The 128-point row transform out[r][:] = in[r][:] S of the double-gyre
// elliptic solves (rows r = c ny + j of back-to-back fields: row r at in + 128 r,
// its output at out + c ldo + 128 j), S a row-major 128 x 128 FP32 matrix packed
// once by rows128_pack into a device buffer of rows128_pack_bytes(); 3xTF32
// products on the tensor cores. in and out 16-byte aligned, ldo a multiple of 4.
size_t rows128_pack_bytes();
int rows128_pack(const float* S, void* out, cudaStream_t st);
int rows128_tc(int ny, int rows, const float* in, const void* Spk, float* out, int ldo, cudaStream_t st);
// SC4DVAR_ERR_TIMEOUT (and clears it) if a tensor-core wait gave up since the last
// call; synchronizes with the device.
int tall_tc_take_error();
}  // namespace sc4
