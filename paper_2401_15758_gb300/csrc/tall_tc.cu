// Tall-skinny products of the sketches on the tensor cores (tcgen05, TMEM).
//
// C (rows x c) = alpha A op(B) + beta C, A (rows x kk) FP32 column-major, the
// small factor B FP64 (kk x c, or c x kk when transposed), C FP32 or FP64. These
// are the products with a tall sketch matrix and an l x l factor in the
// randomized preconditioners: Q = Y R^{-1} of CholeskyQR (Algs. 1, 3, 4 step 3),
// V = W^T U Sigma^{-1} of the thin SVD (Algs. 1-5), the Nystrom W = L^{-1} Y^T
// (Alg. 2 step 6), the Gram-Schmidt updates of the adaptive sketches (Algs. 4, 5)
// and the SingleView W = Z Q_M R_M^{-T} (Alg. 3 step 5).
//
// One CTA of four warps computes a 128-row x N-column tile (N <= 256, a multiple
// of 16) with tcgen05.mma.cta_group::1 (M = 128), the FP32 accumulator living in
// tensor memory (N, rounded up to a power of two, of the 512 TMEM columns of the
// SM). K runs in chunks of 16 through two shared-memory stages: while the tensor
// core multiplies one chunk (issued by one thread, completion signalled on an
// mbarrier by tcgen05.commit), the four warps load the next chunk of A into
// registers, then convert and stage it. The small factor is converted once per
// product by a packing kernel into the operand format of every stage, and each
// stage's B chunk arrives by a bulk copy of the tensor-memory-access engine. Operands sit in shared memory in
// the canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// adjacent in K at LBO = (tile rows / 8) x 128 bytes, adjacent in rows at
// SBO = 128 bytes. The epilogue reads the accumulator with tcgen05.ld (warp w
// owns TMEM lanes 32w .. 32w + 31 = tile rows) and writes C column by column,
// coalesced along the rows.
//
// Modes: TF32 (one product, ~1e-4 relative), BF16 (kind::f16 with BF16 inputs,
// ~1e-3), and 3xTF32 (a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi);
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, Ootomo & Yokota 2022), which gives
// FP32 accuracy (~1e-7 relative) on the tensor pipe and is the default for FP32
// sketches.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets a device error
// word (reported as SC4DVAR_ERR_TIMEOUT by the next synchronizing call), waits a
// bounded time for the products already issued, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include "common.cuh"
#include "dense.cuh"
#include "tall_tc.cuh"

namespace sc4 {
namespace {

__device__ int g_tall_err = 0;

constexpr int kKC = 16;          // K per staged chunk
constexpr int kNmax = 256;       // columns per CTA tile
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: no swizzle, K-major, version field 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: FP32 accumulator, A and B of format fmt (TF32 = 2 for
// kind::tf32, BF16 = 1 for kind::f16), both K-major, M x N.
__device__ __forceinline__ uint32_t instr_desc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

template <int MODE>
struct TallMode {
  static constexpr int E = (MODE == kTallBF16) ? 2 : 4;     // operand bytes
  static constexpr int T = 16 / E;                          // elements per core-matrix row
  static constexpr int KI = 32 / E;                         // K per instruction
  static constexpr int NSPLIT = (MODE == kTall3xTF32) ? 2 : 1;
  static constexpr int kABytes = (kKC / T) * 16 * 128;      // one 128-row operand chunk
  static constexpr int kAStage = NSPLIT * kABytes;
  // B chunk of an N-row operand: (kKC / T) * (N / 8) * 128 bytes per split
  __host__ __device__ static int b_bytes(int N) { return (kKC / T) * (N / 8) * 128; }
  __host__ __device__ static int stage_bytes(int N) { return NSPLIT * (kABytes + b_bytes(N)); }
  __host__ __device__ static int smem_bytes(int N) { return 2 * stage_bytes(N) + 64; }
};

// Writes T consecutive K values of one row (already zero-padded) in the operand
// format: hi (and lo) parts for TF32 modes, BF16 otherwise.
template <int MODE>
__device__ __forceinline__ void put_row(unsigned char* dst, int split_bytes, const float* v) {
  if constexpr (MODE == kTallBF16) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(h);
  } else {
    float hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      hi[i] = tf32_rna(v[i]);
      lo[i] = tf32_rna(v[i] - hi[i]);
    }
    *reinterpret_cast<float4*>(dst) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    if constexpr (MODE == kTall3xTF32)
      *reinterpret_cast<float4*>(dst + split_bytes) = make_float4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// The small factor converted once into the operand format, chunk by chunk, for
// every column tile: block (y, ch) holds NSPLIT x b_bytes(Nt_y) bytes laid out
// exactly as a stage's B region, so a CTA fetches it with one bulk copy.
template <int MODE, typename TB>
__global__ void tall_pack_b_kernel(int kk, int c, const TB* __restrict__ B, int ldb, int transB, int ntl,
                                   int nch, unsigned char* __restrict__ out) {
  using Md = TallMode<MODE>;
  constexpr int T = Md::T;
  const int y = blockIdx.y, ch = blockIdx.x;
  const int c0 = y * kNmax, Nt = min(ntl, (c - c0 + 15) / 16 * 16);
  const int bB = Md::b_bytes(Nt);
  unsigned char* dst = out + ((size_t)y * nch + ch) * Md::NSPLIT * Md::b_bytes(ntl);
  const int k0 = ch * kKC;
  for (int e = threadIdx.x; e < Nt * (kKC / T); e += blockDim.x) {
    const int n = e % Nt, q = e / Nt, j = c0 + n;
    float v[8];
#pragma unroll
    for (int i = 0; i < T; ++i) {
      const int k = k0 + q * T + i;
      v[i] = (j < c && k < kk) ? (float)(transB ? B[(size_t)k * ldb + j] : B[(size_t)j * ldb + k]) : 0.f;
    }
    put_row<MODE>(dst + (q * (Nt / 8) + (n >> 3)) * 128 + (n & 7) * 16, bB, v);
  }
}

// One CTA: rows r0 .. r0 + 127 and columns c0 .. c0 + Nt - 1 (Nt <= ntl, the
// widest tile of the launch, which sizes the shared stages; tcols TMEM columns).
// Thread t stages row t of A (the next chunk's values are loaded into registers
// while the tensor core multiplies); thread 0 brings the chunk of the packed B
// operand with a bulk copy (cp.async.bulk) that completes the stage's B barrier.
template <int MODE, typename TC>
__global__ void __launch_bounds__(128) tall_tc_kernel(int rows, int kk, int c, float alpha,
                                                      const float* __restrict__ A, int lda,
                                                      const unsigned char* __restrict__ Bpk, double beta,
                                                      TC* __restrict__ C, int ldc, int ntl, int tcols) {
  using Md = TallMode<MODE>;
  constexpr int T = Md::T;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.x * 128, c0 = blockIdx.y * kNmax;
  const int Nt = min(ntl, (c - c0 + 15) / 16 * 16);
  const int bB = Md::b_bytes(Nt);
  const int stage = Md::stage_bytes(ntl);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * stage);  // [0, 1] products done, [2, 3] B landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < 4; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar + b)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(MODE == kTallBF16 ? 1 : 2, 128, Nt);
  const int nch = (kk + kKC - 1) / kKC;
  const int gr = r0 + tid;
  const unsigned char* bsrc = Bpk + (size_t)blockIdx.y * nch * Md::NSPLIT * Md::b_bytes(ntl);
  const uint32_t bbytes = Md::NSPLIT * bB;
  float va[kKC];
  auto load = [&](int ch) {
    const int k0 = ch * kKC;
#pragma unroll
    for (int k = 0; k < kKC; ++k)
      va[k] = (gr < rows && k0 + k < kk) ? A[(size_t)(k0 + k) * lda + gr] : 0.f;
  };
  bool ok = true;
  int issued = -1;  // last chunk whose products were committed
  if (nch > 0) load(0);
  for (int ch = 0; ch < nch; ++ch) {
    const int s = ch & 1;
    if (ch >= 2) {
      // every thread waits for the products that read this stage two chunks ago;
      // the verdict is made uniform before anyone leaves the loop
      const bool w = mbar_wait(saddr(bar + s), ((ch - 2) >> 1) & 1);
      if (!__syncthreads_and(w)) {
        ok = false;
        break;
      }
    }
    unsigned char* As = smem + s * stage;
    unsigned char* Bs = As + Md::kAStage;
    if (tid == 0) {
      // the packed B chunk by a bulk copy (TMA) completing the stage's B barrier
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar + 2 + s)),
                   "r"(bbytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              saddr(Bs)),
          "l"(bsrc + (size_t)ch * Md::NSPLIT * Md::b_bytes(ntl)), "r"(bbytes), "r"(saddr(bar + 2 + s))
          : "memory");
    }
#pragma unroll
    for (int q = 0; q < kKC / T; ++q)
      put_row<MODE>(As + (q * 16 + (tid >> 3)) * 128 + (tid & 7) * 16, Md::kABytes, va + q * T);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && !mbar_wait(saddr(bar + 2 + s), (ch >> 1) & 1)) atomicExch(&g_tall_err, 1);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = saddr(As), b0 = saddr(Bs);
      const uint32_t a_lbo = 16 * 128, b_lbo = (Nt / 8) * 128;
#pragma unroll
      for (int ki = 0; ki < kKC / Md::KI; ++ki) {
        const int q = ki * (Md::KI / T);
        constexpr int nterm = (MODE == kTall3xTF32) ? 3 : 1;
#pragma unroll
        for (int tm = 0; tm < nterm; ++tm) {
          const int sa = (tm == 2) ? 1 : 0, sb = (tm == 1) ? 1 : 0;  // hi hi, hi lo, lo hi
          const uint64_t ad = smem_desc(a0 + sa * Md::kABytes + q * 16 * 128, a_lbo, 128);
          const uint64_t bd = smem_desc(b0 + sb * bB + q * (Nt / 8) * 128, b_lbo, 128);
          const uint32_t acc = (ch > 0 || ki > 0 || tm > 0) ? 1u : 0u;
          if constexpr (MODE == kTallBF16) {
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          } else {
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       saddr(bar + s))
                   : "memory");
    }
    issued = ch;
    if (ch + 1 < nch) load(ch + 1);
  }
  // the last commit covers every product issued before it
  if (issued >= 0) {
    const bool w = mbar_wait(saddr(bar + (issued & 1)), (issued >> 1) & 1);
    ok = __syncthreads_and(w && ok);
  }
  if (!ok && tid == 0) atomicExch(&g_tall_err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && issued >= 0) {
    const int row = r0 + warp * 32 + lane;
    for (int cb = 0; cb < Nt; cb += 8) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                     "=r"(v[7])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < rows) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = c0 + cb + i;
          if (j < c) {
            TC* p = &C[(size_t)j * ldc + row];
            double y = (double)(alpha * __uint_as_float(v[i]));
            if (beta != 0.0) y += beta * (double)*p;
            *p = (TC)y;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

template <int MODE>
size_t pack_bytes(int kk, int c) {
  const int ntl = std::min(kNmax, (c + 15) / 16 * 16);
  const size_t nch = (size_t)(kk + kKC - 1) / kKC, ny = (size_t)(c + kNmax - 1) / kNmax;
  return ny * nch * TallMode<MODE>::NSPLIT * TallMode<MODE>::b_bytes(ntl);
}

template <int MODE, typename TC>
int launch_tall(int rows, int kk, int c, double alpha, const float* A, int lda, const double* B, int ldb,
                int transB, double beta, TC* C, int ldc, void* pack, cudaStream_t st) {
  const int ntl = std::min(kNmax, (c + 15) / 16 * 16);
  const int nch = (kk + kKC - 1) / kKC;
  int tcols = 32;
  while (tcols < ntl) tcols *= 2;
  dim3 pgrid(nch, div_up(c, kNmax));
  tall_pack_b_kernel<MODE, double><<<pgrid, 256, 0, st>>>(kk, c, B, ldb, transB, ntl, nch,
                                                         static_cast<unsigned char*>(pack));
  SC4_LAUNCH_CHECK();
  const int smem = TallMode<MODE>::smem_bytes(ntl);
  auto kern = tall_tc_kernel<MODE, TC>;
  SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  dim3 grid(div_up(rows, 128), div_up(c, kNmax));
  kern<<<grid, 128, smem, st>>>(rows, kk, c, (float)alpha, A, lda, static_cast<const unsigned char*>(pack), beta,
                                C, ldc, ntl, tcols);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

// ---------------------------------------------------------------- 128-point row transform
// out[r][p] = sum_i in[r][i] S[i][p] for rows r = c ny + j of k fields (row r at
// in + c ldi + j 128), S a fixed 128 x 128 FP32 matrix packed once
// (tall_pack_factor) in the staged operand format of all eight 16-wide K chunks
// (128 KB for the 3xTF32 split). A persistent CTA keeps the whole packed S in
// shared memory (one bulk copy at start) and walks 128-row tiles: per tile,
// eight K chunks of the rows go through two shared stages, each followed by six
// tcgen05 MMAs (two K steps of 8, three TF32 products each) into a 128-column
// TMEM accumulator; the epilogue writes every row's 128 outputs with vector stores.
constexpr int kRowN = 128;
constexpr int kRowChunks = kRowN / kKC;

__global__ void __launch_bounds__(128, 1) rows128_tc_kernel(int ny, int rows, const float* __restrict__ in, int ldi,
                                                            const unsigned char* __restrict__ Spk,
                                                            float* __restrict__ out, int ldo) {
  using Md = TallMode<kTall3xTF32>;
  constexpr int T = Md::T;
  constexpr int kBChunk = Md::NSPLIT * ((kKC / T) * (kRowN / 8) * 128);  // 16 KB
  constexpr int kBAll = kRowChunks * kBChunk;                             // 128 KB
  const int bB = Md::b_bytes(kRowN);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Bsm = smem;
  unsigned char* Ast = smem + kBAll;                                      // [2][kAStage]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Ast + 2 * Md::kAStage);     // [0, 1] products, [2] S landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(2 * kRowN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar + b)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar + 2)), "r"(kBAll)
                 : "memory");
    for (int ch = 0; ch < kRowChunks; ++ch)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              saddr(Bsm + ch * kBChunk)),
          "l"(Spk + (size_t)ch * kBChunk), "r"(kBChunk), "r"(saddr(bar + 2))
          : "memory");
  }
  const uint32_t idesc = instr_desc(2, 128, kRowN);
  const int tiles = (rows + 127) / 128;
  bool ok = true, have_s = false;
  int g = 0;  // chunks staged by this CTA so far
  for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const int r = tile * 128 + tid;
    const bool valid = r < rows;
    const int c = valid ? r / ny : 0, j = valid ? r - c * ny : 0;
    const float* rin = in + (size_t)c * ldi + (size_t)j * kRowN;
    for (int ch = 0; ch < kRowChunks; ++ch, ++g) {
      const int s = g & 1;
      if (g >= 2) {
        const bool w = mbar_wait(saddr(bar + s), ((g - 2) >> 1) & 1);
        if (!__syncthreads_and(w)) {
          ok = false;
          break;
        }
      }
      float v[kKC];
      if (valid) {
#pragma unroll
        for (int q = 0; q < kKC / 4; ++q) {
          const float4 x = *reinterpret_cast<const float4*>(rin + ch * kKC + 4 * q);
          v[4 * q] = x.x;
          v[4 * q + 1] = x.y;
          v[4 * q + 2] = x.z;
          v[4 * q + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < kKC; ++k) v[k] = 0.f;
      }
      unsigned char* As = Ast + s * Md::kAStage;
#pragma unroll
      for (int q = 0; q < kKC / T; ++q)
        put_row<kTall3xTF32>(As + (q * 16 + (tid >> 3)) * 128 + (tid & 7) * 16, Md::kABytes, v + q * T);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        if (!have_s) {
          if (!mbar_wait(saddr(bar + 2), 0)) atomicExch(&g_tall_err, 1);
          have_s = true;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = saddr(As), b0 = saddr(Bsm + ch * kBChunk);
#pragma unroll
        for (int ki = 0; ki < kKC / Md::KI; ++ki) {
          const int q = ki * (Md::KI / T);
#pragma unroll
          for (int tm = 0; tm < 3; ++tm) {
            // hi hi into columns 0..127; the two correction products hi lo and
            // lo hi into columns 128..255, summed with the first in the epilogue
            const int sa = (tm == 2) ? 1 : 0, sb = (tm == 1) ? 1 : 0;
            const uint64_t ad = smem_desc(a0 + sa * Md::kABytes + q * 16 * 128, 16 * 128, 128);
            const uint64_t bd = smem_desc(b0 + sb * bB + q * (kRowN / 8) * 128, (kRowN / 8) * 128, 128);
            const uint32_t acc = (ch > 0 || ki > 0 || tm == 2) ? 1u : 0u;
            const uint32_t dst = tmem + (tm > 0 ? (uint32_t)kRowN : 0u);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr(bar + s))
                     : "memory");
      }
    }
    if (!ok) break;
    // the tile's products are done: read the accumulator row by row
    const bool w = mbar_wait(saddr(bar + ((g - 1) & 1)), ((g - 1) >> 1) & 1);
    if (!__syncthreads_and(w)) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    float* rout = out + (size_t)c * ldo + (size_t)j * kRowN;
    for (int cb = 0; cb < kRowN; cb += 8) {
      uint32_t x[8], y[8];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]),
                     "=r"(x[7])
                   : "r"(ta));
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]),
                     "=r"(y[7])
                   : "r"(ta + (uint32_t)kRowN));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) o[i] = __uint_as_float(x[i]) + __uint_as_float(y[i]);
      if (valid) {
        *reinterpret_cast<float4*>(rout + cb) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4*>(rout + cb + 4) = make_float4(o[4], o[5], o[6], o[7]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // every warp has read the accumulator before the next tile overwrites it
  }
  if (!ok) {
    if (tid == 0) atomicExch(&g_tall_err, 1);
    if (g > 0) mbar_wait(saddr(bar + ((g - 1) & 1)), ((g - 1) >> 1) & 1);  // products already issued
  }
  if (tid == 0 && !have_s) mbar_wait(saddr(bar + 2), 0);  // the copy of S has landed
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kRowN));
}

}  // namespace

size_t tall_pack_bytes(int mode, int kk, int c) {
  if (kk <= 0 || c <= 0) return 0;
  switch (mode) {
    case kTallTF32: return pack_bytes<kTallTF32>(kk, c);
    case kTallBF16: return pack_bytes<kTallBF16>(kk, c);
    default: return pack_bytes<kTall3xTF32>(kk, c);
  }
}

template <typename TC>
int tall_gemm_tc(int mode, int rows, int kk, int c, double alpha, const float* A, int lda, const double* B,
                 int ldb, int transB, double beta, TC* C, int ldc, void* pack, cudaStream_t st) {
  if (rows <= 0 || c <= 0) return SC4DVAR_OK;
  if (kk <= 0) return gemm_nn<float, TC>(rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C, ldc, st);
  switch (mode) {
    case kTallTF32:
      return launch_tall<kTallTF32, TC>(rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C, ldc, pack, st);
    case kTallBF16:
      return launch_tall<kTallBF16, TC>(rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C, ldc, pack, st);
    default:
      return launch_tall<kTall3xTF32, TC>(rows, kk, c, alpha, A, lda, B, ldb, transB, beta, C, ldc, pack, st);
  }
}

size_t rows128_pack_bytes() { return (size_t)kRowChunks * 2 * (kKC / 4) * (kRowN / 8) * 128; }

int rows128_pack(const float* S, void* out, cudaStream_t st) {
  tall_pack_b_kernel<kTall3xTF32, float><<<dim3(kRowChunks, 1), 256, 0, st>>>(
      kRowN, kRowN, S, kRowN, 1, kRowN, kRowChunks, static_cast<unsigned char*>(out));
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int rows128_tc(int ny, int rows, const float* in, int ldi, const void* Spk, float* out, int ldo, cudaStream_t st) {
  if (rows <= 0) return SC4DVAR_OK;
  const int smem = (int)rows128_pack_bytes() + 2 * TallMode<kTall3xTF32>::kAStage + 64;
  SC4_CUDA(cudaFuncSetAttribute(rows128_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int tiles = div_up(rows, 128);
  rows128_tc_kernel<<<std::min(tiles, 152), 128, smem, st>>>(ny, rows, in, ldi,
                                                            static_cast<const unsigned char*>(Spk), out, ldo);
  SC4_LAUNCH_CHECK();
  return SC4DVAR_OK;
}

int tall_tc_take_error() {
  int h = 0;
  SC4_CUDA(cudaMemcpyFromSymbol(&h, g_tall_err, sizeof(int)));
  if (h) {
    const int z = 0;
    SC4_CUDA(cudaMemcpyToSymbol(g_tall_err, &z, sizeof(int)));
    set_error("tensor-core tall product: a bounded wait on the tensor-core completion gave up");
    return SC4DVAR_ERR_TIMEOUT;
  }
  return SC4DVAR_OK;
}

template int tall_gemm_tc<float>(int, int, int, int, double, const float*, int, const double*, int, int, double,
                                 float*, int, void*, cudaStream_t);
template int tall_gemm_tc<double>(int, int, int, int, double, const float*, int, const double*, int, int,
                                  double, double*, int, void*, cudaStream_t);

}  // namespace sc4
