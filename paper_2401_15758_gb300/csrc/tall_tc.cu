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
#include <cuda.h>
#include <cudaTypedefs.h>
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
      // load and wait in one statement: the registers are defined only once
      // the wait has retired the load
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          "tcgen05.wait::ld.sync.aligned;"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(ta)
          : "memory");
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
// out[r][p] = sum_i in[r][i] S[i][p] for the rows r = c ny + j of k fields held
// back to back (row r at in + 128 r; its output at out + c ldo + 128 j), S a
// fixed 128 x 128 FP32 matrix packed once (rows128_pack) in the staged operand
// format of its eight 16-wide K chunks (128 KB for the 3xTF32 split). A
// persistent CTA keeps the packed S in shared memory and walks 128-row tiles
// with four roles that run ahead of one another through mbarrier rings (every
// wait bounded, its verdict made uniform across the warp):
//   loader warp (one thread)  tensor-memory-access loads of the raw FP32 K
//                        chunks of the rows (2D tensor map, box 16 x 128) into a
//                        ring of kRawSlots slots;
//   splitting warps      two groups of four warps that take the chunks in turn
//                        and split each into TF32 hi and lo parts in the
//                        canonical K-major operand layout (kAStages stages);
//   MMA warp (one thread) six tcgen05 MMAs per chunk: hi hi into accumulator
//                        columns 0..127, hi lo and lo hi into 128..255 (summed
//                        in the epilogue), two such accumulators (all 512 TMEM
//                        columns) so that one tile's products overlap the
//                        previous tile's epilogue;
//   epilogue warps       read an accumulator with tcgen05.ld (epilogue warp w
//                        owns TMEM lanes 32w .. 32w + 31), add its two halves and
//                        write the rows through a per-warp shared slab of 32
//                        columns, so that every store instruction covers four
//                        128-byte row segments.
constexpr int kRowN = 128;
constexpr int kRowChunks = kRowN / kKC;
constexpr int kRawSlots = 4;
constexpr int kAStages = 3;
constexpr int kRawBytes = kKC * kRowN * 4;  // 16 floats of 128 rows
// warps: kConvW splitting warps, 4 epilogue warps, one loader and one MMA warp
template <int CW>
struct RowsRoles {
  static_assert(CW % 4 == 0, "the epilogue warps must start at a multiple of four (TMEM lane quarters)");
  static constexpr int kEpi0 = CW, kLoad = CW + 4, kMma = CW + 5, kThreads = (CW + 6) * 32;
};
constexpr int kConvW = 8;  // two groups: 41.6 -> 36.4 us per k = 384 transform against one group
constexpr int kSlabStride = 36;             // floats per slab row (16-byte rows, no bank conflicts)

struct RowsSmem {
  static constexpr int kStage = 2 * (kKC / 4) * 16 * 128;  // hi + lo of a 128-row chunk
  static constexpr int S = 0;
  static constexpr int raw = kRowChunks * kStage;
  static constexpr int A = raw + kRawSlots * kRawBytes;
  static constexpr int slab = A + kAStages * kStage;
  static constexpr int bar = slab + 4 * 32 * kSlabStride * 4;
  // rawfull[R], rawempty[R], afull[A], aempty[A], accf[2], acce[2], sbar
  static constexpr int nbar = 2 * kRawSlots + 2 * kAStages + 5;
  static constexpr int total = bar + nbar * 8 + 16;
};
static_assert(RowsSmem::total <= 232448, "row transform exceeds the shared memory of a CTA");

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* b, int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

template <int CW>
__global__ void __launch_bounds__(RowsRoles<CW>::kThreads, 1)
    rows128_tc_kernel(const __grid_constant__ CUtensorMap tin, int ny, int rows,
                      const unsigned char* __restrict__ Spk, float* __restrict__ out, int ldo) {
  using Md = TallMode<kTall3xTF32>;
  using Ro = RowsRoles<CW>;
  constexpr int T = Md::T;
  constexpr int kBChunk = RowsSmem::kStage;  // 16 KB of packed S per K chunk
  const int bB = Md::b_bytes(kRowN);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Ssm = smem + RowsSmem::S;
  unsigned char* raw = smem + RowsSmem::raw;
  unsigned char* Ast = smem + RowsSmem::A;
  float* slab = reinterpret_cast<float*>(smem + RowsSmem::slab);
  uint64_t* rawfull = reinterpret_cast<uint64_t*>(smem + RowsSmem::bar);
  uint64_t* rawempty = rawfull + kRawSlots;
  uint64_t* afull = rawempty + kRawSlots;
  uint64_t* aempty = afull + kAStages;
  uint64_t* accf = aempty + kAStages;
  uint64_t* acce = accf + 2;
  uint64_t* sbar = acce + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == Ro::kMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(4 * kRowN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    auto init = [](uint64_t* b, int n) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n));
    };
    for (int i = 0; i < kRawSlots; ++i) {
      init(rawfull + i, 1);
      init(rawempty + i, 4);
    }
    for (int i = 0; i < kAStages; ++i) {
      init(afull + i, 4);
      init(aempty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      init(accf + i, 1);
      init(acce + i, 4);
    }
    init(sbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int tiles = (rows + 127) / 128;
  bool ok = true;
  if (warp == Ro::kLoad) {
    // ---- loads: S once, then the raw K chunks of every tile
    if (lane == 0) {
      mbar_expect(sbar, kRowChunks * kBChunk);
      for (int ch = 0; ch < kRowChunks; ++ch)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                saddr(Ssm + ch * kBChunk)),
            "l"(Spk + (size_t)ch * kBChunk), "r"(kBChunk), "r"(saddr(sbar))
            : "memory");
      const uint64_t tmap = reinterpret_cast<uint64_t>(&tin);
      int g = 0;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x)
        for (int ch = 0; ch < kRowChunks; ++ch, ++g) {
          const int i = g % kRawSlots;
          if (g >= kRawSlots && !mbar_wait(saddr(rawempty + i), ((g / kRawSlots) - 1) & 1)) {
            ok = false;
            break;
          }
          mbar_expect(rawfull + i, kRawBytes);
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
              "[%4];" ::"r"(saddr(raw + i * kRawBytes)),
              "l"(tmap), "r"(ch * kKC), "r"(tile * 128), "r"(saddr(rawfull + i))
              : "memory");
        }
      // every copy issued has landed before the CTA exits
      for (int u = (g > kRawSlots ? g - kRawSlots : 0); u < g; ++u)
        mbar_wait(saddr(rawfull + u % kRawSlots), (u / kRawSlots) & 1);
      mbar_wait(saddr(sbar), 0);
      if (!ok) atomicExch(&g_tall_err, 1);
    }
  } else if (warp < CW) {
    // ---- split: CW / 4 groups of four warps take the K chunks in turn (two
    // chunks in flight with eight warps); in a group, thread t converts K
    // quarter t & 3 of rows t / 4 + 32 u
    constexpr int kGroups = CW / 4;
    const int grp = warp >> 2, gt = tid & 127, q = gt & 3;
    int g = 0;
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x)
      for (int ch = 0; ch < kRowChunks; ++ch, ++g) {
        if (g % kGroups != grp) continue;
        const int i = g % kRawSlots, s = g % kAStages;
        if (!__all_sync(0xffffffffu, mbar_wait(saddr(rawfull + i), (g / kRawSlots) & 1))) {
          ok = false;
          break;
        }
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          v[u] = *reinterpret_cast<const float4*>(raw + i * kRawBytes + ((gt >> 2) + 32 * u) * (kKC * 4) + q * 16);
        if (g >= kAStages && !__all_sync(0xffffffffu, mbar_wait(saddr(aempty + s), ((g / kAStages) - 1) & 1))) {
          ok = false;
          break;
        }
        unsigned char* As = Ast + s * RowsSmem::kStage;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = (gt >> 2) + 32 * u;
          put_row<kTall3xTF32>(As + (q * 16 + (r >> 3)) * 128 + (r & 7) * 16, Md::kABytes, &v[u].x);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        // the raw slot is released only after its values have been consumed, so
        // no read of it is still in flight when the next copy overwrites it
        if (lane == 0) {
          mbar_arrive(afull + s);
          mbar_arrive(rawempty + i);
        }
      }
    if (!ok && lane == 0) atomicExch(&g_tall_err, 1);
  } else if (warp == Ro::kMma) {
    // ---- products
    if (lane == 0) {
      const uint32_t idesc = instr_desc(2, 128, kRowN);
      uint64_t* last = nullptr;
      uint32_t lastpar = 0;
      ok = mbar_wait(saddr(sbar), 0);
      int g = 0, lt = 0;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++lt) {
        const int b = lt & 1;
        if (lt >= 2 && !mbar_wait(saddr(acce + b), ((lt >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int ch = 0; ch < kRowChunks; ++ch, ++g) {
          const int s = g % kAStages;
          if (!mbar_wait(saddr(afull + s), (g / kAStages) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = saddr(Ast + s * RowsSmem::kStage), b0 = saddr(Ssm + ch * kBChunk);
#pragma unroll
          for (int ki = 0; ki < kKC / Md::KI; ++ki) {
            const int qq = ki * (Md::KI / T);
#pragma unroll
            for (int tm = 0; tm < 3; ++tm) {
              const int sa = (tm == 2) ? 1 : 0, sb = (tm == 1) ? 1 : 0;  // hi hi, hi lo, lo hi
              const uint64_t ad = smem_desc(a0 + sa * Md::kABytes + qq * 16 * 128, 16 * 128, 128);
              const uint64_t bd = smem_desc(b0 + sb * bB + qq * (kRowN / 8) * 128, (kRowN / 8) * 128, 128);
              const uint32_t acc = (ch > 0 || ki > 0 || tm == 2) ? 1u : 0u;
              const uint32_t dst = tmem + (uint32_t)(b * 2 * kRowN) + (tm > 0 ? (uint32_t)kRowN : 0u);
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           saddr(aempty + s))
                       : "memory");
          last = aempty + s;
          lastpar = (g / kAStages) & 1;
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr(accf + b))
                     : "memory");
        last = accf + b;
        lastpar = (lt >> 1) & 1;
      }
      if (last) mbar_wait(saddr(last), lastpar);  // the products issued have completed
      if (!ok) atomicExch(&g_tall_err, 1);
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp kEpi0 + e writes rows 32 e .. 32 e + 31 of every tile
    const int e = warp - Ro::kEpi0;
    float* sl = slab + e * 32 * kSlabStride;
    int lt = 0;
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++lt) {
      const int b = lt & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(saddr(accf + b), (lt >> 1) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int r = tile * 128 + e * 32 + lane;
      const int c = r / ny, j = r - c * ny;
      const long long base = r < rows ? (long long)c * ldo + (long long)j * kRowN : -1;
#pragma unroll 1
      for (int cb = 0; cb < kRowN; cb += 32) {
        uint32_t x[32], y[32];
        const uint32_t ta = tmem + ((uint32_t)(e * 32) << 16) + (uint32_t)(b * 2 * kRowN + cb);
        // both halves and the wait in one statement: the registers are defined
        // only once the wait has retired the loads (split statements let their
        // consumers be scheduled ahead of the wait)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n"
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
            "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]),
              "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]),
              "=r"(x[15]), "=r"(x[16]), "=r"(x[17]), "=r"(x[18]), "=r"(x[19]), "=r"(x[20]), "=r"(x[21]),
              "=r"(x[22]), "=r"(x[23]), "=r"(x[24]), "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]),
              "=r"(x[29]), "=r"(x[30]), "=r"(x[31]),
              "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]),
              "=r"(y[8]), "=r"(y[9]), "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]),
              "=r"(y[15]), "=r"(y[16]), "=r"(y[17]), "=r"(y[18]), "=r"(y[19]), "=r"(y[20]), "=r"(y[21]),
              "=r"(y[22]), "=r"(y[23]), "=r"(y[24]), "=r"(y[25]), "=r"(y[26]), "=r"(y[27]), "=r"(y[28]),
              "=r"(y[29]), "=r"(y[30]), "=r"(y[31])
            : "r"(ta), "r"(ta + (uint32_t)kRowN)
            : "memory");
#pragma unroll
        for (int m = 0; m < 8; ++m)
          *reinterpret_cast<float4*>(sl + lane * kSlabStride + 4 * m) =
              make_float4(__uint_as_float(x[4 * m]) + __uint_as_float(y[4 * m]),
                          __uint_as_float(x[4 * m + 1]) + __uint_as_float(y[4 * m + 1]),
                          __uint_as_float(x[4 * m + 2]) + __uint_as_float(y[4 * m + 2]),
                          __uint_as_float(x[4 * m + 3]) + __uint_as_float(y[4 * m + 3]));
        __syncwarp();
        // eight lanes per 128-byte row segment, four rows per store instruction
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = 4 * i + (lane >> 3), cc = (lane & 7) * 4;
          const long long bi = __shfl_sync(0xffffffffu, base, rr);
          const float4 v = *reinterpret_cast<const float4*>(sl + rr * kSlabStride + cc);
          if (bi >= 0) *reinterpret_cast<float4*>(out + bi + cb + cc) = v;
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce + b);
    }
    if (!ok && lane == 0) atomicExch(&g_tall_err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == Ro::kMma) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * kRowN));
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

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

int rows128_tc(int ny, int rows, const float* in, const void* Spk, float* out, int ldo, cudaStream_t st) {
  if (rows <= 0) return SC4DVAR_OK;
  if (ny <= 0 || ((uintptr_t)in % 16) != 0 || ((uintptr_t)out % 16) != 0 || ldo % 4 != 0 || !Spk)
    return SC4DVAR_ERR_INVALID_ARG;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return SC4DVAR_ERR_CUDA;
  CUtensorMap tm;
  const cuuint64_t dims[2] = {(cuuint64_t)kRowN, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kRowN * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, 128u};
  const cuuint32_t estr[2] = {1u, 1u};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(in), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return SC4DVAR_ERR_CUDA;
  auto kern = rows128_tc_kernel<kConvW>;
  SC4_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, RowsSmem::total));
  const int tiles = div_up(rows, 128);
  kern<<<std::min(tiles, 152), RowsRoles<kConvW>::kThreads, RowsSmem::total, st>>>(
      tm, ny, rows, static_cast<const unsigned char*>(Spk), out, ldo);
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
