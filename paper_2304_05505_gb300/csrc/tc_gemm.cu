// Batched complex GEMMs of the mixed build on the 5th-generation tensor cores
// (tcgen05, sm_103a): the dense contractions S1 (Psi = X^T C), S2
// (D = Psi Psi^H), S4a (Y = M Psi) and S4b (KC = conj(X) Y) of the build.
//
// Complex via a real embedding.  C[m][n] = sum_k A[m][k] B[k][n] with A stored
// as interleaved complex rows is the real product C' = A' B'^T where
//   A'[m][2k+d] = (re, im)[d] of A[m][k]                  (A's own layout)
//   B'[2n+c][2k+d] = [[Br, -Bi], [Bi, Br]][c][d]           (built per call)
// and C'[m][2n+c] is C in interleaved form.  conj(A) B uses
//   B'[2n+c][2k+d] = [[Br, Bi], [Bi, -Br]][c][d].
//
// Exact accumulation (fixed-point slices).  The tensor core's FP32 accumulator
// does not round to nearest, so summing floating-point products on it leaves
// a one-sided error of about an ulp per step, which shows up as a bias in E_x.
// Instead every operand row r is scaled by a power of two so that its entries
// lie in [-128, 128] and cut into three fixed-point slices of 8, 11 and 11 bits:
//   x = 2^(e_r - 7) (S0 + 2^-11 S1 + 2^-22 S2),  S0 in [-128, 128], S1, S2 in [-1024, 1024]
// held in fp16 planes P0 = 2^8 S0, P1 = 2^-3 S1, P2 = 2^-14 S2 (all normal
// fp16 numbers or zero, so exact).  Every product P_s P_t is exact in FP32, and
// the product of two rows is 2^(e_a + e_b - 30) sum_{s,t} P_s^a P_t^b.  The
// leading class P0 P0 is 2^16 times a sum of integers of at most 2^14 each; any
// partial sum of up to 1024 of them is below 2^24 in those units, which the
// FP32 accumulator holds exactly whatever its rounding.  The other kept
// classes go to a second accumulator 2^-11 smaller or less:
//   6 products: (0,0) | (0,2) (2,0) (1,1) (0,1) (1,0)       about 2^-27 of the row scales dropped
//   8 products: the same and (1,2) (2,1)                      about 2^-30
// against 10 products for four 8-bit bf16 slices at the same accuracy.  fp16
// and bf16 operands run at the same kind::f16 rate.
//
// Operand A is either three planes written by a preparation kernel, or an
// FP32 matrix that TMA brings into shared memory and converter warps cut into
// the three planes inside the kernel (no planes of A through HBM):
//   CV = 1  A stored [rows][K] (row-major complex): 128 x 32-float boxes, 128B swizzle
//   CV = 2  A stored [K][rows] (A is the transpose of the stored matrix, as
//           X^T in S1): 16 x 256-float boxes, the converters transpose
//   CV = 3  as CV = 1, plus an fp16 tile of A's remainders (A = hi + lo with
//           hi the FP32 matrix; the extended M of S4a), 64B swizzle; the
//           converters add lo to the first remainder before slicing
//
// Work units: a 128 x 128 output tile and a chunk of at most 1024 real K (so
// the leading sum of a unit is exact), the chunks of one product of equal
// length (tc_chunk_blocks).  When K needs more than one chunk the
// units write their exact int32 leading sums and FP32 remainders to a partial
// buffer and tc_combine adds the chunks (split K); otherwise they write the
// scaled result directly.
//
// Kernel structure (persistent: one CTA per SM loops over units):
//   warp 0      TMA producer: A planes (or the FP32 A tile) and B planes per
//               32-wide real-K block into a ring in shared memory, 64B
//               swizzle, running ahead across units
//   warp 1      allocates 512 TMEM columns = two accumulator sets (leading
//               class, the other classes; 128 columns each) so that the
//               epilogue of one unit overlaps the MMAs of the next; lane 0
//               issues tcgen05.mma (M = 128, N = 128, K = 16, f16 x f16 -> f32),
//               6 or 8 per K step
//   CV:  warps 2-9 converters, warps 10-17 epilogue (8 warps, 64 columns each)
//   else warps 2-3 idle, warps 4-19 epilogue (16 warps, 32 columns each)
// The epilogue warps (4 per TMEM lane quadrant) read both accumulators with
// tcgen05.ld, scale by exact powers of two and store (or write the partial
// sums), then release the accumulator set.  Each warp turns its 32-row x
// 16-column blocks around in a 2 KB shared tile so that every store
// instruction writes whole 64-byte row segments; the unit's row and column
// exponents are loaded before its accumulator is ready.
// Every mbarrier wait is bounded (about 2 s of clock64); on expiry the thread
// sets the error word and stops issuing work, the producer waits (bounded) for
// its copies in flight, the MMA thread for its MMAs in flight, and the CTA
// releases TMEM and exits.
#include "thc_internal.cuh"
#include "tc_gemm.cuh"
#include "slices.cuh"
#include "mbarrier.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace {

constexpr int BM = 128, BN = 128, BKR = 32;
constexpr int NPL = 3;                                       // slices per operand
constexpr uint32_t TILE_BYTES = BM * BKR * 2;                // 8 KB (one plane of A or B)
constexpr int MAX_CHUNK_KB = 32;                             // K blocks per exact chunk, at most (1024 real K)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t STAGE_BYTES = 2 * NPL * TILE_BYTES;       // A and B planes of one K block: 48 KB
constexpr uint32_t EPI_TILE = 32 * 16;                       // floats per epilogue warp (32 rows x 16)
// Shared memory: the operand rings, 256 B of barriers, then the epilogue
// warps' staging tiles.  Plane-fed forms: a 192 KB ring and 16 epilogue
// warps; converted forms: 208 KB of rings (see the kernel) and 8 epilogue
// warps.  Both come to the same total.
template <int CV> struct Smem {
  static constexpr uint32_t RING = CV ? 208 * 1024 : 192 * 1024;
  static constexpr size_t BYTES = RING + 1024 + 256 + (CV ? 8 : 16) * EPI_TILE * 4;
};
static_assert(Smem<1>::BYTES <= 232448 && Smem<0>::BYTES <= 232448, "227 KB of shared memory per block");

// Warp roles: 0 TMA, 1 MMA, then (CV) 8 converter warps, then the epilogue.
// The converted-A forms take 8 epilogue warps, the others 16.
template <int CV> struct Roles {
  static constexpr int CONV_WARPS = CV ? 8 : 0;                 // warps 2 .. 2 + CONV_WARPS - 1
  static constexpr int EPI = CV ? 8 : 16;                       // epilogue warps
  static constexpr int EPI0 = CV ? 2 + CONV_WARPS : 4;          // first epilogue warp
  static constexpr int NT = (EPI0 + EPI) * 32;                  // threads
  static constexpr int COLS = 4 * BN / EPI;                     // columns of a unit per epilogue warp
};

// K-major operand tile, 64B swizzle: rows of 64 B, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;               // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                        // SWIZZLE_64B
  return d;
}

// kind::f16 instruction descriptor: D f32 (bits 4-5 = 1), A and B f16 (type
// fields 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 16 consecutive fp32 columns of this thread's TMEM lane, at each of two
// TMEM addresses, both loads in flight before one wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%33];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[16 + i]);
  }
}

// Float offset of 16-byte chunk c (0..3) of row r in a 32 x 16 staging tile;
// the chunk index is XORed with bits 1-2 of the row so that 8 lanes writing
// one chunk of 8 rows, or reading 8 rows of one chunk, hit distinct banks.
__device__ __forceinline__ int stage_off(int r, int c) { return r * 16 + 4 * (c ^ ((r >> 1) & 3)); }

struct Maps {
  CUtensorMap a[NPL];
  CUtensorMap b[NPL];
};

// Exact powers of two built from the exponent bits (ldexp for the rare
// exponents outside the normal range).
__device__ __forceinline__ float pow2f(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : ldexpf(1.0f, e);
}
__device__ __forceinline__ double pow2d(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}

struct Geometry {
  int M, Nr, Kr, batch;
  int mt, nt, nchunk, nkb;   // tiles along M and N, K chunks, K blocks
  int ckb;                   // K blocks per chunk
  long units;
  int herm;                  // Hermitian product: tiles reaching the diagonal only (1: mirrored, 2: upper part)
  long upb;                  // units per batch entry when herm
  int b0;                    // batch offset of the operands' tensor maps (a sub-batch of a product)
};

// First n tile of m tile mi that reaches the diagonal of a Hermitian product
// (its last complex column >= the tile's first row).
__host__ __device__ __forceinline__ int herm_n0(int mi) {
  const int x = mi * BM - (BN / 2 - 1);
  return x > 0 ? (x + BN / 2 - 1) / (BN / 2) : 0;
}

// Exponent sentinel of an all-zero row (the rows' atomicMax starts below it).
__device__ __forceinline__ int row_exp(const int* e, long i) {
  const int x = e[i];
  return x < -1000 ? 0 : x;
}

// The three fp16 planes of 8 consecutive reals x[0..8) of one row (scale sc =
// 2^(7 - e_row)), packed two reals per word: w[p][j] holds reals 2j, 2j + 1 of
// plane p.
__device__ __forceinline__ void slice8_f16(const float* x, float sc, uint32_t w[NPL][4]) {
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    float lo[NPL], hi[NPL];
    slice3_planes(x[j] * sc, lo);
    slice3_planes(x[j + 1] * sc, hi);
#pragma unroll
    for (int p = 0; p < NPL; p++) {
      const __half2 h = __floats2half2_rn(lo[p], hi[p]);
      w[p][j >> 1] = *reinterpret_cast<const uint32_t*>(&h);
    }
  }
}

// The same for values given as an FP32 part x and a small remainder lo
// (already scaled by the row's scale): the leading slice comes from x alone,
// the remainder joins the first remainder (exact up to an FP32 rounding far
// below the last slice).
__device__ __forceinline__ void slice8_f16x(const float* x, const float* lo, float sc, uint32_t w[NPL][4]) {
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    float p0[NPL], p1[NPL];
    slice3_planes_x(x[j] * sc, lo[j], p0);
    slice3_planes_x(x[j + 1] * sc, lo[j + 1], p1);
#pragma unroll
    for (int p = 0; p < NPL; p++) {
      const __half2 h = __floats2half2_rn(p0[p], p1[p]);
      w[p][j >> 1] = *reinterpret_cast<const uint32_t*>(&h);
    }
  }
}

// OUT: 0 = FP32 result, 1 = FP64 result, 2 = partial sums (split K)
// NP: 6 or 8 slice products per real product (see the header).
// AR (A resident, short K in one chunk): the A tile of all K (4 blocks x 3
// planes, 96 KB) stays in shared memory while the CTA runs the N tiles of one
// (batch, M tile) one after another; only B streams through a 4-stage ring of
// 24 KB.  Each CTA takes a contiguous range of units so that consecutive units
// share their A tile.
// CV (A converted in shared memory, 1, 2 or 3): A is an FP32 (interleaved
// complex) matrix; CV = 3 adds its fp16 remainders (map a[1], 64B swizzle).  TMA brings 16 KB FP32 tiles into a 3-stage staging ring;
// converter warps cut each tile into the three fp16 slices with the rows'
// exponents and write them in the 64B-swizzled K-major layout the MMA reads,
// then fence the generic-proxy writes for the async proxy and arrive on the
// stage's full barrier beside the TMA bytes of the B planes.
template <int OUT, int NP, bool AR, int CV>
__global__ void __launch_bounds__(Roles<CV>::NT, 1)
tc_gemm_kernel(const __grid_constant__ Maps maps, Geometry g, const int* __restrict__ eA, long seA,
               const int* __restrict__ eB, long seB, void* out, long ldo, long sbo, int* __restrict__ ps0,
               float* __restrict__ pbc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  static_assert(NP == 6 || NP == 8, "slice products");
  static_assert(!(AR && CV), "A is resident planes or converted, not both");
  constexpr int AKB = 4;                                           // K blocks the resident A tile holds
  constexpr int CONV_WARPS = Roles<CV>::CONV_WARPS;
  constexpr int EPI_W = Roles<CV>::EPI, EPI_W0 = Roles<CV>::EPI0, EPI_COLS = Roles<CV>::COLS;
  constexpr uint32_t RING_BYTES = Smem<CV>::RING;
  // Converted forms: three decoupled rings so that the DRAM stream of A runs
  // well ahead of the MMAs: FP32 A tiles (SA_STAGES x 16 KB, from DRAM), B
  // planes (B_STAGES x 24 KB, TMA only) and the converted A planes (STAGES x
  // 24 KB, written by the converter warps).
  // CV = 3: each FP32 stage also holds the fp16 tile of the remainders (8 KB)
  constexpr int SA_STAGES = CV == 3 ? 3 : 4, B_STAGES = CV == 3 ? 3 : 4;
  constexpr uint32_t SA_HI = BM * BKR * 4;                         // 16 KB: FP32 tile
  constexpr uint32_t SA_BYTES = CV == 3 ? SA_HI + BM * BKR * 2 : SA_HI;
  constexpr uint32_t PL_BYTES = NPL * TILE_BYTES;                  // 24 KB: three planes of one operand
  constexpr uint32_t B_OFF = SA_STAGES * SA_BYTES + 2 * PL_BYTES;  // CV: the B ring after the A plane ring
  // what precedes the plane ring: the resident A tile, or the FP32 staging ring
  constexpr uint32_t A_BYTES = AR ? AKB * NPL * TILE_BYTES : CV ? SA_STAGES * SA_BYTES : 0;
  constexpr uint32_t SBYTES = (AR || CV) ? PL_BYTES : STAGE_BYTES;  // bytes of one plane-ring stage
  constexpr int STAGES = CV ? 2 : (RING_BYTES - A_BYTES) / SBYTES;
  static_assert(STAGES >= 2 && STAGES <= 4, "ring stages");
  static_assert(!CV || B_OFF + B_STAGES * PL_BYTES <= RING_BYTES, "ring size");
  uint64_t* bars = (uint64_t*)(smem + RING_BYTES);
  // barrier slots: full[4], empty[4], acc_full[2], acc_empty[2], resident A
  // loaded / released, FP32 tile landed / converted [SA_STAGES each], B planes
  // landed / consumed [B_STAGES each], MMAs drained.  CV: full / empty are the
  // converted A planes.
  uint32_t* tmem_slot = (uint32_t*)(bars + 31);
  float* epi_stage = (float*)(smem + RING_BYTES + 256);   // EPI_W tiles of EPI_TILE floats
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto FULL = [&](int s) { return bar0 + 8u * s; };
  auto EMPTY = [&](int s) { return bar0 + 8u * (4 + s); };
  auto AFULL = [&](int s) { return bar0 + 8u * (8 + s); };
  auto AEMPTY = [&](int s) { return bar0 + 8u * (10 + s); };
  const uint32_t AOP_FULL = bar0 + 8u * 12;    // resident A tile loaded
  const uint32_t AOP_EMPTY = bar0 + 8u * 13;   // MMAs on the resident A tile done
  auto SFULL = [&](int s) { return bar0 + 8u * (14 + s); };                            // CV: FP32 tile landed
  auto SEMPTY = [&](int s) { return bar0 + 8u * (14 + SA_STAGES + s); };               // CV: FP32 tile converted
  auto BFULL = [&](int s) { return bar0 + 8u * (14 + 2 * SA_STAGES + s); };            // CV: B planes landed
  auto BEMPTY = [&](int s) { return bar0 + 8u * (14 + 2 * SA_STAGES + B_STAGES + s); };  // CV: B planes consumed
  const uint32_t MMA_DONE = bar0 + 8u * 30;    // every MMA of the CTA complete
  static_assert(2 * SA_STAGES + 2 * B_STAGES <= 16, "barrier slots 14 .. 29");

  __shared__ int abort_flag;
  if (threadIdx.x == 0) abort_flag = *(volatile int*)err;
  __syncthreads();
  if (abort_flag) return;   // an earlier CTA gave up a wait: skip the work

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(FULL(s), CV ? CONV_WARPS : 1);   // CV: the converter warps
      mbar_init(EMPTY(s), 1);
    }
    if (CV) {
      for (int s = 0; s < SA_STAGES; s++) {
        mbar_init(SFULL(s), 1);
        mbar_init(SEMPTY(s), CONV_WARPS);
      }
      for (int s = 0; s < B_STAGES; s++) {
        mbar_init(BFULL(s), 1);
        mbar_init(BEMPTY(s), 1);
      }
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(AFULL(s), 1);
      mbar_init(AEMPTY(s), EPI_W);
    }
    if (AR) {
      mbar_init(AOP_FULL, 1);
      mbar_init(AOP_EMPTY, 1);
    }
    mbar_init(MMA_DONE, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  // units of this CTA: strided (CTAs running side by side share the A tile
  // through L2) or, A resident, one contiguous range
  const long u_begin = AR ? g.units * blockIdx.x / gridDim.x : (long)blockIdx.x;
  const long u_end = AR ? g.units * (blockIdx.x + 1) / gridDim.x : g.units;
  const long u_step = AR ? 1 : gridDim.x;
  // unit u -> (b, m tile, n tile, K chunk), K chunk fastest, then n
  auto decode = [&](long u, int& b, int& mi, int& ni, int& kc) {
    if (g.herm) {   // one chunk; per batch entry the tiles n >= herm_n0(m), m ascending
      kc = 0;
      b = (int)(u / g.upb);
      long r = u - (long)b * g.upb;
      int m = 0;
      for (; m < g.mt - 1; m++) {
        const long cnt = g.nt - herm_n0(m);
        if (r < cnt) break;
        r -= cnt;
      }
      mi = m;
      ni = herm_n0(m) + (int)r;
      return;
    }
    kc = (int)(u % g.nchunk);
    long r = u / g.nchunk;
    ni = (int)(r % g.nt);
    r /= g.nt;
    mi = (int)(r % g.mt);
    b = (int)(r / g.mt);
  };

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < NPL; s++) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.a[s]) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.b[s]) : "memory");
      }
      uint32_t it = 0, agen = 0, nfull = 0, nsa = 0;   // K blocks; B (or A and B) and FP32 A copies issued
      long gprev = -1;
      bool ok = true;
      for (long u = u_begin; u < u_end && ok; u += u_step) {
        int b, mi, ni, kc;
        decode(u, b, mi, ni, kc);
        const int bz = b + g.b0;   // the batch coordinate in the operands' tensor maps
        if constexpr (AR) {
          const long grp = (long)b * g.mt + mi;
          if (grp != gprev) {
            // reload the resident A tile once the MMAs on the previous one are done
            if (agen > 0 && !mbar_wait(AOP_EMPTY, (agen - 1) & 1, err, 32)) { ok = false; break; }
            mbar_expect_tx(AOP_FULL, g.nkb * NPL * TILE_BYTES);
            for (int kb = 0; kb < g.nkb; kb++)
              for (int p = 0; p < NPL; p++)
                tma_load_3d(sbase + (kb * NPL + p) * TILE_BYTES, &maps.a[p], AOP_FULL, kb * BKR, mi * BM, bz);
            gprev = grp;
            agen++;
          }
        }
        const int kb1 = min(g.nkb, (kc + 1) * g.ckb);
        for (int kb = kc * g.ckb; kb < kb1; kb++, it++) {
          const int st = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if constexpr (CV != 0) {
            // the FP32 A tile into the staging ring, the B planes into the plane ring
            const int sa = it % SA_STAGES;
            if (!mbar_wait(SEMPTY(sa), ((it / SA_STAGES) & 1) ^ 1, err, 2)) { ok = false; break; }
            mbar_expect_tx(SFULL(sa), SA_BYTES);
            if constexpr (CV == 1 || CV == 3)
              tma_load_3d(sbase + sa * SA_BYTES, &maps.a[0], SFULL(sa), kb * BKR, mi * BM, bz);
            else   // [K][rows] source: 16 complex K values (rows of the box) x 128 complex rows
              tma_load_3d(sbase + sa * SA_BYTES, &maps.a[0], SFULL(sa), mi * 2 * BM, kb * (BKR / 2), bz);
            if constexpr (CV == 3)   // the remainders' fp16 tile beside it
              tma_load_3d(sbase + sa * SA_BYTES + SA_HI, &maps.a[1], SFULL(sa), kb * BKR, mi * BM, bz);
            nsa++;
            const int sb = it % B_STAGES;
            if (!mbar_wait(BEMPTY(sb), ((it / B_STAGES) & 1) ^ 1, err, 2)) { ok = false; break; }
            mbar_expect_tx(BFULL(sb), PL_BYTES);
            for (int p = 0; p < NPL; p++)
              tma_load_3d(sbase + B_OFF + sb * PL_BYTES + p * TILE_BYTES, &maps.b[p], BFULL(sb), kb * BKR,
                          ni * BN, bz);
            nfull++;
            continue;
          }
          if (!mbar_wait(EMPTY(st), ph ^ 1, err, 2)) { ok = false; break; }
          mbar_expect_tx(FULL(st), SBYTES);
          const uint32_t dst = sbase + A_BYTES + st * SBYTES;
          if constexpr (AR) {
            for (int p = 0; p < NPL; p++)
              tma_load_3d(dst + p * TILE_BYTES, &maps.b[p], FULL(st), kb * BKR, ni * BN, bz);
          } else {
            for (int p = 0; p < NPL; p++)
              tma_load_3d(dst + p * TILE_BYTES, &maps.a[p], FULL(st), kb * BKR, mi * BM, bz);
            for (int p = 0; p < NPL; p++)
              tma_load_3d(dst + (NPL + p) * TILE_BYTES, &maps.b[p], FULL(st), kb * BKR, ni * BN, bz);
          }
          nfull++;
        }
      }
      {
        // let the copies already issued land before the CTA exits (another
        // role may have given up a wait, leaving them unconsumed).  Each
        // drained barrier completes on TMA bytes alone, and only the last
        // ring's worth can be outstanding (a stage is reused only after its
        // copy was consumed); on the normal path every phase tested here has
        // completed already.  Every wait here is bounded.
        constexpr uint32_t RS = CV ? B_STAGES : STAGES;
        const uint32_t n = nfull < RS ? nfull : RS;
        for (uint32_t j = nfull - n; j < nfull; j++) mbar_drain(CV ? BFULL(j % RS) : FULL(j % RS), (j / RS) & 1);
        if constexpr (CV != 0) {
          const uint32_t m = nsa < (uint32_t)SA_STAGES ? nsa : (uint32_t)SA_STAGES;
          for (uint32_t j = nsa - m; j < nsa; j++) mbar_drain(SFULL(j % SA_STAGES), (j / SA_STAGES) & 1);
        }
        if constexpr (AR) {
          if (agen > 0) mbar_drain(AOP_FULL, (agen - 1) & 1);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BM, BN);
      const uint64_t dbase = smem_desc(sbase);
      uint32_t it = 0, local = 0, agen = 0;
      long gprev = -1;
      bool ok = true;
      for (long u = u_begin; u < u_end && ok; u += u_step, local++) {
        int b, mi, ni, kc;
        decode(u, b, mi, ni, kc);
        if constexpr (AR) {
          const long grp = (long)b * g.mt + mi;
          if (grp != gprev) {
            if (agen > 0) mma_commit(AOP_EMPTY);      // arrives when the MMAs issued so far are done
            if (!mbar_wait(AOP_FULL, agen & 1, err, 64)) break;
            fence_after();
            gprev = grp;
            agen++;
          }
        }
        const int set = local & 1;
        if (!mbar_wait(AEMPTY(set), ((local >> 1) & 1) ^ 1, err, 4)) break;
        fence_after();
        const uint32_t accA = tmem + 256 * set, accBC = accA + 128;
        const int kb0 = kc * g.ckb, kb1 = min(g.nkb, (kc + 1) * g.ckb);
        for (int kb = kb0; kb < kb1; kb++, it++) {
          const int st = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          const int sb = it % B_STAGES;
          if (!mbar_wait(FULL(st), ph, err, 8)) { ok = false; break; }
          if (CV && !mbar_wait(BFULL(sb), (it / B_STAGES) & 1, err, 8)) { ok = false; break; }
          fence_after();
          // descriptors: one base per stage, planes and K steps are offsets of
          // (bytes >> 4) in the start-address field (no carry: smem < 256 KB)
          const uint64_t aBase = AR ? dbase + (((uint32_t)kb * NPL * TILE_BYTES) >> 4)
                                    : dbase + ((A_BYTES + st * SBYTES) >> 4);
          const uint64_t bBase = AR ? dbase + ((A_BYTES + st * SBYTES) >> 4)
                                 : CV ? dbase + ((B_OFF + sb * PL_BYTES) >> 4)
                                      : aBase + ((NPL * TILE_BYTES) >> 4);
          constexpr uint64_t PL = TILE_BYTES >> 4;
#pragma unroll
          for (int kk = 0; kk < BKR / 16; kk++) {
            const uint64_t a = aBase + 2 * kk, b2 = bBase + 2 * kk;   // 32 B per K step
            const uint32_t acc = (kb == kb0 && kk == 0) ? 0u : 1u;
            mma_f16(accA, a, b2, idesc, acc);                           // exact leading class (0,0)
            // the other classes, smallest first, into the second accumulator
            if constexpr (NP == 8) {
              mma_f16(accBC, a + PL, b2 + 2 * PL, idesc, acc);          // (1,2)
              mma_f16(accBC, a + 2 * PL, b2 + PL, idesc, 1u);           // (2,1)
              mma_f16(accBC, a, b2 + 2 * PL, idesc, 1u);                // (0,2)
            } else {
              mma_f16(accBC, a, b2 + 2 * PL, idesc, acc);               // (0,2)
            }
            mma_f16(accBC, a + 2 * PL, b2, idesc, 1u);                  // (2,0)
            mma_f16(accBC, a + PL, b2 + PL, idesc, 1u);                 // (1,1)
            mma_f16(accBC, a, b2 + PL, idesc, 1u);                      // (0,1)
            mma_f16(accBC, a + PL, b2, idesc, 1u);                      // (1,0)
          }
          mma_commit(EMPTY(st));
          if (CV) mma_commit(BEMPTY(sb));
        }
        if (!ok) break;
        mma_commit(AFULL(set));
      }
      // every MMA issued by this thread complete before TMEM is released
      mma_commit(MMA_DONE);
      mbar_drain(MMA_DONE, 0);
    }
  } else if (CV != 0 && warp >= 2 && warp < 2 + CONV_WARPS) {
    // converter warps: warp w handles rows 32 (w & 3) .. + 31 (one per lane)
    // and K half w >> 2 (16 reals = two 8-real chunks of each plane)
    const int w = warp - 2;
    const int r = 32 * (w & 3) + lane, hf = w >> 2;
    uint32_t it = 0;
    bool ok = true;
    for (long u = u_begin; u < u_end && ok; u += u_step) {
      int b, mi, ni, kc;
      decode(u, b, mi, ni, kc);
      const int row = mi * BM + r;
      // 2^(7 - e): the row's scale, exact
      const int erow = row < g.M ? row_exp(eA, (long)b * seA + row) : 0;
      const float sc = pow2f(7 - erow);
      const int kb1 = min(g.nkb, (kc + 1) * g.ckb);
      for (int kb = kc * g.ckb; kb < kb1; kb++, it++) {
        const int sa = it % SA_STAGES, st = it % STAGES;
        if (!mbar_wait(SFULL(sa), (it / SA_STAGES) & 1, err, 128)) { ok = false; break; }
        if (!mbar_wait(EMPTY(st), ((it / STAGES) & 1) ^ 1, err, 256)) { ok = false; break; }
        const unsigned char* src = smem + sa * SA_BYTES;
        unsigned char* dstp = smem + A_BYTES + st * SBYTES;
#pragma unroll
        for (int k2 = 0; k2 < 2; k2++) {
          const int pc = 2 * hf + k2;               // 8 reals = one 16-byte chunk of each plane
          float x[8];
          if constexpr (CV == 1 || CV == 3) {
            // FP32 row r, 128B swizzle: 16-byte chunk c at r * 128 + 16 (c ^ (r & 7))
            const float4 f0 = *reinterpret_cast<const float4*>(src + r * 128 + 16 * ((2 * pc) ^ (r & 7)));
            const float4 f1 = *reinterpret_cast<const float4*>(src + r * 128 + 16 * ((2 * pc + 1) ^ (r & 7)));
            x[0] = f0.x; x[1] = f0.y; x[2] = f0.z; x[3] = f0.w;
            x[4] = f1.x; x[5] = f1.y; x[6] = f1.z; x[7] = f1.w;
          } else {
            // [16 K rows][256 floats]: the complex value (K j, row r) at (j * 256 + 2 r) floats
#pragma unroll
            for (int j = 0; j < 4; j++) {
              const float2 v = *reinterpret_cast<const float2*>(src + ((4 * pc + j) * 256 + 2 * r) * 4);
              x[2 * j] = v.x;
              x[2 * j + 1] = v.y;
            }
          }
          uint32_t wd[NPL][4];
          if constexpr (CV == 3) {
            // the remainders of these 8 values, fp16 multiples of each value's
            // unit in the last place (64B-swizzled row r of the fp16 tile)
            const uint4 q = *reinterpret_cast<const uint4*>(src + SA_HI + r * 64 + 16 * (pc ^ ((r >> 1) & 3)));
            const uint32_t qw[4] = {q.x, q.y, q.z, q.w};
            float lo[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const uint16_t h16 = (uint16_t)(qw[j >> 1] >> (16 * (j & 1)));
              const int eh = (int)((__float_as_uint(x[j]) >> 23) & 0xffu);
              // q 2^(eh - 150) (the unit in the last place of x[j]) times the row's scale
              lo[j] = eh >= 24 ? __half2float(__ushort_as_half(h16)) * pow2f(eh - 150 + 7 - erow) : 0.f;
            }
            slice8_f16x(x, lo, sc, wd);
          } else {
            slice8_f16(x, sc, wd);
          }
          // plane row r, 64B swizzle: chunk pc at r * 64 + 16 (pc ^ ((r >> 1) & 3))
          const uint32_t off = r * 64 + 16 * (pc ^ ((r >> 1) & 3));
#pragma unroll
          for (int p = 0; p < NPL; p++)
            *reinterpret_cast<uint4*>(dstp + p * TILE_BYTES + off) = make_uint4(wd[p][0], wd[p][1], wd[p][2], wd[p][3]);
        }
        // the planes were written by the generic proxy; the MMA reads them through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(SEMPTY(sa));
          mbar_arrive(FULL(st));
        }
      }
    }
  } else if (warp >= EPI_W0) {
    // epilogue warps: lane quadrant q, column part h (EPI_COLS columns)
    const int q = warp & 3;
    const int h = (warp - EPI_W0) >> 2;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    float* stg = epi_stage + (warp - EPI_W0) * EPI_TILE;
    uint32_t local = 0;
    for (long u = u_begin; u < u_end; u += u_step, local++) {
      int b, mi, ni, kc;
      decode(u, b, mi, ni, kc);
      const int row0 = mi * BM + 32 * q;          // first row of this warp's blocks
      const int cbase = ni * BN + EPI_COLS * h;   // first column of this warp
      // exponents before the accumulator is ready: this lane's row, and the
      // column pairs of the warp's columns (lane l < EPI_COLS / 2 holds pair l)
      int ea = 0, ebl = 0;
      if constexpr (OUT != 2) {
        if (row0 + lane < g.M) ea = row_exp(eA, (long)b * seA + row0 + lane);
        if (lane < EPI_COLS / 2 && cbase + 2 * lane < g.Nr) ebl = eB[(long)b * seB + (cbase >> 1) + lane];
      }
      const int set = local & 1;
      if (!mbar_wait_warp(AFULL(set), (local >> 1) & 1, err, 16)) break;
      fence_after();
      const uint32_t accA = tmem + lane_off + 256 * set, accBC = accA + 128;
#pragma unroll 1
      for (int qq = 0; qq < EPI_COLS / 16; qq++) {
        float va[16], vb[16];
        tmem_ld16x2(accA + EPI_COLS * h + 16 * qq, accBC + EPI_COLS * h + 16 * qq, va, vb);
        const int col0 = cbase + 16 * qq;             // even: complex pairs stay together
        if (col0 >= g.Nr) continue;                   // the whole block is padding (warp-uniform)
        if constexpr (OUT == 1) {
          int ep[8];   // the block's column-pair exponents, shuffled while all lanes are here
#pragma unroll
          for (int j = 0; j < 8; j++) ep[j] = __shfl_sync(0xffffffffu, ebl, 8 * qq + j);
          const int row = row0 + lane;
          if (row >= g.M) continue;
          double* o = (double*)out + (long)b * sbo + (long)row * ldo;
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            if (col0 + j >= g.Nr) break;
            const double sc = pow2d(ea + ep[j >> 1] - 30);
            // va holds 2^16 times an exact integer below 2^24
            const double x0 = ((double)va[j] + (double)vb[j]) * sc;
            const double x1 = ((double)va[j + 1] + (double)vb[j + 1]) * sc;
            if (col0 + j + 1 < g.Nr && (ldo % 2) == 0) {
              *reinterpret_cast<double2*>(o + col0 + j) = make_double2(x0, x1);
            } else {
              o[col0 + j] = x0;
              if (col0 + j + 1 < g.Nr) o[col0 + j + 1] = x1;
            }
          }
        } else {
          // values of this lane's row into the staging tile
          if constexpr (OUT == 2) {
            // the exact leading sum as an int32 (va / 2^16 is an integer below
            // 2^24) and the remainder, both in units of 2^16
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              *reinterpret_cast<float4*>(stg + stage_off(lane, j >> 2)) =
                  make_float4(__int_as_float(__float2int_rn(va[j] * 0x1p-16f)),
                              __int_as_float(__float2int_rn(va[j + 1] * 0x1p-16f)),
                              __int_as_float(__float2int_rn(va[j + 2] * 0x1p-16f)),
                              __int_as_float(__float2int_rn(va[j + 3] * 0x1p-16f)));
          } else {
            float y[16];
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float s0 = pow2f(ea + __shfl_sync(0xffffffffu, ebl, 8 * qq + (j >> 1)) - 30);
              const float s1 = pow2f(ea + __shfl_sync(0xffffffffu, ebl, 8 * qq + (j >> 1) + 1) - 30);
              // va is exact: one rounding in the add
              y[j] = (va[j] + vb[j]) * s0;
              y[j + 1] = (va[j + 1] + vb[j + 1]) * s0;
              y[j + 2] = (va[j + 2] + vb[j + 2]) * s1;
              y[j + 3] = (va[j + 3] + vb[j + 3]) * s1;
              *reinterpret_cast<float4*>(stg + stage_off(lane, j >> 2)) = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
            }
            if (g.herm == 1) {
              // the mirror image below the diagonal: out[Q][P] = conj(out[P][Q]) for Q > P,
              // lanes = consecutive P, so each store instruction writes 256 contiguous bytes
              const int P = row0 + lane;
              if (P < g.M) {
                float* ob = (float*)out + (long)b * sbo + 2L * P;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                  const int Q = (col0 >> 1) + j;
                  if (Q > P && 2 * Q < g.Nr)
                    *reinterpret_cast<float2*>(ob + (long)Q * ldo) = make_float2(y[2 * j], -y[2 * j + 1]);
                }
              }
            }
          }
          __syncwarp();
          // write out: lane -> (row rr, 4 columns f); 8 rows x 64 B per instruction
          const int f = lane >> 3;
          const int col = col0 + 4 * f;
          const bool vec = (OUT == 2) ? (g.Nr % 4 == 0) : ((ldo % 4) == 0 && (sbo % 4) == 0);
#pragma unroll
          for (int pass = 0; pass < (OUT == 2 ? 2 : 1); pass++) {
            if (pass == 1) {   // FP32 remainders of the chunk through the same tile
              __syncwarp();
#pragma unroll
              for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4*>(stg + stage_off(lane, j >> 2)) =
                    make_float4(vb[j] * 0x1p-16f, vb[j + 1] * 0x1p-16f, vb[j + 2] * 0x1p-16f, vb[j + 3] * 0x1p-16f);
              __syncwarp();
            }
#pragma unroll
            for (int it = 0; it < 4; it++) {
              const int rr = (lane & 7) + 8 * it;
              const int row = row0 + rr;
              if (row >= g.M || col >= g.Nr) continue;
              const float4 v = *reinterpret_cast<const float4*>(stg + stage_off(rr, f));
              float* o;
              if constexpr (OUT == 2) {
                const long base = (((long)kc * g.batch + b) * g.M + row) * g.Nr;
                o = pass == 0 ? reinterpret_cast<float*>(ps0 + base) : pbc + base;
              } else {
                o = (float*)out + (long)b * sbo + (long)row * ldo;
              }
              if (OUT == 0 && g.herm && (col >> 1) + 1 <= row) {   // on or below the diagonal
                if ((col >> 1) + 1 == row) *reinterpret_cast<float2*>(o + col + 2) = make_float2(v.z, v.w);
                continue;
              }
              if (vec && col + 4 <= g.Nr) {
                *reinterpret_cast<float4*>(o + col) = v;
              } else {
                const float w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int i = 0; i < 4; i++)
                  if (col + i < g.Nr) o[col + i] = w4[i];
              }
            }
          }
          __syncwarp();   // the tile is rewritten by the next block
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(AEMPTY(set));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

// Adds the K chunks of a split-K product: out = 2^(e_a + e_b - 14) (sum s0 + sum bc).
// V = 4: four consecutive columns per thread (16-byte partial loads; Nr, ldo
// and sbo multiples of 4), V = 1 otherwise.  DOT (FP32 output, V = 4, out
// contiguous): also the block's partial sums of sum conj(w) out over its
// elements for the interleaved complex w laid out as out (the exchange
// energy's <Psi, Y> when out = Y and w = Psi): each product formed in FP32,
// a thread's products summed in a float-float pair, then FP64 across the
// block; dot[2 b], dot[2 b + 1] = real and imaginary part of block b's sum.
template <bool OUT_F64, int V, bool DOT>
__global__ void __launch_bounds__(256) tc_combine_kernel(const int* __restrict__ ps0, const float* __restrict__ pbc,
                                                         int nchunk, int batch, int M, int Nr,
                                                         const int* __restrict__ eA, long seA,
                                                         const int* __restrict__ eB, long seB, void* out, long ldo,
                                                         long sbo, const float* __restrict__ w, double* dot) {
  static_assert(!DOT || (!OUT_F64 && V == 4), "the dot product of an FP32 result, four columns per thread");
  const long total = (long)batch * M * Nr;
  const long nv = total / V;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (long iv = (long)blockIdx.x * blockDim.x + threadIdx.x; iv < nv; iv += (long)gridDim.x * blockDim.x) {
    const long i = iv * V;
    const int col = (int)(i % Nr);
    const long bm = i / Nr;
    const int m = (int)(bm % M);
    const int b = (int)(bm / M);
    long s0[V];
    float bc[V];
#pragma unroll
    for (int j = 0; j < V; j++) {
      s0[j] = 0;
      bc[j] = 0.f;
    }
    for (int c = 0; c < nchunk; c++) {
      if constexpr (V == 4) {
        const int4 a = __ldcs(reinterpret_cast<const int4*>(ps0 + (long)c * total + i));
        const float4 f = __ldcs(reinterpret_cast<const float4*>(pbc + (long)c * total + i));
        s0[0] += a.x; s0[1] += a.y; s0[2] += a.z; s0[3] += a.w;
        bc[0] += f.x; bc[1] += f.y; bc[2] += f.z; bc[3] += f.w;
      } else {
        s0[0] += ps0[(long)c * total + i];
        bc[0] += pbc[(long)c * total + i];
      }
    }
    const int ea = row_exp(eA, (long)b * seA + m) - 14;
    const long o = (long)b * sbo + (long)m * ldo + col;
    if constexpr (OUT_F64) {
      double x[V];
#pragma unroll
      for (int j = 0; j < V; j++)
        x[j] = ((double)s0[j] + (double)bc[j]) * pow2d(ea + eB[(long)b * seB + ((col + j) >> 1)]);
      if constexpr (V == 4) {
        reinterpret_cast<double2*>((double*)out + o)[0] = make_double2(x[0], x[1]);
        reinterpret_cast<double2*>((double*)out + o)[1] = make_double2(x[2], x[3]);
      } else {
        ((double*)out)[o] = x[0];
      }
    } else {
      // FP32 result without the FP64 pipe: the integer sum (|s0| < 2^31) as
      // its rounded float sh plus the exact remainder s0 - sh (at most 2^6),
      // the FP32 classes added to the remainder first, so that the one
      // remaining rounding is the final add
      float x[V];
#pragma unroll
      for (int j = 0; j < V; j++) {
        const int si = (int)s0[j];
        const float sh = __int2float_rn(si);
        const float lo = __int2float_rn(si - __float2int_rz(sh)) + bc[j];
        const int e = ea + eB[(long)b * seB + ((col + j) >> 1)];
        x[j] = (e >= -126 && e <= 127) ? (sh + lo) * pow2f(e) : ldexpf(sh + lo, e);
      }
      if constexpr (V == 4) *reinterpret_cast<float4*>((float*)out + o) = make_float4(x[0], x[1], x[2], x[3]);
      else ((float*)out)[o] = x[0];
      if constexpr (DOT) {
        const float4 p = __ldcs(reinterpret_cast<const float4*>(w + o));
        const float re0 = fmaf(p.x, x[0], p.y * x[1]), im0 = fmaf(p.x, x[1], -p.y * x[0]);
        const float re1 = fmaf(p.z, x[2], p.w * x[3]), im1 = fmaf(p.z, x[3], -p.w * x[2]);
        float sv, ev;
        two_sum_f(rh, re0, sv, ev); rh = sv; rl += ev;
        two_sum_f(ih, im0, sv, ev); ih = sv; il += ev;
        two_sum_f(rh, re1, sv, ev); rh = sv; rl += ev;
        two_sum_f(ih, im1, sv, ev); ih = sv; il += ev;
      }
    }
  }
  if constexpr (DOT) {
    __shared__ double sh[2][8];
    double re = (double)rh + (double)rl, im = (double)ih + (double)il;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
      sh[0][threadIdx.x >> 5] = re;
      sh[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
        tr += sh[0][i];
        ti += sh[1][i];
      }
      dot[2 * blockIdx.x] = tr;
      dot[2 * blockIdx.x + 1] = ti;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

// A 3-D fp16 plane [batch][rows][ld] read as boxes of 32 (K) x 128 (rows).
cudaError_t make_plane_map(void* map_out, const void* base, int batch, int rows, int cols, int ld) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (ld * 2) % 16) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * rows};
  cuuint32_t box[3] = {BKR, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void*)base, dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_f32_map(void* map_out, const void* base, int batch, int rows, int cols, int ld) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (ld * 4) % 16) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)ld * 4 * rows};
  cuuint32_t box[3] = {BKR, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_f32_map_t(void* map_out, const void* base, int batch, int kdim, int rows, int ld) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (ld * 4) % 16) return cudaErrorInvalidValue;
  // [batch][kdim][ld floats], 2 rows floats valid per K row; boxes of 128
  // complex rows (256 floats) by 16 K rows
  cuuint64_t dims[3] = {(cuuint64_t)(2 * rows), (cuuint64_t)kdim, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)ld * 4 * kdim};
  cuuint32_t box[3] = {2 * BM, BKR / 2, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_f32_map_3d(void* map_out, const void* base, long d0, long d1, long d2, long s1_bytes,
                            long s2_bytes, int b0, int b1, int b2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || s1_bytes % 16 || s2_bytes % 16 || (b0 * 4) % 16 || b0 > 256 || b1 > 256 ||
      b2 > 256)
    return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)s1_bytes, (cuuint64_t)s2_bytes};
  cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_f32_map_2d(void* map_out, const void* base, long inner, long outer, long stride_bytes, int box0,
                            int box1) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || stride_bytes % 16 || (box0 * 4) % 16 || box0 > 256 || box1 > 256)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)stride_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box0, (cuuint32_t)box1};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_chunk_blocks(int M, int Nr, int Kr, int batch) {
  const int nkb = std::max(1, (Kr + BKR - 1) / BKR);
  int nchunk = (nkb + MAX_CHUNK_KB - 1) / MAX_CHUNK_KB;
  const long tiles = (long)batch * ((M + BM - 1) / BM) * ((Nr + BN - 1) / BN);
  // split products pay a partial write and a combine whatever the count, so
  // only they buy tail balance with a shorter chunk
  if (nchunk > 1 && nchunk < nkb && tiles * nchunk < 6L * 152) nchunk++;
  return (nkb + nchunk - 1) / nchunk;
}

long tc_partial_elems(int M, int Nr, int Kr, int batch) {
  const int nkb = (Kr + BKR - 1) / BKR;
  const int ckb = tc_chunk_blocks(M, Nr, Kr, batch);
  const int nchunk = (nkb + ckb - 1) / ckb;
  return nchunk > 1 ? (long)nchunk * batch * M * Nr : 0;
}

cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, int M, int Nr, int Kr, int batch,
                    const int* eA, long seA, const int* eB, long seB, void* out, bool out_f64, long ldo,
                    long sbo, int* ps0, float* pbc, int* err, cudaStream_t s,
                    cudaEvent_t gemm_done, int products, int a_conv, int herm, const float* dot_with,
                    double* dot_partial, int dot_max, int* dot_blocks, int b0, int ckb) {
  if (dot_blocks) *dot_blocks = 0;
  if (b0 < 0) return cudaErrorInvalidValue;
  if (products != 6 && products != 8) return cudaErrorInvalidValue;
  if (a_conv < 0 || a_conv > 3) return cudaErrorInvalidValue;
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  Maps maps;
  for (int p = 0; p < NPL; p++) {
    memcpy(&maps.a[p], A.map[p], sizeof(CUtensorMap));
    memcpy(&maps.b[p], B.map[p], sizeof(CUtensorMap));
  }
  Geometry g;
  g.M = M; g.Nr = Nr; g.Kr = Kr; g.batch = batch;
  g.mt = (M + BM - 1) / BM;
  g.nt = (Nr + BN - 1) / BN;
  g.nkb = (Kr + BKR - 1) / BKR;
  g.ckb = ckb > 0 ? std::min(ckb, MAX_CHUNK_KB) : tc_chunk_blocks(M, Nr, Kr, batch);
  g.nchunk = (g.nkb + g.ckb - 1) / g.ckb;
  g.units = (long)batch * g.mt * g.nt * g.nchunk;
  if (herm < 0 || herm > 2) return cudaErrorInvalidValue;
  g.herm = herm;
  g.upb = 0;
  g.b0 = b0;
  if (herm) {
    // a Hermitian FP32 product written whole: square, one chunk, FP32 interleaved output
    if (Nr != 2 * M || g.nchunk != 1 || out_f64 || a_conv || (ldo % 2) || (sbo % 2)) return cudaErrorInvalidValue;
    for (int mi = 0; mi < g.mt; mi++) g.upb += g.nt - herm_n0(mi);
    g.units = (long)batch * g.upb;
  }
  if (g.units <= 0) return cudaSuccess;
  const bool split = g.nchunk > 1;
  if (split && (!ps0 || !pbc)) return cudaErrorInvalidValue;
  if (g.nchunk > 127) return cudaErrorInvalidValue;   // the combined leading sums stay below 2^31
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  const unsigned grid = (unsigned)std::min<long>(g.units, nsm);
  cudaError_t e = cudaSuccess;
#define LAUNCH(OUTK, NPK, ARK, CVK)                                                                       \
  {                                                                                                       \
    e = cudaFuncSetAttribute(tc_gemm_kernel<OUTK, NPK, ARK, CVK>,                                         \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem<CVK>::BYTES);               \
    if (e != cudaSuccess) return e;                                                                       \
    tc_gemm_kernel<OUTK, NPK, ARK, CVK><<<grid, Roles<CVK>::NT, Smem<CVK>::BYTES, s>>>(maps, g, eA, seA, eB, seB, \
                                                                           out, ldo, sbo, ps0, pbc, err); \
  }
#define BY_OUT(NPK, ARK, CVK) \
  { if (split) LAUNCH(2, NPK, ARK, CVK) else if (out_f64) LAUNCH(1, NPK, ARK, CVK) else LAUNCH(0, NPK, ARK, CVK) }
  // A resident when all K fits the resident tile (one chunk of at most 4 K blocks)
  const bool ar = !a_conv && !split && g.nkb <= 4 && products == 6;
  if (a_conv == 1) {
    if (products == 6) BY_OUT(6, false, 1) else BY_OUT(8, false, 1)
  } else if (a_conv == 2) {
    if (products == 6) BY_OUT(6, false, 2) else BY_OUT(8, false, 2)
  } else if (a_conv == 3) {
    if (products == 6) BY_OUT(6, false, 3) else BY_OUT(8, false, 3)
  } else if (ar) {
    if (out_f64) LAUNCH(1, 6, true, 0) else LAUNCH(0, 6, true, 0)
  } else {
    if (products == 6) BY_OUT(6, false, 0) else BY_OUT(8, false, 0)
  }
#undef BY_OUT
#undef LAUNCH
  e = cudaGetLastError();
  if (e == cudaSuccess && gemm_done) e = cudaEventRecord(gemm_done, s);
  if (e != cudaSuccess || !split) return e;
  const long total = (long)batch * M * Nr;
  const bool v4 = Nr % 4 == 0 && ldo % 4 == 0 && sbo % 4 == 0 && ((uintptr_t)out & 31) == 0;
  unsigned cg = (unsigned)std::min<long>((total / (v4 ? 4 : 1) + 255) / 256, 152L * 16);
  // the dot product rides along when the result is a contiguous FP32 array
  // and w has its layout (16-byte aligned)
  const bool dot = dot_with && dot_partial && dot_blocks && dot_max > 0 && !out_f64 && v4 && ldo == Nr &&
                   sbo == (long)M * Nr && ((uintptr_t)dot_with & 15) == 0;
  if (dot) cg = std::min<unsigned>(cg, (unsigned)dot_max);
#define COMBINE(F64, V, D)                                                                                 \
  tc_combine_kernel<F64, V, D><<<cg, 256, 0, s>>>(ps0, pbc, g.nchunk, batch, M, Nr, eA, seA, eB, seB, out, ldo, \
                                                  sbo, dot_with, dot_partial)
  if (out_f64) {
    if (v4) COMBINE(true, 4, false); else COMBINE(true, 1, false);
  } else if (dot) {
    COMBINE(false, 4, true);
    *dot_blocks = (int)cg;
  } else {
    if (v4) COMBINE(false, 4, false); else COMBINE(false, 1, false);
  }
#undef COMBINE
  return cudaGetLastError();
}
