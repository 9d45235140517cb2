// Batched complex GEMMs of the mixed build on the 5th-generation tensor cores
// (tcgen05, sm_103a): the dense contractions S1 (Psi = X^T C), S2
// (D = Psi Psi^H) and S4b (KC = conj(X) Y) of the build.
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
// Instead every operand row r is scaled by a power of two 2^-e_r so that its
// entries lie in [-1, 1], and written as four slices of 8 bits:
//   x = 2^(e_r - 7) (S0 + 2^-8 S1 + 2^-16 S2 + 2^-24 S3),  S_s integers in [-128, 128]
// kept in bf16 planes P_s = 2^(-8 s) S_s (exact).  The product of two rows is
// then 2^(e_a + e_b - 14) sum_{s,t} P_s^a P_t^b.  The leading class P_0 P_0 is a
// sum of integers of at most 2^14 each; any partial sum of up to 1024 of them
// is an integer below 2^24, which the FP32 accumulator holds exactly whatever
// its rounding.  The nine classes with s + t = 1..3 go to a second
// accumulator; their rounding is at least 2^-8 smaller.  Classes with
// s + t >= 4 (below 2^-32 of the row scales) are dropped.
//
// Kernel structure (one 128 x 128 output tile per CTA, 384 threads):
//   warp 0      TMA producer: 4 A planes + 4 B planes per 32-wide real-K block
//               into a 3-stage ring (64 KB a stage, 64B swizzle)
//   warp 1      allocates 512 TMEM columns; lane 0 issues tcgen05.mma
//               (M = 128, N = 128, K = 16, bf16 x bf16 -> f32), 10 per K step
//   warps 2-3   idle (they keep the block at 12 warps)
//   warps 4-11  epilogue: move the exact leading class out of TMEM into int32
//               registers every DRAIN blocks (1024 real K), then scale, combine
//               and store
// Every mbarrier wait is bounded (about 2 s of clock64); on expiry the thread
// sets the error word, stops issuing work and the CTA releases TMEM and exits.
#include "thc_internal.cuh"
#include "tc_gemm.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace {

constexpr int BM = 128, BN = 128, BKR = 32;
constexpr int NPL = 4;                                       // slices per operand
constexpr int STAGES = 3;
constexpr uint32_t TILE_BYTES = BM * BKR * 2;                // 8 KB (one plane of A or B)
constexpr uint32_t STAGE_BYTES = 2 * NPL * TILE_BYTES;       // 64 KB
constexpr int EPI_WARPS = 8;
constexpr int EPI_WARP0 = 4;
constexpr int NTHREADS = (EPI_WARP0 + EPI_WARPS) * 32;
constexpr int DRAIN = 32;                                    // K blocks per exact chunk (1024 real K)
constexpr long long WAIT_LIMIT = 4000000000LL;               // clock64 cycles (~2 s)
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete.  Gives up after
// WAIT_LIMIT cycles (setting `code` in the error word) or as soon as another
// CTA has set the error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *(volatile int*)err != 0) return false;
    if (clock64() - t0 > WAIT_LIMIT) {
      atomicOr(err, code);
      return false;
    }
  }
}

// The same wait taken by a whole warp, with one answer for every lane.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, int* err, int code) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, err, code);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

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

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
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

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

struct Maps {
  CUtensorMap a[NPL];
  CUtensorMap b[NPL];
};

template <bool OUT_F64>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_gemm_kernel(const __grid_constant__ Maps maps, int M, int Nr, int Kr, const int* __restrict__ eA,
               long seA, const int* __restrict__ eB, long seB, void* out, long ldo, long sbo, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  // bars: full[3], empty[3], accA_full[2], accA_empty[2], done[1]
  uint32_t* tmem_slot = (uint32_t*)(bars + 16);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto FULL = [&](int s) { return bar0 + 8u * s; };
  auto EMPTY = [&](int s) { return bar0 + 8u * (3 + s); };
  auto AFULL = [&](int s) { return bar0 + 8u * (6 + s); };
  auto AEMPTY = [&](int s) { return bar0 + 8u * (8 + s); };
  const uint32_t DONE = bar0 + 8u * 10;

  __shared__ int abort_flag;
  if (threadIdx.x == 0) abort_flag = *(volatile int*)err;
  __syncthreads();
  if (abort_flag) return;   // an earlier CTA gave up a wait: skip the tile

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, b = blockIdx.z;
  const int nkb = (Kr + BKR - 1) / BKR;
  const int nchunk = (nkb + DRAIN - 1) / DRAIN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(FULL(s), 1);
      mbar_init(EMPTY(s), 1);
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(AFULL(s), 1);
      mbar_init(AEMPTY(s), EPI_WARPS);
    }
    mbar_init(DONE, 1);
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

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < NPL; s++) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.a[s]) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.b[s]) : "memory");
      }
      for (int kb = 0; kb < nkb; kb++) {
        const int st = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(EMPTY(st), ph ^ 1, err, 2)) break;
        mbar_expect_tx(FULL(st), STAGE_BYTES);
        const uint32_t dst = sbase + st * STAGE_BYTES;
        for (int p = 0; p < NPL; p++)
          tma_load_3d(dst + p * TILE_BYTES, &maps.a[p], FULL(st), kb * BKR, m0, b);
        for (int p = 0; p < NPL; p++)
          tma_load_3d(dst + (NPL + p) * TILE_BYTES, &maps.b[p], FULL(st), kb * BKR, n0, b);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, BN);
      const uint32_t accBC = tmem + 256;
      for (int kb = 0; kb < nkb; kb++) {
        const int st = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        const int chunk = kb / DRAIN;
        const int buf = chunk & 1;
        const bool chunk_start = (kb % DRAIN) == 0;
        if (chunk_start && !mbar_wait(AEMPTY(buf), ((chunk >> 1) & 1) ^ 1, err, 4)) break;
        if (!mbar_wait(FULL(st), ph, err, 8)) break;
        fence_after();
        const uint32_t accA = tmem + 128 * buf;
        const uint32_t tA = sbase + st * STAGE_BYTES;
        const uint32_t tB = tA + NPL * TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < BKR / 16; kk++) {
          const uint32_t off = kk * 32;
          const uint32_t firstA = (chunk_start && kk == 0) ? 0u : 1u;
          const uint32_t firstBC = (kb == 0 && kk == 0) ? 0u : 1u;
          auto da = [&](int s) { return smem_desc(tA + s * TILE_BYTES + off); };
          auto db = [&](int t) { return smem_desc(tB + t * TILE_BYTES + off); };
          mma_bf16(accA, da(0), db(0), idesc, firstA);          // exact leading class
          // classes s + t = 3, 2, 1 (smallest first) into the second accumulator
          mma_bf16(accBC, da(0), db(3), idesc, firstBC);
          mma_bf16(accBC, da(1), db(2), idesc, 1u);
          mma_bf16(accBC, da(2), db(1), idesc, 1u);
          mma_bf16(accBC, da(3), db(0), idesc, 1u);
          mma_bf16(accBC, da(0), db(2), idesc, 1u);
          mma_bf16(accBC, da(1), db(1), idesc, 1u);
          mma_bf16(accBC, da(2), db(0), idesc, 1u);
          mma_bf16(accBC, da(0), db(1), idesc, 1u);
          mma_bf16(accBC, da(1), db(0), idesc, 1u);
        }
        mma_commit(EMPTY(st));
        if ((kb % DRAIN) == DRAIN - 1 || kb == nkb - 1) mma_commit(AFULL(buf));
      }
      mma_commit(DONE);
    }
  } else if (warp >= EPI_WARP0) {
    // epilogue warps: lane quadrant q, column half h
    const int q = warp & 3;
    const int h = (warp - EPI_WARP0) >> 2;
    const int row = m0 + 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    int s0[64];   // exact leading-class sums, |s0| <= 2^14 K
#pragma unroll
    for (int j = 0; j < 64; j++) s0[j] = 0;
    bool ok = true;
    for (int c = 0; c < nchunk; c++) {
      const int buf = c & 1;
      if (!mbar_wait_warp(AFULL(buf), (c >> 1) & 1, err, 16)) { ok = false; break; }
      fence_after();
#pragma unroll
      for (int qq = 0; qq < 4; qq++) {
        float v[16];
        tmem_ld16(tmem + lane_off + 128 * buf + 64 * h + 16 * qq, v);
#pragma unroll
        for (int j = 0; j < 16; j++) s0[16 * qq + j] += __float2int_rn(v[j]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(AEMPTY(buf));
    }
    if (ok && mbar_wait_warp(DONE, 0, err, 32)) {
      fence_after();
      const int ea = (row < M) ? eA[(long)b * seA + row] : 0;
#pragma unroll
      for (int qq = 0; qq < 4; qq++) {
        float v[16];
        tmem_ld16(tmem + lane_off + 256 + 64 * h + 16 * qq, v);   // classes 1..3
        const int col0 = n0 + 64 * h + 16 * qq;
        if (row < M) {
          if constexpr (OUT_F64) {
            double* o = (double*)out + (long)b * sbo + (long)row * ldo;
#pragma unroll
            for (int j = 0; j < 16; j++) {
              const int col = col0 + j;
              if (col < Nr) {
                const int e = ea + eB[(long)b * seB + (col >> 1)] - 14;
                o[col] = ldexp((double)s0[16 * qq + j] + (double)v[j], e);
              }
            }
          } else {
            float* o = (float*)out + (long)b * sbo + (long)row * ldo;
#pragma unroll
            for (int j = 0; j < 16; j++) {
              const int col = col0 + j;
              if (col < Nr) {
                const int e = ea + eB[(long)b * seB + (col >> 1)] - 14;
                o[col] = ldexpf((float)s0[16 * qq + j] + v[j], e);
              }
            }
          }
        }
      }
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

// A 3-D bf16 plane [batch][rows][ld] read as boxes of 32 (K) x 128 (rows).
cudaError_t make_plane_map(void* map_out, const void* base, int batch, int rows, int cols, int ld) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (ld * 2) % 16) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * rows};
  cuuint32_t box[3] = {BKR, 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, int M, int Nr, int Kr, int batch,
                    const int* eA, long seA, const int* eB, long seB, void* out, bool out_f64, long ldo,
                    long sbo, int* err, cudaStream_t s) {
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  if (Kr > 0x7fffffff / 16384) return cudaErrorInvalidValue;   // exact int32 leading sums
  Maps maps;
  for (int p = 0; p < NPL; p++) {
    memcpy(&maps.a[p], A.map[p], sizeof(CUtensorMap));
    memcpy(&maps.b[p], B.map[p], sizeof(CUtensorMap));
  }
  dim3 grid((Nr + BN - 1) / BN, (M + BM - 1) / BM, batch);
  cudaError_t e;
  if (out_f64) {
    e = cudaFuncSetAttribute(tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<true><<<grid, NTHREADS, SMEM_BYTES, s>>>(maps, M, Nr, Kr, eA, seA, eB, seB, out, ldo, sbo,
                                                          err);
  } else {
    e = cudaFuncSetAttribute(tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<false><<<grid, NTHREADS, SMEM_BYTES, s>>>(maps, M, Nr, Kr, eA, seA, eB, seB, out, ldo, sbo,
                                                           err);
  }
  return cudaGetLastError();
}
