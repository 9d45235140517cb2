// Batched complex GEMMs on CUDA cores for the build's contractions S1, S2, S4a
// and S4b (the contractions of Algorithm 2's exchange lines).
//
//   C[b](m, n) = sum_k A[b](m, k) B[b](k, n)
//
// A is read as A[m*lda + k] (A_MK), A[k*lda + m] (A_KM, a transpose) or
// conj(A[m*lda + k]) (A_MK_CONJ); B as B[k*ldb + n] (B_KN),
// conj(B[n*ldb + k]) (B_NK_CONJ) or B[n*ldb + k] (B_NK, FP64 form).  Tiles of 64 x 64 outputs, 16-deep k slabs
// staged in shared memory.  FP64: 256 threads with 4 x 4 outputs each.  FP32:
// 512 threads with 2 x 4 outputs each and double-buffered slabs.
//
// Three arithmetic forms:
//  * FP64 (double2 throughout): the plain FP64 build.
//  * compensated FP32: operands rounded to FP32, products and 16-term partial
//    sums in FP32, partial sums folded into a float-float (hi, lo) pair with
//    an error-free two-sum after every slab, so the long K sums (432, 1200)
//    do not lose the low bits an FP32 running sum would.
//  * plain FP32 (S2, whose K = n_occ is short).
#include "thc_internal.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T> struct Real;
template <> struct Real<double2> { typedef double t; };
template <> struct Real<float2> { typedef float t; };

__device__ __forceinline__ float2 to_c(float2 v, float) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_c(double2 v, double) { return v; }

__device__ __forceinline__ void store_out(float2* p, float2 hi, float2 lo) {
  *p = make_float2(hi.x + lo.x, hi.y + lo.y);
}
__device__ __forceinline__ void store_out(double2* p, float2 hi, float2 lo) {
  *p = make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
}
__device__ __forceinline__ void store_out(double2* p, double2 v, double2) { *p = v; }

__device__ __forceinline__ void store_plain(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void store_plain(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void store_plain(double2* p, float2 v) {
  *p = make_double2((double)v.x, (double)v.y);
}

// error-free two-sum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

template <typename R, int LA, int LB, bool COMP, typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(NT)
gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int lda, long sA,
            const TB* __restrict__ B, int ldb, long sB, TC* __restrict__ C, int ldc, long sC) {
  typedef typename cplx<R>::type CT;
  __shared__ CT As[BK][BM + 1];
  __shared__ CT Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const R zr = (R)0;

  CT acc[4][4];
  CT hi[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      acc[i][j] = CT{zr, zr};
      hi[i][j] = CT{zr, zr};
      lo[i][j] = CT{zr, zr};
    }

  for (int k0 = 0; k0 < K; k0 += BK) {
    // stage A slab (BM x BK)
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; r++) {
      int e = tid + r * NT;
      int mm, kk;
      if (LA == A_KM) { kk = e / BM; mm = e % BM; }
      else { mm = e / BK; kk = e % BK; }
      int gm = m0 + mm, gk = k0 + kk;
      CT v = CT{zr, zr};
      if (gm < M && gk < K) {
        if (LA == A_KM) v = to_c(A[(long)gk * lda + gm], zr);
        else v = to_c(A[(long)gm * lda + gk], zr);
        if (LA == A_MK_CONJ) v.y = -v.y;
      }
      As[kk][mm] = v;
    }
    // stage B slab (BK x BN)
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; r++) {
      int e = tid + r * NT;
      int nn, kk;
      if (LB == B_KN) { kk = e / BN; nn = e % BN; }
      else { nn = e / BK; kk = e % BK; }
      int gn = n0 + nn, gk = k0 + kk;
      CT v = CT{zr, zr};
      if (gn < N && gk < K) {
        if (LB == B_KN) v = to_c(B[(long)gk * ldb + gn], zr);
        else {
          v = to_c(B[(long)gn * ldb + gk], zr);
          if (LB == B_NK_CONJ) v.y = -v.y;
        }
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      CT a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i][j].x = fma(a[i].x, bb[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, bb[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, bb[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, bb[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
    if constexpr (COMP) {
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          float s, e;
          two_sum((float)hi[i][j].x, (float)acc[i][j].x, s, e);
          hi[i][j].x = s; lo[i][j].x += e;
          two_sum((float)hi[i][j].y, (float)acc[i][j].y, s, e);
          hi[i][j].y = s; lo[i][j].y += e;
          acc[i][j] = CT{zr, zr};
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) {
        if constexpr (COMP) store_out(&C[(long)gm * ldc + gn], hi[i][j], lo[i][j]);
        else store_plain(&C[(long)gm * ldc + gn], acc[i][j]);
      }
    }
}

// FP32 form, 512 threads, 2 x 4 complex outputs a thread (rows ty + 32 i,
// columns tx + 16 j), and two shared-memory slabs: the next slab is fetched
// into registers while the current one is multiplied.
constexpr int NT2 = 512;

template <int LA, int LB, bool COMP, typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(NT2)
gemm_c_kernel(int M, int N, int K, const TA* __restrict__ A, int lda, long sA, const TB* __restrict__ B,
              int ldb, long sB, TC* __restrict__ C, int ldc, long sC) {
  __shared__ float2 As[2][BK][BM + 1];
  __shared__ float2 Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long b = blockIdx.z;
  A += b * sA;
  B += b * sB;
  C += b * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  float2 acc[2][4], hi[2][4], lo[2][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      acc[i][j] = make_float2(0.f, 0.f);
      hi[i][j] = make_float2(0.f, 0.f);
      lo[i][j] = make_float2(0.f, 0.f);
    }

  // this thread's two A and two B elements of a slab
  float2 pa[2], pb[2];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const int e = tid + r * NT2;
      int mm, kk;
      if (LA == A_KM) { kk = e / BM; mm = e % BM; }
      else { mm = e / BK; kk = e % BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gm < M && gk < K) {
        v = to_c((LA == A_KM) ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk], 0.f);
        if (LA == A_MK_CONJ) v.y = -v.y;
      }
      pa[r] = v;
    }
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const int e = tid + r * NT2;
      int nn, kk;
      if (LB == B_KN) { kk = e / BN; nn = e % BN; }
      else { nn = e / BK; kk = e % BK; }
      const int gn = n0 + nn, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gn < N && gk < K) {
        if (LB == B_KN) v = to_c(B[(long)gk * ldb + gn], 0.f);
        else { v = to_c(B[(long)gn * ldb + gk], 0.f); v.y = -v.y; }
      }
      pb[r] = v;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const int e = tid + r * NT2;
      if (LA == A_KM) As[buf][e / BM][e % BM] = pa[r];
      else As[buf][e % BK][e / BK] = pa[r];
      if (LB == B_KN) Bs[buf][e / BN][e % BN] = pb[r];
      else Bs[buf][e % BK][e / BK] = pb[r];
    }
  };

  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      float2 a[2], bb[4];
#pragma unroll
      for (int i = 0; i < 2; i++) a[i] = As[buf][kk][ty + 32 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) bb[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          acc[i][j].x = fmaf(a[i].x, bb[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-a[i].y, bb[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(a[i].x, bb[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(a[i].y, bb[j].x, acc[i][j].y);
        }
    }
    if constexpr (COMP) {
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          float s, e;
          two_sum(hi[i][j].x, acc[i][j].x, s, e);
          hi[i][j].x = s; lo[i][j].x += e;
          two_sum(hi[i][j].y, acc[i][j].y, s, e);
          hi[i][j].y = s; lo[i][j].y += e;
          acc[i][j] = make_float2(0.f, 0.f);
        }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gm = m0 + ty + 32 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) {
        if constexpr (COMP) store_out(&C[(long)gm * ldc + gn], hi[i][j], lo[i][j]);
        else store_plain(&C[(long)gm * ldc + gn], acc[i][j]);
      }
    }
}

template <bool COMP, typename TA, typename TB, typename TC>
cudaError_t launch_c(int la, int lb, int M, int N, int K, const TA* A, int lda, long sA, const TB* B, int ldb,
                     long sB, TC* C, int ldc, long sC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
#define L(LA_, LB_)                                                                                         \
  if (la == LA_ && lb == LB_) {                                                                             \
    gemm_c_kernel<LA_, LB_, COMP, TA, TB, TC><<<grid, NT2, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, \
                                                                   sC);                                     \
    return cudaGetLastError();                                                                              \
  }
  L(A_MK, B_KN) L(A_KM, B_KN) L(A_MK_CONJ, B_KN) L(A_MK, B_NK_CONJ)
#undef L
  return cudaErrorInvalidValue;
}

template <typename R, bool COMP, typename TA, typename TB, typename TC>
cudaError_t launch(int la, int lb, int M, int N, int K, const TA* A, int lda, long sA,
                   const TB* B, int ldb, long sB, TC* C, int ldc, long sC, int batch,
                   cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
#define L(LA_, LB_)                                                                     \
  if (la == LA_ && lb == LB_) {                                                         \
    gemm_kernel<R, LA_, LB_, COMP, TA, TB, TC><<<grid, NT, 0, s>>>(M, N, K, A, lda, sA, \
                                                                  B, ldb, sB, C, ldc, sC); \
    return cudaGetLastError();                                                          \
  }
  L(A_MK, B_KN) L(A_KM, B_KN) L(A_MK_CONJ, B_KN) L(A_MK, B_NK_CONJ) L(A_MK, B_NK)
#undef L
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t gemm_z(int la, int lb, int M, int N, int K, const double2* A, int lda, long sA,
                   const double2* B, int ldb, long sB, double2* C, int ldc, long sC, int batch,
                   cudaStream_t s) {
  return launch<double, false>(la, lb, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, s);
}

template <typename TA, typename TB, typename TC>
cudaError_t gemm_c_comp(int la, int lb, int M, int N, int K, const TA* A, int lda, long sA,
                        const TB* B, int ldb, long sB, TC* C, int ldc, long sC, int batch,
                        cudaStream_t s) {
  return launch_c<true>(la, lb, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, s);
}

cudaError_t gemm_c_plain(int la, int lb, int M, int N, int K, const float2* A, int lda, long sA,
                         const float2* B, int ldb, long sB, float2* C, int ldc, long sC,
                         int batch, cudaStream_t s) {
  return launch_c<false>(la, lb, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, s);
}

template cudaError_t gemm_c_comp<float2, double2, float2>(int, int, int, int, int, const float2*,
    int, long, const double2*, int, long, float2*, int, long, int, cudaStream_t);
template cudaError_t gemm_c_comp<float2, float2, float2>(int, int, int, int, int, const float2*,
    int, long, const float2*, int, long, float2*, int, long, int, cudaStream_t);
template cudaError_t gemm_c_comp<float2, float2, double2>(int, int, int, int, int, const float2*,
    int, long, const float2*, int, long, double2*, int, long, int, cudaStream_t);
