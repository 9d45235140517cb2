// Internal declarations shared by the CUDA translation units of libthc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/thc.h"
#include "tc_gemm.cuh"

// ---------------------------------------------------------------------------
// complex helpers (interleaved re, im)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

template <typename T> struct cplx;
template <> struct cplx<double> { typedef double2 type; };
template <> struct cplx<float> { typedef float2 type; };

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct thc_ctx {
  int n1, n2, n3, nk, nbas, nocc, nisdf;
  int precision;
  int device;
  cudaStream_t stream;
  bool have_x, have_v, built;
  // the tensor-core build replayed as a CUDA graph while not profiled: its
  // executable graph and the caller buffers it was captured with
  cudaGraphExec_t gexec;
  const void *g_C, *g_KC, *g_ex;
  // thc_build_host: a copy stream that moves C in and KC out in halves beside
  // the build (events: fork, the two halves in, the two halves out, join),
  // and the captured host-buffer build with its host buffers
  cudaStream_t cstream;
  cudaEvent_t cev[6];
  cudaGraphExec_t gexec_h;
  const void *gh_C, *gh_KC;
  // FP64 state
  double2* X64;     // [nk][nbas][nisdf]
  double2* Vh64;    // [nk][nisdf][nisdf] prepared kernel (FP64 mode)
  // mixed state
  float2* X32;      // [nk][nbas][ldX] (THC_MIXED_SIMT: ldX = nisdf; THC_MIXED: nisdf rounded up to
                    // even, so that the FP32 rows are 16-byte strided for TMA)
  float2* Vh32;     // [nk][nisdf][nisdf]
  uint32_t* Mlo;    // THC_MIXED_EXT: fp16 remainders (re, im) of M below its FP32 values, [nk][nisdf][nisdf]
  int ldX;
  // workspace (element type follows the precision)
  void* Psi;        // [nk][nisdf][nocc]
  void* D;          // [nk][nisdf][nisdf]
  void* M;          // [nk][nisdf][nisdf]
  void* Y;          // [nk][nisdf][nocc]
  double2* Cdev;    // [nk][nbas][nocc] staging for thc_build_host
  double2* KCdev;   // [nk][nbas][nocc] staging for thc_build_host
  double* exdev;    // 2 doubles staging for thc_build_host
  double* partial;  // reduction scratch
  int* flag;        // device flag word (finite checks)
  int n_partial;
  // tensor-core operands (THC_MIXED): three fp16 fixed-point planes each,
  // plane p at base + p * plane elements, rows padded to 8 elements, and one
  // power-of-two exponent per row.  X is A of S1 (as its transpose) and of
  // S4b, read in FP32 from X32 and sliced inside the GEMM (exponents eXT per
  // point, eXn per basis function).
  uint16_t* PsiA_pl;  // [nk][nisdf][ldPs]   Psi, A of S2         ePsi [nk][nisdf]
  uint16_t* Bc_pl;    // [nk][2 nocc][ldC]   embedded C, B of S1  eC [nk][nocc]
  uint16_t* Bd_pl;    // [nk][2 nisdf][ldPs] embedded Psi^H, B of S2 (ePsi)
  uint16_t* By_pl;    // [nk][2 nocc][ldM]   embedded Psi, B of S4a, then embedded Y, B of S4b
                      //                     (column exponents of Psi, then of Y, in eY [nk][nocc])
                      // M (FP32 workspace) is A of S4a, sliced inside the GEMM   eM [nk][nisdf]
  uint16_t* M_pl;     // [nk][nisdf][ldM] M's slices, only for odd nisdf (FP32 rows of 8 nisdf
                      // bytes are not 16-byte strided, which the FP32 tensor map needs)
  int* ex_pl;         // eXn | eXT | ePsi | eC | eY | eM
  int* part_s0;       // split-K partial sums of the tensor-core GEMMs (exact leading class)
  float* part_bc;     // and their FP32 remainders
  int *eXn, *eXT, *ePsi, *eC, *eY, *eM;
  long plPs, plBc, plBd, plBy, plM;
  int ldC, ldM, ldPs;
  TcOperand opXT, opPs, opXn, opBc, opBd, opBy;   // opXT, opXn: FP32 maps of X32
  TcOperand opMf;     // map[0]: FP32 map of M (A of S4a, converted in the GEMM), even nisdf
  TcOperand opM;      // M's slices, odd nisdf
  // THC-AO-K (thc_build_K), allocated by its first call: Z = M X^T and, for
  // the tensor-core form, the embedded planes of X^T (static) and of Z, the
  // column exponents of Z and split-K partials of the two products; for the
  // FP64 form W = conj(X) M
  bool ao_ready, bxt_valid;
  float2* Zao;        // [nk][nisdf][nbas]
  double2* Wao;       // [nk][nbas][nisdf] (FP64)
  uint16_t* BxT_pl;   // [nk][2 nbas][ldAO]  embedded X^T, B of Z = M X^T (exponents eXn)
  uint16_t* Bz_pl;    // [nk][2 nbas][ldAO]  embedded Z, B of K = conj(X) Z (exponents eZ)
  int* eZ;            // [nk][nbas]
  int* ps0_ao;
  float* pbc_ao;
  long plAO;
  int ldAO;
  TcOperand opBxT, opBz;
  int* tc_err;        // device word: nonzero after a device wait gave up
  int* tc_err_host;   // pinned host copy of it, read by thc_sync
  uint32_t* hkeys;    // row and column keys of the Hermitian convolution (when its form applies)
  bool herm_v;        // every V^q Hermitian (to 1e-12 of max |V|): S2 writes D's upper part, S3 mirrors M
  bool d_upper;       // the last build left D's part below the diagonal unwritten
  bool m_ext;         // the last build wrote M's remainders (THC_MIXED_EXT, Hermitian form)
  cudaEvent_t ev[7];               // stage boundaries of the last build
  std::vector<cudaEvent_t> prof;   // per profiled build: 7 stage boundaries, then the
                                   // start and end of each stage's main kernel (12)
  int prof_max, prof_n;            // slots, builds recorded
  float core_ms[6];                // mean main-kernel times of the last profile
  bool core_valid;
  std::string last_error;
};

// ---------------------------------------------------------------------------
// launchers (each queues kernels on `s`; returns cudaGetLastError())
// ---------------------------------------------------------------------------

// GEMM operand layouts.  A(m, k) and B(k, n) for C(m, n) = sum_k A B.
enum GemmA { A_MK = 0, A_KM = 1, A_MK_CONJ = 2 };   // A[m*lda+k], A[k*lda+m], conj(A[m*lda+k])
enum GemmB { B_KN = 0, B_NK_CONJ = 1, B_NK = 2 };  // B[k*ldb+n], conj(B[n*ldb+k]), B[n*ldb+k]

// FP64 complex batched GEMM on CUDA cores.
cudaError_t gemm_z(int la, int lb, int M, int N, int K, const double2* A, int lda, long sA,
                   const double2* B, int ldb, long sB, double2* C, int ldc, long sC, int batch,
                   cudaStream_t s);

// Mixed complex batched GEMM on CUDA cores: operands rounded to FP32, products
// in FP32, sums of 16 products in FP32 then added into a float-float (two-sum)
// accumulator.  TA/TB are float2 or double2 in memory, TC float2 or double2.
template <typename TA, typename TB, typename TC>
cudaError_t gemm_c_comp(int la, int lb, int M, int N, int K, const TA* A, int lda, long sA,
                        const TB* B, int ldb, long sB, TC* C, int ldc, long sC, int batch,
                        cudaStream_t s);

// Plain FP32 complex batched GEMM (S2).
cudaError_t gemm_c_plain(int la, int lb, int M, int N, int K, const float2* A, int lda, long sA,
                         const float2* B, int ldb, long sB, float2* C, int ldc, long sC,
                         int batch, cudaStream_t s);

// k-mesh convolution M = IDFT(DFT(D) o Vh) per (P,Q) element; npq = elements per k.
cudaError_t kconv_z(const double2* D, const double2* Vh, double2* M, long npq, int n1, int n2,
                    int n3, cudaStream_t s);
cudaError_t kconv_c(const float2* D, const float2* Vh, float2* M, long npq, int n1, int n2,
                    int n3, cudaStream_t s);
// As kconv_c with npq = np^2.  On the 2^3, 3^3 and 4^3 meshes with npq even
// (and err non-null) it runs the TMA-fed convolution, which also writes the
// row exponents of M: e[k * np + p] = the smallest e with
// max_q max(|re|, |im|) of M^k[p][q] < 2^e when that maximum is at least
// 2^-133, else 0; *done tells whether e was written.  err receives a nonzero
// code if a device wait gave up.  started / conv_done (may be null) are
// recorded on s right before and right after the convolution kernel.
// Key scratch (32-bit words) of kconv_c_herm for this shape; 0 where the
// Hermitian form does not apply (meshes other than 2^3, 3^3, 4^3, odd np).
long kconv_herm_key_words(int np, int n1, int n2, int n3);
// Writes the tile table of the Hermitian convolution into its key scratch
// (once, when the context is made).
cudaError_t kconv_herm_prepare(uint32_t* keys, int np, int n1, int n2, int n3, cudaStream_t s);
// The convolution for Hermitian D^k and V^q (M^k Hermitian): reads the
// tiles of D and Vh that reach the diagonal only (D's part below it is never
// read), writes all of M, and the row exponents e of M as kconv_c_rowexp.
// keys: kconv_herm_key_words words of scratch.
// Mlo (may be null; radix-2/4 meshes only): the extended form, which also
// writes the fp16 remainders of M below its FP32 values ([N_k][np][np] pairs
// (re, im), each a multiple of its value's unit in the last place: the
// remainder is q * 2^(e - 24) for a value m 2^e, 1/2 <= m < 1, q the fp16).
cudaError_t kconv_c_herm(const float2* D, const float2* Vh, float2* M, int np, int n1, int n2, int n3,
                         uint32_t* keys, int* e, int* err, cudaEvent_t started, cudaEvent_t conv_done,
                         cudaStream_t s, uint32_t* Mlo = nullptr);
cudaError_t kconv_c_rowexp(const float2* D, const float2* Vh, float2* M, int np, int n1, int n2, int n3,
                           int* e, bool* done, int* err, cudaEvent_t started, cudaEvent_t conv_done,
                           cudaStream_t s);
// out = M plus its fp16 remainders (kconv_c_herm's Mlo), complex128.
cudaError_t mlo_combine_c2z(const float2* M, const uint32_t* Mlo, double2* out, long n, cudaStream_t s);
// Vh[a] = (1/N_k) sum_q V[q] w^{+a.q} in FP64; writes FP64 or FP32 output.
cudaError_t prepare_kernel_z(const double2* V, double2* Vh64, float2* Vh32, long npq, int n1,
                             int n2, int n3, cudaStream_t s);

// max |V - V^H| and max |V| over the nk matrices [np][np] of V: out[0], out[1]
// as the bits of non-negative doubles (atomicMax; the caller zeroes out).
cudaError_t hermitian_deviation_z(const double2* V, int np, int nk, unsigned long long* out, cudaStream_t s);
// out (complex128) = D, with the part below each diagonal filled from the
// conjugate of the part above (D written by a herm = 2 GEMM).
cudaError_t hermitian_fill_c2z(const float2* D, double2* out, int np, int nk, cudaStream_t s);

// E_x = -(1/nk) sum conj(Psi) Y, FP64 accumulation, deterministic two-pass.
cudaError_t ex_reduce_z(const double2* Psi, const double2* Y, long n, int nk, double* partial,
                        int npartial, double* ex, cudaStream_t s);
// E_x from block partial sums of <Psi, Y> already written (2 doubles each,
// real and imaginary part), added in a fixed order: ex[0] = -re / nk,
// ex[1] = -im / nk.
cudaError_t ex_finalize(const double* partial, int npartial, int nk, double* ex, cudaStream_t s);
cudaError_t ex_reduce_c(const float2* Psi, const float2* Y, long n, int nk, double* partial,
                        int npartial, double* ex, cudaStream_t s);

// Message returned by thc_last_error(NULL) for calls made without a context.
void set_global_error(const std::string& msg);

// conversions and checks
cudaError_t convert_z2c(const double2* in, float2* out, long n, cudaStream_t s);
// out[r][c] (leading dimension ldo) = in[r][c] (contiguous rows of cols) in FP32.
cudaError_t convert_z2c_rows(const double2* in, float2* out, long rows, int cols, int ldo, cudaStream_t s);
cudaError_t convert_c2z(const float2* in, double2* out, long n, cudaStream_t s);
cudaError_t check_finite_z(const double2* in, long n, int* flag, cudaStream_t s);

