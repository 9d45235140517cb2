// The k-mesh convolution of the build, step S3 (Sec. 2.2: the sum over q of
// M^q against the occupied products is a convolution in k space, done by FFT
// in O(N_k log N_k)):
//
//   M^k[P,Q] = sum_{k'} D^{k'}[P,Q] V^{k'-k}[P,Q]
//            = sum_a w^{+a.k} ( sum_{k'} w^{-a.k'} D^{k'}[P,Q] ) Vh^a[P,Q]
//   Vh^a[P,Q] = (1/N_k) sum_q w^{+a.q} V^q[P,Q]           (prepare_kernel)
//
// with w = exp(2 pi i / n) per mesh axis.  Every (P,Q) element is
// independent; the stage is bound by HBM (3 N_k complex values move per
// element against ~6 N_k L flops).  Forms, fastest first:
//   kconv_herm_kernel  Hermitian D^k and V^q (so M^k Hermitian), meshes 2^3,
//                      3^3, 4^3, N_P even: TMA-fed tiles that reach the
//                      diagonal, M mirrored through shared memory, row
//                      exponents of M from per-tile keys; on 2^3 and 4^3
//                      meshes an extended form (X) also writes M's fp16
//                      remainders, the DFTs run exactly on an 18-bit split
//                      of each element (see split_magic)
//   kconv_pipe_kernel  the same meshes, any V: TMA-fed batches of consecutive
//                      elements, row exponents of M folded in
//   kconv_tile_kernel  other meshes with N_k <= 256 (6^3 among them), N_P^2
//                      even: TMA-fed batches of 32 elements, the 3-D DFT in
//                      place in shared memory (lengths 6 by Good-Thomas)
//   kconv_lanes_kernel the same meshes as kconv_pipe_kernel without TMA (N1
//                      lanes per element, first axis by shuffles)
//   kconv_kernel       any mesh: one thread per element, its N_k values in
//                      shared memory ([k][thread], conflict-free)
// All run the separable 3-D DFT axis by axis with radix-2/3/4 butterflies or
// a direct DFT for other lengths, multiply by Vh and transform back.
//
// FP32 form: a 2- or 4-point DFT has twiddles 1, -1, +-i and is exact up to the
// additions; the only irrational twiddles (sqrt(3)/2 for lengths 3 and 6, the
// table for lengths 5, 7, 8) are applied as an FP32 hi + lo pair so that the
// forward and inverse transforms do not pick up a systematic scale error.
//
#include "thc_internal.cuh"
#include "mbarrier.cuh"
#include "tc_gemm.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <math.h>

#include <algorithm>
#include <cstring>

namespace {

constexpr int MAXL = 8;

struct Twiddles {
  int n[3];
  double c[3][MAXL], s[3][MAXL];      // cos, sin of 2 pi r / n_ax
  float ch[3][MAXL], cl[3][MAXL];     // FP32 hi/lo split of c
  float sh[3][MAXL], sl[3][MAXL];
};

template <typename R> struct Tw;
template <> struct Tw<double> {
  __device__ static double2 mul(double2 v, const Twiddles& t, int ax, int r, int sign) {
    double c = t.c[ax][r], s = sign * t.s[ax][r];
    return make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
  __device__ static double2 mul_s3(double2 d, int sign) {
    // i * sign * sqrt(3)/2 * d
    const double h = 0.86602540378443864676;
    return make_double2(-sign * h * d.y, sign * h * d.x);
  }
};
template <> struct Tw<float> {
  __device__ static float2 mul(float2 v, const Twiddles& t, int ax, int r, int sign) {
    float ch = t.ch[ax][r], cl = t.cl[ax][r];
    float sh = sign * t.sh[ax][r], sl = sign * t.sl[ax][r];
    float re = fmaf(v.x, ch, -v.y * sh) + (v.x * cl - v.y * sl);
    float im = fmaf(v.x, sh, v.y * ch) + (v.x * sl + v.y * cl);
    return make_float2(re, im);
  }
  __device__ static float2 mul_s3(float2 d, int sign) {
    const float hh = 0.866025388240814208984375f;       // float(sqrt(3)/2)
    const float hl = 1.5543625e-8f;                     // sqrt(3)/2 - hh
    float re = -(d.y * hh + d.y * hl);
    float im = d.x * hh + d.x * hl;
    return make_float2(sign * re, sign * im);
  }
};

template <typename R, int L>
__device__ __forceinline__ void line_dft(typename cplx<R>::type* x, int step, const Twiddles& tw,
                                         int ax, int sign) {
  typedef typename cplx<R>::type CT;
  CT v[L];
#pragma unroll
  for (int j = 0; j < L; j++) v[j] = x[j * step];
  if constexpr (L == 2) {
    x[0] = cadd(v[0], v[1]);
    x[step] = csub(v[0], v[1]);
  } else if constexpr (L == 3) {
    CT t = cadd(v[1], v[2]);
    CT d = csub(v[1], v[2]);
    CT m = CT{v[0].x - (R)0.5 * t.x, v[0].y - (R)0.5 * t.y};
    CT s = Tw<R>::mul_s3(d, sign);
    x[0] = cadd(v[0], t);
    x[step] = cadd(m, s);
    x[2 * step] = csub(m, s);
  } else if constexpr (L == 4) {
    CT a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    CT b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
    CT ib1 = CT{-sign * b1.y, sign * b1.x};   // i * sign * b1
    x[0] = cadd(a0, b0);
    x[2 * step] = csub(a0, b0);
    x[step] = cadd(a1, ib1);
    x[3 * step] = csub(a1, ib1);
  } else if constexpr (L == 6) {
    // prime-factor (Good-Thomas) 6 = 2 x 3, no twiddles between the factors:
    // inputs n = (3 n1 + 2 n2) mod 6, outputs m = (3 m1 + 4 m2) mod 6,
    // X[m] = sum_{n1} (-1)^{n1 m1} sum_{n2} x[n] w3^{n2 m2}
    CT y0[3], y1[3];
    auto dft3v = [&](CT a, CT b, CT c, CT* y) {
      const CT t = cadd(b, c), d = csub(b, c);
      const CT m = CT{a.x - (R)0.5 * t.x, a.y - (R)0.5 * t.y};
      const CT sd = Tw<R>::mul_s3(d, sign);
      y[0] = cadd(a, t);
      y[1] = cadd(m, sd);
      y[2] = csub(m, sd);
    };
    dft3v(v[0], v[2], v[4], y0);
    dft3v(v[3], v[5], v[1], y1);
    x[0] = cadd(y0[0], y1[0]);
    x[3 * step] = csub(y0[0], y1[0]);
    x[4 * step] = cadd(y0[1], y1[1]);
    x[step] = csub(y0[1], y1[1]);
    x[2 * step] = cadd(y0[2], y1[2]);
    x[5 * step] = csub(y0[2], y1[2]);
  } else {
#pragma unroll
    for (int m = 0; m < L; m++) {
      CT acc = v[0];
#pragma unroll
      for (int j = 1; j < L; j++) acc = cadd(acc, Tw<R>::mul(v[j], tw, ax, (j * m) % L, sign));
      x[m * step] = acc;
    }
  }
}

template <typename R>
__device__ void dft_axis(typename cplx<R>::type* x, int T, const Twiddles& tw, int ax, int sign) {
  const int n1 = tw.n[0], n2 = tw.n[1], n3 = tw.n[2];
  const int L = tw.n[ax];
  if (L == 1) return;
  int nout, sout, nin, sin_, step;
  if (ax == 0) { nout = n2; sout = n3; nin = n3; sin_ = 1; step = n2 * n3; }
  else if (ax == 1) { nout = n1; sout = n2 * n3; nin = n3; sin_ = 1; step = n3; }
  else { nout = n1; sout = n2 * n3; nin = n2; sin_ = n3; step = 1; }
  for (int o = 0; o < nout; o++)
    for (int i = 0; i < nin; i++) {
      typename cplx<R>::type* base = x + (long)(o * sout + i * sin_) * T;
      const int st = step * T;
      switch (L) {
        case 2: line_dft<R, 2>(base, st, tw, ax, sign); break;
        case 3: line_dft<R, 3>(base, st, tw, ax, sign); break;
        case 4: line_dft<R, 4>(base, st, tw, ax, sign); break;
        case 5: line_dft<R, 5>(base, st, tw, ax, sign); break;
        case 6: line_dft<R, 6>(base, st, tw, ax, sign); break;
        case 7: line_dft<R, 7>(base, st, tw, ax, sign); break;
        default: line_dft<R, 8>(base, st, tw, ax, sign); break;
      }
    }
}

template <typename R>
__device__ __forceinline__ void dft3(typename cplx<R>::type* x, int T, const Twiddles& tw, int sign) {
  dft_axis<R>(x, T, tw, 0, sign);
  dft_axis<R>(x, T, tw, 1, sign);
  dft_axis<R>(x, T, tw, 2, sign);
}

// M = IDFT(DFT(D) o Vh), one element per thread, values in shared memory.
template <typename R>
__global__ void kconv_kernel(const typename cplx<R>::type* __restrict__ D,
                             const typename cplx<R>::type* __restrict__ Vh,
                             typename cplx<R>::type* __restrict__ M, long npq, Twiddles tw) {
  typedef typename cplx<R>::type CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* buf = reinterpret_cast<CT*>(smem_raw);
  const int T = blockDim.x, tid = threadIdx.x;
  const int nk = tw.n[0] * tw.n[1] * tw.n[2];
  const long e = (long)blockIdx.x * T + tid;
  const bool ok = e < npq;
  CT* x = buf + tid;
  // unrolled so that many independent loads are in flight per thread
#pragma unroll 16
  for (int k = 0; k < nk; k++) x[(long)k * T] = ok ? D[(long)k * npq + e] : CT{(R)0, (R)0};
  dft3<R>(x, T, tw, -1);
#pragma unroll 16
  for (int a = 0; a < nk; a++) {
    CT v = ok ? Vh[(long)a * npq + e] : CT{(R)0, (R)0};
    x[(long)a * T] = cmul(x[(long)a * T], v);
  }
  dft3<R>(x, T, tw, +1);
  if (ok)
    for (int k = 0; k < nk; k++) M[(long)k * npq + e] = x[(long)k * T];
}

// Lane-split FP32 form for the meshes 2^3, 3^3 and 4^3 (compile-time N1, N2,
// N3).  N1 lanes of a warp share one element: lane slot t holds the N2 N3
// values with first mesh index t, in registers.  The DFT along the first axis
// runs across the N1 lanes (each lane gathers the N1 values by shuffles and
// keeps output t), the other two axes run locally.  Lane l of a warp is slot
// l / EPW of element l % EPW, so the lanes of one slot read EPW consecutive
// elements of one k plane.  Both D and Vh are loaded up front, so a warp
// waits for DRAM once, and no shared memory holds the data.
// Output m of the N1-point DFT of v (the same operations as line_dft).
template <int N1>
__device__ __forceinline__ float2 dft_one(const float2* v, int m, int sign, const Twiddles& tw) {
  if constexpr (N1 == 2) {
    return m ? csub(v[0], v[1]) : cadd(v[0], v[1]);
  } else if constexpr (N1 == 3) {
    const float2 t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 h = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    const float2 r = Tw<float>::mul_s3(d, sign);
    return m == 0 ? cadd(v[0], t) : m == 1 ? cadd(h, r) : csub(h, r);
  } else {
    static_assert(N1 == 4, "lane-split meshes are 2^3, 3^3 and 4^3");
    const bool odd = m & 1;
    const float2 a = odd ? csub(v[0], v[2]) : cadd(v[0], v[2]);
    const float2 b = odd ? csub(v[1], v[3]) : cadd(v[1], v[3]);
    const float2 bb = odd ? make_float2(-sign * b.y, sign * b.x) : b;   // i * sign * b for odd m
    return (m & 2) ? csub(a, bb) : cadd(a, bb);
  }
}

// The DFTs along the second and third mesh axes of one lane's N2 N3 values.
template <int N2, int N3>
__device__ __forceinline__ void local_dfts(float2* x, const Twiddles& tw, int sign) {
  if constexpr (N2 > 1) {
#pragma unroll
    for (int i = 0; i < N3; i++) line_dft<float, N2>(x + i, N3, tw, 1, sign);
  }
  if constexpr (N3 > 1) {
#pragma unroll
    for (int i = 0; i < N2; i++) line_dft<float, N3>(x + i * N3, 1, tw, 2, sign);
  }
}

// The convolution of one element on N1 lanes: x (this lane's N2 N3 values of
// D, first mesh index = slot) becomes this lane's values of M.
template <int N1, int N2, int N3>
__device__ __forceinline__ void lanes_convolve(float2* x, const float2* vh, const Twiddles& tw, int slot,
                                               int el) {
  constexpr int L = N2 * N3, EPW = 32 / N1;
  // DFT along the first axis across the lanes: gather the N1 values by shuffles
  auto across = [&](int sign) {
#pragma unroll
    for (int j = 0; j < L; j++) {
      float2 v[N1];
#pragma unroll
      for (int t = 0; t < N1; t++) {
        v[t].x = __shfl_sync(0xffffffffu, x[j].x, t * EPW + el);
        v[t].y = __shfl_sync(0xffffffffu, x[j].y, t * EPW + el);
      }
      x[j] = dft_one<N1>(v, slot, sign, tw);
    }
  };
  across(-1);
  local_dfts<N2, N3>(x, tw, -1);
#pragma unroll
  for (int j = 0; j < L; j++) x[j] = cmul(x[j], vh[j]);
  local_dfts<N2, N3>(x, tw, +1);
  across(+1);
}

template <int N1, int N2, int N3>
__global__ void __launch_bounds__(256, 2) kconv_lanes_kernel(const float2* __restrict__ D,
                                                          const float2* __restrict__ Vh, float2* __restrict__ M,
                                                          long npq, Twiddles tw) {
  constexpr int L = N2 * N3, EPW = 32 / N1, EPB = EPW * 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / EPW;                       // first mesh index of this lane's values
  const int el = lane - slot * EPW;                  // element within the warp
  const bool live = slot < N1;                       // lanes past EPW N1 idle
  const long e = (long)blockIdx.x * EPB + warp * EPW + el;
  const bool ok = live && e < npq;
  const long off = (long)(live ? slot : 0) * L * npq + e;
  float2 x[L], vh[L];
#pragma unroll
  for (int j = 0; j < L; j++) x[j] = ok ? __ldcs(D + off + (long)j * npq) : make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < L; j++) vh[j] = ok ? __ldcs(Vh + off + (long)j * npq) : make_float2(0.f, 0.f);
  lanes_convolve<N1, N2, N3>(x, vh, tw, slot, el);
  if (ok) {
#pragma unroll
    for (int j = 0; j < L; j++) M[off + (long)j * npq] = x[j];
  }
}

// Row-exponent key of a value pair's max(|re|, |im|): the top 16 bits of its
// FP32 pattern (sign 0, exponent, 7 mantissa bits), which orders as the value
// does and fixes its frexp exponent whenever the value is at least 2^-133.
__device__ __forceinline__ uint32_t abs_bits(float2 v) {
  return max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu);
}

// Persistent, TMA-fed form of the lane-split convolution (N_P^2 even).  A
// batch is EPB consecutive elements of all N_k planes; one 2-D box of D and
// one of Vh ([N_k][EPB] complex, zero past the end) land in shared memory
// while the block convolves the batch before, so each SM keeps two boxes in
// flight instead of waiting on DRAM once per element.  Each block takes a
// contiguous range of batches.  The DFT along the first mesh axis reads the
// N1 values of an element straight from the D box (one broadcast load each,
// every lane keeping its own output) and, on the way back, from a scratch
// area where the warp's lanes left their values ([j][element][slot], the
// slot index XORed so that the loads of one value index hit distinct banks):
// no shuffles.
//
// With rowkey (np rows of np elements per k), it also folds the row
// exponents of M: rowkey[k * np + p] = the largest abs_bits key over
// M^k[p][q], q < np.  The EPW lanes of one slot reduce the keys of a warp
// whose elements lie in one row by shuffles (two keys per word); the slot's
// first lane keeps the running maximum of its row across the block's batches
// in registers and adds it to memory by atomicMax when the row changes.
// Every mbarrier wait is bounded; on expiry the block sets the error word,
// waits (bounded) for its copy in flight and returns.
template <int N1, int N2, int N3>
__global__ void __launch_bounds__(256, 2) kconv_pipe_kernel(const __grid_constant__ CUtensorMap mapD,
                                                         const __grid_constant__ CUtensorMap mapV,
                                                         float2* __restrict__ M, long npq, long nbatch,
                                                         Twiddles tw, unsigned* __restrict__ rowkey, int np,
                                                         int* err) {
  constexpr int L = N2 * N3, NK = N1 * L, EPW = 32 / N1, EPB = EPW * 8, LP = (L + 1) / 2;
  constexpr uint32_t BOX = NK * EPB * sizeof(float2);
  extern __shared__ __align__(128) unsigned char kc_smem[];   // [D box][Vh box][scratch][mbarrier]
  const float2* sD = reinterpret_cast<const float2*>(kc_smem);
  const float2* sV = reinterpret_cast<const float2*>(kc_smem + BOX);
  float2* scr = reinterpret_cast<float2*>(kc_smem + 2 * BOX);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / EPW, el = lane - slot * EPW;
  const bool live = slot < N1;
  const int eloc = warp * EPW + el;                                  // element within the batch
  const int sbase = (live ? slot : 0) * L * EPB + eloc;               // this lane's first value in a box
  // scratch slot swizzle: the second half of a warp's elements XORs the slot
  constexpr int SW = N1 == 4 ? 2 : N1 == 2 ? 1 : 0;
  const int sw = el >= EPW / 2 ? SW : 0;
  const long b0 = nbatch * blockIdx.x / gridDim.x, b1 = nbatch * (blockIdx.x + 1) / gridDim.x;
  const uint32_t bar = smem_u32(kc_smem + 3 * BOX);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](long bt) {
    mbar_expect_tx(bar, 2 * BOX);
    tma_load_2d(smem_u32(sD), &mapD, bar, (int)(2 * bt * EPB), 0);
    tma_load_2d(smem_u32(sV), &mapV, bar, (int)(2 * bt * EPB), 0);
  };
  if (threadIdx.x == 0 && b0 < b1) issue(b0);
  uint32_t acc[LP];
#pragma unroll
  for (int i = 0; i < LP; i++) acc[i] = 0u;
  long acc_row = -1;
  auto flush = [&]() {
    if (acc_row >= 0) {
#pragma unroll
      for (int i = 0; i < LP; i++) {
        const uint32_t lo = acc[i] & 0xffffu, hi = acc[i] >> 16;
        if (lo) atomicMax(rowkey + (long)(slot * L + 2 * i) * np + acc_row, lo);
        if (hi) atomicMax(rowkey + (long)(slot * L + 2 * i + 1) * np + acc_row, hi);
      }
    }
  };
  bool good = true;
  uint32_t fail_parity = 0;
  for (long bt = b0; bt < b1; bt++) {
    fail_parity = (uint32_t)((bt - b0) & 1);
    good = mbar_wait_warp(bar, fail_parity, err, 1024);
    good = __syncthreads_and(good);
    if (!good) break;
    float2 x[L], vh[L];
    // forward DFT along the first axis, this lane's output, from the D box
#pragma unroll
    for (int j = 0; j < L; j++) {
      float2 v[N1];
#pragma unroll
      for (int t = 0; t < N1; t++) v[t] = sD[(t * L + j) * EPB + eloc];
      x[j] = dft_one<N1>(v, live ? slot : 0, -1, tw);
    }
#pragma unroll
    for (int j = 0; j < L; j++) vh[j] = live ? sV[sbase + j * EPB] : make_float2(0.f, 0.f);
    __syncthreads();                                   // the boxes are free for the next batch
    if (threadIdx.x == 0 && bt + 1 < b1) issue(bt + 1);
    local_dfts<N2, N3>(x, tw, -1);
#pragma unroll
    for (int j = 0; j < L; j++) x[j] = cmul(x[j], vh[j]);
    local_dfts<N2, N3>(x, tw, +1);
    // inverse DFT along the first axis through the scratch (the warp's own elements)
    if (live) {
#pragma unroll
      for (int j = 0; j < L; j++) scr[(j * EPB + eloc) * N1 + (slot ^ sw)] = x[j];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < L; j++) {
      float2 v[N1];
#pragma unroll
      for (int t = 0; t < N1; t++) v[t] = scr[(j * EPB + eloc) * N1 + (t ^ sw)];
      x[j] = dft_one<N1>(v, live ? slot : 0, +1, tw);
    }
    const long ew = bt * EPB + warp * EPW;             // the warp's first element
    const long e = ew + el;
    const bool ok = live && e < npq;
    if (ok) {
      const long off = (long)slot * L * npq + e;
#pragma unroll
      for (int j = 0; j < L; j++) __stcs(M + off + (long)j * npq, x[j]);
    }
    if (rowkey) {
      uint32_t w[LP];
#pragma unroll
      for (int i = 0; i < LP; i++)
        w[i] = __byte_perm(abs_bits(x[2 * i]), 2 * i + 1 < L ? abs_bits(x[2 * i + 1 < L ? 2 * i + 1 : 0]) : 0u,
                           0x7632);
      const bool one = ew < npq && ew / np == (std::min(ew + EPW, npq) - 1) / np;   // warp-uniform
      if (one) {
#pragma unroll
        for (int o = 1; o < EPW; o <<= 1) {
#pragma unroll
          for (int i = 0; i < LP; i++) {
            const uint32_t t = __shfl_down_sync(0xffffffffu, w[i], o);
            if (el + o < EPW) w[i] = __vmaxu2(w[i], t);
          }
        }
        if (el == 0 && live) {
          const long row = ew / np;
          if (row != acc_row) {
            flush();
            acc_row = row;
#pragma unroll
            for (int i = 0; i < LP; i++) acc[i] = w[i];
          } else {
#pragma unroll
            for (int i = 0; i < LP; i++) acc[i] = __vmaxu2(acc[i], w[i]);
          }
        }
      } else if (ok) {                                 // a warp across rows: one atomic per value
        const long row = e / np;
#pragma unroll
        for (int i = 0; i < LP; i++) {
          if (w[i] & 0xffffu) atomicMax(rowkey + (long)(slot * L + 2 * i) * np + row, w[i] & 0xffffu);
          if (w[i] >> 16) atomicMax(rowkey + (long)(slot * L + 2 * i + 1) * np + row, w[i] >> 16);
        }
      }
    }
  }
  if (rowkey && el == 0 && live) flush();
  // the copy of the batch whose wait gave up may still be in flight
  if (!good && threadIdx.x == 0) mbar_drain(bar, fail_parity);
}

// TMA-fed shared-memory form for the other meshes (N_k <= 256, N_P^2 even):
// a batch is TILE_EPB = 32 consecutive (P, Q) elements of all N_k planes; one
// 2-D box of D and one of Vh ([N_k][32] complex) land in shared memory, and
// the 3-D DFT runs in place there, axis by axis: warp w takes the lines w,
// w + 8, ... of an axis and lane l the element l of each, so every access of
// a warp is 256 contiguous bytes.  Two blocks per SM (for N_k <= 216) each
// keep one batch in flight.  M leaves from shared memory in 256-byte rows, and
// the row keys of M (as rowkey of kconv_pipe_kernel) are reduced per k plane
// by the warp and kept per block while consecutive batches stay in one row.
constexpr int TILE_EPB = 32;

template <typename R>
__device__ __forceinline__ void smem_line(float2* x, int L, int step, const Twiddles& tw, int ax, int sign) {
  switch (L) {
    case 2: line_dft<float, 2>(x, step, tw, ax, sign); break;
    case 3: line_dft<float, 3>(x, step, tw, ax, sign); break;
    case 4: line_dft<float, 4>(x, step, tw, ax, sign); break;
    case 5: line_dft<float, 5>(x, step, tw, ax, sign); break;
    case 6: line_dft<float, 6>(x, step, tw, ax, sign); break;
    case 7: line_dft<float, 7>(x, step, tw, ax, sign); break;
    default: line_dft<float, 8>(x, step, tw, ax, sign); break;
  }
}

// The DFT of all elements of the box along every mesh axis (sign -1 forward,
// +1 inverse); the box is [k][TILE_EPB] with k = (i1 n2 + i2) n3 + i3.
__device__ __forceinline__ void tile_dft3(float2* box, const Twiddles& tw, int sign, int warp, int lane) {
  const int n1 = tw.n[0], n2 = tw.n[1], n3 = tw.n[2];
  const int nk = n1 * n2 * n3;
#pragma unroll 1
  for (int ax = 0; ax < 3; ax++) {
    const int L = tw.n[ax];
    if (L > 1) {
      const int nl = nk / L;                         // lines along this axis
      for (int l = warp; l < nl; l += 8) {
        int base, st;
        if (ax == 0) { base = l; st = n2 * n3; }                                  // l = i2 n3 + i3
        else if (ax == 1) { base = (l / n3) * n2 * n3 + (l % n3); st = n3; }       // l = i1 n3 + i3
        else { base = l * n3; st = 1; }                                           // l = i1 n2 + i2
        smem_line<float>(box + base * TILE_EPB + lane, L, st * TILE_EPB, tw, ax, sign);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) kconv_tile_kernel(const __grid_constant__ CUtensorMap mapD,
                                                      const __grid_constant__ CUtensorMap mapV,
                                                      float2* __restrict__ M, long npq, long nbatch, Twiddles tw,
                                                      unsigned* __restrict__ rowkey, int np, int* err) {
  const int nk = tw.n[0] * tw.n[1] * tw.n[2];
  const uint32_t box_bytes = (uint32_t)nk * TILE_EPB * sizeof(float2);
  extern __shared__ __align__(128) unsigned char kt_smem[];   // [D box][Vh box][row maxima][mbarrier]
  float2* sD = reinterpret_cast<float2*>(kt_smem);
  const float2* sV = reinterpret_cast<const float2*>(kt_smem + box_bytes);
  unsigned* rmax = reinterpret_cast<unsigned*>(kt_smem + 2 * box_bytes);
  const uint32_t bar = smem_u32(kt_smem + 2 * box_bytes + ((nk * 4 + 15) & ~15));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long b0 = nbatch * blockIdx.x / gridDim.x, b1 = nbatch * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  for (int k = threadIdx.x; k < nk; k += blockDim.x) rmax[k] = 0u;
  __syncthreads();
  auto issue = [&](long bt) {
    mbar_expect_tx(bar, 2 * box_bytes);
    tma_load_2d(smem_u32(sD), &mapD, bar, (int)(2 * bt * TILE_EPB), 0);
    tma_load_2d(smem_u32(sV), &mapV, bar, (int)(2 * bt * TILE_EPB), 0);
  };
  if (threadIdx.x == 0 && b0 < b1) issue(b0);
  long cur_row = -1;                     // the row whose maxima rmax holds (block-uniform)
  bool good = true;
  uint32_t fail_parity = 0;
  for (long bt = b0; bt < b1; bt++) {
    fail_parity = (uint32_t)((bt - b0) & 1);
    good = mbar_wait_warp(bar, fail_parity, err, 4096);
    good = __syncthreads_and(good);
    if (!good) break;
    tile_dft3(sD, tw, -1, warp, lane);
    for (int k = warp; k < nk; k += 8) sD[k * TILE_EPB + lane] = cmul(sD[k * TILE_EPB + lane], sV[k * TILE_EPB + lane]);
    __syncthreads();
    tile_dft3(sD, tw, +1, warp, lane);
    // M out, and the row keys: warp w owns the k planes w, w + 8, ... of rmax
    const long e0 = bt * TILE_EPB, e = e0 + lane;
    const long rfirst = e0 / np, rlast = (min(e0 + TILE_EPB, npq) - 1) / np;
    if (rowkey && rfirst != cur_row && cur_row >= 0) {
      for (int k = warp; k < nk; k += 8)
        if (lane == 0 && rmax[k]) atomicMax(rowkey + (long)k * np + cur_row, rmax[k]);
      for (int k = warp; k < nk; k += 8)
        if (lane == 0) rmax[k] = 0u;
    }
    for (int k = warp; k < nk; k += 8) {
      const float2 v = sD[k * TILE_EPB + lane];
      unsigned key = 0u;
      if (e < npq) {
        M[(long)k * npq + e] = v;
        key = abs_bits(v) >> 16;
      }
      if (rowkey) {
        if (rfirst == rlast) {
          key = __reduce_max_sync(0xffffffffu, key);
          if (lane == 0) rmax[k] = max(rmax[k], key);
        } else {
          // a batch across a row boundary: each row's part straight to memory
          const bool first = e / np == rfirst;
          const unsigned ka = __reduce_max_sync(0xffffffffu, first ? key : 0u);
          const unsigned kb = __reduce_max_sync(0xffffffffu, first ? 0u : key);
          if (lane == 0) {
            if (ka) atomicMax(rowkey + (long)k * np + rfirst, ka);
            if (kb) atomicMax(rowkey + (long)k * np + rlast, kb);
          }
        }
      }
    }
    if (rfirst == rlast) cur_row = rfirst;
    __syncthreads();                      // the boxes are free again
    if (threadIdx.x == 0 && bt + 1 < b1) issue(bt + 1);
  }
  if (rowkey && cur_row >= 0)
    for (int k = warp; k < nk; k += 8)
      if (lane == 0 && rmax[k]) atomicMax(rowkey + (long)k * np + cur_row, rmax[k]);
  // the copy of the batch whose wait gave up may still be in flight
  if (!good && threadIdx.x == 0) mbar_drain(bar, fail_parity);
}

// Exponent of a 16-bit row key (abs_bits >> 16): the frexp exponent of any
// value of at least 2^-133 with that key, else 0.
__device__ __forceinline__ int key_exponent(unsigned k) {
  return k >= 0x80u ? (int)(k >> 7) - 126 : k ? (32 - __clz((int)k)) - 133 : 0;
}

// First column tile of row tile pb that reaches the diagonal (its last column
// >= the tile's first row); tiles are 8 rows by EPW columns.
__host__ __device__ __forceinline__ int herm_qb0(int pb, int epw) {
  const int x = 8 * pb - (epw - 1);
  return x > 0 ? (x + epw - 1) / epw : 0;
}

// Extended form of the convolution (radix-2/4 meshes, where every DFT is made
// of additions, subtractions and multiplications by +-i).  Each element's
// values are split into a part on the grid of 2^(e - 18), e the exponent of
// the element's largest component (|x| < 2^e), and the remainder.  The DFTs
// of the first part are exact in FP32: a 64-point DFT grows values by at most
// 2^6, so every sum stays an integer multiple of the grid below 2^24 of it.
// The remainders are at most 2^-18 of the largest value, so their DFTs' FP32
// roundings sit near 2^-42 of it.  The product with the prepared kernel is
// formed with error-free products (an FMA gives each product's rounding
// error), so M leaves as an FP32 value and the part of its error below
// 2^-24, which is stored as an fp16 multiple of the value's unit in the last
// place (mlo_scale).

// 1.5 * 2^(e + 5): adding and subtracting it rounds |x| < 2^e to a multiple of
// 2^(e - 18).
__device__ __forceinline__ float split_magic(float mx) {
  int e;
  frexpf(mx, &e);
  e = max(-100, min(e, 100));
  return 1.5f * __int_as_float((e + 5 + 127) << 23);
}
__device__ __forceinline__ float2 split_hi(float2 v, float c) {
  return make_float2(__fsub_rn(__fadd_rn(v.x, c), c), __fsub_rn(__fadd_rn(v.y, c), c));
}
// the largest component of the element held by the N1 slot lanes (EPW apart)
template <int N1, int L>
__device__ __forceinline__ float element_max(const float2* x) {
  constexpr int EPW = 32 / N1;
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < L; j++) m = fmaxf(m, fmaxf(fabsf(x[j].x), fabsf(x[j].y)));
#pragma unroll
  for (int o = EPW; o < 32; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}
// (h + l) * v with the rounding of the h * v products kept: returns the FP32
// product in ph and everything below it in pl.
__device__ __forceinline__ void cmul_x(float2 h, float2 l, float2 v, float2& ph, float2& pl) {
  const float p1 = h.x * v.x, e1 = fmaf(h.x, v.x, -p1);
  const float p2 = h.y * v.y, e2 = fmaf(h.y, v.y, -p2);
  const float p3 = h.x * v.y, e3 = fmaf(h.x, v.y, -p3);
  const float p4 = h.y * v.x, e4 = fmaf(h.y, v.x, -p4);
  // two-sums p1 - p2 and p3 + p4
  const float r = __fsub_rn(p1, p2), rb = __fsub_rn(r, p1), re_err = __fadd_rn(__fsub_rn(p1, __fsub_rn(r, rb)), __fsub_rn(-p2, rb));
  const float i = __fadd_rn(p3, p4), ib = __fsub_rn(i, p3), im_err = __fadd_rn(__fsub_rn(p3, __fsub_rn(i, ib)), __fsub_rn(p4, ib));
  ph = make_float2(r, i);
  pl = make_float2((e1 - e2) + re_err + (l.x * v.x - l.y * v.y), (e3 + e4) + im_err + (l.x * v.y + l.y * v.x));
}
// The remainder l of a value h as an fp16 multiple of h's unit in the last
// place, 2^(e(h) - 24) with h = m 2^e(h), 1/2 <= m < 1 (0 for h = 0 or a
// remainder outside what it can carry).
__device__ __forceinline__ uint16_t mlo_scale(float h, float l) {
  const int eh = (int)((__float_as_uint(h) >> 23) & 0xffu);
  if (eh < 24 || eh == 0xffu) return 0;   // |h| < 2^-103 (or not finite): nothing to carry
  // l * 2^(24 - e(h)) with e(h) = eh - 126
  const float q = l * __int_as_float((150 - eh + 127) << 23);
  return __half_as_ushort(__float2half_rn(q));
}

// out = M + its fp16 remainders (the extended form's pair), complex128.
__global__ void mlo_combine_kernel(const float2* __restrict__ M, const uint32_t* __restrict__ Mlo,
                                   double2* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 h = M[i];
    const uint32_t q = Mlo[i];
    auto one = [](float x, uint16_t qq) {
      const int eh = (int)((__float_as_uint(x) >> 23) & 0xffu);
      return (double)x + (eh >= 24 ? ldexp((double)__half2float(__ushort_as_half(qq)), eh - 150) : 0.0);
    };
    out[i] = make_double2(one(h.x, (uint16_t)(q & 0xffffu)), one(h.y, (uint16_t)(q >> 16)));
  }
}

// Hermitian form of the TMA-fed convolution, for D^k and V^q Hermitian (so
// that M^k is too): only the tiles of 8 rows P by EPW columns Q that reach the
// diagonal are loaded (3-D boxes [N_k][8][EPW] of D and Vh, zero past the
// ends), which halves the bytes read; each lane writes its value of M for
// Q >= P and the conjugate at (Q, P) for Q > P.  Warp w holds row 8 pb + w,
// so the box layout [k][w * EPW + el] is that of the flat form.  Row
// exponents: every tile stores, with plain coalesced stores, the row keys of
// its rows (max over its elements with Q >= P) in rowk[P][qb][..] and the
// column keys of its columns (max over its elements with Q > P, the mirrored
// part of row Q) in colk[Q][pb][..], KWR words per row ([slot][LP] pairs of
// 16-bit keys); herm_keys_to_exponents takes the maxima.
// X (extended form, N1 = 2 or 4): also writes Mlo, the fp16 remainders of M
// (mlo_scale), [N_k][np][np] pairs (re, im).
template <int N1, int N2, int N3, bool X>
__global__ void __launch_bounds__(256, 2) kconv_herm_kernel(const __grid_constant__ CUtensorMap mapD,
                                                         const __grid_constant__ CUtensorMap mapV,
                                                         float2* __restrict__ M, int np, long ntile, Twiddles tw,
                                                         uint32_t* __restrict__ rowk, uint32_t* __restrict__ colk,
                                                         const int* __restrict__ tcum, int* err,
                                                         uint32_t* __restrict__ Mlo) {
  static_assert(!X || N1 == 2 || N1 == 4, "the extended form needs radix-2/4 meshes");
  constexpr int L = N2 * N3, NK = N1 * L, EPW = 32 / N1, EPB = EPW * 8, LP = (L + 1) / 2, KWR = N1 * LP;
  constexpr uint32_t BOX = NK * EPB * sizeof(float2);
  extern __shared__ __align__(128) unsigned char kc_smem[];   // [D box][Vh box][scratch][column keys][mbarrier]
  const float2* sD = reinterpret_cast<const float2*>(kc_smem);
  const float2* sV = reinterpret_cast<const float2*>(kc_smem + BOX);
  float2* scr = reinterpret_cast<float2*>(kc_smem + 2 * BOX);
  uint32_t* ckey = reinterpret_cast<uint32_t*>(kc_smem + 3 * BOX);   // [warp][lane][LP]
  const uint32_t bar = smem_u32(kc_smem + 3 * BOX + 8 * 32 * LP * 4);
  int* tnext = reinterpret_cast<int*>(kc_smem + 3 * BOX + 8 * 32 * LP * 4 + 8);   // (pb, qb) of the next tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / EPW, el = lane - slot * EPW;
  const bool live = slot < N1;
  const int eloc = warp * EPW + el;
  const int sbase = (live ? slot : 0) * L * EPB + eloc;
  constexpr int SW = N1 == 4 ? 2 : N1 == 2 ? 1 : 0;
  const int sw = el >= EPW / 2 ? SW : 0;
  auto tsw = [](int k, int c) { return (EPW == 8 ? (c >> 1) + 2 * (k / L) : (k * EPW + c) >> 1) & 7; };
  const int npb = (np + 7) / 8, nqb = (np + EPW - 1) / EPW;
  // tiles are dealt round robin, so that the blocks running side by side read
  // neighbouring tiles (DRAM pages) at the same time; tile t is (pb, qb) with
  // tcum[pb] <= t < tcum[pb + 1], found by bisection
  auto locate = [&](long t, int& lpb, int& lqb) {
    int lo = 0, hi = npb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tcum[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    lpb = lo;
    lqb = herm_qb0(lo, EPW) + (int)(t - tcum[lo]);
  };
  auto issue = [&](int tpb, int tqb) {
    mbar_expect_tx(bar, 2 * BOX);
    tma_load_3d(smem_u32(sD), &mapD, bar, 2 * EPW * tqb, 8 * tpb, 0);
    tma_load_3d(smem_u32(sV), &mapV, bar, 2 * EPW * tqb, 8 * tpb, 0);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    if ((long)blockIdx.x < ntile) {
      int a, b;
      locate(blockIdx.x, a, b);
      tnext[0] = a;
      tnext[1] = b;
      issue(a, b);
    }
  }
  __syncthreads();
  const long npq = (long)np * np;
  bool good = true;
  uint32_t fail_parity = 0;
  long it = 0;
  for (long t = blockIdx.x; t < ntile; t += gridDim.x, it++) {
    fail_parity = (uint32_t)(it & 1);
    good = mbar_wait_warp(bar, fail_parity, err, 2048);
    good = __syncthreads_and(good);
    if (!good) break;
    const int pb = tnext[0], qb = tnext[1];
    float2 x[L];
    // X: xl holds the remainder part of every value; hi / lo the M pair
    float2 xl[X ? L : 1];
    if constexpr (!X) {
      float2 vh[L];
#pragma unroll
      for (int j = 0; j < L; j++) {
        float2 v[N1];
#pragma unroll
        for (int u = 0; u < N1; u++) v[u] = sD[(u * L + j) * EPB + eloc];
        x[j] = dft_one<N1>(v, live ? slot : 0, -1, tw);
      }
#pragma unroll
      for (int j = 0; j < L; j++) vh[j] = live ? sV[sbase + j * EPB] : make_float2(0.f, 0.f);
      __syncthreads();                                   // the boxes (and tnext) are free for the next tile
      if (threadIdx.x == 0 && t + gridDim.x < ntile) {
        int a, b;
        locate(t + gridDim.x, a, b);
        tnext[0] = a;
        tnext[1] = b;
        issue(a, b);
      }
      local_dfts<N2, N3>(x, tw, -1);
#pragma unroll
      for (int j = 0; j < L; j++) x[j] = cmul(x[j], vh[j]);
      local_dfts<N2, N3>(x, tw, +1);
    } else {
      // the element's own values (this lane's slot) give the split point
#pragma unroll
      for (int j = 0; j < L; j++) x[j] = live ? sD[sbase + j * EPB] : make_float2(0.f, 0.f);
      const float cD = split_magic(element_max<N1, L>(x));
#pragma unroll
      for (int j = 0; j < L; j++) {
        float2 vh[N1], vl[N1];
#pragma unroll
        for (int u = 0; u < N1; u++) {
          const float2 d = sD[(u * L + j) * EPB + eloc];
          vh[u] = split_hi(d, cD);
          vl[u] = csub(d, vh[u]);
        }
        x[j] = dft_one<N1>(vh, live ? slot : 0, -1, tw);
        xl[j] = dft_one<N1>(vl, live ? slot : 0, -1, tw);
      }
      local_dfts<N2, N3>(x, tw, -1);
      local_dfts<N2, N3>(xl, tw, -1);
#pragma unroll
      for (int j = 0; j < L; j++) {
        float2 ph, pl;
        cmul_x(x[j], xl[j], live ? sV[sbase + j * EPB] : make_float2(0.f, 0.f), ph, pl);
        x[j] = ph;
        xl[j] = pl;
      }
      __syncthreads();                                   // the boxes (and tnext) are free for the next tile
      if (threadIdx.x == 0 && t + gridDim.x < ntile) {
        int a, b;
        locate(t + gridDim.x, a, b);
        tnext[0] = a;
        tnext[1] = b;
        issue(a, b);
      }
      // split the products again: the grid part's inverse DFTs are exact
      const float cM = split_magic(element_max<N1, L>(x));
#pragma unroll
      for (int j = 0; j < L; j++) {
        const float2 a = split_hi(x[j], cM);
        xl[j] = cadd(csub(x[j], a), xl[j]);
        x[j] = a;
      }
      local_dfts<N2, N3>(x, tw, +1);
      local_dfts<N2, N3>(xl, tw, +1);
      // the first axis of the remainder part through the scratch (below, the
      // grid part takes the same way)
      if (live) {
#pragma unroll
        for (int j = 0; j < L; j++) scr[(j * EPB + eloc) * N1 + (slot ^ sw)] = xl[j];
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < L; j++) {
        float2 v[N1];
#pragma unroll
        for (int u = 0; u < N1; u++) v[u] = scr[(j * EPB + eloc) * N1 + (u ^ sw)];
        xl[j] = dft_one<N1>(v, live ? slot : 0, +1, tw);
      }
      __syncwarp();
    }
    if (live) {
#pragma unroll
      for (int j = 0; j < L; j++) scr[(j * EPB + eloc) * N1 + (slot ^ sw)] = x[j];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < L; j++) {
      float2 v[N1];
#pragma unroll
      for (int u = 0; u < N1; u++) v[u] = scr[(j * EPB + eloc) * N1 + (u ^ sw)];
      x[j] = dft_one<N1>(v, live ? slot : 0, +1, tw);
    }
    uint32_t lo[X ? L : 1];   // X: the fp16 remainders (re, im) of this lane's values of M
    if constexpr (X) {
#pragma unroll
      for (int j = 0; j < L; j++) {
        const float hx = __fadd_rn(x[j].x, xl[j].x), hy = __fadd_rn(x[j].y, xl[j].y);
        const float lx = __fadd_rn(__fsub_rn(x[j].x, hx), xl[j].x), ly = __fadd_rn(__fsub_rn(x[j].y, hy), xl[j].y);
        x[j] = make_float2(hx, hy);
        lo[j] = (uint32_t)mlo_scale(hx, lx) | ((uint32_t)mlo_scale(hy, ly) << 16);
      }
    }
    const int P = 8 * pb + warp, Q = EPW * qb + el;
    const bool valid = live && P < np && Q < np;
    const bool direct = valid && Q >= P, mirror = valid && Q > P;   // mirror: its conjugate at (Q, P)
    if (direct) {
      const long off = (long)slot * L * npq + (long)P * np + Q;
#pragma unroll
      for (int j = 0; j < L; j++) __stcs(M + off + (long)j * npq, x[j]);
      if constexpr (X) {
#pragma unroll
        for (int j = 0; j < L; j++) __stcs(Mlo + off + (long)j * npq, lo[j]);
      }
    }
    // keys: the row's (Q >= P) reduced over the warp's lanes of each slot, the
    // column's (Q > P) over the warps through shared memory
    uint32_t w[LP];
#pragma unroll
    for (int i = 0; i < LP; i++) {
      const uint32_t k = __byte_perm(abs_bits(x[2 * i]), 2 * i + 1 < L ? abs_bits(x[2 * i + 1 < L ? 2 * i + 1 : 0]) : 0u,
                                     0x7632);
      w[i] = direct ? k : 0u;
      ckey[(warp * 32 + lane) * LP + i] = mirror ? k : 0u;
    }
#pragma unroll
    for (int o = 1; o < EPW; o <<= 1) {
#pragma unroll
      for (int i = 0; i < LP; i++) {
        const uint32_t u = __shfl_down_sync(0xffffffffu, w[i], o);
        if (el + o < EPW) w[i] = __vmaxu2(w[i], u);
      }
    }
    if (el == 0 && live && P < np) {
      uint32_t* dst = rowk + ((long)P * nqb + qb) * KWR + slot * LP;
#pragma unroll
      for (int i = 0; i < LP; i++) dst[i] = w[i];
    }
    // the mirror image goes out row by row: the tile is transposed through the
    // scratch ([k][column][row], the row index XORed by tsw so that the stores
    // of a warp and the loads of 8 consecutive rows hit distinct banks)
    __syncthreads();                                   // every warp has read its part of the scratch
    if (live) {
#pragma unroll
      for (int j = 0; j < L; j++) {
        const int k = slot * L + j;
        scr[(k * EPW + el) * 8 + (warp ^ tsw(k, el))] = x[j];
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NK * EPW * 8; idx += blockDim.x) {
      const int r = idx & 7, c = (idx >> 3) % EPW, k = idx / (8 * EPW);
      const int mP = 8 * pb + r, mQ = EPW * qb + c;
      if (mQ > mP && mQ < np) {
        const float2 v = scr[(k * EPW + c) * 8 + (r ^ tsw(k, c))];
        __stcs(M + ((long)k * np + mQ) * np + mP, make_float2(v.x, -v.y));
      }
    }
    if constexpr (X) {
      // the remainders' mirror image, the same way (conjugate: the imaginary
      // part's sign bit flips)
      uint32_t* scr32 = reinterpret_cast<uint32_t*>(scr);
      __syncthreads();
      if (live) {
#pragma unroll
        for (int j = 0; j < L; j++) {
          const int k = slot * L + j;
          scr32[(k * EPW + el) * 8 + (warp ^ tsw(k, el))] = lo[j];
        }
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < NK * EPW * 8; idx += blockDim.x) {
        const int r = idx & 7, c = (idx >> 3) % EPW, k = idx / (8 * EPW);
        const int mP = 8 * pb + r, mQ = EPW * qb + c;
        if (mQ > mP && mQ < np)
          __stcs(Mlo + ((long)k * np + mQ) * np + mP, scr32[(k * EPW + c) * 8 + (r ^ tsw(k, c))] ^ 0x80000000u);
      }
    }
    for (int idx = threadIdx.x; idx < N1 * EPW * LP; idx += blockDim.x) {
      const int i = idx % LP, ln = idx / LP;          // ln = slot * EPW + column
      const int cs = ln / EPW, cq = EPW * qb + (ln - cs * EPW);
      if (cq >= np) continue;
      uint32_t m = 0u;
#pragma unroll
      for (int v = 0; v < 8; v++) m = __vmaxu2(m, ckey[(v * 32 + ln) * LP + i]);
      colk[((long)cq * npb + pb) * KWR + cs * LP + i] = m;
    }
  }
  if (!good && threadIdx.x == 0) mbar_drain(bar, fail_parity);
}

// e[k * np + P] from the keys of the tiles that hold row P (rowk[P][qb], qb
// from the first tile of row band P / 8 that reaches the diagonal) and of
// those whose mirrored part lands in row P (colk[P][pb], the tiles of column
// band P / EPW): one block of four warps per row, lanes over the key words.
template <int N1, int N2, int N3>
__global__ void __launch_bounds__(128) herm_keys_to_exponents(const uint32_t* __restrict__ rowk,
                                                              const uint32_t* __restrict__ colk, int np,
                                                              int* __restrict__ e) {
  constexpr int L = N2 * N3, EPW = 32 / N1, LP = (L + 1) / 2, KWR = N1 * LP;
  __shared__ uint32_t part[4][32];
  const int nqb = (np + EPW - 1) / EPW, npb = (np + 7) / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int P = blockIdx.x; P < np; P += gridDim.x) {
    uint32_t m0 = 0u, m1 = 0u;
    if (lane < KWR) {
      const uint32_t* r = rowk + (long)P * nqb * KWR + lane;
      int qb = herm_qb0(P / 8, EPW) + warp;
      for (; qb + 4 < nqb; qb += 8) {
        m0 = __vmaxu2(m0, r[(long)qb * KWR]);
        m1 = __vmaxu2(m1, r[(long)(qb + 4) * KWR]);
      }
      if (qb < nqb) m0 = __vmaxu2(m0, r[(long)qb * KWR]);
      const uint32_t* c = colk + (long)P * npb * KWR + lane;
      const int qbP = P / EPW;
      for (int pb = warp; pb < npb && herm_qb0(pb, EPW) <= qbP; pb += 4) m1 = __vmaxu2(m1, c[(long)pb * KWR]);
    }
    part[warp][lane] = __vmaxu2(m0, m1);
    __syncthreads();
    if (warp == 0 && lane < KWR) {
      const uint32_t m = __vmaxu2(__vmaxu2(part[0][lane], part[1][lane]), __vmaxu2(part[2][lane], part[3][lane]));
      const int s = lane / LP, i = lane - s * LP;
      e[(long)(s * L + 2 * i) * np + P] = key_exponent(m & 0xffffu);
      if (2 * i + 1 < L) e[(long)(s * L + 2 * i + 1) * np + P] = key_exponent(m >> 16);
    }
    __syncthreads();
  }
}

// tcum[pb] = the tiles of the row bands before pb that reach the diagonal
// (tcum[npb] = all of them).
__global__ void herm_tile_prefix(int* tcum, int np, int epw) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int npb = (np + 7) / 8, nqb = (np + epw - 1) / epw;
  int c = 0;
  for (int pb = 0; pb < npb; pb++) {
    tcum[pb] = c;
    c += nqb - herm_qb0(pb, epw);
  }
  tcum[npb] = c;
}

// e[i] = the exponent a row key stands for, in place: for a key of a value of
// at least 2^-133 its frexp exponent (normal: biased exponent - 126;
// subnormal: bit length of the 7 kept mantissa bits - 133), else 0.
__global__ void rowkey_to_exponents(unsigned* v, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned k = v[i];
    const int e = k >= 0x80u ? (int)(k >> 7) - 126 : k ? (32 - __clz((int)k)) - 133 : 0;
    reinterpret_cast<int*>(v)[i] = e;
  }
}

// Vh[a] = (1/N_k) sum_q w^{+a.q} V[q], FP64; stored FP64 and/or FP32.
__global__ void prepare_kernel(const double2* __restrict__ V, double2* __restrict__ Vh64,
                               float2* __restrict__ Vh32, long npq, Twiddles tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const int T = blockDim.x, tid = threadIdx.x;
  const int nk = tw.n[0] * tw.n[1] * tw.n[2];
  const long e = (long)blockIdx.x * T + tid;
  const bool ok = e < npq;
  double2* x = buf + tid;
  for (int k = 0; k < nk; k++) x[(long)k * T] = ok ? V[(long)k * npq + e] : make_double2(0, 0);
  dft3<double>(x, T, tw, +1);
  if (!ok) return;
  const double sc = 1.0 / nk;
  for (int a = 0; a < nk; a++) {
    double2 v = x[(long)a * T];
    v.x *= sc;
    v.y *= sc;
    if (Vh64) Vh64[(long)a * npq + e] = v;
    if (Vh32) Vh32[(long)a * npq + e] = make_float2((float)v.x, (float)v.y);
  }
}

Twiddles make_twiddles(int n1, int n2, int n3) {
  Twiddles t;
  t.n[0] = n1; t.n[1] = n2; t.n[2] = n3;
  for (int ax = 0; ax < 3; ax++)
    for (int r = 0; r < MAXL; r++) {
      int L = t.n[ax];
      double c = 1.0, s = 0.0;
      if (r < L && L > 0) {
        // exact values at multiples of pi/2
        if ((4 * r) % L == 0) {
          int q = (4 * r) / L;   // quarter turns
          c = (q == 0) ? 1.0 : (q == 2) ? -1.0 : 0.0;
          s = (q == 1) ? 1.0 : (q == 3) ? -1.0 : 0.0;
        } else {
          c = cos(2.0 * M_PI * r / L);
          s = sin(2.0 * M_PI * r / L);
        }
      }
      t.c[ax][r] = c;
      t.s[ax][r] = s;
      t.ch[ax][r] = (float)c;
      t.cl[ax][r] = (float)(c - (double)t.ch[ax][r]);
      t.sh[ax][r] = (float)s;
      t.sl[ax][r] = (float)(s - (double)t.sh[ax][r]);
    }
  return t;
}

// Threads per block of the one-element-per-thread forms: each thread keeps
// its element's N_k values in shared memory, so blocks shrink (down to 8
// threads: 8 x 512 complex128 values = 64 KB on an 8^3 mesh) to stay within
// about 100 KB of dynamic shared memory.
int pick_threads(int nk, size_t elem) {
  const size_t budget = 100 * 1024;
  int T = 256;
  while (T > 8 && (size_t)T * nk * elem > budget) T /= 2;
  return T;
}

template <int N1, int N2, int N3>
cudaError_t kconv_lanes_launch(const float2* D, const float2* Vh, float2* M, long npq, cudaStream_t s) {
  constexpr int EPB = (32 / N1) * 8;
  const long blocks = (npq + EPB - 1) / EPB;
  kconv_lanes_kernel<N1, N2, N3><<<(unsigned)blocks, 256, 0, s>>>(D, Vh, M, npq, make_twiddles(N1, N2, N3));
  return cudaGetLastError();
}

template <typename R>
cudaError_t kconv_launch(const typename cplx<R>::type* D, const typename cplx<R>::type* Vh,
                         typename cplx<R>::type* M, long npq, int n1, int n2, int n3, cudaStream_t s) {
  if constexpr (sizeof(R) == sizeof(float)) {
    if (n1 == n2 && n2 == n3) {
      if (n1 == 4) return kconv_lanes_launch<4, 4, 4>(D, Vh, M, npq, s);
      if (n1 == 3) return kconv_lanes_launch<3, 3, 3>(D, Vh, M, npq, s);
      if (n1 == 2) return kconv_lanes_launch<2, 2, 2>(D, Vh, M, npq, s);
    }
  }
  const int nk = n1 * n2 * n3;
  const size_t el = sizeof(typename cplx<R>::type);
  const int T = pick_threads(nk, el);
  const size_t sm = (size_t)T * nk * el;
  cudaError_t e = cudaFuncSetAttribute(kconv_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long blocks = (npq + T - 1) / T;
  kconv_kernel<R><<<(unsigned)blocks, T, sm, s>>>(D, Vh, M, npq, make_twiddles(n1, n2, n3));
  return cudaGetLastError();
}

template <int N1, int N2, int N3>
cudaError_t kconv_pipe_launch(const float2* D, const float2* Vh, float2* M, int np, unsigned* rowkey, int* err,
                              cudaStream_t s) {
  constexpr int NK = N1 * N2 * N3, EPB = (32 / N1) * 8;
  constexpr uint32_t BOX = NK * EPB * sizeof(float2);
  const long npq = (long)np * np;
  alignas(64) unsigned char mD[128], mV[128];
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  cudaError_t e = make_f32_map_2d(mD, D, 2 * npq, NK, 8 * npq, 2 * EPB, NK);
  if (e == cudaSuccess) e = make_f32_map_2d(mV, Vh, 2 * npq, NK, 8 * npq, 2 * EPB, NK);
  if (e != cudaSuccess) return e;
  CUtensorMap mapD, mapV;
  memcpy(&mapD, mD, sizeof mapD);
  memcpy(&mapV, mV, sizeof mapV);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  constexpr uint32_t SMEM = 3 * BOX + 16;
  static_assert(BOX % 128 == 0, "boxes start on 128-byte boundaries");
  e = cudaFuncSetAttribute(kconv_pipe_kernel<N1, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (e != cudaSuccess) return e;
  const long nbatch = (npq + EPB - 1) / EPB;
  const unsigned grid = (unsigned)std::min<long>(nbatch, 2L * nsm);
  kconv_pipe_kernel<N1, N2, N3><<<grid, 256, SMEM, s>>>(mapD, mapV, M, npq, nbatch, make_twiddles(N1, N2, N3),
                                                         rowkey, np, err);
  return cudaGetLastError();
}

template <int N1, int N2, int N3, bool X>
cudaError_t kconv_herm_launch(const float2* D, const float2* Vh, float2* M, int np, uint32_t* keys, int* e,
                              int* err, cudaEvent_t conv_done, cudaStream_t s, uint32_t* Mlo) {
  constexpr int L = N2 * N3, NK = N1 * L, EPW = 32 / N1, EPB = EPW * 8, LP = (L + 1) / 2, KWR = N1 * LP;
  constexpr uint32_t BOX = NK * EPB * sizeof(float2);
  constexpr uint32_t SMEM = 3 * BOX + 8 * 32 * LP * 4 + 16;   // + mbarrier and the next tile's (pb, qb)
  static_assert(BOX % 128 == 0, "boxes start on 128-byte boundaries");
  const long npq = (long)np * np;
  alignas(64) unsigned char mD[128], mV[128];
  cudaError_t r = make_f32_map_3d(mD, D, 2L * np, np, NK, 8L * np, 8 * npq, 2 * EPW, 8, NK);
  if (r == cudaSuccess) r = make_f32_map_3d(mV, Vh, 2L * np, np, NK, 8L * np, 8 * npq, 2 * EPW, 8, NK);
  if (r != cudaSuccess) return r;
  CUtensorMap mapD, mapV;
  memcpy(&mapD, mD, sizeof mapD);
  memcpy(&mapV, mV, sizeof mapV);
  const int npb = (np + 7) / 8, nqb = (np + EPW - 1) / EPW;
  long ntile = 0;
  for (int pb = 0; pb < npb; pb++) ntile += nqb - herm_qb0(pb, EPW);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  r = cudaFuncSetAttribute(kconv_herm_kernel<N1, N2, N3, X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (r != cudaSuccess) return r;
  uint32_t* rowk = keys;
  uint32_t* colk = keys + (long)nqb * np * KWR;
  const int* tcum = reinterpret_cast<const int*>(colk + (long)npb * np * KWR);
  const unsigned grid = (unsigned)std::min<long>(ntile, 2L * nsm);
  kconv_herm_kernel<N1, N2, N3, X><<<grid, 256, SMEM, s>>>(mapD, mapV, M, np, ntile, make_twiddles(N1, N2, N3),
                                                         rowk, colk, tcum, err, Mlo);
  r = cudaGetLastError();
  if (r == cudaSuccess && conv_done) r = cudaEventRecord(conv_done, s);
  if (r != cudaSuccess) return r;
  herm_keys_to_exponents<N1, N2, N3><<<(unsigned)std::min(np, 152 * 16), 128, 0, s>>>(rowk, colk, np, e);
  return cudaGetLastError();
}

}  // namespace

long kconv_herm_key_words(int np, int n1, int n2, int n3) {
  if (!(n1 == n2 && n2 == n3 && n1 >= 2 && n1 <= 4) || np < 2 || np % 2) return 0;
  const int L = n2 * n3, EPW = 32 / n1, LP = (L + 1) / 2, KWR = n1 * LP;
  const long nqb = (np + EPW - 1) / EPW, npb = (np + 7) / 8;
  return (nqb + npb) * np * KWR + npb + 1;   // row keys, column keys, tile prefix
}

cudaError_t kconv_herm_prepare(uint32_t* keys, int np, int n1, int n2, int n3, cudaStream_t s) {
  if (kconv_herm_key_words(np, n1, n2, n3) == 0 || !keys) return cudaErrorInvalidValue;
  const int L = n2 * n3, EPW = 32 / n1, LP = (L + 1) / 2, KWR = n1 * LP;
  const long nqb = (np + EPW - 1) / EPW, npb = (np + 7) / 8;
  herm_tile_prefix<<<1, 32, 0, s>>>(reinterpret_cast<int*>(keys + (nqb + npb) * np * KWR), np, EPW);
  return cudaGetLastError();
}

cudaError_t kconv_c_herm(const float2* D, const float2* Vh, float2* M, int np, int n1, int n2, int n3,
                         uint32_t* keys, int* e, int* err, cudaEvent_t started, cudaEvent_t conv_done,
                         cudaStream_t s, uint32_t* Mlo) {
  if (kconv_herm_key_words(np, n1, n2, n3) == 0 || !keys || !err || ((uintptr_t)D & 15) || ((uintptr_t)Vh & 15))
    return cudaErrorInvalidValue;
  if (Mlo && n1 == 3) return cudaErrorInvalidValue;   // the extended form needs a radix-2/4 mesh
  cudaError_t r = started ? cudaEventRecord(started, s) : cudaSuccess;
  if (r != cudaSuccess) return r;
  if (n1 == 4)
    return Mlo ? kconv_herm_launch<4, 4, 4, true>(D, Vh, M, np, keys, e, err, conv_done, s, Mlo)
               : kconv_herm_launch<4, 4, 4, false>(D, Vh, M, np, keys, e, err, conv_done, s, nullptr);
  if (n1 == 3) return kconv_herm_launch<3, 3, 3, false>(D, Vh, M, np, keys, e, err, conv_done, s, nullptr);
  return Mlo ? kconv_herm_launch<2, 2, 2, true>(D, Vh, M, np, keys, e, err, conv_done, s, Mlo)
             : kconv_herm_launch<2, 2, 2, false>(D, Vh, M, np, keys, e, err, conv_done, s, nullptr);
}

// Shared memory of kconv_tile_kernel for N_k k-planes: two boxes, the row
// maxima and the barrier.
size_t tile_smem(int nk) { return 2 * (size_t)nk * TILE_EPB * sizeof(float2) + ((nk * 4 + 15) & ~15) + 16; }

cudaError_t kconv_tile_launch(const float2* D, const float2* Vh, float2* M, int np, int n1, int n2, int n3,
                              unsigned* rowkey, int* err, cudaStream_t s) {
  const int nk = n1 * n2 * n3;
  const long npq = (long)np * np;
  alignas(64) unsigned char mD[128], mV[128];
  cudaError_t e = make_f32_map_2d(mD, D, 2 * npq, nk, 8 * npq, 2 * TILE_EPB, nk);
  if (e == cudaSuccess) e = make_f32_map_2d(mV, Vh, 2 * npq, nk, 8 * npq, 2 * TILE_EPB, nk);
  if (e != cudaSuccess) return e;
  CUtensorMap mapD, mapV;
  memcpy(&mapD, mD, sizeof mapD);
  memcpy(&mapV, mV, sizeof mapV);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  const size_t sm = tile_smem(nk);
  e = cudaFuncSetAttribute(kconv_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long nbatch = (npq + TILE_EPB - 1) / TILE_EPB;
  const int per_sm = sm <= 113 * 1024 ? 2 : 1;
  const unsigned grid = (unsigned)std::min<long>(nbatch, (long)per_sm * nsm);
  kconv_tile_kernel<<<grid, 256, sm, s>>>(mapD, mapV, M, npq, nbatch, make_twiddles(n1, n2, n3), rowkey, np, err);
  return cudaGetLastError();
}

cudaError_t kconv_c_rowexp(const float2* D, const float2* Vh, float2* M, int np, int n1, int n2, int n3, int* e,
                           bool* done, int* err, cudaEvent_t started, cudaEvent_t conv_done, cudaStream_t s) {
  *done = false;
  const long npq = (long)np * np;
  const bool aligned = np >= 1 && npq % 2 == 0 && npq < (1L << 29) && ((uintptr_t)D & 15) == 0 &&
                       ((uintptr_t)Vh & 15) == 0 && err;
  const bool pipe = aligned && n1 == n2 && n2 == n3 && n1 >= 2 && n1 <= 4;
  // the shared-memory form: up to 256 k-planes (one TMA box along k)
  const bool tile = aligned && !pipe && n1 * n2 * n3 <= 256 && n1 * n2 * n3 > 1;
  cudaError_t r = cudaSuccess;
  if (tile) {
    const long rows = (long)n1 * n2 * n3 * np;
    unsigned* key = reinterpret_cast<unsigned*>(e);
    r = cudaMemsetAsync(key, 0, rows * sizeof(unsigned), s);
    if (r == cudaSuccess && started) r = cudaEventRecord(started, s);
    if (r == cudaSuccess) r = kconv_tile_launch(D, Vh, M, np, n1, n2, n3, key, err, s);
    if (r == cudaSuccess && conv_done) r = cudaEventRecord(conv_done, s);
    if (r != cudaSuccess) return r;
    rowkey_to_exponents<<<(unsigned)std::min<long>((rows + 255) / 256, 152L * 8), 256, 0, s>>>(key, rows);
    r = cudaGetLastError();
    *done = r == cudaSuccess;
    return r;
  }
  if (!pipe) {
    if (started) r = cudaEventRecord(started, s);
    if (r == cudaSuccess) r = kconv_c(D, Vh, M, npq, n1, n2, n3, s);
    if (r == cudaSuccess && conv_done) r = cudaEventRecord(conv_done, s);
    return r;
  }
  const long rows = (long)n1 * n2 * n3 * np;
  unsigned* key = reinterpret_cast<unsigned*>(e);
  r = cudaMemsetAsync(key, 0, rows * sizeof(unsigned), s);
  if (r == cudaSuccess && started) r = cudaEventRecord(started, s);
  if (r != cudaSuccess) return r;
  if (n1 == 4) r = kconv_pipe_launch<4, 4, 4>(D, Vh, M, np, key, err, s);
  else if (n1 == 3) r = kconv_pipe_launch<3, 3, 3>(D, Vh, M, np, key, err, s);
  else r = kconv_pipe_launch<2, 2, 2>(D, Vh, M, np, key, err, s);
  if (r == cudaSuccess && conv_done) r = cudaEventRecord(conv_done, s);
  if (r != cudaSuccess) return r;
  rowkey_to_exponents<<<(unsigned)std::min<long>((rows + 255) / 256, 152L * 8), 256, 0, s>>>(key, rows);
  r = cudaGetLastError();
  *done = r == cudaSuccess;
  return r;
}

cudaError_t mlo_combine_c2z(const float2* M, const uint32_t* Mlo, double2* out, long n, cudaStream_t s) {
  mlo_combine_kernel<<<(unsigned)std::min<long>((n + 255) / 256, 152L * 16), 256, 0, s>>>(M, Mlo, out, n);
  return cudaGetLastError();
}

cudaError_t kconv_z(const double2* D, const double2* Vh, double2* M, long npq, int n1, int n2,
                    int n3, cudaStream_t s) {
  return kconv_launch<double>(D, Vh, M, npq, n1, n2, n3, s);
}

cudaError_t kconv_c(const float2* D, const float2* Vh, float2* M, long npq, int n1, int n2,
                    int n3, cudaStream_t s) {
  return kconv_launch<float>(D, Vh, M, npq, n1, n2, n3, s);
}

cudaError_t prepare_kernel_z(const double2* V, double2* Vh64, float2* Vh32, long npq, int n1,
                             int n2, int n3, cudaStream_t s) {
  const int nk = n1 * n2 * n3;
  const int T = pick_threads(nk, sizeof(double2));
  const size_t sm = (size_t)T * nk * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(prepare_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const long blocks = (npq + T - 1) / T;
  prepare_kernel<<<(unsigned)blocks, T, sm, s>>>(V, Vh64, Vh32, npq, make_twiddles(n1, n2, n3));
  return cudaGetLastError();
}


