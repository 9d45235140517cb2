// Operand preparation of the tensor-core GEMMs (tc_gemm.cu): row and column
// exponents, fixed-point slicing of complex rows into three fp16 planes, and
// the real embedding of the thin B operand.
//
// A row r with exponent e_r (max |re|, |im| over the row < 2^e_r) is written
// as x = 2^(e_r - 7) (S0 + 2^-11 S1 + 2^-22 S2) with the integers
//   y = 2^(7 - e_r) x,  S0 = rint(y),  S1 = rint(2^11 (y - S0)),  S2 = rint(2^22 (y - S0) - 2^11 S1)
// held in fp16 planes P0 = 2^8 S0, P1 = 2^-3 S1, P2 = 2^-14 S2 (slices.cuh).
// Every step is exact in FP32, so the planes carry the first 30 bits of x
// relative to its row scale.
#include "thc_internal.cuh"
#include "tc_gemm.cuh"
#include "slices.cuh"


#include <algorithm>
#include <type_traits>

namespace {

template <typename CT>
__device__ __forceinline__ double cmax(CT v) {
  return fmax(fabs((double)v.x), fabs((double)v.y));
}

// Exponent of each contiguous row: e[b * rows + r] over src[b][r][0..cols).
// One warp per row.
template <typename CT>
__global__ void rowexp_kernel(const CT* __restrict__ src, long sbs, int lds, int batch, int rows, int cols,
                              int* __restrict__ e) {
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long)batch * rows) return;
  const int b = (int)(w / rows), r = (int)(w % rows);
  const CT* p = src + (long)b * sbs + (long)r * lds;
  double m = 0.0;
  for (int c = lane; c < cols; c += 32) m = fmax(m, cmax(p[c]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) e[w] = row_exponent(m);
}

// Exponent of each column: e[b * cols + c] = max over r of src[b][r][c].
// Block (b, column slab of 32) of 32 warps: warp w scans rows w, w + 32, ...
// four at a time (lane = column), then the warps' maxima are combined.  The
// maxima are taken on the absolute values' bit patterns (non-negative floats
// order as unsigned integers), exact and off the FP64 pipe.
template <typename CT> struct AbsBits;
template <> struct AbsBits<float2> {
  typedef unsigned T;
  __device__ static T of(float2 v) { return max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu); }
  __device__ static double value(T t) { return (double)__uint_as_float(t); }
};
template <> struct AbsBits<double2> {
  typedef unsigned long long T;
  __device__ static T of(double2 v) {
    const T m = 0x7fffffffffffffffull;
    return max((T)__double_as_longlong(v.x) & m, (T)__double_as_longlong(v.y) & m);
  }
  __device__ static double value(T t) { return __longlong_as_double((long long)t); }
};

constexpr int CE_WARPS = 32;
template <typename CT>
__global__ void __launch_bounds__(CE_WARPS * 32) colexp_kernel(const CT* __restrict__ src, long sbs, int lds,
                                                               int batch, int rows, int cols, int* __restrict__ e) {
  typedef typename AbsBits<CT>::T T;
  __shared__ T red[CE_WARPS][32];
  const int b = blockIdx.y;
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5;
  T m = 0;
  if (c < cols) {
    const CT* p = src + (long)b * sbs + c;
    int r = w;
    for (; r + 3 * CE_WARPS < rows; r += 4 * CE_WARPS) {
      const CT v0 = p[(long)r * lds], v1 = p[(long)(r + CE_WARPS) * lds];
      const CT v2 = p[(long)(r + 2 * CE_WARPS) * lds], v3 = p[(long)(r + 3 * CE_WARPS) * lds];
      m = max(m, max(max(AbsBits<CT>::of(v0), AbsBits<CT>::of(v1)), max(AbsBits<CT>::of(v2), AbsBits<CT>::of(v3))));
    }
    for (; r < rows; r += CE_WARPS) m = max(m, AbsBits<CT>::of(p[(long)r * lds]));
  }
  red[w][threadIdx.x & 31] = m;
  __syncthreads();
  if (w == 0) {
    for (int i = 1; i < CE_WARPS; i++) m = max(m, red[i][threadIdx.x]);
    if (c < cols) e[(long)b * cols + c] = row_exponent(AbsBits<CT>::value(m));
  }
}

// Embedded B planes of B(k, j) = src[b*sbs + k*ldk + j*ldj] (conjugated if
// conj_src), row exponents e[b][j]:
//   planes[p][b][2j + c][2k + d] = slice_p(E_cd(B(k, j)))
// E = [[Br, -Bi], [Bi, Br]] (conj_a = 0) or [[Br, Bi], [Bi, -Br]] (conj_a = 1).
template <typename CT, typename R>
__global__ void embed_kernel(const CT* __restrict__ src, long sbs, long ldk, long ldj, bool conj_src,
                             bool conj_a, int batch, int K, int J, const int* __restrict__ e, uint16_t* planes,
                             long plane, int ldp) {
  // grid: x over K, y over the rows j (blockDim.y per block), z over the batch
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z;
  if (k < K && j < J) {
    const long bj = (long)b * J + j;
    const CT v = src[(long)b * sbs + (long)k * ldk + (long)j * ldj];
    const R br = (R)v.x;
    const R bi = conj_src ? -(R)v.y : (R)v.y;
    const int ex = e[bj];
    const long row0 = ((long)b * 2 * J + 2L * j) * ldp + 2L * k;
    uint16_t s_br[3], s_bi[3], s_nbr[3], s_nbi[3];
    slice3(br, ex, s_br);
    slice3(bi, ex, s_bi);
    negate3(s_br, s_nbr);
    negate3(s_bi, s_nbi);
    if (!conj_a) {
      store3(planes, plane, row0, s_br, s_nbi);
      store3(planes, plane, row0 + ldp, s_bi, s_br);
    } else {
      store3(planes, plane, row0, s_br, s_bi);
      store3(planes, plane, row0 + ldp, s_bi, s_nbr);
    }
  }
}

// Slices of the contiguous rows src[row][0..np) with the exact row exponent,
// one warp per row: the warp reduces max(|re|, |im|) over its row, then
// writes the three planes.  V = 2: two consecutive complex values per lane
// access (16-byte loads, np even).  R > 0: the row stays in registers (R
// accesses per lane, np / V <= 32 R; used for short rows); R = 0: the row is
// read twice, the second time mostly from cache (long rows: holding a row of
// 1200 complex values in registers costs more residency than the re-read).
// EMB: also the embedded B operand of src^H (embed_b with conj_src, conj_a = 0,
// the row exponents of src): rows 2 row and 2 row + 1 of bplanes hold the
// slices of (re, im) and of (-im, re) of each value, the first the same words
// as the row's own planes.
template <int V, int R, bool PLANES = true, bool EMB = false>
__global__ void slice_rowmax_kernel(const float2* __restrict__ src, int np, long rows, int* __restrict__ e,
                                    uint16_t* planes, long plane, int ldp, uint16_t* bplanes = nullptr,
                                    long bplane = 0) {
  typedef typename std::conditional<V == 2, float4, float2>::type VT;
  const long w0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int per = np / V;
  auto amax = [](VT w) {
    if constexpr (V == 2) return fmaxf(fmaxf(fabsf(w.x), fabsf(w.y)), fmaxf(fabsf(w.z), fabsf(w.w)));
    else return fmaxf(fabsf(w.x), fabsf(w.y));
  };
  auto put = [&](long row, int c, VT w, int ex) {
    float2 v[V];
    if constexpr (V == 2) {
      v[0] = make_float2(w.x, w.y);
      v[1] = make_float2(w.z, w.w);
    } else {
      v[0] = w;
    }
    uint16_t sl[V][2][3];
#pragma unroll
    for (int j = 0; j < V; j++) {
      slice3(v[j].x, ex, sl[j][0]);
      slice3(v[j].y, ex, sl[j][1]);
    }
    const long off = row * ldp + 2L * c * V;
    const long bo = 2 * row * ldp + 2L * c * V;
#pragma unroll
    for (int p = 0; p < 3; p++) {
      if constexpr (V == 2) {
        const uint2 wv = make_uint2((uint32_t)sl[0][0][p] | ((uint32_t)sl[0][1][p] << 16),
                                    (uint32_t)sl[1][0][p] | ((uint32_t)sl[1][1][p] << 16));
        *reinterpret_cast<uint2*>(planes + p * plane + off) = wv;
        if constexpr (EMB) {
          *reinterpret_cast<uint2*>(bplanes + p * bplane + bo) = wv;
          *reinterpret_cast<uint2*>(bplanes + p * bplane + bo + ldp) =
              make_uint2(((uint32_t)sl[0][1][p] ^ 0x8000u) | ((uint32_t)sl[0][0][p] << 16),
                         ((uint32_t)sl[1][1][p] ^ 0x8000u) | ((uint32_t)sl[1][0][p] << 16));
        }
      } else {
        const uint32_t wv = (uint32_t)sl[0][0][p] | ((uint32_t)sl[0][1][p] << 16);
        *reinterpret_cast<uint32_t*>(planes + p * plane + off) = wv;
        if constexpr (EMB) {
          *reinterpret_cast<uint32_t*>(bplanes + p * bplane + bo) = wv;
          *reinterpret_cast<uint32_t*>(bplanes + p * bplane + bo + ldp) =
              ((uint32_t)sl[0][1][p] ^ 0x8000u) | ((uint32_t)sl[0][0][p] << 16);
        }
      }
    }
  };
  for (long row = w0; row < rows; row += nw) {
    const VT* r = reinterpret_cast<const VT*>(src + row * np);
    float m = 0.f;
    if constexpr (R > 0) {
      VT buf[R];
#pragma unroll
      for (int t = 0; t < R; t++) {
        const int c = lane + 32 * t;
        if (c < per) {
          buf[t] = __ldcs(r + c);
          m = fmaxf(m, amax(buf[t]));
        }
      }
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const int ex = row_exponent((double)m);
      if (lane == 0) e[row] = ex;
#pragma unroll
      for (int t = 0; t < R; t++) {
        const int c = lane + 32 * t;
        if (c < per) put(row, c, buf[t], ex);
      }
    } else {
#pragma unroll 4
      for (int c = lane; c < per; c += 32) m = fmaxf(m, amax(PLANES ? r[c] : __ldcs(r + c)));
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const int ex = row_exponent((double)m);
      if (lane == 0) e[row] = ex;
      if constexpr (PLANES)
        for (int c = lane; c < per; c += 32) put(row, c, __ldcs(r + c), ex);
    }
  }
}

unsigned grid1(long n) {
  long b = (n + 255) / 256;
  if (b > 152L * 32) b = 152L * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t row_exponents_z(const double2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s) {
  const long warps = (long)batch * rows;
  rowexp_kernel<double2><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(src, sbs, lds, batch, rows, cols, e);
  return cudaGetLastError();
}

cudaError_t row_exponents_c(const float2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s) {
  const long warps = (long)batch * rows;
  rowexp_kernel<float2><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(src, sbs, lds, batch, rows, cols, e);
  return cudaGetLastError();
}

cudaError_t col_exponents_z(const double2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s) {
  colexp_kernel<double2><<<dim3((cols + 31) / 32, batch), CE_WARPS * 32, 0, s>>>(src, sbs, lds, batch, rows, cols,
                                                                                 e);
  return cudaGetLastError();
}

cudaError_t col_exponents_c(const float2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s) {
  colexp_kernel<float2><<<dim3((cols + 31) / 32, batch), CE_WARPS * 32, 0, s>>>(src, sbs, lds, batch, rows, cols,
                                                                                e);
  return cudaGetLastError();
}

cudaError_t slice_rows_exact(const float2* src, int np, long rows, int* e, uint16_t* planes, long plane, int ldp,
                             cudaStream_t s, uint16_t* bplanes, long bplane) {
  const long nb = std::min<long>((rows + 3) / 4, 152L * 128);   // 4 warps (rows) per block
  // 16-byte loads and 8-byte plane stores need even rows and 8-byte aligned plane rows
  const bool v2 = np % 2 == 0 && ldp % 4 == 0 && ((uintptr_t)src & 15) == 0;
  const int per = v2 ? np / 2 : np;   // lane accesses of a row
#define SR(V_, R_, E_)                                                                                    \
  slice_rowmax_kernel<V_, R_, true, E_><<<(unsigned)nb, 128, 0, s>>>(src, np, rows, e, planes, plane, ldp, \
                                                                     bplanes, bplane)
#define SR2(V_, R_) { if (bplanes) SR(V_, R_, true); else SR(V_, R_, false); }
  if (v2) {
    if (per <= 32) SR2(2, 1) else if (per <= 128) SR2(2, 4) else SR2(2, 0)
  } else {
    if (per <= 32) SR2(1, 1) else if (per <= 128) SR2(1, 4) else SR2(1, 0)
  }
#undef SR2
#undef SR
  return cudaGetLastError();
}

cudaError_t row_exponents_rows(const float2* src, int np, long rows, int* e, cudaStream_t s) {
  const long nb = std::min<long>((rows + 3) / 4, 152L * 128);   // 4 warps (rows) per block
  if (np % 2 == 0 && ((uintptr_t)src & 15) == 0)
    slice_rowmax_kernel<2, 0, false><<<(unsigned)nb, 128, 0, s>>>(src, np, rows, e, nullptr, 0, 0);
  else
    slice_rowmax_kernel<1, 0, false><<<(unsigned)nb, 128, 0, s>>>(src, np, rows, e, nullptr, 0, 0);
  return cudaGetLastError();
}

cudaError_t embed_b(const void* src, bool src_f64, long sbs, long ldk, long ldj, bool conj_src, bool conj_a,
                    int batch, int K, int J, const int* e, uint16_t* planes, long plane, int ldp,
                    cudaStream_t s) {
  if ((long)batch * J * K == 0) return cudaSuccess;
  // 256 threads: up to 128 consecutive K (one write segment per plane row), the rest over rows
  const int kw = K > 64 ? 128 : K > 32 ? 64 : 32;
  const dim3 blk(kw, 256 / kw);
  if (batch > 65535 || (J + (int)blk.y - 1) / (int)blk.y > 65535) return cudaErrorInvalidValue;
  const dim3 grid((K + kw - 1) / kw, (J + blk.y - 1) / blk.y, batch);
  if (src_f64)
    embed_kernel<double2, float><<<grid, blk, 0, s>>>((const double2*)src, sbs, ldk, ldj, conj_src, conj_a, batch, K,
                                                   J, e, planes, plane, ldp);
  else
    embed_kernel<float2, float><<<grid, blk, 0, s>>>((const float2*)src, sbs, ldk, ldj, conj_src, conj_a, batch, K, J,
                                                  e, planes, plane, ldp);
  return cudaGetLastError();
}
