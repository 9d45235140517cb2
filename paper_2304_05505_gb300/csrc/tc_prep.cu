// Operand preparation of the tensor-core GEMMs: splitting complex matrices
// into three bf16 planes (x = x0 + x1 + x2, each the bf16 rounding of what
// the previous planes left) and building the real embedding of the thin B
// operand.  See tc_gemm.cu for the layout the planes feed.
#include "thc_internal.cuh"
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

namespace {

__device__ __forceinline__ void split3(float x, uint16_t& a, uint16_t& b, uint16_t& c) {
  __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(h0);
  __nv_bfloat16 h1 = __float2bfloat16_rn(r);
  r -= __bfloat162float(h1);
  __nv_bfloat16 h2 = __float2bfloat16_rn(r);
  a = __bfloat16_as_ushort(h0);
  b = __bfloat16_as_ushort(h1);
  c = __bfloat16_as_ushort(h2);
}

// From FP64: the residuals are formed in FP64 so the planes carry the first
// 24 significant bits of the double, not of its FP32 rounding.
__device__ __forceinline__ void split3(double x, uint16_t& a, uint16_t& b, uint16_t& c) {
  __nv_bfloat16 h0 = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(h0);
  __nv_bfloat16 h1 = __double2bfloat16(r);
  r -= (double)__bfloat162float(h1);
  __nv_bfloat16 h2 = __double2bfloat16(r);
  a = __bfloat16_as_ushort(h0);
  b = __bfloat16_as_ushort(h1);
  c = __bfloat16_as_ushort(h2);
}

__device__ __forceinline__ void store_pair(uint16_t* p0, uint16_t* p1, uint16_t* p2, long off, float re,
                                           float im) {
  uint16_t a0, a1, a2, b0, b1, b2;
  split3(re, a0, a1, a2);
  split3(im, b0, b1, b2);
  *reinterpret_cast<uint32_t*>(p0 + off) = (uint32_t)a0 | ((uint32_t)b0 << 16);
  *reinterpret_cast<uint32_t*>(p1 + off) = (uint32_t)a1 | ((uint32_t)b1 << 16);
  *reinterpret_cast<uint32_t*>(p2 + off) = (uint32_t)a2 | ((uint32_t)b2 << 16);
}

__device__ __forceinline__ void store_pair(uint16_t* p0, uint16_t* p1, uint16_t* p2, long off, double re,
                                           double im) {
  uint16_t a0, a1, a2, b0, b1, b2;
  split3(re, a0, a1, a2);
  split3(im, b0, b1, b2);
  *reinterpret_cast<uint32_t*>(p0 + off) = (uint32_t)a0 | ((uint32_t)b0 << 16);
  *reinterpret_cast<uint32_t*>(p1 + off) = (uint32_t)a1 | ((uint32_t)b1 << 16);
  *reinterpret_cast<uint32_t*>(p2 + off) = (uint32_t)a2 | ((uint32_t)b2 << 16);
}

template <typename CT>
__global__ void split_rows_kernel(const CT* __restrict__ src, long sbs, int lds, int batch, int rows,
                                  int cols, uint16_t* p0, uint16_t* p1, uint16_t* p2, int ldp) {
  const long total = (long)batch * rows * cols;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    const long br = i / cols;
    const int r = (int)(br % rows);
    const int b = (int)(br / rows);
    const CT v = src[(long)b * sbs + (long)r * lds + c];
    store_pair(p0, p1, p2, ((long)b * rows + r) * ldp + 2L * c, v.x, v.y);
  }
}

// planes[b][c][2r + d] of src[b][r][c]; 32 x 32 tiles through shared memory.
__global__ void split_cols_kernel(const double2* __restrict__ src, long sbs, int lds, int rows, int cols,
                                  uint16_t* p0, uint16_t* p1, uint16_t* p2, int ldp) {
  __shared__ double2 t[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? src[(long)b * sbs + (long)r * lds + c] : make_double2(0, 0);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const double2 v = t[threadIdx.x][y];
      store_pair(p0, p1, p2, ((long)b * cols + c) * ldp + 2L * r, v.x, v.y);
    }
  }
}

template <typename CT>
__global__ void embed_kernel(const CT* __restrict__ src, long sbs, long ldk, long ldj, bool conj_src,
                             bool conj_a, int batch, int K, int J, uint16_t* p0, uint16_t* p1, uint16_t* p2,
                             int ldp) {
  const long total = (long)batch * J * K;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int k = (int)(i % K);
    const long bj = i / K;
    const int j = (int)(bj % J);
    const int b = (int)(bj / J);
    const CT v = src[(long)b * sbs + (long)k * ldk + (long)j * ldj];
    const float br = (float)v.x;
    const float bi = conj_src ? -(float)v.y : (float)v.y;
    const long row0 = ((long)b * 2 * J + 2L * j) * ldp + 2L * k;
    const long row1 = row0 + ldp;
    if (!conj_a) {
      store_pair(p0, p1, p2, row0, br, -bi);
      store_pair(p0, p1, p2, row1, bi, br);
    } else {
      store_pair(p0, p1, p2, row0, br, bi);
      store_pair(p0, p1, p2, row1, bi, -br);
    }
  }
}

__global__ void combine_kernel(const uint16_t* p0, const uint16_t* p1, const uint16_t* p2, int batch, int rows,
                               int cols, int ldp, double2* out) {
  const long total = (long)batch * rows * cols;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    const long br = i / cols;
    const long off = br * ldp + 2L * c;
    double re = 0.0, im = 0.0;
    const uint16_t* ps[3] = {p0, p1, p2};
    for (int p = 0; p < 3; p++) {
      re += (double)__bfloat162float(__ushort_as_bfloat16(ps[p][off]));
      im += (double)__bfloat162float(__ushort_as_bfloat16(ps[p][off + 1]));
    }
    out[i] = make_double2(re, im);
  }
}

unsigned grid1(long n) {
  long b = (n + 255) / 256;
  if (b > 152L * 32) b = 152L * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t split_rows_z(const double2* src, long sbs, int lds, int batch, int rows, int cols, uint16_t* p0,
                         uint16_t* p1, uint16_t* p2, int ldp, cudaStream_t s) {
  split_rows_kernel<double2><<<grid1((long)batch * rows * cols), 256, 0, s>>>(src, sbs, lds, batch, rows, cols,
                                                                              p0, p1, p2, ldp);
  return cudaGetLastError();
}

cudaError_t split_rows_c(const float2* src, long sbs, int lds, int batch, int rows, int cols, uint16_t* p0,
                         uint16_t* p1, uint16_t* p2, int ldp, cudaStream_t s) {
  split_rows_kernel<float2><<<grid1((long)batch * rows * cols), 256, 0, s>>>(src, sbs, lds, batch, rows, cols,
                                                                             p0, p1, p2, ldp);
  return cudaGetLastError();
}

cudaError_t split_cols_z(const double2* src, long sbs, int lds, int batch, int rows, int cols, uint16_t* p0,
                         uint16_t* p1, uint16_t* p2, int ldp, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  split_cols_kernel<<<grid, dim3(32, 8), 0, s>>>(src, sbs, lds, rows, cols, p0, p1, p2, ldp);
  return cudaGetLastError();
}

cudaError_t embed_b(const void* src, bool src_f64, long sbs, long ldk, long ldj, bool conj_src, bool conj_a,
                    int batch, int K, int J, uint16_t* p0, uint16_t* p1, uint16_t* p2, int ldp, cudaStream_t s) {
  const long n = (long)batch * J * K;
  if (src_f64)
    embed_kernel<double2><<<grid1(n), 256, 0, s>>>((const double2*)src, sbs, ldk, ldj, conj_src, conj_a, batch,
                                                   K, J, p0, p1, p2, ldp);
  else
    embed_kernel<float2><<<grid1(n), 256, 0, s>>>((const float2*)src, sbs, ldk, ldj, conj_src, conj_a, batch, K,
                                                  J, p0, p1, p2, ldp);
  return cudaGetLastError();
}

cudaError_t combine_planes(const uint16_t* p0, const uint16_t* p1, const uint16_t* p2, int batch, int rows,
                           int cols, int ldp, double2* out, cudaStream_t s) {
  combine_kernel<<<grid1((long)batch * rows * cols), 256, 0, s>>>(p0, p1, p2, batch, rows, cols, ldp, out);
  return cudaGetLastError();
}
