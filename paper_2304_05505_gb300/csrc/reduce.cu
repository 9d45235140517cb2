// Step S5, the exchange energy (Eq. thcoccrik):
//   E_x = -(1/N_k) sum_k sum_{P,i} conj(Psi^k[P,i]) Y^k[P,i],  Y = M Psi,
// plus element-wise conversions and the finite-value check of the inputs.
//
// The sum is deterministic: a fixed grid of blocks writes one FP64 partial per
// block, and a single block adds the partials in a fixed order.  In the mixed
// form each product is formed in FP32 and a thread's products are summed in a
// float-float (two-sum) pair, which is carried into FP64 before any sum across
// threads; every sum across threads and blocks is FP64.
#include "thc_internal.cuh"

namespace {

constexpr int RT = 256;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(RT) ex_partial_z(const double2* __restrict__ Psi,
                                                    const double2* __restrict__ Y, long n,
                                                    double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  double re = 0.0, im = 0.0;
  for (long i = (long)blockIdx.x * RT + threadIdx.x; i < n; i += (long)gridDim.x * RT) {
    double2 p = Psi[i], y = Y[i];
    re += p.x * y.x + p.y * y.y;
    im += p.x * y.y - p.y * y.x;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = re;
    partial[2 * blockIdx.x + 1] = im;
  }
}

__global__ void __launch_bounds__(RT) ex_partial_c(const float2* __restrict__ Psi,
                                                    const float2* __restrict__ Y, long n,
                                                    double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  // unrolled so that the loads of several iterations are in flight together
#pragma unroll 4
  for (long i = (long)blockIdx.x * RT + threadIdx.x; i < n; i += (long)gridDim.x * RT) {
    const float2 p = __ldcs(Psi + i), y = __ldcs(Y + i);
    float re = fmaf(p.x, y.x, p.y * y.y);
    float im = fmaf(p.x, y.y, -p.y * y.x);
    float s, e;
    two_sum(rh, re, s, e); rh = s; rl += e;
    two_sum(ih, im, s, e); ih = s; il += e;
  }
  double re = block_sum((double)rh + (double)rl, sh);
  double im = block_sum((double)ih + (double)il, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = re;
    partial[2 * blockIdx.x + 1] = im;
  }
}

// One block; thread t adds partials t, t + RT, ... and the block tree adds
// the thread sums: a fixed order, so the result is reproducible.
__global__ void __launch_bounds__(RT) ex_final(const double* __restrict__ partial, int np, int nk, double* ex) {
  __shared__ double sh[RT / 32];
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < np; i += RT) {
    re += partial[2 * i];
    im += partial[2 * i + 1];
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) {
    ex[0] = -re / nk;
    ex[1] = -im / nk;
  }
}

__global__ void z2c_kernel(const double2* __restrict__ in, float2* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void z2c_rows_kernel(const double2* __restrict__ in, float2* __restrict__ out, long n, int cols,
                                int ldo) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long r = i / cols;
    const int c = (int)(i - r * cols);
    out[r * ldo + c] = make_float2((float)in[i].x, (float)in[i].y);
  }
}

__global__ void c2z_kernel(const float2* __restrict__ in, double2* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

__global__ void finite_kernel(const double2* __restrict__ in, long n, int* flag) {
  int bad = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    bad |= !(isfinite(in[i].x) && isfinite(in[i].y));
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

unsigned grid_for(long n, int t) {
  long b = (n + t - 1) / t;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

cudaError_t ex_reduce_z(const double2* Psi, const double2* Y, long n, int nk, double* partial,
                        int npartial, double* ex, cudaStream_t s) {
  ex_partial_z<<<npartial, RT, 0, s>>>(Psi, Y, n, partial);
  ex_final<<<1, RT, 0, s>>>(partial, npartial, nk, ex);
  return cudaGetLastError();
}

cudaError_t ex_finalize(const double* partial, int npartial, int nk, double* ex, cudaStream_t s) {
  ex_final<<<1, RT, 0, s>>>(partial, npartial, nk, ex);
  return cudaGetLastError();
}

cudaError_t ex_reduce_c(const float2* Psi, const float2* Y, long n, int nk, double* partial,
                        int npartial, double* ex, cudaStream_t s) {
  ex_partial_c<<<npartial, RT, 0, s>>>(Psi, Y, n, partial);
  ex_final<<<1, RT, 0, s>>>(partial, npartial, nk, ex);
  return cudaGetLastError();
}

__global__ void herm_dev_kernel(const double2* __restrict__ V, int np, long n, unsigned long long* out) {
  double dev = 0.0, mx = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long k = i / ((long)np * np), r = i - k * np * np;
    const int p = (int)(r / np), q = (int)(r - (long)p * np);
    const double2 a = V[i], b = V[k * np * np + (long)q * np + p];
    dev = fmax(dev, fmax(fabs(a.x - b.x), fabs(a.y + b.y)));
    mx = fmax(mx, fmax(fabs(a.x), fabs(a.y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(dev));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(mx));
  }
}

__global__ void herm_fill_kernel(const float2* __restrict__ D, double2* __restrict__ out, int np, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long k = i / ((long)np * np), r = i - k * np * np;
    const int p = (int)(r / np), q = (int)(r - (long)p * np);
    const float2 v = q >= p ? D[i] : D[k * np * np + (long)q * np + p];
    out[i] = make_double2(v.x, q >= p ? v.y : -v.y);
  }
}

cudaError_t hermitian_deviation_z(const double2* V, int np, int nk, unsigned long long* out, cudaStream_t s) {
  const long n = (long)nk * np * np;
  herm_dev_kernel<<<grid_for(n, 256), 256, 0, s>>>(V, np, n, out);
  return cudaGetLastError();
}

cudaError_t hermitian_fill_c2z(const float2* D, double2* out, int np, int nk, cudaStream_t s) {
  const long n = (long)nk * np * np;
  herm_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(D, out, np, n);
  return cudaGetLastError();
}

cudaError_t convert_z2c(const double2* in, float2* out, long n, cudaStream_t s) {
  z2c_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t convert_z2c_rows(const double2* in, float2* out, long rows, int cols, int ldo, cudaStream_t s) {
  const long n = rows * cols;
  z2c_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n, cols, ldo);
  return cudaGetLastError();
}

cudaError_t convert_c2z(const float2* in, double2* out, long n, cudaStream_t s) {
  c2z_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t check_finite_z(const double2* in, long n, int* flag, cudaStream_t s) {
  finite_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, n, flag);
  return cudaGetLastError();
}
