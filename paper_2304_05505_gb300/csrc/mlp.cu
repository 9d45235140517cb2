// Learned interpolation-point proposal (setup, not part of the timed build).
// The paper has no learned part: its points come from a deterministic
// decomposition (Sec. 2.1) or k-means on the density (Sec. 4).  Here a small
// network scores grid points, the highest-scoring candidates are kept, and the
// FP64 pivoted Cholesky of thc_select_points picks the points among them.
//
//  * features of grid point r (FP64 arithmetic, stored FP32):
//      log(rho + 1e-8), log(|grad rho| + 1e-8), nearest-centre distance,
//    rho(r) = (1/N_k) sum_f |U[f][r]|^2, gradient by periodic second-order
//    central differences, the distance over the 27 nearest lattice images;
//  * network 3 -> 64 -> 64 -> 64 -> 1, SiLU, FP32, on standardised features;
//    one thread per grid point, parameters in shared memory;
//  * training step: mean weighted binary cross-entropy with logits,
//    backpropagation per point (pre-activations and deltas kept point-major
//    in the workspace), weight gradients summed over fixed chunks of points
//    and then over chunks in order (deterministic), one Adam update;
//  * candidates: the k highest scores (lower index first among equals) by a
//    single-block radix select on order-preserving keys.
#include "thc_internal.cuh"

#include <math.h>

#include <vector>

namespace {

constexpr int H = 64;
constexpr int NP = 3 * H + H + H * H + H + H * H + H + H + 1;   // 8641
constexpr int oW1 = 0, oB1 = 3 * H, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H, oB3 = oW3 + H * H,
              oW4 = oB3 + H, oB4 = oW4 + H;
static_assert(oB4 + 1 == NP, "parameter layout");
constexpr int MT = 128;          // points per block
constexpr int NCHUNK = 64;       // point chunks of the weight-gradient sums
constexpr int PER_POINT = 3 + 3 * H + 3 * H + 1;   // x, a1..a3, d1..d3, d4

struct Norm {
  float mean[3], inv_std[3];
};

__device__ __forceinline__ float sigm(float a) { return 1.0f / (1.0f + __expf(-a)); }
__device__ __forceinline__ float silu(float a) { return a * sigm(a); }
__device__ __forceinline__ float silu_d(float a) {
  const float s = sigm(a);
  return s * (1.0f + a * (1.0f - s));
}
__device__ __forceinline__ float softplus(float a) { return fmaxf(a, 0.0f) + log1pf(__expf(-fabsf(a))); }

// ----------------------------------------------------------------------------
// features
// ----------------------------------------------------------------------------

__global__ void rho_kernel(const double2* __restrict__ U, int nf, long ng, double inv_nk, double* __restrict__ rho) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ng) return;
  double s = 0.0;
  for (int f = 0; f < nf; f++) {
    const double2 u = U[(long)f * ng + r];
    s += u.x * u.x + u.y * u.y;
  }
  rho[r] = s * inv_nk;
}

struct Geo {
  int g[3];
  double lat[9];     // rows a1, a2, a3
  double rec[9];     // rows b_a / (2 pi): d f_a / d r
};

__global__ void feat_kernel(const double* __restrict__ rho, Geo geo, const double* __restrict__ cf, int ncent,
                            float* __restrict__ feat) {
  const int g1 = geo.g[0], g2 = geo.g[1], g3 = geo.g[2];
  const long ng = (long)g1 * g2 * g3;
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ng) return;
  const int i1 = (int)(r / ((long)g2 * g3)), i2 = (int)((r / g3) % g2), i3 = (int)(r % g3);
  auto at = [&](int a, int b, int c) {
    a = (a + g1) % g1;
    b = (b + g2) % g2;
    c = (c + g3) % g3;
    return rho[((long)a * g2 + b) * g3 + c];
  };
  const double d0 = (at(i1 + 1, i2, i3) - at(i1 - 1, i2, i3)) * g1 * 0.5;
  const double d1 = (at(i1, i2 + 1, i3) - at(i1, i2 - 1, i3)) * g2 * 0.5;
  const double d2 = (at(i1, i2, i3 + 1) - at(i1, i2, i3 - 1)) * g3 * 0.5;
  double gn = 0.0;
  for (int x = 0; x < 3; x++) {
    const double v = d0 * geo.rec[x] + d1 * geo.rec[3 + x] + d2 * geo.rec[6 + x];
    gn += v * v;
  }
  const double f[3] = {(double)i1 / g1, (double)i2 / g2, (double)i3 / g3};
  double best = INFINITY;
  for (int c = 0; c < ncent; c++) {
    double d[3];
    for (int a = 0; a < 3; a++) {
      d[a] = f[a] - cf[3 * c + a];
      d[a] -= rint(d[a]);
    }
    for (int n0 = -1; n0 <= 1; n0++)
      for (int n1 = -1; n1 <= 1; n1++)
        for (int n2 = -1; n2 <= 1; n2++) {
          const double e0 = d[0] + n0, e1 = d[1] + n1, e2 = d[2] + n2;
          double s = 0.0;
          for (int x = 0; x < 3; x++) {
            const double v = e0 * geo.lat[x] + e1 * geo.lat[3 + x] + e2 * geo.lat[6 + x];
            s += v * v;
          }
          best = fmin(best, s);
        }
  }
  feat[3 * r] = (float)log(rho[r] + 1e-8);
  feat[3 * r + 1] = (float)log(sqrt(gn) + 1e-8);
  feat[3 * r + 2] = (float)sqrt(best);
}

// ----------------------------------------------------------------------------
// network
// ----------------------------------------------------------------------------

// Forward (and, when TRAIN, the loss and backward deltas) of one point per
// thread.  Workspace layout (point-major): ws[p * PER_POINT + ...] = x[3],
// a1[64], a2[64], a3[64], d1[64], d2[64], d3[64], d4.  Dynamic shared memory:
// the parameters, then one 64-vector per thread in column layout
// vec[j * MT + thread]; the other 64-vector of a layer lives in registers.
constexpr size_t kMlpSmem = sizeof(float) * (NP + 3 + (size_t)H * MT);   // NP + 3: 16-byte aligned vec

template <bool TRAIN>
__global__ void __launch_bounds__(MT) mlp_kernel(const float* __restrict__ params, Norm nm,
                                                 const float* __restrict__ feat, const float* __restrict__ labels,
                                                 int n, float pos_weight, float* __restrict__ score,
                                                 float* __restrict__ ws, float* __restrict__ loss_part) {
  extern __shared__ __align__(16) float sm[];
  float* w = sm;
  float* vec = sm + NP + 3;
  __shared__ float red[MT];
  for (int i = threadIdx.x; i < NP; i += MT) w[i] = params[i];
  __syncthreads();
  const int t = threadIdx.x;
  const int p = blockIdx.x * MT + t;
  const bool ok = p < n;
  float x[3];
  for (int c = 0; c < 3; c++) x[c] = ok ? (feat[3L * p + c] - nm.mean[c]) * nm.inv_std[c] : 0.f;
  float* row = ws + (long)p * PER_POINT;
  const bool keep = TRAIN && ok;
  float u[H];
  // layer 1 -> u (registers)
#pragma unroll
  for (int j = 0; j < H; j++) {
    const float a = w[oB1 + j] + w[oW1 + 3 * j] * x[0] + w[oW1 + 3 * j + 1] * x[1] + w[oW1 + 3 * j + 2] * x[2];
    if (keep) row[3 + j] = a;
    u[j] = silu(a);
  }
  // layer 2 -> vec
#pragma unroll 1
  for (int j = 0; j < H; j++) {
    float a = w[oB2 + j];
#pragma unroll
    for (int i = 0; i < H; i++) a = fmaf(w[oW2 + H * j + i], u[i], a);
    if (keep) row[3 + H + j] = a;
    vec[j * MT + t] = silu(a);
  }
#pragma unroll
  for (int i = 0; i < H; i++) u[i] = vec[i * MT + t];
  // layer 3 -> vec (pre-activations a3)
#pragma unroll 1
  for (int j = 0; j < H; j++) {
    float a = w[oB3 + j];
#pragma unroll
    for (int i = 0; i < H; i++) a = fmaf(w[oW3 + H * j + i], u[i], a);
    vec[j * MT + t] = a;
    if (keep) row[3 + 2 * H + j] = a;
  }
  float z = w[oB4];
#pragma unroll
  for (int j = 0; j < H; j++) z = fmaf(w[oW4 + j], silu(vec[j * MT + t]), z);
  if constexpr (!TRAIN) {
    if (ok) score[p] = z;
    return;
  } else {
    const float y = ok ? labels[p] : 0.f;
    const float l = ok ? pos_weight * y * softplus(-z) + (1.f - y) * softplus(z) : 0.f;
    const float s = sigm(z);
    const float d4 = ok ? (pos_weight * y * (s - 1.f) + (1.f - y) * s) / (float)n : 0.f;
    if (ok) {
      for (int c = 0; c < 3; c++) row[c] = x[c];
      row[3 + 6 * H] = d4;
    }
    // d3 -> u
#pragma unroll
    for (int j = 0; j < H; j++) {
      u[j] = w[oW4 + j] * d4 * silu_d(vec[j * MT + t]);
      if (ok) row[3 + 5 * H + j] = u[j];
    }
    // d2 -> vec
#pragma unroll 1
    for (int i = 0; i < H; i++) {
      float a = 0.f;
#pragma unroll
      for (int j = 0; j < H; j++) a = fmaf(w[oW3 + H * j + i], u[j], a);
      const float d = a * silu_d(ok ? row[3 + H + i] : 0.f);
      vec[i * MT + t] = d;
      if (ok) row[3 + 4 * H + i] = d;
    }
#pragma unroll
    for (int i = 0; i < H; i++) u[i] = vec[i * MT + t];
    // d1 -> workspace
#pragma unroll 1
    for (int i = 0; i < H; i++) {
      float a = 0.f;
#pragma unroll
      for (int j = 0; j < H; j++) a = fmaf(w[oW2 + H * j + i], u[j], a);
      if (ok) row[3 + 3 * H + i] = a * silu_d(row[3 + i]);
    }
    red[t] = l;
    __syncthreads();
    for (int o = MT / 2; o > 0; o >>= 1) {
      if (t < o) red[t] += red[t + o];
      __syncthreads();
    }
    if (t == 0) loss_part[blockIdx.x] = red[0];
  }
}

// part[c][k] = the gradient of parameter k summed over point chunk c.
__global__ void wgrad_kernel(const float* __restrict__ ws, int n, float* __restrict__ part) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (k >= NP) return;
  const int per = (n + NCHUNK - 1) / NCHUNK;
  const int p0 = c * per, p1 = min(n, p0 + per);
  // which delta (offset in the row) and which input (offset, kind) this parameter pairs
  int dofs, iofs, kind;   // kind 0: raw x, 1: silu(a), 2: bias (input 1)
  if (k < oB1) { dofs = 3 + 3 * H + k / 3; iofs = k % 3; kind = 0; }
  else if (k < oW2) { dofs = 3 + 3 * H + (k - oB1); iofs = 0; kind = 2; }
  else if (k < oB2) { dofs = 3 + 4 * H + (k - oW2) / H; iofs = 3 + (k - oW2) % H; kind = 1; }
  else if (k < oW3) { dofs = 3 + 4 * H + (k - oB2); iofs = 0; kind = 2; }
  else if (k < oB3) { dofs = 3 + 5 * H + (k - oW3) / H; iofs = 3 + H + (k - oW3) % H; kind = 1; }
  else if (k < oW4) { dofs = 3 + 5 * H + (k - oB3); iofs = 0; kind = 2; }
  else if (k < oB4) { dofs = 3 + 6 * H; iofs = 3 + 2 * H + (k - oW4); kind = 1; }
  else { dofs = 3 + 6 * H; iofs = 0; kind = 2; }
  float s = 0.f;
  for (int p = p0; p < p1; p++) {
    const float* row = ws + (long)p * PER_POINT;
    const float in = kind == 0 ? row[iofs] : kind == 1 ? silu(row[iofs]) : 1.f;
    s = fmaf(row[dofs], in, s);
  }
  part[(long)c * NP + k] = s;
}

// Sum of the chunk partials in order, then Adam (bias-corrected).
__global__ void adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ part, int t, float lr, float* __restrict__ grad_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NP) return;
  float g = 0.f;
  for (int c = 0; c < NCHUNK; c++) g += part[(long)c * NP + k];
  if (grad_out) grad_out[k] = g;
  if (lr == 0.f) return;   // gradient only
  const float b1 = 0.9f, b2 = 0.999f;
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / (1.f - powf(b1, (float)t));
  const float vh = vk / (1.f - powf(b2, (float)t));
  params[k] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// The mean loss: block partial sums added in order, divided by n.
__global__ void loss_kernel(const float* __restrict__ part, int nb, int n, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; b++) s += part[b];
  *loss = (float)(s / n);
}

// ----------------------------------------------------------------------------
// candidates: top k of n scores, one block
// ----------------------------------------------------------------------------

constexpr int KT = 1024;

__device__ __forceinline__ unsigned okey(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // ascending with f
}

// Exclusive block prefix sum of v (KT threads); returns the total in *tot.
__device__ int block_scan(int v, int* sh, int* tot) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < KT; o <<= 1) {
    const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  const int incl = sh[threadIdx.x];
  *tot = sh[KT - 1];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(KT) topk_kernel(const float* __restrict__ score, int n, int k,
                                                  int* __restrict__ out) {
  __shared__ int hist[256];
  __shared__ int sh[KT];
  __shared__ unsigned prefix_s, mask_s;
  __shared__ int need_s;
  if (threadIdx.x == 0) {
    prefix_s = 0;
    mask_s = 0;
    need_s = k;   // how many of the keys matching the prefix are still to take from the top
  }
  __syncthreads();
  // radix select of the k-th largest key, 8 bits at a time from the top
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += KT) hist[i] = 0;
    __syncthreads();
    const unsigned pre = prefix_s, msk = mask_s;
    for (int i = threadIdx.x; i < n; i += KT) {
      const unsigned key = okey(score[i]);
      if ((key & msk) == pre) atomicAdd(&hist[(key >> shift) & 255], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int need = need_s, b = 255;
      for (; b > 0; b--) {
        if (hist[b] >= need) break;
        need -= hist[b];
      }
      prefix_s = pre | ((unsigned)b << shift);
      mask_s = msk | (255u << shift);
      need_s = need;
    }
    __syncthreads();
  }
  const unsigned T = prefix_s;   // the k-th largest key
  const int take_eq = need_s;    // keys equal to T to take, lowest indices first
  // contiguous segments per thread so that index order is the scan order
  const int per = (n + KT - 1) / KT;
  const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
  int eq = 0;
  for (int i = i0; i < i1; i++) eq += okey(score[i]) == T;
  int tot;
  int eq_before = block_scan(eq, sh, &tot);
  int sel = 0;
  {
    int e = eq_before;
    for (int i = i0; i < i1; i++) {
      const unsigned key = okey(score[i]);
      if (key > T || (key == T && e++ < take_eq)) sel++;
    }
  }
  int pos = block_scan(sel, sh, &tot);
  int e = eq_before;
  for (int i = i0; i < i1; i++) {
    const unsigned key = okey(score[i]);
    if (key > T || (key == T && e++ < take_eq)) out[pos++] = i;
  }
}

// Uc[f][j] = U[f][cand[j]]
__global__ void gather_cand(const double2* __restrict__ U, int nf, long ng, const int* __restrict__ cand, int nc,
                            double2* __restrict__ Uc) {
  const long i = (long)blockIdx.x * 256 + threadIdx.x;
  if (i >= (long)nf * nc) return;
  const int f = (int)(i / nc), j = (int)(i % nc);
  Uc[i] = U[(long)f * ng + cand[j]];
}

bool norm_of(const float* h, Norm* nm) {
  for (int c = 0; c < 3; c++) {
    if (!(h[3 + c] > 0.f)) return false;
    nm->mean[c] = h[c];
    nm->inv_std[c] = 1.f / h[3 + c];
  }
  return true;
}

thc_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return THC_OK;
  set_global_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
}

}  // namespace

extern "C" {

thc_status thc_mlp_features(const double* U, int nfunc, int nk, const int* grid_host, const double* lattice_host,
                            const double* centres_host, int ncent, float* feat, void* stream) {
  if (!U || !grid_host || !lattice_host || !centres_host || !feat || nfunc < 1 || nk < 1 || ncent < 1)
    return THC_ERR_ARG;
  if (((uintptr_t)U & 15) || ((uintptr_t)feat & 3)) return THC_ERR_ARG;
  Geo geo;
  for (int a = 0; a < 3; a++) {
    geo.g[a] = grid_host[a];
    if (geo.g[a] < 3) return THC_ERR_ARG;   // central differences need three points per axis
  }
  const double* a = lattice_host;
  for (int i = 0; i < 9; i++) geo.lat[i] = a[i];
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  if (!(fabs(det) > 0)) return THC_ERR_ARG;
  // rows of inv(lattice)^T = b_a / (2 pi)
  auto cross = [](const double* x, const double* y, double* o) {
    o[0] = x[1] * y[2] - x[2] * y[1];
    o[1] = x[2] * y[0] - x[0] * y[2];
    o[2] = x[0] * y[1] - x[1] * y[0];
  };
  cross(a + 3, a + 6, geo.rec);
  cross(a + 6, a, geo.rec + 3);
  cross(a, a + 3, geo.rec + 6);
  for (double& x : geo.rec) x /= det;
  // centres in fractional coordinates: f = r . rec rows
  std::vector<double> cf(3 * (size_t)ncent);
  for (int c = 0; c < ncent; c++)
    for (int k = 0; k < 3; k++) {
      const double* r = centres_host + 3 * c;
      cf[3 * c + k] = r[0] * geo.rec[3 * k] + r[1] * geo.rec[3 * k + 1] + r[2] * geo.rec[3 * k + 2];
    }
  const long ng = (long)geo.g[0] * geo.g[1] * geo.g[2];
  cudaStream_t s = (cudaStream_t)stream;
  double *rho = nullptr, *cfd = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&rho, sizeof(double) * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&cfd, sizeof(double) * cf.size())) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(cfd, cf.data(), sizeof(double) * cf.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    const unsigned nb = (unsigned)((ng + 255) / 256);
    rho_kernel<<<nb, 256, 0, s>>>((const double2*)U, nfunc, ng, 1.0 / nk, rho);
    feat_kernel<<<nb, 256, 0, s>>>(rho, geo, cfd, ncent, feat);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    e = cudaStreamSynchronize(s);
  } while (0);
  if (rho) cudaFree(rho);
  if (cfd) cudaFree(cfd);
  return cuda_status(e, "thc_mlp_features");
}

thc_status thc_mlp_score(const float* params, const float* norm_host, const float* feat, int n, float* score,
                         void* stream) {
  Norm nm;
  if (!params || !norm_host || !feat || !score || n < 1 || !norm_of(norm_host, &nm)) return THC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaFuncSetAttribute(mlp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e != cudaSuccess) return cuda_status(e, "thc_mlp_score");
  mlp_kernel<false><<<(n + MT - 1) / MT, MT, kMlpSmem, s>>>(params, nm, feat, nullptr, n, 0.f, score, nullptr,
                                                            nullptr);
  return cuda_status(cudaGetLastError(), "thc_mlp_score");
}

thc_status thc_mlp_workspace_bytes(int n, size_t* bytes) {
  if (n < 1 || !bytes) return THC_ERR_ARG;
  const size_t nb = (size_t)(n + MT - 1) / MT;
  *bytes = sizeof(float) * ((size_t)n * PER_POINT + (size_t)NCHUNK * NP + nb);
  return THC_OK;
}

thc_status thc_mlp_train_step(float* params, float* adam_m, float* adam_v, int t, float lr, const float* norm_host,
                              const float* feat, const float* labels, int n, float pos_weight, void* workspace,
                              size_t ws_bytes, float* loss_out, float* grad_out, void* stream) {
  Norm nm;
  if (!params || !adam_m || !adam_v || !norm_host || !feat || !labels || !workspace || n < 1 || t < 1 ||
      !(lr >= 0.f) || !(pos_weight > 0.f) || !norm_of(norm_host, &nm))
    return THC_ERR_ARG;
  size_t need = 0;
  thc_mlp_workspace_bytes(n, &need);
  if (ws_bytes < need || ((uintptr_t)workspace & 15)) return THC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float* ws = (float*)workspace;
  float* part = ws + (size_t)n * PER_POINT;
  float* lpart = part + (size_t)NCHUNK * NP;
  const int nb = (n + MT - 1) / MT;
  cudaError_t e = cudaFuncSetAttribute(mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
  if (e != cudaSuccess) return cuda_status(e, "thc_mlp_train_step");
  mlp_kernel<true><<<nb, MT, kMlpSmem, s>>>(params, nm, feat, labels, n, pos_weight, nullptr, ws, lpart);
  wgrad_kernel<<<dim3((NP + 255) / 256, NCHUNK), 256, 0, s>>>(ws, n, part);
  adam_kernel<<<(NP + 255) / 256, 256, 0, s>>>(params, adam_m, adam_v, part, t, lr, grad_out);
  if (loss_out) loss_kernel<<<1, 32, 0, s>>>(lpart, nb, n, loss_out);
  return cuda_status(cudaGetLastError(), "thc_mlp_train_step");
}

thc_status thc_mlp_candidates(const float* score, int n, int k, int* cand_host, void* stream) {
  if (!score || !cand_host || n < 1 || k < 1 || k > n) return THC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int* d = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&d, sizeof(int) * k)) != cudaSuccess) break;
    topk_kernel<<<1, KT, 0, s>>>(score, n, k, d);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(cand_host, d, sizeof(int) * k, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    e = cudaStreamSynchronize(s);
  } while (0);
  if (d) cudaFree(d);
  return cuda_status(e, "thc_mlp_candidates");
}

thc_status thc_select_points_among(const double* U, int nfunc, int ng, const int* cand_host, int ncand, int npts,
                                   double rel_tol, int* points_host, int* npoints_host, void* stream) {
  if (!U || !cand_host || !points_host || !npoints_host || nfunc < 1 || ng < 1 || ncand < 1 || ncand > ng ||
      npts < 1 || npts > ncand)
    return THC_ERR_ARG;
  for (int j = 0; j < ncand; j++)
    if (cand_host[j] < 0 || cand_host[j] >= ng) return THC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int* cd = nullptr;
  double2* Uc = nullptr;
  cudaError_t e = cudaSuccess;
  thc_status st = THC_OK;
  do {
    if ((e = cudaMalloc(&cd, sizeof(int) * ncand)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Uc, sizeof(double2) * (size_t)nfunc * ncand)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(cd, cand_host, sizeof(int) * ncand, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    gather_cand<<<(unsigned)(((long)nfunc * ncand + 255) / 256), 256, 0, s>>>((const double2*)U, nfunc, ng, cd,
                                                                              ncand, Uc);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    st = thc_select_points((const double*)Uc, nfunc, ncand, npts, rel_tol, points_host, npoints_host, nullptr,
                           stream);
    if (st == THC_OK)
      for (int j = 0; j < *npoints_host; j++) points_host[j] = cand_host[points_host[j]];
  } while (0);
  if (cd) cudaFree(cd);
  if (Uc) cudaFree(Uc);
  if (e != cudaSuccess) return cuda_status(e, "thc_select_points_among");
  return st;
}

}  // extern "C"
