// Interpolation-point selection (setup, not part of the timed build):
// greedy pivoted Cholesky, in FP64, of the Gram matrix of occupied pair
// products
//   A(r, r') = | sum_f conj(U[f][r]) U[f][r'] |^2,   f = (k, i), U[f][r] = u^k_i(r)
// (the metric of the least-squares fit of Eq. pbcinterpvec restricted to
// occupied orbitals, Eq. orbprodoo).  Pivoted Cholesky picks the same points
// as the QR decomposition with column pivoting of Sec. 2.1 in exact
// arithmetic.  A is never formed: each step builds one column from U.
//
// Per step j (host loop):
//   argmax  p = argmax_r d[r] (lowest r among equal values), d[p], sum_r d[r]
//           (block partials, then one block)
//   column  a = |B(:, p)|^2, l = (a - sum_{t<j} L[t][:] L[t][p]) / sqrt(d[p]),
//           L[j][:] = l, d = max(d - l^2, 0), d[p] = 0; a block takes 32
//           candidates (one per lane, coalesced) and its 8 warps split the
//           sums over f and over t, added in a fixed order
// The loop stops after npts pivots or when sum d <= rel_tol * trace(A).
#include "thc_internal.cuh"

namespace {

constexpr int PT = 256;

__global__ void diag_kernel(const double2* __restrict__ U, int nfunc, int ncand, double* __restrict__ d) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand) return;
  double rho = 0.0;
  for (int f = 0; f < nfunc; f++) {
    const double2 u = U[(long)f * ncand + c];
    rho += u.x * u.x + u.y * u.y;
  }
  d[c] = rho * rho;
}

struct Best {
  double v;
  int i;
};

__device__ __forceinline__ Best better(Best a, Best b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

// Block partials of (max d, its lowest index) and of sum d.
__global__ void __launch_bounds__(PT) argmax_partial(const double* __restrict__ d, int n, double* pv, int* pi,
                                                     double* ps) {
  __shared__ double sv[PT];
  __shared__ int si[PT];
  __shared__ double ss[PT];
  Best b{-1.0, 0x7fffffff};
  double s = 0.0;
  for (int c = blockIdx.x * PT + threadIdx.x; c < n; c += gridDim.x * PT) {
    b = better(b, Best{d[c], c});
    s += d[c];
  }
  sv[threadIdx.x] = b.v;
  si[threadIdx.x] = b.i;
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int o = PT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      Best x = better(Best{sv[threadIdx.x], si[threadIdx.x]}, Best{sv[threadIdx.x + o], si[threadIdx.x + o]});
      sv[threadIdx.x] = x.v;
      si[threadIdx.x] = x.i;
      ss[threadIdx.x] += ss[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
    ps[blockIdx.x] = ss[0];
  }
}

// One block: final (p, d[p], trace) into sel (int) and selv[0..1].
__global__ void __launch_bounds__(PT) argmax_final(const double* pv, const int* pi, const double* ps, int nb,
                                                   int* sel, double* selv) {
  __shared__ double sv[PT];
  __shared__ int si[PT];
  __shared__ double ss[PT];
  Best b{-1.0, 0x7fffffff};
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += PT) {
    b = better(b, Best{pv[i], pi[i]});
    s += ps[i];
  }
  sv[threadIdx.x] = b.v;
  si[threadIdx.x] = b.i;
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int o = PT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      Best x = better(Best{sv[threadIdx.x], si[threadIdx.x]}, Best{sv[threadIdx.x + o], si[threadIdx.x + o]});
      sv[threadIdx.x] = x.v;
      si[threadIdx.x] = x.i;
      ss[threadIdx.x] += ss[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sel[0] = si[0];
    selv[0] = sv[0];
    selv[1] = ss[0];
  }
}

constexpr int CW = 8;   // warps of a column block

__global__ void __launch_bounds__(32 * CW) column_kernel(const double2* __restrict__ U, int nfunc, int ncand, int j,
                                                         const int* __restrict__ sel,
                                                         const double* __restrict__ selv, double* __restrict__ L,
                                                         double* __restrict__ d) {
  __shared__ double sr[CW][32], si[CW][32], sl[CW][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const int p = sel[0];
  double br = 0.0, bi = 0.0, ll = 0.0;   // B(c, p) = sum_f conj(U[f][c]) U[f][p]; sum_t L[t][c] L[t][p]
  if (c < ncand) {
    for (int f = w; f < nfunc; f += CW) {
      const double2 u = U[(long)f * ncand + c];
      const double2 v = U[(long)f * ncand + p];
      br += u.x * v.x + u.y * v.y;
      bi += u.x * v.y - u.y * v.x;
    }
    for (int t = w; t < j; t += CW) ll += L[(long)t * ncand + c] * L[(long)t * ncand + p];
  }
  sr[w][lane] = br;
  si[w][lane] = bi;
  sl[w][lane] = ll;
  __syncthreads();
  if (w != 0 || c >= ncand) return;
  for (int k = 1; k < CW; k++) {
    br += sr[k][lane];
    bi += si[k][lane];
    ll += sl[k][lane];
  }
  const double l = (br * br + bi * bi - ll) / sqrt(selv[0]);
  L[(long)j * ncand + c] = l;
  d[c] = (c == p) ? 0.0 : fmax(d[c] - l * l, 0.0);
}

}  // namespace

extern "C" thc_status thc_select_points(const double* U, int nfunc, int ncand, int npts, double rel_tol,
                                        int* points_host, int* npoints_host, double* resid_diag, void* stream) {
  if (!U || !points_host || !npoints_host || nfunc < 1 || ncand < 1 || npts < 1 || npts > ncand || rel_tol < 0)
    return THC_ERR_ARG;
  if ((uintptr_t)U & 15) return THC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)std::min<long>((ncand + PT - 1) / PT, 1024);
  double *d = nullptr, *L = nullptr, *pv = nullptr, *ps = nullptr, *selv = nullptr, *host = nullptr;
  int *pi = nullptr, *sel = nullptr;
  thc_status st = THC_OK;
  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err) {
    set_global_error(std::string("thc_select_points: ") + cudaGetErrorString(err));
    return err == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
  };
  do {
    if ((e = cudaMalloc(&d, sizeof(double) * ncand)) != cudaSuccess) break;
    if ((e = cudaMalloc(&L, sizeof(double) * (size_t)npts * ncand)) != cudaSuccess) break;
    if ((e = cudaMalloc(&pv, sizeof(double) * nb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ps, sizeof(double) * nb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&pi, sizeof(int) * nb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&sel, sizeof(int) * 4)) != cudaSuccess) break;
    if ((e = cudaMalloc(&selv, sizeof(double) * 2)) != cudaSuccess) break;
    if ((e = cudaMallocHost(&host, sizeof(double) * 4)) != cudaSuccess) break;
    const double2* u = (const double2*)U;
    const unsigned g = (unsigned)((ncand + PT - 1) / PT);
    diag_kernel<<<g, PT, 0, s>>>(u, nfunc, ncand, d);
    double tr0 = -1.0;
    int count = 0;
    for (int j = 0; j < npts; j++) {
      argmax_partial<<<nb, PT, 0, s>>>(d, ncand, pv, pi, ps);
      argmax_final<<<1, PT, 0, s>>>(pv, pi, ps, nb, sel, selv);
      if ((e = cudaMemcpyAsync(host, selv, 2 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync((int*)(host + 2), sel, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        break;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
      const double trace = host[1];
      if (j == 0) tr0 = trace;
      if (!(trace > rel_tol * tr0) || !(host[0] > 0.0)) break;   // rank reached
      points_host[j] = *(int*)(host + 2);
      column_kernel<<<(unsigned)((ncand + 31) / 32), 32 * CW, 0, s>>>(u, nfunc, ncand, j, sel, selv, L, d);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      count = j + 1;
    }
    if (e != cudaSuccess) break;
    for (int j = count; j < npts; j++) points_host[j] = -1;
    *npoints_host = count;
    if (resid_diag &&
        (e = cudaMemcpyAsync(resid_diag, d, sizeof(double) * ncand, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      break;
    e = cudaStreamSynchronize(s);
  } while (0);
  if (e != cudaSuccess) st = fail(e);
  if (d) cudaFree(d);
  if (L) cudaFree(L);
  if (pv) cudaFree(pv);
  if (ps) cudaFree(ps);
  if (pi) cudaFree(pi);
  if (sel) cudaFree(sel);
  if (selv) cudaFree(selv);
  if (host) cudaFreeHost(host);
  return st;
}
