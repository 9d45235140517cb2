// The THC-oo-K orbital gradient: the vo block of the exchange matrix with the
// kernel's response to the orbitals (Sec. 2.3, the K_ai expression and
// Algorithm 2's dM/dtheta step), in FP64, with the dominant contraction on
// the tensor cores in the THC_MIXED form.
//
// With D^k = Psi^k Psi^kH at the points (Psi^k[P][i] = psi^k_i(r_P)) the
// energy is a sum over q,
//   E_x = -(1/N_k) sum_q sum_PQ W^q[P,Q] V^q[P,Q],   W^q = sum_k conj(D^k) o D^{k+q},
// W^q being the k-correlation of the densities the paper calls W.  THC-oo-K
// fits the interpolation vectors, and so V, to the occupied pair products
// (Eq. orbprodoo), so V moves with the orbitals.  For the rotation
// C^k -> C^k + Cv^k theta^k the gradient g = dE/dRe(theta) + i dE/dIm(theta)
// has two parts:
//   * the kernel held fixed (the K_ai expression's first term):
//       g_e^k = -(4/N_k) Psi_v^kH Y^k,  Y^k = M^k Psi^k,  M^k = sum_k' D^k' o V^(k'-k);
//   * the kernel's response (its W^q terms), the adjoint of the fit run
//     backwards from W: with xh the raw DFT of xi, ph_P = e^{-i q_r.r_P} and
//     w_q = (Omega/N_g)^2 / (n_reps N_k Omega) as in the fit,
//       Gam_P(G)  = -(2/N_k) sum_{q, reps} w_q v(G+q_r) ph_P sum_Q W^q[P,Q] conj(ph_Q xh_Q(G))
//       Xbar_P(r) = Re sum_G Gam_P(G) e^{-i G.r}          (the same forward DFT as the fit's)
//       Lam = S^-1 Xbar;  Rbar = Lam;  Rbar[:, points] -= Lam xi^T      (xi = S^-1 R)
//       Y2 = 2 Rbar o conj(B)                              (R = |B|^2)
//       T1[P][f] = sum_r Y2[P][r] U[f][r],  T2[f][r] = sum_P conj(U[f][r_P]) Y2[P][r]
//       g_r^k[a][i] = conj(sum_r Uv[(k,a)][r] T2[(k,i)][r]) + sum_P conj(Uv[(k,a)][r_P]) T1[P][(k,i)]
//     (B = conj(U_P)^T U, so dE/dconj(U) = conj(T2) plus T1 at the point columns).
// The fit (B, R, S, its Cholesky factor, xi and xh) is recomputed here from the
// orbitals with the same kernels as thc_fit_kernel; V is the caller's (the fit
// of the same orbitals at the same points).  Every contraction is an FP64
// complex GEMM on CUDA cores, except that with THC_MIXED the O(N_k N_P^2 N_G)
// one over (q, G), which dominates as the fit's own V contraction does, and
// the grid contractions T1, T2 and the projection of T2 run on the tcgen05
// tensor cores in the form of the rebuild's contraction.
#include "isdf_common.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <string>

namespace {

// out = ph * U[k*nb + b][pts[P]], ph = e^{2 pi i kfrac_k . pfrac_P} when
// `phase` (the Bloch factor that makes psi from its periodic part u), else 1.
// trans: out[(k*nb + b)*np + P]; else out[(k*np + P)*nb + b].
__global__ void point_values(const double2* __restrict__ U, int nk, int nb, long ng, const int* __restrict__ pts,
                             int np, int g1, int g2, int g3, int n1, int n2, int n3, bool phase, bool trans,
                             double2* __restrict__ out) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)nk * nb * np) return;
  int k, b, P;
  if (trans) {
    P = (int)(i % np);
    const long row = i / np;
    b = (int)(row % nb);
    k = (int)(row / nb);
  } else {
    b = (int)(i % nb);
    const long kp = i / nb;
    P = (int)(kp % np);
    k = (int)(kp / np);
  }
  const int p = pts[P];
  double2 u = U[((long)k * nb + b) * ng + p];
  if (phase) {
    const long c0 = k / (n2 * n3), c1 = (k / n3) % n2, c2 = k % n3;
    const long p0 = p / (g2 * g3), p1 = (p / g3) % g2, p2 = p % g3;
    // the turn fraction sum_j c_j p_j / (n_j g_j), each term reduced mod 1 in integers
    const double t = (double)(c0 * p0 % ((long)n1 * g1)) / ((double)n1 * g1) +
                     (double)(c1 * p1 % ((long)n2 * g2)) / ((double)n2 * g2) +
                     (double)(c2 * p2 % ((long)n3 * g3)) / ((double)n3 * g3);
    double s, c;
    sincospi(2.0 * t, &s, &c);
    u = make_double2(u.x * c - u.y * s, u.x * s + u.y * c);
  }
  out[i] = u;
}

// For every (P,Q) element e of the N_k matrices D^k:
//   W[q][e] = sum_k conj(D[k][e]) D[kq[k][q]][e]     (kq: the mesh index of k + q)
//   M[k][e] = sum_k' D[k'][e] V[qk[k][k']][e]        (qk: the mesh index of k' - k)
__global__ void kcorr_kernel(const double2* __restrict__ D, const double2* __restrict__ V, const int* __restrict__ kq,
                             const int* __restrict__ qk, int nk, long npq, double2* __restrict__ W,
                             double2* __restrict__ M) {
  const long e = (long)blockIdx.x * TB + threadIdx.x;
  if (e >= npq) return;
  for (int q = 0; q < nk; q++) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nk; k++) {
      const double2 a = D[(long)k * npq + e], b = D[(long)kq[k * nk + q] * npq + e];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
    W[(long)q * npq + e] = make_double2(re, im);
  }
  for (int k = 0; k < nk; k++) {
    double re = 0.0, im = 0.0;
    for (int kp = 0; kp < nk; kp++) {
      const double2 a = D[(long)kp * npq + e], v = V[(long)qk[k * nk + kp] * npq + e];
      re += a.x * v.x - a.y * v.y;
      im += a.x * v.y + a.y * v.x;
    }
    M[(long)k * npq + e] = make_double2(re, im);
  }
}

// Per-block FP64 sums of Re(W[i] V[i]) over i < n (a fixed grid and a fixed
// tree, so the sum is the same on every run).
__global__ void wv_partial(const double2* __restrict__ W, const double2* __restrict__ V, long n,
                           double* __restrict__ part) {
  __shared__ double sm[TB];
  double acc = 0.0;
  for (long i = (long)blockIdx.x * TB + threadIdx.x; i < n; i += (long)gridDim.x * TB) {
    const double2 a = W[i], b = V[i];
    acc += a.x * b.x - a.y * b.y;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int h = TB / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// A[P][Q] = c e^{-i q.r_P} W[P][Q] e^{+i q.r_Q}   (q Cartesian)
__global__ void phase_w(const double2* __restrict__ W, int np, const double* __restrict__ rP, double qx, double qy,
                        double qz, double c, double2* __restrict__ A) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * np) return;
  const int P = (int)(i / np), Q = (int)(i % np);
  double sp, cp, sq, cq;
  sincos(-(qx * rP[3 * P] + qy * rP[3 * P + 1] + qz * rP[3 * P + 2]), &sp, &cp);
  sincos(-(qx * rP[3 * Q] + qy * rP[3 * Q + 1] + qz * rP[3 * Q + 2]), &sq, &cq);
  // e^{-i q.r_P} conj(e^{-i q.r_Q}) = e^{i (aP - aQ)} with aP = -q.r_P
  const double cr = cp * cq + sp * sq, ci = sp * cq - cp * sq;
  const double2 w = W[i];
  A[i] = make_double2(c * (w.x * cr - w.y * ci), c * (w.x * ci + w.y * cr));
}

// The same, rounded to FP32, rows lda complex apart (the A operand of the
// tensor-core contraction).
__global__ void phase_w32(const double2* __restrict__ W, int np, const double* __restrict__ rP, double qx, double qy,
                          double qz, double c, float2* __restrict__ A, int lda) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * np) return;
  const int P = (int)(i / np), Q = (int)(i % np);
  double sp, cp, sq, cq;
  sincos(-(qx * rP[3 * P] + qy * rP[3 * P + 1] + qz * rP[3 * P + 2]), &sp, &cp);
  sincos(-(qx * rP[3 * Q] + qy * rP[3 * Q + 1] + qz * rP[3 * Q + 2]), &sq, &cq);
  const double cr = cp * cq + sp * sq, ci = sp * cq - cp * sq;
  const double2 w = W[i];
  A[(long)P * lda + Q] = make_float2((float)(c * (w.x * cr - w.y * ci)), (float)(c * (w.x * ci + w.y * cr)));
}

// Bq[Q][G] = v(G + q) conj(F[Q][flat[G]]), K = (gm[G] + qf) B, v(K) = 4 pi / |K|^2 (0 for K = 0)
__global__ void coulomb_conj(const double2* __restrict__ F, long ng, const int* __restrict__ flat,
                             const int* __restrict__ gm, int nG, int np, Recip B, double q0, double q1, double q2,
                             double2* __restrict__ Bq) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * nG) return;
  const int Q = (int)(i / nG), G = (int)(i % nG);
  const double f0 = gm[3 * G] + q0, f1 = gm[3 * G + 1] + q1, f2 = gm[3 * G + 2] + q2;
  const double kx = f0 * B.b[0] + f1 * B.b[3] + f2 * B.b[6];
  const double ky = f0 * B.b[1] + f1 * B.b[4] + f2 * B.b[7];
  const double kz = f0 * B.b[2] + f1 * B.b[5] + f2 * B.b[8];
  const double k2 = kx * kx + ky * ky + kz * kz;
  const double v = k2 > 1e-12 ? 4.0 * M_PI / k2 : 0.0;
  const double2 x = F[(long)Q * ng + flat[G]];
  Bq[i] = make_double2(v * x.x, -v * x.y);
}

// Y += X (complex)
__global__ void axpy_z(double2* __restrict__ Y, const double2* __restrict__ X, long n) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= n) return;
  Y[i] = make_double2(Y[i].x + X[i].x, Y[i].y + X[i].y);
}

// Gfull[P][flat[G]] = Gam[P][G] (Gfull zeroed before; flat entries distinct)
__global__ void scatter_g(const double2* __restrict__ Gam, int np, int nG, const int* __restrict__ flat, long ng,
                          double2* __restrict__ Gfull) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * nG) return;
  const int P = (int)(i / nG), G = (int)(i % nG);
  Gfull[(long)P * ng + flat[G]] = Gam[i];
}

// out[i] = Re X[i]
__global__ void real_part(const double2* __restrict__ X, long n, double* __restrict__ out) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= n) return;
  out[i] = X[i].x;
}

// C[m][n] = alpha sum_k A[m][k] B[n][k] (real, both operands k-contiguous);
// 32 x 32 output tiles, 256 threads with 2 x 2 outputs each, 32-deep k slabs.
constexpr int DT = 32;
__global__ void gemm_d_nt(int M, int N, long K, const double* __restrict__ A, long lda, const double* __restrict__ B,
                          long ldb, double* __restrict__ C, int ldc, double alpha) {
  __shared__ double As[DT][DT + 1], Bs[DT][DT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * DT, n0 = blockIdx.x * DT;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (long k0 = 0; k0 < K; k0 += DT) {
    for (int e = threadIdx.x; e < DT * DT; e += TB) {
      const int r = e / DT, kk = e % DT;
      const long gk = k0 + kk;
      As[r][kk] = (m0 + r < M && gk < K) ? A[(long)(m0 + r) * lda + gk] : 0.0;
      Bs[r][kk] = (n0 + r < N && gk < K) ? B[(long)(n0 + r) * ldb + gk] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < DT; kk++) {
      const double a0 = As[ty][kk], a1 = As[ty + 16][kk];
      const double b0 = Bs[tx][kk], b1 = Bs[tx + 16][kk];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) C[(long)m * ldc + n] = alpha * acc[i][j];
    }
}

// Lam[P][pts[Q]] += Sbar[P][Q]   (points distinct: no two threads share an address)
__global__ void add_point_cols(double* __restrict__ Lam, long ng, const int* __restrict__ pts, int np,
                               const double* __restrict__ Sbar) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * np) return;
  const int P = (int)(i / np), Q = (int)(i % np);
  Lam[(long)P * ng + pts[Q]] += Sbar[i];
}

// Bm[i] = 2 Rbar[i] conj(Bm[i])   (the adjoint of R = |B|^2, in place)
__global__ void abs2_adjoint(double2* __restrict__ Bm, const double* __restrict__ Rbar, long n) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= n) return;
  const double2 b = Bm[i];
  const double r = 2.0 * Rbar[i];
  Bm[i] = make_double2(r * b.x, -r * b.y);
}

// g = ce Ge + conj(G1) + G2; gexp = ce Ge (when given)
__global__ void combine_g(const double2* __restrict__ Ge, const double2* __restrict__ G1,
                          const double2* __restrict__ G2, long n, double ce, double2* __restrict__ g,
                          double2* __restrict__ gexp) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= n) return;
  const double2 e = make_double2(ce * Ge[i].x, ce * Ge[i].y);
  g[i] = make_double2(e.x + G1[i].x + G2[i].x, e.y - G1[i].y + G2[i].y);
  if (gexp) gexp[i] = e;
}

// dst[r][c] = (float2) src[r][c] for r < rows, c < cols (rows lds / ldd apart)
__global__ void to_f32_rows(const double2* __restrict__ src, long rows, int cols, long lds, float2* __restrict__ dst,
                            int ldd) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= rows * cols) return;
  const long r = i / cols;
  const int c = (int)(i % cols);
  const double2 v = src[r * lds + c];
  dst[r * ldd + c] = make_float2((float)v.x, (float)v.y);
}

// A[f][P] = conj(U[f][pts[P]]) in FP32, rows lda apart
__global__ void gather_conj_t32(const double2* __restrict__ U, int nf, long ng, const int* __restrict__ pts, int np,
                                float2* __restrict__ A, int lda) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)nf * np) return;
  const int f = (int)(i / np), P = (int)(i % np);
  const double2 u = U[(long)f * ng + pts[P]];
  A[(long)f * lda + P] = make_float2((float)u.x, (float)-u.y);
}

// out[b][m][n] = sum_k A[b][m][k] B[b](k, n) on the tensor cores, in the form of
// the kernel rebuild's contraction: A complex FP32 [batch][M][lda] (contiguous
// batches) sliced in the GEMM with its row exponents eA[b M + m]; B(k, n) =
// src[b sbs + k ldk + n ldj] complex128, embedded as three fp16 slices with
// exponents eB[b N + n] (no smaller than the exponent of max_k |B(k, n)|); 8
// slice products, exact K chunks of at most 1024 reals combined in FP64; out
// complex128 with rows ldo and batches sbo complex apart.  Allocates its planes
// and partial sums and frees them before returning.
cudaError_t tc_product(const float2* A, int lda, const int* eA, const double2* src, long sbs, long ldk, long ldj,
                       const int* eB, int batch, int M, int N, int K, double2* out, long ldo, long sbo, int* err,
                       cudaStream_t s) {
  if (batch > 1 && N > 65536) return cudaErrorInvalidValue;   // the embedding takes one slab of N per batch
  const int ldp = (2 * K + 7) & ~7;
  const long plane = (long)batch * 2 * N * ldp;
  const long npart = tc_partial_elems(M, 2 * N, 2 * K, batch);
  uint16_t* pl = nullptr;
  int* ps0 = nullptr;
  float* pbc = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&pl, sizeof(uint16_t) * 3 * (size_t)plane)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(pl, 0, sizeof(uint16_t) * 3 * (size_t)plane, s)) != cudaSuccess) break;
    if (npart > 0) {
      if ((e = cudaMalloc(&ps0, sizeof(int) * npart)) != cudaSuccess) break;
      if ((e = cudaMalloc(&pbc, sizeof(float) * npart)) != cudaSuccess) break;
    }
    TcOperand opA, opB;
    if ((e = make_f32_map(opA.map[0], A, batch, M, 2 * K, 2 * lda)) != cudaSuccess) break;
    for (int p = 0; p < 3 && e == cudaSuccess; p++) e = make_plane_map(opB.map[p], pl + p * plane, batch, 2 * N, 2 * K, ldp);
    if (e != cudaSuccess) break;
    if (batch == 1) {
      for (int n0 = 0; n0 < N && e == cudaSuccess; n0 += 65536)
        e = embed_b(src + n0 * ldj, true, 0, ldk, ldj, false, false, 1, K, std::min(65536, N - n0), eB + n0,
                    pl + 2L * n0 * ldp, plane, ldp, s);
    } else {
      e = embed_b(src, true, sbs, ldk, ldj, false, false, batch, K, N, eB, pl, plane, ldp, s);
    }
    if (e != cudaSuccess) break;
    e = tc_gemm(opA, opB, M, 2 * N, 2 * K, batch, eA, M, eB, N, out, true, 2 * ldo, 2 * sbo, ps0, pbc, err, s,
                nullptr, 8, 1, 0);
  } while (0);
  void* ptrs[] = {pl, ps0, pbc};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  return e;
}

}  // namespace

extern "C" thc_status thc_vo_gradient(const double* U, int nocc, const double* Uv, int nvir, const int* grid_host,
                                      const double* lattice_host, const int* mesh_host, const int* points_host,
                                      int npts, const double* V, int precision, double* g_out,
                                      double* g_explicit_out, double* ex_host, float* step_ms_host, void* stream) {
  if (!U || !Uv || !V || !g_out || !grid_host || !lattice_host || !mesh_host || !points_host || nocc < 1 ||
      nvir < 1 || npts < 1)
    return THC_ERR_ARG;
  if (precision != THC_FP64 && precision != THC_MIXED) return THC_ERR_ARG;
  if (((uintptr_t)U & 15) || ((uintptr_t)Uv & 15) || ((uintptr_t)V & 15) || ((uintptr_t)g_out & 15) ||
      ((uintptr_t)g_explicit_out & 15))
    return THC_ERR_ARG;
  FitGeom geo;
  if (!fit_geometry(grid_host, lattice_host, mesh_host, points_host, npts, geo)) return THC_ERR_ARG;
  const int g1 = geo.g[0], g2 = geo.g[1], g3 = geo.g[2];
  const int n1 = geo.n[0], n2 = geo.n[1], n3 = geo.n[2];
  const int nk = geo.nk;
  const long ng = geo.ng;
  const int nG = (int)geo.flat.size();
  const int np = npts;
  const long npq = (long)np * np;
  const int nf = nk * nocc;
  if ((long)nk * nocc > (1L << 30) || (long)nk * nvir > (1L << 30)) return THC_ERR_ARG;
  // mesh index tables: kq[k][q] = index of k + q, qk[k][k'] = index of k' - k
  std::vector<int> kq((size_t)nk * nk), qk((size_t)nk * nk);
  for (int k = 0; k < nk; k++)
    for (int j = 0; j < nk; j++) {
      const int a[3] = {k / (n2 * n3), (k / n3) % n2, k % n3};
      const int b[3] = {j / (n2 * n3), (j / n3) % n2, j % n3};
      kq[(size_t)k * nk + j] = (((a[0] + b[0]) % n1) * n2 + (a[1] + b[1]) % n2) * n3 + (a[2] + b[2]) % n3;
      qk[(size_t)k * nk + j] =
          (((b[0] - a[0] + n1) % n1) * n2 + (b[1] - a[1] + n2) % n2) * n3 + (b[2] - a[2] + n3) % n3;
    }

  cudaStream_t s = (cudaStream_t)stream;
  // step boundaries: 0 start, 1 after the fixed-kernel part (D, W, M, Y, g_e),
  // 2 after the fit, 3 after the (q, G) contraction, 4 after the DFT adjoint,
  // the solve and S-bar, 5 after the orbital adjoint and the sum
  cudaEvent_t ev[6] = {};
  if (step_ms_host)
    for (auto& x : ev)
      if (cudaEventCreate(&x) != cudaSuccess) x = nullptr;
  auto mark = [&](int i) {
    if (step_ms_host && ev[i]) cudaEventRecord(ev[i], s);
  };
  const int NPART = 1024;
  double2 *Psi = nullptr, *Psivt = nullptr, *D = nullptr, *M = nullptr, *W = nullptr, *Y = nullptr, *Ge = nullptr;
  double2 *Ugc = nullptr, *Bm = nullptr, *F = nullptr, *T = nullptr, *Gam = nullptr, *Aq = nullptr, *Bq = nullptr;
  double2 *Z = nullptr, *T1 = nullptr, *T2 = nullptr, *Uvp = nullptr, *G1 = nullptr, *G2 = nullptr, *twd = nullptr;
  double *R = nullptr, *S = nullptr, *L = nullptr, *Lam = nullptr, *Sbar = nullptr, *rPd = nullptr, *part = nullptr;
  int *ptsd = nullptr, *gmd = nullptr, *flatd = nullptr, *bad = nullptr, *kqd = nullptr, *qkd = nullptr;
  // tensor-core state of the (q, G) contraction (THC_MIXED)
  float2* Aq32 = nullptr;
  uint16_t* Bpl = nullptr;
  int *eA = nullptr, *eB = nullptr, *ps0 = nullptr, *tcerr = nullptr;
  float* pbc = nullptr;
  // ... and of the orbital contractions
  float2 *Y32 = nullptr, *A2 = nullptr, *Uv32 = nullptr;
  int* eOrb = nullptr;
  cudaError_t e = cudaSuccess;
  thc_status st = THC_OK;
  int hbad = 0;
  std::vector<double> hpart(NPART, 0.0);
  const long ngo = (long)nk * nvir * nocc;
  do {
#define ALLOC(p, n) \
  if ((e = cudaMalloc(&p, sizeof(*p) * (size_t)(n))) != cudaSuccess) break
    ALLOC(ptsd, np);
    ALLOC(kqd, (long)nk * nk);
    ALLOC(qkd, (long)nk * nk);
    ALLOC(twd, geo.tw.size());
    ALLOC(gmd, geo.gm.size());
    ALLOC(flatd, geo.flat.size());
    ALLOC(rPd, geo.rP.size());
    ALLOC(bad, 1);
    ALLOC(part, NPART);
    ALLOC(Psi, (long)nk * np * nocc);
    ALLOC(Psivt, (long)nk * nvir * np);
    ALLOC(D, nk * npq);
    ALLOC(M, nk * npq);
    ALLOC(W, nk * npq);
    ALLOC(Y, (long)nk * np * nocc);
    ALLOC(Ge, ngo);
#undef ALLOC
    if ((e = cudaMemcpyAsync(ptsd, points_host, sizeof(int) * np, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(kqd, kq.data(), sizeof(int) * kq.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(qkd, qk.data(), sizeof(int) * qk.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(twd, geo.tw.data(), sizeof(double2) * geo.tw.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(gmd, geo.gm.data(), sizeof(int) * geo.gm.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(flatd, geo.flat.data(), sizeof(int) * geo.flat.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(rPd, geo.rP.data(), sizeof(double) * geo.rP.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemsetAsync(bad, 0, sizeof(int), s)) != cudaSuccess) break;

    // 1. the kernel held fixed: Psi, Psi_v at the points, D, W, M, Y, E_x, g_e
    mark(0);
    const double2* U2 = (const double2*)U;
    const double2* Uv2 = (const double2*)Uv;
    point_values<<<blocks((long)nk * nocc * np), TB, 0, s>>>(U2, nk, nocc, ng, ptsd, np, g1, g2, g3, n1, n2, n3,
                                                             true, false, Psi);
    point_values<<<blocks((long)nk * nvir * np), TB, 0, s>>>(Uv2, nk, nvir, ng, ptsd, np, g1, g2, g3, n1, n2, n3,
                                                             true, true, Psivt);
    if ((e = gemm_z(A_MK, B_NK_CONJ, np, np, nocc, Psi, nocc, (long)np * nocc, Psi, nocc, (long)np * nocc, D, np,
                    npq, nk, s)) != cudaSuccess)
      break;
    kcorr_kernel<<<blocks(npq), TB, 0, s>>>(D, (const double2*)V, kqd, qkd, nk, npq, W, M);
    wv_partial<<<NPART, TB, 0, s>>>(W, (const double2*)V, nk * npq, part);
    if (ex_host &&
        (e = cudaMemcpyAsync(hpart.data(), part, sizeof(double) * NPART, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      break;
    if ((e = gemm_z(A_MK, B_KN, np, nocc, np, M, np, npq, Psi, nocc, (long)np * nocc, Y, nocc, (long)np * nocc, nk,
                    s)) != cudaSuccess)
      break;
    if ((e = gemm_z(A_MK_CONJ, B_KN, nvir, nocc, np, Psivt, np, (long)nvir * np, Y, nocc, (long)np * nocc, Ge, nocc,
                    (long)nvir * nocc, nk, s)) != cudaSuccess)
      break;
    cudaFree(D);
    cudaFree(M);
    cudaFree(Y);
    cudaFree(Psi);
    cudaFree(Psivt);
    D = M = Y = Psi = Psivt = nullptr;

    // 2. the fit: B = conj(U_P)^T U, R = |B|^2, S = R[:, points], L L^T = S, xi = S^-1 R, F = DFT(xi)
    mark(1);
    if ((e = cudaMalloc(&Ugc, sizeof(double2) * (size_t)np * nf)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Bm, sizeof(double2) * (size_t)np * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&R, sizeof(double) * (size_t)np * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&S, sizeof(double) * npq)) != cudaSuccess) break;
    if ((e = cudaMalloc(&L, sizeof(double) * npq)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(L, 0, sizeof(double) * npq, s)) != cudaSuccess) break;
    gather_conj<<<blocks((long)np * nf), TB, 0, s>>>(U2, nf, ng, ptsd, np, Ugc);
    if ((e = gemm_z(A_MK, B_KN, np, (int)ng, nf, Ugc, nf, 0, U2, (int)ng, 0, Bm, (int)ng, 0, 1, s)) != cudaSuccess)
      break;
    abs2_kernel<<<blocks((long)np * ng), TB, 0, s>>>(Bm, (long)np * ng, R);
    gather_cols<<<blocks(npq), TB, 0, s>>>(R, ng, ptsd, np, S);
    for (int j = 0; j < np; j++) chol_column<<<blocks(np - j), TB, 0, s>>>(S, L, np, j, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    if (hbad) {
      st = THC_ERR_ARG;
      set_global_error("thc_vo_gradient: the Gram matrix of the points is not positive definite");
      break;
    }
    chol_solve<<<blocks(ng), TB, 0, s>>>(L, R, np, ng);   // R now holds xi
    if ((e = cudaMalloc(&F, sizeof(double2) * (size_t)np * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&T, sizeof(double2) * (size_t)np * ng)) != cudaSuccess) break;
    const long tot = (long)np * ng;
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(R, true, F, tot, g3, 1, twd + geo.off[2]);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(F, false, T, tot, g2, g3, twd + geo.off[1]);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(T, false, F, tot, g1, (long)g2 * g3, twd + geo.off[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) break;

    // 3. Gam = sum over q and its representatives of (c ph W^q ph^H) (v o conj(xh))
    mark(2);
    if ((e = cudaMalloc(&Gam, sizeof(double2) * (size_t)np * nG)) != cudaSuccess) break;
    if (precision == THC_FP64 && (e = cudaMalloc(&Aq, sizeof(double2) * npq)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Bq, sizeof(double2) * (size_t)np * nG)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Z, sizeof(double2) * (size_t)np * nG)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(Gam, 0, sizeof(double2) * (size_t)np * nG, s)) != cudaSuccess) break;
    // THC_MIXED: Z = A Bq on the tensor cores, A (FP32, sliced in the GEMM with
    // its row exponents) against the embedded Bq (three fp16 slices with the
    // exact column exponents of the FP64 Bq), 8 slice products, exact K chunks
    // of at most 1024 reals combined in FP64
    const bool tc = precision == THC_MIXED;
    const int lda = np + (np & 1);                    // FP32 rows 16-byte strided
    const int ldp = (2 * np + 7) & ~7;                // B plane rows: 2 np reals, padded
    const long plane = 2L * nG * ldp;
    TcOperand opA, opB;
    if (tc) {
      const long npart = tc_partial_elems(np, 2 * nG, 2 * np, 1);
      if ((e = cudaMalloc(&Aq32, sizeof(float2) * (size_t)np * lda)) != cudaSuccess) break;
      if ((e = cudaMalloc(&Bpl, sizeof(uint16_t) * 3 * (size_t)plane)) != cudaSuccess) break;
      if ((e = cudaMalloc(&eA, sizeof(int) * np)) != cudaSuccess) break;
      if ((e = cudaMalloc(&eB, sizeof(int) * nG)) != cudaSuccess) break;
      if ((e = cudaMalloc(&tcerr, 64)) != cudaSuccess) break;
      if (npart > 0) {
        if ((e = cudaMalloc(&ps0, sizeof(int) * npart)) != cudaSuccess) break;
        if ((e = cudaMalloc(&pbc, sizeof(float) * npart)) != cudaSuccess) break;
      }
      if ((e = cudaMemsetAsync(tcerr, 0, 64, s)) != cudaSuccess) break;
      if ((e = cudaMemsetAsync(Aq32, 0, sizeof(float2) * (size_t)np * lda, s)) != cudaSuccess) break;
      if ((e = cudaMemsetAsync(Bpl, 0, sizeof(uint16_t) * 3 * (size_t)plane, s)) != cudaSuccess) break;
      if ((e = make_f32_map(opA.map[0], Aq32, 1, np, 2 * np, 2 * lda)) != cudaSuccess) break;
      for (int p = 0; p < 3 && e == cudaSuccess; p++)
        e = make_plane_map(opB.map[p], Bpl + p * plane, 1, 2 * nG, 2 * np, ldp);
      if (e != cudaSuccess) break;
    }
    const double sc = geo.vol / ng;
    const Recip& B = geo.B;
    for (int q = 0; q < nk && e == cudaSuccess; q++) {
      const int qc[3] = {q / (n2 * n3), (q / n3) % n2, q % n3};
      const std::vector<double> r0 = axis_reps(qc[0], n1), r1 = axis_reps(qc[1], n2), r2 = axis_reps(qc[2], n3);
      const double nrep = (double)(r0.size() * r1.size() * r2.size());
      const double c = -2.0 / nk * sc * sc / (nrep * nk * geo.vol);
      for (double x0 : r0)
        for (double x1 : r1)
          for (double x2 : r2) {
            if (e != cudaSuccess) break;
            const double qx = x0 * B.b[0] + x1 * B.b[3] + x2 * B.b[6];
            const double qy = x0 * B.b[1] + x1 * B.b[4] + x2 * B.b[7];
            const double qz = x0 * B.b[2] + x1 * B.b[5] + x2 * B.b[8];
            coulomb_conj<<<blocks((long)np * nG), TB, 0, s>>>(F, ng, flatd, gmd, nG, np, B, x0, x1, x2, Bq);
            if (!tc) {
              phase_w<<<blocks(npq), TB, 0, s>>>(W + (long)q * npq, np, rPd, qx, qy, qz, c, Aq);
              if ((e = gemm_z(A_MK, B_KN, np, nG, np, Aq, np, 0, Bq, nG, 0, Z, nG, 0, 1, s)) != cudaSuccess) break;
            } else {
              phase_w32<<<blocks(npq), TB, 0, s>>>(W + (long)q * npq, np, rPd, qx, qy, qz, c, Aq32, lda);
              if ((e = row_exponents_c(Aq32, 0, lda, 1, np, np, eA, s)) != cudaSuccess) break;
              if ((e = col_exponents_z(Bq, 0, nG, 1, np, nG, eB, s)) != cudaSuccess) break;
              // embedded in slabs of G (the embedding's grid holds at most 131,070 rows j)
              for (int g0 = 0; g0 < nG && e == cudaSuccess; g0 += 65536)
                e = embed_b(Bq + g0, true, 0, nG, 1, false, false, 1, np, std::min(65536, nG - g0), eB + g0,
                            Bpl + 2L * g0 * ldp, plane, ldp, s);
              if (e != cudaSuccess) break;
              if ((e = tc_gemm(opA, opB, np, 2 * nG, 2 * np, 1, eA, np, eB, nG, Z, true, 2L * nG, 2L * np * nG, ps0,
                               pbc, tcerr, s, nullptr, 8, 1, 0)) != cudaSuccess)
                break;
            }
            axpy_z<<<blocks((long)np * nG), TB, 0, s>>>(Gam, Z, (long)np * nG);
          }
    }
    if (e != cudaSuccess) break;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    cudaFree(Aq);
    cudaFree(Bq);
    cudaFree(Z);
    cudaFree(W);
    Aq = Bq = Z = W = nullptr;

    // 4. Xbar = Re DFT(Gam on the grid), Lam = S^-1 Xbar, Rbar = Lam + (S-bar at the point columns)
    mark(3);
    if ((e = cudaMemsetAsync(F, 0, sizeof(double2) * (size_t)np * ng, s)) != cudaSuccess) break;
    scatter_g<<<blocks((long)np * nG), TB, 0, s>>>(Gam, np, nG, flatd, ng, F);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(F, false, T, tot, g3, 1, twd + geo.off[2]);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(T, false, F, tot, g2, g3, twd + geo.off[1]);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(F, false, T, tot, g1, (long)g2 * g3, twd + geo.off[0]);
    if ((e = cudaMalloc(&Lam, sizeof(double) * (size_t)np * ng)) != cudaSuccess) break;
    real_part<<<blocks(tot), TB, 0, s>>>(T, tot, Lam);
    chol_solve<<<blocks(ng), TB, 0, s>>>(L, Lam, np, ng);
    if ((e = cudaMalloc(&Sbar, sizeof(double) * npq)) != cudaSuccess) break;
    {
      dim3 grid((np + DT - 1) / DT, (np + DT - 1) / DT);
      gemm_d_nt<<<grid, TB, 0, s>>>(np, np, ng, Lam, ng, R, ng, Sbar, np, -1.0);
    }
    add_point_cols<<<blocks(npq), TB, 0, s>>>(Lam, ng, ptsd, np, Sbar);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    cudaFree(F);
    cudaFree(T);
    cudaFree(Gam);
    F = T = Gam = nullptr;

    // 5. Y2 = 2 Rbar conj(B); T1[P][f] = sum_r Y2[P][r] U[f][r], T2 = conj(U_P)^T Y2; g_r from Uv;
    //    g = g_e + g_r
    mark(4);
    abs2_adjoint<<<blocks(tot), TB, 0, s>>>(Bm, Lam, tot);
    if ((e = cudaMalloc(&T1, sizeof(double2) * (size_t)nf * np)) != cudaSuccess) break;
    if ((e = cudaMalloc(&T2, sizeof(double2) * (size_t)nf * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Uvp, sizeof(double2) * (size_t)nk * nvir * np)) != cudaSuccess) break;
    if ((e = cudaMalloc(&G1, sizeof(double2) * ngo)) != cudaSuccess) break;
    if ((e = cudaMalloc(&G2, sizeof(double2) * ngo)) != cudaSuccess) break;
    // THC_MIXED: T1, T2 and the projection of T2 on the tensor cores when the
    // grid sum fits the exact K chunks of one product (2 N_g reals in at most
    // 126 chunks of 1024); else, and in THC_FP64, FP64 GEMMs
    const bool tc_orb = tc && 2L * ng <= 126L * 1024;
    if (!tc_orb) {
      if ((e = gemm_z(A_MK, B_NK, np, nf, (int)ng, Bm, (int)ng, 0, U2, (int)ng, 0, T1, nf, 0, 1, s)) != cudaSuccess)
        break;
      if ((e = gemm_z(A_KM, B_KN, nf, (int)ng, np, Ugc, nf, 0, Bm, (int)ng, 0, T2, (int)ng, 0, 1, s)) !=
          cudaSuccess)
        break;
      if ((e = gemm_z(A_MK, B_NK, nvir, nocc, (int)ng, Uv2, (int)ng, (long)nvir * ng, T2, (int)ng, (long)nocc * ng,
                      G1, nocc, (long)nvir * nocc, nk, s)) != cudaSuccess)
        break;
    } else {
      const int ldy = (int)(ng + (ng & 1));           // FP32 grid rows 16-byte strided
      const int lda2 = np + (np & 1);
      const long nfv = (long)nk * nvir;
      if ((e = cudaMalloc(&Y32, sizeof(float2) * (size_t)np * ldy)) != cudaSuccess) break;
      if ((e = cudaMalloc(&A2, sizeof(float2) * (size_t)nf * lda2)) != cudaSuccess) break;
      if ((e = cudaMalloc(&Uv32, sizeof(float2) * (size_t)nfv * ldy)) != cudaSuccess) break;
      if ((e = cudaMalloc(&eOrb, sizeof(int) * (size_t)(np + 3L * nf + ng + nfv))) != cudaSuccess) break;
      int* eY = eOrb;
      int* eU = eY + np;
      int* eA2 = eU + nf;
      int* eT2 = eA2 + nf;
      int* eBm = eT2 + nf;
      int* eUv = eBm + ng;
      // T1[P][f] = sum_r Y2[P][r] U[f][r]
      to_f32_rows<<<blocks((long)np * ng), TB, 0, s>>>(Bm, np, (int)ng, ng, Y32, ldy);
      if ((e = row_exponents_c(Y32, 0, ldy, 1, np, (int)ng, eY, s)) != cudaSuccess) break;
      if ((e = row_exponents_z(U2, 0, (int)ng, 1, nf, (int)ng, eU, s)) != cudaSuccess) break;
      if ((e = tc_product(Y32, ldy, eY, U2, 0, 1, ng, eU, 1, np, nf, (int)ng, T1, nf, 0, tcerr, s)) != cudaSuccess)
        break;
      // T2[f][r] = sum_P conj(U[f][r_P]) Y2[P][r]
      gather_conj_t32<<<blocks((long)nf * np), TB, 0, s>>>(U2, nf, ng, ptsd, np, A2, lda2);
      if ((e = row_exponents_c(A2, 0, lda2, 1, nf, np, eA2, s)) != cudaSuccess) break;
      if ((e = col_exponents_z(Bm, 0, (int)ng, 1, np, (int)ng, eBm, s)) != cudaSuccess) break;
      if ((e = tc_product(A2, lda2, eA2, Bm, 0, ng, 1, eBm, 1, nf, (int)ng, np, T2, ng, 0, tcerr, s)) !=
          cudaSuccess)
        break;
      // G1^k[a][i] = sum_r Uv[(k,a)][r] T2[(k,i)][r]
      to_f32_rows<<<blocks(nfv * ng), TB, 0, s>>>(Uv2, nfv, (int)ng, ng, Uv32, ldy);
      if ((e = row_exponents_c(Uv32, 0, ldy, 1, (int)nfv, (int)ng, eUv, s)) != cudaSuccess) break;
      if ((e = row_exponents_z(T2, 0, (int)ng, 1, nf, (int)ng, eT2, s)) != cudaSuccess) break;
      if ((e = tc_product(Uv32, ldy, eUv, T2, (long)nocc * ng, 1, ng, eT2, nk, nvir, nocc, (int)ng, G1, nocc,
                          (long)nvir * nocc, tcerr, s)) != cudaSuccess)
        break;
    }
    point_values<<<blocks((long)nk * nvir * np), TB, 0, s>>>(Uv2, nk, nvir, ng, ptsd, np, g1, g2, g3, n1, n2, n3,
                                                             false, true, Uvp);
    if ((e = gemm_z(A_MK_CONJ, B_KN, nvir, nocc, np, Uvp, np, (long)nvir * np, T1, nf, nocc, G2, nocc,
                    (long)nvir * nocc, nk, s)) != cudaSuccess)
      break;
    combine_g<<<blocks(ngo), TB, 0, s>>>(Ge, G1, G2, ngo, -4.0 / nk, (double2*)g_out, (double2*)g_explicit_out);
    mark(5);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    if (tcerr) {
      int h = 0;
      if ((e = cudaMemcpy(&h, tcerr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
      if (h) {
        st = THC_ERR_TIMEOUT;
        set_global_error("thc_vo_gradient: a device wait of the tensor-core contraction timed out");
        break;
      }
    }
    if (ex_host) {
      double acc = 0.0;
      for (int i = 0; i < NPART; i++) acc += hpart[i];
      *ex_host = -acc / nk;
    }
    if (step_ms_host)
      for (int i = 0; i < 5; i++) {
        step_ms_host[i] = 0.f;
        if (ev[i] && ev[i + 1]) cudaEventElapsedTime(&step_ms_host[i], ev[i], ev[i + 1]);
      }
  } while (0);
  if (e != cudaSuccess) {
    set_global_error(std::string("thc_vo_gradient: ") + cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
  }
  void* ptrs[] = {Psi, Psivt, D,   M,   W,  Y,  Ge,  Ugc,   Bm,    F,    T,     Gam,  Aq,  Bq,  Z,
                  T1,  T2,    Uvp, G1,  G2, twd, R,  S,     L,     Lam,  Sbar,  rPd,  part, ptsd, gmd,
                  flatd, bad, kqd, qkd, Aq32, Bpl, eA,  eB,  ps0, pbc, tcerr, Y32, A2, Uv32, eOrb};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  return st;
}
