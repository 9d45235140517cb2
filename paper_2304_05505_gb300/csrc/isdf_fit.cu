// ISDF kernel fit (setup, not part of the timed build), FP64 throughout.
//
// Given the occupied orbitals' periodic parts on the grid, U[f][r] = u^k_i(r)
// with f = (k, i), and the interpolation points r_P:
//   1. the fit's right-hand side and metric (the least-squares fit of
//      Eq. pbcinterpvec restricted to occupied products, Eq. orbprodoo):
//        B[P][r] = sum_f conj(U[f][r_P]) U[f][r],   R[P][r] = |B[P][r]|^2,
//        S = R[:, points]
//   2. the interpolation vectors xi = S^-1 R (Cholesky S = L L^T, then one
//      forward and one backward substitution per grid column);
//   3. their reciprocal-space form xh_P(G) = (Omega/N_g) sum_r xi_P(r) e^{-iG.r}
//      (a separable 3-D DFT, one axis at a time, on the G set without the
//      Nyquist planes);
//   4. the kernel of every q (Sec. 2.2), with the pair phase folded in:
//        V^q[P,Q] = 1/(N_k Omega) mean over the representatives q_r of q of
//                   sum_G v(G + q_r) (xh_P(G) e^{-i q_r.r_P}) conj(xh_Q(G) e^{-i q_r.r_Q})
//      one Hermitian product per representative (v(K) = 4 pi / |K|^2, K = 0
//      left out).
// Steps 1-3 and the Cholesky factor run in FP64 (the ill-conditioned
// least-squares metric).  Step 4, the O(N_k N_P^2 N_G) contraction that
// dominates the per-iteration rebuild of Algorithm 2, runs in FP64 on CUDA
// cores (THC_FP64) or on the tcgen05 tensor cores (THC_MIXED): each scaled
// vector set Xq is rounded to FP32 and sliced inside the GEMM, three fp16
// slices, 8 slice products, the leading products summed exactly in K chunks of
// at most 1024 reals; chunks are combined in FP64.
#include "isdf_common.cuh"
#include "tc_gemm.cuh"

namespace {

// Xq[P][G] = F[P][flat[G]] * sqrt(w v(G + q)) * exp(-i q.r_P), with
// K = (gm[G] + qf) B (Cartesian) and v(K) = 4 pi / |K|^2 (0 for K = 0).
__global__ void scale_xi(const double2* __restrict__ F, long ng, const int* __restrict__ flat,
                         const int* __restrict__ gm, int nG, const double* __restrict__ rP, int np, Recip B,
                         double q0, double q1, double q2, double w, double2* __restrict__ Xq) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * nG) return;
  const int P = (int)(i / nG), G = (int)(i % nG);
  const double f0 = gm[3 * G] + q0, f1 = gm[3 * G + 1] + q1, f2 = gm[3 * G + 2] + q2;
  const double kx = f0 * B.b[0] + f1 * B.b[3] + f2 * B.b[6];
  const double ky = f0 * B.b[1] + f1 * B.b[4] + f2 * B.b[7];
  const double kz = f0 * B.b[2] + f1 * B.b[5] + f2 * B.b[8];
  const double k2 = kx * kx + ky * ky + kz * kz;
  const double sv = k2 > 1e-12 ? sqrt(w * 4.0 * M_PI / k2) : 0.0;
  const double qx = q0 * B.b[0] + q1 * B.b[3] + q2 * B.b[6];
  const double qy = q0 * B.b[1] + q1 * B.b[4] + q2 * B.b[7];
  const double qz = q0 * B.b[2] + q1 * B.b[5] + q2 * B.b[8];
  double s, c;
  sincos(-(qx * rP[3 * P] + qy * rP[3 * P + 1] + qz * rP[3 * P + 2]), &s, &c);
  const double2 x = F[(long)P * ng + flat[G]];
  Xq[i] = make_double2(sv * (x.x * c - x.y * s), sv * (x.x * s + x.y * c));
}

// The same, rounded to FP32, rows ldq complex apart.
__global__ void scale_xi_f32(const double2* __restrict__ F, long ng, const int* __restrict__ flat,
                             const int* __restrict__ gm, int nG, const double* __restrict__ rP, int np, Recip B,
                             double q0, double q1, double q2, double w, float2* __restrict__ Xq, int ldq) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * nG) return;
  const int P = (int)(i / nG), G = (int)(i % nG);
  const double f0 = gm[3 * G] + q0, f1 = gm[3 * G + 1] + q1, f2 = gm[3 * G + 2] + q2;
  const double kx = f0 * B.b[0] + f1 * B.b[3] + f2 * B.b[6];
  const double ky = f0 * B.b[1] + f1 * B.b[4] + f2 * B.b[7];
  const double kz = f0 * B.b[2] + f1 * B.b[5] + f2 * B.b[8];
  const double k2 = kx * kx + ky * ky + kz * kz;
  const double sv = k2 > 1e-12 ? sqrt(w * 4.0 * M_PI / k2) : 0.0;
  const double qx = q0 * B.b[0] + q1 * B.b[3] + q2 * B.b[6];
  const double qy = q0 * B.b[1] + q1 * B.b[4] + q2 * B.b[7];
  const double qz = q0 * B.b[2] + q1 * B.b[5] + q2 * B.b[8];
  double s, c;
  sincos(-(qx * rP[3 * P] + qy * rP[3 * P + 1] + qz * rP[3 * P + 2]), &s, &c);
  const double2 x = F[(long)P * ng + flat[G]];
  Xq[(long)P * ldq + G] = make_float2((float)(sv * (x.x * c - x.y * s)), (float)(sv * (x.x * s + x.y * c)));
}

// V += W (complex)
__global__ void add_kernel(double2* __restrict__ V, const double2* __restrict__ W, long n) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= n) return;
  V[i] = make_double2(V[i].x + W[i].x, V[i].y + W[i].y);
}

// V += (W + W^H) / 2 for one [np][np] matrix (complex): the tensor-core
// product computes W[P][Q] and W[Q][P] apart, so their roundings differ; its
// Hermitian part is the same quantity, exactly Hermitian.
__global__ void add_herm_kernel(double2* __restrict__ V, const double2* __restrict__ W, int np) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * np) return;
  const int P = (int)(i / np), Q = (int)(i % np);
  const double2 a = W[i], b = W[(long)Q * np + P];
  V[i] = make_double2(V[i].x + 0.5 * (a.x + b.x), V[i].y + 0.5 * (a.y - b.y));
}


// G vectors per tensor-core product of step 4: at most 60,000 complex (120,000
// real K, under the 127 exact K chunks of 1024 a product may take), even so
// that every slab starts 16-byte aligned.
constexpr int G_SLAB = 60000;

thc_status fit_impl(const double* U, int nfunc, const int* grid_host, const double* lattice_host,
                    const int* mesh_host, const int* points_host, int npts, double* V_out, double* xi_out,
                    int precision, float* step_ms, void* stream) {
  if (precision != THC_FP64 && precision != THC_MIXED) return THC_ERR_ARG;
  if (!U || !grid_host || !lattice_host || !mesh_host || !points_host || !V_out || nfunc < 1 || npts < 1)
    return THC_ERR_ARG;
  if (((uintptr_t)U & 15) || ((uintptr_t)V_out & 15) || ((uintptr_t)xi_out & 7)) return THC_ERR_ARG;
  FitGeom geo;
  if (!fit_geometry(grid_host, lattice_host, mesh_host, points_host, npts, geo)) return THC_ERR_ARG;
  const int g1 = geo.g[0], g2 = geo.g[1], g3 = geo.g[2];
  const int n1 = geo.n[0], n2 = geo.n[1], n3 = geo.n[2];
  const long ng = geo.ng;
  const double vol = geo.vol;
  const Recip B = geo.B;
  const std::vector<int>& gm = geo.gm;
  const std::vector<int>& flat = geo.flat;
  const int nG = (int)flat.size();
  const std::vector<double>& rP = geo.rP;
  const std::vector<double2>& tw = geo.tw;
  const int* off = geo.off;

  cudaStream_t s = (cudaStream_t)stream;
  const int nk = n1 * n2 * n3;
  const long npq = (long)npts * npts;
  // step boundaries: 0 start, 1 after B R S, 2 after Cholesky, 3 after the
  // solve, 4 after the DFT, 5 after the kernel contraction
  cudaEvent_t ev[6] = {};
  if (step_ms)
    for (auto& x : ev)
      if (cudaEventCreate(&x) != cudaSuccess) x = nullptr;
  auto mark = [&](int i) {
    if (step_ms && ev[i]) cudaEventRecord(ev[i], s);
  };
  // tensor-core state of step 4 (THC_MIXED)
  float2* Xq32 = nullptr;
  uint16_t* Bpl = nullptr;
  int *eX = nullptr, *ps0 = nullptr, *tcerr = nullptr;
  float* pbc = nullptr;
  double2 *Ugc = nullptr, *Bm = nullptr, *F = nullptr, *Xq = nullptr, *W = nullptr, *twd = nullptr;
  double *R = nullptr, *S = nullptr, *L = nullptr, *rPd = nullptr;
  int *ptsd = nullptr, *gmd = nullptr, *flatd = nullptr, *bad = nullptr;
  cudaError_t e = cudaSuccess;
  thc_status st = THC_OK;
  int hbad = 0;
  do {
    if ((e = cudaMalloc(&ptsd, sizeof(int) * npts)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Ugc, sizeof(double2) * (size_t)npts * nfunc)) != cudaSuccess) break;
    if ((e = cudaMalloc(&Bm, sizeof(double2) * (size_t)npts * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&R, sizeof(double) * (size_t)npts * ng)) != cudaSuccess) break;
    if ((e = cudaMalloc(&S, sizeof(double) * npq)) != cudaSuccess) break;
    if ((e = cudaMalloc(&L, sizeof(double) * npq)) != cudaSuccess) break;
    if ((e = cudaMalloc(&bad, sizeof(int))) != cudaSuccess) break;
    if ((e = cudaMalloc(&twd, sizeof(double2) * tw.size())) != cudaSuccess) break;
    if ((e = cudaMalloc(&gmd, sizeof(int) * gm.size())) != cudaSuccess) break;
    if ((e = cudaMalloc(&flatd, sizeof(int) * flat.size())) != cudaSuccess) break;
    if ((e = cudaMalloc(&rPd, sizeof(double) * rP.size())) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(ptsd, points_host, sizeof(int) * npts, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(twd, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(gmd, gm.data(), sizeof(int) * gm.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(flatd, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(rPd, rP.data(), sizeof(double) * rP.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      break;
    if ((e = cudaMemsetAsync(bad, 0, sizeof(int), s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(L, 0, sizeof(double) * npq, s)) != cudaSuccess) break;
    // 1. B = conj(U[:, points])^T U, R = |B|^2, S = R[:, points]
    mark(0);
    gather_conj<<<blocks((long)npts * nfunc), TB, 0, s>>>((const double2*)U, nfunc, ng, ptsd, npts, Ugc);
    if ((e = gemm_z(A_MK, B_KN, npts, (int)ng, nfunc, Ugc, nfunc, 0, (const double2*)U, (int)ng, 0, Bm, (int)ng,
                    0, 1, s)) != cudaSuccess)
      break;
    abs2_kernel<<<blocks((long)npts * ng), TB, 0, s>>>(Bm, (long)npts * ng, R);
    gather_cols<<<blocks(npq), TB, 0, s>>>(R, ng, ptsd, npts, S);
    // 2. xi = S^-1 R
    mark(1);
    for (int j = 0; j < npts; j++) chol_column<<<blocks(npts - j), TB, 0, s>>>(S, L, npts, j, bad);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    if (hbad) {
      st = THC_ERR_ARG;   // the metric of these points is not positive definite
      set_global_error("thc_fit_kernel: the Gram matrix of the points is not positive definite");
      break;
    }
    mark(2);
    chol_solve<<<blocks(ng), TB, 0, s>>>(L, R, npts, ng);
    mark(3);
    if (xi_out &&
        (e = cudaMemcpyAsync(xi_out, R, sizeof(double) * npts * ng, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      break;
    // 3. xh = DFT of xi, axis by axis (Bm holds the last two passes' input/output)
    cudaFree(Ugc);
    Ugc = nullptr;
    if ((e = cudaMalloc(&F, sizeof(double2) * (size_t)npts * ng)) != cudaSuccess) break;
    const long tot = (long)npts * ng;
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(R, true, F, tot, g3, 1, twd + off[2]);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(F, false, Bm, tot, g2, g3, twd + off[1]);
    dft_axis_kernel<<<blocks(tot), TB, 0, s>>>(Bm, false, F, tot, g1, (long)g2 * g3, twd + off[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    mark(4);
    // 4. V^q, one Hermitian product per representative of q
    cudaFree(Bm);
    Bm = nullptr;
    const bool tc = precision == THC_MIXED;
    const int ldq = nG + (nG & 1);                    // FP32 rows 16-byte strided
    const int slab = std::min(nG, G_SLAB);
    const int ldb = (2 * slab + 7) & ~7;              // B plane rows: 2 slab reals, padded
    const long plane = 2L * npts * ldb;
    long npart = 0;
    if (tc) {
      for (int g0 = 0; g0 < nG; g0 += slab) npart = std::max(npart, tc_partial_elems(npts, 2 * npts, 2 * std::min(slab, nG - g0), 1));
      if ((e = cudaMalloc(&Xq32, sizeof(float2) * (size_t)npts * ldq)) != cudaSuccess) break;
      if ((e = cudaMalloc(&Bpl, 3 * 2 * (size_t)plane)) != cudaSuccess) break;
      if ((e = cudaMalloc(&eX, sizeof(int) * npts)) != cudaSuccess) break;
      if ((e = cudaMalloc(&tcerr, 64)) != cudaSuccess) break;
      if ((e = cudaMemsetAsync(tcerr, 0, 64, s)) != cudaSuccess) break;
      if ((e = cudaMemsetAsync(Xq32, 0, sizeof(float2) * (size_t)npts * ldq, s)) != cudaSuccess) break;
      if ((e = cudaMemsetAsync(Bpl, 0, 3 * 2 * (size_t)plane, s)) != cudaSuccess) break;
      if (npart > 0) {
        if ((e = cudaMalloc(&ps0, sizeof(int) * npart)) != cudaSuccess) break;
        if ((e = cudaMalloc(&pbc, sizeof(float) * npart)) != cudaSuccess) break;
      }
    } else if ((e = cudaMalloc(&Xq, sizeof(double2) * (size_t)npts * nG)) != cudaSuccess) {
      break;
    }
    if ((e = cudaMalloc(&W, sizeof(double2) * npq)) != cudaSuccess) break;
    double2* V = (double2*)V_out;
    if ((e = cudaMemsetAsync(V, 0, sizeof(double2) * nk * npq, s)) != cudaSuccess) break;
    const double sc = vol / ng;   // xh = (Omega / N_g) DFT(xi)
    for (int q = 0; q < nk && e == cudaSuccess; q++) {
      const int qc[3] = {q / (n2 * n3), (q / n3) % n2, q % n3};
      const std::vector<double> r0 = axis_reps(qc[0], n1), r1 = axis_reps(qc[1], n2), r2 = axis_reps(qc[2], n3);
      const double nrep = (double)(r0.size() * r1.size() * r2.size());
      const double w = sc * sc / (nrep * nk * vol);
      for (double x0 : r0)
        for (double x1 : r1)
          for (double x2 : r2) {
            if (!tc) {
              scale_xi<<<blocks((long)npts * nG), TB, 0, s>>>(F, ng, flatd, gmd, nG, rPd, npts, B, x0, x1, x2, w,
                                                              Xq);
              if ((e = gemm_z(A_MK, B_NK_CONJ, npts, npts, nG, Xq, nG, 0, Xq, nG, 0, W, npts, 0, 1, s)) !=
                  cudaSuccess)
                break;
              add_kernel<<<blocks(npq), TB, 0, s>>>(V + (long)q * npq, W, npq);
              continue;
            }
            // Xq Xq^H on tensor cores: A = Xq (FP32, sliced in the GEMM), B =
            // the embedded conj(Xq)^T, both with the exact row exponents of Xq
            scale_xi_f32<<<blocks((long)npts * nG), TB, 0, s>>>(F, ng, flatd, gmd, nG, rPd, npts, B, x0, x1, x2, w,
                                                                Xq32, ldq);
            if ((e = row_exponents_c(Xq32, 0, ldq, 1, npts, nG, eX, s)) != cudaSuccess) break;
            for (int g0 = 0; g0 < nG && e == cudaSuccess; g0 += slab) {
              const int gn = std::min(slab, nG - g0);
              TcOperand opA, opB;
              if ((e = make_f32_map(opA.map[0], Xq32 + g0, 1, npts, 2 * gn, 2 * ldq)) != cudaSuccess) break;
              for (int p = 0; p < 3 && e == cudaSuccess; p++)
                e = make_plane_map(opB.map[p], Bpl + p * plane, 1, 2 * npts, 2 * gn, ldb);
              if (e != cudaSuccess) break;
              if ((e = embed_b(Xq32 + g0, false, 0, 1, ldq, true, false, 1, gn, npts, eX, Bpl, plane, ldb, s)) !=
                  cudaSuccess)
                break;
              if ((e = tc_gemm(opA, opB, npts, 2 * npts, 2 * gn, 1, eX, npts, eX, npts, W, true, 2 * npts, 2 * npq,
                               ps0, pbc, tcerr, s, nullptr, 8, 1, 0)) != cudaSuccess)
                break;
              add_herm_kernel<<<blocks(npq), TB, 0, s>>>(V + (long)q * npq, W, npts);
            }
            if (e != cudaSuccess) break;
          }
    }
    if (e != cudaSuccess) break;
    mark(5);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    if (tcerr) {
      int h = 0;
      if ((e = cudaMemcpy(&h, tcerr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
      if (h) {
        st = THC_ERR_TIMEOUT;
        set_global_error("thc_rebuild_kernel: a device wait of the tensor-core contraction timed out");
        break;
      }
    }
    if (step_ms)
      for (int i = 0; i < 5; i++) {
        step_ms[i] = 0.f;
        if (ev[i] && ev[i + 1]) cudaEventElapsedTime(&step_ms[i], ev[i], ev[i + 1]);
      }
  } while (0);
  if (e != cudaSuccess) {
    set_global_error(std::string("thc_fit_kernel: ") + cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
  }
  void* ptrs[] = {Ugc, Bm, F, Xq, W, twd, R, S, L, rPd, ptsd, gmd, flatd, bad, Xq32, Bpl, eX, ps0, pbc, tcerr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  return st;
}

}  // namespace

extern "C" thc_status thc_fit_kernel(const double* U, int nfunc, const int* grid_host, const double* lattice_host,
                                     const int* mesh_host, const int* points_host, int npts, double* V_out,
                                     double* xi_out, void* stream) {
  return fit_impl(U, nfunc, grid_host, lattice_host, mesh_host, points_host, npts, V_out, xi_out, THC_FP64, nullptr,
                  stream);
}

extern "C" thc_status thc_rebuild_kernel(const double* U, int nfunc, const int* grid_host,
                                         const double* lattice_host, const int* mesh_host, const int* points_host,
                                         int npts, int precision, double* V_out, float* step_ms_host, void* stream) {
  return fit_impl(U, nfunc, grid_host, lattice_host, mesh_host, points_host, npts, V_out, nullptr, precision,
                  step_ms_host, stream);
}
