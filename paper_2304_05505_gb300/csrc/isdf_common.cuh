// Pieces shared by the ISDF fit (isdf_fit.cu) and the adjoint of the fit in
// the orbital gradient (vo_grad.cu): the FP64 kernels of the fit's steps 1-3
// and the host-side geometry of a (grid, lattice, k mesh, points) problem.
#pragma once

#include "thc_internal.cuh"

#include <math.h>

#include <vector>

namespace {

constexpr int TB = 256;

unsigned blocks(long n) { return (unsigned)((n + TB - 1) / TB); }

// Ugc[P][f] = conj(U[f][pts[P]])
__global__ void gather_conj(const double2* __restrict__ U, int nf, long ng, const int* __restrict__ pts, int np,
                            double2* __restrict__ Ugc) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * nf) return;
  const int P = (int)(i / nf), f = (int)(i % nf);
  const double2 u = U[(long)f * ng + pts[P]];
  Ugc[i] = make_double2(u.x, -u.y);
}

// R[i] = |B[i]|^2
__global__ void abs2_kernel(const double2* __restrict__ B, long n, double* __restrict__ R) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= n) return;
  const double2 b = B[i];
  R[i] = b.x * b.x + b.y * b.y;
}

// S[P][Q] = R[P][pts[Q]]
__global__ void gather_cols(const double* __restrict__ R, long ng, const int* __restrict__ pts, int np,
                            double* __restrict__ S) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= (long)np * np) return;
  const int P = (int)(i / np), Q = (int)(i % np);
  S[i] = R[(long)P * ng + pts[Q]];
}

// Column j of the Cholesky factor L (row-major, lower), left-looking: every
// thread recomputes the pivot d_j = S_jj - sum_t L_jt^2 and forms its L_ij.
// A pivot below 1e-12 S_jj marks the metric numerically singular.
__global__ void chol_column(const double* __restrict__ S, double* __restrict__ L, int n, int j, int* bad) {
  const int i = j + (int)((long)blockIdx.x * TB + threadIdx.x);
  if (i >= n) return;
  double d = S[(long)j * n + j];
  const double sjj = d;
  for (int t = 0; t < j; t++) d -= L[(long)j * n + t] * L[(long)j * n + t];
  if (!(d > 1e-12 * sjj)) {
    if (i == j) atomicOr(bad, 1);
    return;
  }
  const double ljj = sqrt(d);
  if (i == j) {
    L[(long)j * n + j] = ljj;
    return;
  }
  double a = S[(long)i * n + j];
  for (int t = 0; t < j; t++) a -= L[(long)i * n + t] * L[(long)j * n + t];
  L[(long)i * n + j] = a / ljj;
}

// X = L^-T L^-1 X for every column r of X[n][ng], in place.
__global__ void chol_solve(const double* __restrict__ L, double* __restrict__ X, int n, long ng) {
  const long r = (long)blockIdx.x * TB + threadIdx.x;
  if (r >= ng) return;
  for (int j = 0; j < n; j++) {
    double a = X[(long)j * ng + r];
    for (int t = 0; t < j; t++) a -= L[(long)j * n + t] * X[(long)t * ng + r];
    X[(long)j * ng + r] = a / L[(long)j * n + j];
  }
  for (int j = n - 1; j >= 0; j--) {
    double a = X[(long)j * ng + r];
    for (int t = j + 1; t < n; t++) a -= L[(long)t * n + j] * X[(long)t * ng + r];
    X[(long)j * ng + r] = a / L[(long)j * n + j];
  }
}

// One axis of the forward DFT of [np][g1][g2][g3]: out = sum_j in(j) tw[(j m) mod g].
// `real_in` reads a real array (the vectors themselves) for the first axis.
__global__ void dft_axis_kernel(const void* __restrict__ in, bool real_in, double2* __restrict__ out, long total,
                                int g, long st, const double2* __restrict__ tw) {
  const long i = (long)blockIdx.x * TB + threadIdx.x;
  if (i >= total) return;
  const int m = (int)((i / st) % g);
  const long base = i - (long)m * st;
  double re = 0.0, im = 0.0;
  for (int j = 0, jm = 0; j < g; j++, jm = (jm + m) % g) {
    const double2 w = tw[jm];
    if (real_in) {
      const double x = ((const double*)in)[base + (long)j * st];
      re += x * w.x;
      im += x * w.y;
    } else {
      const double2 x = ((const double2*)in)[base + (long)j * st];
      re += x.x * w.x - x.y * w.y;
      im += x.x * w.y + x.y * w.x;
    }
  }
  out[i] = make_double2(re, im);
}

// Minimum-image fractional representatives of q = qco / mesh along one axis.
std::vector<double> axis_reps(int qc, int n) {
  const double f = (double)(((qc % n) + n) % n) / n;
  if (fabs(f - 0.5) < 1e-12) return {0.5, -0.5};
  if (f > 0.5) return {f - 1.0};
  return {f};
}


// Reciprocal rows b_i with a_i . b_j = 2 pi delta_ij.
struct Recip {
  double b[9];   // rows b1, b2, b3
};

// The geometry of one fit: grid and mesh sizes, cell volume, reciprocal rows,
// the G set without Nyquist planes (integer coordinates and the flat grid
// index of each), the Cartesian point positions, and the per-axis twiddles
// e^{-2 pi i t / g} (axis a's at tw[off[a]]).
struct FitGeom {
  int g[3], n[3];
  long ng;
  int nk;
  double vol;
  Recip B;
  std::vector<int> gm, flat;
  std::vector<double> rP;
  std::vector<double2> tw;
  int off[3];
};

// Checks the arguments a fit shares (grid sizes >= 1, mesh sizes in 1..8,
// 1 <= npts <= N_g distinct grid indices, a cell of positive volume) and fills
// `geo`; false on a bad one.
inline bool fit_geometry(const int* grid_host, const double* lattice_host, const int* mesh_host,
                         const int* points_host, int npts, FitGeom& geo) {
  const int g1 = grid_host[0], g2 = grid_host[1], g3 = grid_host[2];
  const int n1 = mesh_host[0], n2 = mesh_host[1], n3 = mesh_host[2];
  if (g1 < 1 || g2 < 1 || g3 < 1 || n1 < 1 || n2 < 1 || n3 < 1 || n1 > 8 || n2 > 8 || n3 > 8) return false;
  const long ng = (long)g1 * g2 * g3;
  if (npts < 1 || npts > ng) return false;
  std::vector<char> seen(ng, 0);
  for (int P = 0; P < npts; P++) {
    const int p = points_host[P];
    if (p < 0 || p >= ng || seen[p]) return false;   // points must be distinct grid indices
    seen[p] = 1;
  }
  const double* a = lattice_host;
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  const double vol = fabs(det);
  if (!(vol > 0)) return false;
  geo.g[0] = g1, geo.g[1] = g2, geo.g[2] = g3;
  geo.n[0] = n1, geo.n[1] = n2, geo.n[2] = n3;
  geo.ng = ng;
  geo.nk = n1 * n2 * n3;
  geo.vol = vol;
  {
    const double c = 2.0 * M_PI / det;
    const double* a1 = a;
    const double* a2 = a + 3;
    const double* a3 = a + 6;
    auto cross = [](const double* x, const double* y, double* o) {
      o[0] = x[1] * y[2] - x[2] * y[1];
      o[1] = x[2] * y[0] - x[0] * y[2];
      o[2] = x[0] * y[1] - x[1] * y[0];
    };
    cross(a2, a3, geo.B.b);
    cross(a3, a1, geo.B.b + 3);
    cross(a1, a2, geo.B.b + 6);
    for (double& x : geo.B.b) x *= c;
  }
  const int h1 = (g1 - 1) / 2, h2 = (g2 - 1) / 2, h3 = (g3 - 1) / 2;
  geo.gm.clear();
  geo.flat.clear();
  for (int i = -h1; i <= h1; i++)
    for (int j = -h2; j <= h2; j++)
      for (int l = -h3; l <= h3; l++) {
        geo.gm.push_back(i);
        geo.gm.push_back(j);
        geo.gm.push_back(l);
        geo.flat.push_back((((i % g1) + g1) % g1 * g2 + ((j % g2) + g2) % g2) * g3 + ((l % g3) + g3) % g3);
      }
  geo.rP.assign(3 * (size_t)npts, 0.0);
  for (int P = 0; P < npts; P++) {
    const int p = points_host[P];
    const double f0 = (double)(p / (g2 * g3)) / g1, f1 = (double)((p / g3) % g2) / g2, f2 = (double)(p % g3) / g3;
    for (int x = 0; x < 3; x++) geo.rP[3 * P + x] = f0 * a[x] + f1 * a[3 + x] + f2 * a[6 + x];
  }
  geo.tw.assign(g1 + g2 + g3, make_double2(0.0, 0.0));
  geo.off[0] = 0, geo.off[1] = g1, geo.off[2] = g1 + g2;
  const int gs[3] = {g1, g2, g3};
  for (int ax = 0; ax < 3; ax++)
    for (int t = 0; t < gs[ax]; t++) {
      const double ang = -2.0 * M_PI * t / gs[ax];
      geo.tw[geo.off[ax] + t] = make_double2(cos(ang), sin(ang));
    }
  return true;
}

}  // namespace
