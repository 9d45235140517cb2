/*
 * thc.h -- C ABI of the GB300 THC-oo-K exact-exchange build.
 *
 * One build is the per-SCF-iteration exchange step of THC-oo-K
 * (Rettig, Lee, Head-Gordon, arXiv 2304.05505, Algorithm 2: the steps that
 * form X^k_PQ by FFT convolution and K_ij):
 *
 *   S1  Psi^k[P,i] = sum_mu X^k[mu,P] C^k[mu,i]        orbitals at the points
 *                                                      (u^k_i(r_P) of Eq. thcoccrik)
 *   S2  D^k[P,Q]   = sum_i Psi^k[P,i] conj(Psi^k[Q,i]) point-space density
 *   S3  M^k[P,Q]   = sum_k' D^k'[P,Q] V^(k'-k)[P,Q]     k-convolution (Sec. 2.2:
 *                                                      done as DFT over the mesh,
 *                                                      Hadamard product, inverse DFT)
 *   S4  (KC)^k     = conj(X^k) (M^k Psi^k)             K^k C^k, K^k = conj(X) M X^T
 *   S5  E_x        = -(1/N_k) sum_k sum_{P,i} conj(Psi^k[P,i]) (M^k Psi^k)[P,i]
 *                                                      (Eq. thcoccrik, closed shell,
 *                                                      per cell)
 *
 * Conventions.
 *  - Complex numbers are interleaved (re, im) doubles, i.e. C99 double _Complex
 *    / numpy complex128.  Arrays are dense and row-major with k slowest.
 *  - k and q share one index on the Gamma-centred n1 x n2 x n3 mesh:
 *    k = (a1 * n2 + a2) * n3 + a3 for k = sum_a (a_a / n_a) b_a.
 *    q = k' - k (Sec. 2.2) is wrapped onto the mesh.
 *  - X^k[mu,P] is the Bloch basis at the points with its Bloch phase,
 *    normalised per cell (no 1/sqrt(N_k)).  V^q[P,Q] is the ISDF Coulomb
 *    kernel M^q_PQ of Sec. 2.2 times exp(-i q.(r_P - r_Q)) and carries the
 *    1/N_k of the k sum.  The library only needs V^q Hermitian in (P,Q).
 *  - Pointers named *_host are host memory; every other pointer is device
 *    memory on the context's device.  Device pointers must be 16-byte aligned.
 *  - The caller owns every buffer it passes.  The library owns its context,
 *    its copies of X and of the prepared kernel, and its workspace; it never
 *    keeps a caller pointer past the call.
 *  - Device work is queued on the context's stream.  thc_build returns as
 *    soon as its work is queued; thc_build_host returns when the results
 *    are in host memory.
 *  - No call throws.  Every call returns a thc_status.  On THC_ERR_CUDA the
 *    CUDA error string is kept and thc_last_error() returns it.
 *  - Calls on one context are not thread-safe.  Contexts are independent.
 */
#ifndef THC_H
#define THC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  THC_OK = 0,
  THC_ERR_ARG = 1,         /* bad dimension, null or misaligned pointer, bad enum */
  THC_ERR_OOM = 2,         /* device allocation failed; nothing leaked */
  THC_ERR_CUDA = 3,        /* a CUDA call failed; see thc_last_error() */
  THC_ERR_NONFINITE = 4,   /* a NaN or Inf in an input checked by the call */
  THC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  THC_ERR_STATE = 6,       /* call order: build before set_collocation/set_kernel */
  THC_ERR_UNSUPPORTED = 7  /* valid request this build of the library cannot run */
} thc_status;

typedef enum {
  THC_FP64 = 0,            /* every step in FP64 on CUDA cores */
  THC_MIXED = 1,           /* S1, S2, S4a, S4b on tensor cores (tcgen05): each
                              operand row scaled by a power of two and cut into
                              three fixed-point slices of 8, 11 and 11 bits held
                              as fp16, the leading products summed exactly, 6 or 8
                              slice products per product; S3 in FP32; E_x summed
                              in FP64 */
  THC_MIXED_SIMT = 2,      /* the same precision on CUDA cores: FP32 operands,
                              float-float compensated sums in S1, S4a, S4b */
  THC_MIXED_EXT = 3        /* THC_MIXED with the extended k-convolution where it
                              applies (2^3 or 4^3 mesh, Hermitian V, nisdf a
                              multiple of 4): the DFTs run exactly on an 18-bit
                              split of each element's values, the product with
                              the prepared kernel keeps its roundings, and M
                              leaves as FP32 values plus fp16 remainders that S4a
                              slices with them (about 35 bits of M instead of
                              24); elsewhere it is THC_MIXED */
} thc_precision;

typedef struct {
  int n1, n2, n3;          /* k mesh, each >= 1 and <= 8 */
  int nbas;                /* N, basis functions, >= 1 */
  int nocc;                /* n, occupied orbitals, >= 1 */
  int nisdf;               /* N_P, interpolation points, >= 1 */
} thc_dims;

typedef struct thc_ctx thc_ctx;

/* Create a context on the current CUDA device.  `stream` is a cudaStream_t
 * (NULL = legacy default stream).  Allocates the context's device memory
 * (thc_memory_bytes tells how much) up front.  *ctx is NULL on failure. */
thc_status thc_create(thc_ctx** ctx, const thc_dims* dims, int precision, void* stream);

/* Device bytes the context holds (X copy, prepared kernel, workspace). */
thc_status thc_memory_bytes(const thc_dims* dims, int precision, size_t* bytes);

/* X: device, [N_k][nbas][nisdf] complex128.  Copied (and converted for
 * THC_MIXED) into the context; checked for NaN/Inf (THC_ERR_NONFINITE).
 * Synchronises the context's stream. */
thc_status thc_set_collocation(thc_ctx* ctx, const double* X);

/* V: device, [N_k][nisdf][nisdf] complex128, V[q] for q on the mesh index.
 * Prepares the DFT of V over the mesh, Vcheck[a] = (1/N_k) sum_q V[q] w^{+a.q}
 * (w = exp(2 pi i / n) per axis), in FP64, and keeps it (complex64 for
 * THC_MIXED).  Checked for NaN/Inf.  THC_MIXED also measures
 * max |V[q] - V[q]^H| against max |V|; within 1e-12 the builds take the
 * Hermitian form (thc_hermitian_kernel), else the general one.  Synchronises
 * the context's stream. */
thc_status thc_set_kernel(thc_ctx* ctx, const double* V);

/* One build.  C: device [N_k][nbas][nocc] complex128 (read only).
 * KC: device [N_k][nbas][nocc] complex128 (written; must not alias C).
 * ex: device, 2 doubles: ex[0] = E_x (Hartree per cell), ex[1] = the
 * imaginary part of the S5 sum (a residual, zero for Hermitian V).
 * Asynchronous on the context's stream.  In the tensor-core forms a build
 * that is not being profiled runs as one CUDA graph launch: its kernels are
 * captured from the stream on the first build with these (C, KC, ex)
 * pointers and replayed on later ones (the contents of C may change between
 * builds; new pointers, thc_set_collocation or thc_set_kernel capture anew;
 * a capture the driver refuses falls back to launching the kernels). */
thc_status thc_build(thc_ctx* ctx, const double* C, double* KC, double* ex);

/* The same build from and to host memory: copies C_host in, runs the build,
 * copies KC and E_x out, and waits for the stream.  Host buffers should be
 * pinned for full copy bandwidth (pageable memory works, more slowly).
 * ex_host: 2 doubles as in thc_build. */
thc_status thc_build_host(thc_ctx* ctx, const double* C_host, double* KC_host, double* ex_host);

/* The THC-AO-K form of the build (Algorithm 1 of the paper: its convolution
 * step forms X^k_PQ, and its K step the full AO exchange matrix):
 *   S1-S3 as thc_build, then K^k[mu,nu] = sum_PQ conj(X^k[mu,P]) M^k[P,Q] X^k[nu,Q]
 * (K^k = conj(X^k) M^k X^{kT}) and E_x = -(1/N_k) sum_k sum_PQ conj(D^k[P,Q]) M^k[P,Q]
 * (the energy of thc_build).  For THC-AO-K the points and V^q are those of
 * the fit of all basis-function products (thc_fit_kernel with U the
 * cell-periodic parts of the basis functions instead of the occupied
 * orbitals); the build takes any V.  C: device [N_k][nbas][nocc] complex128;
 * K: device [N_k][nbas][nbas] complex128 (written, must not overlap C); ex:
 * device, 2 doubles as in thc_build.  THC_FP64: every step in FP64 (the two
 * products on CUDA cores).  THC_MIXED: Z = M X^T and K = conj(X) Z on the
 * tensor cores (three fp16 slices, 8 slice products, exact leading sums; the
 * planes of X^T are made once per thc_set_collocation).  THC_MIXED_SIMT:
 * THC_ERR_UNSUPPORTED.  The first call on a context allocates the form's
 * extra workspace (THC_ERR_OOM if the device cannot hold it; the context
 * stays usable).  Asynchronous on the context's stream.  thc_profile_* and
 * thc_stage_times report its stages in the slots S1, S2, S3, then Z, K and
 * the energy in place of S4a, S4b and S5. */
thc_status thc_build_K(thc_ctx* ctx, const double* C, double* K, double* ex);

/* Intermediates of the last build, copied to device buffers the caller owns
 * (for tests).  which: 0 = Psi [N_k][nisdf][nocc], 1 = D [N_k][nisdf][nisdf],
 * 2 = M [N_k][nisdf][nisdf], 3 = Y = M Psi [N_k][nisdf][nocc].  Written as
 * complex128 whatever the precision (M with its remainders under
 * THC_MIXED_EXT).  which = 4 (THC_MIXED only): the row
 * exponents of M that S4a slices it with, [N_k][nisdf] doubles, each the
 * smallest e with max_Q max(|Re|, |Im|) of M^k[P][Q] < 2^e (0 for a zero
 * row; a row whose maximum is below 2^-133 may also get 0, which still bounds
 * it).  Synchronises the stream. */
thc_status thc_get_intermediate(thc_ctx* ctx, int which, double* out);

/* Per-stage device time of the last build in milliseconds (CUDA events on
 * the context's stream; 0 until a build ran).  stage_ms[0..5] = S1, S2, S3,
 * S4a, S4b, S5.  Synchronises the stream. */
thc_status thc_stage_times(thc_ctx* ctx, float stage_ms[6]);

/* Stage timing over many builds.  After thc_profile_begin(ctx, max_builds)
 * each thc_build records CUDA events around its stages on the context's
 * stream into a slot of its own, for up to max_builds builds (1..4096).
 * thc_profile_end waits for those events, writes the mean device time per
 * build of each stage in milliseconds (mean_ms[0..5] = S1, S2, S3, S4a, S4b,
 * S5) and the number of builds recorded, and stops recording. */
thc_status thc_profile_begin(thc_ctx* ctx, int max_builds);
thc_status thc_profile_end(thc_ctx* ctx, float mean_ms[6], int* nbuilds);

/* Mean device time (ms) of each stage's main kernel over the builds of the
 * last completed profile: the GEMM of S1, S2, S4a and S4b (without operand
 * preparation or the combine of split-K partials), the convolution of S3, the
 * reduction of S5 (its final sum when S4a's split-K combine formed the partial
 * sums, else both of its kernels).  In the FP64 and CUDA-core forms each stage is
 * one kernel and this equals the stage time.  THC_ERR_STATE before a profile
 * has completed. */
thc_status thc_profile_kernels(const thc_ctx* ctx, float core_ms[6]);

/* Wait for the context's stream.  Returns THC_ERR_TIMEOUT if a device-side
 * wait of a tensor-core kernel gave up since the last thc_sync (its outputs
 * are then invalid; the context stays usable), else THC_OK. */
thc_status thc_sync(thc_ctx* ctx);

/* Test hooks for failure detection (no GPU fault is involved in either).
 *
 * thc_debug_set_wait_limit: the limit, in SM clock cycles, of the bounded
 * device-side waits of the context's kernels (THC_MIXED; THC_ERR_UNSUPPORTED
 * for the forms without such waits).  cycles <= 0 restores the default (about
 * 2 s).  A limit of a few hundred cycles makes the waits of the next build
 * give up before their data arrives: each kernel then lets its copies and
 * MMAs in flight finish (with the default limit), stops, and thc_sync returns
 * THC_ERR_TIMEOUT; after the default is restored the context builds
 * correctly again.  Synchronises the context's stream.
 *
 * thc_debug_fail_alloc: the allocation with index nth (0-based, in the order
 * thc_create makes them) of the next thc_create on the calling thread fails
 * as if the device were out of memory, without calling the allocator; that
 * thc_create then returns THC_ERR_OOM having freed everything it allocated.
 * nth < 0 disables the hook. */
thc_status thc_debug_set_wait_limit(thc_ctx* ctx, long long cycles);
thc_status thc_debug_fail_alloc(int nth);

/* The FP64 fused multiply-add rate of the current device, measured: a kernel
 * of independent FMA chains on every SM, timed with CUDA events on `stream`
 * (a cudaStream_t) after one warm-up launch.  *tflops_host = FP64 TFLOP/s
 * (2 flops per FMA).  The FP64 build's stages are reported against it.
 * Synchronises the stream; changes no device setting. */
thc_status thc_measure_fp64_rate(void* stream, double* tflops_host);

/* Number of kernel launches one thc_build makes. */
thc_status thc_launches_per_build(const thc_ctx* ctx, int* launches);

/* *hermitian = 1 when the builds take the Hermitian form (THC_MIXED on a
 * 2^3, 3^3 or 4^3 mesh with even nisdf, and the V of the last thc_set_kernel
 * Hermitian for every q to 1e-12 of max |V|): then M^k is Hermitian, S2
 * writes D on and above the diagonal only and S3 reads that half of D and of
 * the prepared kernel; else 0.  THC_ERR_STATE before thc_set_kernel. */
thc_status thc_hermitian_kernel(const thc_ctx* ctx, int* hermitian);

thc_status thc_destroy(thc_ctx* ctx);

/* Interpolation points (setup, outside the timed build).  Greedy pivoted
 * Cholesky, in FP64, of the Gram matrix of occupied pair products
 *   A(r, r') = | sum_f conj(U[f][r]) U[f][r'] |^2
 * over candidate points r: the metric of the least-squares fit of Eq.
 * pbcinterpvec restricted to occupied orbitals (Eq. orbprodoo); in exact
 * arithmetic the points of the QR decomposition with column pivoting of
 * Sec. 2.1.  Each step takes the candidate with the largest residual diagonal
 * (the lowest index among equal ones).
 * U: device, [nfunc][ncand] complex128, U[f][r] = u^k_i(r_c) for f = (k, i)
 * (the cell-periodic parts of the occupied orbitals at the candidates).
 * Stops after npts points or when the residual trace falls to rel_tol times
 * trace(A).  points_host (host, npts ints) receives the candidate indices in
 * selection order, -1 past the end; npoints_host the number chosen.
 * resid_diag (device, ncand doubles, may be NULL) receives the residual
 * diagonal.  Allocates its own scratch (npts * ncand doubles) and waits for
 * `stream`. */
thc_status thc_select_points(const double* U, int nfunc, int ncand, int npts, double rel_tol,
                             int* points_host, int* npoints_host, double* resid_diag, void* stream);

/* The ISDF kernel of a set of interpolation points (setup, outside the timed
 * build), in FP64.  The interpolation vectors are the least-squares fit of
 * the occupied pair products (Eq. pbcinterpvec restricted to occupied
 * orbitals, Eq. orbprodoo): xi = S^-1 R with R[P][r] = |B[P][r]|^2,
 * B[P][r] = sum_f conj(U[f][r_P]) U[f][r] and S = R[:, points].  The kernel is
 * their Coulomb interaction in reciprocal space (Sec. 2.2), with the pair phase
 * folded in as thc_set_kernel expects:
 *   V^q[P,Q] = 1/(N_k Omega) exp(-i q.(r_P - r_Q)) sum_G v(G + q) xh_P(G) conj(xh_Q(G)),
 *   xh_P(G) = (Omega / N_g) sum_r xi_P(r) exp(-i G.r),  v(K) = 4 pi / |K|^2 (K = 0 left out),
 * G over the grid's frequencies without the Nyquist planes of even sizes, and
 * for a q on the zone boundary the mean over its minimum-image
 * representatives.
 * U: device, [nfunc][N_g] complex128, u^k_i(r) on the whole grid (f = (k, i);
 * grid index r = (i1 * g2 + i2) * g3 + i3 for fractional position
 * (i1/g1, i2/g2, i3/g3)).  grid_host[3] = (g1, g2, g3); lattice_host[9] the
 * cell vectors a1, a2, a3 as rows (bohr); mesh_host[3] the k-mesh (each 1..8).
 * points_host: npts distinct grid indices (host).  V_out: device,
 * [N_k][npts][npts] complex128 (q on the mesh index).  xi_out: device,
 * [npts][N_g] doubles, or NULL.  Allocates its own scratch (about
 * 40 npts N_g bytes) and waits for `stream`.  THC_ERR_ARG for bad sizes,
 * repeated or out-of-range points, or points whose metric S is numerically
 * singular (a Cholesky pivot below 1e-12 of its diagonal entry; message in
 * thc_last_error(NULL)). */
thc_status thc_fit_kernel(const double* U, int nfunc, const int* grid_host, const double* lattice_host,
                          const int* mesh_host, const int* points_host, int npts, double* V_out,
                          double* xi_out, void* stream);

/* The per-iteration kernel rebuild of THC-oo-K (Algorithm 2: the fit of the
 * interpolation vectors to the current orbitals, their FFT, and M^q as a sum
 * over G; Sec. 2.2).  Computes what thc_fit_kernel computes, with the same
 * arguments, conventions and errors (no xi output), and times its steps.
 * precision THC_FP64: every step in FP64 (the result equals thc_fit_kernel's
 * bit for bit).  THC_MIXED: the fit's metric, its Cholesky factor, the solve
 * and the FFT stay FP64; the contraction
 *   V^q[P,Q] = sum_G Xq[P][G] conj(Xq[Q][G]),  Xq = xh sqrt(v(G+q)) e^{-i q.r_P} (scaled),
 * which dominates the rebuild (N_k N_P^2 N_G complex multiply-adds), runs on
 * the tcgen05 tensor cores: Xq rounded to FP32 and cut into three fp16
 * slices inside the GEMM, 8 slice products, the leading products summed
 * exactly in chunks of at most 1024 real K and the chunks combined in FP64
 * (relative error of V about 1e-7 of its largest entries, from the FP32
 * rounding of Xq).  step_ms_host (host, 5 floats, may be NULL) receives the
 * device time of each step in ms: metric (B, R = |B|^2, S), Cholesky, solve,
 * FFT, contraction.  Allocates its own scratch and waits for `stream`;
 * THC_ERR_TIMEOUT if a device wait of the tensor-core contraction gave up. */
thc_status thc_rebuild_kernel(const double* U, int nfunc, const int* grid_host, const double* lattice_host,
                              const int* mesh_host, const int* points_host, int npts, int precision, double* V_out,
                              float* step_ms_host, void* stream);

/* The THC-oo-K orbital gradient: the vo block of the exchange matrix with the
 * kernel's response to the orbitals (Sec. 2.3, the K_ai expression; Algorithm
 * 2's dM/dtheta step), in FP64.  THC-oo-K fits the interpolation vectors to
 * the occupied pair products (Eq. orbprodoo), so V moves with the orbitals.
 * For the rotation C^k -> C^k + Cv^k theta^k (theta^k [n_vir][n_occ]) the
 * call returns
 *   g^k[a][i] = dE_x/dRe(theta^k[a][i]) + i dE_x/dIm(theta^k[a][i])   at theta = 0,
 * the points fixed and the fit (xi = S^-1 R, as thc_fit_kernel computes it)
 * and V redone along theta.  It is the sum of
 *   g_explicit^k = -(4/N_k) Psi_v^kH M^k Psi^k   (the kernel held fixed: the
 *     first term of K_ai; equal to -(4/N_k) Cv^kH (K C)^k with K C from thc_build),
 * and the kernel's response (the two W^q terms of K_ai): the derivative of
 *   E_x = -(1/N_k) sum_q sum_PQ W^q[P,Q] V^q[P,Q],  W^q = sum_k conj(D^k) o D^{k+q},
 * through V^q, xh, xi = S^-1 R, R = |B|^2 and B to the orbitals.
 * U: device, [N_k n_occ][N_g] complex128, the occupied orbitals' periodic
 * parts u^k_i(r) on the grid, row k n_occ + i, as for thc_fit_kernel.  Uv:
 * device, [N_k n_vir][N_g] complex128, the virtual orbitals' periodic parts,
 * row k n_vir + a.  psi = e^{i k.r} u with k = (n1/N1, n2/N2, n3/N3) in
 * reciprocal-lattice units (the mesh index order of thc_create).  grid_host,
 * lattice_host, mesh_host, points_host, npts: as for thc_fit_kernel.  V:
 * device, [N_k][npts][npts] complex128, the kernel fitted to U at these points
 * (thc_fit_kernel's or thc_rebuild_kernel's output); the response terms use
 * the fit recomputed here.  precision THC_FP64: every step in FP64 on CUDA
 * cores.  THC_MIXED: the (q, G) contraction of the response, the
 * O(N_k npts^2 N_G) step that dominates, runs on the tcgen05 tensor cores as
 * thc_rebuild_kernel's contraction does (W^q with its phases rounded to FP32
 * and sliced in the GEMM, v(G+q) conj(xh) cut into three fp16 slices with
 * exact exponents, 8 slice products, exact K chunks combined in FP64), and so
 * do the three grid contractions back to the orbitals (sum over r of the
 * adjoint of |B|^2 with U, over the points with conj(U) at them, and over r
 * of Uv with the result) when 2 N_g <= 126 * 1024; the fixed-kernel part, the
 * fit and the adjoint DFT and solve stay FP64 (g about 1e-7 to 1e-5 of
 * max|g| from the FP64 form, depending on the metric's conditioning).
 * g_out: device, [N_k][n_vir][n_occ] complex128.
 * g_explicit_out: the same shape, or NULL.  ex_host (host, may be NULL):
 * E_x from W and V.  step_ms_host (host, 5 floats, may be NULL): the device
 * ms of the fixed-kernel part, the fit, the (q, G) contraction, the adjoint
 * DFT with the solve, and the orbital contractions.  Outputs must not overlap
 * inputs.  Allocates its own scratch, at most about the largest of
 * 48 N_k npts^2, 16 npts (N_k npts + 7 N_g) and 16 N_k n_occ N_g + 32 npts N_g
 * bytes, and waits for `stream`.  THC_ERR_ARG for
 * bad sizes, null or misaligned pointers, repeated or out-of-range points, or
 * points whose metric S is numerically singular (as thc_fit_kernel);
 * THC_ERR_TIMEOUT if a device wait of the tensor-core contraction gave up. */
thc_status thc_vo_gradient(const double* U, int nocc, const double* Uv, int nvir, const int* grid_host,
                           const double* lattice_host, const int* mesh_host, const int* points_host, int npts,
                           const double* V, int precision, double* g_out, double* g_explicit_out, double* ex_host,
                           float* step_ms_host, void* stream);

/* Learned interpolation-point proposal (setup, outside the timed build).  The
 * paper has no learned part (its points come from a QR decomposition with
 * column pivoting, Sec. 2.1, or from k-means on the density, Sec. 4); these
 * calls add a small network that scores grid points so that the pivoted
 * Cholesky of thc_select_points_among only has to search a few candidates.
 *
 * Network: 3 -> 64 -> 64 -> 64 -> 1, SiLU, FP32, output a logit.  Parameters
 * (device, THC_MLP_NPARAM floats): W1 [64][3], b1 [64], W2 [64][64], b2 [64],
 * W3 [64][64], b3 [64], W4 [64], b4.  Features are standardised inside the
 * calls with norm_host = {mean[3], std[3]} (host, std > 0). */
#define THC_MLP_NPARAM 8641

/* Per-grid-point features (device, [N_g][3] floats): log(rho + 1e-8),
 * log(|grad rho| + 1e-8) and the minimum-image distance to the nearest of the
 * ncent centres (host, [ncent][3] Cartesian bohr), with
 * rho(r) = (1/nk) sum_f |U[f][r]|^2 (U as for thc_fit_kernel) and the gradient
 * from periodic second-order central differences (each grid size >= 3).
 * Waits for `stream`. */
thc_status thc_mlp_features(const double* U, int nfunc, int nk, const int* grid_host, const double* lattice_host,
                            const double* centres_host, int ncent, float* feat, void* stream);

/* score[p] = network logit of feat[p] (device, n points).  Queued on `stream`. */
thc_status thc_mlp_score(const float* params, const float* norm_host, const float* feat, int n, float* score,
                         void* stream);

/* Device workspace one thc_mlp_train_step over n points needs. */
thc_status thc_mlp_workspace_bytes(int n, size_t* bytes);

/* One training step over n points (labels: device floats, 1 for a point the
 * full-grid pivoted Cholesky picks, else 0): the mean of the weighted binary
 * cross-entropy with logits, pos_weight y softplus(-z) + (1 - y) softplus(z);
 * its gradient by backpropagation (summed over fixed point chunks, in a fixed
 * order, so repeated calls give identical results); then the Adam update
 * (beta 0.9, 0.999, eps 1e-8, bias-corrected for step t >= 1) of params,
 * adam_m and adam_v (device, THC_MLP_NPARAM floats each) with rate lr.
 * lr = 0 computes the gradient only.  loss_out (device float) and grad_out
 * (device, THC_MLP_NPARAM floats) may be NULL.  Queued on `stream`. */
thc_status thc_mlp_train_step(float* params, float* adam_m, float* adam_v, int t, float lr, const float* norm_host,
                              const float* feat, const float* labels, int n, float pos_weight, void* workspace,
                              size_t ws_bytes, float* loss_out, float* grad_out, void* stream);

/* The k highest of n scores (device), the lower index first among equal
 * scores; cand_host (host, k ints) receives their indices in ascending order.
 * Waits for `stream`. */
thc_status thc_mlp_candidates(const float* score, int n, int k, int* cand_host, void* stream);

/* thc_select_points restricted to the candidate columns cand_host[0..ncand)
 * (host, indices into the ng columns of U, ascending for the lowest-index
 * tie rule); points_host receives grid indices. */
thc_status thc_select_points_among(const double* U, int nfunc, int ng, const int* cand_host, int ncand, int npts,
                                   double rel_tol, int* points_host, int* npoints_host, void* stream);

/* The k-mesh convolution alone, M^k[P,Q] = sum_k' D^k'[P,Q] V^(k'-k)[P,Q] in
 * FP64, for callers that cannot allocate device memory when they call: for
 * example a host framework that has already reserved the device's memory in
 * its own pool, or a caller that must not let cudaMalloc/cudaFree synchronise
 * the device.  The paper has no counterpart; this is a deployment variant of
 * step S3.
 *
 * D, V, M: device, [N_k][npq] complex128 (npq = elements per k, e.g. N_P^2),
 * V indexed by q on the mesh index; M must not alias D or V.  Work is queued
 * on `stream` (a cudaStream_t; NULL = legacy default stream).  It allocates
 * nothing: its scratch (the DFT of V over the mesh) is one static device array
 * of 2,097,152 complex128 elements (32 MiB) that every GPU loading the library
 * holds until the process exits, so N_k * npq must be at most 2,097,152
 * (THC_ERR_ARG otherwise, message in thc_last_error(NULL)).  The first call on
 * each device looks up that array's device address, so make it before any
 * stream capture.  All calls on a device share the array: calls that overlap
 * on the GPU race and must be ordered by the caller. */
thc_status thc_kconv_noalloc(const double* D, const double* V, double* M, int n1, int n2, int n3,
                             long npq, void* stream);

const char* thc_status_string(thc_status s);
const char* thc_last_error(const thc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* THC_H */
