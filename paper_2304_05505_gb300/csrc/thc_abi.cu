// C ABI of the THC-oo-K exchange build (declared in include/thc.h).
//
// Owns the context: the copy of the collocation X, the prepared kernel
// Vh = DFT_q(V)/N_k, and the workspace for Psi, D, M and Y.  thc_build queues
// the five steps of the build on the context's stream:
//   S1  Psi = X^T C            gemm   (A = X transposed, B = C)
//   S2  D   = Psi Psi^H        gemm   (B = Psi conjugate-transposed)
//   S3  M   = IDFT(DFT(D) o Vh) kconv
//   S4a Y   = M Psi            gemm
//   S4b KC  = conj(X) Y        gemm   (A = X conjugated)
//   S5  E_x = -(1/N_k) <Psi, Y> ex_reduce
#include "thc_internal.cuh"

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

namespace {

thread_local std::string g_create_error;
thread_local int g_fail_alloc = -1;   // test hook: index of the next thc_create allocation to fail

#define CKC(ctx, call)                                                       \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return THC_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// The tensor-core forms: THC_MIXED and THC_MIXED_EXT.
bool tc_form(int precision) { return precision == THC_MIXED || precision == THC_MIXED_EXT; }

// THC_MIXED_EXT's extended k-convolution applies (its remainders of M are
// kept): a 2^3 or 4^3 mesh, the Hermitian form's keys, N_P a multiple of 4
// (16-byte strided fp16 rows of the remainders).
bool ext_form(const thc_dims* d, int precision) {
  return precision == THC_MIXED_EXT && d->n1 == d->n2 && d->n2 == d->n3 && (d->n1 == 2 || d->n1 == 4) &&
         d->nisdf % 4 == 0 && kconv_herm_key_words(d->nisdf, d->n1, d->n2, d->n3) > 0;
}

struct Sizes {
  long nk, x, v, psi, kc;
  size_t el;  // bytes of a workspace complex element
  // tensor-core operands: FP32 X with even leading dimension, planes (elements of one plane)
  int ldX;
  long x32;
  int ldC, ldM, ldPs;
  long plPs, plBc, plBd, plBy, plM;
  long nexp;  // exponents: eXn + eXT + ePsi + eC + eY + eM
  long npart; // split-K partial elements (max over the tensor-core GEMMs)
  long hkey;  // key words of the Hermitian convolution (0 where it does not apply)
  long mlo;   // fp16 remainder pairs of M (THC_MIXED_EXT where its convolution applies)
};

int pad8(int x) { return (x + 7) & ~7; }

Sizes sizes_of(const thc_dims* d, int precision) {
  Sizes s;
  s.nk = (long)d->n1 * d->n2 * d->n3;
  s.x = s.nk * d->nbas * d->nisdf;
  s.v = s.nk * d->nisdf * d->nisdf;
  s.psi = s.nk * d->nisdf * d->nocc;
  s.kc = s.nk * d->nbas * d->nocc;
  s.el = precision == THC_FP64 ? sizeof(double2) : sizeof(float2);
  s.ldX = d->nisdf + (d->nisdf & 1);
  s.x32 = s.nk * d->nbas * (long)s.ldX;
  s.ldC = pad8(2 * d->nbas);
  s.ldM = pad8(2 * d->nisdf);
  s.ldPs = pad8(2 * d->nocc);
  s.plPs = s.nk * d->nisdf * s.ldPs;
  s.plBc = s.nk * 2 * d->nocc * s.ldC;
  s.plBd = s.nk * 2L * d->nisdf * s.ldPs;
  s.plBy = s.nk * 2 * d->nocc * (long)s.ldM;
  s.plM = (d->nisdf % 2) ? s.nk * d->nisdf * (long)s.ldM : 0;   // M's slices only for odd N_P
  s.nexp = s.nk * (d->nbas + 3L * d->nisdf + 2L * d->nocc);
  s.npart = std::max({tc_partial_elems(d->nisdf, 2 * d->nocc, 2 * d->nbas, (int)s.nk),
                      tc_partial_elems(d->nisdf, 2 * d->nisdf, 2 * d->nocc, (int)s.nk),
                      tc_partial_elems(d->nisdf, 2 * d->nocc, 2 * d->nisdf, (int)s.nk),
                      tc_partial_elems(d->nbas, 2 * d->nocc, 2 * d->nisdf, (int)s.nk)});
  s.hkey = tc_form(precision) ? kconv_herm_key_words(d->nisdf, d->n1, d->n2, d->n3) : 0;
  s.mlo = ext_form(d, precision) ? s.v : 0;
  return s;
}

constexpr int kPartials = 1216;  // 152 SMs x 8 blocks

thc_status check_dims(const thc_dims* d, int precision) {
  if (!d) return THC_ERR_ARG;
  if (d->n1 < 1 || d->n2 < 1 || d->n3 < 1 || d->n1 > 8 || d->n2 > 8 || d->n3 > 8) return THC_ERR_ARG;
  if (d->nbas < 1 || d->nocc < 1 || d->nisdf < 1) return THC_ERR_ARG;
  if (d->nocc > d->nbas) return THC_ERR_ARG;
  if (precision != THC_FP64 && !tc_form(precision) && precision != THC_MIXED_SIMT) return THC_ERR_ARG;
  // element counts must fit the kernels' index arithmetic
  const double v = (double)d->n1 * d->n2 * d->n3 * d->nisdf * (double)d->nisdf;
  if (v > 4.0e10) return THC_ERR_UNSUPPORTED;
  if ((double)d->nisdf * d->nisdf > 2.0e9) return THC_ERR_UNSUPPORTED;
  return THC_OK;
}

size_t memory_bytes(const thc_dims* d, int precision) {
  Sizes s = sizes_of(d, precision);
  size_t b = 0;
  b += s.v * s.el;               // prepared kernel
  b += 2 * s.psi * s.el;         // Psi, Y
  b += 2 * s.v * s.el;           // D, M
  if (tc_form(precision)) {
    b += sizeof(uint32_t) * s.mlo;                                           // remainders of M (THC_MIXED_EXT)
    b += s.x32 * sizeof(float2);                                             // X in FP32
    b += 3 * 2 * (s.plPs + s.plBc + s.plBd + s.plBy + s.plM);               // fp16 slices
    b += sizeof(int) * s.nexp + 64;                                         // exponents, error word
    b += (sizeof(int) + sizeof(float)) * s.npart;                           // split-K partial sums
    b += sizeof(uint32_t) * s.hkey;                                          // Hermitian convolution keys
  } else {
    b += s.x * s.el;             // X copy
  }
  b += 2 * s.kc * sizeof(double2) + 2 * sizeof(double);  // host-build staging
  b += 2 * kPartials * sizeof(double) + 64 + 64;
  return b;
}

void free_all(thc_ctx* c) {
  void* ptrs[] = {c->X64, c->Vh64, c->X32, c->Vh32, c->Psi, c->D, c->M, c->Y,
                  c->Cdev, c->KCdev, c->exdev, c->partial, c->flag,
                  c->PsiA_pl, c->Bc_pl, c->Bd_pl, c->By_pl, c->ex_pl, c->tc_err, c->part_s0,
                  c->part_bc, c->M_pl, c->hkeys, c->Zao, c->Wao, c->BxT_pl, c->Bz_pl, c->eZ, c->ps0_ao,
                  c->pbc_ao, c->Mlo};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < 7; i++)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (cudaEvent_t e : c->prof) cudaEventDestroy(e);
  c->prof.clear();
  if (c->tc_err_host) cudaFreeHost(c->tc_err_host);
  c->tc_err_host = nullptr;
  for (cudaEvent_t& e : c->cev)
    if (e) cudaEventDestroy(e), e = nullptr;
  if (c->cstream) cudaStreamDestroy(c->cstream);
  c->cstream = nullptr;
}

constexpr int kStages = 6;

}  // namespace

void set_global_error(const std::string& msg) { g_create_error = msg; }

extern "C" {

const char* thc_status_string(thc_status s) {
  switch (s) {
    case THC_OK: return "ok";
    case THC_ERR_ARG: return "invalid argument";
    case THC_ERR_OOM: return "device out of memory";
    case THC_ERR_CUDA: return "CUDA error";
    case THC_ERR_NONFINITE: return "non-finite input";
    case THC_ERR_TIMEOUT: return "device wait timed out";
    case THC_ERR_STATE: return "call out of order";
    case THC_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

const char* thc_last_error(const thc_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->last_error.c_str();
}

thc_status thc_memory_bytes(const thc_dims* dims, int precision, size_t* bytes) {
  thc_status st = check_dims(dims, precision);
  if (st != THC_OK) return st;
  if (!bytes) return THC_ERR_ARG;
  *bytes = memory_bytes(dims, precision);
  return THC_OK;
}

thc_status thc_create(thc_ctx** out, const thc_dims* d, int precision, void* stream) {
  if (!out) return THC_ERR_ARG;
  *out = nullptr;
  thc_status st = check_dims(d, precision);
  if (st != THC_OK) return st;
  thc_ctx* c = new (std::nothrow) thc_ctx();
  if (!c) return THC_ERR_OOM;
  c->n1 = d->n1; c->n2 = d->n2; c->n3 = d->n3;
  c->nk = d->n1 * d->n2 * d->n3;
  c->nbas = d->nbas; c->nocc = d->nocc; c->nisdf = d->nisdf;
  c->precision = precision;
  c->stream = (cudaStream_t)stream;
  c->n_partial = kPartials;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    delete c;
    return THC_ERR_CUDA;
  }
  Sizes s = sizes_of(d, precision);
  struct Want { void** p; size_t bytes; };
  Want want[32];
  int nw = 0;
  auto W = [&](void** p, size_t bytes) { want[nw++] = Want{p, bytes}; };
  if (precision == THC_FP64) {
    W((void**)&c->X64, s.x * s.el);
    W((void**)&c->Vh64, s.v * s.el);
    W(&c->M, s.v * s.el);
  } else if (precision == THC_MIXED_SIMT) {
    W((void**)&c->X32, s.x * s.el);
    W((void**)&c->Vh32, s.v * s.el);
    W(&c->M, s.v * s.el);
  } else {
    W((void**)&c->Vh32, s.v * s.el);
    W(&c->M, s.v * s.el);
    if (s.mlo) W((void**)&c->Mlo, sizeof(uint32_t) * s.mlo);
    W((void**)&c->X32, s.x32 * sizeof(float2));
    if (s.plM) W((void**)&c->M_pl, 3 * 2 * s.plM);
    W((void**)&c->PsiA_pl, 3 * 2 * s.plPs);
    W((void**)&c->Bc_pl, 3 * 2 * s.plBc);
    W((void**)&c->Bd_pl, 3 * 2 * s.plBd);
    W((void**)&c->By_pl, 3 * 2 * s.plBy);
    W((void**)&c->ex_pl, sizeof(int) * s.nexp);
    W((void**)&c->tc_err, 64);
    if (s.npart > 0) {
      W((void**)&c->part_s0, sizeof(int) * s.npart);
      W((void**)&c->part_bc, sizeof(float) * s.npart);
    }
    if (s.hkey > 0) W((void**)&c->hkeys, sizeof(uint32_t) * s.hkey);
  }
  W(&c->Psi, s.psi * s.el);
  W(&c->Y, s.psi * s.el);
  W(&c->D, s.v * s.el);
  W((void**)&c->Cdev, s.kc * sizeof(double2));
  W((void**)&c->KCdev, s.kc * sizeof(double2));
  W((void**)&c->exdev, 2 * sizeof(double));
  W((void**)&c->partial, 2 * kPartials * sizeof(double));
  W((void**)&c->flag, 64);
  const int fail_at = g_fail_alloc;
  g_fail_alloc = -1;
  for (int i = 0; i < nw; i++) {
    Want& w = want[i];
    e = i == fail_at ? cudaErrorMemoryAllocation : cudaMalloc(w.p, w.bytes);
    if (e == cudaSuccess) e = cudaMemset(*w.p, 0, w.bytes);   // plane padding stays zero
    if (e != cudaSuccess) {
      if (*w.p) cudaFree(*w.p);
      *w.p = nullptr;
      cudaGetLastError();
      g_create_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      free_all(c);
      delete c;
      return e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
    }
  }
  if (tc_form(precision)) {
    c->ldX = s.ldX; c->ldC = s.ldC; c->ldM = s.ldM; c->ldPs = s.ldPs;
    c->plPs = s.plPs;
    c->plBc = s.plBc; c->plBd = s.plBd; c->plBy = s.plBy; c->plM = s.plM;
    const int nk = (int)s.nk, N = d->nbas, n = d->nocc, P = d->nisdf;
    c->eXn = c->ex_pl;
    c->eXT = c->eXn + (long)nk * N;
    c->ePsi = c->eXT + (long)nk * P;
    c->eC = c->ePsi + (long)nk * P;
    c->eY = c->eC + (long)nk * n;
    c->eM = c->eY + (long)nk * n;
    struct MapReq { TcOperand* op; uint16_t* base; long pl; int rows, cols, ld; };
    MapReq reqs[] = {
        {&c->opPs, c->PsiA_pl, s.plPs, P, 2 * n, s.ldPs},
        {&c->opBc, c->Bc_pl, s.plBc, 2 * n, 2 * N, s.ldC},
        {&c->opBd, c->Bd_pl, s.plBd, 2 * P, 2 * n, s.ldPs},
        {&c->opBy, c->By_pl, s.plBy, 2 * n, 2 * P, s.ldM},
    };
    // X in FP32: A of S1 read as the transpose [mu][P] -> rows P, and A of S4b (rows mu)
    e = make_f32_map_t(c->opXT.map[0], c->X32, nk, N, P, 2 * s.ldX);
    if (e == cudaSuccess) e = make_f32_map(c->opXn.map[0], c->X32, nk, N, 2 * P, 2 * s.ldX);
    for (auto& r : reqs)
      for (int p = 0; p < 3 && e == cudaSuccess; p++) {
        e = make_plane_map(r.op->map[p], r.base + p * r.pl, nk, r.rows, r.cols, r.ld);
        if (e != cudaSuccess) {
          g_create_error = std::string("cuTensorMapEncodeTiled: ") + cudaGetErrorString(e);
          free_all(c);
          delete c;
          return e == cudaErrorNotSupported ? THC_ERR_UNSUPPORTED : THC_ERR_CUDA;
        }
      }
    if (s.plM)
      for (int p = 0; p < 3 && e == cudaSuccess; p++)
        e = make_plane_map(c->opM.map[p], c->M_pl + p * s.plM, nk, P, 2 * P, s.ldM);
    else
      e = make_f32_map(c->opMf.map[0], c->M, nk, P, 2 * P, 2 * P);
    if (e == cudaSuccess && c->Mlo) e = make_plane_map(c->opMf.map[1], c->Mlo, nk, P, 2 * P, 2 * P);
    if (e == cudaSuccess && c->hkeys) {
      e = kconv_herm_prepare(c->hkeys, P, d->n1, d->n2, d->n3, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
      g_create_error = std::string("cuTensorMapEncodeTiled: ") + cudaGetErrorString(e);
      free_all(c);
      delete c;
      return e == cudaErrorNotSupported ? THC_ERR_UNSUPPORTED : THC_ERR_CUDA;
    }
  }
  e = cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking);
  for (int i = 0; i < 6 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&c->cev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    g_create_error = std::string("copy stream: ") + cudaGetErrorString(e);
    free_all(c);
    delete c;
    return THC_ERR_CUDA;
  }
  if (c->tc_err && (e = cudaMallocHost(&c->tc_err_host, sizeof(int))) != cudaSuccess) {
    g_create_error = std::string("cudaMallocHost: ") + cudaGetErrorString(e);
    free_all(c);
    delete c;
    return THC_ERR_OOM;
  }
  for (int i = 0; i < 7; i++) {
    e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
      g_create_error = std::string("cudaEventCreate: ") + cudaGetErrorString(e);
      free_all(c);
      delete c;
      return THC_ERR_CUDA;
    }
  }
  *out = c;
  return THC_OK;
}

// Drops the captured build (the inputs or the kernel form changed).
static void drop_graph(thc_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->g_C = c->g_KC = c->g_ex = nullptr;
  if (c->gexec_h) cudaGraphExecDestroy(c->gexec_h);
  c->gexec_h = nullptr;
  c->gh_C = c->gh_KC = nullptr;
}

thc_status thc_destroy(thc_ctx* c) {
  if (!c) return THC_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  drop_graph(c);
  free_all(c);
  delete c;
  return THC_OK;
}

static thc_status finite_check(thc_ctx* c, const double2* p, long n) {
  CKC(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
  CKC(c, check_finite_z(p, n, c->flag, c->stream));
  int h = 0;
  CKC(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return h ? THC_ERR_NONFINITE : THC_OK;
}

thc_status thc_set_collocation(thc_ctx* c, const double* X) {
  if (!c || !X || !aligned16(X)) return THC_ERR_ARG;
  const long n = (long)c->nk * c->nbas * c->nisdf;
  const double2* x = (const double2*)X;
  thc_status st = finite_check(c, x, n);
  if (st != THC_OK) return st;
  drop_graph(c);
  if (c->precision == THC_FP64) {
    CKC(c, cudaMemcpyAsync(c->X64, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  } else if (c->precision == THC_MIXED_SIMT) {
    CKC(c, convert_z2c(x, c->X32, n, c->stream));
  } else {
    // X in FP32 (rows padded to an even length), and the exponents that slice
    // it inside the GEMMs: per basis function (rows of A in S4b) and per point
    // (rows of A = X^T in S1), taken on the FP32 values
    CKC(c, convert_z2c_rows(x, c->X32, (long)c->nk * c->nbas, c->nisdf, c->ldX, c->stream));
    const long sb = (long)c->nbas * c->ldX;
    CKC(c, row_exponents_c(c->X32, sb, c->ldX, c->nk, c->nbas, c->nisdf, c->eXn, c->stream));
    CKC(c, col_exponents_c(c->X32, sb, c->ldX, c->nk, c->nbas, c->nisdf, c->eXT, c->stream));
  }
  CKC(c, cudaStreamSynchronize(c->stream));
  c->have_x = true;
  c->bxt_valid = false;   // the THC-AO-K planes of X^T follow the collocation
  return THC_OK;
}

thc_status thc_set_kernel(thc_ctx* c, const double* V) {
  if (!c || !V || !aligned16(V)) return THC_ERR_ARG;
  const long npq = (long)c->nisdf * c->nisdf;
  const double2* v = (const double2*)V;
  thc_status st = finite_check(c, v, npq * c->nk);
  if (st != THC_OK) return st;
  drop_graph(c);
  CKC(c, prepare_kernel_z(v, c->Vh64, c->Vh32, npq, c->n1, c->n2, c->n3, c->stream));
  c->herm_v = false;
  if (c->hkeys) {
    // every V^q Hermitian to 1e-12 of max |V|: then M^k is Hermitian and the
    // build convolves the part of D on and above the diagonal only
    unsigned long long* dv = reinterpret_cast<unsigned long long*>(c->partial);
    CKC(c, cudaMemsetAsync(dv, 0, 2 * sizeof(unsigned long long), c->stream));
    CKC(c, hermitian_deviation_z(v, c->nisdf, c->nk, dv, c->stream));
    unsigned long long h[2] = {0, 0};
    CKC(c, cudaMemcpyAsync(h, dv, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CKC(c, cudaStreamSynchronize(c->stream));
    double dev, mx;
    memcpy(&dev, &h[0], sizeof dev);
    memcpy(&mx, &h[1], sizeof mx);
    c->herm_v = dev <= 1e-12 * mx;
  }
  CKC(c, cudaStreamSynchronize(c->stream));
  c->have_v = true;
  return THC_OK;
}

constexpr int kProfEv = 7 + 12;

static bool profiling(const thc_ctx* c) { return c->prof_max > 0 && c->prof_n < c->prof_max; }

// Event marking the start of stage i (i = 6: end of the build).
static cudaEvent_t stage_event(thc_ctx* c, int i) {
  if (profiling(c)) return c->prof[(size_t)c->prof_n * kProfEv + i];
  return c->ev[i];
}

// Start (which = 0) or end (1) of stage st's main kernel; null unless profiling.
static cudaEvent_t core_event(thc_ctx* c, int st, int which) {
  if (!profiling(c)) return nullptr;
  return c->prof[(size_t)c->prof_n * kProfEv + 7 + 2 * st + which];
}

static cudaError_t record_core(thc_ctx* c, int st, int which, cudaStream_t s) {
  cudaEvent_t e = core_event(c, st, which);
  return e ? cudaEventRecord(e, s) : cudaSuccess;
}

// Stage boundary i.  In the one-kernel-per-stage forms (simple) the stage's
// main kernel is the whole stage, so its core events sit on the boundaries.
static cudaError_t mark(thc_ctx* c, int i, cudaStream_t s, bool simple) {
  cudaError_t e = cudaSuccess;
  if (simple && i > 0) e = record_core(c, i - 1, 1, s);
  if (e == cudaSuccess) e = cudaEventRecord(stage_event(c, i), s);
  if (e == cudaSuccess && simple && i < 6) e = record_core(c, i, 0, s);
  return e;
}

// Kao (THC-AO-K): after S3, K^k = conj(X^k) M^k X^{kT} into Kao instead of S4a,
// S4b, and E_x = -(1/N_k) sum_k sum_PQ conj(D^k_PQ) M^k_PQ (the same energy).
static thc_status build_fp64(thc_ctx* c, const double2* C, double2* KC, double* ex, double2* Kao = nullptr) {
  const int nk = c->nk, N = c->nbas, n = c->nocc, P = c->nisdf;
  const long PP = (long)P * P;
  double2* Psi = (double2*)c->Psi;
  double2* D = (double2*)c->D;
  double2* M = (double2*)c->M;
  double2* Y = (double2*)c->Y;
  cudaStream_t s = c->stream;
  CKC(c, mark(c, 0, s, true));
  CKC(c, gemm_z(A_KM, B_KN, P, n, N, c->X64, P, (long)N * P, C, n, (long)N * n, Psi, n,
                (long)P * n, nk, s));
  CKC(c, mark(c, 1, s, true));
  CKC(c, gemm_z(A_MK, B_NK_CONJ, P, P, n, Psi, n, (long)P * n, Psi, n, (long)P * n, D, P, PP,
                nk, s));
  CKC(c, mark(c, 2, s, true));
  CKC(c, kconv_z(D, c->Vh64, M, PP, c->n1, c->n2, c->n3, s));
  CKC(c, mark(c, 3, s, true));
  if (Kao) {
    CKC(c, gemm_z(A_MK_CONJ, B_KN, N, P, P, c->X64, P, (long)N * P, M, P, PP, c->Wao, P, (long)N * P, nk, s));
    CKC(c, mark(c, 4, s, true));
    CKC(c, gemm_z(A_MK, B_NK, N, N, P, c->Wao, P, (long)N * P, c->X64, P, (long)N * P, Kao, N, (long)N * N, nk, s));
    CKC(c, mark(c, 5, s, true));
    CKC(c, ex_reduce_z(D, M, (long)nk * PP, nk, c->partial, c->n_partial, ex, s));
    CKC(c, mark(c, 6, s, true));
    return THC_OK;
  }
  CKC(c, gemm_z(A_MK, B_KN, P, n, P, M, P, PP, Psi, n, (long)P * n, Y, n, (long)P * n, nk, s));
  CKC(c, mark(c, 4, s, true));
  CKC(c, gemm_z(A_MK_CONJ, B_KN, N, n, P, c->X64, P, (long)N * P, Y, n, (long)P * n, KC, n,
                (long)N * n, nk, s));
  CKC(c, mark(c, 5, s, true));
  CKC(c, ex_reduce_z(Psi, Y, (long)nk * P * n, nk, c->partial, c->n_partial, ex, s));
  CKC(c, mark(c, 6, s, true));
  return THC_OK;
}

static thc_status build_mixed(thc_ctx* c, const double2* C, double2* KC, double* ex) {
  const int nk = c->nk, N = c->nbas, n = c->nocc, P = c->nisdf;
  const long PP = (long)P * P;
  float2* Psi = (float2*)c->Psi;
  float2* D = (float2*)c->D;
  float2* M = (float2*)c->M;
  float2* Y = (float2*)c->Y;
  cudaStream_t s = c->stream;
  CKC(c, mark(c, 0, s, true));
  CKC(c, (gemm_c_comp<float2, double2, float2>(A_KM, B_KN, P, n, N, c->X32, P, (long)N * P, C, n,
                                               (long)N * n, Psi, n, (long)P * n, nk, s)));
  CKC(c, mark(c, 1, s, true));
  CKC(c, gemm_c_plain(A_MK, B_NK_CONJ, P, P, n, Psi, n, (long)P * n, Psi, n, (long)P * n, D, P,
                      PP, nk, s));
  CKC(c, mark(c, 2, s, true));
  CKC(c, kconv_c(D, c->Vh32, M, PP, c->n1, c->n2, c->n3, s));
  CKC(c, mark(c, 3, s, true));
  CKC(c, (gemm_c_comp<float2, float2, float2>(A_MK, B_KN, P, n, P, M, P, PP, Psi, n, (long)P * n,
                                              Y, n, (long)P * n, nk, s)));
  CKC(c, mark(c, 4, s, true));
  CKC(c, (gemm_c_comp<float2, float2, double2>(A_MK_CONJ, B_KN, N, n, P, c->X32, P, (long)N * P,
                                               Y, n, (long)P * n, KC, n, (long)N * n, nk, s)));
  CKC(c, mark(c, 5, s, true));
  CKC(c, ex_reduce_c(Psi, Y, (long)nk * P * n, nk, c->partial, c->n_partial, ex, s));
  CKC(c, mark(c, 6, s, true));
  return THC_OK;
}

// Slice products of the tensor-core GEMMs S1, S2, S4a and S4b (6 or 8, see
// tc_gemm.cu).  Measured at 4x4x4 k, N_P = 1200 against the FP64 oracle: the
// back-projections S4a and S4b, whose outputs carry the final precision, take
// 8; S1 (rounded to FP32 Psi) and S2 (FP32 D) take 6.  THC_MIXED_EXT takes 8
// in S1 as well: with M carried to about 35 bits, the slices of Psi are the
// next limit on a fitted kernel.
constexpr int kProducts[4] = {6, 6, 8, 8};
constexpr int kProductsExt[4] = {8, 6, 8, 8};

// Host buffers of a host-buffer build that moves C in and KC out in halves on
// the context's copy stream, beside S1 and S4b, which then run per half.
struct HostIO {
  const double2* C;
  double2* KC;
};

static thc_status build_tc(thc_ctx* c, const double2* C, double2* KC, double* ex, double2* Kao = nullptr,
                           const HostIO* io = nullptr) {
  const int* kProducts = c->precision == THC_MIXED_EXT ? kProductsExt : ::kProducts;
  const int nk = c->nk, N = c->nbas, n = c->nocc, P = c->nisdf;
  const long PP = (long)P * P, Pn = (long)P * n, Nn = (long)N * n;
  float2* Psi = (float2*)c->Psi;
  float2* D = (float2*)c->D;
  float2* M = (float2*)c->M;
  float2* Y = (float2*)c->Y;
  cudaStream_t s = c->stream;
  CKC(c, mark(c, 0, s, false));
  // host-buffer build: the copy stream brings C in two halves of the k
  // points, and S1 starts on the first while the second is in flight (the
  // halves keep the whole product's K chunks, so the results are the same bits)
  const int nh = io ? 2 : 1;
  auto kb = [&](int h) { return nk * h / nh; };
  cudaStream_t cs = c->cstream;
  if (io) {
    CKC(c, cudaEventRecord(c->cev[0], s));
    CKC(c, cudaStreamWaitEvent(cs, c->cev[0], 0));
    for (int h = 0; h < nh; h++) {
      CKC(c, cudaMemcpyAsync((double2*)C + kb(h) * Nn, io->C + kb(h) * Nn, sizeof(double2) * Nn * (kb(h + 1) - kb(h)),
                             cudaMemcpyHostToDevice, cs));
      CKC(c, cudaEventRecord(c->cev[1 + h], cs));
    }
  }
  for (int h = 0; h < nh; h++) {
    const int b0 = kb(h), nb = kb(h + 1) - kb(h);
    if (io) CKC(c, cudaStreamWaitEvent(s, c->cev[1 + h], 0));
    // S1  Psi = X^T C on tensor cores: B = embedded C, one exponent per orbital
    CKC(c, col_exponents_z(C + b0 * Nn, Nn, n, nb, N, n, c->eC + b0 * n, s));
    CKC(c, embed_b(C + b0 * Nn, true, Nn, n, 1, false, false, nb, N, n, c->eC + b0 * n,
                   c->Bc_pl + (long)b0 * 2 * n * c->ldC, c->plBc, c->ldC, s));
    if (h == 0) CKC(c, record_core(c, 0, 0, s));
    // A = X^T, read from FP32 X [mu][P] and sliced (transposed) inside the GEMM
    CKC(c, tc_gemm(c->opXT, c->opBc, P, 2 * n, 2 * N, nb, c->eXT + (long)b0 * P, P, c->eC + b0 * n, n,
                   Psi + b0 * Pn, false, 2 * n, 2 * Pn, c->part_s0, c->part_bc, c->tc_err, s,
                   h == nh - 1 ? core_event(c, 0, 1) : nullptr, kProducts[0], 2, 0, nullptr, nullptr, 0, nullptr,
                   b0, tc_chunk_blocks(P, 2 * n, 2 * N, nk)));
  }
  CKC(c, mark(c, 1, s, false));
  // S2  D = Psi Psi^H on tensor cores: A = Psi and B = embedded Psi^H share the
  // row exponents of Psi
  // (one kernel: the slices of Psi with its row exponents, and the embedded Psi^H)
  CKC(c, slice_rows_exact(Psi, n, (long)nk * P, c->ePsi, c->PsiA_pl, c->plPs, c->ldPs, s, c->Bd_pl, c->plBd));
  CKC(c, record_core(c, 1, 0, s));
  // D is Hermitian, so only the tiles that reach the diagonal are multiplied
  // (Hermitian V: M^k is Hermitian too, and S3 reads D on and above the
  // diagonal only, so S2 leaves the part below it unwritten)
  const bool a_f32 = c->plM == 0;
  const bool herm = c->herm_v && c->hkeys && a_f32;
  // (THC-AO-K reads all of D for its energy, so D is written whole there)
  const bool upper = herm && !Kao;
  CKC(c, tc_gemm(c->opPs, c->opBd, P, 2 * P, 2 * n, nk, c->ePsi, P, c->ePsi, P, D, false, 2 * P, 2 * PP,
                 c->part_s0, c->part_bc, c->tc_err, s, core_event(c, 1, 1), kProducts[1], 0, upper ? 2 : 1));
  c->d_upper = upper;
  c->m_ext = herm && c->Mlo;
  CKC(c, mark(c, 2, s, false));
  // S3  M = IDFT(DFT(D) o Vh) in FP32
  // (2^3, 3^3 and 4^3 meshes: the convolution also finds the exact row
  // exponents of M that S4a slices it with)
  bool have_eM = false;
  if (herm) {
    CKC(c, kconv_c_herm(D, c->Vh32, M, P, c->n1, c->n2, c->n3, c->hkeys, c->eM, c->tc_err, core_event(c, 2, 0),
                        core_event(c, 2, 1), s, c->Mlo));
    have_eM = true;
  } else if (a_f32) {
    CKC(c, kconv_c_rowexp(D, c->Vh32, M, P, c->n1, c->n2, c->n3, c->eM, &have_eM, c->tc_err,
                          core_event(c, 2, 0), core_event(c, 2, 1), s));
  } else {
    CKC(c, record_core(c, 2, 0, s));
    CKC(c, kconv_c(D, c->Vh32, M, PP, c->n1, c->n2, c->n3, s));
    CKC(c, record_core(c, 2, 1, s));
  }
  CKC(c, mark(c, 3, s, false));
  if (Kao) {
    // THC-AO-K: Z = M X^T (A = M as in S4a; B = the embedded X^T, made once
    // per collocation), then K = conj(X) Z (A = X as in S4b; B = embedded Z)
    if (a_f32) {
      if (!have_eM) CKC(c, row_exponents_rows(M, P, (long)nk * P, c->eM, s));
    } else {
      CKC(c, slice_rows_exact(M, P, (long)nk * P, c->eM, c->M_pl, c->plM, c->ldM, s));
    }
    if (!c->bxt_valid) {
      CKC(c, embed_b(c->X32, false, (long)N * c->ldX, 1, c->ldX, false, false, nk, P, N, c->eXn, c->BxT_pl, c->plAO,
                     c->ldAO, s));
      c->bxt_valid = true;
    }
    CKC(c, record_core(c, 3, 0, s));
    CKC(c, tc_gemm(a_f32 ? c->opMf : c->opM, c->opBxT, P, 2 * N, 2 * P, nk, c->eM, P, c->eXn, N, c->Zao, false,
                   2 * N, 2L * P * N, c->ps0_ao, c->pbc_ao, c->tc_err, s, core_event(c, 3, 1), 8,
                   !a_f32 ? 0 : (herm && c->Mlo) ? 3 : 1));
    CKC(c, mark(c, 4, s, false));
    CKC(c, col_exponents_c(c->Zao, (long)P * N, N, nk, P, N, c->eZ, s));
    CKC(c, embed_b(c->Zao, false, (long)P * N, N, 1, false, true, nk, P, N, c->eZ, c->Bz_pl, c->plAO, c->ldAO, s));
    CKC(c, record_core(c, 4, 0, s));
    CKC(c, tc_gemm(c->opXn, c->opBz, N, 2 * N, 2 * P, nk, c->eXn, N, c->eZ, N, Kao, true, 2 * N, 2L * N * N,
                   c->ps0_ao, c->pbc_ao, c->tc_err, s, core_event(c, 4, 1), 8, 1));
    CKC(c, mark(c, 5, s, false));
    CKC(c, record_core(c, 5, 0, s));
    CKC(c, ex_reduce_c(D, M, (long)nk * PP, nk, c->partial, c->n_partial, ex, s));
    CKC(c, record_core(c, 5, 1, s));
    CKC(c, mark(c, 6, s, false));
    return THC_OK;
  }
  // S4a Y = M Psi on tensor cores: A = M in FP32, cut into its slices inside
  // the GEMM with the exact row exponents of M; B = embedded Psi with one
  // exponent per orbital
  // (odd N_P: M's slices go through HBM, written by the warp-per-row kernel)
  if (a_f32) {
    if (!have_eM) CKC(c, row_exponents_rows(M, P, (long)nk * P, c->eM, s));
  } else {
    CKC(c, slice_rows_exact(M, P, (long)nk * P, c->eM, c->M_pl, c->plM, c->ldM, s));
  }
  CKC(c, col_exponents_c(Psi, Pn, n, nk, P, n, c->eY, s));
  CKC(c, embed_b(Psi, false, Pn, n, 1, false, false, nk, P, n, c->eY, c->By_pl, c->plBy, c->ldM, s));
  CKC(c, record_core(c, 3, 0, s));
  // (THC_MIXED_EXT with the Hermitian form: M's fp16 remainders join its FP32 values)
  const int m_conv = !a_f32 ? 0 : (herm && c->Mlo) ? 3 : 1;
  // (the split-K combine that writes Y also forms the block sums of <Psi, Y> for S5)
  int ex_blocks = 0;
  CKC(c, tc_gemm(a_f32 ? c->opMf : c->opM, c->opBy, P, 2 * n, 2 * P, nk, c->eM, P, c->eY, n, Y, false, 2 * n,
                 2 * Pn, c->part_s0, c->part_bc, c->tc_err, s, core_event(c, 3, 1), kProducts[2], m_conv, 0,
                 (const float*)Psi, c->partial, c->n_partial, &ex_blocks));
  CKC(c, mark(c, 4, s, false));
  // S4b KC = conj(X) Y on tensor cores: A = X (FP32, sliced inside the GEMM),
  // B = embedded Y (conj-A form)
  CKC(c, col_exponents_c(Y, Pn, n, nk, P, n, c->eY, s));
  CKC(c, embed_b(Y, false, Pn, n, 1, false, true, nk, P, n, c->eY, c->By_pl, c->plBy, c->ldM, s));
  CKC(c, record_core(c, 4, 0, s));
  // (host-buffer build: per half of the k points, its KC going out on the
  // copy stream while the next half is computed)
  for (int h = 0; h < nh; h++) {
    const int b0 = kb(h), nb = kb(h + 1) - kb(h);
    CKC(c, tc_gemm(c->opXn, c->opBy, N, 2 * n, 2 * P, nb, c->eXn + (long)b0 * N, N, c->eY + b0 * n, n,
                   KC + b0 * Nn, true, 2 * n, 2 * Nn, c->part_s0, c->part_bc, c->tc_err, s,
                   h == nh - 1 ? core_event(c, 4, 1) : nullptr, kProducts[3], 1, 0, nullptr, nullptr, 0, nullptr,
                   b0, tc_chunk_blocks(N, 2 * n, 2 * P, nk)));
    if (io) {
      CKC(c, cudaEventRecord(c->cev[3 + h], s));
      CKC(c, cudaStreamWaitEvent(cs, c->cev[3 + h], 0));
      CKC(c, cudaMemcpyAsync(io->KC + b0 * Nn, KC + b0 * Nn, sizeof(double2) * Nn * nb, cudaMemcpyDeviceToHost, cs));
    }
  }
  CKC(c, mark(c, 5, s, false));
  CKC(c, record_core(c, 5, 0, s));
  if (ex_blocks > 0)
    CKC(c, ex_finalize(c->partial, ex_blocks, nk, ex, s));
  else
    CKC(c, ex_reduce_c(Psi, Y, (long)nk * P * n, nk, c->partial, c->n_partial, ex, s));
  CKC(c, record_core(c, 5, 1, s));
  CKC(c, mark(c, 6, s, false));
  if (io) {   // the copies out joined to the context's stream
    CKC(c, cudaEventRecord(c->cev[5], cs));
    CKC(c, cudaStreamWaitEvent(s, c->cev[5], 0));
  }
  return THC_OK;
}

// The tensor-core build as one CUDA graph launch: its 16-odd kernels (and the
// stage-boundary events) are captured from the stream once per (C, KC, ex)
// triple and replayed.  If the capture fails the build runs directly.
static thc_status build_tc_graph(thc_ctx* c, const double2* C, double2* KC, double* ex) {
  if (!c->gexec || c->g_C != C || c->g_KC != KC || c->g_ex != ex) {
    drop_graph(c);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      return build_tc(c, C, KC, ex);
    }
    const thc_status st = build_tc(c, C, KC, ex);
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    cudaGraphExec_t x = nullptr;
    if (st == THC_OK && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
      c->gexec = x;
      c->g_C = C;
      c->g_KC = KC;
      c->g_ex = ex;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // a failed capture leaves no sticky error: run the build directly
    if (!c->gexec) return build_tc(c, C, KC, ex);
  }
  CKC(c, cudaGraphLaunch(c->gexec, c->stream));
  return THC_OK;
}

thc_status thc_build(thc_ctx* c, const double* C, double* KC, double* ex) {
  if (!c || !C || !KC || !ex) return THC_ERR_ARG;
  if (!aligned16(C) || !aligned16(KC) || ((uintptr_t)ex & 7u)) return THC_ERR_ARG;
  const size_t kcb = (size_t)c->nk * c->nbas * c->nocc * sizeof(double2);
  const char* a = (const char*)C;
  const char* b = (const char*)KC;
  if (a < b + kcb && b < a + kcb) return THC_ERR_ARG;  // KC aliases C
  if (!c->have_x || !c->have_v) return THC_ERR_STATE;
  thc_status st;
  if (c->precision == THC_FP64) st = build_fp64(c, (const double2*)C, (double2*)KC, ex);
  else if (c->precision == THC_MIXED_SIMT) st = build_mixed(c, (const double2*)C, (double2*)KC, ex);
  else if (profiling(c)) st = build_tc(c, (const double2*)C, (double2*)KC, ex);
  else st = build_tc_graph(c, (const double2*)C, (double2*)KC, ex);
  if (st == THC_OK) {
    c->built = true;
    if (c->prof_max > 0 && c->prof_n < c->prof_max) {
      c->prof_n++;
    }
  }
  return st;
}

// The THC-AO-K workspace, made by the first thc_build_K of a context.
static thc_status ao_prepare(thc_ctx* c) {
  if (c->ao_ready) return THC_OK;
  const int nk = c->nk, N = c->nbas, P = c->nisdf;
  struct Want { void** p; size_t bytes; };
  std::vector<Want> want;
  if (c->precision == THC_FP64) {
    want.push_back({(void**)&c->Wao, sizeof(double2) * (size_t)nk * N * P});
  } else {
    c->ldAO = pad8(2 * P);
    c->plAO = (long)nk * 2 * N * c->ldAO;
    const long npart = std::max(tc_partial_elems(P, 2 * N, 2 * P, nk), tc_partial_elems(N, 2 * N, 2 * P, nk));
    want.push_back({(void**)&c->Zao, sizeof(float2) * (size_t)nk * P * N});
    want.push_back({(void**)&c->BxT_pl, 3 * 2 * (size_t)c->plAO});
    want.push_back({(void**)&c->Bz_pl, 3 * 2 * (size_t)c->plAO});
    want.push_back({(void**)&c->eZ, sizeof(int) * (size_t)nk * N});
    if (npart > 0) {
      want.push_back({(void**)&c->ps0_ao, sizeof(int) * (size_t)npart});
      want.push_back({(void**)&c->pbc_ao, sizeof(float) * (size_t)npart});
    }
  }
  for (auto& w : want) {
    cudaError_t e = cudaMalloc(w.p, w.bytes);
    if (e == cudaSuccess) e = cudaMemset(*w.p, 0, w.bytes);   // plane padding stays zero
    if (e != cudaSuccess) {
      cudaGetLastError();
      for (auto& x : want)
        if (*x.p) {
          cudaFree(*x.p);
          *x.p = nullptr;
        }
      c->last_error = std::string("thc_build_K workspace: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? THC_ERR_OOM : THC_ERR_CUDA;
    }
  }
  if (tc_form(c->precision)) {
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < 3 && e == cudaSuccess; p++) {
      e = make_plane_map(c->opBxT.map[p], c->BxT_pl + p * c->plAO, nk, 2 * N, 2 * P, c->ldAO);
      if (e == cudaSuccess) e = make_plane_map(c->opBz.map[p], c->Bz_pl + p * c->plAO, nk, 2 * N, 2 * P, c->ldAO);
    }
    if (e != cudaSuccess) {
      c->last_error = std::string("thc_build_K maps: ") + cudaGetErrorString(e);
      return THC_ERR_CUDA;
    }
  }
  c->ao_ready = true;
  return THC_OK;
}

thc_status thc_build_K(thc_ctx* c, const double* C, double* K, double* ex) {
  if (!c || !C || !K || !ex) return THC_ERR_ARG;
  if (!aligned16(C) || !aligned16(K) || ((uintptr_t)ex & 7u)) return THC_ERR_ARG;
  if (c->precision == THC_MIXED_SIMT) return THC_ERR_UNSUPPORTED;
  const size_t cb = (size_t)c->nk * c->nbas * c->nocc * sizeof(double2);
  const size_t kb = (size_t)c->nk * c->nbas * c->nbas * sizeof(double2);
  const char* a = (const char*)C;
  const char* b = (const char*)K;
  if (a < b + kb && b < a + cb) return THC_ERR_ARG;   // K overlaps C
  if (!c->have_x || !c->have_v) return THC_ERR_STATE;
  thc_status st = ao_prepare(c);
  if (st != THC_OK) return st;
  if (c->precision == THC_FP64) st = build_fp64(c, (const double2*)C, nullptr, ex, (double2*)K);
  else st = build_tc(c, (const double2*)C, nullptr, ex, (double2*)K);
  if (st == THC_OK) {
    c->built = true;
    if (c->prof_max > 0 && c->prof_n < c->prof_max) c->prof_n++;
  }
  return st;
}

// The host-buffer tensor-core build with its copies overlapped (build_tc with
// HostIO), as one CUDA graph launch captured per pair of host buffers; if the
// capture is refused (pageable host memory, for one) it runs directly.
static thc_status build_host_overlapped(thc_ctx* c, const double2* C_host, double2* KC_host) {
  const HostIO io{C_host, KC_host};
  const double2* C = (const double2*)c->Cdev;
  double2* KC = (double2*)c->KCdev;
  if (!c->gexec_h || c->gh_C != C_host || c->gh_KC != KC_host) {
    if (c->gexec_h) cudaGraphExecDestroy(c->gexec_h);
    c->gexec_h = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      return build_tc(c, C, KC, c->exdev, nullptr, &io);
    }
    const thc_status st = build_tc(c, C, KC, c->exdev, nullptr, &io);
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    cudaGraphExec_t x = nullptr;
    if (st == THC_OK && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
      c->gexec_h = x;
      c->gh_C = C_host;
      c->gh_KC = KC_host;
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!c->gexec_h) return build_tc(c, C, KC, c->exdev, nullptr, &io);
  }
  CKC(c, cudaGraphLaunch(c->gexec_h, c->stream));
  return THC_OK;
}

thc_status thc_build_host(thc_ctx* c, const double* C_host, double* KC_host, double* ex_host) {
  if (!c || !C_host || !KC_host || !ex_host) return THC_ERR_ARG;
  if (!c->have_x || !c->have_v) return THC_ERR_STATE;
  if (tc_form(c->precision) && !profiling(c) && c->nk >= 2) {
    const thc_status st = build_host_overlapped(c, (const double2*)C_host, (double2*)KC_host);
    if (st != THC_OK) return st;
    c->built = true;
    CKC(c, cudaMemcpyAsync(ex_host, c->exdev, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return thc_sync(c);
  }
  const size_t kcb = (size_t)c->nk * c->nbas * c->nocc * sizeof(double2);
  CKC(c, cudaMemcpyAsync(c->Cdev, C_host, kcb, cudaMemcpyHostToDevice, c->stream));
  thc_status st = thc_build(c, (const double*)c->Cdev, (double*)c->KCdev, c->exdev);
  if (st != THC_OK) return st;
  CKC(c, cudaMemcpyAsync(KC_host, c->KCdev, kcb, cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaMemcpyAsync(ex_host, c->exdev, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return thc_sync(c);
}

thc_status thc_debug_set_wait_limit(thc_ctx* c, long long cycles) {
  if (!c) return THC_ERR_ARG;
  if (!c->tc_err) return THC_ERR_UNSUPPORTED;   // only the tensor-core form has device-side waits
  const long long v = cycles > 0 ? cycles : 0;
  CKC(c, cudaMemcpyAsync(reinterpret_cast<char*>(c->tc_err) + 8, &v, sizeof v, cudaMemcpyHostToDevice, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return THC_OK;
}

thc_status thc_debug_fail_alloc(int nth) {
  g_fail_alloc = nth >= 0 ? nth : -1;
  return THC_OK;
}

thc_status thc_sync(thc_ctx* c) {
  if (!c) return THC_ERR_ARG;
  // the error word comes back with the stream's last work: one wait
  if (c->tc_err) CKC(c, cudaMemcpyAsync(c->tc_err_host, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  if (!c->tc_err) return THC_OK;
  const int h = *c->tc_err_host;
  if (h) {
    CKC(c, cudaMemset(c->tc_err, 0, sizeof(int)));
    c->last_error = "device wait timed out, code " + std::to_string(h);
    return THC_ERR_TIMEOUT;
  }
  return THC_OK;
}

__global__ void ints_to_doubles(const int* __restrict__ v, double* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = (double)v[i];
}

thc_status thc_get_intermediate(thc_ctx* c, int which, double* out) {
  if (!c || !out || !aligned16(out) || which < 0 || which > 4) return THC_ERR_ARG;
  if (which == 4 && !tc_form(c->precision)) return THC_ERR_ARG;
  if (!c->built) return THC_ERR_STATE;
  if (which == 4) {
    const long n = (long)c->nk * c->nisdf;
    ints_to_doubles<<<(unsigned)std::min<long>((n + 255) / 256, 152L * 8), 256, 0, c->stream>>>(c->eM, out, n);
    CKC(c, cudaGetLastError());
    CKC(c, cudaStreamSynchronize(c->stream));
    return THC_OK;
  }
  const long n = (which == 0 || which == 3) ? (long)c->nk * c->nisdf * c->nocc
                                            : (long)c->nk * c->nisdf * c->nisdf;
  void* src = which == 0 ? c->Psi : which == 1 ? c->D : which == 2 ? c->M : c->Y;
  if (which == 2 && c->Mlo && c->m_ext)
    CKC(c, mlo_combine_c2z((const float2*)src, c->Mlo, (double2*)out, n, c->stream));
  else if (which == 1 && tc_form(c->precision) && c->d_upper)
    CKC(c, hermitian_fill_c2z((const float2*)src, (double2*)out, c->nisdf, c->nk, c->stream));
  else if (c->precision == THC_FP64)
    CKC(c, cudaMemcpyAsync(out, src, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  else
    CKC(c, convert_c2z((const float2*)src, (double2*)out, n, c->stream));
  CKC(c, cudaStreamSynchronize(c->stream));
  return THC_OK;
}

thc_status thc_stage_times(thc_ctx* c, float ms[6]) {
  if (!c || !ms) return THC_ERR_ARG;
  for (int i = 0; i < kStages; i++) ms[i] = 0.f;
  if (!c->built) return THC_OK;
  if (c->prof_max > 0) return THC_ERR_STATE;  // events are going to the profile slots
  CKC(c, cudaEventSynchronize(c->ev[6]));
  for (int i = 0; i < kStages; i++) CKC(c, cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]));
  return THC_OK;
}

thc_status thc_profile_begin(thc_ctx* c, int max_builds) {
  if (!c || max_builds < 1 || max_builds > 4096) return THC_ERR_ARG;
  for (cudaEvent_t e : c->prof) cudaEventDestroy(e);
  c->prof.assign((size_t)max_builds * kProfEv, nullptr);
  for (auto& e : c->prof) CKC(c, cudaEventCreate(&e));
  c->prof_max = max_builds;
  c->prof_n = 0;
  return THC_OK;
}

thc_status thc_profile_end(thc_ctx* c, float mean_ms[6], int* nbuilds) {
  if (!c || !mean_ms || !nbuilds) return THC_ERR_ARG;
  if (c->prof_max <= 0) return THC_ERR_STATE;
  for (int i = 0; i < kStages; i++) mean_ms[i] = 0.f;
  const int nb = c->prof_n;
  float core[kStages] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int b = 0; b < nb; b++) {
    cudaEvent_t* e = &c->prof[(size_t)b * kProfEv];
    CKC(c, cudaEventSynchronize(e[6]));
    for (int i = 0; i < kStages; i++) {
      float t = 0.f;
      CKC(c, cudaEventElapsedTime(&t, e[i], e[i + 1]));
      mean_ms[i] += t;
      CKC(c, cudaEventElapsedTime(&t, e[7 + 2 * i], e[8 + 2 * i]));
      core[i] += t;
    }
  }
  if (nb > 0)
    for (int i = 0; i < kStages; i++) {
      mean_ms[i] /= nb;
      c->core_ms[i] = core[i] / nb;
    }
  c->core_valid = nb > 0;
  *nbuilds = nb;
  for (cudaEvent_t e : c->prof) cudaEventDestroy(e);
  c->prof.clear();
  c->prof_max = 0;
  c->prof_n = 0;
  return THC_OK;
}

thc_status thc_profile_kernels(const thc_ctx* c, float core_ms[6]) {
  if (!c || !core_ms) return THC_ERR_ARG;
  if (!c->core_valid) return THC_ERR_STATE;
  for (int i = 0; i < kStages; i++) core_ms[i] = c->core_ms[i];
  return THC_OK;
}

thc_status thc_hermitian_kernel(const thc_ctx* c, int* hermitian) {
  if (!c || !hermitian) return THC_ERR_ARG;
  if (!c->have_v) return THC_ERR_STATE;
  *hermitian = (tc_form(c->precision) && c->herm_v && c->hkeys && c->plM == 0) ? 1 : 0;
  return THC_OK;
}

thc_status thc_launches_per_build(const thc_ctx* c, int* launches) {
  if (!c || !launches) return THC_ERR_ARG;
  // FP64 and CUDA-core forms: S1, S2, S3, S4a, S4b, E_x partial, E_x final.
  // Tensor-core form: S1 3 (exponents, embed, GEMM), S2 2 (slices with their
  // row exponents and the embedded Psi^H, GEMM), S3 + S4a 5 (the convolution, the row
  // exponents of M: in the convolution plus a conversion kernel on the
  // 2^3 .. 4^3 meshes, else a kernel of their own; exponents of Psi, embed,
  // GEMM), S4b 3, E_x 2; S1, S4a and S4b add a combine kernel when split
  // along K, and S4a's combine then forms the partial sums of E_x (E_x 1)
  // when its result rows are 16-byte strided (n_occ even).
  if (tc_form(c->precision)) {
    const int s1 = tc_partial_elems(c->nisdf, 2 * c->nocc, 2 * c->nbas, c->nk) > 0 ? 1 : 0;
    const int s4a = tc_partial_elems(c->nisdf, 2 * c->nocc, 2 * c->nisdf, c->nk) > 0 ? 1 : 0;
    const int s4b = tc_partial_elems(c->nbas, 2 * c->nocc, 2 * c->nisdf, c->nk) > 0 ? 1 : 0;
    *launches = 3 + s1 + 2 + 1 + 4 + s4a + 3 + s4b + (s4a && c->nocc % 2 == 0 ? 1 : 2);
  } else {
    *launches = 7;
  }
  return THC_OK;
}

}  // extern "C"
