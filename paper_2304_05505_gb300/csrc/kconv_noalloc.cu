// thc_kconv_noalloc: the k-mesh convolution (step S3) for callers that cannot
// allocate device memory at the point of the call.
//
// The convolution needs scratch for the prepared kernel Vh = DFT_q(V)/N_k.
// The rest of the library allocates that inside a context; this entry point
// instead uses one file-scope device array, g_vh_scratch, of kScratchElems
// complex128 elements (32 MiB).  The array exists on every GPU that loads the
// library, for the life of the process.
//
// In host code the name g_vh_scratch is only a host-side stand-in for the
// device array, not a device address: handing it to a kernel would fault or,
// where the GPU can reach host memory, silently use the wrong memory.  The
// device address is therefore fetched with cudaGetSymbolAddress, once per
// device, with that device current, on the first call made while that device
// is current, and cached.  Because that first call does this set-up, it should
// come before any stream capture.
//
// Every call on a device shares the one array and leaves the last call's
// prepared kernel in it.  Nothing in it has to start at zero: each call
// overwrites the part it reads.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array and give wrong results;
// the caller must order them.
#include "thc_internal.cuh"

#include <mutex>

namespace {

constexpr long kScratchElems = 1L << 21;   // 2,097,152 complex128 elements = 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_vh_scratch[kScratchElems];

std::mutex g_setup_mutex;
double2* g_scratch_addr[kMaxDevices];       // device address per device, nullptr until set up

}  // namespace

extern "C" thc_status thc_kconv_noalloc(const double* D, const double* V, double* M, int n1, int n2, int n3,
                                        long npq, void* stream) {
  if (!D || !V || !M) return THC_ERR_ARG;
  if (((uintptr_t)D | (uintptr_t)V | (uintptr_t)M) & 15u) return THC_ERR_ARG;
  if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > 8 || n2 > 8 || n3 > 8 || npq < 1) return THC_ERR_ARG;
  const long nk = (long)n1 * n2 * n3;
  // M must not overlap D or V: the convolution reads D while it writes M
  const size_t bytes = (size_t)nk * (size_t)npq * sizeof(double2);
  const char* m0 = (const char*)M;
  for (const char* in : {(const char*)D, (const char*)V})
    if (npq <= kScratchElems / nk && m0 < in + bytes && in < m0 + bytes) {
      set_global_error("thc_kconv_noalloc: M overlaps D or V");
      return THC_ERR_ARG;
    }
  if (npq > kScratchElems / nk) {
    set_global_error("thc_kconv_noalloc: N_k * npq exceeds the static scratch of 2097152 complex "
                     "elements (32 MiB)");
    return THC_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_global_error(e != cudaSuccess ? cudaGetErrorString(e) : "thc_kconv_noalloc: device index too large");
    return THC_ERR_CUDA;
  }
  double2* scratch;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_vh_scratch);
      if (e != cudaSuccess || !p) {
        set_global_error(std::string("thc_kconv_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return THC_ERR_CUDA;
      }
      g_scratch_addr[dev] = (double2*)p;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  e = prepare_kernel_z((const double2*)V, scratch, nullptr, npq, n1, n2, n3, s);
  if (e == cudaSuccess) e = kconv_z((const double2*)D, scratch, (double2*)M, npq, n1, n2, n3, s);
  if (e != cudaSuccess) {
    set_global_error(std::string("thc_kconv_noalloc: ") + cudaGetErrorString(e));
    return THC_ERR_CUDA;
  }
  return THC_OK;
}
