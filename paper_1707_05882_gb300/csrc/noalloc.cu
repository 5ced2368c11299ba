// Batched eigen-decomposition that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns
// the device memory budget (a framework's caching allocator, a fixed-size pool on a
// shared GPU), and code on a path where an allocation would synchronize the device or is
// forbidden (stream-ordered callbacks, latency-critical loops). For them this entry
// point runs the library's eigensolver with its Hessenberg/Schur/eigenvector scratch
// taken from a file-scope device array instead of a plan workspace.
#include <mutex>

#include "vrte_internal.cuh"

namespace vrte {
void batched_eigen(int n, const double* A, double* H, double* Z, double* V, double* X,
                   double* lam_re, double* lam_im, double* scale, int batch, unsigned* status,
                   cudaStream_t s, const int* mask);
}  // namespace vrte

namespace {

// Scratch for H, Z, V (n*n each) and the balancing scale (n) of every matrix in a call:
// (3 n^2 + n) * batch doubles at most, plus a reserved tail that receives the device
// status bits when the caller passes no status word. 2^21 doubles = 16 MiB, held by
// every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratch = size_t(1) << 21;
constexpr size_t kReserved = 8;
constexpr size_t kNoAllocUsable = kNoAllocScratch - kReserved;
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

// Device address of the scratch array per device, resolved once per device with that
// device current (the host-side name is only a stand-in for the symbol).
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

vrte_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VRTE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return VRTE_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return VRTE_OK;
}

}  // namespace

extern "C" vrte_status vrte_eigen_noalloc(const double* d_A, int n, int batch, double* d_lam_re,
                                          double* d_lam_im, double* d_X, unsigned* d_status,
                                          void* stream) {
  // batch <= 65535: the eigenvector kernels take the batch in a grid y or z dimension
  if (!d_A || !d_lam_re || !d_lam_im || !d_X || n < 1 || n > 768 || batch < 1 || batch > 65535)
    return VRTE_ERR_INVALID_ARG;
  size_t per = 3 * (size_t)n * n + (size_t)n;
  if (per * (size_t)batch > kNoAllocUsable) return VRTE_ERR_INVALID_ARG;
  // a launch error left pending by earlier, unrelated work is not this call's failure:
  // it is cleared here so that the check after the launches sees only this call's own
  cudaGetLastError();
  double* base = nullptr;
  vrte_status st = scratch_for_current_device(&base);
  if (st != VRTE_OK) return st;
  size_t nn = (size_t)n * n * batch;
  double* H = base;
  double* Z = H + nn;
  double* V = Z + nn;
  double* scale = V + nn;
  // the kernels initialise every scratch entry they read (H from A, Z = I, V = 0,
  // scale = 1), so the contents left by the previous call need no clearing
  unsigned* status = d_status ? d_status : (unsigned*)(base + kNoAllocUsable);
  vrte::batched_eigen(n, d_A, H, Z, V, d_X, d_lam_re, d_lam_im, scale, batch, status,
                      (cudaStream_t)stream, nullptr);
  if (cudaGetLastError() != cudaSuccess) return VRTE_ERR_CUDA;
  return VRTE_OK;
}
