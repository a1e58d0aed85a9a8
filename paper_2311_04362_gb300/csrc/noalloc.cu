// noalloc.cu -- ls_residual_gradient_noalloc: the fused residual/gradient
// pass (the same kernels as ls_residual_gradient) for callers that must not
// allocate device memory, e.g. code running inside a memory pool or arena it
// does not own, or under a framework that forbids cudaMalloc on its hot path.
//
// The pass needs scratch for one partial result per CTA.  Here that scratch is
// a file-scope __device__ array of fixed size, so the call allocates nothing:
// every GPU that loads this library keeps kNoAllocBytes of it until the
// process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "ls_internal.cuh"

namespace {

constexpr int kNoAllocMaxN = 1024;      // columns
constexpr int kNoAllocMaxCtas = 160;    // one partial per CTA (one CTA per SM)
constexpr int kNoAllocMaxDevices = 64;
// partials (kNoAllocMaxCtas x (n + 2) doubles) followed by 4 status words
constexpr size_t kPartDoubles = (size_t)kNoAllocMaxCtas * (kNoAllocMaxN + 2);
constexpr size_t kNoAllocBytes = kPartDoubles * sizeof(double) + 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device (host code may not use the
// symbol itself as a device pointer: on the host it is only a stand-in), with
// the device's SM count and compute capability, looked up once per device.
void* g_scratch_addr[kNoAllocMaxDevices] = {nullptr};
int g_num_sms[kNoAllocMaxDevices] = {0};
int g_cc[kNoAllocMaxDevices] = {0};     // 10 * major + minor
std::mutex g_setup_mu;

cudaError_t scratch_for_device(int dev, void** out, int* num_sms, int* cc) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // device `dev` is current
    if (e != cudaSuccess) return e;
    int sms = 0, major = 0, minor = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess) return e;
    g_num_sms[dev] = sms;
    g_cc[dev] = 10 * major + minor;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  *num_sms = g_num_sms[dev];
  *cc = g_cc[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" LS_API ls_status ls_residual_gradient_noalloc(void* cuda_stream, const double* A, int64_t m, int64_t n,
                                                         int64_t lda, const double* b, const double* x,
                                                         const double* r_prev, double* r_out, double* c,
                                                         double* norms) {
  if (!A || !b || !x || !c || !norms) return LS_EINVAL;
  if (m < 1 || n < 1 || n > m) return LS_EINVAL;
  if (n > kNoAllocMaxN) return LS_EINVAL;                       // scratch holds n <= 1024 columns
  if (lda < n || (lda & 1) || (reinterpret_cast<uintptr_t>(A) & 15)) return LS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LS_ECUDA;
  void* scratch = nullptr;
  int sms = 0, cc = 0;
  if (scratch_for_device(dev, &scratch, &sms, &cc) != cudaSuccess) return LS_ECUDA;
  if (cc != 103) return LS_ECUDA;                                 // built for sm_103a only

  // A context on the stack: only what the launch helpers read (no allocation).
  ls_ctx ctx;
  ctx.device = dev;
  ctx.num_sms = sms;
  ctx.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  double* part = reinterpret_cast<double*>(scratch);
  ctx.d_status = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(scratch) + kPartDoubles * sizeof(double));

  lsk::PassGeom g = lsk::pass_geometry(&ctx, n, m);
  // the pass walks its tiles with a grid stride, so fewer CTAs than SMs is
  // still correct; the partial count below follows g.grid
  g.grid = std::min(g.grid, kNoAllocMaxCtas);
  CUtensorMap map;
  if (lsk::make_tensor_map(&ctx, &map, A, m, n, lda, g) != cudaSuccess) return LS_ECUDA;
  // the status words must start at zero; the partials are fully overwritten
  if (cudaMemsetAsync(ctx.d_status, 0, 4 * sizeof(unsigned int), ctx.stream) != cudaSuccess) return LS_ECUDA;
  if (lsk::launch_fused_pass(&ctx, map, g, m, n, b, x, r_prev, r_out, part, nullptr) != cudaSuccess) return LS_ECUDA;
  if (lsk::launch_reduce_partials(&ctx, part, g.grid, n, c, norms) != cudaSuccess) return LS_ECUDA;
  if (!r_prev && cudaMemsetAsync(norms + 1, 0, sizeof(double), ctx.stream) != cudaSuccess) return LS_ECUDA;
  unsigned int status = 0;
  if (cudaMemcpyAsync(&status, ctx.d_status, sizeof status, cudaMemcpyDeviceToHost, ctx.stream) != cudaSuccess)
    return LS_ECUDA;
  if (cudaStreamSynchronize(ctx.stream) != cudaSuccess) return LS_ECUDA;
  if (status & LS_DEV_TIMEOUT) return LS_ETIMEOUT;
  return LS_OK;
}
