// snn_noalloc.cu -- network construction into caller-owned device memory,
// without any device allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: a host program whose
// device memory is owned by one pool allocator (a framework that hands every
// byte out itself and must account for it), a real-time loop that cannot
// afford the implicit device synchronisation and latency of cudaMalloc /
// cudaFree, or a process that has already reserved nearly all device memory.
// For them snn_build_rows_static runs the same construction kernel as
// snn_build_network, but its scratch -- the Eq. 1 module thresholds and the
// Gaussian quantile table -- lives in one file-scope device array of fixed
// size, and the rows are written into memory the caller passes in.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/snn.h"
#include "snn_internal.h"

namespace {

// Largest grid the static scratch serves: 1024 modules (for example 32 x 32).
constexpr uint32_t kMaxModules = 1024;
constexpr size_t kCdfBytes = (size_t)kMaxModules * (kMaxModules - 1) * 4;   // 4,190,208 B
constexpr size_t kZtabOffset = (kCdfBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kZtabOffset + (size_t)snn::kZTab * 4;      // about 4.2 MB

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) uint8_t g_build_scratch[kScratchBytes];

// Device address of g_build_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

int scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return snn_fail(SNN_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return snn_fail(SNN_ERR_LIMIT, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    // first call on this device, with it current: the symbol's device address
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_build_scratch);
    if (e != cudaSuccess || !p)
      return snn_fail(SNN_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SNN_OK;
}

}  // namespace

extern "C" int snn_build_rows_static(const snn_params *p, uint64_t seed, void *rows_out, size_t *rows_bytes,
                                     void *cuda_stream) {
  using namespace snn;
  if (!p || !rows_bytes) return snn_fail(SNN_ERR_ARG, "null argument");
  int rc = snn_validate_params(*p);
  if (rc) return rc;
  const uint32_t G = (uint32_t)(p->gx * p->gy);
  if (G > kMaxModules)
    return snn_fail(SNN_ERR_LIMIT, "snn_build_rows_static serves at most 1024 modules (static scratch of " +
                                       std::to_string(kScratchBytes) + " bytes); use snn_build_network");
  const uint32_t N = G * (uint32_t)kK;
  const uint32_t M = (uint32_t)p->out_degree;
  const uint32_t M_pad = (M + 7u) / 8u * 8u;
  const uint32_t row_bytes = M_pad * 4u + M_pad * (p->record_format == SNN_REC_I16 ? 2u : 4u);
  const size_t need = (size_t)N * row_bytes;
  // The size query also looks up the scratch array's device address (which
  // loads this module and places the array on the device), so that a caller
  // can make it before reserving the rest of its device memory.
  void *scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc) return rc;
  if (!rows_out) {           // size query
    *rows_bytes = need;
    return SNN_OK;
  }
  if (*rows_bytes < need) {
    *rows_bytes = need;
    return snn_fail(SNN_ERR_BUFFER, "rows_out holds fewer than N * row_bytes bytes");
  }
  if (reinterpret_cast<uintptr_t>(rows_out) % 16 != 0) return snn_fail(SNN_ERR_ARG, "rows_out must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // The table uploads below read host vectors that are freed on return: a
  // captured copy node would read them again at every replay.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return snn_fail(SNN_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return snn_fail(SNN_ERR_ARG, "snn_build_rows_static must not be called on a capturing stream");
  e = prepare_kernels();
  if (e != cudaSuccess) return snn_fail(SNN_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));

  // host tables: module thresholds and Gaussian quantiles
  std::vector<uint32_t> cdf;
  module_thresholds(*p, cdf);
  std::vector<float> ztab;
  gaussian_table(ztab);
  uint8_t *base = static_cast<uint8_t *>(scratch);
  // every entry the kernel reads is overwritten here: the last call's contents never leak in
  if (!cdf.empty()) {
    e = cudaMemcpyAsync(base, cdf.data(), cdf.size() * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return snn_fail(SNN_ERR_CUDA, std::string("threshold upload: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(base + kZtabOffset, ztab.data(), ztab.size() * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return snn_fail(SNN_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));

  NetDev nd;
  std::memset(&nd, 0, sizeof(nd));
  nd.N = N;
  nd.N_pad = (N + kNeuronAlign - 1) / kNeuronAlign * kNeuronAlign;
  nd.G = G;
  nd.gx = (uint32_t)p->gx;
  nd.M = M;
  nd.M_pad = M_pad;
  nd.D = (uint32_t)p->n_delay + 1u;
  nd.fmt = (uint32_t)p->record_format;
  nd.row_bytes = row_bytes;
  nd.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
  nd.key1 = (uint32_t)(seed >> 32);
  nd.rows = static_cast<uint8_t *>(rows_out);
  BuildDev bd{};
  build_inputs(*p, bd);
  bd.cdf = reinterpret_cast<const uint32_t *>(base);
  bd.ztab = reinterpret_cast<const float *>(base + kZtabOffset);
  e = launch_build_rows(nd, bd, s);
  if (e != cudaSuccess) return snn_fail(SNN_ERR_CUDA, std::string("construction kernel: ") + cudaGetErrorString(e));
  *rows_bytes = need;
  return SNN_OK;
}
