// leaf_noalloc.cu -- the batched leaf inverse Cholesky for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// moment they need this routine: code inside a host framework that owns the
// whole device-memory budget and forbids hidden allocations (its own caching
// allocator would otherwise be bypassed), or latency-critical loops where an
// allocation's implicit synchronisation with the device is not acceptable.  leaf_invchol_batched allocates its
// scratch (the inverses of the diagonal tiles, and identity-padded copies when
// nl is not a multiple of 32) from the context's pool; this variant takes that
// scratch from one fixed array in device memory instead and allocates nothing.
//
// The array below is part of the library image: every GPU that loads the
// library holds IFAC_NOALLOC_SCRATCH_DOUBLES doubles (32 MiB) until the
// process exits.  In host code `g_leaf_scratch` names a host-side stand-in,
// not device memory, so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.  The cached address belongs
// to the device's current context: resetting the device (cudaDeviceReset)
// between calls is not supported.
#include <mutex>

#include "internal.cuh"

namespace ifac {
cudaError_t leaf_invchol_launch_scratch(cudaStream_t stream, int count, int nl, double* A, int* info, double* wd,
                                        double* pad);
}

#define IFAC_NOALLOC_SCRATCH_DOUBLES (4u << 20)

static __device__ __align__(256) double g_leaf_scratch[IFAC_NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_leaf_scratch on the current device (looked up once).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IFAC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_leaf_scratch);
    if (e != cudaSuccess || !p) return IFAC_ERR_CUDA;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return IFAC_OK;
}
}  // namespace

extern "C" int leaf_invchol_batched_noalloc(void* stream, int count, int nl, const double* S, double* Z, int* info) {
  if (count < 0 || nl <= 0 || nl > 1024 || !S || !Z || !info) return IFAC_ERR_INVALID;
  if (count == 0) return IFAC_OK;
  const int64_t np = ((int64_t)nl + 31) / 32 * 32;
  const int64_t wd_need = (int64_t)count * (np / 32) * 32 * 32;
  const int64_t pad_need = (np == nl) ? 0 : (int64_t)count * np * np;
  if (wd_need + pad_need > (int64_t)IFAC_NOALLOC_SCRATCH_DOUBLES) return IFAC_ERR_TOO_LARGE;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != IFAC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // in place (S == Z) or disjoint: a partial overlap has no defined copy
  const uintptr_t bytes = sizeof(double) * (uintptr_t)count * (uintptr_t)nl * (uintptr_t)nl;
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(S), z0 = reinterpret_cast<uintptr_t>(Z);
  if (S != Z && s0 < z0 + bytes && z0 < s0 + bytes) return IFAC_ERR_INVALID;
  if (S != Z) {
    if (cudaMemcpyAsync(Z, S, sizeof(double) * (size_t)count * nl * nl, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return IFAC_ERR_CUDA;
  }
  double* wd = scratch;
  double* pad = pad_need ? scratch + wd_need : nullptr;
  cudaError_t e = ifac::leaf_invchol_launch_scratch(s, count, nl, Z, info, wd, pad);
  return e == cudaSuccess ? IFAC_OK : IFAC_ERR_CUDA;
}
