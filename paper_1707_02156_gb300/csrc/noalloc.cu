// Allocation-free variant of the SH rotation entry point.
//
// bie_rotate stages each drop's rotation tables (the real Wigner blocks, the e^{i m alpha}
// phases and the per-component offsets) in device buffers it allocates and frees on every
// call.  Some callers cannot allow that: code that owns the device's memory through its own
// pool or arena and forbids foreign allocations, and latency-critical loops that must not hit
// the allocator or its implicit synchronisation.  bie_rotate_noalloc does the same rotation
// with those tables staged in one fixed array that lives in the library's device image
// (below), so it never allocates or frees device memory; the host side builds the tables in a
// fixed host buffer, so it does not allocate host memory either.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "tables.h"

namespace bie {
namespace {

// Staging area for one drop's tables: Wigner blocks (at most wigner_block_stride(BIE_NOALLOC_MAX_P)
// doubles), then 2(p+1) phases, then ncomp offsets stored as doubles' worth of bytes.
// Every GPU that loads the library holds this array until the process exits.
constexpr long long kScratchDoubles = BIE_NOALLOC_SCRATCH_DOUBLES;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};

// Host staging buffer of the same size, guarded by g_mu for the whole call: cudaMemcpyAsync from
// pageable host memory has copied the source out before it returns, so the next drop may
// overwrite it.
static double g_host_stage[kScratchDoubles];

// Makes `device` current for the guard's lifetime and restores the caller's current device.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int device) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != device) err = cudaSetDevice(device);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Device address of the staging array on the current device (looked up once per device).
int scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("bie_rotate_noalloc: device ordinal out of range");
    return BIE_EINVAL;
  }
  if (!g_dev_ptr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error(std::string("bie_rotate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return BIE_ECUDA;
    }
    g_dev_ptr[device] = static_cast<double*>(ptr);
  }
  *out = g_dev_ptr[device];
  return BIE_OK;
}

}  // namespace
}  // namespace bie

using namespace bie;

extern "C" int bie_rotate_noalloc(bie_ctx* ctx, int ndrop, const int* p, int ncomp, const double* coef,
                                  const double* euler, double* coef_out, void* stream) {
  if (!ctx || !coef || !coef_out || !euler || !p || ndrop <= 0 || ncomp <= 0) {
    set_error("bie_rotate_noalloc: null or empty argument");
    return BIE_EINVAL;
  }
  // sizes: every drop's tables must fit the staging array
  for (int d = 0; d < ndrop; ++d) {
    if (p[d] < 1 || p[d] > BIE_NOALLOC_MAX_P) {
      set_error("bie_rotate_noalloc: degree must satisfy 1 <= p <= BIE_NOALLOC_MAX_P (" +
                std::to_string(BIE_NOALLOC_MAX_P) + ")");
      return BIE_EINVAL;
    }
    const long long need = wigner_block_stride(p[d]) + 2LL * (p[d] + 1) + ncomp;
    if (need > kScratchDoubles) {
      set_error("bie_rotate_noalloc: tables of " + std::to_string(need) + " doubles exceed the staging array of " +
                std::to_string(kScratchDoubles) + " doubles (reduce ncomp)");
      return BIE_EINVAL;
    }
  }
  const int device = ctx_device(ctx);
  DeviceGuard guard(device);
  if (guard.err != cudaSuccess) {
    set_error(std::string("bie_rotate_noalloc: selecting the device: ") + cudaGetErrorString(guard.err));
    return BIE_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  double* scratch = nullptr;
  BIE_TRY(scratch_address(device, &scratch));
  cudaStream_t s = (cudaStream_t)stream;
  long long co = 0;
  double* host = g_host_stage;
  for (int d = 0; d < ndrop; ++d) {
    const int pd = p[d];
    const long long stride = wigner_block_stride(pd);
    const long long len = stride + 2 * (pd + 1) + ncomp;
    std::memset(host, 0, len * sizeof(double));
    wigner_blocks(pd, euler[3 * d + 1], host);
    double* ph = host + stride;
    for (int m = 0; m <= pd; ++m) {
      ph[2 * m] = std::cos(m * euler[3 * d]);
      ph[2 * m + 1] = std::sin(m * euler[3 * d]);
    }
    long long* foff = reinterpret_cast<long long*>(ph + 2 * (pd + 1));
    for (int c = 0; c < ncomp; ++c) foff[c] = co + c * (long long)(pd + 1) * (pd + 1);
    // the copy is stream-ordered after the previous drop's kernel, which read the same array
    BIE_CUDA_TRY(cudaMemcpyAsync(scratch, host, len * sizeof(double), cudaMemcpyHostToDevice, s));
    const double* dblk = scratch;
    const double* dph = scratch + stride;
    const long long* dfo = reinterpret_cast<const long long*>(scratch + stride + 2 * (pd + 1));
    BIE_TRY((launch_rotate<double, double>(coef, dfo, ncomp, 1, pd, dblk, stride, 1, 1, dph, coef_out + co, 0, s)));
    BIE_TRY(launch_phase(coef_out + co, ncomp, pd, euler[3 * d + 2], s));
    co += ncomp * (long long)(pd + 1) * (pd + 1);
  }
  return BIE_OK;
}
