// wd_norm2_noalloc: the FP64 squared norm of one single-parity field, for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// wanted -- for instance a host framework that owns all device memory
// through its own pool and forbids other allocations on its hot path, or a
// caller that is about to capture work into a CUDA graph -- and that
// therefore cannot create a wd_ctx (wd_create allocates the reduction
// scratch, staging and workspace).  This entry point takes only the caller's
// input field and output location and allocates nothing.
//
// The reduction needs scratch memory beyond its input and output: one FP64
// partial sum per block and a ticket counter that picks the last block.  Here
// that scratch is a file-scope static __device__ array, so every GPU that
// loads the library holds it (kScratchBytes, about 512 KB) until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call in each CUDA context looks the address up with
// cudaGetSymbolAddress (with that context current) and caches it under the
// context's unique id; make that first call before any stream capture.  The
// address belongs to the context, not to the device: a driver-API caller with
// its own context, or a caller that reset the device (which ends the primary
// context), gets a fresh lookup in the new context.  Every call shares the
// array: the counter is cleared on the stream before each launch, and calls
// that overlap on the GPU (different streams, or different host threads at
// once) race on it.
#include <cuda.h>

#include <mutex>
#include <unordered_map>

#include "wd_kernels.cuh"

namespace wd {
namespace {

constexpr int kNoallocBlock = 256;
constexpr int kMaxPartials = 65536;  // one per block: Vh <= 65536 * 256 = 16,777,216 sites
constexpr size_t kCounterOffset = (size_t)kMaxPartials * sizeof(double);
constexpr size_t kScratchBytes = kCounterOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
std::unordered_map<unsigned long long, void*> g_scratch_addr;  // context id -> address

void put_err(char* err, size_t len, const char* msg) {
  if (!err || len == 0) return;
  size_t i = 0;
  for (; i + 1 < len && msg[i]; ++i) err[i] = msg[i];
  err[i] = 0;
}

// The current context's unique id, through the driver entry points that the
// runtime hands out (no link against the driver library).  0 when no context
// is current yet.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorNotSupported;
    get_current = (CtxGetCurrentFn)f1;
    get_id = (CtxGetIdFn)f2;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Once per context, with that context current: the device address of the
// array.  The runtime binds the device's primary context on its first call
// when none is current, so the id is read again after the lookup.
cudaError_t scratch_address(void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long id = 0;
  cudaError_t e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  if (id) {
    auto it = g_scratch_addr.find(id);
    if (it != g_scratch_addr.end()) {
      *out = it->second;
      return cudaSuccess;
    }
  }
  void* p = nullptr;
  if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
  if ((e = current_context_id(&id)) != cudaSuccess) return e;
  if (!id) return cudaErrorDeviceUninitialized;
  g_scratch_addr[id] = p;
  *out = p;
  return cudaSuccess;
}

template <int P>
void launch_norm2(const Geom& g, const void* field, double* result, void* scratch, cudaStream_t s) {
  using T = Tr<P>;
  RedScratch rs{(double*)scratch, (unsigned*)((char*)scratch + kCounterOffset)};
  OpNorm2<typename T::S> op{T::view(field, g), rs, FinStore{result, 1}};
  const int grid = (g.Vh + kNoallocBlock - 1) / kNoallocBlock;  // one site per thread
  site_kernel<OpNorm2<typename T::S>><<<grid, kNoallocBlock, 0, s>>>(g.Vh, op);
}

}  // namespace
}  // namespace wd

extern "C" wd_status wd_norm2_noalloc(double* result, const void* field, const int dims[4], wd_prec prec,
                                      void* cuda_stream, char* err, size_t err_len) {
  using namespace wd;
  put_err(err, err_len, "");
  if (!result || !field || !dims || prec < WD_F64 || prec > WD_B16N) {
    put_err(err, err_len, "wd_norm2_noalloc: null pointer or bad precision");
    return WD_ERR_INVALID_ARG;
  }
  long long v = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 2 || (dims[m] & 1)) {
      put_err(err, err_len, "wd_norm2_noalloc: every dimension must be even and >= 2");
      return WD_ERR_INVALID_ARG;
    }
    v *= dims[m];
  }
  const long long vh = v / 2;
  if (vh > (long long)kMaxPartials * kNoallocBlock) {
    put_err(err, err_len,
            "wd_norm2_noalloc: field too large for the static scratch (at most 16777216 sites per parity, "
            "65536 partial sums)");
    return WD_ERR_INVALID_ARG;
  }
  const Geom g = make_geom(dims, 0);
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    put_err(err, err_len, "wd_norm2_noalloc: no usable current context, or cudaGetSymbolAddress of the static "
                          "scratch failed");
    return WD_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the ticket counter must start at zero
  if ((e = cudaMemsetAsync((char*)scratch + kCounterOffset, 0, sizeof(unsigned), s)) != cudaSuccess) {
    put_err(err, err_len, "wd_norm2_noalloc: clearing the counter failed");
    return WD_ERR_CUDA;
  }
  switch (prec) {
    case WD_F64: launch_norm2<WD_F64>(g, field, result, scratch, s); break;
    case WD_F32: launch_norm2<WD_F32>(g, field, result, scratch, s); break;
    case WD_Q16: launch_norm2<WD_Q16>(g, field, result, scratch, s); break;
    case WD_H16N: launch_norm2<WD_H16N>(g, field, result, scratch, s); break;
    case WD_B16N: launch_norm2<WD_B16N>(g, field, result, scratch, s); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) {
    put_err(err, err_len, "wd_norm2_noalloc: kernel launch failed");
    return WD_ERR_CUDA;
  }
  return WD_OK;
}
