// pa_noalloc.cu -- log compression that allocates no memory at all.
//
// The plan-based path (pa_beamform) keeps the per-image envelope maxima that
// log compression divides by in scratch memory the plan allocated with
// cudaMalloc.  Some callers cannot allocate device memory once they are
// running: a scanner's real-time acquisition loop that must never stall
// (cudaMalloc can synchronise the whole device), a host framework that owns
// every device allocation and hands the beamformer fixed buffers, or code
// that has already frozen its memory footprint before streaming starts.
// pa_log_compress_noalloc serves them: the maxima live in a fixed,
// file-scope device array that exists as soon as this library is loaded on
// a device, so the call needs only the caller's input and output buffers.
#include <mutex>

#include <cudaTypedefs.h>

#include "pa_internal.cuh"
#include "pa_logdb.cuh"

namespace {

// Scratch for the per-image maxima (float bits of non-negative values).
// Every GPU that loads this library holds these 16 KiB until the process
// exits.
static __device__ __align__(256) int g_noalloc_max[PA_NOALLOC_MAX_IMAGES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Device address of the array, per device, with the context it was looked up
// in: a context created later on the same device (after cudaDeviceReset, or
// one the caller made current) loads the library's module afresh, so the
// address is looked up again there.
int* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The current driver context (cuCtxGetCurrent, reached through the runtime
// so that the library needs no link against the driver); null if unknown.
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Largest value of each image (negative inputs count as zero).
__global__ void k_noalloc_image_max(const float* env, long long elems, int* slots) {
  const int img = blockIdx.y;
  const float* src = env + (size_t)img * elems;
  float mx = 0.f;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < elems;
       q += (long long)gridDim.x * blockDim.x)
    mx = fmaxf(mx, src[q]);
  for (int s = 16; s >= 1; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(slots + img, __float_as_int(mx));
}

// 20 log10(env / image max), clipped to [-dr, 0]; -dr where env or max is 0.
__global__ void k_noalloc_log(const float* env, float* out, long long elems, const int* slots,
                              float dr) {
  const int img = blockIdx.y;
  const float mx = __int_as_float(slots[img]);
  const float inv = mx > 0.f ? 1.0f / mx : 0.f;
  const float* src = env + (size_t)img * elems;
  float* dst = out + (size_t)img * elems;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < elems;
       q += (long long)gridDim.x * blockDim.x) {
    dst[q] = pa::log_db(src[q], mx, inv, dr);
  }
}

pa_status noalloc_fail(pa_status s, const char* msg) {
  pa::set_error_message(msg);  // readable through pa_last_error()
  return s;
}

}  // namespace

extern "C" pa_status pa_log_compress_noalloc(const float* env_dev, int32_t n_images,
                                             int64_t image_elems, float dyn_range_db,
                                             float* log_dev, void* cuda_stream) {
  if (n_images < 0 || image_elems < 0)
    return noalloc_fail(PA_EINVAL, "pa_log_compress_noalloc: negative size");
  if (n_images > PA_NOALLOC_MAX_IMAGES)
    return noalloc_fail(PA_EINVAL,
                        "pa_log_compress_noalloc: more images than the static scratch holds "
                        "(PA_NOALLOC_MAX_IMAGES)");
  if (n_images == 0 || image_elems == 0) return PA_OK;
  if (!env_dev || !log_dev) return noalloc_fail(PA_EINVAL, "pa_log_compress_noalloc: null buffer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(PA_ECUDA, "pa_log_compress_noalloc: no current CUDA device");
  int* slots = nullptr;
  {
    // One-time set-up per device (and context): the host-side name of the
    // array is not a device address, so ask the runtime for the address on
    // this device, with the device current.
    std::lock_guard<std::mutex> lk(g_mu);
    const CUcontext ctx = current_context();
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_max);
      if (e != cudaSuccess || !p)
        return noalloc_fail(PA_ECUDA, "pa_log_compress_noalloc: cudaGetSymbolAddress failed");
      g_scratch_addr[dev] = static_cast<int*>(p);
      g_scratch_ctx[dev] = current_context();  // the lookup may have created it
    }
    slots = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // as in pa_plan_desc: a range that is not positive (or NaN) means 60 dB
  const float dr = dyn_range_db > 0.f ? dyn_range_db : 60.f;
  // The array keeps the previous call's maxima: clear the slots this call uses.
  if (cudaMemsetAsync(slots, 0, (size_t)n_images * sizeof(int), st) != cudaSuccess)
    return noalloc_fail(PA_ECUDA, "pa_log_compress_noalloc: clearing the scratch failed");
  long long per_img = (image_elems + 255) / 256;
  if (per_img > 1024) per_img = 1024;
  dim3 grid((unsigned)per_img, (unsigned)n_images);
  k_noalloc_image_max<<<grid, 256, 0, st>>>(env_dev, image_elems, slots);
  k_noalloc_log<<<grid, 256, 0, st>>>(env_dev, log_dev, image_elems, slots, dr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(PA_ECUDA, cudaGetErrorString(e));
  return PA_OK;
}
