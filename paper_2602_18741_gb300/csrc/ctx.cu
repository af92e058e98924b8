// Context, scratch and error handling of libhsc.
#include "common.cuh"

#include <mutex>

namespace hsc {

static thread_local std::string t_last_error;

hsc_status set_error(hsc_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

hsc_status clear_error() {
  t_last_error.clear();
  return HSC_OK;
}

hsc_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(HSC_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return HSC_OK;
}

// Grows the context's large scratch to at least `bytes`.  Growing frees the
// old block after a device synchronisation, so it must not happen while a
// stream is being captured; hsc_reserve() lets callers size it up front.
hsc_status ensure_big(hsc_ctx* ctx, size_t bytes, cudaStream_t stream) {
  if (bytes <= ctx->big_bytes) return HSC_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (stream && cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return set_error(HSC_ERR_INVALID_ARG, "scratch must grow during stream capture; call hsc_reserve first");
  if (ctx->d_big) {
    HSC_CUDA(cudaDeviceSynchronize());
    HSC_CUDA(cudaFree(ctx->d_big));
    ctx->d_big = nullptr;
    ctx->big_bytes = 0;
  }
  size_t want = (bytes + 0xFFFFF) & ~size_t(0xFFFFF);
  cudaError_t e = cudaMalloc(&ctx->d_big, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->d_big = nullptr;
    return set_error(HSC_ERR_OOM, "cannot allocate %zu bytes of scratch: %s", want, cudaGetErrorString(e));
  }
  ctx->big_bytes = want;
  return HSC_OK;
}

// Launches on one stream run in order, so the last CTA of one launch resets
// the pair before the next launch on that stream reads it; launches on two
// streams may run at the same time and get two pairs.
unsigned int* stream_queue(hsc_ctx* ctx, cudaStream_t stream) {
  unsigned int* base = reinterpret_cast<unsigned int*>(ctx->d_small + HSC_OFF_QUEUE);
  void* key = reinterpret_cast<void*>(stream);
  auto it = ctx->queue_slots.find(key);
  if (it != ctx->queue_slots.end()) return base + 2 * it->second;
  const int slot = (int)ctx->queue_slots.size();
  if (slot >= HSC_QUEUE_SLOTS) return nullptr;
  ctx->queue_slots[key] = slot;
  return base + 2 * slot;
}

static_assert(HSC_OFF_QUEUE + 2u * 4u * HSC_QUEUE_SLOTS <= HSC_SMALL_SCRATCH, "tile counters outside the scratch block");

}  // namespace hsc

extern "C" {

const char* hsc_last_error(void) { return hsc::t_last_error.c_str(); }

hsc_status hsc_create(hsc_ctx** out, int device) {
  hsc::clear_error();
  HSC_REQUIRE(out != nullptr, "out is null");
  *out = nullptr;
  int count = 0;
  HSC_CUDA(cudaGetDeviceCount(&count));
  HSC_REQUIRE(device >= 0 && device < count, "device %d out of range (%d devices)", device, count);
  HSC_CUDA(cudaSetDevice(device));
  hsc_ctx* ctx = new hsc_ctx();
  ctx->device = device;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete ctx;
    return hsc::set_error(HSC_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  }
  ctx->sm_count = prop.multiProcessorCount;
  ctx->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
  if (cudaMalloc(&ctx->d_err, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_small, HSC_SMALL_SCRATCH) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return hsc::set_error(HSC_ERR_OOM, "cannot allocate context scratch");
  }
  HSC_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned int)));
  HSC_CUDA(cudaMemset(ctx->d_small, 0, HSC_SMALL_SCRATCH));
  *out = ctx;
  return HSC_OK;
}

void hsc_destroy(hsc_ctx* ctx) {
  if (!ctx) return;
  hsc::DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->d_small) cudaFree(ctx->d_small);
  if (ctx->d_big) cudaFree(ctx->d_big);
  for (auto& slot : ctx->desc_ring) {
    if (slot.h) cudaFreeHost(slot.h);
    if (slot.d) cudaFree(slot.d);
    if (slot.ev) cudaEventDestroy(slot.ev);
  }
  delete ctx;
}

hsc_status hsc_sync(hsc_ctx* ctx, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_GUARD(ctx);
  HSC_CUDA(cudaStreamSynchronize(hsc::as_stream(stream)));
  HSC_CUDA(cudaGetLastError());
  unsigned int err = 0;
  HSC_CUDA(cudaMemcpy(&err, ctx->d_err, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) {
    HSC_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned int)));
    if (err & HSC_DEVERR_TIMEOUT)
      return hsc::set_error(HSC_ERR_TIMEOUT, "a bounded device wait expired (flags 0x%x)", err);
    return hsc::set_error(HSC_ERR_DEVICE_CHECK, "device check failed (flags 0x%x)%s", err,
                          (err & HSC_DEVERR_MATERIAL) ? ": material index out of range" : "");
  }
  return HSC_OK;
}

hsc_status hsc_reserve(hsc_ctx* ctx, size_t bytes) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_GUARD(ctx);
  return hsc::ensure_big(ctx, bytes, nullptr);
}

}  // extern "C"
