// Per-channel fp8 e4m3 quantisation of an FP32 latent image.
//   scale_c = max_p z_c(p) / 448 (1 for an all-zero channel), codes RNE(z * (1/scale_c)).
// Latent values are non-negative (non-negative codec and spectra, Sec. 4.3), so
// the channel maximum is an unsigned max over the float bit patterns.
// Both kernels are HBM streams over the P x k image.
#include "common.cuh"
#include "shade_latent.cuh"

#include <mutex>

namespace hsc {

namespace {

constexpr int kQBlock = 256;

// Every thread keeps one channel: the grid stride is a multiple of k.
__global__ void __launch_bounds__(kQBlock) channel_max_kernel(const float* __restrict__ z, int64_t total, int k,
                                                              int64_t stride, unsigned int* __restrict__ out) {
  __shared__ unsigned int s_max[HSC_MAX_K];
  for (int c = threadIdx.x; c < k; c += blockDim.x) s_max[c] = 0u;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 < stride) {
    unsigned int m = 0u;
    for (int64_t i = t0; i < total; i += stride) m = max(m, __float_as_uint(fmaxf(__ldg(z + i), 0.0f)));
    if (m) atomicMax(&s_max[(int)(t0 % k)], m);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x)
    if (s_max[c]) atomicMax(out + c, s_max[c]);
}

__device__ __forceinline__ float channel_scale(unsigned int bits) {
  const float mx = __uint_as_float(bits);
  return mx > 0.0f ? __fdiv_rn(mx, 448.0f) : 1.0f;
}

__global__ void __launch_bounds__(kQBlock) quantize_kernel(const float* __restrict__ z, int64_t total, int k,
                                                           const unsigned int* __restrict__ chan_max,
                                                           uint8_t* __restrict__ codes, float* __restrict__ scales) {
  __shared__ float s_inv[HSC_MAX_K];
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const float sc = channel_scale(chan_max[c]);
    s_inv[c] = __frcp_rn(sc);
    if (blockIdx.x == 0) scales[c] = sc;
  }
  __syncthreads();
  // 4 consecutive elements per thread, one 32-bit store
  const int64_t n4 = total / 4;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 4 * q;
    const float4 v = __ldg(reinterpret_cast<const float4*>(z) + q);
    int c = (int)(i % k);
    unsigned int w = float_to_fp8_e4m3(__fmul_rn(v.x, s_inv[c]));
    c = (c + 1 == k) ? 0 : c + 1;
    w |= float_to_fp8_e4m3(__fmul_rn(v.y, s_inv[c])) << 8;
    c = (c + 1 == k) ? 0 : c + 1;
    w |= float_to_fp8_e4m3(__fmul_rn(v.z, s_inv[c])) << 16;
    c = (c + 1 == k) ? 0 : c + 1;
    w |= float_to_fp8_e4m3(__fmul_rn(v.w, s_inv[c])) << 24;
    reinterpret_cast<unsigned int*>(codes)[q] = w;
  }
  // tail (total not a multiple of 4)
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total - 4 * n4) {
    const int64_t i = 4 * n4 + t;
    codes[i] = (uint8_t)float_to_fp8_e4m3(__fmul_rn(__ldg(z + i), s_inv[(int)(i % k)]));
  }
}

int64_t grid_for(int64_t work, int sm_count) {
  int64_t g = (work + kQBlock - 1) / kQBlock;
  const int64_t cap = (int64_t)sm_count * 8;
  if (g > cap) g = cap;
  return g < 1 ? 1 : g;
}

}  // namespace

hsc_status launch_channel_max(const float* latent, int64_t P, int k, unsigned int* chan_max, int sm_count,
                              cudaStream_t s) {
  const int64_t total = P * k;
  int64_t grid = grid_for(total, sm_count);
  int64_t stride = grid * kQBlock;
  stride -= stride % k;
  if (stride < k) {  // fewer threads than channels: widen the grid
    grid = (k + kQBlock - 1) / kQBlock;
    stride = grid * kQBlock;
    stride -= stride % k;
  }
  channel_max_kernel<<<(unsigned)grid, kQBlock, 0, s>>>(latent, total, k, stride, chan_max);
  return check_launch("channel_max_kernel");
}

hsc_status launch_quantize(const float* latent, int64_t P, int k, const unsigned int* chan_max, uint8_t* codes,
                           float* scales, int sm_count, cudaStream_t s) {
  const int64_t total = P * k;
  const int64_t grid = grid_for((total + 3) / 4, sm_count);
  quantize_kernel<<<(unsigned)grid, kQBlock, 0, s>>>(latent, total, k, chan_max, codes, scales);
  return check_launch("quantize_kernel");
}

}  // namespace hsc

extern "C" hsc_status hsc_quantize_fp8(hsc_ctx* ctx, const float* latent, int64_t pixels, int k, uint8_t* codes_out,
                                       float* scales_out, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(k >= 1 && k <= HSC_MAX_K, "k=%d out of range", k);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  HSC_REQUIRE(latent && codes_out && scales_out, "null pointer");
  HSC_REQUIRE(hsc::aligned(latent, 16) && hsc::aligned(codes_out, 4) && hsc::aligned(scales_out, 4),
              "latent must be 16-byte and codes 4-byte aligned");
  HSC_GUARD(ctx);
  cudaStream_t s = hsc::as_stream(stream);
  unsigned int* chan_max = reinterpret_cast<unsigned int*>(ctx->d_small + HSC_OFF_CHANMAX);
  HSC_CUDA(cudaMemsetAsync(chan_max, 0, sizeof(unsigned int) * k, s));
  if (pixels > 0) HSC_TRY(hsc::launch_channel_max(latent, pixels, k, chan_max, ctx->sm_count, s));
  return hsc::launch_quantize(latent, pixels, k, chan_max, codes_out, scales_out, ctx->sm_count, s);
}

namespace hsc {

// ---------------------------------------------------------------------------
// Allocation-free variant of the quantiser.
//
// Some callers of this library may not allocate device memory at all: a
// plugin that runs inside a host renderer which owns the GPU's whole memory
// budget through its own allocator, or a frame loop with a hard deadline in
// which cudaMalloc (which can synchronise the whole device) is not allowed.
// Such callers cannot create an hsc_ctx either, because hsc_create allocates
// the context's scratch.  hsc_quantize_fp8_noalloc serves them: its only
// scratch, one max word per channel, is the file-scope array below.  The
// array is part of the library's device code, so every GPU on which the
// library is loaded holds its 384 bytes until the process exits.
static __device__ __align__(256) unsigned int g_noalloc_chan_max[HSC_NOALLOC_MAX_K];
// launch_channel_max stages one word per channel in a shared array of
// HSC_MAX_K words, which must hold every channel this entry point accepts
static_assert(HSC_NOALLOC_MAX_K <= HSC_MAX_K, "the channel-max kernel stages at most HSC_MAX_K channels");

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned int* g_noalloc_ptr[kMaxDevices];  // device address of g_noalloc_chan_max, per device
int g_noalloc_sms[kMaxDevices];

// One-time set-up per device, with that device current: the array's name in
// host code is only a host-side stand-in, so its device address is fetched
// with cudaGetSymbolAddress and cached.
hsc_status noalloc_setup(int dev, unsigned int** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_chan_max);
    if (e != cudaSuccess) return set_error(HSC_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    int sm = 0;
    e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(HSC_ERR_CUDA, "cudaDeviceGetAttribute failed: %s", cudaGetErrorString(e));
    g_noalloc_sms[dev] = sm > 0 ? sm : 1;
    g_noalloc_ptr[dev] = reinterpret_cast<unsigned int*>(p);
  }
  *ptr = g_noalloc_ptr[dev];
  *sms = g_noalloc_sms[dev];
  return HSC_OK;
}

}  // namespace

}  // namespace hsc

extern "C" hsc_status hsc_quantize_fp8_noalloc(const float* latent, int64_t pixels, int k, uint8_t* codes_out,
                                               float* scales_out, void* stream) {
  hsc::clear_error();
  HSC_REQUIRE(k >= 1 && k <= HSC_NOALLOC_MAX_K,
              "k=%d exceeds the allocation-free quantiser's maximum of %d channels", k, HSC_NOALLOC_MAX_K);
  HSC_REQUIRE(pixels >= 0, "negative pixel count");
  HSC_REQUIRE(latent && codes_out && scales_out, "null pointer");
  HSC_REQUIRE(hsc::aligned(latent, 16) && hsc::aligned(codes_out, 4) && hsc::aligned(scales_out, 4),
              "latent must be 16-byte and codes 4-byte aligned");
  int dev = 0;
  HSC_CUDA(cudaGetDevice(&dev));
  HSC_REQUIRE(dev >= 0 && dev < hsc::kMaxDevices, "device %d beyond the supported %d", dev, hsc::kMaxDevices);
  unsigned int* chan_max = nullptr;
  int sms = 1;
  HSC_TRY(hsc::noalloc_setup(dev, &chan_max, &sms));
  cudaStream_t s = hsc::as_stream(stream);
  // the array keeps the previous call's maxima: clear the channels used here
  HSC_CUDA(cudaMemsetAsync(chan_max, 0, sizeof(unsigned int) * k, s));
  if (pixels > 0) HSC_TRY(hsc::launch_channel_max(latent, pixels, k, chan_max, sms, s));
  return hsc::launch_quantize(latent, pixels, k, chan_max, codes_out, scales_out, sms, s);
}
