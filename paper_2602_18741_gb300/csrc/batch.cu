// Batched latent shading of many frames of uneven size in one persistent
// launch, replayed as a CUDA graph.
//
// Each frame brings its own G-buffer, codes (its own codec), lights, k and
// folded decode matrix.  The frames' pixel tiles form one global tile space;
// persistent CTAs take tiles from an atomic queue (frames differ 64x in light
// count, so a static split would leave SMs idle), locate the frame by binary
// search over the frames' first tiles, stage that frame's lights in shared
// memory when the frame changes, and run the same shade_tile code as the
// single-frame launch -- so every frame's output is bit-identical to shading
// it alone.  XYZ is decoded in the epilogue with the frame's M = T D.
#include "common.cuh"
#include "shade_latent.cuh"
#include "shade_latent_kernel.cuh"
#include "tune.cuh"

#include <vector>

namespace hsc {

namespace {

struct FrameDesc {
  ShadeArgs a;
  int64_t tile0;  // first global tile of the frame
  int sec;
};

struct BatchArgs {
  const FrameDesc* frames;
  int count;
  int64_t total_tiles;
  unsigned int* queue;  // tile counter, zeroed before every launch
};

__device__ __forceinline__ int find_frame(const BatchArgs& b, int64_t tile) {
  int lo = 0, hi = b.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&b.frames[mid].tile0) <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Paired (f32x2) points need an even point count: a direct-only frame with
// one pixel per thread falls back to the scalar form (same results).
template <int KC, bool SEC, int PPT, int BLOCK, int VEC>
__device__ __forceinline__ void run_tile(const ShadeArgs& a, int64_t local_tile, float4* s_light, float* s_M,
                                         bool restage, bool staged) {
  constexpr int V = (VEC == 2 && !SEC && PPT == 1) ? 1 : VEC;
  if (restage) {
    __syncthreads();
    if (staged) restage_light_codes<KC, V, BLOCK>(a, s_light, 0, a.L);
    stage_decode_matrix<KC, BLOCK>(a, s_M);
    __syncthreads();
  }
  shade_tile<KC, PPT, SEC, BLOCK, V>(a, local_tile, s_light, staged, s_M);
}

template <int PPT, int BLOCK, int VEC>
__global__ void __launch_bounds__(BLOCK) shade_batch_kernel(const BatchArgs b) {
  extern __shared__ float4 s_light[];
  __shared__ int64_t s_tile;
  __shared__ float s_M[3 * 9];
  int staged_frame = -1;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(b.queue, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile >= b.total_tiles) break;
    const int f = find_frame(b, tile);
    const FrameDesc& fd = b.frames[f];
    const ShadeArgs a = fd.a;
    const bool restage = f != staged_frame;
    staged_frame = f;
    const bool staged = a.L <= kLightTile;
    const int64_t local = tile - fd.tile0;
    if (a.k == 6) {
      if (fd.sec) run_tile<6, true, PPT, BLOCK, VEC>(a, local, s_light, s_M, restage, staged);
      else run_tile<6, false, PPT, BLOCK, VEC>(a, local, s_light, s_M, restage, staged);
    } else {
      if (fd.sec) run_tile<9, true, PPT, BLOCK, VEC>(a, local, s_light, s_M, restage, staged);
      else run_tile<9, false, PPT, BLOCK, VEC>(a, local, s_light, s_M, restage, staged);
    }
    if (!staged) staged_frame = -1;  // the light tiles were streamed; restage next time
  }
}

template <int PPT, int BLOCK, int VEC>
hsc_status launch_batch(const BatchArgs& b, int sm_count, cudaStream_t s) {
  auto kern = shade_batch_kernel<PPT, BLOCK, VEC>;
  const size_t smem = (size_t)kLightTile * LightStage<9, VEC>::F4 * sizeof(float4);
  static int occ = -1;
  if (occ < 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, BLOCK, smem) != cudaSuccess) o = 1;
    occ = o > 0 ? o : 1;
  }
  int64_t grid = (int64_t)sm_count * occ;
  if (grid > b.total_tiles) grid = b.total_tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, BLOCK, smem, s>>>(b);
  return check_launch("shade_batch_kernel");
}

hsc_status launch_batch_cfg(const BatchArgs& b, const LaunchCfg& c, cudaStream_t s) {
  if (c.vec == 2) {
    if (c.block == 256)
      return c.ppt == 1 ? launch_batch<1, 256, 2>(b, c.sm_count, s) : launch_batch<2, 256, 2>(b, c.sm_count, s);
    return c.ppt == 1 ? launch_batch<1, 128, 2>(b, c.sm_count, s) : launch_batch<2, 128, 2>(b, c.sm_count, s);
  }
  if (c.block == 256)
    return c.ppt == 1 ? launch_batch<1, 256, 1>(b, c.sm_count, s) : launch_batch<2, 256, 1>(b, c.sm_count, s);
  return c.ppt == 1 ? launch_batch<1, 128, 1>(b, c.sm_count, s) : launch_batch<2, 128, 1>(b, c.sm_count, s);
}

}  // namespace

hsc_status validate_gbuffer(const hsc_gbuffer* g, const char* name, int64_t pixels);
hsc_status validate_lights(const hsc_lights* l);

// Fills the device descriptors of `count` frames for tiles of c.block * c.ppt
// pixels; returns the total tile count.
static int64_t build_frame_descs(hsc_ctx* ctx, const hsc_frame* frames, int count, const LaunchCfg& c, FrameDesc* h) {
  int64_t tile0 = 0;
  const int64_t tile_px = (int64_t)c.block * c.ppt;
  for (int i = 0; i < count; ++i) {
    const hsc_frame& f = frames[i];
    ShadeArgs a{};
    a.n1 = f.g1.normal;
    a.x1 = f.g1.pos;
    a.m1 = f.g1.mat;
    if (f.has_g2) {
      a.n2 = f.g2.normal;
      a.x2 = f.g2.pos;
      a.m2 = f.g2.mat;
    }
    a.P = f.pixels;
    a.mat_codes = f.mat_codes;
    a.n_mat = f.n_mat;
    a.lpos = f.lights.pos;
    a.linten = f.lights.intensity;
    a.L = f.lights.count;
    a.light_codes = f.light_codes;
    a.code_dt = (int)f.code_dt;
    a.k = f.k;
    a.c0 = 0;
    a.out = f.latent_out;
    a.out_stride = f.k;
    a.out_c0 = 0;
    a.xyz = f.xyz_out;
    a.M = f.M_xyz;
    a.chan_max = nullptr;
    a.err = ctx->d_err;
    a.tiles = (f.pixels + tile_px - 1) / tile_px;
    h[i].a = a;
    h[i].tile0 = tile0;
    h[i].sec = f.has_g2 ? 1 : 0;
    tile0 += a.tiles;
  }
  return tile0;
}

static hsc_status validate_frames(const hsc_frame* frames, int count) {
  HSC_REQUIRE(frames != nullptr && count >= 1, "need at least one frame");
  for (int i = 0; i < count; ++i) {
    const hsc_frame& f = frames[i];
    HSC_REQUIRE(f.k == 6 || f.k == 9, "frame %d: the batched launch supports k = 6 and 9 (got %d)", i, f.k);
    HSC_REQUIRE(f.pixels >= 1, "frame %d: empty frame", i);
    HSC_REQUIRE(f.code_dt == HSC_F32 || f.code_dt == HSC_BF16 || f.code_dt == HSC_F16, "frame %d: bad code dtype", i);
    HSC_REQUIRE(f.mat_codes && f.light_codes && f.M_xyz && f.xyz_out, "frame %d: null pointer", i);
    HSC_REQUIRE(f.n_mat >= 1 && f.n_mat <= HSC_MAX_MAT, "frame %d: n_mat out of range", i);
    HSC_REQUIRE(!f.latent_out || aligned(f.latent_out, 4), "frame %d: latent_out misaligned", i);
    HSC_TRY(validate_gbuffer(&f.g1, "g1", f.pixels));
    if (f.has_g2) HSC_TRY(validate_gbuffer(&f.g2, "g2", f.pixels));
    HSC_TRY(validate_lights(&f.lights));
  }
  return HSC_OK;
}

}  // namespace hsc

struct hsc_batch {
  hsc_ctx* ctx = nullptr;
  hsc::FrameDesc* d_frames = nullptr;
  unsigned int* d_queue = nullptr;
  int count = 0;
  int64_t total_tiles = 0;
  hsc::LaunchCfg cfg;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string report;
};

static void batch_free(hsc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_frames) cudaFree(b->d_frames);
  if (b->d_queue) cudaFree(b->d_queue);
  delete b;
}

extern "C" {

hsc_status hsc_batch_create(hsc_ctx* ctx, const hsc_frame* frames, int count, hsc_batch** out) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(out != nullptr, "out is null");
  *out = nullptr;
  HSC_TRY(hsc::validate_frames(frames, count));
  HSC_GUARD(ctx);
  hsc_batch* b = new hsc_batch();
  b->ctx = ctx;
  b->count = count;
  // Configuration candidates: the tile shape changes the global tile space,
  // so descriptors are rebuilt per candidate.
  std::vector<hsc::LaunchCfg> cands;
  for (int vec : {1, 2})
    for (int ppt : {1, 2})
      for (int block : {128, 256}) {
        hsc::LaunchCfg c;
        c.sm_count = ctx->sm_count;
        c.ppt = ppt;
        c.block = block;
        c.vec = vec;
        c.waves = 1;
        cands.push_back(c);
      }
  if (ctx->forced.ppt > 0) {
    hsc::LaunchCfg c = ctx->forced;
    c.sm_count = ctx->sm_count;
    if (c.ppt > 2) c.ppt = 2;
    cands.assign(1, c);
  } else if (!ctx->autotune) {
    cands.resize(1);  // default: ppt 1, 128 threads, scalar
  }
  std::vector<hsc::FrameDesc> h(count);
  auto build_desc = [&](const hsc::LaunchCfg& c) -> int64_t { return hsc::build_frame_descs(ctx, frames, count, c, h.data()); };
  cudaError_t e = cudaMalloc(&b->d_frames, sizeof(hsc::FrameDesc) * count);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(unsigned int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    return hsc::set_error(HSC_ERR_OOM, "batch descriptors: %s", cudaGetErrorString(e));
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hsc_status status = HSC_OK;
  float best = 1e30f;
  hsc::LaunchCfg best_cfg = cands[0];
  char line[256];
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    status = hsc::set_error(HSC_ERR_CUDA, "batch set-up: stream/event creation failed");
  }
  for (size_t ci = 0; status == HSC_OK && ci < cands.size(); ++ci) {
    const hsc::LaunchCfg& c = cands[ci];
    const int64_t total = build_desc(c);
    if (total >= (int64_t)0xFFFFFFF0ll) {
      status = hsc::set_error(HSC_ERR_INVALID_ARG, "batch has too many pixel tiles");
      break;
    }
    if (cudaMemcpy(b->d_frames, h.data(), sizeof(hsc::FrameDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
      status = hsc::set_error(HSC_ERR_CUDA, "batch descriptor upload failed");
      break;
    }
    hsc::BatchArgs ba{b->d_frames, count, total, b->d_queue};
    if (cands.size() == 1) {
      best_cfg = c;
      break;
    }
    float ms = 0.0f;
    for (int rep = 0; rep < 4 && status == HSC_OK; ++rep) {
      if (rep == 1) cudaEventRecord(e0, st);
      cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), st);
      status = hsc::launch_batch_cfg(ba, c, st);
    }
    if (status != HSC_OK) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      status = hsc::set_error(HSC_ERR_CUDA, "batch tuning failed");
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= 3.0f;
    snprintf(line, sizeof(line), " [ppt=%d block=%d vec=%d %.4f ms]", c.ppt, c.block, c.vec, ms);
    b->report += line;
    if (ms < best) {
      best = ms;
      best_cfg = c;
    }
  }
  if (status == HSC_OK) {
    // final descriptors for the chosen configuration, then the graph:
    // queue reset + one persistent kernel
    b->cfg = best_cfg;
    b->total_tiles = build_desc(best_cfg);
    if (cudaMemcpy(b->d_frames, h.data(), sizeof(hsc::FrameDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess)
      status = hsc::set_error(HSC_ERR_CUDA, "batch descriptor upload failed");
  }
  if (status == HSC_OK) {
    hsc::BatchArgs ba{b->d_frames, count, b->total_tiles, b->d_queue};
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      status = hsc::set_error(HSC_ERR_CUDA, "batch graph capture could not start");
    } else {
      cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), st);
      hsc_status ls = hsc::launch_batch_cfg(ba, best_cfg, st);
      cudaError_t ce = cudaStreamEndCapture(st, &g);
      if (ls != HSC_OK) status = ls;
      else if (ce != cudaSuccess) status = hsc::set_error(HSC_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(ce));
      else if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) status = hsc::set_error(HSC_ERR_CUDA, "graph instantiate failed");
      b->graph = g;
    }
  }
  snprintf(line, sizeof(line), " -> ppt=%d block=%d vec=%d, %lld tiles\n", b->cfg.ppt, b->cfg.block, b->cfg.vec,
           (long long)b->total_tiles);
  b->report = "batch of " + std::to_string(count) + " frames:" + b->report + line;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (status != HSC_OK) {
    batch_free(b);
    return status;
  }
  ctx->tune_report += b->report;
  *out = b;
  return HSC_OK;
}

hsc_status hsc_batch_shade(hsc_ctx* ctx, hsc_batch* batch, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(batch != nullptr && batch->exec != nullptr, "null batch");
  HSC_REQUIRE(batch->ctx == ctx, "batch belongs to another context");
  HSC_GUARD(ctx);
  HSC_CUDA(cudaGraphLaunch(batch->exec, hsc::as_stream(stream)));
  return HSC_OK;
}

hsc_status hsc_shade_frames(hsc_ctx* ctx, const hsc_frame* frames, int count, void* stream) {
  hsc::clear_error();
  HSC_CHECK_CTX(ctx);
  HSC_REQUIRE(count >= 0 && count <= HSC_MAX_FRAMES_PER_CALL, "0 to %d frames per call", HSC_MAX_FRAMES_PER_CALL);
  if (count > 0) HSC_TRY(hsc::validate_frames(frames, count));
  HSC_GUARD(ctx);
  cudaStream_t s = hsc::as_stream(stream);
  // the whole descriptor ring is allocated by the first call (pinned host
  // memory and device memory: allocations that can wait for the device)
  if (!ctx->desc_ring[0].h) {
    for (int i = 0; i < hsc_ctx::kDescSlots; ++i) {
      hsc_ctx::DescSlot& sl = ctx->desc_ring[i];
      if (cudaMallocHost(&sl.h, sizeof(hsc::FrameDesc) * HSC_MAX_FRAMES_PER_CALL) != cudaSuccess ||
          cudaMalloc(&sl.d, sizeof(hsc::FrameDesc) * HSC_MAX_FRAMES_PER_CALL + 256) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(sl.ev, s) != cudaSuccess) {
        cudaGetLastError();
        return hsc::set_error(HSC_ERR_OOM, "cannot allocate the frame descriptor ring");
      }
    }
  }
  if (count == 0) return HSC_OK;
  // descriptor ring: a slot is reused only after its previous launch has
  // consumed the descriptors (its event), so host writes never race a copy.
  // Launches on different streams finish out of order, so take the first
  // slot whose launch is done and wait only when every slot is busy.
  int pick = -1;
  for (int i = 0; i < hsc_ctx::kDescSlots && pick < 0; ++i) {
    const int j = (ctx->desc_next + i) % hsc_ctx::kDescSlots;
    const cudaError_t q = cudaEventQuery(ctx->desc_ring[j].ev);
    if (q == cudaSuccess) pick = j;
    else if (q != cudaErrorNotReady) HSC_CUDA(q);
  }
  if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();  // a query's "not ready" is no error
  if (pick < 0) pick = ctx->desc_next;
  ctx->desc_next = (pick + 1) % hsc_ctx::kDescSlots;
  hsc_ctx::DescSlot& slot = ctx->desc_ring[pick];
  HSC_CUDA(cudaEventSynchronize(slot.ev));
  hsc::LaunchCfg c;
  c.sm_count = ctx->sm_count;
  c.ppt = 2;
  c.block = 128;
  c.vec = 1;
  if (ctx->forced.ppt > 0) {
    c = ctx->forced;
    c.sm_count = ctx->sm_count;
    if (c.ppt > 2) c.ppt = 2;
  }
  hsc::FrameDesc* h = reinterpret_cast<hsc::FrameDesc*>(slot.h);
  hsc::FrameDesc* d = reinterpret_cast<hsc::FrameDesc*>(slot.d);
  unsigned int* queue = reinterpret_cast<unsigned int*>(reinterpret_cast<unsigned char*>(slot.d) +
                                                        sizeof(hsc::FrameDesc) * HSC_MAX_FRAMES_PER_CALL);
  const int64_t total = hsc::build_frame_descs(ctx, frames, count, c, h);
  HSC_REQUIRE(total < (int64_t)0xFFFFFFF0ll, "too many pixel tiles in one call");
  HSC_CUDA(cudaMemcpyAsync(d, h, sizeof(hsc::FrameDesc) * count, cudaMemcpyHostToDevice, s));
  HSC_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned int), s));
  hsc::BatchArgs ba{d, count, total, queue};
  HSC_TRY(hsc::launch_batch_cfg(ba, c, s));
  HSC_CUDA(cudaEventRecord(slot.ev, s));
  return HSC_OK;
}

void hsc_batch_destroy(hsc_batch* batch) {
  if (!batch) return;
  hsc::DeviceGuard g(batch->ctx->device);
  cudaDeviceSynchronize();
  batch_free(batch);
}

}  // extern "C"
