// Many concurrent trackers on one GPU: the serving and batching form of the per-frame
// update (Alg. 3 with one coil, then the line draw of Alg. 4 for the next frame).
//
// Every stream (a cine slice with its own Nx, Ny, R, lambda_forget, mu, K, rate) is a
// tracker handle whose device state lives in one slot of a device arena that the engine
// reserves once; admission asks the arena for the stream's footprint and is refused when
// it has no room. One engine step takes one frame for each of a set of slots and runs
//   (1) all their MM iterations in one persistent launch: clusters of C CTAs pull frames
//       from a queue ordered largest first, each frame staying on one cluster;
//   (2) all their images X_t = A diag(gamma) B^T in one launch over the union of tiles;
//   (3) all their next-frame line draws in one launch, one CTA per stream;
// with the parameters of the step in one block copied from pinned host memory. The four
// operations are captured once in a CUDA graph and replayed; the kernels read the step's
// counts from the parameter block, so one graph serves any subset of the slots.
// Each stream's arithmetic is exactly that of its handle run alone (same cluster size,
// same chunking), so its results do not depend on what else is in the step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "tts_handle.cuh"

namespace {

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

struct BlockHeader {
  int queue;        // frame queue counter (0 at launch)
  int n_frames;
  int n_samplers;
  int n_images;
  int pad[60];
};
static_assert(sizeof(BlockHeader) == 256, "parameter block header is 256 bytes");

#define ECK(call)                                               \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return tts_cuda_fail(e_, #call);     \
  } while (0)

}  // namespace

struct tts_engine {
  int dev = 0;
  cudaStream_t stream = nullptr;   // every step and every slot's work
  cudaStream_t admin = nullptr;    // initialisation of newly admitted slots
  bool own_stream = false;
  int C = 8;
  int max_slots = 0;
  bool use_graph = true;
  int sms = 0;
  // device arena: slot memory, first fit, freed blocks coalesced
  char* arena = nullptr;
  size_t arena_bytes = 0, used = 0;
  std::map<size_t, size_t> free_blocks;   // offset -> bytes
  std::vector<tts_handle*> slot;
  std::vector<size_t> slot_off, slot_len;
  int active = 0;
  // parameter block: header | FrameParams[max] | SamplerJob[max] | ImageJob[max]
  size_t off_frames = 0, off_samplers = 0, off_images = 0, block_bytes = 0;
  char* d_block = nullptr;
  char* h_block[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool pending[2] = {false, false};
  int cur = 0;
  // launch shape of the persistent frame kernel
  int own = 0, frame_smem = 0, frame_clusters = 0, image_grid = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int graph_own[2] = {0, 0};
  int64_t steps = 0;
};

namespace {

bool arena_take(tts_engine* e, size_t bytes, size_t* off) {
  for (auto it = e->free_blocks.begin(); it != e->free_blocks.end(); ++it) {
    if (it->second < bytes) continue;
    *off = it->first;
    const size_t rest = it->second - bytes;
    const size_t roff = it->first + bytes;
    e->free_blocks.erase(it);
    if (rest) e->free_blocks[roff] = rest;
    e->used += bytes;
    return true;
  }
  return false;
}

void arena_give(tts_engine* e, size_t off, size_t bytes) {
  e->used -= bytes;
  auto it = e->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != e->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    e->free_blocks.erase(nx);
  }
  if (it != e->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      e->free_blocks.erase(it);
    }
  }
}

// OWN of the persistent launch: the largest that any admitted slot needs.
int refresh_shape(tts_engine* e) {
  int own = 1;
  for (tts_handle* h : e->slot)
    if (h) own = std::max(own, frame_own(h->fp));
  if (own == e->own && e->frame_clusters > 0) return TTS_OK;
  int dyn = 0, clusters = 0;
  const int rc = frame_batch_limits(own, e->C, &dyn, &clusters);
  if (rc != TTS_OK) return tts_fail(rc, "cannot size the persistent frame launch%s");
  e->own = own;
  e->frame_smem = dyn;
  e->frame_clusters = clusters;
  return TTS_OK;
}

int enqueue_step(tts_engine* e, int b) {
  char* d = e->d_block;
  BlockHeader* hd = (BlockHeader*)d;
  ECK(cudaMemcpyAsync(d, e->h_block[b], e->block_bytes, cudaMemcpyHostToDevice, e->stream));
  int rc = launch_frame_batch(e->own, e->C, e->frame_clusters, e->frame_smem, (const FrameParams*)(d + e->off_frames),
                              &hd->queue, e->stream);
  if (rc == TTS_OK)
    rc = launch_image_batch((const ImageJob*)(d + e->off_images), &hd->n_images, e->image_grid, e->stream);
  if (rc == TTS_OK)
    rc = launch_sampler_batch((const SamplerJob*)(d + e->off_samplers), &hd->n_samplers, e->max_slots, e->stream);
  if (rc != TTS_OK) return tts_fail(rc, "engine kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  return TTS_OK;
}

int capture_step(tts_engine* e, int b) {
  if (e->gexec[b]) {
    cudaGraphExecDestroy(e->gexec[b]);
    e->gexec[b] = nullptr;
  }
  ECK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_step(e, b);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
  if (rc != TTS_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) return tts_cuda_fail(ce, "cudaStreamEndCapture");
  const cudaError_t ie = cudaGraphInstantiate(&e->gexec[b], g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return tts_cuda_fail(ie, "cudaGraphInstantiate");
  e->graph_own[b] = e->own;
  return TTS_OK;
}

double frame_cost(const FrameParams& p) {
  // shared-memory passes over the factor rows per MM iteration, plus the ridge system
  return (double)p.K * ((double)(p.Nx + p.Ny) * p.R + (double)p.R * p.R * p.R / 8.0) + (double)p.Nx * p.Ny / 4.0;
}

}  // namespace

extern "C" {

int tts_stream_footprint(const tts_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return tts_fail(TTS_EINVAL, "NULL argument%s");
  const int rc = handle_check_config(cfg);
  if (rc) return rc;
  tts_config c = *cfg;
  if (c.cluster_ctas == 0) c.cluster_ctas = 8;
  const size_t b = handle_footprint(c);
  if (!b) return tts_fail(TTS_EINVAL, "no cluster size fits the shared memory for these Nx, Ny, R%s");
  *bytes = b;
  return TTS_OK;
}

int tts_engine_create(size_t arena_bytes, int max_slots, int cluster_ctas, int flags, void* cuda_stream,
                      tts_engine** out) {
  if (!out) return tts_fail(TTS_EINVAL, "out is NULL%s");
  *out = nullptr;
  if (max_slots < 1 || max_slots > TTS_ENGINE_MAX_SLOTS) return tts_fail(TTS_EINVAL, "max_slots must be 1..4096%s");
  if (cluster_ctas != 0 && cluster_ctas != 1 && cluster_ctas != 2 && cluster_ctas != 4 && cluster_ctas != 8 &&
      cluster_ctas != 16)
    return tts_fail(TTS_EINVAL, "cluster_ctas must be 0, 1, 2, 4, 8 or 16%s");
  if (flags & ~TTS_ENGINE_GRAPH) return tts_fail(TTS_EINVAL, "unknown engine flags%s");
  if (arena_bytes < 4096) return tts_fail(TTS_EINVAL, "arena_bytes is too small%s");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return tts_fail(TTS_ECUDA, "no CUDA device available (no CPU fallback)%s");
  tts_engine* e = new tts_engine();
  cudaGetDevice(&e->dev);
  e->C = cluster_ctas ? cluster_ctas : 8;
  e->max_slots = max_slots;
  e->use_graph = (flags & TTS_ENGINE_GRAPH) != 0;
  cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->dev);
  e->image_grid = std::max(1, e->sms) * 8;
  auto bail = [&](int rc) {
    tts_engine_destroy(e);
    return rc;
  };
  cudaError_t ce;
  if (cuda_stream) {
    e->stream = (cudaStream_t)cuda_stream;
  } else {
    ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(tts_cuda_fail(ce, "cudaStreamCreate"));
    e->own_stream = true;
  }
  ce = cudaStreamCreateWithFlags(&e->admin, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(tts_cuda_fail(ce, "cudaStreamCreate"));
  e->arena_bytes = arena_bytes & ~size_t(255);
  ce = cudaMalloc((void**)&e->arena, e->arena_bytes);
  if (ce != cudaSuccess) {
    e->arena = nullptr;
    return bail(tts_fail(TTS_ENOMEM, "device allocation of the engine arena failed%s"));
  }
  e->free_blocks[0] = e->arena_bytes;
  e->slot.assign(max_slots, nullptr);
  e->slot_off.assign(max_slots, 0);
  e->slot_len.assign(max_slots, 0);
  e->off_frames = sizeof(BlockHeader);
  e->off_samplers = e->off_frames + up256(sizeof(FrameParams) * max_slots);
  e->off_images = e->off_samplers + up256(sizeof(SamplerJob) * max_slots);
  e->block_bytes = e->off_images + up256(sizeof(ImageJob) * max_slots);
  ce = cudaMalloc((void**)&e->d_block, e->block_bytes);
  if (ce != cudaSuccess) {
    e->d_block = nullptr;
    return bail(tts_fail(TTS_ENOMEM, "device allocation of the parameter block failed%s"));
  }
  for (int b = 0; b < 2; ++b) {
    ce = cudaMallocHost((void**)&e->h_block[b], e->block_bytes);
    if (ce != cudaSuccess) {
      e->h_block[b] = nullptr;
      return bail(tts_fail(TTS_ENOMEM, "pinned allocation of the parameter block failed%s"));
    }
    memset(e->h_block[b], 0, e->block_bytes);
    ce = cudaEventCreateWithFlags(&e->done[b], cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(tts_cuda_fail(ce, "cudaEventCreate"));
  }
  // kernel attributes are set here, outside any capture
  int rc = refresh_shape(e);
  if (rc == TTS_OK) rc = launch_sampler_batch(nullptr, nullptr, 0, e->stream);
  if (rc != TTS_OK) return bail(rc);
  *out = e;
  return TTS_OK;
}

void tts_engine_destroy(tts_engine* e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  for (tts_handle* h : e->slot)
    if (h) tts_destroy(h);
  for (int b = 0; b < 2; ++b) {
    if (e->gexec[b]) cudaGraphExecDestroy(e->gexec[b]);
    if (e->done[b]) cudaEventDestroy(e->done[b]);
    if (e->h_block[b]) cudaFreeHost(e->h_block[b]);
  }
  if (e->d_block) cudaFree(e->d_block);
  if (e->arena) cudaFree(e->arena);
  if (e->admin) cudaStreamDestroy(e->admin);
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

int tts_engine_admit(tts_engine* e, const tts_config* cfg, int* slot_out) {
  if (!e || !cfg || !slot_out) return tts_fail(TTS_EINVAL, "NULL argument%s");
  *slot_out = -1;
  tts_config c = *cfg;
  c.cluster_ctas = e->C;
  c.launch = TTS_LAUNCH_FUSED;
  c.cuda_stream = e->admin;
  int rc = handle_check_config(&c);
  if (rc) return rc;
  const size_t need = handle_footprint(c);
  if (!need) return tts_fail(TTS_EINVAL, "no layout of this stream fits the engine's cluster size%s");
  int s = -1;
  for (int i = 0; i < e->max_slots; ++i)
    if (!e->slot[i]) {
      s = i;
      break;
    }
  if (s < 0) return tts_fail(TTS_EBUSY, "every engine slot is taken%s");
  size_t off = 0;
  if (!arena_take(e, need, &off)) return tts_fail(TTS_EBUSY, "the engine arena has no room for this stream%s");
  tts_handle* h = nullptr;
  rc = handle_create(&c, e->arena + off, &h);
  if (rc != TTS_OK) {
    arena_give(e, off, need);
    return rc;
  }
  // from now on the slot's work is ordered on the engine stream
  h->stream = e->stream;
  h->cfg.cuda_stream = e->stream;
  e->slot[s] = h;
  e->slot_off[s] = off;
  e->slot_len[s] = need;
  e->active += 1;
  rc = refresh_shape(e);
  if (rc != TTS_OK) {
    e->slot[s] = nullptr;
    e->active -= 1;
    tts_destroy(h);
    arena_give(e, off, need);
    return rc;
  }
  *slot_out = s;
  return TTS_OK;
}

int tts_engine_release(tts_engine* e, int slot) {
  if (!e) return tts_fail(TTS_EINVAL, "NULL engine%s");
  if (slot < 0 || slot >= e->max_slots || !e->slot[slot]) return tts_fail(TTS_EINVAL, "no stream in this slot%s");
  // the slot's memory may still be in use by steps in flight
  ECK(cudaStreamSynchronize(e->stream));
  tts_destroy(e->slot[slot]);
  e->slot[slot] = nullptr;
  arena_give(e, e->slot_off[slot], e->slot_len[slot]);
  e->active -= 1;
  return refresh_shape(e);
}

int tts_engine_handle(tts_engine* e, int slot, tts_handle** h) {
  if (!e || !h) return tts_fail(TTS_EINVAL, "NULL argument%s");
  if (slot < 0 || slot >= e->max_slots || !e->slot[slot]) return tts_fail(TTS_EINVAL, "no stream in this slot%s");
  *h = e->slot[slot];
  return TTS_OK;
}

int tts_engine_step(tts_engine* e, int n, const int* slots, const tts_c64* const* y_rows,
                    const uint8_t* const* line_masks, const double* rates, const uint64_t* seeds, int flags) {
  if (!e) return tts_fail(TTS_EINVAL, "NULL engine%s");
  if (n < 0 || n > e->max_slots) return tts_fail(TTS_EINVAL, "n must be 0..max_slots%s");
  if (n == 0) return TTS_OK;
  if (!slots || !y_rows || !rates || !seeds) return tts_fail(TTS_EINVAL, "NULL argument%s");
  if (flags & ~(TTS_DEVICE_PTRS | TTS_FULL_FRAME)) return tts_fail(TTS_EINVAL, "unknown flags%s");
  std::vector<char> seen(e->max_slots, 0);
  for (int i = 0; i < n; ++i) {
    const int s = slots[i];
    if (s < 0 || s >= e->max_slots || !e->slot[s]) return tts_fail(TTS_EINVAL, "no stream in a listed slot%s");
    if (seen[s]) return tts_fail(TTS_EINVAL, "a slot is listed twice in one step%s");
    seen[s] = 1;
    if (!y_rows[i]) return tts_fail(TTS_EINVAL, "NULL frame%s");
    if (!(rates[i] > 0.0 && rates[i] <= 1.0)) return tts_fail(TTS_EINVAL, "rate must lie in (0, 1]%s");
  }
  const int b = e->cur;
  if (e->pending[b]) {
    ECK(cudaEventSynchronize(e->done[b]));
    e->pending[b] = false;
  }
  char* blk = e->h_block[b];
  BlockHeader* hd = (BlockHeader*)blk;
  FrameParams* fps = (FrameParams*)(blk + e->off_frames);
  SamplerJob* sjs = (SamplerJob*)(blk + e->off_samplers);
  ImageJob* ijs = (ImageJob*)(blk + e->off_images);
  // stage every frame first: a refused frame leaves every slot's state as it was
  std::vector<FrameParams> staged(n);
  for (int i = 0; i < n; ++i) {
    tts_handle* h = e->slot[slots[i]];
    const uint8_t* m = line_masks ? line_masks[i] : nullptr;
    if (!m && !(flags & TTS_DEVICE_PTRS) && (flags & TTS_FULL_FRAME)) {
      // full host frame with the drawn mask: copy the frame, keep the mask on the device
      // (non-finite samples are then caught by the frame kernel, as for device inputs)
      if (!h->have_next) return tts_fail(TTS_ESTATE, "no mask given and none drawn yet%s");
      FrameParams p = h->fp;
      p.full_frame = 1;
      p.mask = h->dmask_next;
      ECK(cudaMemcpyAsync(h->ystage, y_rows[i], sizeof(float2) * (size_t)h->cfg.Nx * h->cfg.Ny,
                          cudaMemcpyHostToDevice, e->stream));
      p.yrows = h->ystage;
      staged[i] = p;
      continue;
    }
    const int rc = handle_stage_frame(h, y_rows[i], m, flags, &staged[i]);
    if (rc != TTS_OK) return rc;
  }
  // the queue hands out the largest frames first
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return frame_cost(staged[a]) > frame_cost(staged[c]); });
  for (int k = 0; k < n; ++k) fps[k] = staged[order[k]];
  int tile0 = 0;
  for (int i = 0; i < n; ++i) {
    tts_handle* h = e->slot[slots[i]];
    const tts_config& c = h->cfg;
    // the draw follows this frame: its counter is that of frame t + 1
    h->t += 1;
    const uint64_t ctr = handle_draw_counter(h);
    h->t -= 1;
    sjs[i] = sampler_job(h->fp.A, c.Nx, c.Ny, c.R, nullptr, h->dp, c.policy, c.vd_alpha, handle_k_lines(h, rates[i]),
                         c.central_lines, seeds[i], ctr, c.with_replacement, h->fp.Wx, h->dmask_next, nullptr);
    ImageJob& ij = ijs[i];
    ij.A = h->fp.A;
    ij.B = h->fp.B;
    ij.gamma = h->fp.gamma;
    ij.X = h->X;
    ij.Nx = c.Nx;
    ij.Ny = c.Ny;
    ij.R = c.R;
    ij.tile0 = tile0;
    ij.tiles = ((c.Nx + 31) / 32) * ((c.Ny + 31) / 32);
    tile0 += ij.tiles;
  }
  hd->queue = 0;
  hd->n_frames = n;
  hd->n_samplers = n;
  hd->n_images = n;
  int rc = TTS_OK;
  if (e->use_graph) {
    if (!e->gexec[b] || e->graph_own[b] != e->own) rc = capture_step(e, b);
    if (rc == TTS_OK) {
      const cudaError_t ge = cudaGraphLaunch(e->gexec[b], e->stream);
      if (ge != cudaSuccess) rc = tts_cuda_fail(ge, "cudaGraphLaunch");
    }
  } else {
    rc = enqueue_step(e, b);
  }
  if (rc != TTS_OK) return rc;
  ECK(cudaEventRecord(e->done[b], e->stream));
  e->pending[b] = true;
  e->cur = b ^ 1;
  e->steps += 1;
  for (int i = 0; i < n; ++i) {
    tts_handle* h = e->slot[slots[i]];
    h->t += 1;
    h->have_next = true;
    h->next_on_host = false;
  }
  return TTS_OK;
}

int tts_engine_image(tts_engine* e, int slot, tts_c64* out, int flags) {
  if (!e || !out) return tts_fail(TTS_EINVAL, "NULL argument%s");
  if (slot < 0 || slot >= e->max_slots || !e->slot[slot]) return tts_fail(TTS_EINVAL, "no stream in this slot%s");
  tts_handle* h = e->slot[slot];
  if (h->t == 0) return tts_fail(TTS_ERANGE, "the stream has no frame yet%s");
  const size_t bytes = sizeof(float2) * (size_t)h->cfg.Nx * h->cfg.Ny;
  if (flags & TTS_DEVICE_PTRS) {
    ECK(cudaMemcpyAsync(out, h->X, bytes, cudaMemcpyDeviceToDevice, e->stream));
  } else {
    ECK(cudaMemcpyAsync(out, h->X, bytes, cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
  }
  return TTS_OK;
}

int tts_engine_mask(tts_engine* e, int slot, uint8_t* out, int flags) {
  if (!e || !out) return tts_fail(TTS_EINVAL, "NULL argument%s");
  if (slot < 0 || slot >= e->max_slots || !e->slot[slot]) return tts_fail(TTS_EINVAL, "no stream in this slot%s");
  tts_handle* h = e->slot[slot];
  if (!h->have_next) return tts_fail(TTS_ESTATE, "no mask drawn for this stream yet%s");
  if (flags & TTS_DEVICE_PTRS) {
    ECK(cudaMemcpyAsync(out, h->dmask_next, h->cfg.Nx, cudaMemcpyDeviceToDevice, e->stream));
  } else {
    ECK(cudaMemcpyAsync(out, h->dmask_next, h->cfg.Nx, cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
  }
  return TTS_OK;
}

int tts_engine_synchronize(tts_engine* e) {
  if (!e) return tts_fail(TTS_EINVAL, "NULL engine%s");
  ECK(cudaStreamSynchronize(e->stream));
  int bad = 0;
  for (tts_handle* h : e->slot)
    if (h && tts_synchronize(h) != TTS_OK) bad = 1;
  if (bad) return tts_fail(TTS_ENONFINITE, "a frame held NaN or Inf and was skipped%s");
  return TTS_OK;
}

int tts_engine_info(tts_engine* e, tts_engine_stats* st) {
  if (!e || !st) return tts_fail(TTS_EINVAL, "NULL argument%s");
  size_t largest = 0;
  for (auto& kv : e->free_blocks) largest = std::max(largest, kv.second);
  st->arena_bytes = e->arena_bytes;
  st->arena_used = e->used;
  st->arena_largest_free = largest;
  st->active = e->active;
  st->max_slots = e->max_slots;
  st->cluster_ctas = e->C;
  st->resident_clusters = e->frame_clusters;
  st->owned_outputs = e->own;
  st->steps = e->steps;
  return TTS_OK;
}

}  // extern "C"
