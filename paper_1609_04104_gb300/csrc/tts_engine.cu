// Many concurrent trackers on one GPU: the serving and batching form of the per-frame
// update (Alg. 3 with one coil, then the line draw of Alg. 4 for the next frame).
//
// Every stream (a cine slice with its own Nx, Ny, R, lambda_forget, mu, K, rate) is a
// tracker handle whose device state lives in one slot of a device arena that the engine
// reserves once; admission asks the arena for the stream's footprint and is refused when
// it has no room. A stream runs its frames on a cluster of C CTAs: the engine's preferred
// C when the stream's layout fits it, else the next larger size that fits. One engine step
// takes one frame for each of a set of slots and runs
//   (1) their MM iterations in one persistent launch per cluster size (launched on forked
//       streams, so the groups overlap): clusters pull frames from a queue ordered
//       largest first, each frame staying on one cluster;
//   (2) all their images X_t = A diag(gamma) B^T in one launch over the union of tiles;
//   (3) all their next-frame line draws in one launch, one CTA per stream;
// with the parameters of the step in one block copied from pinned host memory. The
// operations are captured once in a CUDA graph and replayed; the kernels read the step's
// counts from the parameter block, so one graph serves any subset of the slots.
// Each stream's arithmetic is exactly that of its handle run alone with the same cluster
// size, so its results do not depend on what else is in the step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "tts_handle.cuh"

namespace {

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int kMaxGroups = 5;   // cluster sizes 1, 2, 4, 8, 16

struct BlockHeader {
  int q[8][4];      // per group: queue counter (0 at launch), frames, offset of its blocks
  int n_samplers;
  int n_images;
  int pad[30];
};
static_assert(sizeof(BlockHeader) == 256, "parameter block header is 256 bytes");

struct Group {
  int C = 0, own = 0, smem = 0, clusters = 0;
};

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
  // one persistent frame launch per cluster size in use, on its own forked stream
  std::vector<Group> groups;
  Group limits[4][kMaxGroups];     // launch limits per (OWN 1/2/4/8, C 1/2/4/8/16), at creation
  cudaStream_t side[kMaxGroups] = {};
  cudaEvent_t fork = nullptr, join[kMaxGroups] = {};
  int image_grid = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::vector<Group> graph_groups[2];
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

bool same_groups(const std::vector<Group>& a, const std::vector<Group>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].C != b[i].C || a[i].own != b[i].own) return false;
  return true;
}

// The cluster sizes in use and, per size, the largest per-thread output count (OWN) of
// its streams and the launch limits.
int refresh_groups(tts_engine* e) {
  std::vector<Group> g;
  for (tts_handle* h : e->slot) {
    if (!h) continue;
    const int C = h->fp.C, own = frame_own(h->fp);
    bool found = false;
    for (Group& x : g)
      if (x.C == C) {
        x.own = std::max(x.own, own);
        found = true;
      }
    if (!found) {
      Group x;
      x.C = C;
      x.own = own;
      g.push_back(x);
    }
  }
  std::sort(g.begin(), g.end(), [](const Group& a, const Group& b) { return a.C < b.C; });
  for (Group& x : g) {
    const Group& l = e->limits[x.own == 1 ? 0 : x.own == 2 ? 1 : x.own == 4 ? 2 : 3][__builtin_ctz(x.C)];
    if (l.clusters <= 0) return tts_fail(TTS_ECUDA, "no launch limits for this cluster size%s");
    x = l;
  }
  e->groups = g;
  return TTS_OK;
}

// Launch limits of every kernel variant a stream may need, computed (and the variants
// loaded) once, so that admitting a stream never waits on module loading.
int prepare_limits(tts_engine* e) {
  static const int owns[4] = {1, 2, 4, 8};
  for (int oi = 0; oi < 4; ++oi)
    for (int ci = 0; ci < kMaxGroups; ++ci) {
      Group& l = e->limits[oi][ci];
      l.C = 1 << ci;
      l.own = owns[oi];
      if (l.C < e->C) continue;
      const int rc = frame_batch_limits(l.own, l.C, &l.smem, &l.clusters);
      if (rc != TTS_OK) return tts_fail(rc, "cannot size the persistent frame launch%s");
    }
  return TTS_OK;
}

int group_index(const tts_engine* e, int C) {
  for (size_t i = 0; i < e->groups.size(); ++i)
    if (e->groups[i].C == C) return (int)i;
  return -1;
}

int enqueue_step(tts_engine* e, int b) {
  char* d = e->d_block;
  BlockHeader* hd = (BlockHeader*)d;
  ECK(cudaMemcpyAsync(d, e->h_block[b], e->block_bytes, cudaMemcpyHostToDevice, e->stream));
  ECK(cudaEventRecord(e->fork, e->stream));
  int rc = TTS_OK;
  for (size_t g = 0; g < e->groups.size() && rc == TTS_OK; ++g) {
    const Group& x = e->groups[g];
    ECK(cudaStreamWaitEvent(e->side[g], e->fork, 0));
    rc = launch_frame_batch(x.own, x.C, std::min(x.clusters, e->max_slots), x.smem,
                            (const FrameParams*)(d + e->off_frames), &hd->q[g][0], e->side[g]);
    ECK(cudaEventRecord(e->join[g], e->side[g]));
    ECK(cudaStreamWaitEvent(e->stream, e->join[g], 0));
  }
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
  e->graph_groups[b] = e->groups;
  return TTS_OK;
}

// Footprint of a stream on the preferred cluster size, else on the next larger size that
// holds its layout (0 if none does); the size in *C_out.
size_t engine_footprint(tts_config c, int C_pref, int* C_out) {
  for (int C = C_pref; C <= TTS_MAX_CLUSTER; C *= 2) {
    c.cluster_ctas = C;
    const size_t f = handle_footprint(c);
    if (f) {
      if (C_out) *C_out = C;
      return f;
    }
  }
  return 0;
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
  if (c.cluster_ctas == 0) c.cluster_ctas = 4;
  const size_t b = handle_footprint(c);
  if (!b) return tts_fail(TTS_EINVAL, "the stream's layout does not fit clusters of this size%s");
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
  e->C = cluster_ctas ? cluster_ctas : 4;
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
  for (int g = 0; g < kMaxGroups; ++g) {
    ce = cudaStreamCreateWithFlags(&e->side[g], cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->join[g], cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(tts_cuda_fail(ce, "engine streams"));
  }
  ce = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
  if (ce != cudaSuccess) return bail(tts_cuda_fail(ce, "cudaEventCreate"));
  // kernel attributes are set here, outside any capture
  int rc = launch_sampler_batch(nullptr, nullptr, 0, e->stream);
  if (rc == TTS_OK) rc = launch_image_batch(nullptr, nullptr, 0, e->stream);
  if (rc == TTS_OK) rc = prepare_limits(e);
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
  for (int g = 0; g < kMaxGroups; ++g) {
    if (e->join[g]) cudaEventDestroy(e->join[g]);
    if (e->side[g]) cudaStreamDestroy(e->side[g]);
  }
  if (e->fork) cudaEventDestroy(e->fork);
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
  c.launch = TTS_LAUNCH_FUSED;
  c.cuda_stream = e->admin;
  int rc = handle_check_config(&c);
  if (rc) return rc;
  if (c.row_dft != TTS_ROWDFT_FFT) return tts_fail(TTS_EINVAL, "engine streams transform rows in the frame kernel%s");
  if (c.kspace) return tts_fail(TTS_EINVAL, "engine streams track image-domain factors%s");
  // the preferred cluster size, else the next larger one that holds the stream's layout
  int C = 0;
  const size_t need = engine_footprint(c, e->C, &C);
  if (!need) return tts_fail(TTS_EINVAL, "no cluster size holds this stream's layout%s");
  c.cluster_ctas = C;
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
  h->in_engine = true;
  h->stream = e->stream;
  h->cfg.cuda_stream = e->stream;
  e->slot[s] = h;
  e->slot_off[s] = off;
  e->slot_len[s] = need;
  e->active += 1;
  rc = refresh_groups(e);
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
  return refresh_groups(e);
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
  // frames grouped by cluster size; each group's queue hands out its largest frames first
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    if (staged[a].C != staged[c].C) return staged[a].C < staged[c].C;
    return frame_cost(staged[a]) > frame_cost(staged[c]);
  });
  memset(hd->q, 0, sizeof(hd->q));
  for (int k = 0; k < n; ++k) {
    fps[k] = staged[order[k]];
    const int g = group_index(e, fps[k].C);
    if (g < 0) return tts_fail(TTS_ESTATE, "a stream's cluster size has no launch group%s");
    if (hd->q[g][1] == 0) hd->q[g][2] = k;
    hd->q[g][1] += 1;
  }
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
  hd->n_samplers = n;
  hd->n_images = n;
  int rc = TTS_OK;
  if (e->use_graph) {
    if (!e->gexec[b] || !same_groups(e->graph_groups[b], e->groups)) rc = capture_step(e, b);
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

int tts_engine_autotune(const tts_config* cfgs, int n, int steps, int* best_C, double* step_ms) {
  if (!cfgs || !best_C || n < 1 || n > TTS_ENGINE_MAX_SLOTS || steps < 1)
    return tts_fail(TTS_EINVAL, "bad autotune arguments%s");
  static const int kCand[5] = {1, 2, 4, 8, 16};
  *best_C = 0;
  double best = 0.0;
  for (int ci = 0; ci < 5; ++ci) {
    const int C = kCand[ci];
    if (step_ms) step_ms[ci] = -1.0;
    // every stream runs on this size or, as in an engine, the next larger that fits it;
    // a candidate no stream can use is skipped
    size_t arena = 64u << 20;
    bool ok = true, used = false;
    for (int k = 0; k < n && ok; ++k) {
      tts_config c = cfgs[k];
      if (handle_check_config(&c) != TTS_OK) return TTS_EINVAL;
      int Ck = 0;
      const size_t f = engine_footprint(c, C, &Ck);
      if (!f) ok = false;
      used = used || Ck == C;
      arena += f;
    }
    if (!ok || !used) continue;
    tts_engine* e = nullptr;
    int rc = tts_engine_create(arena, n, C, TTS_ENGINE_GRAPH, nullptr, &e);
    if (rc != TTS_OK) return rc;
    std::vector<int> slots(n);
    std::vector<const tts_c64*> frames(n);
    std::vector<const uint8_t*> masks(n, nullptr);
    std::vector<double> rates(n);
    std::vector<uint64_t> seeds(n);
    size_t fbytes = 0, mbytes = 0;
    for (int k = 0; k < n; ++k) {
      fbytes += up256(sizeof(float2) * (size_t)cfgs[k].Nx * cfgs[k].Ny);
      mbytes += up256((size_t)cfgs[k].Nx);
    }
    char* dbuf = nullptr;
    cudaError_t ce = cudaMalloc((void**)&dbuf, fbytes + mbytes);
    if (ce != cudaSuccess) {
      tts_engine_destroy(e);
      return tts_fail(TTS_ENOMEM, "autotune frame buffers%s");
    }
    // synthetic fully sampled frames: CN(0, 1) samples from the factor initialiser
    size_t fo = 0, mo = fbytes;
    for (int k = 0; k < n && rc == TTS_OK; ++k) {
      tts_config c = cfgs[k];
      rc = tts_engine_admit(e, &c, &slots[k]);
      if (rc != TTS_OK) break;
      frames[k] = (const tts_c64*)(dbuf + fo);
      masks[k] = (const uint8_t*)(dbuf + mo);
      rc = launch_init_factors((float2*)(dbuf + fo), c.Nx, c.Ny, 0x7u + k, 3, e->stream);
      if (cudaMemsetAsync(dbuf + mo, 1, c.Nx, e->stream) != cudaSuccess) rc = TTS_ECUDA;
      fo += up256(sizeof(float2) * (size_t)c.Nx * c.Ny);
      mo += up256((size_t)c.Nx);
      rates[k] = 1.0 / 8.0;
      seeds[k] = 1 + k;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == TTS_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = TTS_ECUDA;
    float ms = 0.f;
    if (rc == TTS_OK) {
      // the first step is fully sampled and untimed (graph capture); later steps use the
      // drawn masks
      rc = tts_engine_step(e, n, slots.data(), frames.data(), masks.data(), rates.data(), seeds.data(),
                           TTS_DEVICE_PTRS | TTS_FULL_FRAME);
      if (rc == TTS_OK) rc = tts_engine_step(e, n, slots.data(), frames.data(), nullptr, rates.data(), seeds.data(),
                                             TTS_DEVICE_PTRS | TTS_FULL_FRAME);
      if (rc == TTS_OK && cudaEventRecord(e0, e->stream) != cudaSuccess) rc = TTS_ECUDA;
      for (int s = 0; s < steps && rc == TTS_OK; ++s)
        rc = tts_engine_step(e, n, slots.data(), frames.data(), nullptr, rates.data(), seeds.data(),
                             TTS_DEVICE_PTRS | TTS_FULL_FRAME);
      if (rc == TTS_OK && (cudaEventRecord(e1, e->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = TTS_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    tts_engine_destroy(e);
    cudaFree(dbuf);
    if (rc != TTS_OK) return rc;
    const double per = (double)ms / steps;
    if (step_ms) step_ms[ci] = per;
    if (*best_C == 0 || per < best) {
      best = per;
      *best_C = C;
    }
  }
  if (*best_C == 0) return tts_fail(TTS_EINVAL, "no cluster size fits every stream%s");
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
  st->groups = (int)e->groups.size();
  st->resident_clusters = 0;
  for (const Group& g : e->groups) st->resident_clusters += g.clusters;
  st->steps = e->steps;
  return TTS_OK;
}

}  // extern "C"
