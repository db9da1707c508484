// The tracker handle behind the C ABI (tts_handle in include/tts.h) and the host-side
// pieces that the single-stream calls (tts_api.cu) and the multi-stream engine
// (tts_engine.cu) share.
#pragma once

#include <string>
#include <vector>

#include "tts_internal.cuh"

struct MultiCoil;   // coil maps and workspace of the multi-coil tracker (tts_multicoil.cu)

struct tts_handle {
  tts_config cfg;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool own_mem = true;          // dmem came from cudaMalloc (else from an engine arena)
  void* dmem = nullptr;
  size_t dbytes = 0;
  FrameParams fp;
  float2* X = nullptr;          // image
  float2* ystage = nullptr;     // acquired rows from host pushes
  uint8_t* dmask_push = nullptr;
  uint8_t* dmask_next = nullptr;
  double* dp = nullptr;
  int64_t t = 0;                // frames processed
  bool have_next = false;
  bool next_on_host = false;
  bool in_engine = false;       // a slot of an engine (no coil maps)
  std::vector<uint8_t> next_host;
  MultiCoil* mc = nullptr;      // set by tts_set_coil_maps
  // pinned host staging of the acquired rows of host pushes (tts_push_frame): two buffers
  // of Nx x Ny, mapped into the device address space when possible (hstage_dev: the kernels
  // read the rows in place), each reused once the work recorded by its event has completed
  float2* hstage[2] = {nullptr, nullptr};
  float2* hstage_dev[2] = {nullptr, nullptr};
  cudaEvent_t hstage_done[2] = {nullptr, nullptr};
  int hstage_next = 0;
  int hstage_pending = -1;      // staged buffer whose event follows the frame's launches
  // the drawn mask for host callers: mapped pinned memory the sampler writes directly
  // (mask_map on the host, mask_map_dev its device address), so no copy follows the draw
  uint8_t* mask_map = nullptr;
  uint8_t* mask_map_dev = nullptr;
  // completion word of the last draw in the same mapped allocation (after the mask, 64-byte
  // aligned): the sampler sets it to draw_seq once the mask is written, the host polls it
  unsigned int* draw_done = nullptr;
  unsigned int* draw_done_dev = nullptr;
  unsigned int draw_seq = 0;
  // test hook (tts_test_withhold_row_transform): the next row transform withholds this K'
  // chunk's arrival and waits at most test_wait_cycles; -1: none
  int test_withhold = -1;
  long long test_wait_cycles = 0;
};

// Validates a configuration (message through tts_last_error on failure).
int handle_check_config(const tts_config* c);
// Device bytes one tracker holds, for a cluster of C CTAs (C = 0: the size frame_configure
// picks); 0 if no cluster size fits.
size_t handle_footprint(const tts_config& cfg);
// Creates a tracker whose device state lives in `mem` (at least handle_footprint bytes,
// 256-byte aligned), or in its own allocation when mem is NULL. Initialisation runs on
// cfg->cuda_stream (or a stream of its own) and is complete on return.
int handle_create(const tts_config* cfg, void* mem, tts_handle** out);
// Fills p (a copy of h->fp) with the frame's mask and rows, staging host inputs into the
// handle's device buffers on h->stream, with the checks of tts_push_frame. With
// pinned_gather, host rows go through the handle's pinned staging (only the acquired rows,
// also of a full frame, checked for NaN/Inf while they are gathered) and a line mask of
// NULL is read from the device copy of the last draw; otherwise the rows are copied from
// y_rows as they are.
int handle_stage_frame(tts_handle* h, const tts_c64* y_rows, const uint8_t* line_mask, int flags, FrameParams* p,
                       bool pinned_gather = false);
// Philox counter of the next draw: stream_id in the high bits, frames processed below.
uint64_t handle_draw_counter(const tts_handle* h);
// Lines a draw at this rate keeps: max(central, round(rate Nx)).
int handle_k_lines(const tts_handle* h, double rate);
int tts_fail(int code, const char* fmt, const char* detail = nullptr);
// multi-coil tracker (tts_multicoil.cu)
int mc_attach(tts_handle* h, const float2* maps, int C, bool device);
void mc_detach(tts_handle* h);
int mc_push(tts_handle* h, const tts_c64* y, const uint8_t* mask, int flags);
int tts_cuda_fail(cudaError_t e, const char* where);
