// Host side of the C ABI declared in include/tts.h: handle life cycle, argument checks,
// device workspace, and the enqueueing of the kernels for each call.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "tts_handle.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, const char* detail = nullptr) {
  char buf[512];
  snprintf(buf, sizeof(buf), fmt, detail ? detail : "");
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_err = buf;
  return TTS_ECUDA;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

std::vector<float2> twiddles(int N) {
  std::vector<float2> w(N);
  for (int k = 0; k < N; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)N;
    w[k] = make_float2((float)cos(a), (float)-sin(a));
  }
  return w;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

struct Piece {
  void** ptr;
  size_t bytes;
};

// The device workspace of a tracker, in allocation order.
std::vector<Piece> handle_pieces(tts_handle* h, int Nx, int Ny, int R, int C) {
  FrameParams& p = h->fp;
  return {
      {(void**)&p.A, sizeof(float2) * Nx * R},          {(void**)&p.B, sizeof(float2) * Ny * R},
      {(void**)&p.A0, sizeof(float2) * Nx * R},         {(void**)&p.B0, sizeof(float2) * Ny * R},
      {(void**)&h->ystage, sizeof(float2) * Nx * Ny},   {(void**)&p.Yt, sizeof(float2) * Nx * Ny},
      {(void**)&p.rows, sizeof(int) * Nx},              {(void**)&p.nrows, sizeof(int) * 4},
      {(void**)&p.AhS[0], sizeof(float2) * Nx * R},     {(void**)&p.AhS[1], sizeof(float2) * Nx * R},
      {(void**)&p.nA[0], sizeof(float) * R},            {(void**)&p.nA[1], sizeof(float) * R},
      {(void**)&p.MB, sizeof(float2) * R * R},          {(void**)&p.P, sizeof(float2) * Nx * R},
      {(void**)&p.MBlo, sizeof(float2) * R * R},        {(void**)&p.Plo, sizeof(float2) * Nx * R},
      {(void**)&p.MA, sizeof(float2) * R * R},          {(void**)&p.MAlo, sizeof(float2) * R * R},
      {(void**)&p.partA, sizeof(float2) * C * Nx * R},  {(void**)&p.partNA, sizeof(float) * C * R},
      {(void**)&p.partMB, sizeof(float4) * C * R * R},  {(void**)&p.partP, sizeof(float4) * C * Nx * R},
      {(void**)&p.partMA, sizeof(float4) * C * R * R},
      {(void**)&p.sc, sizeof(double) * SC_COUNT},
      {(void**)&p.sf, sizeof(double) * SF_COUNT},       {(void**)&p.gamma, sizeof(float2) * R},
      {(void**)&p.gamma_d, sizeof(double2) * R},        {(void**)&p.status, sizeof(int) * (3 + TTS_MAX_CLUSTER)},
      {(void**)&p.Wx, sizeof(float2) * Nx},             {(void**)&p.Wy, sizeof(float2) * Ny},
      {(void**)&h->X, sizeof(float2) * Nx * Ny},        {(void**)&h->dmask_push, (size_t)Nx},
      {(void**)&h->dmask_next, (size_t)Nx},             {(void**)&h->dp, sizeof(double) * Nx},
  };
}

}  // namespace

void tts_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }
int tts_fail(int code, const char* fmt, const char* detail) { return fail(code, fmt, detail); }
int tts_cuda_fail(cudaError_t e, const char* where) { return cuda_fail(e, where); }

int handle_check_config(const tts_config* c) {
  if (!c) return fail(TTS_EINVAL, "config is NULL%s");
  if (c->Nx < 1 || c->Nx > TTS_MAX_N || !smooth235(c->Nx)) return fail(TTS_EINVAL, "Nx must be 1..512 with prime factors in {2,3,5}%s");
  if (c->Ny < 1 || c->Ny > TTS_MAX_N || !smooth235(c->Ny)) return fail(TTS_EINVAL, "Ny must be 1..512 with prime factors in {2,3,5}%s");
  if (c->R < 1 || c->R > TTS_MAX_R) return fail(TTS_EINVAL, "R must be 1..64%s");
  if (!(c->lambda_forget > 0.0 && c->lambda_forget <= 1.0)) return fail(TTS_EINVAL, "lambda_forget must lie in (0, 1]%s");
  if (!(c->mu > 0.0) || !isfinite(c->mu)) return fail(TTS_EINVAL, "mu must be positive and finite%s");
  if (c->mm_iters < 1 || c->mm_iters > 1000) return fail(TTS_EINVAL, "mm_iters must be 1..1000%s");
  if (c->central_lines < 0 || c->central_lines > c->Nx) return fail(TTS_EINVAL, "central_lines must be 0..Nx%s");
  if (c->policy < TTS_POLICY_UNIFORM || c->policy > TTS_POLICY_INFORMATIVE) return fail(TTS_EINVAL, "unknown policy%s");
  if (c->update != TTS_UPDATE_GAUSS_SEIDEL && c->update != TTS_UPDATE_JACOBI) return fail(TTS_EINVAL, "unknown update order%s");
  if (c->launch != TTS_LAUNCH_FUSED && c->launch != TTS_LAUNCH_PHASES) return fail(TTS_EINVAL, "unknown launch mode%s");
  if (c->cluster_ctas < 0 || c->cluster_ctas > TTS_MAX_CLUSTER) return fail(TTS_EINVAL, "cluster_ctas must be 0..16%s");
  if (!isfinite(c->vd_alpha)) return fail(TTS_EINVAL, "vd_alpha must be finite%s");
  if (c->row_dft < TTS_ROWDFT_FFT || c->row_dft > TTS_ROWDFT_BF16) return fail(TTS_EINVAL, "unknown row_dft%s");
  if (c->kspace != 0 && c->kspace != 1) return fail(TTS_EINVAL, "kspace must be 0 or 1%s");
  if (c->ridge_precision != TTS_RIDGE_FF_ALL && c->ridge_precision != TTS_RIDGE_FF_LAST)
    return fail(TTS_EINVAL, "unknown ridge_precision%s");
  if (c->kspace && c->row_dft != TTS_ROWDFT_FFT) return fail(TTS_EINVAL, "the k-space tracker transforms no rows%s");
  if (c->row_dft != TTS_ROWDFT_FFT && !dft_gemm_size_ok(c->Ny))
    return fail(TTS_EINVAL, "the tensor-core row transform needs Ny a multiple of 32 in [32, 256]%s");
  return TTS_OK;
}

size_t handle_footprint(const tts_config& cfg) {
  tts_handle tmp;
  memset(&tmp.fp, 0, sizeof(tmp.fp));
  tmp.fp.Nx = cfg.Nx;
  tmp.fp.Ny = cfg.Ny;
  tmp.fp.R = cfg.R;
  if (frame_configure(tmp.fp, cfg.cluster_ctas) != TTS_OK) return 0;
  size_t total = 0;
  for (auto& pc : handle_pieces(&tmp, cfg.Nx, cfg.Ny, cfg.R, tmp.fp.C)) total += align_up(pc.bytes);
  return total;
}

int handle_create(const tts_config* cfg, void* mem, tts_handle** out) {
  if (!out) return fail(TTS_EINVAL, "out is NULL%s");
  *out = nullptr;
  int rc = handle_check_config(cfg);
  if (rc) return rc;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail(TTS_ECUDA, "no CUDA device available (no CPU fallback)%s");
  tts_handle* h = new tts_handle();
  h->cfg = *cfg;
  cudaGetDevice(&h->dev);
  const int Nx = cfg->Nx, Ny = cfg->Ny, R = cfg->R;
  FrameParams& p = h->fp;
  memset(&p, 0, sizeof(p));
  p.Nx = Nx;
  p.Ny = Ny;
  p.R = R;
  if (frame_configure(p, cfg->cluster_ctas) != TTS_OK) {
    delete h;
    return fail(TTS_EINVAL, "no cluster size fits the shared memory for these Nx, Ny, R%s");
  }
  const int C = p.C;
  h->cfg.cluster_ctas = C;
  if (cfg->cuda_stream) {
    h->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "cudaStreamCreate");
    }
    h->own_stream = true;
  }
  std::vector<Piece> pieces = handle_pieces(h, Nx, Ny, R, C);
  size_t total = 0;
  for (auto& pc : pieces) total += align_up(pc.bytes);
  if (mem) {
    h->dmem = mem;
    h->own_mem = false;
  } else {
    e = cudaMalloc(&h->dmem, total);
    if (e != cudaSuccess) {
      if (h->own_stream) cudaStreamDestroy(h->stream);
      delete h;
      return fail(TTS_ENOMEM, "device allocation of the tracker workspace failed%s");
    }
  }
  h->dbytes = total;
  size_t off = 0;
  for (auto& pc : pieces) {
    *pc.ptr = (char*)h->dmem + off;
    off += align_up(pc.bytes);
  }
  p.K = cfg->mm_iters;
  p.refine = 5;
  p.ridge_ff_all = cfg->ridge_precision == TTS_RIDGE_FF_ALL ? 1 : 0;
  p.jacobi = cfg->update == TTS_UPDATE_JACOBI;
  p.lf = cfg->lambda_forget;
  p.mu = cfg->mu;
  p.kspace = cfg->kspace;
  p.isx = cfg->kspace ? 1.f : (float)(1.0 / sqrt((double)Nx));
  p.isy = cfg->kspace ? 1.f : (float)(1.0 / sqrt((double)Ny));
  p.plan_y = fft_plan(Ny);
  std::vector<float2> wx = twiddles(Nx), wy = twiddles(Ny);
  rc = TTS_OK;
  auto ck = [&](cudaError_t ee, const char* where) {
    if (ee != cudaSuccess && rc == TTS_OK) rc = cuda_fail(ee, where);
  };
  ck(cudaMemsetAsync(h->dmem, 0, total, h->stream), "memset workspace");
  ck(cudaMemcpyAsync((void*)p.Wx, wx.data(), sizeof(float2) * Nx, cudaMemcpyHostToDevice, h->stream), "twiddles");
  ck(cudaMemcpyAsync((void*)p.Wy, wy.data(), sizeof(float2) * Ny, cudaMemcpyHostToDevice, h->stream), "twiddles");
  if (rc == TTS_OK) rc = launch_init_factors(p.A, Nx, R, cfg->init_seed, 0, h->stream);
  if (rc == TTS_OK) rc = launch_init_factors(p.B, Ny, R, cfg->init_seed, 1, h->stream);
  if (rc == TTS_OK) ck(cudaStreamSynchronize(h->stream), "create");
  if (rc != TTS_OK) {
    if (g_err.empty()) g_err = "kernel launch failed during create";
    if (h->own_mem) cudaFree(h->dmem);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return rc;
  }
  h->next_host.assign(Nx, 0);
  *out = h;
  return TTS_OK;
}

// Gathers the acquired rows of a host frame (compact |S| x Ny, or a full Nx x Ny frame) into
// the next pinned staging buffer, checking every value for NaN/Inf on the way; *out is the
// buffer. The buffer's previous copy has completed before it is overwritten.
static int gather_host_rows(tts_handle* h, const float* y, const uint8_t* m, bool full, float2** out) {
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny;
  const int b = h->hstage_next;
  if (!h->hstage[b]) {
    const size_t bytes = sizeof(float2) * (size_t)Nx * Ny;
    void* d = nullptr;
    if (cudaHostAlloc((void**)&h->hstage[b], bytes, cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer(&d, h->hstage[b], 0) == cudaSuccess) {
      h->hstage_dev[b] = (float2*)d;
    } else {   // no mapping: plain pinned memory and a copy per push
      if (h->hstage[b]) cudaFreeHost(h->hstage[b]);
      h->hstage[b] = nullptr;
      cudaGetLastError();
      CK(cudaMallocHost((void**)&h->hstage[b], bytes));
    }
    CK(cudaEventCreateWithFlags(&h->hstage_done[b], cudaEventDisableTiming));
  } else {
    CK(cudaEventSynchronize(h->hstage_done[b]));
  }
  float* dst = (float*)h->hstage[b];
  const size_t row = 2 * (size_t)Ny;   // floats per row
  uint32_t bad = 0;
  for (int i = 0, m_ = 0; i < Nx; ++i) {
    if (!m[i]) continue;
    const float* src = y + row * (full ? (size_t)i : (size_t)m_);
    float* d = dst + row * (size_t)m_;
    memcpy(d, src, sizeof(float) * row);
    for (size_t e = 0; e < row; ++e) {   // exponent all ones: Inf or NaN
      uint32_t u;
      memcpy(&u, d + e, sizeof(u));
      bad |= (uint32_t)((u & 0x7f800000u) == 0x7f800000u);
    }
    ++m_;
  }
  if (bad) return fail(TTS_ENONFINITE, "frame holds NaN or Inf; not applied%s");
  *out = h->hstage[b];
  return TTS_OK;
}

// Poll a word in mapped host memory until it reads v (acquire), for at most ~10 s; false if
// it never did.
static bool wait_word(unsigned int* w, unsigned int v) {
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned int i = 0;; ++i) {
    if (__atomic_load_n(w, __ATOMIC_ACQUIRE) == v) return true;
    if ((i & 4095u) == 4095u && std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10)) return false;
  }
}

int handle_stage_frame(tts_handle* h, const tts_c64* y_rows, const uint8_t* line_mask, int flags, FrameParams* pout,
                       bool pinned_gather) {
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny;
  FrameParams p = h->fp;
  p.full_frame = (flags & TTS_FULL_FRAME) ? 1 : 0;
  if (flags & TTS_DEVICE_PTRS) {
    if (!line_mask && !h->have_next) return fail(TTS_ESTATE, "no mask given and none drawn yet%s");
    p.mask = line_mask ? line_mask : h->dmask_next;
    p.yrows = (const float2*)y_rows;
  } else {
    const uint8_t* m = line_mask;
    if (!m) {
      if (!h->have_next) return fail(TTS_ESTATE, "no mask given and none drawn yet%s");
      if (!h->next_on_host) {
        CK(cudaMemcpyAsync(h->next_host.data(), h->dmask_next, Nx, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->next_on_host = true;
      }
      m = h->next_host.data();
    }
    int s = 0;
    for (int i = 0; i < Nx; ++i) s += m[i] != 0;
    if (s == 0) return fail(TTS_EINVAL, "the line mask selects no line%s");
    if (pinned_gather && (flags & TTS_HOST_PINNED) && h->cfg.row_dft == TTS_ROWDFT_FFT) {
      // page-locked caller memory: the kernels read the acquired rows in place
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, y_rows) != cudaSuccess || a.type != cudaMemoryTypeHost ||
          a.devicePointer == nullptr) {
        cudaGetLastError();
        return fail(TTS_EINVAL, "TTS_HOST_PINNED: y_rows is not page-locked host memory%s");
      }
      if (line_mask) CK(cudaMemcpyAsync(h->dmask_push, m, Nx, cudaMemcpyHostToDevice, h->stream));
      p.mask = line_mask ? h->dmask_push : h->dmask_next;
      p.yrows = (const float2*)a.devicePointer;
      *pout = p;
      return TTS_OK;
    }
    if (pinned_gather) {
      float2* staged = nullptr;
      const int rg = gather_host_rows(h, (const float*)y_rows, m, (flags & TTS_FULL_FRAME) != 0, &staged);
      if (rg != TTS_OK) return rg;
      const int b = h->hstage_next;
      if (line_mask) CK(cudaMemcpyAsync(h->dmask_push, m, Nx, cudaMemcpyHostToDevice, h->stream));
      if (h->hstage_dev[b]) {
        p.yrows = h->hstage_dev[b];   // read in place by the frame's kernels
        h->hstage_pending = b;        // its event follows their launches (tts_push_frame)
      } else {
        CK(cudaMemcpyAsync(h->ystage, staged, sizeof(float2) * (size_t)s * Ny, cudaMemcpyHostToDevice, h->stream));
        CK(cudaEventRecord(h->hstage_done[b], h->stream));
        p.yrows = h->ystage;
      }
      h->hstage_next ^= 1;
      p.mask = line_mask ? h->dmask_push : h->dmask_next;
      p.full_frame = 0;   // compact rows on the device
      *pout = p;
      return TTS_OK;
    }
    const size_t nrows_in = (flags & TTS_FULL_FRAME) ? (size_t)Nx : (size_t)s;
    const float* f = (const float*)y_rows;
    for (int i = 0, m_ = 0; i < Nx; ++i) {
      if (!m[i]) continue;
      const float* row = f + 2 * (size_t)Ny * ((flags & TTS_FULL_FRAME) ? (size_t)i : (size_t)m_++);
      for (int e = 0; e < 2 * Ny; ++e)
        if (!isfinite(row[e])) return fail(TTS_ENONFINITE, "frame holds NaN or Inf; not applied%s");
    }
    CK(cudaMemcpyAsync(h->dmask_push, m, Nx, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->ystage, y_rows, sizeof(float2) * nrows_in * Ny, cudaMemcpyHostToDevice, h->stream));
    p.mask = h->dmask_push;
    p.yrows = h->ystage;
  }
  *pout = p;
  return TTS_OK;
}

uint64_t handle_draw_counter(const tts_handle* h) {
  return ((uint64_t)(h->cfg.stream_id & 0xFFFFFFu) << 40) | ((uint64_t)h->t & ((1ull << 40) - 1));
}

int handle_k_lines(const tts_handle* h, double rate) {
  return std::max(h->cfg.central_lines, (int)floor(rate * h->cfg.Nx + 0.5));
}

extern "C" {

const char* tts_last_error(void) { return g_err.c_str(); }

void tts_config_init(tts_config* c, int Nx, int Ny, int R, double lambda_forget, double mu) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->Nx = Nx;
  c->Ny = Ny;
  c->R = R;
  c->lambda_forget = lambda_forget;
  c->mu = mu;
  c->mm_iters = 1;
  c->central_lines = 8;
  c->policy = TTS_POLICY_INFORMATIVE;
  c->vd_alpha = -1.0;
  c->with_replacement = 0;
  c->update = TTS_UPDATE_GAUSS_SEIDEL;
  c->launch = TTS_LAUNCH_FUSED;
  c->cluster_ctas = 0;
  c->init_seed = 0;
  c->stream_id = 0;
  c->cuda_stream = nullptr;
  c->row_dft = TTS_ROWDFT_FFT;
  c->kspace = 0;
  c->ridge_precision = TTS_RIDGE_FF_LAST;
}

int tts_create(int Nx, int Ny, int R, double lambda_forget, double mu, tts_handle** out) {
  tts_config c;
  tts_config_init(&c, Nx, Ny, R, lambda_forget, mu);
  return tts_create_ex(&c, out);
}

int tts_create_ex(const tts_config* cfg, tts_handle** out) { return handle_create(cfg, nullptr, out); }

void tts_destroy(tts_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  mc_detach(h);
  for (int b = 0; b < 2; ++b) {
    if (h->hstage[b]) cudaFreeHost(h->hstage[b]);
    if (h->hstage_done[b]) cudaEventDestroy(h->hstage_done[b]);
  }
  if (h->mask_map) cudaFreeHost(h->mask_map);
  if (h->own_mem) cudaFree(h->dmem);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

int tts_set_factors(tts_handle* h, const tts_c64* A, const tts_c64* B, int flags) {
  if (!h || !A || !B) return fail(TTS_EINVAL, "NULL argument%s");
  const cudaMemcpyKind k = (flags & TTS_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(h->fp.A, A, sizeof(float2) * h->cfg.Nx * h->cfg.R, k, h->stream));
  CK(cudaMemcpyAsync(h->fp.B, B, sizeof(float2) * h->cfg.Ny * h->cfg.R, k, h->stream));
  if (!(flags & TTS_DEVICE_PTRS)) CK(cudaStreamSynchronize(h->stream));
  return TTS_OK;
}

int tts_get_factors(tts_handle* h, tts_c64* A, tts_c64* B, int flags) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  const cudaMemcpyKind k = (flags & TTS_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (A) CK(cudaMemcpyAsync(A, h->fp.A, sizeof(float2) * h->cfg.Nx * h->cfg.R, k, h->stream));
  if (B) CK(cudaMemcpyAsync(B, h->fp.B, sizeof(float2) * h->cfg.Ny * h->cfg.R, k, h->stream));
  if (!(flags & TTS_DEVICE_PTRS)) CK(cudaStreamSynchronize(h->stream));
  return TTS_OK;
}

int tts_get_stats(tts_handle* h, double* abar_A, double* abar_B, double* w, int64_t* t) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  double sc[SC_COUNT];
  CK(cudaMemcpyAsync(sc, h->fp.sc, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (abar_A) *abar_A = sc[SC_ABAR_A];
  if (abar_B) *abar_B = sc[SC_ABAR_B];
  if (w) *w = sc[SC_W];
  if (t) *t = h->t;
  return TTS_OK;
}

int tts_set_stats(tts_handle* h, double abar_A, double abar_B, double w, int64_t t) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  if (!(abar_A >= 0.0) || !(abar_B >= 0.0) || !(w >= 0.0) || t < 0) return fail(TTS_EINVAL, "statistics must be non-negative%s");
  double sc[SC_COUNT] = {0};
  sc[SC_W] = w;
  sc[SC_ABAR_A] = abar_A;
  sc[SC_ABAR_B] = abar_B;
  sc[SC_T] = (double)t;
  CK(cudaMemcpyAsync(h->fp.sc, sc, sizeof(sc), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->t = t;
  return TTS_OK;
}

int tts_get_gamma(tts_handle* h, tts_c64* gamma) {
  if (!h || !gamma) return fail(TTS_EINVAL, "NULL argument%s");
  CK(cudaMemcpyAsync(gamma, h->fp.gamma, sizeof(float2) * h->cfg.R, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return TTS_OK;
}

int tts_get_gamma_fp64(tts_handle* h, double* gamma) {
  if (!h || !gamma) return fail(TTS_EINVAL, "NULL argument%s");
  CK(cudaMemcpyAsync(gamma, h->fp.gamma_d, sizeof(double2) * h->cfg.R, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return TTS_OK;
}

int tts_get_ridge_operands(tts_handle* h, tts_c64* Ahat_S, tts_c64* Yt, int* rows, int* nrows) {
  if (!h || !Ahat_S || !Yt || !rows || !nrows) return fail(TTS_EINVAL, "NULL argument%s");
  if (h->mc) return fail(TTS_EINVAL, "the multi-coil tracker has no separable operands%s");
  int s = 0;
  CK(cudaMemcpyAsync(&s, h->fp.nrows, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (s < 0 || s > h->cfg.Nx) return fail(TTS_ESTATE, "no frame processed yet%s");
  *nrows = s;
  CK(cudaMemcpyAsync(Ahat_S, h->fp.AhS[0], sizeof(float2) * (size_t)s * h->cfg.R, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(Yt, h->fp.Yt, sizeof(float2) * (size_t)s * h->cfg.Ny, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(rows, h->fp.rows, sizeof(int) * (size_t)s, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return TTS_OK;
}

int tts_get_config(tts_handle* h, tts_config* cfg) {
  if (!h || !cfg) return fail(TTS_EINVAL, "NULL argument%s");
  *cfg = h->cfg;
  cfg->cluster_ctas = h->fp.C;
  cfg->cuda_stream = (void*)h->stream;
  return TTS_OK;
}

int tts_set_coil_maps(tts_handle* h, const tts_c64* maps, int C, int flags) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  if (h->in_engine) return fail(TTS_EINVAL, "engine streams are single-coil%s");
  if (h->cfg.kspace) return fail(TTS_EINVAL, "the k-space tracker is single-coil%s");
  if (flags & ~TTS_DEVICE_PTRS) return fail(TTS_EINVAL, "unknown flags%s");
  if (!maps || C == 0) {
    CK(cudaStreamSynchronize(h->stream));
    mc_detach(h);
    return TTS_OK;
  }
  if (C < 1 || C > TTS_MAX_COILS) return fail(TTS_EINVAL, "C must be 1..64%s");
  if (h->cfg.update != TTS_UPDATE_GAUSS_SEIDEL || h->cfg.row_dft != TTS_ROWDFT_FFT)
    return fail(TTS_EINVAL, "the multi-coil tracker runs Gauss-Seidel iterations with the FFT row transform%s");
  if ((size_t)h->cfg.R * (h->cfg.Ny + 1) + h->cfg.Ny > 16384 + 512)
    return fail(TTS_EINVAL, "the multi-coil tracker needs R (Ny + 1) <= 16384%s");
  CK(cudaStreamSynchronize(h->stream));
  return mc_attach(h, (const float2*)maps, C, (flags & TTS_DEVICE_PTRS) != 0);
}

int tts_push_frame(tts_handle* h, const tts_c64* y_rows, const uint8_t* line_mask, int flags) {
  if (!h || !y_rows) return fail(TTS_EINVAL, "NULL argument%s");
  if (h->mc) return mc_push(h, y_rows, line_mask, flags);
  if (h->cfg.row_dft != TTS_ROWDFT_FFT && (flags & TTS_DEVICE_PTRS) && (uintptr_t)y_rows % 16 != 0)
    return fail(TTS_EINVAL, "the tensor-core row transform reads 16-byte aligned device rows%s");
  FrameParams p;
  const int rs = handle_stage_frame(h, y_rows, line_mask, flags, &p, true);
  if (rs != TTS_OK) return rs;
  // a staging buffer the kernels read in place is free again once they are done
  auto release_staging = [h]() {
    if (h->hstage_pending >= 0) {
      cudaEventRecord(h->hstage_done[h->hstage_pending], h->stream);
      h->hstage_pending = -1;
    }
  };
  if (h->cfg.row_dft != TTS_ROWDFT_FFT) {
    // the acquired rows' transform on the tensor cores, straight into Yt; it reports a wait
    // that ran out in the frame's own status word, which the frame kernel reads (and then
    // skips the frame and raises the handle's sticky timeout word)
    int* frame_tmo = p.status + 2 + TTS_MAX_CLUSTER;
    const int withhold = h->test_withhold;
    const long long limit = withhold >= 0 ? h->test_wait_cycles : 2000000000LL;
    h->test_withhold = -1;
    if (cudaMemsetAsync(frame_tmo, 0, sizeof(int), h->stream) != cudaSuccess) {
      release_staging();
      return fail(TTS_ECUDA, "status reset failed%s");
    }
    const int rr = launch_row_dft(p.yrows, p.Yt, p.mask, h->cfg.Nx, h->cfg.Ny, p.full_frame,
                                  h->cfg.row_dft == TTS_ROWDFT_BF16X3 ? 1 : 0, frame_tmo, h->stream, withhold, limit);
    if (rr != TTS_OK) {
      release_staging();
      return fail(rr, "row transform launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    p.yt_ready = 1;
  }
  const int rc = launch_frame(p, h->cfg.launch, h->stream);
  release_staging();
  if (rc != TTS_OK) return fail(rc, "frame kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->t += 1;
  return TTS_OK;
}

int tts_image(tts_handle* h, int64_t t, tts_c64* out, int flags) {
  if (!h || !out) return fail(TTS_EINVAL, "NULL argument%s");
  if (h->t == 0 || t != h->t - 1) return fail(TTS_ERANGE, "only the most recent frame's image is available%s");
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny;
  float2* dst = (flags & TTS_DEVICE_PTRS) ? (float2*)out : h->X;
  int rc = launch_image(h->fp.A, h->fp.B, h->fp.gamma, dst, Nx, Ny, h->cfg.R, h->stream);
  if (rc != TTS_OK) return fail(rc, "image kernel launch failed%s");
  if (h->cfg.kspace) {
    // Alg. 2: the interpolated k-space frame back to the image domain
    rc = tts_fft2d((const tts_c64*)dst, (tts_c64*)dst, 1, Nx, Ny, 1, h->stream);
    if (rc != TTS_OK) return rc;
  }
  if (!(flags & TTS_DEVICE_PTRS)) {
    CK(cudaMemcpyAsync(out, h->X, sizeof(float2) * (size_t)Nx * Ny, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return TTS_OK;
}

int tts_next_mask(tts_handle* h, double rate, uint64_t seed, uint8_t* line_mask_out, int flags) {
  if (!h || !line_mask_out) return fail(TTS_EINVAL, "NULL argument%s");
  if (!(rate > 0.0 && rate <= 1.0)) return fail(TTS_EINVAL, "rate must lie in (0, 1]%s");
  const int Nx = h->cfg.Nx;
  const int k_lines = handle_k_lines(h, rate);
  const bool host = !(flags & TTS_DEVICE_PTRS);
  if (host) {
    // a host mask is a wait for the draw, which a stream being captured never runs
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return fail(TTS_ESTATE, "a host line mask cannot be drawn while the stream is captured%s");
    }
  }
  if (host && !h->mask_map) {
    uint8_t* m = nullptr;
    void* d = nullptr;
    const size_t at = ((size_t)Nx + 63) & ~(size_t)63;   // the completion word after the mask
    if (cudaHostAlloc((void**)&m, at + 64, cudaHostAllocMapped) == cudaSuccess) {
      if (cudaHostGetDevicePointer(&d, m, 0) == cudaSuccess) {
        h->mask_map = m;
        h->mask_map_dev = (uint8_t*)d;
        h->draw_done = (unsigned int*)(m + at);
        h->draw_done_dev = (unsigned int*)((uint8_t*)d + at);
        *h->draw_done = h->draw_seq;
      } else {
        cudaFreeHost(m);
      }
    }
    cudaGetLastError();   // without mapped memory the mask is copied back instead
  }
  uint8_t* out2 = host ? h->mask_map_dev : line_mask_out;
  const unsigned int seq = h->draw_seq + 1;
  int rc = launch_sampler(h->fp.A, Nx, h->cfg.Ny, h->cfg.R, nullptr, h->dp, h->cfg.policy, h->cfg.vd_alpha, k_lines,
                          h->cfg.central_lines, seed, handle_draw_counter(h), h->cfg.with_replacement, h->fp.Wx,
                          h->dmask_next, out2, h->stream, h->cfg.kspace, host ? h->draw_done_dev : nullptr, seq);
  if (rc != TTS_OK) return fail(rc, "sampler kernel launch failed%s");
  h->have_next = true;
  if (flags & TTS_DEVICE_PTRS) {
    h->next_on_host = false;
  } else {
    if (!h->mask_map) CK(cudaMemcpyAsync(h->next_host.data(), h->dmask_next, Nx, cudaMemcpyDeviceToHost, h->stream));
    // the mask is on the host once the sampler has set its completion word: poll that word
    // (the scanner waits on these lines) instead of synchronising the stream; a stream
    // synchronisation after a bounded wait reports any error of the work before it
    if (!(h->mask_map && wait_word(h->draw_done, seq))) CK(cudaStreamSynchronize(h->stream));
    if (h->mask_map && __atomic_load_n(h->draw_done, __ATOMIC_ACQUIRE) != seq)
      return fail(TTS_ECUDA, "the line draw did not complete%s");
    h->draw_seq = seq;
    if (h->mask_map) memcpy(h->next_host.data(), h->mask_map, Nx);
    memcpy(line_mask_out, h->next_host.data(), Nx);
    h->next_on_host = true;
  }
  return TTS_OK;
}

int tts_line_probs(tts_handle* h, double* p, int flags) {
  if (!h || !p) return fail(TTS_EINVAL, "NULL argument%s");
  const int Nx = h->cfg.Nx;
  double* dst = (flags & TTS_DEVICE_PTRS) ? p : h->dp;
  int rc = launch_sampler(h->fp.A, Nx, h->cfg.Ny, h->cfg.R, nullptr, dst, h->cfg.policy, h->cfg.vd_alpha, 0,
                          h->cfg.central_lines, 0, 0, 0, h->fp.Wx, h->dmask_next, nullptr, h->stream, h->cfg.kspace);
  if (rc != TTS_OK) return fail(rc, "sampler kernel launch failed%s");
  if (!(flags & TTS_DEVICE_PTRS)) {
    CK(cudaMemcpyAsync(p, h->dp, sizeof(double) * Nx, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return TTS_OK;
}

int tts_sample_lines_from_probs(const double* p, int Nx, int k_lines, int central, uint64_t seed, uint64_t ctr,
                                int with_replacement, uint8_t* out, int flags) {
  if (!p || !out) return fail(TTS_EINVAL, "NULL argument%s");
  if (Nx < 1 || Nx > TTS_MAX_N) return fail(TTS_EINVAL, "Nx must be 1..512%s");
  if (k_lines < 0 || central < 0 || central > Nx) return fail(TTS_EINVAL, "bad k_lines or central%s");
  if (flags & TTS_DEVICE_PTRS) {
    int rc = launch_sampler(nullptr, Nx, 1, 1, p, nullptr, TTS_POLICY_UNIFORM, -1.0, std::max(k_lines, 1), central,
                            seed, ctr, with_replacement, nullptr, out, nullptr, 0);
    return rc == TTS_OK ? TTS_OK : fail(rc, "sampler kernel launch failed%s");
  }
  for (int i = 0; i < Nx; ++i)
    if (!(p[i] >= 0.0) || !isfinite(p[i])) return fail(TTS_EINVAL, "probabilities must be finite and >= 0%s");
  double* dp = nullptr;
  uint8_t* dm = nullptr;
  CK(cudaMalloc(&dp, sizeof(double) * Nx));
  cudaError_t e = cudaMalloc(&dm, Nx);
  if (e != cudaSuccess) {
    cudaFree(dp);
    return cuda_fail(e, "cudaMalloc");
  }
  int rc = TTS_OK;
  e = cudaMemcpy(dp, p, sizeof(double) * Nx, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    rc = launch_sampler(nullptr, Nx, 1, 1, dp, nullptr, TTS_POLICY_UNIFORM, -1.0, std::max(k_lines, 1), central, seed,
                        ctr, with_replacement, nullptr, dm, nullptr, 0);
    if (rc == TTS_OK) e = cudaMemcpy(out, dm, Nx, cudaMemcpyDeviceToHost);
  }
  cudaFree(dp);
  cudaFree(dm);
  if (e != cudaSuccess) return cuda_fail(e, "sample_lines_from_probs");
  if (rc != TTS_OK) return fail(rc, "sampler kernel launch failed%s");
  return TTS_OK;
}

// ---- checkpoint ---------------------------------------------------------------------
namespace {
struct SaveHeader {
  char magic[8];
  int32_t Nx, Ny, R, mm_iters, central, policy, update, launch, C, with_repl;
  double lf, mu, vd_alpha;
  uint64_t init_seed;
  uint32_t stream_id;
  int32_t have_next;
  int64_t t;
};
const char kMagic[8] = {'T', 'T', 'S', 'S', 'T', 'A', 'T', '1'};
}  // namespace

int tts_save(tts_handle* h, void* buf, size_t* len) {
  if (!h || !len) return fail(TTS_EINVAL, "NULL argument%s");
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny, R = h->cfg.R;
  const size_t need = sizeof(SaveHeader) + sizeof(double) * SC_COUNT + Nx + sizeof(float2) * ((size_t)Nx * R + (size_t)Ny * R + R);
  if (!buf) {
    *len = need;
    return TTS_OK;
  }
  if (*len < need) return fail(TTS_EINVAL, "buffer too small for the checkpoint%s");
  SaveHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, 8);
  hd.Nx = Nx; hd.Ny = Ny; hd.R = R; hd.mm_iters = h->cfg.mm_iters; hd.central = h->cfg.central_lines;
  hd.policy = h->cfg.policy; hd.update = h->cfg.update; hd.launch = h->cfg.launch; hd.C = h->cfg.cluster_ctas;
  hd.with_repl = h->cfg.with_replacement; hd.lf = h->cfg.lambda_forget; hd.mu = h->cfg.mu; hd.vd_alpha = h->cfg.vd_alpha;
  hd.init_seed = h->cfg.init_seed; hd.stream_id = h->cfg.stream_id; hd.have_next = h->have_next; hd.t = h->t;
  char* o = (char*)buf;
  memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  CK(cudaMemcpyAsync(o, h->fp.sc, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, h->stream));
  o += sizeof(double) * SC_COUNT;
  CK(cudaMemcpyAsync(o, h->dmask_next, Nx, cudaMemcpyDeviceToHost, h->stream));
  o += Nx;
  CK(cudaMemcpyAsync(o, h->fp.A, sizeof(float2) * Nx * R, cudaMemcpyDeviceToHost, h->stream));
  o += sizeof(float2) * Nx * R;
  CK(cudaMemcpyAsync(o, h->fp.B, sizeof(float2) * Ny * R, cudaMemcpyDeviceToHost, h->stream));
  o += sizeof(float2) * Ny * R;
  CK(cudaMemcpyAsync(o, h->fp.gamma, sizeof(float2) * R, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *len = need;
  return TTS_OK;
}

int tts_load(tts_handle* h, const void* buf, size_t len) {
  if (!h || !buf) return fail(TTS_EINVAL, "NULL argument%s");
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny, R = h->cfg.R;
  const size_t need = sizeof(SaveHeader) + sizeof(double) * SC_COUNT + Nx + sizeof(float2) * ((size_t)Nx * R + (size_t)Ny * R + R);
  if (len < need) return fail(TTS_EINVAL, "checkpoint is truncated%s");
  SaveHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  if (memcmp(hd.magic, kMagic, 8) != 0) return fail(TTS_EINVAL, "not a tracker checkpoint%s");
  if (hd.Nx != Nx || hd.Ny != Ny || hd.R != R) return fail(TTS_EINVAL, "checkpoint has other Nx, Ny or R%s");
  const char* i = (const char*)buf + sizeof(hd);
  CK(cudaMemcpyAsync(h->fp.sc, i, sizeof(double) * SC_COUNT, cudaMemcpyHostToDevice, h->stream));
  i += sizeof(double) * SC_COUNT;
  CK(cudaMemcpyAsync(h->dmask_next, i, Nx, cudaMemcpyHostToDevice, h->stream));
  memcpy(h->next_host.data(), i, Nx);
  i += Nx;
  CK(cudaMemcpyAsync(h->fp.A, i, sizeof(float2) * Nx * R, cudaMemcpyHostToDevice, h->stream));
  i += sizeof(float2) * Nx * R;
  CK(cudaMemcpyAsync(h->fp.B, i, sizeof(float2) * Ny * R, cudaMemcpyHostToDevice, h->stream));
  i += sizeof(float2) * Ny * R;
  CK(cudaMemcpyAsync(h->fp.gamma, i, sizeof(float2) * R, cudaMemcpyHostToDevice, h->stream));
  // the drawn mask on the device too (a push with no mask reads the device copy)
  CK(cudaMemcpyAsync(h->dmask_next, h->next_host.data(), Nx, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->t = hd.t;
  h->have_next = hd.have_next != 0;
  h->next_on_host = true;
  return TTS_OK;
}

int tts_synchronize(tts_handle* h) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  int st = 0, tmo = 0;
  CK(cudaMemcpyAsync(&st, h->fp.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&tmo, h->fp.status + 1 + TTS_MAX_CLUSTER, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (tmo) {
    CK(cudaMemsetAsync(h->fp.status + 1 + TTS_MAX_CLUSTER, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(TTS_ETIMEOUT, "a bounded wait of the tensor-core row transform ran out%s");
  }
  if (st) {
    CK(cudaMemsetAsync(h->fp.status, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(TTS_ENONFINITE, "a frame held NaN or Inf and was skipped%s");
  }
  return TTS_OK;
}

int tts_launches_per_frame(tts_handle* h) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  return h->cfg.launch == TTS_LAUNCH_FUSED ? 1 : frame_num_steps(h->cfg.mm_iters);
}

int tts_ridge_solve(const double* G, const double* h, int R, double* gamma) {
  if (!G || !h || !gamma) return fail(TTS_EINVAL, "NULL argument%s");
  if (R < 1 || R > TTS_MAX_R) return fail(TTS_EINVAL, "R must be 1..64%s");
  double2 *dG = nullptr, *dh = nullptr, *dg = nullptr;
  const size_t bG = sizeof(double2) * R * R, bh = sizeof(double2) * R;
  CK(cudaMalloc(&dG, bG + 2 * bh));
  dh = dG + R * R;
  dg = dh + R;
  cudaError_t e = cudaMemcpy(dG, G, bG, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dh, h, bh, cudaMemcpyHostToDevice);
  int rc = TTS_OK;
  if (e == cudaSuccess) rc = launch_ridge(dG, dh, R, dg, 0);
  if (e == cudaSuccess && rc == TTS_OK) e = cudaMemcpy(gamma, dg, bh, cudaMemcpyDeviceToHost);
  cudaFree(dG);
  if (e != cudaSuccess) return cuda_fail(e, "ridge_solve");
  if (rc != TTS_OK) return fail(rc, "ridge kernel launch failed%s");
  return TTS_OK;
}

// ---- standalone batched 2D DFT ----------------------------------------------------
namespace {
std::mutex g_status_mu;
int* g_status[64];

// A device status word per device for the standalone transforms' bounded waits.
int* device_status(int* rc) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) {
    *rc = TTS_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!g_status[dev]) {
    if (cudaMalloc(&g_status[dev], sizeof(int)) != cudaSuccess || cudaMemset(g_status[dev], 0, sizeof(int)) != cudaSuccess) {
      *rc = TTS_ECUDA;
      return nullptr;
    }
  }
  return g_status[dev];
}
std::mutex g_tw_mu;
struct TwEntry {
  int dev, n;
  float2* d;
};
std::vector<TwEntry> g_tw;

const float2* device_twiddles(int n, int* rc) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tw_mu);
  for (auto& e : g_tw)
    if (e.dev == dev && e.n == n) return e.d;
  std::vector<float2> w = twiddles(n);
  float2* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(float2) * n);
  if (e == cudaSuccess) e = cudaMemcpy(d, w.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "twiddle table");
    return nullptr;
  }
  g_tw.push_back({dev, n, d});
  return d;
}
}  // namespace

int tts_fft2d(const tts_c64* in, tts_c64* out, int batch, int Nx, int Ny, int inverse, void* cuda_stream) {
  if (!in || !out) return fail(TTS_EINVAL, "NULL argument%s");
  if (batch < 0 || Nx < 1 || Ny < 1 || Nx > TTS_MAX_N || Ny > TTS_MAX_N || !smooth235(Nx) || !smooth235(Ny))
    return fail(TTS_EINVAL, "sizes must be 1..512 with prime factors in {2,3,5}%s");
  if (batch == 0) return TTS_OK;
  int rc = TTS_OK;
  const float2* wx = device_twiddles(Nx, &rc);
  if (!wx) return rc;
  const float2* wy = device_twiddles(Ny, &rc);
  if (!wy) return rc;
  if (fft2d_square_ok(Nx, Ny)) {
    int* st = device_status(&rc);
    if (!st) return fail(rc, "device status word%s");
    rc = launch_fft2d_square((const float2*)in, (float2*)out, batch, Nx, inverse, wx, st, (cudaStream_t)cuda_stream);
  } else if (fft2d_lines_ok(Nx, Ny)) {
    rc = launch_fft2d_lines((const float2*)in, (float2*)out, batch, Nx, Ny, inverse, wx, wy, (cudaStream_t)cuda_stream);
  } else {
    rc = launch_fft2d((const float2*)in, (float2*)out, batch, Nx, Ny, inverse, wx, wy, nullptr,
                      (cudaStream_t)cuda_stream);
  }
  return rc == TTS_OK ? TTS_OK : fail(rc, "fft kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
}


int tts_fft2d_autotune(int N, int batch, int inverse, int reps, double* best_ms, int* per_sm, double* lag) {
  if (!fft2d_square_ok(N, N)) return fail(TTS_EINVAL, "the autotuner covers the square band-task sizes%s");
  if (batch < 1 || reps < 1) return fail(TTS_EINVAL, "batch and reps must be positive%s");
  int rc = TTS_OK;
  const float2* w = device_twiddles(N, &rc);
  if (!w) return rc;
  int* st = device_status(&rc);
  if (!st) return fail(rc, "device status word%s");
  float2* buf = nullptr;
  const size_t n = (size_t)batch * N * N;
  CK(cudaMalloc(&buf, 2 * n * sizeof(float2)));
  cudaError_t e = cudaMemset(buf, 0, 2 * n * sizeof(float2));
  if (e == cudaSuccess)
    rc = tune_fft2d_square(buf, buf + n, batch, N, inverse, w, st, reps, best_ms, per_sm, lag);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "autotune buffers");
  return rc == TTS_OK ? TTS_OK : fail(rc, "autotune launch failed%s");
}

int tts_test_withheld_wait(int kind, const tts_c64* in, tts_c64* out, tts_c64* tmp, int batch, int N, int index,
                           long long wait_cycles, int* dev_status, void* cuda_stream) {
  if (!in || !out || !dev_status) return fail(TTS_EINVAL, "NULL argument%s");
  if (batch < 1 || index < 0 || wait_cycles < 1) return fail(TTS_EINVAL, "bad batch, index or wait_cycles%s");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (kind == 0) {
    if (!fft2d_square_ok(N, N) || index >= batch) return fail(TTS_EINVAL, "kind 0: square band size, index < batch%s");
    int rc = TTS_OK;
    const float2* w = device_twiddles(N, &rc);
    if (!w) return rc;
    rc = launch_fft2d_square((const float2*)in, (float2*)out, batch, N, 0, w, dev_status, st, index, wait_cycles);
    return rc == TTS_OK ? TTS_OK : fail(rc, "square FFT launch failed%s");
  }
  if (kind == 1) {
    if (!tmp || !dft_gemm_size_ok(N) || index >= 2 * N / 16) return fail(TTS_EINVAL, "kind 1: N, tmp, chunk index%s");
    if (((uintptr_t)in | (uintptr_t)out | (uintptr_t)tmp) % 16 != 0) return fail(TTS_EINVAL, "16-byte alignment%s");
    const int rc = launch_dft2d_gemm((const float2*)in, (float2*)out, (float2*)tmp, batch, N, N, 0, 1, dev_status, st,
                                     index, wait_cycles);
    return rc == TTS_OK ? TTS_OK : fail(rc, "tensor-core DFT launch failed%s");
  }
  return fail(TTS_EINVAL, "kind must be 0 or 1%s");
}

int tts_test_withhold_row_transform(tts_handle* h, int chunk, long long wait_cycles) {
  if (!h) return fail(TTS_EINVAL, "NULL handle%s");
  if (h->cfg.row_dft == TTS_ROWDFT_FFT) return fail(TTS_EINVAL, "the handle has no tensor-core row transform%s");
  if (chunk < 0 || chunk >= 2 * h->cfg.Ny / 16 || wait_cycles < 1) return fail(TTS_EINVAL, "bad chunk or wait_cycles%s");
  h->test_withhold = chunk;
  h->test_wait_cycles = wait_cycles;
  return TTS_OK;
}

int tts_dft2d_gemm(const tts_c64* in, tts_c64* out, tts_c64* tmp, int batch, int Nx, int Ny, int inverse,
                   int precision, int* dev_status, void* cuda_stream) {
  if (!in || !out || !tmp) return fail(TTS_EINVAL, "NULL argument%s");
  if (batch < 0 || !dft_gemm_size_ok(Nx) || !dft_gemm_size_ok(Ny))
    return fail(TTS_EINVAL, "sizes must be multiples of 32 in [32, 256]%s");
  if (precision != TTS_DFT_BF16X3 && precision != TTS_DFT_BF16) return fail(TTS_EINVAL, "unknown precision%s");
  if ((const void*)tmp == (const void*)in || (const void*)tmp == (const void*)out)
    return fail(TTS_EINVAL, "tmp must not alias in or out%s");
  if (((uintptr_t)in | (uintptr_t)out | (uintptr_t)tmp) % 16 != 0)
    return fail(TTS_EINVAL, "in, out and tmp must be 16-byte aligned%s");
  if (batch == 0) return TTS_OK;
  int* st = dev_status;
  if (!st) {
    int rs = TTS_OK;
    st = device_status(&rs);
    if (!st) return fail(rs, "device status word%s");
  }
  const int rc = launch_dft2d_gemm((const float2*)in, (float2*)out, (float2*)tmp, batch, Nx, Ny, inverse,
                                   precision == TTS_DFT_BF16X3 ? 1 : 0, st, (cudaStream_t)cuda_stream);
  return rc == TTS_OK ? TTS_OK : fail(rc, "tensor-core DFT launch failed: %s", cudaGetErrorString(cudaGetLastError()));
}

}  // extern "C"
