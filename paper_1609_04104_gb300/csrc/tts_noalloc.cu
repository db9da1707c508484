// Frame update that allocates nothing: the caller passes the tracker state and the frame
// in device memory, and every temporary the frame kernel needs lives in one fixed
// file-scope device array. For callers that cannot allocate device memory at run time,
// e.g. code running under an allocator they do not control, inside a pre-sized real-time
// budget, or that must not trigger the implicit synchronisation of cudaMalloc/cudaFree.
#include <math.h>
#include <string.h>

#include <mutex>

#include "tts_internal.cuh"

namespace {

// Largest problem the fixed scratch serves (see tts.h): Nx, Ny <= 256, R <= 32, which
// the frame kernel runs on a cluster of at most 8 CTAs.
constexpr int kMaxN = TTS_NOALLOC_MAX_N;
constexpr int kMaxR = TTS_NOALLOC_MAX_R;
constexpr int kMaxC = 8;

size_t up(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of scratch a problem of the given size uses (same pieces as a tracker handle,
// without the factors, the statistics and gamma, which the caller owns).
size_t scratch_bytes(int Nx, int Ny, int R, int C) {
  size_t b = 0;
  b += up(sizeof(float2) * Nx) + up(sizeof(float2) * Ny);                 // twiddles
  b += up(sizeof(float2) * Nx * R) + up(sizeof(float2) * Ny * R);         // anchors
  b += up(sizeof(float2) * (size_t)Nx * Ny);                              // Yt
  b += up(sizeof(int) * Nx) + up(sizeof(int) * 4);                        // rows, |S|
  b += 2 * up(sizeof(float2) * Nx * R) + 2 * up(sizeof(float) * R);       // AhS, nA
  b += 2 * (up(sizeof(float2) * R * R) + up(sizeof(float2) * Nx * R));    // MB, P (hi, lo)
  b += 2 * up(sizeof(float2) * R * R);                                     // MA (hi, lo)
  b += up(sizeof(float2) * (size_t)C * Nx * R) + up(sizeof(float) * C * R);  // partials of A
  b += up(sizeof(float4) * (size_t)C * R * R) + up(sizeof(float4) * (size_t)C * Nx * R);  // partials of B
  b += up(sizeof(float4) * (size_t)C * R * R);                             // partials of MA
  b += up(sizeof(double) * SF_COUNT) + up(sizeof(double2) * R);           // frame scalars, gamma (FP64)
  b += up(sizeof(int) * (3 + TTS_MAX_CLUSTER));                           // status words
  return b;
}

}  // namespace

// The shared scratch of every tts_push_frame_noalloc call on a device. Each GPU that
// loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TTS_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_mu;
void* g_addr[64];         // device address of g_noalloc_scratch, per device ordinal

// Per call, before the frame kernel: the twiddle tables exp(-2 pi i k / N) of this call's
// sizes (from double-precision sincospi, rounded to float) and the zeroed status words,
// written into the scratch on the device, so the call copies nothing from host memory.
__global__ void noalloc_setup_kernel(float2* Wx, int Nx, float2* Wy, int Ny, int* status, int nstatus) {
  const int n = Nx + Ny + nstatus;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    if (k < Nx + Ny) {
      const bool x = k < Nx;
      const int i = x ? k : k - Nx, N = x ? Nx : Ny;
      double sn, cs;
      sincospi(2.0 * (double)i / (double)N, &sn, &cs);
      (x ? Wx : Wy)[i] = make_float2((float)cs, (float)-sn);
    } else {
      status[k - Nx - Ny] = 0;
    }
  }
}

int na_fail(int code, const char* msg) {
  tts_internal_set_error(msg);
  return code;
}

// Host code only knows g_noalloc_scratch as a host-side stand-in symbol: its device
// address is looked up once per device, with that device current.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TTS_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TTS_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TTS_OK;
}

bool smooth235(int n) {
  if (n < 1) return false;
  for (int q : {2, 3, 5})
    while (n % q == 0) n /= q;
  return n == 1;
}

}  // namespace

extern "C" int tts_push_frame_noalloc(const tts_frame_args* a, void* cuda_stream) {
  if (!a || !a->A || !a->B || !a->stats || !a->gamma || !a->y_rows || !a->line_mask)
    return na_fail(TTS_EINVAL, "tts_push_frame_noalloc: NULL argument");
  if (a->Nx < 1 || a->Ny < 1 || a->Nx > kMaxN || a->Ny > kMaxN || !smooth235(a->Nx) || !smooth235(a->Ny))
    return na_fail(TTS_EINVAL,
                   "tts_push_frame_noalloc: Nx and Ny must be 1..256 with prime factors in {2,3,5} "
                   "(the fixed scratch holds no larger frame)");
  if (a->R < 1 || a->R > kMaxR)
    return na_fail(TTS_EINVAL, "tts_push_frame_noalloc: R must be 1..32 (the fixed scratch holds no larger rank)");
  if (!(a->lambda_forget > 0.0 && a->lambda_forget <= 1.0) || !(a->mu > 0.0) || a->mm_iters < 1 ||
      a->mm_iters > 1000 || (a->update != TTS_UPDATE_GAUSS_SEIDEL && a->update != TTS_UPDATE_JACOBI) ||
      (a->flags & ~TTS_FULL_FRAME))
    return na_fail(TTS_EINVAL, "tts_push_frame_noalloc: bad lambda_forget, mu, mm_iters, update or flags");
  const int Nx = a->Nx, Ny = a->Ny, R = a->R;
  // the parameters a tracker handle would use for the same sizes
  FrameParams p;
  memset(&p, 0, sizeof(p));
  p.Nx = Nx;
  p.Ny = Ny;
  p.R = R;
  if (frame_configure(p, 0) != TTS_OK || p.C > kMaxC)
    return na_fail(TTS_EINVAL, "tts_push_frame_noalloc: no frame configuration fits the fixed scratch");
  if (scratch_bytes(Nx, Ny, R, p.C) > sizeof(g_noalloc_scratch))
    return na_fail(TTS_EINVAL, "tts_push_frame_noalloc: problem exceeds the fixed scratch");
  p.K = a->mm_iters;
  p.refine = 5;
  p.ridge_ff_all = 1;
  p.jacobi = a->update == TTS_UPDATE_JACOBI;
  p.lf = a->lambda_forget;
  p.mu = a->mu;
  p.isx = (float)(1.0 / sqrt((double)Nx));
  p.isy = (float)(1.0 / sqrt((double)Ny));
  p.plan_y = fft_plan(Ny);
  p.A = (float2*)a->A;
  p.B = (float2*)a->B;
  p.sc = a->stats;
  p.gamma = (float2*)a->gamma;
  p.yrows = (const float2*)a->y_rows;
  p.mask = a->line_mask;
  p.full_frame = (a->flags & TTS_FULL_FRAME) ? 1 : 0;

  void* base = nullptr;
  if (scratch_address(&base) != TTS_OK)
    return na_fail(TTS_ECUDA, "tts_push_frame_noalloc: cannot resolve the device scratch");
  char* q = (char*)base;
  auto take = [&](size_t bytes) {
    void* r = q;
    q += up(bytes);
    return r;
  };
  float2* Wx = (float2*)take(sizeof(float2) * Nx);
  float2* Wy = (float2*)take(sizeof(float2) * Ny);
  p.Wx = Wx;
  p.Wy = Wy;
  p.A0 = (float2*)take(sizeof(float2) * Nx * R);
  p.B0 = (float2*)take(sizeof(float2) * Ny * R);
  p.Yt = (float2*)take(sizeof(float2) * (size_t)Nx * Ny);
  p.rows = (int*)take(sizeof(int) * Nx);
  p.nrows = (int*)take(sizeof(int) * 4);
  p.AhS[0] = (float2*)take(sizeof(float2) * Nx * R);
  p.AhS[1] = (float2*)take(sizeof(float2) * Nx * R);
  p.nA[0] = (float*)take(sizeof(float) * R);
  p.nA[1] = (float*)take(sizeof(float) * R);
  p.MB = (float2*)take(sizeof(float2) * R * R);
  p.P = (float2*)take(sizeof(float2) * Nx * R);
  p.MBlo = (float2*)take(sizeof(float2) * R * R);
  p.Plo = (float2*)take(sizeof(float2) * Nx * R);
  p.MA = (float2*)take(sizeof(float2) * R * R);
  p.MAlo = (float2*)take(sizeof(float2) * R * R);
  p.partA = (float2*)take(sizeof(float2) * (size_t)p.C * Nx * R);
  p.partNA = (float*)take(sizeof(float) * p.C * R);
  p.partMB = (float4*)take(sizeof(float4) * (size_t)p.C * R * R);
  p.partP = (float4*)take(sizeof(float4) * (size_t)p.C * Nx * R);
  p.partMA = (float4*)take(sizeof(float4) * (size_t)p.C * R * R);
  p.sf = (double*)take(sizeof(double) * SF_COUNT);
  p.gamma_d = (double2*)take(sizeof(double2) * R);
  p.status = (int*)take(sizeof(int) * (3 + TTS_MAX_CLUSTER));

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nstatus = 3 + TTS_MAX_CLUSTER;
  noalloc_setup_kernel<<<(Nx + Ny + nstatus + 255) / 256, 256, 0, st>>>(Wx, Nx, Wy, Ny, p.status, nstatus);
  if (cudaGetLastError() != cudaSuccess)
    return na_fail(TTS_ECUDA, "tts_push_frame_noalloc: set-up of the device scratch failed");
  if (launch_frame(p, TTS_LAUNCH_FUSED, st) != TTS_OK)
    return na_fail(TTS_ECUDA, "tts_push_frame_noalloc: frame kernel launch failed");
  return TTS_OK;
}
