// Batched unitary 2D DFT for square N (64, 96, 128, 144, 160, 192, 256, 288, 320, 384; the
// band length divides N) as one
// persistent launch over band tasks, with the intermediate image kept in L2, so that HBM
// sees about one read and one write of every image.
//
// The image splits into NB = N / BAND bands of BAND rows and NB bands of BAND columns
// (BAND = 16). A row task (image i, band b) transforms rows [BAND b, BAND (b + 1)) of in[i]
// and writes them, unscaled, to out[i]; a column task transforms columns
// [BAND b, BAND (b + 1)) of out[i] in place and scales by 1 / N (the two unitary 1 / sqrt N
// factors); both are the band transforms of tts_fft_band.cuh. Tasks are taken in a fixed
// order from one counter: the row tasks of image i come L images ahead of its column tasks
// (L about 3 CTAs / (2 NB)), so a column task almost never waits, and the L
// images between the two passes (a few MB) stay in L2. A column task waits until the NB row
// tasks of its image have published (a per-image counter: thread 0 of a row task's CTA
// raises it with a release reduction after the barrier that follows the task's stores,
// thread 0 of a column task's CTA reads it with acquire loads; GPU scope; the wait is
// bounded). A row task never waits, and every task waits only on tasks taken before it, so
// the launch cannot deadlock. Small CTAs (BAND x T threads, at most 52 KB of shared memory,
// two to eight per SM) let the other CTAs of an SM run through one CTA's barrier and memory
// waits.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "tts_fft_band.cuh"
#include "tts_internal.cuh"

namespace {

using fftband::Shape;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Task q of the fixed order: row tasks of images [0, L) first, then per image i >= L the
// column tasks of image i - L followed by the row tasks of image i, then the column tasks
// of the last L images. Returns the image; *band the band, *col whether a column task.
__device__ __forceinline__ int decode(int q, int NB, int L, int batch, int* band, bool* col) {
  const int Lb = min(L, batch);
  const int head = NB * Lb;
  const int mid_imgs = batch - Lb;
  const int mid = 2 * NB * mid_imgs;
  if (q < head) {
    *col = false;
    *band = q % NB;
    return q / NB;
  }
  if (q < head + mid) {
    const int qq = q - head, pair = qq / (2 * NB), r = qq - pair * 2 * NB;
    *col = r < NB;
    *band = *col ? r : r - NB;
    return *col ? pair : pair + Lb;
  }
  const int qq = q - head - mid;
  *col = true;
  *band = qq % NB;
  return mid_imgs + qq / NB;
}

// CTAs per SM the square kernel is compiled for: above the band shape's default for 96, 160
// and 192, whose registers still fit the tighter budget without spills (more warps in flight
// to cover the memory latency)
template <int N>
constexpr int square_minb() {
  return N == 96 ? 8 : (N == 160 ? 5 : (N == 192 ? 4 : Shape<N>::MINB));
}

template <int N, bool INV>
__global__ void __launch_bounds__(Shape<N>::NT, square_minb<N>())
    fft2d_square_kernel(const float2* in, float2* out, int batch, int L, const float2* __restrict__ Wg, float scale,
                        int* ctrl, int* err, int withhold, long long limit) {
  constexpr int BAND = Shape<N>::BAND, NT = Shape<N>::NT, NB = N / BAND;
  static_assert(BAND * Shape<N>::T == NT && N % BAND == 0, "one line of the band per thread");
  extern __shared__ __align__(16) unsigned char smem[];
  float2* S = (float2*)smem;                                 // band transposes
  float2* W = S + BAND * fftband::row_stride<N>();           // fsz(N), padded
  __shared__ int s_task[2];
  int* next = ctrl;                         // task counter
  int* done = ctrl + 1;                     // row tasks published, per image
  const int tid = threadIdx.x;
  const int total = 2 * NB * batch;
  for (int k = tid; k < N; k += NT) W[fpad(k)] = Wg[k];
  // thread 0 takes the next task index while the current task runs, and publishes a
  // finished row task at the top of the next iteration (after the barrier that follows
  // the task's last store)
  int nq = 0, pub = -1;
  if (tid == 0) s_task[0] = atomicAdd(next, 1);
  __syncthreads();
  for (int it = 0;; ++it) {
    const int q = s_task[it & 1];
    if (tid == 0) {
      if (pub >= 0) {
        // cumulative over the CTA's stores (the barrier before); the test hook withholds
        // the publication of one image, so that its column tasks' waits run out
        if (pub != withhold) red_release_add(done + pub, 1);
        pub = -1;
      }
      if (q < total) nq = atomicAdd(next, 1);
    }
    if (q >= total) break;
    int band;
    bool col;
    const int img = decode(q, NB, L, batch, &band, &col);
    float2* ob = out + (size_t)img * N * N;
    if (!col) {
      fftband::row_band<N, INV, false>(in + (size_t)img * N * N, ob, N, band * BAND, W, S);
      if (tid == 0) pub = img;
    } else {
      if (tid == 0) {   // acquire the NB row tasks of the image
        const long long t0 = clock64();
        while (ld_acquire(done + img) < NB) {
          if (clock64() - t0 > limit) {
            atomicOr(err, 1);
            break;
          }
        }
      }
      __syncthreads();
      fftband::col_band<N, INV, false>(ob, N, band * BAND, W, S, scale);
    }
    if (tid == 0) s_task[(it + 1) & 1] = nq;
    __syncthreads();   // the task's stores are issued; S and s_task[it & 1] are free
  }
}

// Stream-ordered memory for the task counters of a call, from a pool of this library that
// keeps its memory between calls (the device's default pool returns it at every
// synchronisation, and mapping it again costs more than a small transform). One pool per
// device, created on first use.
cudaMemPool_t ctrl_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return nullptr;
    }
    pools[dev] = p;
  }
  return pools[dev];
}

// Launch shape of the square kernel per (device, N, direction): CTAs per SM of the
// persistent grid (0: as many as fit) and the multiplier of the row-ahead lag L. The defaults
// (all that fit, multiplier 1) stand until tts_fft2d_autotune records a measured pick.
struct SquareShape {
  int per_sm;
  float lag;
};
std::mutex g_shape_mu;
SquareShape g_shape[TTS_MAX_DEVICES][2][10];

int size_slot(int N) {
  switch (N) {
    case 64: return 0;
    case 96: return 1;
    case 128: return 2;
    case 144: return 3;
    case 160: return 4;
    case 192: return 5;
    case 256: return 6;
    case 288: return 7;
    case 320: return 8;
    case 384: return 9;
    default: return -1;
  }
}

SquareShape square_shape(int N, bool inv) {
  int dev = 0;
  const int k = size_slot(N);
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TTS_MAX_DEVICES || k < 0) return {0, 1.f};
  std::lock_guard<std::mutex> lk(g_shape_mu);
  const SquareShape sh = g_shape[dev][inv ? 1 : 0][k];
  return sh.lag > 0.f ? sh : SquareShape{0, 1.f};
}

// CTAs of the kernel that fit on one SM (*fit) and the SM count, set up once per device
template <int N, bool INV>
int grid_info(int* fit, int* sms_out) {
  constexpr int smem = fftband::smem_bytes<N>();
  static PerDevice grids;
  int grid = 0;
  if (per_device(grids,
                 [](int dev, int* v) {
                   if (cudaFuncSetAttribute(fft2d_square_kernel<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            smem) != cudaSuccess)
                     return TTS_ECUDA;
                   int per_sm = 0, sms = 0;
                   if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fft2d_square_kernel<N, INV>,
                                                                     Shape<N>::NT, smem) != cudaSuccess ||
                       cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
                     return TTS_ECUDA;
                   *v = per_sm * 1000 + sms;
                   return TTS_OK;
                 },
                 &grid) != TTS_OK)
    return TTS_ECUDA;
  *fit = grid / 1000;
  *sms_out = grid % 1000;
  return TTS_OK;
}

template <int N, bool INV>
int launch_t(const float2* in, float2* out, int batch, const float2* W, int* err, cudaStream_t st, int withhold,
             long long limit, SquareShape shape) {
  constexpr int NB = N / Shape<N>::BAND;
  constexpr int smem = fftband::smem_bytes<N>();
  int fit = 0, sms = 0;
  if (grid_info<N, INV>(&fit, &sms) != TTS_OK) return TTS_ECUDA;
  const int per_sm = shape.per_sm > 0 ? std::min(shape.per_sm, fit) : fit;
  const int tasks = 2 * NB * batch;
  const int g = std::min(per_sm * sms, tasks);
  // lag between an image's row and column tasks: by default the 2 NB L tasks in between are
  // about three times the tasks in flight (measured at 256^2: half of it, 62 % of HBM; this,
  // 66 %; twice it, 63 %); the autotuner may scale it
  const int L = std::max(1, (int)(shape.lag * (float)((3 * g) / (2 * NB))) + 1);
  int* ctrl = nullptr;
  const size_t cb = sizeof(int) * (1 + (size_t)batch);
  cudaMemPool_t pool = ctrl_pool();
  if (!pool || cudaMallocFromPoolAsync((void**)&ctrl, cb, pool, st) != cudaSuccess) return TTS_ECUDA;
  if (cudaMemsetAsync(ctrl, 0, cb, st) != cudaSuccess) return TTS_ECUDA;
  fft2d_square_kernel<N, INV><<<g, Shape<N>::NT, smem, st>>>(in, out, batch, L, W, 1.0f / (float)N, ctrl, err,
                                                               withhold, limit);
  const cudaError_t e = cudaGetLastError();
  if (cudaFreeAsync(ctrl, st) != cudaSuccess || e != cudaSuccess) return TTS_ECUDA;
  return TTS_OK;
}

template <int N>
int launch_n(const float2* in, float2* out, int batch, int inverse, const float2* W, int* err, cudaStream_t st,
             int withhold, long long limit, const SquareShape* forced) {
  const SquareShape sh = forced ? *forced : square_shape(N, inverse != 0);
  return inverse ? launch_t<N, true>(in, out, batch, W, err, st, withhold, limit, sh)
                 : launch_t<N, false>(in, out, batch, W, err, st, withhold, limit, sh);
}

template <int N>
int fit_n(int inverse, int* fit) {
  int sms = 0;
  return inverse ? grid_info<N, true>(fit, &sms) : grid_info<N, false>(fit, &sms);
}

int square_fit(int N, int inverse, int* fit) {
  switch (N) {
    case 64: return fit_n<64>(inverse, fit);
    case 96: return fit_n<96>(inverse, fit);
    case 128: return fit_n<128>(inverse, fit);
    case 144: return fit_n<144>(inverse, fit);
    case 160: return fit_n<160>(inverse, fit);
    case 192: return fit_n<192>(inverse, fit);
    case 256: return fit_n<256>(inverse, fit);
    case 288: return fit_n<288>(inverse, fit);
    case 320: return fit_n<320>(inverse, fit);
    case 384: return fit_n<384>(inverse, fit);
    default: return TTS_EINVAL;
  }
}

int launch_any(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
               cudaStream_t st, int withhold, long long limit, const SquareShape* forced) {
  switch (N) {
    case 64: return launch_n<64>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 96: return launch_n<96>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 128: return launch_n<128>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 144: return launch_n<144>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 160: return launch_n<160>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 192: return launch_n<192>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 256: return launch_n<256>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 288: return launch_n<288>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 320: return launch_n<320>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    case 384: return launch_n<384>(in, out, batch, inverse, W, err, st, withhold, limit, forced);
    default: return TTS_EINVAL;
  }
}

}  // namespace

bool fft2d_square_ok(int Nx, int Ny) {
  if (Nx != Ny) return false;
  switch (Nx) {
    case 64: case 96: case 128: case 144: case 160: case 192: case 256: case 288: case 320: case 384: return true;
    default: return false;
  }
}

int launch_fft2d_square(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
                        cudaStream_t st, int withhold, long long limit) {
  if (batch <= 0) return TTS_OK;
  return launch_any(in, out, batch, N, inverse, W, err, st, withhold, limit, nullptr);
}

int tune_fft2d_square(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
                      int reps, double* best_ms, int* best_per_sm, double* best_lag) {
  const int k = size_slot(N);
  int dev = 0;
  if (k < 0 || batch < 1 || reps < 1 || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TTS_MAX_DEVICES)
    return TTS_EINVAL;
  int fit = 0;
  if (square_fit(N, inverse, &fit) != TTS_OK || fit < 1) return TTS_ECUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TTS_ECUDA;
  const float lags[] = {0.5f, 1.f, 1.5f, 2.f, 3.f};
  float best = 0.f;
  SquareShape pick{0, 1.f};
  int rc = TTS_OK;
  // candidates: the CTAs per SM that fit and up to two fewer (more registers and cache per
  // CTA), each with five lags; one untimed launch each, then the best of `reps`
  for (int per_sm = fit; per_sm >= std::max(1, fit - 2) && rc == TTS_OK; --per_sm)
    for (float lag : lags) {
      const SquareShape sh{per_sm, lag};
      rc = launch_any(in, out, batch, N, inverse, W, err, 0, -1, 2000000000LL, &sh);
      float t_best = 0.f;
      for (int r = 0; r < reps && rc == TTS_OK; ++r) {
        cudaEventRecord(e0, 0);
        rc = launch_any(in, out, batch, N, inverse, W, err, 0, -1, 2000000000LL, &sh);
        cudaEventRecord(e1, 0);
        float t = 0.f;
        if (rc == TTS_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
          rc = TTS_ECUDA;
        if (rc == TTS_OK && (t_best == 0.f || t < t_best)) t_best = t;
      }
      if (rc != TTS_OK) break;
      if (best == 0.f || t_best < best) {
        best = t_best;
        pick = sh;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TTS_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape[dev][inverse ? 1 : 0][k] = pick;
  }
  if (best_ms) *best_ms = best;
  if (best_per_sm) *best_per_sm = pick.per_sm;
  if (best_lag) *best_lag = pick.lag;
  return TTS_OK;
}