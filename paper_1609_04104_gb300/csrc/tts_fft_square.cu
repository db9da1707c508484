// Batched unitary 2D DFT for square N in {64, 128, 256} as one persistent launch over band
// tasks, with the intermediate image kept in L2, so that HBM sees about one read and one
// write of every image.
//
// The image splits into NB = N / BAND bands of BAND rows and NB bands of BAND columns
// (BAND = 16). A row task (image i, band b) transforms rows
// [BAND b, BAND (b + 1)) of in[i] and writes them, unscaled, to out[i]; a column task
// transforms columns [BAND b, BAND (b + 1)) of out[i] in place and scales by 1 / N (the two
// unitary 1 / sqrt N factors). Tasks are taken in a fixed order from one counter: the row
// tasks of image i come L images ahead of its column tasks (L about 1.5 times the CTAs
// over 2 NB), so a column task almost never waits, and the L images between the two passes
// (a few MB) stay in L2. A column task waits until the NB row tasks of its image have
// published (a per-image counter, release / acquire at GPU scope; the wait is bounded). A
// row task never waits, and every task waits only on tasks taken before it, so the launch
// cannot deadlock. Small CTAs (BAND x T threads, at most 35 KB of shared memory, four or
// eight per SM) let the other CTAs of an SM run through one CTA's barrier and memory waits.
//
// Both task kinds run the four-step FFT N = T x R per line: a length-R DFT in registers over
// the elements t + T n2, twiddles w_N^(t k2), a transpose through shared memory, length-T
// DFTs.
//   rows:    T threads per row (a half-warp or a quarter-warp), loads and stores of T
//            consecutive values; the transpose through the row's own region;
//   columns: thread (t, c) for column c of the band, every load and store of BAND
//            consecutive values of one row, the transpose through the band's N x BAND buffer.
// Global loads bypass L1 (the data of a column task was written by other SMs).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "tts_fft_small.cuh"
#include "tts_internal.cuh"

namespace {

// T x R = N (T a power of two, threads per line in a row task; R the register length); BAND
// rows (row task) or columns (column task) per task; NT = BAND T threads, one line of the
// band each; MINB CTAs per SM (registers: 64 for R <= 16, more for the longer R)
template <int N>
struct Shape;
template <>
struct Shape<64> {
  static constexpr int T = 8, R = 8, BAND = 16, NT = 128, MINB = 8;
};
template <>
struct Shape<96> {
  static constexpr int T = 8, R = 12, BAND = 16, NT = 128, MINB = 6;
};
template <>
struct Shape<128> {
  static constexpr int T = 8, R = 16, BAND = 16, NT = 128, MINB = 8;
};
template <>
struct Shape<160> {
  static constexpr int T = 16, R = 10, BAND = 16, NT = 256, MINB = 4;
};
template <>
struct Shape<192> {
  static constexpr int T = 16, R = 12, BAND = 16, NT = 256, MINB = 3;
};
template <>
struct Shape<256> {
  static constexpr int T = 16, R = 16, BAND = 16, NT = 256, MINB = 4;
};
template <>
struct Shape<320> {
  static constexpr int T = 16, R = 20, BAND = 16, NT = 256, MINB = 2;
};
template <>
struct Shape<384> {
  static constexpr int T = 16, R = 24, BAND = 16, NT = 256, MINB = 2;
};

using fftsmall::twn;

template <int L, bool INV>
__device__ __forceinline__ void dft_small(float2* v, const float2* W, int N) {
  fftsmall::Dft<L, INV>::run(v, W, N);
}

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

// Row regions of a row task: with quarter-warp rows (T = 8) a pad of 64 bytes puts the two
// rows of a half-warp on different banks.
template <int N>
__host__ __device__ constexpr int row_stride() {
  return N + (Shape<N>::T == 8 ? 8 : 0);
}

template <int N, bool INV>
__global__ void __launch_bounds__(Shape<N>::NT, Shape<N>::MINB)
    fft2d_square_kernel(const float2* in, float2* out, int batch, int L, const float2* __restrict__ Wg, float scale,
                        int* ctrl, int* err) {
  constexpr int T = Shape<N>::T, R = Shape<N>::R, BAND = Shape<N>::BAND, NT = Shape<N>::NT;
  constexpr int J = (R + T - 1) / T, NB = N / BAND;   // second-stage lines per thread
  static_assert(BAND * T == NT, "one line of the band per thread");
  constexpr int RS = row_stride<N>();       // row regions of a row task in S
  extern __shared__ __align__(16) unsigned char smem[];
  float2* S = (float2*)smem;                // transposes: BAND x RS (rows), N x BAND (columns)
  float2* W = S + BAND * RS;                // fsz(N), padded
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
        red_release_add(done + pub, 1);   // cumulative over the CTA's stores (the barrier before)
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
      // ---- row task: group g = tid / T takes row g of the band
      const int g = tid / T, t = tid % T;
      float2 v[R];
      const float2* src = in + (size_t)img * N * N + (size_t)(band * BAND + g) * N + t;
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) v[n2] = __ldcs(src + T * n2);
      float2* sc = S + g * RS;
      dft_small<R, INV>(v, W, N);
#pragma unroll
      for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twn<INV>(W, t * k2));   // t k2 < N
      // Y[n1 = t][k2] to slot k2 T + (n1 ^ (k2 mod T))
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) sc[k2 * T + (t ^ (k2 % T))] = v[k2];
      __syncwarp();
      float2* dst = ob + (size_t)(band * BAND + g) * N;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int k2 = t + T * j;
        if (J * T == R || k2 < R) {
          float2 u[T];
#pragma unroll
          for (int n1 = 0; n1 < T; ++n1) u[n1] = sc[k2 * T + (n1 ^ (k2 % T))];
          dft_small<T, INV>(u, W, N);
#pragma unroll
          for (int k1 = 0; k1 < T; ++k1) __stcg(dst + k2 + R * k1, u[k1]);   // X[k2 + R k1]
        }
      }
      if (tid == 0) pub = img;
    } else {
      // ---- column task: c = tid mod BAND is column band * BAND + c, t = tid / BAND the
      // four-step index (a warp holds 32 / BAND values of t)
      if (tid == 0) {
        const long long t0 = clock64();
        while (ld_acquire(done + img) < NB) {
          if (clock64() - t0 > 2000000000LL) {
            atomicOr(err, 1);
            break;
          }
        }
      }
      __syncthreads();
      const int c = tid % BAND, t = tid / BAND;
      float2* cb = ob + band * BAND + c;
      float2 v[R];
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) v[n2] = __ldcg(cb + (size_t)(t + T * n2) * N);
      dft_small<R, INV>(v, W, N);
#pragma unroll
      for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twn<INV>(W, t * k2));
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) S[(k2 * T + t) * BAND + c] = v[k2];
      __syncthreads();
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int k2 = t + T * j;
        if (J * T == R || k2 < R) {
          float2 u[T];
#pragma unroll
          for (int n1 = 0; n1 < T; ++n1) u[n1] = S[(k2 * T + n1) * BAND + c];
          dft_small<T, INV>(u, W, N);
#pragma unroll
          for (int k1 = 0; k1 < T; ++k1) __stcs(cb + (size_t)(k2 + R * k1) * N, cscale(u[k1], scale));
        }
      }
    }
    if (tid == 0) s_task[(it + 1) & 1] = nq;
    __syncthreads();   // the task's stores are issued; S and s_task[it & 1] are free
  }
}

template <int N>
constexpr int smem_bytes() {
  return (int)sizeof(float2) * (Shape<N>::BAND * row_stride<N>() + N + (N - 1) / 16);   // S and fsz(N)
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

template <int N, bool INV>
int launch_t(const float2* in, float2* out, int batch, const float2* W, int* err, cudaStream_t st) {
  constexpr int NB = N / Shape<N>::BAND;
  constexpr int smem = smem_bytes<N>();
  static int grid = 0;
  if (grid == 0) {
    if (cudaFuncSetAttribute(fft2d_square_kernel<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return TTS_ECUDA;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fft2d_square_kernel<N, INV>, Shape<N>::NT, smem) !=
            cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return TTS_ECUDA;
    grid = per_sm * sms;
  }
  const int tasks = 2 * NB * batch;
  const int g = std::min(grid, tasks);
  // lag between an image's row and column tasks: about 1.5 times the tasks in flight
  const int L = std::max(1, (3 * g) / (4 * NB) + 1);
  int* ctrl = nullptr;
  const size_t cb = sizeof(int) * (1 + (size_t)batch);
  cudaMemPool_t pool = ctrl_pool();
  if (!pool || cudaMallocFromPoolAsync((void**)&ctrl, cb, pool, st) != cudaSuccess) return TTS_ECUDA;
  if (cudaMemsetAsync(ctrl, 0, cb, st) != cudaSuccess) return TTS_ECUDA;
  fft2d_square_kernel<N, INV><<<g, Shape<N>::NT, smem, st>>>(in, out, batch, L, W, 1.0f / (float)N, ctrl, err);
  const cudaError_t e = cudaGetLastError();
  if (cudaFreeAsync(ctrl, st) != cudaSuccess || e != cudaSuccess) return TTS_ECUDA;
  return TTS_OK;
}

template <int N>
int launch_n(const float2* in, float2* out, int batch, int inverse, const float2* W, int* err, cudaStream_t st) {
  return inverse ? launch_t<N, true>(in, out, batch, W, err, st) : launch_t<N, false>(in, out, batch, W, err, st);
}

}  // namespace

bool fft2d_square_ok(int Nx, int Ny) {
  if (Nx != Ny) return false;
  switch (Nx) {
    case 64: case 96: case 128: case 160: case 192: case 256: case 320: case 384: return true;
    default: return false;
  }
}

int launch_fft2d_square(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
                        cudaStream_t st) {
  if (batch <= 0) return TTS_OK;
  switch (N) {
    case 64: return launch_n<64>(in, out, batch, inverse, W, err, st);
    case 96: return launch_n<96>(in, out, batch, inverse, W, err, st);
    case 128: return launch_n<128>(in, out, batch, inverse, W, err, st);
    case 160: return launch_n<160>(in, out, batch, inverse, W, err, st);
    case 192: return launch_n<192>(in, out, batch, inverse, W, err, st);
    case 256: return launch_n<256>(in, out, batch, inverse, W, err, st);
    case 320: return launch_n<320>(in, out, batch, inverse, W, err, st);
    case 384: return launch_n<384>(in, out, batch, inverse, W, err, st);
    default: return TTS_EINVAL;
  }
}
