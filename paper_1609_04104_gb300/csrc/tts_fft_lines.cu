// Batched unitary 2D DFT of Nx x Ny images with Nx != Ny, both line lengths among the band
// shapes of tts_fft_band.cuh (64 ... 384, see fftband::supported): per group of
// images, one launch transforms every row band (rows of length Ny, from in to out,
// unscaled) and a second one every column band of out in place (columns of length Nx,
// scaled by 1 / sqrt(Nx Ny)). A group holds at most ~40 MB, so the row pass's output is still
// in L2 when the column pass reads it and HBM sees about one read and one write of every
// image. Both kernels are persistent (one wave of CTAs walks the bands of the group), so a
// CTA loads its twiddle table once.
#include <algorithm>
#include <cstdint>

#include "tts_fft_band.cuh"
#include "tts_internal.cuh"

namespace {

using fftband::Shape;

// CTAs per SM for the launch bounds: the runtime image dimensions cost the length-16 shapes a
// few registers more than their 64, so they run a quarter fewer CTAs per SM than in the
// square form
template <int N>
constexpr int lines_minb() {
  return Shape<N>::R == 16 ? (3 * Shape<N>::MINB) / 4 : Shape<N>::MINB;
}

template <int NY, bool INV>
__global__ void __launch_bounds__(Shape<NY>::NT, lines_minb<NY>())
    fft_row_bands_kernel(const float2* in, float2* out, int nimg, int Nx, const float2* __restrict__ Wg) {
  constexpr int BAND = Shape<NY>::BAND;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* S = (float2*)smem;
  float2* W = S + BAND * fftband::row_stride<NY>();
  for (int k = threadIdx.x; k < NY; k += blockDim.x) W[fpad(k)] = Wg[k];
  const int nb = (Nx + BAND - 1) / BAND;
  const size_t img_elems = (size_t)Nx * NY;
  for (int task = blockIdx.x; task < nimg * nb; task += gridDim.x) {
    __syncthreads();   // the table; the previous band's last use of S
    const int img = task / nb, band = task - img * nb;
    fftband::row_band<NY, INV, true>(in + img * img_elems, out + img * img_elems, Nx, band * BAND, W, S);
  }
}

template <int NX, bool INV>
__global__ void __launch_bounds__(Shape<NX>::NT, lines_minb<NX>())
    fft_col_bands_kernel(float2* data, int nimg, int Ny, const float2* __restrict__ Wg, float scale) {
  constexpr int BAND = Shape<NX>::BAND;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* S = (float2*)smem;
  float2* W = S + BAND * fftband::row_stride<NX>();
  for (int k = threadIdx.x; k < NX; k += blockDim.x) W[fpad(k)] = Wg[k];
  const int nb = (Ny + BAND - 1) / BAND;
  const size_t img_elems = (size_t)NX * Ny;
  for (int task = blockIdx.x; task < nimg * nb; task += gridDim.x) {
    __syncthreads();   // the table; the previous band's last use of S
    const int img = task / nb, band = task - img * nb;
    fftband::col_band<NX, INV, true>(data + img * img_elems, Ny, band * BAND, W, S, scale);
  }
}

// resident CTAs of a kernel (occupancy x SMs), computed once per instantiation and device
template <typename K>
int resident(K kernel, int threads, int smem, PerDevice* cache) {
  int res = 0;
  if (per_device(*cache,
                 [&](int dev, int* v) {
                   int per_sm = 0, sms = 0;
                   if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                           cudaSuccess ||
                       cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
                       cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
                     return TTS_ECUDA;
                   *v = per_sm * sms;
                   return TTS_OK;
                 },
                 &res) != TTS_OK)
    return 0;
  return res;
}

template <int NY, bool INV>
int rows_t(const float2* in, float2* out, int nimg, int Nx, const float2* W, cudaStream_t st) {
  static PerDevice cache;
  constexpr int smem = fftband::smem_bytes<NY>();
  const int res = resident(fft_row_bands_kernel<NY, INV>, Shape<NY>::NT, smem, &cache);
  if (res < 1) return TTS_ECUDA;
  const int tasks = nimg * ((Nx + Shape<NY>::BAND - 1) / Shape<NY>::BAND);
  fft_row_bands_kernel<NY, INV><<<std::min(res, tasks), Shape<NY>::NT, smem, st>>>(in, out, nimg, Nx, W);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

template <int NX, bool INV>
int cols_t(float2* data, int nimg, int Ny, const float2* W, float scale, cudaStream_t st) {
  static PerDevice cache;
  constexpr int smem = fftband::smem_bytes<NX>();
  const int res = resident(fft_col_bands_kernel<NX, INV>, Shape<NX>::NT, smem, &cache);
  if (res < 1) return TTS_ECUDA;
  const int tasks = nimg * ((Ny + Shape<NX>::BAND - 1) / Shape<NX>::BAND);
  fft_col_bands_kernel<NX, INV><<<std::min(res, tasks), Shape<NX>::NT, smem, st>>>(data, nimg, Ny, W, scale);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

template <bool INV>
int rows(const float2* in, float2* out, int nimg, int Nx, int Ny, const float2* W, cudaStream_t st) {
  switch (Ny) {
    case 64: return rows_t<64, INV>(in, out, nimg, Nx, W, st);
    case 96: return rows_t<96, INV>(in, out, nimg, Nx, W, st);
    case 120: return rows_t<120, INV>(in, out, nimg, Nx, W, st);
    case 128: return rows_t<128, INV>(in, out, nimg, Nx, W, st);
    case 144: return rows_t<144, INV>(in, out, nimg, Nx, W, st);
    case 160: return rows_t<160, INV>(in, out, nimg, Nx, W, st);
    case 192: return rows_t<192, INV>(in, out, nimg, Nx, W, st);
    case 200: return rows_t<200, INV>(in, out, nimg, Nx, W, st);
    case 216: return rows_t<216, INV>(in, out, nimg, Nx, W, st);
    case 240: return rows_t<240, INV>(in, out, nimg, Nx, W, st);
    case 256: return rows_t<256, INV>(in, out, nimg, Nx, W, st);
    case 288: return rows_t<288, INV>(in, out, nimg, Nx, W, st);
    case 320: return rows_t<320, INV>(in, out, nimg, Nx, W, st);
    case 384: return rows_t<384, INV>(in, out, nimg, Nx, W, st);
    default: return TTS_EINVAL;
  }
}

template <bool INV>
int cols(float2* data, int nimg, int Nx, int Ny, const float2* W, float scale, cudaStream_t st) {
  switch (Nx) {
    case 64: return cols_t<64, INV>(data, nimg, Ny, W, scale, st);
    case 96: return cols_t<96, INV>(data, nimg, Ny, W, scale, st);
    case 120: return cols_t<120, INV>(data, nimg, Ny, W, scale, st);
    case 128: return cols_t<128, INV>(data, nimg, Ny, W, scale, st);
    case 144: return cols_t<144, INV>(data, nimg, Ny, W, scale, st);
    case 160: return cols_t<160, INV>(data, nimg, Ny, W, scale, st);
    case 192: return cols_t<192, INV>(data, nimg, Ny, W, scale, st);
    case 200: return cols_t<200, INV>(data, nimg, Ny, W, scale, st);
    case 216: return cols_t<216, INV>(data, nimg, Ny, W, scale, st);
    case 240: return cols_t<240, INV>(data, nimg, Ny, W, scale, st);
    case 256: return cols_t<256, INV>(data, nimg, Ny, W, scale, st);
    case 288: return cols_t<288, INV>(data, nimg, Ny, W, scale, st);
    case 320: return cols_t<320, INV>(data, nimg, Ny, W, scale, st);
    case 384: return cols_t<384, INV>(data, nimg, Ny, W, scale, st);
    default: return TTS_EINVAL;
  }
}

}  // namespace

bool fft2d_lines_ok(int Nx, int Ny) { return fftband::supported(Nx) && fftband::supported(Ny); }

int launch_fft2d_lines(const float2* in, float2* out, int batch, int Nx, int Ny, int inverse, const float2* Wx,
                       const float2* Wy, cudaStream_t st) {
  if (batch <= 0) return TTS_OK;
  if (!fft2d_lines_ok(Nx, Ny)) return TTS_EINVAL;
  const size_t img = (size_t)Nx * Ny;
  const int group = (int)std::max<size_t>(1, std::min<size_t>((size_t)batch, (40u << 20) / (img * sizeof(float2))));
  const float scale = 1.0f / sqrtf((float)Nx * (float)Ny);
  for (int g0 = 0; g0 < batch; g0 += group) {
    const int n = std::min(group, batch - g0);
    const float2* src = in + (size_t)g0 * img;
    float2* dst = out + (size_t)g0 * img;
    int rc = inverse ? rows<true>(src, dst, n, Nx, Ny, Wy, st) : rows<false>(src, dst, n, Nx, Ny, Wy, st);
    if (rc != TTS_OK) return rc;
    rc = inverse ? cols<true>(dst, n, Nx, Ny, Wx, scale, st) : cols<false>(dst, n, Nx, Ny, Wx, scale, st);
    if (rc != TTS_OK) return rc;
  }
  return TTS_OK;
}
