// Single-pass batched unitary 2D DFT for square N in {64, 128, 256}: one image per thread-
// block cluster of CL CTAs, the image held in the cluster's distributed shared memory, so
// that HBM sees one read and one write of every image (the two-pass form in
// tts_kernels.cu moves each image through L2 twice).
//
// Per image, CTA c of the cluster:
//   1. transforms rows [c RW, (c+1) RW) (RW = N / CL) along the rows: four-step FFT in
//      registers, N = T x R, T threads per row holding R values each, loaded straight from
//      global memory (T consecutive values per load: coalesced); length-R DFT, twiddles
//      w_N^(n1 k2), transpose through a per-group shared-memory scratch with an XOR swizzle,
//      length-T DFTs; each output is stored into the column buffer of the CTA that owns its
//      column (distributed shared memory; column block [c CW, (c+1) CW), row stride CW + 1);
//   2. after a cluster barrier, transforms its CW columns the same way in place and writes
//      them out, one 256-byte row segment per warp store;
//   3. a second cluster barrier frees every column buffer for the next image's stores.
// Two CTAs fit on one SM, so one CTA's loads overlap the other's transforms. Clusters are
// persistent: cluster k takes images k, k + clusters, ...
#include <cooperative_groups.h>

#include <algorithm>

#include "tts_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kFftThreads = 256;

template <int N>
struct Shape;
template <>
struct Shape<256> {
  static constexpr int CL = 8, T = 16, R = 16;
};
template <>
struct Shape<128> {
  static constexpr int CL = 4, T = 8, R = 16;
};
template <>
struct Shape<64> {
  static constexpr int CL = 2, T = 8, R = 8;
};

template <int L>
__device__ __forceinline__ void dft_small(float2* v, const float2* W, int N, int sign) {
  if (L == 16) dft16(v, W, N, sign);
  else dft8(v, W, N, sign);
}

// One length-N line transformed by the T threads of a group (t = thread within the group):
// v holds the line's elements t + T n2 (n2 < R); sc is N slots of scratch (slot i at
// sc[i * ss]) for the transpose; the output element k goes to put(k, value). All lanes of
// the warp call it together.
template <int N, typename Put>
__device__ __forceinline__ void fft_line(float2* v, float2* sc, int ss, const float2* W, int sign, int t, Put put) {
  constexpr int T = Shape<N>::T, R = Shape<N>::R, J = R / T;
  dft_small<R>(v, W, N, sign);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], tw(W, t * k2, sign));   // t k2 < N
  __syncwarp();
  // Y[n1 = t][k2] to slot k2 T + (n1 ^ (k2 mod T))
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) sc[(k2 * T + (t ^ (k2 % T))) * ss] = v[k2];
  __syncwarp();
  float2 u[J][T];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k2 = t + T * j;
#pragma unroll
    for (int n1 = 0; n1 < T; ++n1) u[j][n1] = sc[(k2 * T + (n1 ^ t)) * ss];
    dft_small<T>(u[j], W, N, sign);
  }
  __syncwarp();
  // X[k2 + R k1]
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int k1 = 0; k1 < T; ++k1) put(t + T * j + R * k1, u[j][k1]);
  __syncwarp();
}

template <int N>
__global__ void __launch_bounds__(kFftThreads, 2) fft2d_cluster_kernel(const float2* __restrict__ in, float2* out,
                                                                       int batch, const float2* __restrict__ Wg,
                                                                       int sign, float scale, int* err) {
  constexpr int CL = Shape<N>::CL, T = Shape<N>::T, R = Shape<N>::R;
  constexpr int RW = N / CL, CW = N / CL, GS = CW + 1, GROUPS = kFftThreads / T;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* G = (float2*)smem;                          // N x GS: this CTA's columns
  float2* scr = G + N * GS;                           // GROUPS x N: row-transpose scratch
  float2* W = scr + GROUPS * N;                       // fsz(N), padded
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int nclusters = gridDim.x / CL, cid = blockIdx.x / CL;
  const int g = tid / T, t = tid % T;
  for (int k = tid; k < N; k += kFftThreads) W[fpad(k)] = Wg[k];
  // the first row of each group for the next image, loaded while the current image's
  // columns are written out and the cluster synchronises
  float2 pv[R];
  auto load_row = [&](float2* v, int img, int r) {
    const float2* src = in + ((size_t)img * N + rank * RW + r) * N;
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) v[n2] = src[t + T * n2];
  };
  if (cid < batch && g < RW) load_row(pv, cid, g);
  __syncthreads();
  for (int img = cid; img < batch; img += nclusters) {
    cluster.sync();   // every column buffer is free (and every peer has started)
    // rows, straight from global memory
    for (int r = g; r < RW; r += GROUPS) {
      const int gr = rank * RW + r;
      float2 v[R];
      if (r == g) {
#pragma unroll
        for (int n2 = 0; n2 < R; ++n2) v[n2] = pv[n2];
      } else {
        load_row(v, img, r);
      }
      fft_line<N>(v, scr + g * N, 1, W, sign, t, [&](int k, float2 x) {
        float2* dst = cluster.map_shared_rank(G, k / CW);
        dst[gr * GS + (k % CW)] = x;
      });
    }
    cluster.sync();   // this image's column buffers are complete in every CTA
    // columns, in place
    for (int c = g; c < CW; c += GROUPS) {
      float2* col = G + c;
      float2 v[R];
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) v[n2] = col[(t + T * n2) * GS];
      fft_line<N>(v, col, GS, W, sign, t, [&](int k, float2 x) { col[k * GS] = x; });
    }
    if (img + nclusters < batch && g < RW) load_row(pv, img + nclusters, g);
    __syncthreads();
    // write: one row segment of CW values (CW * 8 bytes) per warp instruction
    float2* ob = out + (size_t)img * N * N + rank * CW;
    const int lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < N; r += kFftThreads / 32)
      for (int c = lane; c < CW; c += 32) ob[(size_t)r * N + c] = cscale(G[r * GS + c], scale);
  }
  cluster.sync();   // no CTA leaves while a peer may still store into its shared memory
  (void)err;
}

template <int N>
int launch_t(const float2* in, float2* out, int batch, const float2* W, int inverse, int* err, cudaStream_t st) {
  constexpr int CL = Shape<N>::CL, CW = N / CL;
  const int smem = (int)(sizeof(float2) * (N * (CW + 1) + (kFftThreads / Shape<N>::T) * N + fsz(N) + 1) + 16);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(fft2d_cluster_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return TTS_ECUDA;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kFftThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = CL;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(CL, 1, 1);
  int maxc = 0;
  if (cudaOccupancyMaxActiveClusters(&maxc, fft2d_cluster_kernel<N>, &cfg) != cudaSuccess || maxc < 1)
    return TTS_ECUDA;
  const int clusters = std::min(batch, maxc);
  cfg.gridDim = dim3(clusters * CL, 1, 1);
  const float scale = 1.0f / (float)N;   // (1 / sqrt N)^2: unitary in both directions
  const cudaError_t e =
      cudaLaunchKernelEx(&cfg, fft2d_cluster_kernel<N>, in, out, batch, W, inverse ? 1 : -1, scale, err);
  return e == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

}  // namespace

bool fft2d_cluster_ok(int Nx, int Ny) { return Nx == Ny && (Nx == 64 || Nx == 128 || Nx == 256); }

int launch_fft2d_cluster(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
                         cudaStream_t st) {
  if (batch <= 0) return TTS_OK;
  switch (N) {
    case 256: return launch_t<256>(in, out, batch, W, inverse, err, st);
    case 128: return launch_t<128>(in, out, batch, W, inverse, err, st);
    case 64: return launch_t<64>(in, out, batch, W, inverse, err, st);
    default: return TTS_EINVAL;
  }
}
