// Image formation, line sampler (S0 of Alg. 5), factor initialisation and the
// batched unitary 2D DFT.
#include <algorithm>

#include "tts_fft_band.cuh"
#include "tts_internal.cuh"

namespace {

// ------------------------------------------------------------------------------------
// X = A diag(gamma) B^T  (the image of the most recent frame, cf. §IV-A X_t)
// 32 x 32 output tile per CTA; A and B rows of the tile staged in shared memory.
// ------------------------------------------------------------------------------------
// One TR x 32 tile of X (TR in {8, 32}) by 256 threads. Every output sums its R terms in
// the order r = 0 .. R - 1, so the tile shape does not change a single bit of X.
template <int TR>
__device__ __forceinline__ void image_tile(const float2* __restrict__ A, const float2* __restrict__ B,
                                           const float2* __restrict__ gamma, float2* __restrict__ X, int Nx, int Ny,
                                           int R, int i0, int j0, unsigned char* smem_raw) {
  float2* sA = (float2*)smem_raw;     // TR x (R+1), A[i][r] gamma_r
  float2* sB = sA + 32 * (R + 1);     // 32 x (R+1)
  const int tid = threadIdx.x;
  for (int base = tid; base < 32 * R; base += 4 * blockDim.x) {
    float2 va[4], vb[4], vg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * blockDim.x;
      if (e < 32 * R) {
        const int ii = e / R, r = e - ii * R;
        const int i = i0 + ii, j = j0 + ii;
        va[u] = (ii < TR && i < Nx) ? A[i * R + r] : make_float2(0.f, 0.f);
        vb[u] = j < Ny ? B[j * R + r] : make_float2(0.f, 0.f);
        vg[u] = gamma[r];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * blockDim.x;
      if (e < 32 * R) {
        const int ii = e / R, r = e - ii * R;
        if (ii < TR) sA[ii * (R + 1) + r] = cmul(va[u], vg[u]);
        sB[ii * (R + 1) + r] = vb[u];
      }
    }
  }
  __syncthreads();
  constexpr int Q = TR / 8;
  const int jj = tid & 31, ib = tid >> 5;  // each thread: column jj, rows ib, ib+8, ... (Q rows)
  float2 acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int r = 0; r < R; ++r) {
    const float2 b = sB[jj * (R + 1) + r];
#pragma unroll
    for (int q = 0; q < Q; ++q) cfma(acc[q], sA[(ib + 8 * q) * (R + 1) + r], b);
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = i0 + ib + 8 * q, j = j0 + jj;
    if (i < Nx && j < Ny) X[(size_t)i * Ny + j] = acc[q];
  }
}

template <int TR>
__global__ void __launch_bounds__(256) image_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                    const float2* __restrict__ gamma, float2* __restrict__ X,
                                                    int Nx, int Ny, int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_release();
  pdl_wait();
  image_tile<TR>(A, B, gamma, X, Nx, Ny, R, blockIdx.y * TR, blockIdx.x * 32, smem_raw);
}

// Images of many trackers: the 32 x 32 tiles of all jobs form one list (job k owns tiles
// [tile0, tile0 + tiles) in row-major tile order), walked grid-stride; the number of jobs
// is read from device memory (*n).
__global__ void __launch_bounds__(256) image_batch_kernel(const ImageJob* __restrict__ jobs, const int* n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nj = *n;
  if (nj <= 0) return;
  const int total = jobs[nj - 1].tile0 + jobs[nj - 1].tiles;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = nj - 1;   // last job with tile0 <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const ImageJob& j = jobs[lo];
    const int tl = t - j.tile0, tx = (j.Ny + 31) / 32;
    const int ti = tl / tx, tj = tl - ti * tx;
    image_tile<32>(j.A, j.B, j.gamma, j.X, j.Nx, j.Ny, j.R, ti * 32, tj * 32, smem_raw);
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// Line sampler, one CTA.
//  (1) probabilities: informative scores of §V-B marginalised over readout (§VI-C),
//      p_i = (Ny sum_r |Ahat_ir|^2 / ||ahat_r||^2 + R) / (R (Nx + Ny)), Ahat = F_Nx A
//      (a zero column counts as uniform); or uniform; or variable density d_i^alpha;
//      or given.
//  (2) draw (Alg. 4 on lines): central lines kept; integer weights q = floor(p 2^52)
//      with inclusive prefix sums over the other lines; Philox4x32-10 draws
//      x = mulhi(u, Q_total), line = first with Q > x; duplicates rejected; fallback
//      fill by decreasing q.
// ------------------------------------------------------------------------------------
constexpr int SAMPLER_THREADS = 512;

__device__ __forceinline__ int upper_bound_u64(const unsigned long long* Q, int n, unsigned long long x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (Q[mid] > x) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Row scores of the informative sampler for a line length with a band shape: per pass, one
// group of T threads per column r of A (up to `cols` columns at once): the column's length-N
// DFT Ahat[:, r] = F_N a_r by the four-step FFT of tts_fft_band.cuh (or the column itself
// with no_fft), its squared norm by a reduction over the group, and the weights
// |Ahat_kr|^2 / ||ahat_r||^2 (1 / N for a zero column) into a cols x N table; then every row
// k adds its weights in column order to rowacc[k]. buf holds the transposes and the table
// (cols (row_stride + (N + 16) / 2) float2, within the sampler's FFT buffer).
template <int N>
__device__ __forceinline__ void sampler_scores_band(const float2* __restrict__ A, int R, int no_fft, const float2* W,
                                                    float2* buf, float* rowacc, int cols) {
  using fftband::Shape;
  constexpr int T = Shape<N>::T, RL = Shape<N>::R, J = (RL + T - 1) / T, RS = fftband::row_stride<N>();
  constexpr int WS = N + 16;   // weight-table row stride (floats): neighbouring groups on other banks
  float* Wt = (float*)(buf + cols * RS);
  const int tid = threadIdx.x, g = tid / T, t = tid % T;
  const unsigned gmask = T == 32 ? 0xffffffffu : (((1u << T) - 1u) << ((tid & 31) & ~(T - 1)));
  for (int r0 = 0; r0 < R; r0 += cols) {
    const int nc = min(cols, R - r0);
    if (g < nc) {   // uniform over the group
      const float2* a = A + r0 + g;
      float2 v[RL];
#pragma unroll
      for (int n2 = 0; n2 < RL; ++n2) v[n2] = a[(size_t)(t + T * n2) * R];
      float* wrow = Wt + g * WS;
      if (no_fft) {
        float s = 0.f;
#pragma unroll
        for (int n2 = 0; n2 < RL; ++n2) s += cabs2(v[n2]);
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        const float inv = s > 0.f ? 1.f / s : 0.f;
#pragma unroll
        for (int n2 = 0; n2 < RL; ++n2) wrow[t + T * n2] = inv > 0.f ? cabs2(v[n2]) * inv : 1.f / (float)N;
      } else {
        float2* sc = buf + g * RS;
        fftband::dft_small<RL, false>(v, W, N);
#pragma unroll
        for (int k2 = 1; k2 < RL; ++k2) v[k2] = cmul(v[k2], fftsmall::twn<false>(W, t * k2));
#pragma unroll
        for (int k2 = 0; k2 < RL; ++k2) sc[k2 * T + (t ^ (k2 % T))] = v[k2];
        __syncwarp(gmask);
        float2 u[J][T];
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int k2 = t + T * j;
          if (J * T == RL || k2 < RL) {
#pragma unroll
            for (int n1 = 0; n1 < T; ++n1) u[j][n1] = sc[k2 * T + (n1 ^ (k2 % T))];
            fftband::dft_small<T, false>(u[j], W, N);
#pragma unroll
            for (int k1 = 0; k1 < T; ++k1) s += cabs2(u[j][k1]);
          }
        }
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        const float inv = s > 0.f ? 1.f / s : 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int k2 = t + T * j;
          if (J * T == RL || k2 < RL) {
#pragma unroll
            for (int k1 = 0; k1 < T; ++k1)
              wrow[k2 + RL * k1] = inv > 0.f ? cabs2(u[j][k1]) * inv : 1.f / (float)N;   // row k2 + RL k1
          }
        }
      }
    }
    __syncthreads();
    for (int k = tid; k < N; k += blockDim.x) {
      float acc = rowacc[k];
      for (int c = 0; c < nc; ++c) acc += Wt[c * WS + k];
      rowacc[k] = acc;
    }
    __syncthreads();
  }
}

// The same scores with the T = 16 threads of a column in 16 different warps, one column per
// lane (T warps, up to 32 columns a pass): every load of A is a coalesced piece of a row, the
// transpose goes through the column's region of shared memory (stride N + 1, so that the 32
// columns of a warp fall on different banks) with a CTA barrier, and the column norm is summed
// through shared memory (red, T x 32 floats) in the order of the shuffle butterfly of
// sampler_scores_band, so the weights are bit-identical to it.
template <int N>
__device__ __forceinline__ void sampler_scores_lanes(const float2* __restrict__ A, int R, int no_fft,
                                                     const float2* W, float2* buf, float* rowacc, int cols,
                                                     float* red) {
  using fftband::Shape;
  constexpr int T = Shape<N>::T, RL = Shape<N>::R, J = (RL + T - 1) / T, CS = N + 1;
  static_assert(T == 16, "one warp per thread of a column");
  constexpr int WS = N + 16;
  float* Wt = (float*)(buf + cols * CS);
  const int tid = threadIdx.x, t = tid >> 5, c = tid & 31;
  for (int r0 = 0; r0 < R; r0 += cols) {
    const int nc = min(cols, R - r0);
    const bool act = c < nc;
    float2 v[RL];
    float2 u[J][T];
    float s = 0.f;
    if (act) {
#pragma unroll
      for (int n2 = 0; n2 < RL; ++n2) v[n2] = A[(size_t)(t + T * n2) * R + r0 + c];
    }
    if (no_fft) {
      if (act) {
#pragma unroll
        for (int n2 = 0; n2 < RL; ++n2) s += cabs2(v[n2]);
      }
    } else {
      float2* sc = buf + c * CS;
      if (act) {
        fftband::dft_small<RL, false>(v, W, N);
#pragma unroll
        for (int k2 = 1; k2 < RL; ++k2) v[k2] = cmul(v[k2], fftsmall::twn<false>(W, t * k2));
#pragma unroll
        for (int k2 = 0; k2 < RL; ++k2) sc[k2 * T + (t ^ (k2 % T))] = v[k2];
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int k2 = t + T * j;
          if (J * T == RL || k2 < RL) {
#pragma unroll
            for (int n1 = 0; n1 < T; ++n1) u[j][n1] = sc[k2 * T + (n1 ^ (k2 % T))];
            fftband::dft_small<T, false>(u[j], W, N);
#pragma unroll
            for (int k1 = 0; k1 < T; ++k1) s += cabs2(u[j][k1]);
          }
        }
      }
    }
    // column norm: the butterfly x1[i] = s[i] + s[i ^ 8], x2[i] = x1[i] + x1[i ^ 4], ... of
    // the 16 per-thread sums, whose value is the same for every i
    red[t * 32 + c] = s;
    __syncthreads();
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = red[i * 32 + c];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < o) x[i] = x[i] + x[i + o];   // x[i] for i < o holds the value of both i and i + o
    const float tot = x[0];
    const float inv = tot > 0.f ? 1.f / tot : 0.f;
    if (act) {
      float* wrow = Wt + c * WS;
      if (no_fft) {
#pragma unroll
        for (int n2 = 0; n2 < RL; ++n2) wrow[t + T * n2] = inv > 0.f ? cabs2(v[n2]) * inv : 1.f / (float)N;
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int k2 = t + T * j;
          if (J * T == RL || k2 < RL) {
#pragma unroll
            for (int k1 = 0; k1 < T; ++k1) wrow[k2 + RL * k1] = inv > 0.f ? cabs2(u[j][k1]) * inv : 1.f / (float)N;
          }
        }
      }
    }
    __syncthreads();
    for (int k = tid; k < N; k += blockDim.x) {
      float acc = rowacc[k];
      for (int cc = 0; cc < nc; ++cc) acc += Wt[cc * WS + k];
      rowacc[k] = acc;
    }
    __syncthreads();
  }
}

// scores for one band-shape length: up to blockDim / T columns per pass (T threads each); for
// the 16-thread shapes with 16 warps, one column per lane instead (coalesced loads of A)
template <int N>
__device__ __forceinline__ void sampler_scores_for(const float2* A, int R, int no_fft, const float2* W, float2* buf,
                                                   float* rowacc, int fft_cols, float* red) {
  if constexpr (fftband::Shape<N>::T == 16) {
    if (blockDim.x == 512) {
      sampler_scores_lanes<N>(A, R, no_fft, W, buf, rowacc, min(min(32, R), fft_cols), red);
      return;
    }
  }
  const int cols = min(min((int)blockDim.x / fftband::Shape<N>::T, R), fft_cols);
  sampler_scores_band<N>(A, R, no_fft, W, buf, rowacc, cols);
}

// the band-shape lengths: scores through sampler_scores_band; false for any other Nx
__device__ __forceinline__ bool sampler_scores_fast(int Nx, const float2* A, int R, int no_fft, const float2* W,
                                                    float2* buf, float* rowacc, int fft_cols, float* red) {
  switch (Nx) {
#define SCORES(N) \
  case N: sampler_scores_for<N>(A, R, no_fft, W, buf, rowacc, fft_cols, red); return true;
    SCORES(64) SCORES(96) SCORES(120) SCORES(128) SCORES(144) SCORES(160) SCORES(192) SCORES(200) SCORES(216)
    SCORES(240) SCORES(256) SCORES(288) SCORES(320) SCORES(384)
#undef SCORES
    default: return false;
  }
}

__device__ __forceinline__ void sampler_run(const SamplerJob& job, unsigned char* smem_raw) {
  const float2* __restrict__ A = job.A;
  const int Nx = job.Nx, Ny = job.Ny, R = job.R;
  const double* __restrict__ p_in = job.p_in;
  double* p_out = job.p_out;
  const int policy = job.policy;
  const double vd_alpha = job.vd_alpha;
  const int k_lines = job.k_lines, central = job.central;
  const unsigned long long seed = job.seed, ctr = job.ctr;
  const int with_replacement = job.with_replacement;
  const float2* __restrict__ Wx = job.Wx;
  uint8_t* mask_out = job.mask_out;
  uint8_t* mask_out2 = job.mask_out2;
  const int fft_cols = job.fft_cols;
  double* p = (double*)smem_raw;                                   // Nx
  unsigned long long* Q = (unsigned long long*)(p + TTS_MAX_N);    // Nx
  float* rowacc = (float*)(Q + TTS_MAX_N);                          // Nx
  float* nrm = rowacc + TTS_MAX_N;                                  // fft_cols
  int* cand = (int*)(nrm + 64);                                     // Nx
  uint8_t* mask = (uint8_t*)(cand + TTS_MAX_N);                     // Nx
  int* misc = (int*)(mask + TTS_MAX_N);                             // 8
  float2* W = (float2*)(misc + 8);                                  // fsz(Nx), padded
  float2* buf = W + fsz(TTS_MAX_N);                                 // 2 x fft_cols x ld
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;

  // (1) probabilities
  if (p_in != nullptr) {
    for (int i = tid; i < Nx; i += blockDim.x) p[i] = p_in[i];
  } else if (policy == TTS_POLICY_INFORMATIVE) {
    for (int i = tid; i < Nx; i += blockDim.x) {
      W[fpad(i)] = Wx[i];
      rowacc[i] = 0.f;
    }
    __syncthreads();
    const FftPlan plan = fft_plan(Nx);
    const int ld = fsz(Nx) | 1;   // padded column stride (odd) in shared memory
    // p (probabilities, written after the scores) serves as the scores' reduction scratch
    const bool fast = sampler_scores_fast(Nx, A, R, job.no_fft, W, buf, rowacc, fft_cols, (float*)p);
    for (int r0 = 0; r0 < (fast ? 0 : R); r0 += fft_cols) {
      const int nc = min(fft_cols, R - r0);
      // coalesced along the rows of A, transposed into columns
      for (int base = tid; base < nc * Nx; base += 8 * blockDim.x) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = base + u * blockDim.x;
          if (e < nc * Nx) {
            const int n = e / nc, c = e - n * nc;
            v[u] = A[n * R + r0 + c];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = base + u * blockDim.x;
          if (e < nc * Nx) {
            const int n = e / nc, c = e - n * nc;
            buf[c * ld + fpad(n)] = v[u];
          }
        }
      }
      __syncthreads();
      float2* res = job.no_fft ? buf : fft_smem(buf, buf + fft_cols * ld, plan, nc, ld, W, -1, tid, blockDim.x);
      for (int c = warp; c < nc; c += nwarp) {
        float acc = 0.f;
        for (int n = lane; n < Nx; n += 32) acc += cabs2(res[c * ld + fpad(n)]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) nrm[c] = acc > 0.f ? 1.f / acc : 0.f;
      }
      __syncthreads();
      for (int i = tid; i < Nx; i += blockDim.x) {
        float acc = rowacc[i];
        for (int c = 0; c < nc; ++c) acc += nrm[c] > 0.f ? cabs2(res[c * ld + fpad(i)]) * nrm[c] : 1.f / (float)Nx;
        rowacc[i] = acc;
      }
      __syncthreads();
    }
    // one FP64 division for the block (FP64 is slow on this part), then FMAs
    double* dinv = (double*)(misc + 4);
    if (tid == 0) *dinv = 1.0 / ((double)R * (double)(Nx + Ny));
    __syncthreads();
    const double inv = *dinv;
    for (int i = tid; i < Nx; i += blockDim.x) p[i] = ((double)Ny * (double)rowacc[i] + (double)R) * inv;
  } else {
    // uniform or variable density: weights then a fixed-order tree normalisation
    for (int i = tid; i < TTS_MAX_N; i += blockDim.x) {
      double wgt = 0.0;
      if (i < Nx) {
        if (policy == TTS_POLICY_UNIFORM) {
          wgt = 1.0;
        } else {
          double d = (double)min(i, Nx - i);
          d = d < 1.0 ? 1.0 : d;
          wgt = vd_alpha == -1.0 ? 1.0 / d : (vd_alpha == -0.5 ? 1.0 / sqrt(d) : pow(d, vd_alpha));
        }
      }
      p[i] = wgt;
      ((double*)Q)[i] = wgt;
    }
    __syncthreads();
    double* tsum = (double*)Q;
    for (int half = TTS_MAX_N / 2; half > 0; half >>= 1) {
      for (int i = tid; i < half; i += blockDim.x) tsum[i] += tsum[i + half];
      __syncthreads();
    }
    const double total = tsum[0];
    __syncthreads();
    for (int i = tid; i < Nx; i += blockDim.x) p[i] = p[i] / total;   // exact division: fixed policies only
  }
  __syncthreads();
  if (p_out != nullptr)
    for (int i = tid; i < Nx; i += blockDim.x) p_out[i] = p[i];
  if (k_lines <= 0) return;

  // (2) draw. Central set {-c/2 .. c/2-1} mod Nx.
  const int c = min(central, Nx);
  for (int i = tid; i < Nx; i += blockDim.x) {
    const int off = (i + c / 2) % Nx;   // i == (k - c/2) mod Nx  <=>  off == k < c
    mask[i] = off < c ? 1 : 0;
  }
  __syncthreads();
  // candidate list (non-central lines, increasing) and their integer weights
  if (warp == 0) {
    int count = 0;
    for (int base = 0; base < Nx; base += 32) {
      const int i = base + lane;
      const bool on = i < Nx && mask[i] == 0;
      const unsigned bal = __ballot_sync(0xffffffffu, on);
      if (on) cand[count + __popc(bal & ((1u << lane) - 1u))] = i;
      count += __popc(bal);
    }
    if (lane == 0) misc[0] = count;
  }
  __syncthreads();
  const int ncand = misc[0];
  const int kl = min(k_lines, Nx);
  const int need = kl - c;
  if (need > 0 && ncand > 0) {
    const double two52 = 4503599627370496.0;
    for (int k = tid; k < ncand; k += blockDim.x) {
      const double v = p[cand[k]];
      Q[k] = v > 0.0 ? (unsigned long long)floor(v * two52) : 0ull;
    }
    __syncthreads();
    // inclusive prefix sum by one warp (integer, exact): blocks of 32 entries in order, a
    // shuffle scan within each block and the running total carried across blocks, so no
    // CTA barrier is needed between the steps
    if (warp == 0) {
      unsigned long long carry = 0ull;
      for (int b0 = 0; b0 < ncand; b0 += 32) {
        const int k = b0 + lane;
        unsigned long long v = k < ncand ? Q[k] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += t;
        }
        v += carry;
        if (k < ncand) Q[k] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
      }
    }
    __syncthreads();
    const unsigned long long Qtot = Q[ncand - 1];
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c2 = (uint32_t)ctr, c3 = (uint32_t)(ctr >> 32);
    if (warp == 0) {
      int got = 0;
      if (Qtot > 0) {
        const int ndraws = with_replacement ? need : 64 * need;
        for (int base = 0; base < ndraws; base += 32) {
          if (!with_replacement && got >= need) break;
          const int d = base + lane;
          const bool valid = d < ndraws;
          int line = -1 - lane;
          if (valid) {
            const U32x4 w = philox4x32_10((uint32_t)d, TTS_PURPOSE_LINES, c2, c3, k0, k1);
            const unsigned long long u = (unsigned long long)w.v[0] | ((unsigned long long)w.v[1] << 32);
            const unsigned long long x = __umul64hi(u, Qtot);
            line = cand[upper_bound_u64(Q, ncand, x)];
          }
          if (with_replacement) {
            if (valid) mask[line] = 1;
            __syncwarp();
            continue;
          }
          const unsigned peers = __match_any_sync(0xffffffffu, line);
          const bool first = (__ffs(peers) - 1) == lane;
          const bool acc0 = valid && first && mask[line] == 0;
          const unsigned bal = __ballot_sync(0xffffffffu, acc0);
          const int rank = __popc(bal & ((1u << lane) - 1u));
          __syncwarp();
          if (acc0 && got + rank < need) mask[line] = 1;
          got = min(need, got + __popc(bal));
          __syncwarp();
        }
      }
      if (lane == 0) misc[1] = got;
    }
    __syncthreads();
    const int got = misc[1];
    if (!with_replacement && got < need) {
      // fill by decreasing q, lower index first on ties (q recomputed from p)
      const int rest = need - got;
      for (int k = tid; k < ncand; k += blockDim.x) {
        const int i = cand[k];
        if (mask[i]) continue;
        const double vi = p[i];
        const unsigned long long qi = vi > 0.0 ? (unsigned long long)floor(vi * two52) : 0ull;
        int rank = 0;
        for (int k2 = 0; k2 < ncand; ++k2) {
          const int i2 = cand[k2];
          if (mask[i2] || i2 == i) continue;
          const double v2 = p[i2];
          const unsigned long long q2 = v2 > 0.0 ? (unsigned long long)floor(v2 * two52) : 0ull;
          if (q2 > qi || (q2 == qi && i2 < i)) ++rank;
        }
        rowacc[i] = rank < rest ? 1.f : 0.f;
      }
      __syncthreads();
      for (int k = tid; k < ncand; k += blockDim.x) {
        const int i = cand[k];
        if (!mask[i] && rowacc[i] == 1.f) mask[i] = 2;
      }
      __syncthreads();
      for (int i = tid; i < Nx; i += blockDim.x)
        if (mask[i] == 2) mask[i] = 1;
    }
  }
  __syncthreads();
  for (int i = tid; i < Nx; i += blockDim.x) {
    mask_out[i] = mask[i];
    if (mask_out2) mask_out2[i] = mask[i];
  }
}

__global__ void __launch_bounds__(SAMPLER_THREADS) sampler_kernel(SamplerJob job) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_release();
  pdl_wait();
  sampler_run(job, smem_raw);
  if (job.done) {
    // the masks are in memory the host polls: every thread's writes are made visible system
    // wide before the completion word is set
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) *(volatile unsigned int*)job.done = job.done_value;
  }
}

// One CTA per job; the number of jobs is read from device memory (*n), so a captured
// launch sized for the capacity serves any smaller batch.
__global__ void __launch_bounds__(SAMPLER_THREADS) sampler_batch_kernel(const SamplerJob* __restrict__ jobs,
                                                                        const int* n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if ((int)blockIdx.x >= *n) return;
  const SamplerJob job = jobs[blockIdx.x];
  sampler_run(job, smem_raw);
}

// ------------------------------------------------------------------------------------
// CN(0, 1/N) factor entries from Philox4x32-10 and the Box-Muller transform.
// ------------------------------------------------------------------------------------
__global__ void init_kernel(float2* A, int N, int R, unsigned long long seed, uint32_t which) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * R) return;
  const U32x4 w = philox4x32_10((uint32_t)e, TTS_PURPOSE_INIT, which, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = ((float)(w.v[0] >> 8) + 1.0f) * (1.0f / 16777216.0f);  // (0, 1]
  const float u2 = (float)(w.v[1] >> 8) * (1.0f / 16777216.0f);           // [0, 1)
  const float rad = sqrtf(-2.0f * logf(u1)) * sqrtf(0.5f / (float)N);
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  A[e] = make_float2(rad * cs, rad * sn);
}

// ------------------------------------------------------------------------------------
// Batched unitary 2D DFT, two passes through global memory: row transforms (length Ny,
// contiguous), then column transforms (length Nx) on column blocks staged in shared
// memory.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) fft_rows_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                       long nrows, int Ny, int rows_per_cta, int sign,
                                                       const float2* __restrict__ Wy, float scale, int vec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = fsz(Ny);   // padded row stride in shared memory
  float2* W = (float2*)smem_raw;
  float2* buf = W + fsz(Ny);
  float2* tmp = buf + rows_per_cta * ld;
  const int tid = threadIdx.x;
  for (int e = tid; e < Ny; e += blockDim.x) W[fpad(e)] = Wy[e];
  const long r0 = (long)blockIdx.x * rows_per_cta;
  const int nr = (int)min((long)rows_per_cta, nrows - r0);
  if (nr <= 0) return;
  const int n2 = nr * Ny;
  if (vec) {
    // float4 global loads (Ny even, in and out 16-byte aligned): two elements of one row
    // (a pair never straddles a pad slot)
    const float4* src = (const float4*)(in + r0 * Ny);
    for (int e = tid; e < n2 / 2; e += blockDim.x) {
      const float4 v = src[e];
      const int i0 = 2 * e, r = i0 / Ny, c = i0 - r * Ny;
      buf[r * ld + fpad(c)] = make_float2(v.x, v.y);
      buf[r * ld + fpad(c + 1)] = make_float2(v.z, v.w);
    }
  } else {
    for (int e = tid; e < n2; e += blockDim.x) {
      const int r = e / Ny, c = e - r * Ny;
      buf[r * ld + fpad(c)] = in[r0 * Ny + e];
    }
  }
  __syncthreads();
  const FftPlan plan = fft_plan(Ny);
  float2* res = fft_smem(buf, tmp, plan, nr, ld, W, sign, tid, blockDim.x);
  if (vec) {
    float4* dst = (float4*)(out + r0 * Ny);
    for (int e = tid; e < n2 / 2; e += blockDim.x) {
      const int i0 = 2 * e, r = i0 / Ny, c = i0 - r * Ny;
      const float2 x0 = res[r * ld + fpad(c)], x1 = res[r * ld + fpad(c + 1)];
      dst[e] = make_float4(x0.x * scale, x0.y * scale, x1.x * scale, x1.y * scale);
    }
  } else {
    for (int e = tid; e < n2; e += blockDim.x) {
      const int r = e / Ny, c = e - r * Ny;
      out[r0 * Ny + e] = cscale(res[r * ld + fpad(c)], scale);
    }
  }
}

__global__ void __launch_bounds__(256) fft_cols_kernel(float2* data, int Nx, int Ny, int cols_per_cta, int sign,
                                                       const float2* __restrict__ Wx, float scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* W = (float2*)smem_raw;
  const int ld = fsz(Nx) | 1;   // padded column stride (odd) in shared memory
  float2* buf = W + fsz(Nx);
  float2* tmp = buf + cols_per_cta * ld;
  const int tid = threadIdx.x;
  for (int e = tid; e < Nx; e += blockDim.x) W[fpad(e)] = Wx[e];
  const int nblk = (Ny + cols_per_cta - 1) / cols_per_cta;
  const long img = blockIdx.x / nblk;
  const int j0 = (blockIdx.x % nblk) * cols_per_cta;
  const int nc = min(cols_per_cta, Ny - j0);
  float2* base = data + img * (long)Nx * Ny;
  // stage column block transposed: column c of the block at c * ld, element i at fpad(i)
  for (int e = tid; e < Nx * nc; e += blockDim.x) {
    const int i = e / nc, c = e - i * nc;
    buf[c * ld + fpad(i)] = base[(long)i * Ny + j0 + c];
  }
  __syncthreads();
  const FftPlan plan = fft_plan(Nx);
  float2* res = fft_smem(buf, tmp, plan, nc, ld, W, sign, tid, blockDim.x);
  for (int e = tid; e < Nx * nc; e += blockDim.x) {
    const int i = e / nc, c = e - i * nc;
    base[(long)i * Ny + j0 + c] = cscale(res[c * ld + fpad(i)], scale);
  }
}

}  // namespace

int launch_image(const float2* A, const float2* B, const float2* gamma, float2* X, int Nx, int Ny, int R,
                 cudaStream_t st) {
  // 32-row tiles while they fill every SM, else 8-row tiles (four times the CTAs)
  const int smem = 2 * 32 * (R + 1) * (int)sizeof(float2);
  static PerDevice sm_count;
  int sms = 0;
  if (per_device(sm_count,
                 [](int dev, int* v) {
                   // the largest shared-memory carveout, as the frame kernel runs with: SMs
                   // then keep one L1 / shared split across a frame's launches
                   if (cudaFuncSetAttribute(image_kernel<32>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                            cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
                       cudaFuncSetAttribute(image_kernel<8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                            cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                     return TTS_ECUDA;
                   return cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess ? TTS_OK
                                                                                                      : TTS_ECUDA;
                 },
                 &sms) != TTS_OK)
    return TTS_ECUDA;
  const int tiles32 = ((Ny + 31) / 32) * ((Nx + 31) / 32);
  if (tiles32 >= sms) {
    dim3 grid((Ny + 31) / 32, (Nx + 31) / 32);
    if (launch_pdl(image_kernel<32>, grid, dim3(256), smem, st, 0, A, B, gamma, X, Nx, Ny, R) != cudaSuccess)
      return TTS_ECUDA;
  } else {
    dim3 grid((Ny + 31) / 32, (Nx + 7) / 8);
    if (launch_pdl(image_kernel<8>, grid, dim3(256), smem, st, 0, A, B, gamma, X, Nx, Ny, R) != cudaSuccess)
      return TTS_ECUDA;
  }
  return TTS_OK;
}

SamplerJob sampler_job(const float2* A, int Nx, int Ny, int R, const double* p_in, double* p_out, int policy,
                       double vd_alpha, int k_lines, int central, uint64_t seed, uint64_t ctr, int with_replacement,
                       const float2* Wx, uint8_t* mask_out, uint8_t* mask_out2) {
  SamplerJob j;
  j.A = A;
  j.Nx = Nx;
  j.Ny = Ny;
  j.R = R;
  j.p_in = p_in;
  j.p_out = p_out;
  j.policy = policy;
  j.vd_alpha = vd_alpha;
  j.k_lines = k_lines;
  j.central = central;
  j.seed = (unsigned long long)seed;
  j.ctr = (unsigned long long)ctr;
  j.with_replacement = with_replacement;
  j.Wx = Wx;
  j.mask_out = mask_out;
  j.mask_out2 = mask_out2;
  j.fft_cols = max(1, min(min(R, 64), 8192 / max(Nx, 1)));
  j.no_fft = 0;
  j.done = nullptr;
  j.done_value = 0;
  return j;
}

size_t sampler_smem(int Nx, int fft_cols) {
  return sizeof(double) * TTS_MAX_N + sizeof(unsigned long long) * TTS_MAX_N + sizeof(float) * TTS_MAX_N +
         sizeof(float) * 64 + sizeof(int) * TTS_MAX_N + TTS_MAX_N + sizeof(int) * 8 +
         sizeof(float2) * fsz(TTS_MAX_N) + sizeof(float2) * 2 * fft_cols * (fsz(Nx) | 1) + 64;
}

// grid 0 only loads the kernel (done before any capture).
int launch_image_batch(const ImageJob* jobs, const int* n, int grid, cudaStream_t st) {
  const int smem = 2 * 32 * (TTS_MAX_R + 1) * (int)sizeof(float2);
  if (grid <= 0) {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, image_batch_kernel) == cudaSuccess ? TTS_OK : TTS_ECUDA;
  }
  image_batch_kernel<<<grid, 256, smem, st>>>(jobs, n);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

size_t sampler_smem_max();

int launch_sampler(const float2* A, int Nx, int Ny, int R, const double* p_in, double* p_out, int policy,
                   double vd_alpha, int k_lines, int central, uint64_t seed, uint64_t ctr, int with_replacement,
                   const float2* Wx, uint8_t* mask_out, uint8_t* mask_out2, cudaStream_t st, int no_fft,
                   unsigned int* done_word, unsigned int done_value) {
  SamplerJob j = sampler_job(A, Nx, Ny, R, p_in, p_out, policy, vd_alpha, k_lines, central, seed, ctr,
                             with_replacement, Wx, mask_out, mask_out2);
  j.no_fft = no_fft;
  j.done = done_word;
  j.done_value = done_value;
  const size_t smem = sampler_smem(Nx, j.fft_cols);
  static PerDevice attrs;
  int done = 0;
  if (per_device(attrs,
                 [](int, int* v) {
                   // room for any job, and the largest carveout (see launch_image)
                   if (cudaFuncSetAttribute(sampler_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sampler_smem_max()) != cudaSuccess ||
                       cudaFuncSetAttribute(sampler_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                            cudaSharedmemCarveoutMaxShared) != cudaSuccess)
                     return TTS_ECUDA;
                   *v = 1;
                   return TTS_OK;
                 },
                 &done) != TTS_OK)
    return TTS_ECUDA;
  return launch_pdl(sampler_kernel, dim3(1), dim3(SAMPLER_THREADS), smem, st, 0, j) == cudaSuccess ? TTS_OK
                                                                                         : TTS_ECUDA;
}

// Largest shared memory any sampler job needs (Nx <= TTS_MAX_N, at most 8192 staged
// entries of A): the capacity of a batched launch.
size_t sampler_smem_max() {
  size_t m = 0;
  for (int Nx = 1; Nx <= TTS_MAX_N; ++Nx) m = std::max(m, sampler_smem(Nx, std::max(1, std::min(64, 8192 / Nx))));
  return m;
}

// capacity 0 only sets the kernel's shared-memory attribute (done before any capture).
int launch_sampler_batch(const SamplerJob* jobs, const int* n, int capacity, cudaStream_t st) {
  const size_t smem = sampler_smem_max();
  if (capacity <= 0) {
    const cudaError_t e =
        cudaFuncSetAttribute(sampler_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e == cudaSuccess ? TTS_OK : TTS_ECUDA;
  }
  sampler_batch_kernel<<<capacity, SAMPLER_THREADS, smem, st>>>(jobs, n);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

int launch_init_factors(float2* A, int N, int R, uint64_t seed, uint32_t which, cudaStream_t st) {
  const int n = N * R;
  init_kernel<<<(n + 255) / 256, 256, 0, st>>>(A, N, R, (unsigned long long)seed, which);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

int launch_fft2d(const float2* in, float2* out, int batch, int Nx, int Ny, int inverse, const float2* Wx,
                 const float2* Wy, float2* scratch, cudaStream_t st) {
  (void)scratch;
  const int sign = inverse ? +1 : -1;
  const int rows_per_cta = max(1, 4096 / Ny);
  const size_t smem_r = sizeof(float2) * (fsz(Ny) + 2 * (size_t)rows_per_cta * fsz(Ny));
  cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r);
  if (e != cudaSuccess) return TTS_ECUDA;
  const int cols_per_cta = max(1, min(Ny, 4096 / Nx));
  const size_t smem_c = sizeof(float2) * (fsz(Nx) + 2 * (size_t)cols_per_cta * (fsz(Nx) | 1));
  e = cudaFuncSetAttribute(fft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c);
  if (e != cudaSuccess) return TTS_ECUDA;
  // Images go in groups whose row-pass result (written to out) stays in L2 until the
  // column pass reads it back: DRAM then sees about one read of in and one write of out.
  const size_t img = (size_t)Nx * Ny * sizeof(float2);
  const size_t l2_budget = 32u << 20;
  // 16-byte vector accesses need even rows and 16-byte aligned images
  const int vec = (Ny % 2 == 0) && ((uintptr_t)in % 16 == 0) && ((uintptr_t)out % 16 == 0);
  const int group = (int)std::max<size_t>(1, std::min<size_t>((size_t)batch, l2_budget / img));
  for (int g0 = 0; g0 < batch; g0 += group) {
    const int gb = std::min(group, batch - g0);
    const long nrows = (long)gb * Nx;
    const long grid_r = (nrows + rows_per_cta - 1) / rows_per_cta;
    fft_rows_kernel<<<(unsigned)grid_r, 256, smem_r, st>>>(in + (size_t)g0 * Nx * Ny, out + (size_t)g0 * Nx * Ny, nrows,
                                                            Ny, rows_per_cta, sign, Wy, 1.0f / sqrtf((float)Ny), vec);
    if (cudaGetLastError() != cudaSuccess) return TTS_ECUDA;
    const long grid_c = (long)gb * ((Ny + cols_per_cta - 1) / cols_per_cta);
    fft_cols_kernel<<<(unsigned)grid_c, 256, smem_c, st>>>(out + (size_t)g0 * Nx * Ny, Nx, Ny, cols_per_cta, sign, Wx,
                                                            1.0f / sqrtf((float)Nx));
    if (cudaGetLastError() != cudaSuccess) return TTS_ECUDA;
  }
  return TTS_OK;
}

// ---------------------------------------------------------------------------------
// FP32 fused multiply-add throughput of the device, the denominator of the frame kernel's
// ALU roofline (a calibration; the paper has no counterpart). Every thread runs eight
// independent chains a <- a b + c (b < 1, so the values stay bounded); the sum of the chains
// is stored only if it equals -1, which it never does, so no chain is dead code.
// ---------------------------------------------------------------------------------
namespace {
__device__ float g_fma_sink;

__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, float b, float c) {
  float a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = (float)(threadIdx.x + u) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fmaf(a[u], b, c);
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fmaf(a[u], b, c);
  }
  const float s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  if (s == -1.0f) g_fma_sink = s;
}
}  // namespace

extern "C" int tts_fp32_fma_rate(int iters, int reps, double* tflops, double* ms) {
  if (!tflops || iters < 1 || reps < 1) {
    tts_internal_set_error("tts_fp32_fma_rate: NULL output or non-positive iters / reps");
    return TTS_EINVAL;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel, 256, 0) != cudaSuccess || per_sm < 1) {
    tts_internal_set_error("tts_fp32_fma_rate: no device");
    return TTS_ECUDA;
  }
  const int grid = sms * per_sm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TTS_ECUDA;
  float best = 0.f;
  int rc = TTS_OK;
  for (int r = 0; r <= reps && rc == TTS_OK; ++r) {   // the first launch is a warm-up
    cudaEventRecord(e0, 0);
    fma_rate_kernel<<<grid, 256>>>(iters, 0.99999f, 1e-5f);
    cudaEventRecord(e1, 0);
    float t = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = TTS_ECUDA;
    if (r > 0 && (best == 0.f || t < best)) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TTS_OK || best <= 0.f) {
    tts_internal_set_error("tts_fp32_fma_rate: kernel failed");
    return TTS_ECUDA;
  }
  const double flops = 2.0 * 16.0 * (double)iters * (double)grid * 256.0;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return TTS_OK;
}
