// Band transforms of the batched 2D DFT: BAND consecutive rows, or BAND consecutive
// columns, of one image, each line a four-step FFT N = T x R (T a power of two): a length-R
// DFT in registers over the elements t + T n2, twiddles w_N^(t k2), a transpose through
// shared memory, length-T DFTs, output X[k2 + R k1].
//   rows:    T threads per row (a half-warp or a quarter-warp), loads and stores of T
//            consecutive values; the transpose through the row's own region of S (XOR
//            swizzle, quarter-warp rows padded so that the two rows of a half-warp use
//            different banks);
//   columns: thread (t, c) for column c of the band; every load and store of BAND
//            consecutive values of one row; the transpose through the band's N x BAND
//            region of S.
// Rows are written unscaled; columns are scaled on the way out. Global loads bypass L1 (a
// column band reads rows that other SMs wrote).
#pragma once

#include "tts_fft_small.cuh"
#include "tts_internal.cuh"

namespace fftband {

using fftsmall::twn;

// T x R = N; BAND lines per band; NT = BAND T threads, one line each; MINB CTAs per SM for
// the register budget (64 registers for R <= 16, more for the longer R)
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
struct Shape<120> {
  static constexpr int T = 8, R = 15, BAND = 16, NT = 128, MINB = 6;
};
template <>
struct Shape<128> {
  static constexpr int T = 8, R = 16, BAND = 16, NT = 128, MINB = 8;
};
template <>
struct Shape<144> {
  static constexpr int T = 16, R = 9, BAND = 16, NT = 256, MINB = 4;
};
template <>
struct Shape<200> {
  static constexpr int T = 8, R = 25, BAND = 16, NT = 128, MINB = 4;
};
template <>
struct Shape<216> {
  static constexpr int T = 8, R = 27, BAND = 16, NT = 128, MINB = 4;
};
template <>
struct Shape<288> {
  static constexpr int T = 16, R = 18, BAND = 16, NT = 256, MINB = 3;
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
struct Shape<240> {
  static constexpr int T = 16, R = 15, BAND = 16, NT = 256, MINB = 3;
};
template <>
struct Shape<256> {
  static constexpr int T = 16, R = 16, BAND = 16, NT = 256, MINB = 4;
};
template <>
struct Shape<320> {
  static constexpr int T = 16, R = 20, BAND = 16, NT = 256, MINB = 3;
};
template <>
struct Shape<384> {
  static constexpr int T = 16, R = 24, BAND = 16, NT = 256, MINB = 3;
};

// the line lengths with a Shape
__host__ __device__ constexpr bool supported(int N) {
  return N == 64 || N == 96 || N == 120 || N == 128 || N == 144 || N == 160 || N == 192 || N == 200 || N == 216 ||
         N == 240 || N == 256 || N == 288 || N == 320 || N == 384;
}

// row regions in S: quarter-warp rows (T = 8) padded by 64 bytes
template <int N>
__host__ __device__ constexpr int row_stride() {
  return N + (Shape<N>::T == 8 ? 8 : 0);
}

// shared memory of a band transform: S (BAND x row_stride for rows, N x BAND for columns)
// and the padded length-N twiddle table
template <int N>
__host__ __device__ constexpr int smem_bytes() {
  return (int)sizeof(float2) * (Shape<N>::BAND * row_stride<N>() + N + (N - 1) / 16);
}

template <int L, bool INV>
__device__ __forceinline__ void dft_small(float2* v, const float2* W, int N) {
  fftsmall::Dft<L, INV>::run(v, W, N);
}

// Rows [r0, r0 + BAND) (with RAGGED, those below nrows) of length N, element j of row i
// given by load(i, j), to dst rows (row stride N), unscaled, stored with L2 caching (they are
// read back soon). W: the padded length-N table.
template <int N, bool INV, bool RAGGED, typename Load>
__device__ __forceinline__ void row_band_f(Load load, float2* dst, int nrows, int r0, const float2* W, float2* S) {
  constexpr int T = Shape<N>::T, R = Shape<N>::R, J = (R + T - 1) / T;
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  const int row = r0 + g;
  if (RAGGED && row >= nrows) return;   // uniform over the row's T threads
  float2 v[R];
#pragma unroll
  for (int n2 = 0; n2 < R; ++n2) v[n2] = load(row, t + T * n2);
  float2* sc = S + g * row_stride<N>();
  dft_small<R, INV>(v, W, N);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twn<INV>(W, t * k2));   // t k2 < N
  // Y[n1 = t][k2] to slot k2 T + (n1 ^ (k2 mod T))
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) sc[k2 * T + (t ^ (k2 % T))] = v[k2];
  if (RAGGED) __syncwarp(T == 32 ? 0xffffffffu : (((1u << T) - 1u) << ((threadIdx.x & 31) & ~(T - 1))));
  else __syncwarp();
  float2* d = dst + (size_t)row * N;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k2 = t + T * j;
    if (J * T == R || k2 < R) {
      float2 u[T];
#pragma unroll
      for (int n1 = 0; n1 < T; ++n1) u[n1] = sc[k2 * T + (n1 ^ (k2 % T))];
      dft_small<T, INV>(u, W, N);
#pragma unroll
      for (int k1 = 0; k1 < T; ++k1) __stcg(d + k2 + R * k1, u[k1]);   // X[k2 + R k1]
    }
  }
}

// row_band_f over the rows of src (row stride N), read streaming
template <int N, bool INV, bool RAGGED>
__device__ __forceinline__ void row_band(const float2* src, float2* dst, int nrows, int r0, const float2* W, float2* S) {
  row_band_f<N, INV, RAGGED>([src](int i, int j) { return __ldcs(src + (size_t)i * N + j); }, dst, nrows, r0, W, S);
}

// Columns [c0, c0 + BAND) (with RAGGED, those below ncols) of length N of an image with row
// stride ncols; output k of column c goes to store(k, c, value) unscaled. Every thread of the
// CTA must call it (it synchronises the CTA once, after its shared-memory stores).
template <int N, bool INV, bool RAGGED, typename Store>
__device__ __forceinline__ void col_band_f(const float2* img, int ncols, int c0, const float2* W, float2* S,
                                           Store store) {
  constexpr int T = Shape<N>::T, R = Shape<N>::R, BAND = Shape<N>::BAND, J = (R + T - 1) / T;
  const int c = threadIdx.x % BAND, t = threadIdx.x / BAND;
  const bool live = !RAGGED || c0 + c < ncols;
  const float2* cb = img + c0 + c;
  const float2* p = cb + (size_t)t * ncols;   // rows t + T n2 of the column
  const size_t step = (size_t)T * ncols;
  float2 v[R];
  if (live) {
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) v[n2] = __ldcg(p + n2 * step);
  } else {
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) v[n2] = make_float2(0.f, 0.f);
  }
  dft_small<R, INV>(v, W, N);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twn<INV>(W, t * k2));
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) S[(k2 * T + t) * BAND + c] = v[k2];
  __syncthreads();
  if (!live) return;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k2 = t + T * j;
    if (J * T == R || k2 < R) {
      float2 u[T];
#pragma unroll
      for (int n1 = 0; n1 < T; ++n1) u[n1] = S[(k2 * T + n1) * BAND + c];
      dft_small<T, INV>(u, W, N);
#pragma unroll
      for (int k1 = 0; k1 < T; ++k1) store(k2 + R * k1, c0 + c, u[k1]);   // X[k2 + R k1]
    }
  }
}

// Columns [c0, c0 + BAND) (with RAGGED, those below ncols) of length N of an image with row
// stride ncols, in place, scaled by `scale`, stored streaming: the same transform as
// col_band_f with the output addressed by pointer steps (fewer live registers). Every thread
// of the CTA must call it.
template <int N, bool INV, bool RAGGED>
__device__ __forceinline__ void col_band(float2* img, int ncols, int c0, const float2* W, float2* S, float scale) {
  constexpr int T = Shape<N>::T, R = Shape<N>::R, BAND = Shape<N>::BAND, J = (R + T - 1) / T;
  const int c = threadIdx.x % BAND, t = threadIdx.x / BAND;
  const bool live = !RAGGED || c0 + c < ncols;
  float2* cb = img + c0 + c;
  const float2* p = cb + (size_t)t * ncols;   // rows t + T n2 of the column
  const size_t step = (size_t)T * ncols;
  float2 v[R];
  if (live) {
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) v[n2] = __ldcg(p + n2 * step);
  } else {
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) v[n2] = make_float2(0.f, 0.f);
  }
  dft_small<R, INV>(v, W, N);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], twn<INV>(W, t * k2));
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) S[(k2 * T + t) * BAND + c] = v[k2];
  __syncthreads();
  if (!live) return;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k2 = t + T * j;
    if (J * T == R || k2 < R) {
      float2 u[T];
#pragma unroll
      for (int n1 = 0; n1 < T; ++n1) u[n1] = S[(k2 * T + n1) * BAND + c];
      dft_small<T, INV>(u, W, N);
      float2* q = cb + (size_t)k2 * ncols;   // rows k2 + R k1
      const size_t rstep = (size_t)R * ncols;
#pragma unroll
      for (int k1 = 0; k1 < T; ++k1) __stcs(q + k1 * rstep, cscale(u[k1], scale));
    }
  }
}

}  // namespace fftband
