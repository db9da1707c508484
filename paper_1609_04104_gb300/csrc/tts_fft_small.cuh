// Small DFTs of compile-time length R held in registers, for the four-step FFTs of the
// batched 2D DFT: radix 2, 3, 4, 5, 8, 16 as straight-line butterflies with constant
// twiddles, and any product of those lengths as a four-step split R = A x B (a length-A DFT
// over every stride-B subsequence, twiddles w_R^(n2 k1), length-B DFTs). The twiddles of a
// split come from the padded length-N table of exp(-2 pi i k / N) in shared memory (R divides
// N; every thread reads the same entry, so the reads are broadcasts).
//
// Conventions: v[n] is the input sequence, v[k] the output X[k] = sum_n v[n] w_R^(n k) with
// w_R = exp(-2 pi i / R) (forward) or its conjugate (INV).
#pragma once

#include "tts_internal.cuh"

namespace fftsmall {

// cos / sin of the angles the straight-line kernels use
constexpr float kC8 = 0.92387953251128675613f;    // cos(pi / 8)
constexpr float kS8 = 0.38268343236508977173f;    // sin(pi / 8)
constexpr float kH = 0.70710678118654752440f;     // cos(pi / 4)
constexpr float kS3 = 0.86602540378443864676f;    // sin(pi / 3)
constexpr float kC5a = 0.30901699437494742410f;   // cos(2 pi / 5)
constexpr float kC5b = -0.80901699437494742410f;  // cos(4 pi / 5)
constexpr float kS5a = 0.95105651629515357212f;   // sin(2 pi / 5)
constexpr float kS5b = 0.58778525229247312917f;   // sin(4 pi / 5)

// w_16^k for the k the 8- and 16-point kernels use (conjugated for the inverse)
template <bool INV>
__device__ __forceinline__ float2 w16(int k) {
  float2 w;
  switch (k & 15) {
    case 1: w = make_float2(kC8, -kS8); break;
    case 2: w = make_float2(kH, -kH); break;
    case 3: w = make_float2(kS8, -kC8); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 6: w = make_float2(-kH, -kH); break;
    default: w = make_float2(-kC8, kS8); break;   // k = 9
  }
  return INV ? make_float2(w.x, -w.y) : w;
}

// multiplication by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// w_N^idx from the padded table
template <bool INV>
__device__ __forceinline__ float2 twn(const float2* W, int idx) {
  const float2 w = W[fpad(idx)];
  return INV ? make_float2(w.x, -w.y) : w;
}

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2* v, const float2*, int) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<3, INV> {
  // y1 = a - s / 2 -+ i sin(pi / 3) d, y2 = a - s / 2 +- i sin(pi / 3) d (s = b + c, d = b - c)
  __device__ __forceinline__ static void run(float2* v, const float2*, int) {
    const float2 a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 m = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
    const float2 r = rot<INV>(cscale(d, kS3));   // -i sin(pi/3) d forward
    v[0] = cadd(a, s);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2* v, const float2*, int) {
    const float2 s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
    const float2 s1 = cadd(v[1], v[3]), d1 = rot<INV>(csub(v[1], v[3]));
    v[0] = cadd(s0, s1);
    v[1] = cadd(d0, d1);
    v[2] = csub(s0, s1);
    v[3] = csub(d0, d1);
  }
};

template <bool INV>
struct Dft<5, INV> {
  // pairs (1, 4) and (2, 3): y_k = a + cos terms of the sums -+ i sin terms of the
  // differences
  __device__ __forceinline__ static void run(float2* v, const float2*, int) {
    const float2 a = v[0];
    const float2 s1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
    const float2 s2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
    const float2 m1 = make_float2(fmaf(kC5a, s1.x, fmaf(kC5b, s2.x, a.x)), fmaf(kC5a, s1.y, fmaf(kC5b, s2.y, a.y)));
    const float2 m2 = make_float2(fmaf(kC5b, s1.x, fmaf(kC5a, s2.x, a.x)), fmaf(kC5b, s1.y, fmaf(kC5a, s2.y, a.y)));
    // sin parts before the factor -i (forward): n1 = s5a d1 + s5b d2, n2 = s5b d1 - s5a d2
    const float2 n1 = make_float2(fmaf(kS5a, d1.x, kS5b * d2.x), fmaf(kS5a, d1.y, kS5b * d2.y));
    const float2 n2 = make_float2(fmaf(kS5b, d1.x, -kS5a * d2.x), fmaf(kS5b, d1.y, -kS5a * d2.y));
    const float2 r1 = rot<INV>(n1), r2 = rot<INV>(n2);
    v[0] = cadd(a, cadd(s1, s2));
    v[1] = cadd(m1, r1);
    v[4] = csub(m1, r1);
    v[2] = cadd(m2, r2);
    v[3] = csub(m2, r2);
  }
};

template <bool INV>
struct Dft<8, INV> {
  // n = 4 n1 + n2 (n1 < 2), k = k1 + 2 k2, inner twiddles w_8^(n2)
  __device__ __forceinline__ static void run(float2* v, const float2*, int) {
    float2 t0[4], t1[4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      t0[n2] = cadd(v[n2], v[4 + n2]);
      const float2 d = csub(v[n2], v[4 + n2]);
      t1[n2] = n2 == 0 ? d : cmul(d, w16<INV>(2 * n2));
    }
    Dft<4, INV>::run(t0, nullptr, 0);
    Dft<4, INV>::run(t1, nullptr, 0);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      v[2 * k2] = t0[k2];
      v[2 * k2 + 1] = t1[k2];
    }
  }
};

template <bool INV>
struct Dft<16, INV> {
  // n = 4 n1 + n2, k = k1 + 4 k2, inner twiddles w_16^(n2 k1)
  __device__ __forceinline__ static void run(float2* v, const float2*, int) {
    float2 t[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
      Dft<4, INV>::run(a, nullptr, 0);
      t[n2 * 4 + 0] = a[0];
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) t[n2 * 4 + k1] = n2 == 0 ? a[k1] : cmul(a[k1], w16<INV>(n2 * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 b[4] = {t[k1], t[4 + k1], t[8 + k1], t[12 + k1]};
      Dft<4, INV>::run(b, nullptr, 0);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
  }
};

// R = A x B: n = B n1 + n2, k = k1 + A k2; w_R^(n2 k1) = w_N^((N / R) n2 k1)
template <int A, int B, bool INV>
struct Split {
  __device__ __forceinline__ static void run(float2* v, const float2* W, int N) {
    constexpr int R = A * B;
    const int s = N / R;
    float2 y[R];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
      float2 a[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) a[n1] = v[n2 + B * n1];
      Dft<A, INV>::run(a, W, N);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1)
        y[n2 * A + k1] = (n2 == 0 || k1 == 0) ? a[k1] : cmul(a[k1], twn<INV>(W, s * n2 * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      float2 b[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) b[n2] = y[n2 * A + k1];
      Dft<B, INV>::run(b, W, N);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = b[k2];
    }
  }
};

template <bool INV>
struct Dft<6, INV> : Split<2, 3, INV> {};
template <bool INV>
struct Dft<10, INV> : Split<2, 5, INV> {};
template <bool INV>
struct Dft<12, INV> : Split<4, 3, INV> {};
template <bool INV>
struct Dft<15, INV> : Split<3, 5, INV> {};
template <bool INV>
struct Dft<20, INV> : Split<4, 5, INV> {};
template <bool INV>
struct Dft<24, INV> : Split<8, 3, INV> {};
template <bool INV>
struct Dft<9, INV> : Split<3, 3, INV> {};
template <bool INV>
struct Dft<18, INV> : Split<2, 9, INV> {};
template <bool INV>
struct Dft<25, INV> : Split<5, 5, INV> {};
template <bool INV>
struct Dft<27, INV> : Split<3, 9, INV> {};

}  // namespace fftsmall
