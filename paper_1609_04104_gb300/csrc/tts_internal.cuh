// Internal declarations of the GB300 tracker library: complex helpers, the
// shared-memory Stockham FFT, Philox4x32-10, and the per-handle device workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/tts.h"

#define TTS_MAX_N 512
#define TTS_MAX_R 64
#define TTS_MAX_CLUSTER 16
#define TTS_THREADS 512
#define TTS_MAX_OWN 8     // register-owned outputs per thread (64 x 64 / 512)

// ------------------------------------------------------------------------------------
// Per-device set-up of a kernel (shared-memory opt-in, cluster permission, occupancy):
// kernel attributes belong to the device that was current when they were set, so a value
// is computed once per device ordinal, with that device current, and reused. Thread-safe;
// a failed computation is not remembered.
// ------------------------------------------------------------------------------------
#define TTS_MAX_DEVICES 64
struct PerDevice {
  std::mutex mu;
  int val[TTS_MAX_DEVICES] = {};
  bool have[TTS_MAX_DEVICES] = {};
};

// *out = compute(dev, &v) result v for the current device dev (computed on first use).
template <typename F>
inline int per_device(PerDevice& c, F&& compute, int* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TTS_MAX_DEVICES) return TTS_ECUDA;
  std::lock_guard<std::mutex> lk(c.mu);
  if (!c.have[dev]) {
    int v = 0;
    const int rc = compute(dev, &v);
    if (rc != TTS_OK) return rc;
    c.val[dev] = v;
    c.have[dev] = true;
  }
  *out = c.val[dev];
  return TTS_OK;
}

// ------------------------------------------------------------------------------------
// Programmatic dependent launch between the per-frame kernels of one stream (line draw,
// frame, image). Each is launched with programmatic stream serialization, so its CTAs may
// become resident while the kernel before it in the stream still runs; it calls pdl_wait()
// before its first global access, which returns once every earlier kernel of the stream has
// completed and its writes are visible (each of these kernels waits before it finishes, so
// the chain is transitive). pdl_release() at the top of a kernel lets the next one launch
// as soon as all of this kernel's CTAs have started. Launched without the attribute, both
// are no-ops.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch `kernel` on `st` with programmatic stream serialization (and a cluster of
// `cluster` CTAs along x when cluster > 0).
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              int cluster, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int n = 0;
  attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[n].val.programmaticStreamSerializationAllowed = 1;
  ++n;
  if (cluster > 0) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = cluster;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = 1;
    ++n;
  }
  cfg.attrs = attr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------------------------------
// complex float / double helpers
// ------------------------------------------------------------------------------------
// Products are written with explicit fused multiply-adds and the library is compiled
// without automatic contraction (-fmad=false): every rounding is fixed by the source, so a
// routine gives bit-identical results in every kernel that inlines it.
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -(a.y * b.x)));
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
// acc -= a * b
__device__ __forceinline__ void cfms(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 zmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -(a.y * b.x)));
}
__host__ __device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// ------------------------------------------------------------------------------------
// Block-wide copy of n elements with U loads in flight per thread before the stores, so
// that global-memory latency is paid once per U elements rather than per element.
// ------------------------------------------------------------------------------------
template <typename T, int U = 4>
__device__ __forceinline__ void block_copy(T* __restrict__ dst, const T* __restrict__ src, int n) {
  const int nth = blockDim.x;
  for (int base = threadIdx.x; base < n; base += U * nth) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * nth;
      if (e < n) v[u] = src[e];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * nth;
      if (e < n) dst[e] = v[u];
    }
  }
}

// ------------------------------------------------------------------------------------
// Mixed-radix Stockham autosort FFT in shared memory.
//
// Unnormalised DFT  y_k = sum_n x_n w^{nk},  w = exp(sign * 2 pi i / N),
// N = 16^a 8^b 4^c 2^d 3^e 5^f (radices in that order; 16 and 8 are computed in registers
// as radix-4 x radix-4 and radix-2 x radix-4). Stage with radix p and
// Ns points already combined: work item j in [0, N/p) reads x[j + q N/p], q < p,
// twiddles element q by w_{Ns p}^{(j mod Ns) q}, takes a p-point DFT and writes
// y[(j / Ns) Ns p + (j mod Ns) + q Ns]. The result is in natural order.
//
// `W` is a shared-memory table of exp(-2 pi i k / N), k < N (forward sign); the inverse
// uses its conjugate. Several transforms of length N stored back to back (stride N) are
// processed together. All threads of the block must call it. Returns the buffer
// (buf or tmp) that holds the result.
// ------------------------------------------------------------------------------------
struct FftPlan {
  int n;
  int nrad;
  int rad[12];
};

__host__ __device__ inline FftPlan fft_plan(int N) {
  FftPlan p;
  p.n = N;
  p.nrad = 0;
  int n = N;
  const int order[6] = {16, 8, 4, 2, 3, 5};
  for (int o = 0; o < 6; ++o) {
    while (n % order[o] == 0 && p.nrad < 12) {
      p.rad[p.nrad++] = order[o];
      n /= order[o];
    }
  }
  if (n != 1) p.nrad = -1;  // unsupported length
  return p;
}

// Shared-memory layout of FFT data and FFT twiddle tables: one pad slot per 16 elements,
// so that the strided Stockham stores y[j P + u] and twiddle reads W[k q] hit distinct banks.
__host__ __device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int fsz(int n) { return n > 0 ? fpad(n - 1) + 1 : 0; }

// twiddle idx of a padded table of exp(-2 pi i k / N)
__device__ __forceinline__ float2 tw(const float2* W, int idx, int sign) {
  float2 w = W[fpad(idx)];
  return sign < 0 ? w : make_float2(w.x, -w.y);
}

// n / d for 0 <= n < 2^32 / d with a precomputed multiplier m = floor((2^32 - 1) / d) + 1
// (exact in that range: n m / 2^32 lies in [n/d, n/d + n/2^32) and frac(n/d) <= 1 - 1/d).
// For d = 1 the multiplier wraps to 0, which stands for "divide by one".
__device__ __forceinline__ unsigned fast_div(unsigned n, unsigned m) { return m ? __umulhi(n, m) : n; }
__host__ __device__ __forceinline__ unsigned div_magic(unsigned d) { return 0xFFFFFFFFu / d + 1u; }

// radix-4 butterfly: out_k = sum_n a_n w_4^{nk} (w_4 = -i forward, +i inverse)
__device__ __forceinline__ void bfly4(float2 a0, float2 a1, float2 a2, float2 a3, int sign, float2& o0, float2& o1,
                                      float2& o2, float2& o3) {
  const float2 s0 = cadd(a0, a2), d0 = csub(a0, a2);
  const float2 s1 = cadd(a1, a3), d1 = csub(a1, a3);
  const float2 d1w = sign < 0 ? make_float2(d1.y, -d1.x) : make_float2(-d1.y, d1.x);
  o0 = cadd(s0, s1);
  o1 = cadd(d0, d1w);
  o2 = csub(s0, s1);
  o3 = csub(d0, d1w);
}

// 16-point DFT in registers: n = 4 n1 + n2, k = k1 + 4 k2; inner twiddles w_16^{n2 k1}
// taken from the length-N table (16 divides N)
__device__ __forceinline__ void dft16(float2* v, const float2* W, int N, int sign) {
  const int s16 = N / 16;
  float2 t[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 r0, r1, r2, r3;
    bfly4(v[n2], v[4 + n2], v[8 + n2], v[12 + n2], sign, r0, r1, r2, r3);
    t[n2 * 4 + 0] = r0;
    t[n2 * 4 + 1] = n2 == 0 ? r1 : cmul(r1, tw(W, n2 * 1 * s16, sign));
    t[n2 * 4 + 2] = n2 == 0 ? r2 : cmul(r2, tw(W, n2 * 2 * s16, sign));
    t[n2 * 4 + 3] = n2 == 0 ? r3 : cmul(r3, tw(W, n2 * 3 * s16, sign));
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
    bfly4(t[0 * 4 + k1], t[1 * 4 + k1], t[2 * 4 + k1], t[3 * 4 + k1], sign, v[k1], v[k1 + 4], v[k1 + 8], v[k1 + 12]);
}

// 8-point DFT in registers: n = 4 n1 + n2 (n1 < 2), k = k1 + 2 k2; inner twiddles w_8^{n2 k1}
__device__ __forceinline__ void dft8(float2* v, const float2* W, int N, int sign) {
  const int s8 = N / 8;
  float2 t0[4], t1[4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    t0[n2] = cadd(v[n2], v[4 + n2]);
    const float2 d = csub(v[n2], v[4 + n2]);
    t1[n2] = n2 == 0 ? d : cmul(d, tw(W, n2 * s8, sign));
  }
  bfly4(t0[0], t0[1], t0[2], t0[3], sign, v[0], v[2], v[4], v[6]);
  bfly4(t1[0], t1[1], t1[2], t1[3], sign, v[1], v[3], v[5], v[7]);
}

template <int P>
__device__ __forceinline__ void fft_stage(const float2* x, float2* y, int N, int Ns, int batch, int bstride,
                                          const float2* W, int sign, int tid, int nthreads) {
  const int Np = N / P;
  const int step = N / (Ns * P);
  const int items = batch * Np;
  const unsigned mNp = div_magic((unsigned)Np), mNs = div_magic((unsigned)Ns);
  for (int it = tid; it < items; it += nthreads) {
    const int b = (int)fast_div((unsigned)it, mNp);
    const int j = it - b * Np;
    const float2* xb = x + b * bstride;
    float2* yb = y + b * bstride;
    const int jd = (int)fast_div((unsigned)j, mNs);
    const int k = j - jd * Ns;
    float2 v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = xb[fpad(j + q * Np)];
#pragma unroll
    for (int q = 1; q < P; ++q) v[q] = cmul(v[q], tw(W, k * q * step, sign));   // k q step < N
    const int base = jd * Ns * P + k;
    if (P == 16 || P == 8) {
      if (P == 16) dft16(v, W, N, sign);
      else dft8(v, W, N, sign);
#pragma unroll
      for (int u = 0; u < P; ++u) yb[fpad(base + u * Ns)] = v[u];
    } else if (P == 2) {
      yb[fpad(base)] = cadd(v[0], v[1]);
      yb[fpad(base + Ns)] = csub(v[0], v[1]);
    } else if (P == 4) {
      const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
      const float2 b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
      // b1 times w_4: forward (-i) -> (b1.y, -b1.x); inverse (+i) -> (-b1.y, b1.x)
      const float2 b1w = sign < 0 ? make_float2(b1.y, -b1.x) : make_float2(-b1.y, b1.x);
      yb[fpad(base)] = cadd(a0, b0);
      yb[fpad(base + Ns)] = cadd(a1, b1w);
      yb[fpad(base + 2 * Ns)] = csub(a0, b0);
      yb[fpad(base + 3 * Ns)] = csub(a1, b1w);
    } else {
      // p-point DFT with the table: w_p^{qu} = W[((q u) mod p) N/p]
#pragma unroll
      for (int u = 0; u < P; ++u) {
        float2 acc = v[0];
#pragma unroll
        for (int q = 1; q < P; ++q) cfma(acc, v[q], tw(W, ((q * u) % P) * Np, sign));
        yb[fpad(base + u * Ns)] = acc;
      }
    }
  }
}

// Transforms `batch` sequences of length plan.n stored bstride apart in buf (element i of a
// sequence at fpad(i); bstride >= fsz(n)); W is the padded twiddle table (element k at
// fpad(k)); tmp is the ping-pong buffer of the same shape. Every thread of the block must
// call it.
__device__ inline float2* fft_smem(float2* buf, float2* tmp, const FftPlan& plan, int batch, int bstride,
                                   const float2* W, int sign, int tid, int nthreads) {
  const int N = plan.n;
  float2* x = buf;
  float2* y = tmp;
  int Ns = 1;
  for (int st = 0; st < plan.nrad; ++st) {
    const int p = plan.rad[st];
    if (p == 16) fft_stage<16>(x, y, N, Ns, batch, bstride, W, sign, tid, nthreads);
    else if (p == 8) fft_stage<8>(x, y, N, Ns, batch, bstride, W, sign, tid, nthreads);
    else if (p == 4) fft_stage<4>(x, y, N, Ns, batch, bstride, W, sign, tid, nthreads);
    else if (p == 2) fft_stage<2>(x, y, N, Ns, batch, bstride, W, sign, tid, nthreads);
    else if (p == 3) fft_stage<3>(x, y, N, Ns, batch, bstride, W, sign, tid, nthreads);
    else fft_stage<5>(x, y, N, Ns, batch, bstride, W, sign, tid, nthreads);
    __syncthreads();
    float2* t = x;
    x = y;
    y = t;
    Ns *= p;
  }
  return x;
}

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): round (c0,c1,c2,c3) ->
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); key += (W0, W1).
// ------------------------------------------------------------------------------------
struct U32x4 {
  uint32_t v[4];
};

__host__ __device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                         uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  U32x4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

#define TTS_PURPOSE_LINES 1u
#define TTS_PURPOSE_INIT 2u

// ------------------------------------------------------------------------------------
// Per-handle device workspace and the frame kernel's parameters.
// ------------------------------------------------------------------------------------
// scalars (double) kept across frames
enum { SC_W = 0, SC_ABAR_A = 1, SC_ABAR_B = 2, SC_T = 3, SC_COUNT = 8 };
// scalars of the frame in flight
enum { SF_W = 0, SF_RHO = 1, SF_ABAR_A = 2, SF_ABAR_B = 3, SF_ALPHA_A = 4, SF_ALPHA_B = 5, SF_COUNT = 8 };

// Shared-memory layout of the frame kernel (bytes offsets), computed identically on the
// host (launch size) and the device (carving).
struct FrameLayout {
  int Wx, Wy, rows, misc, red, myA, myA0, myB, myB0, Gf, GJa, GJb, gjx, vec, yb, chunk;
  int chunk_f2;   // capacity of the chunk region in float2
  int bytes;
};

__host__ __device__ inline FrameLayout frame_layout(int Nx, int Ny, int R, int rA, int rB, int MC) {
  FrameLayout L;
  int off = 0;
  auto take = [&](int bytes) {
    off = (off + 15) & ~15;
    int o = off;
    off += bytes;
    return o;
  };
  const int f2 = 8;
  L.Wx = take(f2 * Nx);
  L.Wy = take(f2 * fsz(Ny));       // padded FFT twiddle table
  L.rows = take(4 * Nx);
  L.misc = take(4 * 8);
  L.red = take(4 * 2 * TTS_THREADS);
  L.myA = take(f2 * rA * R);
  L.myA0 = take(f2 * rA * R);
  L.myB = take(f2 * rB * R);
  L.myB0 = take(f2 * rB * R);
  const int Rq = R <= 32 ? 32 : 64;   // ridge inverse padded to 32 or 64, row stride + 8
  L.Gf = take(f2 * R * R);
  L.GJa = take(f2 * Rq * (Rq + 8));
  L.GJb = take(f2 * R * R);        // low parts of the ridge matrix; B^H B for the factor step
  L.gjx = take(f2 * 136);          // pivot rows of the inverse (2 slots x 64), sweep flags
  L.vec = take(f2 * (6 * R + 16));
  L.yb = take(f2 * MC * rB);       // Yt block of this CTA's B rows, kept when |S| <= MC
  const int rmax = rA > rB ? rA : rB;
  int cf = MC * (rmax + rB + 3 * R);
  if (cf < 2 * fsz(Ny)) cf = 2 * fsz(Ny);     // at least one row transform (ping-pong)
  L.chunk_f2 = cf;
  L.chunk = take(f2 * cf);
  L.bytes = off + 16;
  return L;
}

struct FrameParams {
  int Nx, Ny, R, K, C;
  int rA, rB, MC;                 // rows of A / B per CTA, m-chunk length
  int jacobi;
  int refine;                     // refinement sweeps of the ridge solve
  int ridge_ff_all;               // every MM iteration's readout sums in float-float (else the last one's)
  double lf, mu;
  float isx, isy;                 // 1/sqrt(Nx), 1/sqrt(Ny)
  FrameLayout lay;
  FftPlan plan_y;                 // length-Ny transform of the acquired rows
  float2* A;                      // Nx x R (state)
  float2* B;                      // Ny x R (state)
  float2* A0;                     // anchors A[t-1], B[t-1]
  float2* B0;
  const uint8_t* mask;            // Nx bytes
  const float2* yrows;            // |S| x Ny acquired rows (or the full Nx x Ny frame)
  int full_frame;                 // yrows is the full frame: row m of S is yrows[rows[m]]
  int yt_ready;                   // Yt was formed before the launch (tensor-core row transform)
  int kspace;                     // k-space factors (Alg. 2): selection instead of F_Nx[S,:], rows untransformed
  float2* Yt;                     // |S| x Ny: acquired rows times conj(F_Ny)
  int* rows;                      // S, increasing
  int* nrows;                     // |S|
  float2* AhS[2];                 // (F_Nx A)[S,:]  (|S| x R), ping-pong over iterations
  float* nA[2];                   // ||a_r||^2
  // The ridge system's sums in float-float: value = hi + lo (the hi array alone is the FP32
  // value the factor steps use)
  float2* MB;                     // B^H B (R x R), hi
  float2* MBlo;                   //   lo
  float2* P;                      // Yt conj(B) (|S| x R), hi
  float2* Plo;                    //   lo
  float2* MA;                     // Ahat_S^H Ahat_S (R x R), hi
  float2* MAlo;                   //   lo
  float2* partA;                  // [C][Nx][R] partial sums of AhS over row slices
  float* partNA;                  // [C][R]
  float4* partMB;                 // [C][R][R]  float-float partials (hi.x, hi.y, lo.x, lo.y)
  float4* partP;                  // [C][Nx][R]
  float4* partMA;                 // [C][R][R]
  double* sc;                     // SC_* (persistent)
  double* sf;                     // SF_* (frame in flight)
  float2* gamma;                  // R
  double2* gamma_d;               // R
  int* status;                    // [0] sticky non-finite flag, [1 + c] per-CTA flag of the frame
  const float2* Wx;               // exp(-2 pi i k / Nx), k < Nx
  const float2* Wy;               // exp(-2 pi i k / Ny)
};

// Steps of one frame: 0 = ingest (row transforms, anchors, partial sums over the rows of
// A and of B^H B), 1 = Ahat_S by rows with its Gram partials, partial sums of P, 2 = reduce
// the float-float sums; then per MM iteration k: 3 + 4k + {0: ridge solve and A step,
// 1: Ahat'_S by rows with its Gram partials, 2: B step, 3: reduce the float-float sums};
// the last iteration has no step 3.
__host__ __device__ inline int frame_num_steps(int K) { return 4 * K + 2; }

// One line-sampler call (probabilities, then the draw) as a job of a batched launch.
struct SamplerJob {
  const float2* A;
  int Nx, Ny, R;
  const double* p_in;   // given probabilities, or NULL
  double* p_out;        // probabilities out, or NULL
  int policy;
  double vd_alpha;
  int k_lines, central;
  unsigned long long seed, ctr;
  int with_replacement;
  const float2* Wx;
  uint8_t* mask_out;
  uint8_t* mask_out2;   // optional second copy, or NULL
  int fft_cols;         // columns of A transformed together
  int no_fft;           // scores on the rows of A itself (k-space factor)
  unsigned int* done;   // optional word set to done_value once the masks are written (mapped memory)
  unsigned int done_value;
};

// One image X = A diag(gamma) B^T as a job of a batched launch: tiles [tile0, tile0 + tiles).
struct ImageJob {
  const float2* A;
  const float2* B;
  const float2* gamma;
  float2* X;
  int Nx, Ny, R;
  int tile0, tiles;
};

// host-side launchers (tts_kernels.cu, tts_frame.cu)
int launch_frame(const FrameParams& p, int launch_mode, cudaStream_t st);
// Cluster size and chunk length: requested_C = 0 picks the smallest preferred size whose
// layout fits; smem_limit = 0 means the device's opt-in maximum.
int frame_configure(FrameParams& p, int requested_C, int smem_limit = 0);
int frame_own(const FrameParams& p);
// Persistent launch over a queue of frames (queue_n[0] = 0, queue_n[1] = count): `clusters`
// clusters of C CTAs with `smem` bytes of dynamic shared memory each.
int frame_batch_limits(int own, int C, int* max_dyn_smem, int* max_clusters);
int launch_frame_batch(int own, int C, int clusters, int smem, const FrameParams* ps, int* queue_n, cudaStream_t st);
SamplerJob sampler_job(const float2* A, int Nx, int Ny, int R, const double* p_in, double* p_out, int policy,
                       double vd_alpha, int k_lines, int central, uint64_t seed, uint64_t ctr, int with_replacement,
                       const float2* Wx, uint8_t* mask_out, uint8_t* mask_out2);
int launch_sampler_batch(const SamplerJob* jobs, const int* n, int capacity, cudaStream_t st);
int launch_image_batch(const ImageJob* jobs, const int* n, int grid, cudaStream_t st);
int launch_image(const float2* A, const float2* B, const float2* gamma, float2* X, int Nx, int Ny, int R,
                 cudaStream_t st);
int launch_sampler(const float2* A, int Nx, int Ny, int R, const double* p_in, double* p_out, int policy,
                   double vd_alpha, int k_lines, int central, uint64_t seed, uint64_t ctr, int with_replacement,
                   const float2* Wx, uint8_t* mask_out, uint8_t* mask_out2, cudaStream_t st, int no_fft = 0,
                   unsigned int* done = nullptr, unsigned int done_value = 0);
void tts_internal_set_error(const char* msg);   // message returned by tts_last_error
int launch_fft2d(const float2* in, float2* out, int batch, int Nx, int Ny, int inverse, const float2* Wx,
                 const float2* Wy, float2* scratch, cudaStream_t st);
int launch_ridge(const double2* G, const double2* h, int R, double2* gamma, cudaStream_t st);
// batched 2D DFT for square N in {64, 128, 256} as one persistent launch over row and
// column band tasks (tts_fft_square.cu)
bool fft2d_square_ok(int Nx, int Ny);
// Times the square kernel's launch shapes (CTAs per SM, row-ahead lag) on in/out (batch
// images of N x N) and records the fastest for later launches of (device, N, direction);
// synchronous on the legacy default stream.
int tune_fft2d_square(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
                      int reps, double* best_ms, int* best_per_sm, double* best_lag);
// withhold >= 0 (test hook): the image whose row tasks publish nothing, so that the waits of
// its column tasks run out after `limit` SM clocks
int launch_fft2d_square(const float2* in, float2* out, int batch, int N, int inverse, const float2* W, int* err,
                        cudaStream_t st, int withhold = -1, long long limit = 2000000000LL);
// batched 2D DFT for other Nx x Ny whose line lengths both have a band shape: a row-band and a
// column-band launch per group of images that fits L2 (tts_fft_lines.cu)
bool fft2d_lines_ok(int Nx, int Ny);
int launch_fft2d_lines(const float2* in, float2* out, int batch, int Nx, int Ny, int inverse, const float2* Wx,
                       const float2* Wy, cudaStream_t st);
// 2D DFT as tensor-core matrix products (tts_dft_gemm.cu)
bool dft_gemm_size_ok(int N);
// Inverse unitary DFT of the acquired rows (mask lines) of a frame, Yt = y_S conj(F_Ny),
// row-major |S| x Ny, on the tensor cores.
int launch_row_dft(const float2* y, float2* yt, const uint8_t* mask, int Nx, int Ny, int full_frame, int split,
                   int* err, cudaStream_t st, int withhold = -1, long long limit = 2000000000LL);
// withhold >= 0 (test hook): the first pass's K' chunk whose copy and producer arrival are
// withheld, so that the waits for it run out after `limit` SM clocks
int launch_dft2d_gemm(const float2* in, float2* out, float2* tmp, int batch, int Nx, int Ny, int inverse,
                      int split, int* err, cudaStream_t st, int withhold = -1, long long limit = 2000000000LL);
int launch_init_factors(float2* A, int N, int R, uint64_t seed, uint32_t which, cudaStream_t st);
