// Per-frame MM iterations of the online tensor-subspace tracker (Alg. 3 with one coil,
// S1 ridge step for gamma_t and S2 majorized factor steps, §III-A), GB300 design.
//
// Everything a frame needs is computed from factor-sized quantities, using the
// separability of the 2D DFT with Cartesian line masks (Omega = S x [Ny]):
//   F(a b^T) = (F_Nx a)(F_Ny b)^T, F unitary and symmetric, so with
//   Ahat_S = (F_Nx A)[S,:] (|S| x R) and Yt = y_S conj(F_Ny) (|S| x Ny, once per frame):
//     Phi^H Phi = (Ahat_S^H Ahat_S) .* (B^H B)            (Gram of the masked rank-one DFTs)
//     Phi^H y   = colsum(conj(Ahat_S) .* P),  P = Yt conj(B)
//     Theta conj(B)    = conj(F_Nx)[:,S] (P - Ahat_S diag(gamma) (B^H B)^T)
//     Theta'^T conj(A) = Yt^T conj(Ahat'_S) - B diag(gamma) (Ahat'_S^H Ahat'_S)^T
// with Theta = F^{-1}(P_Omega(y - F(A diag(gamma) B^T))) the back-projected residual of
// Alg. 3 (S2). These are the masked 2D DFTs of the rank-one images and the inverse 2D DFT
// of the residual, evaluated in a different order.
//
// The frame runs as one kernel on a thread-block cluster of C CTAs. CTA c owns a slice of
// the rows of A and of B and keeps them, with their anchors, in shared memory for the
// whole frame. Sums over rows go through per-CTA partial sums that one phase writes and
// the next phase reduces (each CTA a slice of the entries). Quantities indexed by the
// acquired rows m stream through shared memory in chunks of MC rows, so shared memory
// stays bounded for any |S|. Phases are separated by cluster barriers (or run as
// separate launches). The R x R ridge system is solved in FP32 (Gauss-Jordan inverse)
// with iterative refinement whose residuals are formed in float-float arithmetic, which
// gives FP64-grade solutions on the FP32 pipes.
#include <cooperative_groups.h>

#include <algorithm>

#include "tts_fft_band.cuh"
#include "tts_internal.cuh"

namespace cg = cooperative_groups;

namespace {

struct Slice {
  int lo, hi;
};
__device__ __forceinline__ Slice slice_of(int n, int parts, int idx) {
  const int per = (n + parts - 1) / parts;
  const int lo = min(n, idx * per);
  return {lo, min(n, lo + per)};
}

struct SM {
  float2 *Wx, *Wy;
  int* rows;
  int* misc;  // [0] |S|, [1] non-finite flag
  float* red;
  float2 *A, *A0, *B, *B0;  // this CTA's rows (rA x R, rB x R)
  float2 *Gf;               // R x R ridge matrix (hi)
  float2 *GJa, *GJb;        // the ridge inverse (32 x 40 or 64 x 72) / R x R products
  float2* Pk;               // pivot rows of the inverse and the refinement flags
  float2 *gam, *glo, *h, *rr, *tmpv;  // R each
  double* ds;               // 8 doubles
  float* fs;                // 8 floats
  float2* yb;               // Yt[m][j] for this CTA's B rows j (|S| <= MC)
  bool yb_ready;
  float2* chunk;
};

__device__ SM carve(const FrameParams& p, unsigned char* base) {
  const FrameLayout& L = p.lay;
  SM s;
  s.Wx = (float2*)(base + L.Wx);
  s.Wy = (float2*)(base + L.Wy);
  s.rows = (int*)(base + L.rows);
  s.misc = (int*)(base + L.misc);
  s.red = (float*)(base + L.red);
  s.A = (float2*)(base + L.myA);
  s.A0 = (float2*)(base + L.myA0);
  s.B = (float2*)(base + L.myB);
  s.B0 = (float2*)(base + L.myB0);
  s.Gf = (float2*)(base + L.Gf);
  s.GJa = (float2*)(base + L.GJa);
  s.GJb = (float2*)(base + L.GJb);
  s.Pk = (float2*)(base + L.gjx);
  float2* v = (float2*)(base + L.vec);
  const int R = p.R;
  s.gam = v;
  s.glo = v + R;
  s.h = v + 2 * R;
  s.rr = v + 3 * R;
  s.tmpv = v + 4 * R;
  s.ds = (double*)(v + 6 * R);   // vec region holds 8R float2: 6R for vectors, then 8 doubles + 8 floats
  s.fs = (float*)(s.ds + 8);
  s.yb = (float2*)(base + L.yb);
  s.yb_ready = false;
  s.chunk = (float2*)(base + L.chunk);
  return s;
}

// ---------------------------------------------------------------------------------
// float-float helpers (error-free transformations)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
// (hi, lo) += v, renormalised
__device__ __forceinline__ void ff_add_f(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  e += lo;
  fast_two_sum(s, e, hi, lo);
}
__device__ __forceinline__ void ff_add_ff(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  e += lo + l2;
  fast_two_sum(s, e, hi, lo);
}

// Float-float accumulation of sums of products of FP32 numbers (the ridge system's sums):
// every product exact (two_prod), every addition to the high part error-free (two_sum), the
// product and addition errors summed in the low part (the compensated dot product of Ogita,
// Rump and Oishi, 2005: the result is as accurate as if computed with twice the working
// precision); the pair is renormalised where it is read (cff_pack, ff_add_ff).
// hi + lo += a1 b1 + a2 b2
__device__ __forceinline__ void ff_acc2(float& hi, float& lo, float a1, float b1, float a2, float b2) {
  float p, pe, s, e;
  two_prod(a1, b1, p, pe);
  two_sum(hi, p, s, e);
  lo = lo + (e + pe);
  two_prod(a2, b2, p, pe);
  two_sum(s, p, hi, e);
  lo = lo + (e + pe);
}
// complex float-float accumulator (re: rh + rl, im: ih + il)
struct CFF {
  float rh, rl, ih, il;
};
__device__ __forceinline__ CFF cff_zero() { return CFF{0.f, 0.f, 0.f, 0.f}; }
// acc += conj(a) b
__device__ __forceinline__ void cff_macc(CFF& c, float2 a, float2 b) {
  ff_acc2(c.rh, c.rl, a.x, b.x, a.y, b.y);
  ff_acc2(c.ih, c.il, a.x, b.y, -a.y, b.x);
}
// acc += conj(a) (b + bl): the product with the hi part exact, with the lo part rounded
__device__ __forceinline__ void cff_macc_ff(CFF& c, float2 a, float2 b, float2 bl) {
  cff_macc(c, a, b);
  const float2 t = cmulc(a, bl);
  float s, e;
  two_sum(c.rh, t.x, s, e);
  c.rh = s;
  c.rl = c.rl + e;
  two_sum(c.ih, t.y, s, e);
  c.ih = s;
  c.il = c.il + e;
}
__device__ __forceinline__ float4 cff_pack(const CFF& c) {
  float rh, rl, ih, il;
  fast_two_sum(c.rh, c.rl, rh, rl);
  fast_two_sum(c.ih, c.il, ih, il);
  return make_float4(rh, ih, rl, il);
}
// float-float sum of n float4 partials (hi.x, hi.y, lo.x, lo.y) `stride` apart, in order; for
// n <= 8 every load is issued before the first addition
__device__ __forceinline__ float4 ff_sum_partials(const float4* src, size_t stride, int n) {
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  if (n <= 8) {
    float4 v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = c < n ? src[c * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      ff_add_ff(rh, rl, v[c].x, v[c].z);
      ff_add_ff(ih, il, v[c].y, v[c].w);
    }
    return make_float4(rh, ih, rl, il);
  }
  for (int c = 0; c < n; c += 4) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = c + u < n ? src[(c + u) * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ff_add_ff(rh, rl, v[u].x, v[u].z);
      ff_add_ff(ih, il, v[u].y, v[u].w);
    }
  }
  return make_float4(rh, ih, rl, il);
}
// (q, r), q <= r, of entry idx of the row-major upper triangle of an R x R matrix
__device__ __forceinline__ void tri_pair(int idx, int R, int& q, int& r) {
  const float b = 2.f * (float)R + 1.f;
  int qq = (int)((b - sqrtf(b * b - 8.f * (float)idx)) * 0.5f);
  qq = max(0, min(R - 1, qq));
  while (qq > 0 && qq * R - qq * (qq - 1) / 2 > idx) --qq;
  while (qq + 1 < R && (qq + 1) * R - (qq + 1) * qq / 2 <= idx) ++qq;
  q = qq;
  r = qq + (idx - (qq * R - qq * (qq - 1) / 2));
}

// ---------------------------------------------------------------------------------
// Ridge solve (S1): (G_hi + G_lo) gamma = h_hi + h_lo, G Hermitian positive definite.
// An FP32 Gauss-Jordan inverse of G_hi (diagonal pivots: each is a Schur complement of a
// positive-definite matrix), gamma_0 = Ginv h_hi, then refinement sweeps
// gamma += Ginv (h - G gamma) with the residual formed in float-float arithmetic and gamma
// held as a float-float pair (gam + glo). Each sweep multiplies the error by about
// kappa(G) u_32, so two sweeps reach the float-float accuracy of the system; the sweeps
// stop once every correction is below sqrt(tol2) relative.
// ---------------------------------------------------------------------------------
// rows of the ridge matrix each warp of the Gauss-Jordan inverse keeps in registers (four:
// eight warps share each pivot step for R <= 32; measured 6.9 us against 7.4 us with eight rows)
#define TTS_GJ_ROWS 4

__device__ __forceinline__ void bar_named(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Gauss-Jordan inverse of G (R x R, row stride R; padded with the identity to RP x RP) into
// Gi (row stride RP + 8) by warps 0 .. RP/RW - 1: warp w keeps rows RW w .. RW w + RW - 1 in
// registers, lane l the columns l + 32q. Each pivot step publishes the scaled pivot row through `prow`
// (two slots, 2 RP float2) and the warps meet at named barrier 1; the pivot column comes
// from the lane that holds it by shuffles. The pivot loop is not unrolled (the kernel's
// phases run once per MM iteration, so compact code matters more than loop overhead):
// registers of the pivot row and column are picked by selects. Other warps return at once.
// Not inlined: its registers are then allocated apart from the rest of the frame code, whose
// changes otherwise moved its time per inverse between 6.6 and 8.3 us.
template <int RP, int RW>
__device__ __noinline__ void gj_inverse_warps(const float2* G, int R, float2* Gi, float2* prow) {
  constexpr int NW = RP / RW, CPL = RP / 32, LD = RP + 8;
  const unsigned FULL = 0xffffffffu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= NW) return;
  float2 M[RW][CPL];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int i = warp * RW + r, j = lane + 32 * q;
      M[r][q] = (i < R && j < R) ? G[i * R + j] : make_float2(i == j ? 1.f : 0.f, 0.f);
    }
#pragma unroll 1
  for (int k = 0; k < RP; ++k) {
    const int ow = k / RW, kr = k % RW, kl = k & 31, kq = k >> 5;
    float2* pr = prow + (k & 1) * RP;
    if (warp == ow) {
      float2 rowk[CPL];
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        rowk[q] = M[0][q];
#pragma unroll
        for (int r = 1; r < RW; ++r) rowk[q] = r == kr ? M[r][q] : rowk[q];
      }
      float2 dk = rowk[0];
#pragma unroll
      for (int q = 1; q < CPL; ++q) dk = q == kq ? rowk[q] : dk;
      float2 d;
      d.x = __shfl_sync(FULL, dk.x, kl);
      d.y = __shfl_sync(FULL, dk.y, kl);
      // approximate reciprocal: the inverse is only the refinement's preconditioner, and
      // this is on the dependent chain of the 32 pivot steps (pivots >= mu, never subnormal)
      const float inv = __fdividef(1.0f, cabs2(d));
      const float2 piv = make_float2(d.x * inv, -d.y * inv);   // 1 / d
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const float2 v = (lane + 32 * q == k) ? piv : cmul(rowk[q], piv);
        pr[lane + 32 * q] = v;
#pragma unroll
        for (int r = 0; r < RW; ++r) M[r][q] = r == kr ? v : M[r][q];
      }
    }
    bar_named(1, NW * 32);
    float2 rk[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) rk[q] = pr[lane + 32 * q];
    const float2 piv = pr[k];
    const bool own = warp == ow;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      float2 src = M[r][0];
#pragma unroll
      for (int q = 1; q < CPL; ++q) src = q == kq ? M[r][q] : src;
      float2 c;
      c.x = __shfl_sync(FULL, src.x, kl);
      c.y = __shfl_sync(FULL, src.y, kl);
      const float2 col = cmul(c, piv);
      const bool skip = own && r == kr;   // the pivot row itself
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        float2 gen = M[r][q];
        cfms(gen, c, rk[q]);
        const float2 v = (lane + 32 * q == k) ? make_float2(-col.x, -col.y) : gen;
        M[r][q] = skip ? M[r][q] : v;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int q = 0; q < CPL; ++q) Gi[(warp * RW + r) * LD + lane + 32 * q] = M[r][q];
}

// sum over the TPR lanes of a row group (lanes TPR g .. TPR g + TPR - 1) of a float2
template <int TPR>
__device__ __forceinline__ float2 sum_group(float2 v) {
#pragma unroll
  for (int o = TPR / 2; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Refinement against G_hi (sm.Gf, row stride R) + Glo and h_hi (sm.h) + hlo with the inverse
// Gi (row stride RP + 8): 8 threads per row (all R <= 64 rows in one pass of 512 threads).
// The result is gamma = sm.gam + sm.glo. Returns true once a sweep's largest correction is
// within sqrt(tol2) of the largest |gamma_r|. With slow2 > 0 (Gi the inverse of a nearby
// system, not of this one) it gives up, returning false, when a correction has not shrunk
// by sqrt(slow2) against the one before or when `iters` sweeps did not converge. Ends with a
// block barrier; the return value is the same in every thread.
template <int RP>
__device__ bool ridge_refine(SM& sm, int R, const float2* Gi, const float2* Glo, const float2* hlo, int iters,
                             float tol2, float slow2) {
  constexpr int LD = RP + 8, TPR = 8;   // 16 a row for R <= 32 measured slower
  const int tid = threadIdx.x, i = tid / TPR, u = tid % TPR;
  const bool row = i < R;
  // three (max |delta|^2, max |gamma|^2) pairs used in turn: sweep `it` reads pair it % 3
  // after its last barrier and clears pair (it + 1) % 3, last read two sweeps earlier
  unsigned* flags = (unsigned*)(sm.Pk + 128);
  if (tid < 6) flags[tid] = 0u;
  // gamma_0 = Ginv h_hi
  {
    float2 acc = make_float2(0.f, 0.f);
    if (row)
      for (int j = u; j < R; j += TPR) cfma(acc, Gi[i * LD + j], sm.h[j]);
    acc = sum_group<TPR>(acc);
    if (row && u == 0) {
      sm.gam[i] = acc;
      sm.glo[i] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  float prev = 0.f;
  for (int it = 0; it < iters; ++it) {
    unsigned* fl = flags + 2 * (it % 3);
    // r = h - G gamma, every product exact (two_prod), sums in float-float
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (row)
      for (int j = u; j < R; j += TPR) {
        const float2 g = sm.Gf[i * R + j];
        const float2 x = sm.gam[j], xl = sm.glo[j];
        float pp, e;
        two_prod(g.x, x.x, pp, e);
        ff_add_ff(rh, rl, pp, e);
        two_prod(-g.y, x.y, pp, e);
        ff_add_ff(rh, rl, pp, e);
        two_prod(g.x, x.y, pp, e);
        ff_add_ff(ih, il, pp, e);
        two_prod(g.y, x.x, pp, e);
        ff_add_ff(ih, il, pp, e);
        float2 cc = cmul(g, xl);
        if (Glo) cfma(cc, Glo[i * R + j], x);
        ff_add_f(rh, rl, cc.x);
        ff_add_f(ih, il, cc.y);
      }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) {
      const float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
      const float c = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
      ff_add_ff(rh, rl, a, b);
      ff_add_ff(ih, il, c, d);
    }
    if (row && u == 0) {
      float sh = sm.h[i].x, sl = hlo ? hlo[i].x : 0.f;
      ff_add_ff(sh, sl, -rh, -rl);
      float th = sm.h[i].y, tl = hlo ? hlo[i].y : 0.f;
      ff_add_ff(th, tl, -ih, -il);
      sm.rr[i] = make_float2(sh + sl, th + tl);
    }
    if (tid < 2) flags[2 * ((it + 1) % 3) + tid] = 0u;   // the next sweep's pair
    __syncthreads();
    // gamma += Ginv r
    float2 acc = make_float2(0.f, 0.f);
    if (row)
      for (int j = u; j < R; j += TPR) cfma(acc, Gi[i * LD + j], sm.rr[j]);
    acc = sum_group<TPR>(acc);
    if (row && u == 0) {
      float2 g = sm.gam[i], gl = sm.glo[i];
      atomicMax(fl, __float_as_uint(cabs2(acc)));
      atomicMax(fl + 1, __float_as_uint(cabs2(g)));
      ff_add_ff(g.x, gl.x, acc.x, 0.f);
      ff_add_ff(g.y, gl.y, acc.y, 0.f);
      sm.gam[i] = g;
      sm.glo[i] = gl;
    }
    __syncthreads();
    // float bits of non-negative floats order like unsigned integers
    const float d2 = __uint_as_float(fl[0]);
    if (d2 <= tol2 * __uint_as_float(fl[1])) return true;
    if (slow2 > 0.f && it > 0 && d2 > slow2 * prev) return false;
    prev = d2;
  }
  return slow2 <= 0.f;
}

// The whole solve; G_hi in sm.Gf, h_hi in sm.h. Uses sm.GJa (64 x 72 float2 at most) for the
// inverse and sm.Pk (136 float2) for the pivot rows and the sweep flags. With reuse > 0,
// sm.GJa still holds the inverse of the previous MM iteration's system, which the factor
// steps changed only a little: refinement with it as the preconditioner (up to `reuse`
// sweeps, each required to shrink the correction at least tenfold) replaces the
// Gauss-Jordan inverse, which is computed only when that does not converge. Ends with a block
// barrier.
__device__ void ridge_solve(SM& sm, int R, const float2* Glo, const float2* hlo, int iters, float tol2,
                            int reuse = 0) {
  if (R <= 32) {
    if (reuse > 0 && ridge_refine<32>(sm, R, sm.GJa, Glo, hlo, reuse, tol2, 1e-2f)) return;
    gj_inverse_warps<32, TTS_GJ_ROWS>(sm.Gf, R, sm.GJa, sm.Pk);
    __syncthreads();
    ridge_refine<32>(sm, R, sm.GJa, Glo, hlo, iters, tol2, 0.f);
  } else {
    if (reuse > 0 && ridge_refine<64>(sm, R, sm.GJa, Glo, hlo, reuse, tol2, 1e-2f)) return;
    gj_inverse_warps<64, TTS_GJ_ROWS>(sm.Gf, R, sm.GJa, sm.Pk);
    __syncthreads();
    ridge_refine<64>(sm, R, sm.GJa, Glo, hlo, iters, tol2, 0.f);
  }
}

// twiddles F[S_m, n] (without 1/sqrt(Nx)) for chunk rows m0.. and the rows lo.. of this CTA
__device__ __forceinline__ void fill_twiddles(const FrameParams& p, SM& sm, float2* TW, int m0, int mc, int lo,
                                              int nrows) {
  for (int e = threadIdx.x; e < mc * nrows; e += blockDim.x) {
    const int mm = e / nrows, nl = e - mm * nrows;
    if (p.kspace) {
      // k-space factors: F_Nx[S, :] becomes the row selection of S
      TW[e] = make_float2(sm.rows[m0 + mm] == lo + nl ? 1.f : 0.f, 0.f);
    } else {
      const int idx = (sm.rows[m0 + mm] * (lo + nl)) % p.Nx;
      TW[e] = sm.Wx[idx];
    }
  }
}

// ---------------------------------------------------------------------------------
// partial sums over this CTA's rows (shared by the ingest and the MM steps)
// ---------------------------------------------------------------------------------
// Ahat_S[m][r] = sum over this CTA's rows n of F[S_m, n] A[n][r] / sqrt(Nx), and ||a_r||^2;
// TW is chunk scratch of MC x (rows of A). With tw_ready the twiddles of a single chunk
// are already in TW.
template <bool SC>
__device__ void partials_A(const FrameParams& p, SM& sm, int cta, float2* TW, bool tw_ready) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nx = p.Nx, R = p.R, MC = p.MC;
  const int s = sm.misc[0];
  const Slice as = slice_of(Nx, p.C, cta);
  const int na = as.hi - as.lo;
  float2* part = p.partA + (size_t)cta * Nx * R;
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    if (!(tw_ready && s <= MC)) fill_twiddles(p, sm, TW, m0, mc, as.lo, na);
    __syncthreads();
    if (SC || (nth % R == 0 && mc * R <= 2 * nth)) {
      // the thread's (at most two) outputs share the column r = tid % R: A[n][r] is loaded
      // once for both, the two sums run as independent chains (arithmetic as below)
      const int cc = tid % R, q0 = tid / R, q1 = q0 + nth / R;
      const int ma = q0 < mc ? q0 : 0, mb = q1 < mc ? q1 : 0;
      float2 x0 = make_float2(0.f, 0.f), x1 = x0, y0 = x0, y1 = x0;
      int nl = 0;
      for (; nl + 1 < na; nl += 2) {
        const float2 av = sm.A[nl * R + cc], aw = sm.A[(nl + 1) * R + cc];
        cfma(x0, TW[ma * na + nl], av);
        cfma(x1, TW[ma * na + nl + 1], aw);
        cfma(y0, TW[mb * na + nl], av);
        cfma(y1, TW[mb * na + nl + 1], aw);
      }
      if (nl < na) {
        const float2 av = sm.A[nl * R + cc];
        cfma(x0, TW[ma * na + nl], av);
        cfma(y0, TW[mb * na + nl], av);
      }
      if (q0 < mc) part[(m0 + q0) * R + cc] = cscale(cadd(x0, x1), p.isx);
      if (q1 < mc) part[(m0 + q1) * R + cc] = cscale(cadd(y0, y1), p.isx);
    } else {
      for (int e = tid; e < mc * R; e += nth) {
        const int mm = e / R, r = e - mm * R;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        int nl = 0;
        for (; nl + 1 < na; nl += 2) {
          cfma(a0, TW[mm * na + nl], sm.A[nl * R + r]);
          cfma(a1, TW[mm * na + nl + 1], sm.A[(nl + 1) * R + r]);
        }
        if (nl < na) cfma(a0, TW[mm * na + nl], sm.A[nl * R + r]);
        part[(m0 + mm) * R + r] = cscale(cadd(a0, a1), p.isx);
      }
    }
    __syncthreads();
  }
  for (int r = tid; r < R; r += nth) {
    float acc = 0.f;
    for (int nl = 0; nl < na; ++nl) {
      const float2 v = sm.A[nl * R + r];
      acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
    }
    p.partNA[cta * R + r] = acc;
  }
}

// Yt[m][j] for m in [m0, m0 + mc) and this CTA's B rows j, into YB (mc x nb)
__device__ __forceinline__ void load_yb(const FrameParams& p, float2* YB, int m0, int mc, int lo, int nb) {
  const int n = mc * nb, nth = blockDim.x;
  for (int base = threadIdx.x; base < n; base += 4 * nth) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * nth;
      if (e < n) {
        const int mm = e / nb, jl = e - mm * nb;
        v[u] = p.Yt[(size_t)(m0 + mm) * p.Ny + lo + jl];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * nth;
      if (e < n) YB[e] = v[u];
    }
  }
}

// (B^H B)[q][r] and P[m][r] = sum over this CTA's rows j of Yt[m][j] conj(B[j][r]), as float4
// partials (hi, lo). With ff, the sums are accumulated in float-float (B^H B on its upper
// triangle, mirrored); else in FP32 (lo = 0).
template <int OWN>
__device__ void partials_B(const FrameParams& p, SM& sm, int cta, bool do_mb, bool do_p, bool ff) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nx = p.Nx, R = p.R, MC = p.MC, RR = R * R;
  const int s = sm.misc[0];
  const Slice bs = slice_of(p.Ny, p.C, cta);
  const int nb = bs.hi - bs.lo;
  if (do_mb) {
    float4* pmb = p.partMB + (size_t)cta * RR;
    if (ff) {
      const int RT = R * (R + 1) / 2;
      // whole blocks of nth pairs one thread a pair; the pairs of a last partial block (16 at
      // R = 32) one warp a pair, its rows over the lanes and the lanes' sums combined in
      // float-float by shuffles, so that a few threads do not run a whole pair alone
      const int full = RT - RT % nth;
      for (int idx = tid; idx < full; idx += nth) {
        int q, r;
        tri_pair(idx, R, q, r);
        CFF acc = cff_zero();
        for (int jl = 0; jl < nb; ++jl) cff_macc(acc, sm.B[jl * R + q], sm.B[jl * R + r]);
        const float4 v = cff_pack(acc);
        pmb[q * R + r] = v;
        if (q != r) pmb[r * R + q] = make_float4(v.x, -v.y, v.z, -v.w);
      }
      const int warp = tid >> 5, lane = tid & 31;
      for (int idx = full + warp; idx < RT; idx += nth >> 5) {
        int q, r;
        tri_pair(idx, R, q, r);
        CFF acc = cff_zero();
        for (int jl = lane; jl < nb; jl += 32) cff_macc(acc, sm.B[jl * R + q], sm.B[jl * R + r]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float a = __shfl_xor_sync(0xffffffffu, acc.rh, o), b = __shfl_xor_sync(0xffffffffu, acc.rl, o);
          const float c = __shfl_xor_sync(0xffffffffu, acc.ih, o), d = __shfl_xor_sync(0xffffffffu, acc.il, o);
          ff_add_ff(acc.rh, acc.rl, a, b);
          ff_add_ff(acc.ih, acc.il, c, d);
        }
        if (lane == 0) {
          const float4 v = cff_pack(acc);
          pmb[q * R + r] = v;
          if (q != r) pmb[r * R + q] = make_float4(v.x, -v.y, v.z, -v.w);
        }
      }
    } else {
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        const int e = tid + o * nth;
        if (e < RR) {
          const int q = e / R, r = e - q * R;
          float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
          int jl = 0;
          for (; jl + 1 < nb; jl += 2) {
            cfmac(a0, sm.B[jl * R + q], sm.B[jl * R + r]);
            cfmac(a1, sm.B[(jl + 1) * R + q], sm.B[(jl + 1) * R + r]);
          }
          if (jl < nb) cfmac(a0, sm.B[jl * R + q], sm.B[jl * R + r]);
          const float2 v = cadd(a0, a1);
          pmb[e] = make_float4(v.x, v.y, 0.f, 0.f);
        }
      }
    }
  }
  if (!do_p) return;
  float4* pp = p.partP + (size_t)cta * Nx * R;
  float2* YB = s <= MC ? sm.yb : sm.chunk;
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    if (s > MC || !sm.yb_ready) load_yb(p, YB, m0, mc, bs.lo, nb);
    __syncthreads();
    if (s <= MC) sm.yb_ready = true;
    for (int e = tid; e < mc * R; e += nth) {
      const int mm = e / R, r = e - mm * R;
      if (ff) {
        // Yt[m][j] conj(B[j][r]) = conj(B[j][r]) Yt[m][j]
        CFF acc = cff_zero();
        for (int jl = 0; jl < nb; ++jl) cff_macc(acc, sm.B[jl * R + r], YB[mm * nb + jl]);
        pp[(m0 + mm) * R + r] = cff_pack(acc);
      } else {
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        int jl = 0;
        for (; jl + 1 < nb; jl += 2) {
          cfma(a0, YB[mm * nb + jl], cconj(sm.B[jl * R + r]));
          cfma(a1, YB[mm * nb + jl + 1], cconj(sm.B[(jl + 1) * R + r]));
        }
        if (jl < nb) cfma(a0, YB[mm * nb + jl], cconj(sm.B[jl * R + r]));
        const float2 v = cadd(a0, a1);
        pp[(m0 + mm) * R + r] = make_float4(v.x, v.y, 0.f, 0.f);
      }
    }
    __syncthreads();
  }
}

// Rows [lo, hi) of S transformed by the register four-step FFT of the batched 2D DFT (line
// length N with a band shape): Yt[m] = y_m conj(F_N) / sqrt(N), T threads a row, as many rows a
// pass as there are thread groups and room in sm.chunk; bad |= 1 on a non-finite sample.
template <int N>
__device__ void rows_band(const FrameParams& p, SM& sm, int lo, int hi, int& bad) {
  using fftband::Shape;
  constexpr int T = Shape<N>::T, RL = Shape<N>::R, J = (RL + T - 1) / T;
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  const int per = min((int)blockDim.x / T, p.lay.chunk_f2 / N);
  const unsigned gmask = ((1u << T) - 1u) << ((threadIdx.x & 31) & ~(T - 1));
  for (int m0 = lo; m0 < hi; m0 += per) {
    const int m = m0 + g;
    if (g < per && m < hi) {   // uniform over the row's T threads
      const float2* src = p.yrows + (p.full_frame ? (size_t)sm.rows[m] * N : (size_t)m * N);
      float2 v[RL];
#pragma unroll
      for (int n2 = 0; n2 < RL; ++n2) v[n2] = src[t + T * n2];
#pragma unroll
      for (int n2 = 0; n2 < RL; ++n2)
        if (!isfinite(v[n2].x) || !isfinite(v[n2].y)) bad = 1;
      float2* sc = sm.chunk + g * N;
      fftband::dft_small<RL, true>(v, sm.Wy, N);
#pragma unroll
      for (int k2 = 1; k2 < RL; ++k2) v[k2] = cmul(v[k2], fftsmall::twn<true>(sm.Wy, t * k2));
#pragma unroll
      for (int k2 = 0; k2 < RL; ++k2) sc[k2 * T + (t ^ (k2 % T))] = v[k2];
      __syncwarp(gmask);
      float2* d = p.Yt + (size_t)m * N;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int k2 = t + T * j;
        if (J * T == RL || k2 < RL) {
          float2 u[T];
#pragma unroll
          for (int n1 = 0; n1 < T; ++n1) u[n1] = sc[k2 * T + (n1 ^ (k2 % T))];
          fftband::dft_small<T, true>(u, sm.Wy, N);
#pragma unroll
          for (int k1 = 0; k1 < T; ++k1) d[k2 + RL * k1] = cscale(u[k1], p.isy);
        }
      }
    }
    __syncthreads();   // the scratch rows are free for the next pass
  }
}

// the band-shape line lengths of the common cine sizes: rows by rows_band; false otherwise
__device__ __forceinline__ bool rows_band_any(const FrameParams& p, SM& sm, int lo, int hi, int& bad) {
  switch (p.Ny) {
    case 128: rows_band<128>(p, sm, lo, hi, bad); return true;
    case 192: rows_band<192>(p, sm, lo, hi, bad); return true;
    case 256: rows_band<256>(p, sm, lo, hi, bad); return true;
    default: return false;
  }
}

// ---------------------------------------------------------------------------------
// step 0: ingest the frame: inverse row transforms of this CTA's slice of S (Yt), the
// anchors A[t-1], B[t-1], and partial sums of Ahat_S, ||a||^2 and B^H B over this CTA's rows
// ---------------------------------------------------------------------------------
template <int OWN, bool SC>
__device__ void step_ingest(const FrameParams& p, SM& sm, int cta) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nx = p.Nx, Ny = p.Ny, R = p.R, C = p.C;
  const int s = sm.misc[0];
  const Slice ms = slice_of(s, C, cta);
  const int bsy = fsz(Ny);   // padded row stride of the transform buffers
  const int fft_rows = max(1, p.lay.chunk_f2 / (2 * bsy));
  int bad = 0;
  if (p.yt_ready)   // rows already transformed: check them only
    for (int e = ms.lo * Ny + tid; e < ms.hi * Ny; e += nth) {
      const float2 v = p.Yt[e];
      if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
    }
  const bool band = !p.yt_ready && !p.kspace && rows_band_any(p, sm, ms.lo, ms.hi, bad);
  for (int m0 = ms.lo; m0 < ms.hi && !p.yt_ready && !band; m0 += fft_rows) {
    const int nr = min(fft_rows, ms.hi - m0);
    float2* buf = sm.chunk;
    float2* tmp = sm.chunk + fft_rows * bsy;
    for (int base = tid; base < nr * Ny; base += 4 * nth) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = base + u * nth;
        if (e < nr * Ny) {
          const int mr = e / Ny;
          const size_t src = p.full_frame ? (size_t)sm.rows[m0 + mr] * Ny + (e - mr * Ny) : (size_t)m0 * Ny + e;
          v[u] = p.yrows[src];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = base + u * nth;
        if (e < nr * Ny) {
          if (!isfinite(v[u].x) || !isfinite(v[u].y)) bad = 1;
          const int mr = e / Ny;
          buf[mr * bsy + fpad(e - mr * Ny)] = v[u];
        }
      }
    }
    __syncthreads();
    float2* res = p.kspace ? buf : fft_smem(buf, tmp, p.plan_y, nr, bsy, sm.Wy, +1, tid, nth);
    for (int e = tid; e < nr * Ny; e += nth) {
      const int mr = e / Ny;
      p.Yt[(size_t)m0 * Ny + e] = cscale(res[mr * bsy + fpad(e - mr * Ny)], p.isy);
    }
    __syncthreads();
  }
  // a tensor-core row transform whose bounded wait ran out left Yt invalid: skip the frame
  if (p.yt_ready && ((volatile int*)p.status)[2 + TTS_MAX_CLUSTER]) bad |= 2;
  if (bad) atomicOr(&sm.misc[1], bad);
  // anchors A[t-1], B[t-1] (the rows this CTA holds in shared memory)
  for (int e = tid; e < p.rA * R; e += nth) sm.A0[e] = sm.A[e];
  for (int e = tid; e < p.rB * R; e += nth) sm.B0[e] = sm.B[e];
  const Slice as = slice_of(Nx, C, cta), bs = slice_of(Ny, C, cta);
  for (int e = tid; e < (as.hi - as.lo) * R; e += nth) p.A0[as.lo * R + e] = sm.A[e];
  for (int e = tid; e < (bs.hi - bs.lo) * R; e += nth) p.B0[bs.lo * R + e] = sm.B[e];
  partials_A<SC>(p, sm, cta, sm.chunk, false);
  partials_B<OWN>(p, sm, cta, true, false, p.ridge_ff_all || p.K == 1);
  __syncthreads();
  if (tid == 0) p.status[1 + cta] = sm.misc[1];
  if (cta == 0 && tid == 0) {
    const double w = p.lf * p.sc[SC_W] + 1.0;
    p.sf[SF_W] = w;
    p.sf[SF_RHO] = p.mu / w;
    p.sf[SF_ABAR_A] = p.sc[SC_ABAR_A];
    p.sf[SF_ABAR_B] = p.sc[SC_ABAR_B];
    *p.nrows = s;
  }
  if (cta == 0)
    for (int m = tid; m < s; m += nth) p.rows[m] = sm.rows[m];
}

// ---------------------------------------------------------------------------------
// step A: ridge solve for gamma (S1), majorized A step (S2) on this CTA's rows, then the
// partial sums of Ahat'_S and ||a'_r||^2 over those rows. OWN = outputs per thread.
// ---------------------------------------------------------------------------------
// Whether the ridge inverse stays in sm.GJa from one MM iteration to the next (the fused
// launch, with the gamma-weighted products gM / gMA then in sm.GJb and B^H B in the twiddle
// region of every CTA): the same answer in every CTA of the cluster.
__device__ __forceinline__ bool keep_inverse(const FrameParams& p, int fused) {
  const int per = (p.Nx + p.C - 1) / p.C;
  const int least = max(0, min(per, p.Nx - (p.C - 1) * per));   // rows of A in the smallest slice
  return fused && p.MC * least >= p.R * p.R;
}

// warp 0: alpha = sum_r |gamma_r|^2 w_r + rho and the MM step coefficients
// c0 = lf abar / den, c1 = alpha / den, c2 = 1 / den (den = lf abar + alpha) into sm.fs,
// alpha into sm.ds[0]
__device__ __forceinline__ void step_coefficients(const FrameParams& p, SM& sm, const float* wr, int wstride,
                                                  double rho, double abar) {
  const int tid = threadIdx.x;
  if (tid < 32) {
    float acc = 0.f;
    for (int r = tid; r < p.R; r += 32) acc = fmaf(cabs2(sm.gam[r]), wr[r * wstride], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (tid == 0) {
      const double alpha = rho + (double)acc;
      const float den = (float)(p.lf * abar + alpha);
      const float inv = 1.0f / den;
      sm.ds[0] = alpha;
      sm.ds[1] = abar;
      sm.fs[0] = (float)(p.lf * abar) * inv;
      sm.fs[1] = (float)alpha * inv;
      sm.fs[2] = inv;
      sm.fs[3] = (float)rho;
    }
  }
}

template <int OWN, bool LOADS_FIRST, bool SC>
__device__ void step_solve_A(const FrameParams& p, SM& sm, int cta, int k, int fused) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nx = p.Nx, R = p.R, C = p.C, MC = p.MC;
  const int s = sm.misc[0];
  const float2* AhS = p.AhS[k & 1];
  const Slice as = slice_of(Nx, C, cta);
  const int na = as.hi - as.lo;
  float2* AH = sm.chunk;                 // MC x R
  float2* PC = AH + MC * R;              // MC x R
  float2* QC = PC + MC * R;              // MC x R
  float2* TW = QC + MC * R;              // MC x na
  const int RR = R * R;
  int orow[OWN], ocol[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    orow[o] = e / R;
    ocol[o] = e - orow[o] * R;
  }
  // The ridge system (S1) in float-float: G = (Ahat_S^H Ahat_S) .* (B^H B) + mu I, the Gram of
  // the masked DFTs of the rank-one images (separable form), from the reduced float-float
  // sums; h = sum_m conj(Ahat_S[m][r]) P[m][r] = (Phi^H y)_r with P = hi + lo.
  float2* Glo = sm.GJb;   // low parts of G
  float2* hlo = sm.tmpv;
  // B^H B (hi) for the factor step after the solve: kept from the loads below in the twiddle
  // region, which the solve leaves alone (it is filled after gM is formed), when that region
  // is large enough; else read again into GJb after the solve
  const bool mb_tw = MC * na >= RR;
  float2* MBt = mb_tw ? TW : sm.GJb;
  // the loads of the system first, so that their L2 latencies overlap: this thread's first LF
  // entries of the reduced Gram factors and of the first chunk of Ahat_S, P and P's low part
  // (two each at most, one in the kernels with four or more outputs a thread, to bound the
  // registers they hold; none in the persistent multi-stream kernel, whose other state leaves
  // no registers for them; any further entries follow in loops, in the same arithmetic)
  constexpr int LF = !LOADS_FIRST ? 0 : (OWN >= 4 ? 1 : OWN);
  constexpr int LFA = LF > 0 ? LF : 1;
  const int mc0 = min(MC, s);
  float2 gah[LFA], gal[LFA], gbh[LFA], gbl[LFA], sa[LFA], sp[LFA], sl[LFA];
#pragma unroll
  for (int o = 0; o < LF; ++o) {
    const int e = tid + o * nth;
    if (e < RR) {
      gah[o] = p.MA[e];
      gal[o] = p.MAlo[e];
      gbh[o] = p.MB[e];
      gbl[o] = p.MBlo[e];
    }
  }
#pragma unroll
  for (int o = 0; o < LF; ++o) {
    const int e = tid + o * nth;
    if (e < mc0 * R) {
      sa[o] = AhS[e];
      sp[o] = p.P[e];
      sl[o] = p.Plo[e];
    }
  }
  {
    const float mu_hi = (float)p.mu, mu_lo = (float)(p.mu - (double)mu_hi);
    // (ah + al)(bh + bl) + mu [q == r] in float-float: ah bh exactly, ah bl + al bh rounded
    auto entry = [&](int e, float2 ah, float2 al, float2 bh, float2 bl) {
      if (mb_tw) MBt[e] = bh;
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      ff_acc2(rh, rl, ah.x, bh.x, -ah.y, bh.y);
      ff_acc2(ih, il, ah.x, bh.y, ah.y, bh.x);
      const float2 c1 = cmul(ah, bl), c2 = cmul(al, bh);
      float t, u;
      two_sum(rh, c1.x + c2.x, t, u);
      rh = t;
      rl = rl + u;
      two_sum(ih, c1.y + c2.y, t, u);
      ih = t;
      il = il + u;
      const int q = e / R, r = e - q * R;
      if (q == r) {
        ff_add_ff(rh, rl, mu_hi, mu_lo);
        ih = il = 0.f;
      }
      two_sum(rh, rl, rh, rl);
      two_sum(ih, il, ih, il);
      sm.Gf[e] = make_float2(rh, ih);
      Glo[e] = make_float2(rl, il);
    };
#pragma unroll
    for (int o = 0; o < LF; ++o) {
      const int e = tid + o * nth;
      if (e < RR) entry(e, gah[o], gal[o], gbh[o], gbl[o]);
    }
    for (int e = tid + LF * nth; e < RR; e += nth) entry(e, p.MA[e], p.MAlo[e], p.MB[e], p.MBlo[e]);
  }
  {
    // T threads per output r (T a power of two dividing 32), m strided over them
    int T = 32;
    while (T * R > nth) T >>= 1;
    const int r = tid / T, u = tid - r * T;
    const bool valid = r < R;
    CFF hacc = cff_zero();
    float2* QL = QC;   // low parts of P, staged
    for (int m0 = 0; m0 < s; m0 += MC) {
      const int mc = min(MC, s - m0);
      if (m0 == 0) {
#pragma unroll
        for (int o = 0; o < LF; ++o) {
          const int e = tid + o * nth;
          if (e < mc * R) {
            AH[e] = sa[o];
            PC[e] = sp[o];
            QL[e] = sl[o];
          }
        }
        for (int e = tid + LF * nth; e < mc * R; e += nth) {
          AH[e] = AhS[e];
          PC[e] = p.P[e];
          QL[e] = p.Plo[e];
        }
      } else {
        for (int e = tid; e < mc * R; e += nth) {
          AH[e] = AhS[m0 * R + e];
          PC[e] = p.P[m0 * R + e];
          QL[e] = p.Plo[m0 * R + e];
        }
      }
      __syncthreads();
      if (valid)
        for (int mm = u; mm < mc; mm += T) cff_macc_ff(hacc, AH[mm * R + r], PC[mm * R + r], QL[mm * R + r]);
      if (m0 + MC < s) __syncthreads();
    }
    for (int o = T >> 1; o > 0; o >>= 1) {
      const float a = __shfl_xor_sync(0xffffffffu, hacc.rh, o), b = __shfl_xor_sync(0xffffffffu, hacc.rl, o);
      const float c = __shfl_xor_sync(0xffffffffu, hacc.ih, o), d = __shfl_xor_sync(0xffffffffu, hacc.il, o);
      ff_add_ff(hacc.rh, hacc.rl, a, b);
      ff_add_ff(hacc.ih, hacc.il, c, d);
    }
    if (valid && u == 0) {
      const float4 v = cff_pack(hacc);
      sm.h[r] = make_float2(v.x, v.y);
      hlo[r] = make_float2(v.z, v.w);
    }
  }
  __syncthreads();
  const bool ffk = p.ridge_ff_all || k == p.K - 1;   // readout sums of this system in float-float
  // float-float readout sums: refine until the corrections fall below ~1e-13 relative; FP32
  // readout sums (an MM iteration before the last with TTS_RIDGE_FF_LAST): one sweep takes the
  // FP32 inverse's kappa u error to the accuracy of that system. After the first MM iteration
  // the previous iteration's inverse serves as the preconditioner (on the cine workloads
  // I - Ginv_prev G has spectral radius ~4e-3 from the first to the second iteration and
  // ~2e-4 from the second to the third), so the corrections shrink about a hundredfold per
  // sweep: at most 4 sweeps to 1e-6 relative, 12 to 1e-13
  const bool keep = keep_inverse(p, fused);
  ridge_solve(sm, R, Glo, hlo, ffk ? p.refine : 1, ffk ? 1e-26f : 1e-12f, keep && k > 0 ? (ffk ? 12 : 4) : 0);
  if (!mb_tw) {
    for (int e = tid; e < RR; e += nth) MBt[e] = p.MB[e];
    __syncthreads();
  }
  // alpha_A = sum |gamma_r|^2 ||b_r||^2 + rho (||b_r||^2 = (B^H B)[r][r])
  step_coefficients(p, sm, (const float*)MBt, 2 * (R + 1), p.sf[SF_RHO], p.sf[SF_ABAR_A]);
  if (cta == 0)
    for (int r = tid; r < R; r += nth) {
      p.gamma[r] = sm.gam[r];
      p.gamma_d[r] = make_double2((double)sm.gam[r].x + (double)sm.glo[r].x,
                                  (double)sm.gam[r].y + (double)sm.glo[r].y);
    }
  // gM[q][r] = gamma_q (B^H B)[r][q]
  float2* gM = keep ? sm.GJb : sm.GJa;
  for (int e = tid; e < RR; e += nth) {
    const int q = e / R, r = e - q * R;
    gM[e] = cmul(sm.gam[q], MBt[r * R + q]);
  }
  __syncthreads();
  if (cta == 0 && tid == 0) p.sf[SF_ALPHA_A] = sm.ds[0];
  // Theta conj(B) on this CTA's rows: T[n][r] = sum_m conj(F[S_m, n]) Q[m][r],
  // Q = P - Ahat_S diag(gamma) (B^H B)^T, accumulated over chunks of m
  float2 t0[OWN], t1[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) t0[o] = t1[o] = make_float2(0.f, 0.f);
  const int NO = na * R;
  const bool one_chunk = s <= MC;   // AH and PC still hold the whole of Ahat_S and P (staged for h)
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    if (!one_chunk)
      for (int e = tid; e < mc * R; e += nth) {
        AH[e] = AhS[m0 * R + e];
        PC[e] = p.P[m0 * R + e];
      }
    fill_twiddles(p, sm, TW, m0, mc, as.lo, na);
    __syncthreads();
    // with R dividing the block, every output of a thread (of Q and of Theta conj(B)) has column
    // tid % R: gM[q][r] and Q[m][r] are loaded once for all of them and the outputs' sums run as
    // independent chains (the same arithmetic per output as the general loops)
    const bool shared_col = SC || (OWN <= 4 && nth % R == 0 && mc * R <= OWN * nth);
    if (shared_col) {
      const int cc = tid % R, q0 = tid / R, step = nth / R;
      float2 a0[OWN], a1[OWN];
      int mr[OWN];
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        mr[o] = q0 + o * step < mc ? q0 + o * step : 0;
        a0[o] = PC[mr[o] * R + cc];
        a1[o] = make_float2(0.f, 0.f);
      }
      int q = 0;
      for (; q + 1 < R; q += 2) {
        const float2 g0 = gM[q * R + cc], g1 = gM[(q + 1) * R + cc];
#pragma unroll
        for (int o = 0; o < OWN; ++o) {
          cfms(a0[o], AH[mr[o] * R + q], g0);
          cfms(a1[o], AH[mr[o] * R + q + 1], g1);
        }
      }
      if (q < R) {
        const float2 g0 = gM[q * R + cc];
#pragma unroll
        for (int o = 0; o < OWN; ++o) cfms(a0[o], AH[mr[o] * R + q], g0);
      }
#pragma unroll
      for (int o = 0; o < OWN; ++o)
        if (q0 + o * step < mc) QC[(q0 + o * step) * R + cc] = cadd(a0[o], a1[o]);
    } else {
      for (int e = tid; e < mc * R; e += nth) {
        const int mm = e / R, r = e - mm * R;
        float2 a0 = PC[e], a1 = make_float2(0.f, 0.f);
        int q = 0;
        for (; q + 1 < R; q += 2) {
          cfms(a0, AH[mm * R + q], gM[q * R + r]);
          cfms(a1, AH[mm * R + q + 1], gM[(q + 1) * R + r]);
        }
        if (q < R) cfms(a0, AH[mm * R + q], gM[q * R + r]);
        QC[e] = cadd(a0, a1);
      }
    }
    __syncthreads();
    int ir[OWN], ic[OWN];
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const bool v = tid + o * nth < NO;
      ir[o] = v ? orow[o] : 0;
      ic[o] = v ? ocol[o] : 0;
    }
    int mm = 0;
    if (SC || (OWN <= 4 && nth % R == 0)) {
      const int cc = tid % R;
      for (; mm + 1 < mc; mm += 2) {
        const float2 qa = QC[mm * R + cc], qb = QC[(mm + 1) * R + cc];
#pragma unroll
        for (int o = 0; o < OWN; ++o) {
          cfmac(t0[o], TW[mm * na + ir[o]], qa);
          cfmac(t1[o], TW[(mm + 1) * na + ir[o]], qb);
        }
      }
      if (mm < mc) {
        const float2 qa = QC[mm * R + cc];
#pragma unroll
        for (int o = 0; o < OWN; ++o) cfmac(t0[o], TW[mm * na + ir[o]], qa);
      }
    } else {
      for (; mm + 1 < mc; mm += 2) {
#pragma unroll
        for (int o = 0; o < OWN; ++o) {
          cfmac(t0[o], TW[mm * na + ir[o]], QC[mm * R + ic[o]]);
          cfmac(t1[o], TW[(mm + 1) * na + ir[o]], QC[(mm + 1) * R + ic[o]]);
        }
      }
      if (mm < mc) {
#pragma unroll
        for (int o = 0; o < OWN; ++o) cfmac(t0[o], TW[mm * na + ir[o]], QC[mm * R + ic[o]]);
      }
    }
    __syncthreads();
  }
  // A step: grad = rho A - T diag(conj gamma); A <- c0 A0 + c1 A - c2 grad
  const float c0 = sm.fs[0], c1 = sm.fs[1], c2 = sm.fs[2], frho = sm.fs[3];
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    if (e < NO) {
      const float2 a = sm.A[e], a0 = sm.A0[e];
      const float2 tt = cscale(cadd(t0[o], t1[o]), p.isx);
      const float2 grad = csub(cscale(a, frho), cmul(tt, cconj(sm.gam[ocol[o]])));
      float2 an;
      an.x = fmaf(-c2, grad.x, fmaf(c1, a.x, c0 * a0.x));
      an.y = fmaf(-c2, grad.y, fmaf(c1, a.y, c0 * a0.y));
      sm.A[e] = an;
      p.A[as.lo * R + e] = an;
    }
  }
  __syncthreads();
  // partial sums over this CTA's rows: Ahat'_S[m][r] and ||a'_r||^2
  partials_A<SC>(p, sm, cta, TW, one_chunk);
}

// sum of C per-CTA partials stride apart, loads issued four at a time
__device__ __forceinline__ float2 sum_partials(const float2* src, size_t stride, int C) {
  float2 acc = make_float2(0.f, 0.f);
  for (int c = 0; c < C; c += 4) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = c + u < C ? src[(c + u) * stride] : make_float2(0.f, 0.f);
    acc = cadd(acc, cadd(cadd(v[0], v[1]), cadd(v[2], v[3])));
  }
  return acc;
}

// Reduce the per-CTA partials of Ahat_S by rows: this CTA sums the rows m of its slice of
// [0, |S|) (all R columns) into AhS[dst]; with ma, it then accumulates (Ahat_S^H Ahat_S) over
// those rows in float-float (upper triangle, mirrored) into its float4 partial partMA[cta],
// so that the Gram's other factor needs only one more cross-CTA reduction. It also reduces
// ||a_r||^2 for r in its slice of [0, R) into nA[dst].
__device__ void reduce_A_rows(const FrameParams& p, SM& sm, int cta, int dst, bool ma) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int R = p.R, C = p.C, Nx = p.Nx, RR = R * R;
  const int s = sm.misc[0];
  const Slice rs = slice_of(R, C, cta);
  for (int r = rs.lo + tid; r < rs.hi; r += nth) {
    float acc = 0.f;
    for (int c = 0; c < C; c += 4) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c + u < C ? p.partNA[(c + u) * R + r] : 0.f;
      acc += (v[0] + v[1]) + (v[2] + v[3]);
    }
    p.nA[dst][r] = acc;
  }
  const Slice ms = slice_of(s, C, cta);
  float2* out = p.AhS[dst];
  float2* rowbuf = sm.chunk;
  const int cap = max(1, min(ms.hi - ms.lo, p.lay.chunk_f2 / R));
  const int RT = R * (R + 1) / 2;
  constexpr int NI = (TTS_MAX_R * (TTS_MAX_R + 1) / 2 + TTS_THREADS - 1) / TTS_THREADS;
  CFF acc[NI];
#pragma unroll
  for (int u = 0; u < NI; ++u) acc[u] = cff_zero();
  for (int m0 = ms.lo; m0 < ms.hi; m0 += cap) {
    const int mc = min(cap, ms.hi - m0);
    for (int e = tid; e < mc * R; e += nth) {
      const float2 v = sum_partials(p.partA + (size_t)m0 * R + e, (size_t)Nx * R, C);
      out[(size_t)m0 * R + e] = v;
      if (ma) rowbuf[e] = v;
    }
    if (!ma) continue;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NI; ++u) {
      const int idx = tid + u * nth;
      if (idx < RT) {
        int q, r;
        tri_pair(idx, R, q, r);
        for (int mm = 0; mm < mc; ++mm) cff_macc(acc[u], rowbuf[mm * R + q], rowbuf[mm * R + r]);
      }
    }
    __syncthreads();
  }
  if (!ma) return;
  float4* pma = p.partMA + (size_t)cta * RR;
#pragma unroll
  for (int u = 0; u < NI; ++u) {
    const int idx = tid + u * nth;
    if (idx < RT) {
      int q, r;
      tri_pair(idx, R, q, r);
      const float4 v = cff_pack(acc[u]);
      pma[q * R + r] = v;
      if (q != r) pma[r * R + q] = make_float4(v.x, -v.y, v.z, -v.w);
    }
  }
}

// The single-chunk form of reduce_A_rows (|S| <= MC), run at the start of the phase that
// needs the result, with no cluster barrier of its own: every CTA sums the per-CTA partials
// of all |S| rows of Ahat_S into shared memory AR for itself and writes its slice of the rows
// to AhS[dst]; it sums ||a_r||^2 into nAs (shared, when given) and, on CTA 0, into nA[dst];
// with ma it accumulates its slice of the upper triangle of Ahat_S^H Ahat_S over all |S| rows
// in float-float (eight threads a pair, combined by shuffles) and writes those entries of
// MA / MAlo, which are then final. Ends with a block barrier.
__device__ void reduce_A_full(const FrameParams& p, SM& sm, int cta, int dst, float2* AR, float* nAs, bool ma) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int R = p.R, C = p.C, Nx = p.Nx;
  const int s = sm.misc[0];
  const Slice ms = slice_of(s, C, cta);
  if (C <= 8) {
    // two entries a thread at a time, all their loads issued before the first addition (the
    // additions in the order of sum_partials)
    for (int e0 = tid; e0 < s * R; e0 += 2 * nth) {
      float2 v[2][8];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int e = e0 + u * nth;
          v[u][c] = (e < s * R && c < C) ? p.partA[(size_t)c * Nx * R + e] : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = e0 + u * nth;
        if (e >= s * R) continue;
        float2 acc = make_float2(0.f, 0.f);
        acc = cadd(acc, cadd(cadd(v[u][0], v[u][1]), cadd(v[u][2], v[u][3])));
        if (C > 4) acc = cadd(acc, cadd(cadd(v[u][4], v[u][5]), cadd(v[u][6], v[u][7])));
        AR[e] = acc;
        if (e >= ms.lo * R && e < ms.hi * R) p.AhS[dst][e] = acc;
      }
    }
  } else {
    for (int e = tid; e < s * R; e += nth) {
      const float2 v = sum_partials(p.partA + e, (size_t)Nx * R, C);
      AR[e] = v;
      if (e >= ms.lo * R && e < ms.hi * R) p.AhS[dst][e] = v;
    }
  }
  for (int r = tid; r < R; r += nth) {
    float acc = 0.f;
    for (int c = 0; c < C; c += 4) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c + u < C ? p.partNA[(c + u) * R + r] : 0.f;
      acc += (v[0] + v[1]) + (v[2] + v[3]);
    }
    if (nAs) nAs[r] = acc;
    if (cta == 0) p.nA[dst][r] = acc;
  }
  __syncthreads();
  if (!ma) return;
  const int RT = R * (R + 1) / 2;
  const Slice ps = slice_of(RT, C, cta);
  // eight threads a pair when the slice fits one pass of the block that way, else four (one
  // pass for up to nth / 4 pairs: 66 at R = 32 with 8 CTAs)
  const int tpp = ps.hi - ps.lo <= nth / 8 ? 8 : 4;
  const int g = tid / tpp, u = tid % tpp;
  for (int base = ps.lo; base < ps.hi; base += nth / tpp) {   // uniform trip count
    const int idx = base + g;
    const bool valid = idx < ps.hi;
    int q = 0, r = 0;
    if (valid) tri_pair(idx, R, q, r);
    CFF acc = cff_zero();
    if (valid)
      for (int m = u; m < s; m += tpp) cff_macc(acc, AR[m * R + q], AR[m * R + r]);
    for (int o = tpp >> 1; o > 0; o >>= 1) {
      const float a = __shfl_xor_sync(0xffffffffu, acc.rh, o), b = __shfl_xor_sync(0xffffffffu, acc.rl, o);
      const float c = __shfl_xor_sync(0xffffffffu, acc.ih, o), d = __shfl_xor_sync(0xffffffffu, acc.il, o);
      ff_add_ff(acc.rh, acc.rl, a, b);
      ff_add_ff(acc.ih, acc.il, c, d);
    }
    if (valid && u == 0) {
      const float4 v = cff_pack(acc);
      p.MA[q * R + r] = make_float2(v.x, v.y);
      p.MAlo[q * R + r] = make_float2(v.z, v.w);
      if (q != r) {
        p.MA[r * R + q] = make_float2(v.x, -v.y);
        p.MAlo[r * R + q] = make_float2(v.z, -v.w);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// step B: majorized B step (S2) on this CTA's rows, then partials of B^H B and P
// ---------------------------------------------------------------------------------
template <int OWN, bool SC>
__device__ void step_B(const FrameParams& p, SM& sm, int cta, int k, bool last, int fused) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Ny = p.Ny, R = p.R, C = p.C, MC = p.MC;
  const int s = sm.misc[0];
  const int src = p.jacobi ? (k & 1) : ((k + 1) & 1);
  const float2* Ah = p.AhS[src];
  const float* nA = p.nA[src];
  const Slice bs = slice_of(Ny, C, cta);
  const int nb = bs.hi - bs.lo;
  float2* AH = sm.chunk;                 // MC x R
  float2* YB = s <= MC ? sm.yb : AH + MC * R;   // MC x nb
  const int RR = R * R;
  int orow[OWN], ocol[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    orow[o] = e / R;
    ocol[o] = e - orow[o] * R;
  }
  float* nAs = (float*)sm.tmpv;   // ||a_r||^2 in shared memory
  // |S| <= MC: Ahat'_S (and ||a'||^2, and the next Gram's Ahat'^H Ahat') reduced here, every
  // CTA for itself, instead of in a phase of its own
  const bool merged = s <= MC;
  float2* AR = sm.chunk + MC * R;
  if (merged) reduce_A_full(p, sm, cta, (k + 1) & 1, AR, p.jacobi ? nullptr : nAs, k + 1 < p.K);
  const bool own_ah = merged && !p.jacobi;   // the reduced rows are this step's Ahat
  // gamma: in a fused launch every CTA still holds the one it solved for (the same in all
  // CTAs); a launch per step reads CTA 0's copy
  for (int r = tid; r < R; r += nth) {
    if (!fused) sm.gam[r] = p.gamma[r];
    if (!own_ah) nAs[r] = nA[r];
  }
  // MA = Ahat^H Ahat (thread-owned entries) and U[j][r] = sum_m Yt[m][j] conj(Ahat[m][r])
  float2 ma[OWN], u[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) ma[o] = u[o] = make_float2(0.f, 0.f);
  const int NO = nb * R;
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    if (!own_ah)
      for (int e = tid; e < mc * R; e += nth) AH[e] = Ah[m0 * R + e];
    if (s > MC || !sm.yb_ready) load_yb(p, YB, m0, mc, bs.lo, nb);
    __syncthreads();
    if (s <= MC) sm.yb_ready = true;
    int mr[OWN], mq[OWN], uj[OWN], ur[OWN];
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const bool vm = tid + o * nth < RR, vu = tid + o * nth < NO;
      mr[o] = vm ? orow[o] : 0;
      mq[o] = vm ? ocol[o] : 0;
      uj[o] = vu ? orow[o] : 0;
      ur[o] = vu ? ocol[o] : 0;
    }
    const float2* AHm = own_ah ? AR : AH;
    if (SC || (OWN <= 4 && nth % R == 0)) {
      // every output of this thread has column tid % R (R divides the block): that column's
      // entry of Ahat is loaded once per m for all of them (same arithmetic as below)
      const int cc = tid % R;
      for (int mm = 0; mm < mc; ++mm) {
        const float2 ac = AHm[mm * R + cc];
#pragma unroll
        for (int o = 0; o < OWN; ++o) {
          cfmac(ma[o], AHm[mm * R + mr[o]], ac);
          cfmac(u[o], ac, YB[mm * nb + uj[o]]);
        }
      }
    } else {
      for (int mm = 0; mm < mc; ++mm) {
#pragma unroll
        for (int o = 0; o < OWN; ++o) {
          cfmac(ma[o], AHm[mm * R + mr[o]], AHm[mm * R + mq[o]]);
          cfmac(u[o], AHm[mm * R + ur[o]], YB[mm * nb + uj[o]]);
        }
      }
    }
    __syncthreads();
  }
  // gMA[q][r] = gamma_q MA[r][q]
  float2* gMA = keep_inverse(p, fused) ? sm.GJb : sm.GJa;
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    if (e < RR) gMA[ocol[o] * R + orow[o]] = cmul(sm.gam[ocol[o]], ma[o]);
  }
  // alpha_B = sum |gamma_r|^2 ||a_r||^2 + rho
  step_coefficients(p, sm, nAs, 1, p.sf[SF_RHO], p.sf[SF_ABAR_B]);
  __syncthreads();
  const float c0 = sm.fs[0], c1 = sm.fs[1], c2 = sm.fs[2], frho = sm.fs[3];
  // B step: T_B = U - B diag(gamma) MA^T, grad = rho B - T_B diag(conj gamma)
  float2 nbv[OWN];
  // the majorized step of output o from its T_B entry tb
  auto bstep = [&](int o, float2 tb) {
    const int e = tid + o * nth, r = ocol[o];
    const float2 b = sm.B[e], b0 = sm.B0[e];
    const float2 grad = csub(cscale(b, frho), cmul(tb, cconj(sm.gam[r])));
    nbv[o].x = fmaf(-c2, grad.x, fmaf(c1, b.x, c0 * b0.x));
    nbv[o].y = fmaf(-c2, grad.y, fmaf(c1, b.y, c0 * b0.y));
  };
  if (SC || (OWN <= 4 && nth % R == 0)) {
    // column tid % R for every output: gMA[q][r] loaded once per q for all of them, the
    // sums of all outputs as independent chains (same arithmetic as below)
    const int cc = tid % R;
    float2 t0[OWN], t1[OWN];
    int jr[OWN];
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      t0[o] = u[o];
      t1[o] = make_float2(0.f, 0.f);
      jr[o] = tid + o * nth < NO ? orow[o] : 0;
    }
    int q = 0;
    for (; q + 1 < R; q += 2) {
      const float2 g0 = gMA[q * R + cc], g1 = gMA[(q + 1) * R + cc];
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        cfms(t0[o], sm.B[jr[o] * R + q], g0);
        cfms(t1[o], sm.B[jr[o] * R + q + 1], g1);
      }
    }
    if (q < R) {
      const float2 g0 = gMA[q * R + cc];
#pragma unroll
      for (int o = 0; o < OWN; ++o) cfms(t0[o], sm.B[jr[o] * R + q], g0);
    }
#pragma unroll
    for (int o = 0; o < OWN; ++o)
      if (tid + o * nth < NO) bstep(o, cadd(t0[o], t1[o]));
  } else {
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const int e = tid + o * nth;
      if (e < NO) {
        const int jl = orow[o], r = ocol[o];
        float2 tb0 = u[o], tb1 = make_float2(0.f, 0.f);
        int q = 0;
        for (; q + 1 < R; q += 2) {
          cfms(tb0, sm.B[jl * R + q], gMA[q * R + r]);
          cfms(tb1, sm.B[jl * R + q + 1], gMA[(q + 1) * R + r]);
        }
        if (q < R) cfms(tb0, sm.B[jl * R + q], gMA[q * R + r]);
        bstep(o, cadd(tb0, tb1));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    if (e < NO) {
      sm.B[e] = nbv[o];
      p.B[bs.lo * R + e] = nbv[o];
    }
  }
  if (last) {
    if (cta == 0 && tid == 0) {
      p.sc[SC_W] = p.sf[SF_W];
      p.sc[SC_ABAR_A] = p.lf * p.sf[SF_ABAR_A] + p.sf[SF_ALPHA_A];
      p.sc[SC_ABAR_B] = p.lf * sm.ds[1] + sm.ds[0];
      p.sc[SC_T] += 1.0;
      p.sf[SF_ALPHA_B] = sm.ds[0];
    }
    return;
  }
  __syncthreads();
  // partials over this CTA's rows: B'^H B' and Yt conj(B'), in float-float for the last
  // MM iteration's ridge system (every iteration's with ridge_ff_all)
  partials_B<OWN>(p, sm, cta, true, true, p.ridge_ff_all || k + 1 == p.K - 1);
}

// Reduce the float-float per-CTA partials of B^H B, P and (with ma) Ahat_S^H Ahat_S, each CTA a
// slice of the entries, into their hi / lo arrays.
__device__ void reduce_sums(const FrameParams& p, SM& sm, int cta, bool ma) {
  const int R = p.R, C = p.C, Nx = p.Nx, RR = R * R;
  const int s = sm.misc[0];
  const int E1 = RR, E2 = E1 + s * R, E = E2 + (ma ? RR : 0);
  const Slice es = slice_of(E, C, cta);
  for (int e = es.lo + threadIdx.x; e < es.hi; e += blockDim.x) {
    const float4* src;
    size_t stride;
    float2 *hi, *lo;
    int o;
    if (e < E1) {
      src = p.partMB + e, stride = (size_t)RR, hi = p.MB, lo = p.MBlo, o = e;
    } else if (e < E2) {
      src = p.partP + (e - E1), stride = (size_t)Nx * R, hi = p.P, lo = p.Plo, o = e - E1;
    } else {
      src = p.partMA + (e - E2), stride = (size_t)RR, hi = p.MA, lo = p.MAlo, o = e - E2;
    }
    const float4 v = ff_sum_partials(src, stride, C);
    hi[o] = make_float2(v.x, v.y);
    lo[o] = make_float2(v.z, v.w);
  }
}

// Steps [step_begin, step_end) of one frame, run by CTA `cta` of the cluster that owns it.
template <int OWN, bool LOADS_FIRST, bool SC>
__device__ __forceinline__ void frame_run(const FrameParams& p, unsigned char* smem_raw, int cta, int step_begin,
                                          int step_end, int fused) {
  SM sm = carve(p, smem_raw);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int R = p.R;
  for (int e = tid; e < p.Nx; e += nth) sm.Wx[e] = p.Wx[e];
  for (int e = tid; e < p.Ny; e += nth) sm.Wy[fpad(e)] = p.Wy[e];
  if (tid < 8) sm.misc[tid] = 0;
  // this CTA's rows of the factors (and of the anchors after the ingest step)
  const Slice as = slice_of(p.Nx, p.C, cta), bs = slice_of(p.Ny, p.C, cta);
  block_copy(sm.A, p.A + as.lo * R, (as.hi - as.lo) * R);
  block_copy(sm.B, p.B + bs.lo * R, (bs.hi - bs.lo) * R);
  if (step_begin > 0) {
    block_copy(sm.A0, p.A0 + as.lo * R, (as.hi - as.lo) * R);
    block_copy(sm.B0, p.B0 + bs.lo * R, (bs.hi - bs.lo) * R);
  }
  __syncthreads();
  if (step_begin == 0) {
    // compact the line mask into the increasing list S (warp 0)
    if (tid < 32) {
      int count = 0;
      for (int base = 0; base < p.Nx; base += 32) {
        const int i = base + tid;
        const bool on = i < p.Nx && p.mask[i] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) sm.rows[count + __popc(bal & ((1u << tid) - 1u))] = i;
        count += __popc(bal);
      }
      if (tid == 0) sm.misc[0] = count;
    }
  } else {
    if (tid == 0) sm.misc[0] = *p.nrows;
    __syncthreads();
    for (int e = tid; e < sm.misc[0]; e += nth) sm.rows[e] = p.rows[e];
  }
  __syncthreads();
  cg::cluster_group cluster = cg::this_cluster();
  // |S| <= MC: the reduction of Ahat'_S after each A step runs at the start of the B step
  // (reduce_A_full), so its own step and the barrier before it are skipped (uniform: every
  // CTA has the same |S|)
  const bool merged = sm.misc[0] <= p.MC;
  for (int step = step_begin; step < step_end; ++step) {
    if (merged && step >= 3 && (step - 3) % 4 == 1) continue;
    if (step > step_begin) {
      // the cluster barrier releases every thread's earlier writes (shared and global) to
      // the cluster and acquires the others': the partial sums in global memory need no
      // separate fence (separate launches are ordered by the stream)
      if (fused) cluster.sync();
      else __syncthreads();
    }
    if (step > 0 && (step == 1 || step == step_begin)) {
      // the frame is rejected when any CTA saw a non-finite input sample (the flags are set by
      // the ingest step only, so one look after it suffices in a fused launch; a launch that
      // starts later in the frame looks again)
      int bad = 0;
      for (int c = 0; c < p.C; ++c) bad |= ((volatile int*)p.status)[1 + c];
      if (bad) {
        if (step == 1 && cta == 0 && tid == 0) {
          if (bad & 1) atomicOr(p.status, 1);                      // non-finite input sample
          if (bad & 2) atomicOr(p.status + 1 + TTS_MAX_CLUSTER, 1);   // row transform ran out of time
        }
        return;
      }
    }
    if (step == 0) {
      step_ingest<OWN, SC>(p, sm, cta);
      __syncthreads();
      continue;
    }
    if (step == 1) {
      // Ahat_S of A[t-1] and its Gram (partials by rows, or final in the single-chunk form);
      // P of B[t-1] over this CTA's rows
      if (merged) reduce_A_full(p, sm, cta, 0, sm.chunk + p.MC * R, nullptr, true);
      else reduce_A_rows(p, sm, cta, 0, true);
      __syncthreads();
      partials_B<OWN>(p, sm, cta, false, true, p.ridge_ff_all || p.K == 1);
      __syncthreads();
      continue;
    }
    if (step == 2) {
      reduce_sums(p, sm, cta, !merged);
      __syncthreads();
      continue;
    }
    const int k = (step - 3) / 4, sub = (step - 3) % 4;
    if (sub == 0) step_solve_A<OWN, LOADS_FIRST, SC>(p, sm, cta, k, fused);
    else if (sub == 1) reduce_A_rows(p, sm, cta, (k + 1) & 1, k + 1 < p.K);
    else if (sub == 2) step_B<OWN, SC>(p, sm, cta, k, k == p.K - 1, fused);
    else reduce_sums(p, sm, cta, !merged);
    __syncthreads();
  }
}

template <int OWN, bool SC>
__global__ void __launch_bounds__(TTS_THREADS, 1) frame_kernel(FrameParams p, int step_begin, int step_end,
                                                               int fused) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_release();
  pdl_wait();
  frame_run<OWN, true, SC>(p, smem_raw, blockIdx.x, step_begin, step_end, fused);
}

// Frames of many independent trackers (streams of any Nx, Ny, R) in one persistent
// launch: each cluster takes the next frame from a queue of parameter blocks, runs all
// its steps, and takes another until the queue is empty. queue_n = {counter (zero at
// launch), number of frames, offset of the first block in ps}: read from device memory,
// so a captured launch serves any batch up to its parameter capacity.
template <int OWN>
__global__ void __launch_bounds__(TTS_THREADS, 1) frame_batch_kernel(const FrameParams* __restrict__ ps,
                                                                     int* queue_n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FrameParams sp;
  __shared__ int item;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int n = ((volatile int*)queue_n)[1];
  ps += ((volatile int*)queue_n)[2];
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) item = atomicAdd(queue_n, 1);
    cluster.sync();
    const int it = *cluster.map_shared_rank(&item, 0);
    cluster.sync();   // every CTA has read the item before rank 0 may overwrite it or exit
    if (it >= n) break;
    const int* src = (const int*)(ps + it);
    int* dst = (int*)&sp;
    for (int e = threadIdx.x; e < (int)(sizeof(FrameParams) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
    __syncthreads();
    frame_run<OWN, false, false>(sp, smem_raw, rank, 0, frame_num_steps(sp.K), 1);
    __syncthreads();
  }
}

// The ridge solve alone on a given Hermitian positive-definite system (test hook): G and
// h in FP64, split into float hi + lo parts; the same Gauss-Jordan + float-float
// refinement as the frame kernel.
__global__ void __launch_bounds__(TTS_THREADS, 1) ridge_kernel(const double2* G, const double2* h, int R, int iters,
                                                               double2* gamma) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM sm;
  float2* base = (float2*)smem_raw;
  const int RR = R * R;
  sm.Gf = base;
  float2* Glo = base + RR;
  sm.GJa = base + 2 * RR;
  sm.Pk = sm.GJa + 64 * 72;
  sm.gam = sm.Pk + 136;
  sm.glo = sm.gam + R;
  sm.h = sm.gam + 2 * R;
  sm.rr = sm.gam + 3 * R;
  float2* hlo = sm.gam + 4 * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const double2 g = G[e];
    const float hx = (float)g.x, hy = (float)g.y;
    sm.Gf[e] = make_float2(hx, hy);
    Glo[e] = make_float2((float)(g.x - (double)hx), (float)(g.y - (double)hy));
  }
  for (int e = threadIdx.x; e < R; e += blockDim.x) {
    const double2 v = h[e];
    const float hx = (float)v.x, hy = (float)v.y;
    sm.h[e] = make_float2(hx, hy);
    hlo[e] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
  __syncthreads();
  ridge_solve(sm, R, Glo, hlo, iters, 1e-28f);
  for (int e = threadIdx.x; e < R; e += blockDim.x)
    gamma[e] = make_double2((double)sm.gam[e].x + (double)sm.glo[e].x, (double)sm.gam[e].y + (double)sm.glo[e].y);
}

}  // namespace

int launch_ridge(const double2* G, const double2* h, int R, double2* gamma, cudaStream_t st) {
  const int smem = (int)(sizeof(float2) * (2 * R * R + 64 * 72 + 136 + 5 * R));
  if (cudaFuncSetAttribute(ridge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return TTS_ECUDA;
  ridge_kernel<<<1, TTS_THREADS, smem, st>>>(G, h, R, 12, gamma);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

// Choose the cluster size and chunk length so that the shared-memory layout fits.
int frame_configure(FrameParams& p, int requested_C, int smem_limit) {
  int maxsm = smem_limit;
  if (maxsm <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || maxsm <= 0)
      maxsm = 227 * 1024;
    // the persistent multi-stream kernel keeps its frame parameters in static shared
    // memory: leave room for them so that one layout serves both kernels
    maxsm -= 1024;
  }
  const int preferred = std::max(1, std::min(8, std::min(p.Nx, p.Ny) / 8));
  const int cands[] = {1, 2, 4, 8, 16};
  for (int ci = 0; ci < 5; ++ci) {
    const int C = requested_C > 0 ? requested_C : cands[ci];
    if (requested_C == 0 && C < preferred) continue;
    for (int MC : {32, 16, 8}) {
      const int rA = (p.Nx + C - 1) / C, rB = (p.Ny + C - 1) / C;
      if (rA * p.R > TTS_MAX_OWN * TTS_THREADS || rB * p.R > TTS_MAX_OWN * TTS_THREADS) continue;
      if (((p.R + 15) & ~15) * ((p.R + 15) & ~15) > TTS_MAX_OWN * TTS_THREADS) continue;
      const FrameLayout L = frame_layout(p.Nx, p.Ny, p.R, rA, rB, MC);
      if (L.bytes <= maxsm) {
        p.C = C;
        p.rA = rA;
        p.rB = rB;
        p.MC = MC;
        p.lay = L;
        return TTS_OK;
      }
    }
    if (requested_C > 0) break;
  }
  return TTS_EINVAL;
}

template <int OWN, bool SC>
static int launch_frame_t(const FrameParams& p, int launch_mode, cudaStream_t st) {
  static PerDevice attrs;
  int done = 0;
  if (per_device(attrs,
                 [](int, int* v) {
                   if (cudaFuncSetAttribute(frame_kernel<OWN, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            227 * 1024) != cudaSuccess ||
                       cudaFuncSetAttribute(frame_kernel<OWN, SC>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                            1) != cudaSuccess)
                     return TTS_ECUDA;
                   *v = 1;
                   return TTS_OK;
                 },
                 &done) != TTS_OK)
    return TTS_ECUDA;
  cudaError_t e;
  const int smem = p.lay.bytes;
  const int nsteps = frame_num_steps(p.K);
  if (launch_mode == TTS_LAUNCH_FUSED) {
    e = launch_pdl(frame_kernel<OWN, SC>, dim3(p.C), dim3(TTS_THREADS), (size_t)smem, st, p.C, p, 0, nsteps, 1);
    if (e != cudaSuccess) return TTS_ECUDA;
  } else {
    for (int s = 0; s < nsteps; ++s) {
      frame_kernel<OWN, SC><<<p.C, TTS_THREADS, smem, st>>>(p, s, s + 1, 0);
      if (cudaGetLastError() != cudaSuccess) return TTS_ECUDA;
    }
  }
  return TTS_OK;
}

// outputs each thread owns: R x R entries of the Gram and Gauss-Jordan updates, and the
// (row, r) entries of this CTA's rows of A and B
int frame_own(const FrameParams& p) {
  const int Rp = (p.R + 15) & ~15;
  const int n = std::max(Rp * Rp, std::max(p.rA, p.rB) * p.R);
  const int own = (n + TTS_THREADS - 1) / TTS_THREADS;
  return own <= 1 ? 1 : own <= 2 ? 2 : own <= 4 ? 4 : 8;
}

int launch_frame(const FrameParams& p, int launch_mode, cudaStream_t st) {
  // R dividing the block and R <= 32: every output a thread owns in the factor-sized loops
  // has the same column, so the kernel is compiled with only the shared-column form of them
  // (the others keep both forms and choose at run time)
  const bool sc = TTS_THREADS % p.R == 0 && p.R <= 32;
  switch (frame_own(p)) {
    case 1: return sc ? launch_frame_t<1, true>(p, launch_mode, st) : launch_frame_t<1, false>(p, launch_mode, st);
    case 2: return sc ? launch_frame_t<2, true>(p, launch_mode, st) : launch_frame_t<2, false>(p, launch_mode, st);
    case 4: return sc ? launch_frame_t<4, true>(p, launch_mode, st) : launch_frame_t<4, false>(p, launch_mode, st);
    default: return launch_frame_t<8, false>(p, launch_mode, st);
  }
}

template <int OWN>
static int frame_batch_limits_t(int C, int* max_dyn_smem, int* max_clusters) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, frame_batch_kernel<OWN>) != cudaSuccess) return TTS_ECUDA;
  int optin = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return TTS_ECUDA;
  const int dyn = optin - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(frame_batch_kernel<OWN>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess ||
      cudaFuncSetAttribute(frame_batch_kernel<OWN>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return TTS_ECUDA;
  *max_dyn_smem = dyn;
  if (max_clusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(TTS_THREADS, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, frame_batch_kernel<OWN>, &cfg) != cudaSuccess || nc < 1) return TTS_ECUDA;
    *max_clusters = nc;
  }
  return TTS_OK;
}

int frame_batch_limits(int own, int C, int* max_dyn_smem, int* max_clusters) {
  switch (own) {
    case 1: return frame_batch_limits_t<1>(C, max_dyn_smem, max_clusters);
    case 2: return frame_batch_limits_t<2>(C, max_dyn_smem, max_clusters);
    case 4: return frame_batch_limits_t<4>(C, max_dyn_smem, max_clusters);
    default: return frame_batch_limits_t<8>(C, max_dyn_smem, max_clusters);
  }
}

template <int OWN>
static int launch_frame_batch_t(int C, int clusters, int smem, const FrameParams* ps, int* queue_n, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * C, 1, 1);
  cfg.blockDim = dim3(TTS_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, frame_batch_kernel<OWN>, ps, queue_n) == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

int launch_frame_batch(int own, int C, int clusters, int smem, const FrameParams* ps, int* queue_n, cudaStream_t st) {
  if (clusters <= 0) return TTS_OK;
  switch (own) {
    case 1: return launch_frame_batch_t<1>(C, clusters, smem, ps, queue_n, st);
    case 2: return launch_frame_batch_t<2>(C, clusters, smem, ps, queue_n, st);
    case 4: return launch_frame_batch_t<4>(C, clusters, smem, ps, queue_n, st);
    default: return launch_frame_batch_t<8>(C, clusters, smem, ps, queue_n, st);
  }
}
