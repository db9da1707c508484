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
  float2 *Gf;               // R x R
  float2 *GJa, *GJb;        // Rp x Rp (R padded to a multiple of 16)
  float2 *Pk, *Tk;          // 16 x 16 block inverse, 16 x Rp block row
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
  s.Tk = s.Pk + 256;
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

// ---------------------------------------------------------------------------------
// Ridge solve (S1): (G_hi + G_lo) gamma = h_hi + h_lo. FP32 Gauss-Jordan inverse of G_hi
// (pivots on the diagonal; G is Hermitian positive definite), then `iters` refinement
// sweeps gamma += Ginv (h - G gamma) with the residual in float-float arithmetic and
// gamma held as a float-float pair (gam + glo); the sweeps stop once every correction is
// below sqrt(tol2) relative. G_hi in sm.Gf, h_hi in sm.h.
// ---------------------------------------------------------------------------------
// Inverse of the 16 x 16 diagonal block at [kb, kb+16) of M (row stride ld), by one warp:
// Gauss-Jordan in registers, lane = column (lane & 15) of rows 8 (lane >> 4) + 0..7;
// rows and columns of the pivot are exchanged with shuffles. Result into P (16 x 16).
__device__ __forceinline__ void warp_inverse16(const float2* M, int ld, int kb, float2* P) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, c = lane & 15, h = lane >> 4;
  float2 m[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) m[e] = M[(kb + 8 * h + e) * ld + kb + c];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int qe = q & 7, qh = q >> 3;
    float2 d, rq, cq[8];
    d.x = __shfl_sync(FULL, m[qe].x, q + 16 * qh);
    d.y = __shfl_sync(FULL, m[qe].y, q + 16 * qh);
    rq.x = __shfl_sync(FULL, m[qe].x, c + 16 * qh);
    rq.y = __shfl_sync(FULL, m[qe].y, c + 16 * qh);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      cq[e].x = __shfl_sync(FULL, m[e].x, q + 16 * h);
      cq[e].y = __shfl_sync(FULL, m[e].y, q + 16 * h);
    }
    const float inv = __frcp_rn(cabs2(d));
    const float2 piv = make_float2(d.x * inv, -d.y * inv);
    const float2 rqp = cmul(rq, piv);
    // branch-free update (the row and column of the pivot are lane dependent)
    const bool colq = (c == q);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const bool rowq = (h == qh) && (e == qe);
      float2 gen = m[e];
      cfms(gen, cq[e], rqp);
      const float2 t = cmul(cq[e], piv);
      const float2 colv = make_float2(-t.x, -t.y);
      const float2 rv = colq ? piv : rqp;
      const float2 ov = colq ? colv : gen;
      m[e] = rowq ? rv : ov;
    }
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) P[(8 * h + e) * 16 + c] = m[e];
}

template <int OWN>
__device__ void ridge_solve(SM& sm, int R, const float2* Glo, const float2* hlo, int iters, float tol2) {
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const int Rp = (R + 15) & ~15;
  const int RP2 = Rp * Rp;
  int oi[OWN], oj[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    oi[o] = e / Rp;
    oj[o] = e - oi[o] * Rp;
  }
  // G padded with the identity to Rp x Rp
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    if (e < RP2) {
      const int i = oi[o], j = oj[o];
      sm.GJa[e] = (i < R && j < R) ? sm.Gf[i * R + j] : make_float2(i == j ? 1.f : 0.f, 0.f);
    }
  }
  __syncthreads();
  // blocked Gauss-Jordan inverse with 16 x 16 pivot blocks (Hermitian positive definite:
  // every pivot block is a Schur complement and invertible)
  float2* M = sm.GJa;
  float2* N = sm.GJb;
  for (int kb = 0; kb < Rp; kb += 16) {
    if (warp == 0) warp_inverse16(M, Rp, kb, sm.Pk);
    __syncthreads();
    // block row k of the update: T = P M[kb:kb+16, :]
    for (int e = tid; e < 16 * Rp; e += nth) {
      const int t = e / Rp, cc = e - t * Rp;
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        cfma(a0, sm.Pk[t * 16 + u], M[(kb + u) * Rp + cc]);
        cfma(a1, sm.Pk[t * 16 + u + 1], M[(kb + u + 1) * Rp + cc]);
      }
      sm.Tk[e] = cadd(a0, a1);
    }
    __syncthreads();
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const int e = tid + o * nth;
      if (e < RP2) {
        const int i = oi[o], cc = oj[o];
        const bool bi = (i >= kb) && (i < kb + 16), bc = (cc >= kb) && (cc < kb + 16);
        float2 v;
        if (bi) {
          v = bc ? sm.Pk[(i - kb) * 16 + (cc - kb)] : sm.Tk[(i - kb) * Rp + cc];
        } else {
          // column source: the block inverse for pivot-block columns, else T (no divergence)
          const float2* src = bc ? sm.Pk + (cc - kb) : sm.Tk + cc;
          const int ld = bc ? 16 : Rp;
          float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 16; u += 2) {
            cfma(a0, M[i * Rp + kb + u], src[u * ld]);
            cfma(a1, M[i * Rp + kb + u + 1], src[(u + 1) * ld]);
          }
          const float2 a = cadd(a0, a1);
          const float2 base = bc ? make_float2(0.f, 0.f) : M[e];
          v = csub(base, a);
        }
        N[e] = v;
      }
    }
    __syncthreads();
    float2* t = M;
    M = N;
    N = t;
  }
  const float2* Gi = M;   // inverse, row stride Rp
  // gamma_0 = Ginv h (one warp per row)
  for (int i = warp; i < R; i += nwarp) {
    float2 acc = make_float2(0.f, 0.f);
    for (int j = lane; j < R; j += 32) cfma(acc, Gi[i * Rp + j], sm.h[j]);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      sm.gam[i] = acc;
      sm.glo[i] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  // convergence: max_i |delta_i|^2 <= tol2 max_i |gamma_i|^2 (float bits of non-negative
  // floats order like unsigned integers)
  unsigned* dmax = (unsigned*)(sm.tmpv);
  unsigned* gmax = dmax + 1;
  for (int it = 0; it < iters; ++it) {
    if (tid == 0) {
      *dmax = 0u;
      *gmax = 0u;
    }
    // r = h - G gamma in float-float (warp per row)
    for (int i = warp; i < R; i += nwarp) {
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      for (int j = lane; j < R; j += 32) {
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
        const float cr = cc.x, ci = cc.y;
        ff_add_f(rh, rl, cr);
        ff_add_f(ih, il, ci);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, rh, o), b = __shfl_xor_sync(0xffffffffu, rl, o);
        const float c = __shfl_xor_sync(0xffffffffu, ih, o), d = __shfl_xor_sync(0xffffffffu, il, o);
        ff_add_ff(rh, rl, a, b);
        ff_add_ff(ih, il, c, d);
      }
      if (lane == 0) {
        float sh = sm.h[i].x, sl = hlo ? hlo[i].x : 0.f;
        ff_add_ff(sh, sl, -rh, -rl);
        float th = sm.h[i].y, tl = hlo ? hlo[i].y : 0.f;
        ff_add_ff(th, tl, -ih, -il);
        sm.rr[i] = make_float2(sh + sl, th + tl);
      }
    }
    __syncthreads();
    // gamma += Ginv r
    for (int i = warp; i < R; i += nwarp) {
      float2 acc = make_float2(0.f, 0.f);
      for (int j = lane; j < R; j += 32) cfma(acc, Gi[i * Rp + j], sm.rr[j]);
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) {
        float2 g = sm.gam[i], gl = sm.glo[i];
        atomicMax(dmax, __float_as_uint(cabs2(acc)));
        atomicMax(gmax, __float_as_uint(cabs2(g)));
        ff_add_ff(g.x, gl.x, acc.x, 0.f);
        ff_add_ff(g.y, gl.y, acc.y, 0.f);
        sm.gam[i] = g;
        sm.glo[i] = gl;
      }
    }
    __syncthreads();
    if (__uint_as_float(*dmax) <= tol2 * __uint_as_float(*gmax)) break;
    __syncthreads();
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

// (B^H B)[q][r] and P[m][r] = sum over this CTA's rows j of Yt[m][j] conj(B[j][r])
template <int OWN>
__device__ void partials_B(const FrameParams& p, SM& sm, int cta, bool do_mb, bool do_p) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nx = p.Nx, R = p.R, MC = p.MC, RR = R * R;
  const int s = sm.misc[0];
  const Slice bs = slice_of(p.Ny, p.C, cta);
  const int nb = bs.hi - bs.lo;
  if (do_mb) {
    float2* pmb = p.partMB + (size_t)cta * RR;
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
        pmb[e] = cadd(a0, a1);
      }
    }
  }
  if (!do_p) return;
  float2* pp = p.partP + (size_t)cta * Nx * R;
  float2* YB = s <= MC ? sm.yb : sm.chunk;
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    if (s > MC || !sm.yb_ready) load_yb(p, YB, m0, mc, bs.lo, nb);
    __syncthreads();
    if (s <= MC) sm.yb_ready = true;
    for (int e = tid; e < mc * R; e += nth) {
      const int mm = e / R, r = e - mm * R;
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
      int jl = 0;
      for (; jl + 1 < nb; jl += 2) {
        cfma(a0, YB[mm * nb + jl], cconj(sm.B[jl * R + r]));
        cfma(a1, YB[mm * nb + jl + 1], cconj(sm.B[(jl + 1) * R + r]));
      }
      if (jl < nb) cfma(a0, YB[mm * nb + jl], cconj(sm.B[jl * R + r]));
      pp[(m0 + mm) * R + r] = cadd(a0, a1);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// step 0: ingest the frame: inverse row transforms of this CTA's slice of S (Yt), the
// anchors A[t-1], B[t-1], and partial sums of Ahat_S, ||a||^2 and B^H B over this CTA's rows
// ---------------------------------------------------------------------------------
template <int OWN>
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
  for (int m0 = ms.lo; m0 < ms.hi && !p.yt_ready; m0 += fft_rows) {
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
  if (bad) atomicOr(&sm.misc[1], 1);
  // anchors A[t-1], B[t-1]
  for (int e = tid; e < p.rA * R; e += nth) sm.A0[e] = sm.A[e];
  for (int e = tid; e < p.rB * R; e += nth) sm.B0[e] = sm.B[e];
  const Slice as = slice_of(Nx, C, cta), bs = slice_of(Ny, C, cta);
  for (int e = as.lo * R + tid; e < as.hi * R; e += nth) p.A0[e] = p.A[e];
  for (int e = bs.lo * R + tid; e < bs.hi * R; e += nth) p.B0[e] = p.B[e];
  partials_A(p, sm, cta, sm.chunk, false);
  partials_B<OWN>(p, sm, cta, true, false);
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

template <int OWN>
__device__ void step_solve_A(const FrameParams& p, SM& sm, int cta, int k) {
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
  // Gram of the masked rank-one DFTs (all R x R entries) and the right-hand side;
  // two accumulators per output (even / odd m)
  float2 g0[OWN], g1[OWN], h0 = make_float2(0.f, 0.f), h1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int o = 0; o < OWN; ++o) g0[o] = g1[o] = make_float2(0.f, 0.f);
  float2* MBs = sm.GJb;   // B^H B staged for the Gram (GJb is free until the solve)
  for (int e = tid; e < RR; e += nth) MBs[e] = p.MB[e];
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    for (int e = tid; e < mc * R; e += nth) {
      AH[e] = AhS[m0 * R + e];
      PC[e] = p.P[m0 * R + e];
    }
    __syncthreads();
    int ir[OWN], ic[OWN];
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const bool v = tid + o * nth < RR;
      ir[o] = v ? orow[o] : 0;
      ic[o] = v ? ocol[o] : 0;
    }
    int mm = 0;
    for (; mm + 1 < mc; mm += 2) {
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        cfmac(g0[o], AH[mm * R + ir[o]], AH[mm * R + ic[o]]);
        cfmac(g1[o], AH[(mm + 1) * R + ir[o]], AH[(mm + 1) * R + ic[o]]);
      }
      if (tid < R) {
        cfmac(h0, AH[mm * R + tid], PC[mm * R + tid]);
        cfmac(h1, AH[(mm + 1) * R + tid], PC[(mm + 1) * R + tid]);
      }
    }
    if (mm < mc) {
#pragma unroll
      for (int o = 0; o < OWN; ++o) cfmac(g0[o], AH[mm * R + ir[o]], AH[mm * R + ic[o]]);
      if (tid < R) cfmac(h0, AH[mm * R + tid], PC[mm * R + tid]);
    }
    __syncthreads();
  }
  const float fmu = (float)p.mu;
#pragma unroll
  for (int o = 0; o < OWN; ++o) {
    const int e = tid + o * nth;
    if (e < RR) {
      float2 v = cmul(cadd(g0[o], g1[o]), MBs[e]);
      if (orow[o] == ocol[o]) v = make_float2(v.x + fmu, 0.f);
      sm.Gf[e] = v;
    }
  }
  if (tid < R) sm.h[tid] = cadd(h0, h1);
  __syncthreads();
  ridge_solve<OWN>(sm, R, nullptr, nullptr, p.refine, 1e-20f);
  // B^H B again in shared memory (the solve overwrote GJb)
  float2* MBt = sm.GJb;
  for (int e = tid; e < RR; e += nth) MBt[e] = p.MB[e];
  __syncthreads();
  // alpha_A = sum |gamma_r|^2 ||b_r||^2 + rho (||b_r||^2 = (B^H B)[r][r])
  step_coefficients(p, sm, (const float*)MBt, 2 * (R + 1), p.sf[SF_RHO], p.sf[SF_ABAR_A]);
  if (cta == 0)
    for (int r = tid; r < R; r += nth) {
      p.gamma[r] = sm.gam[r];
      p.gamma_d[r] = make_double2((double)sm.gam[r].x + (double)sm.glo[r].x,
                                  (double)sm.gam[r].y + (double)sm.glo[r].y);
    }
  // gM[q][r] = gamma_q (B^H B)[r][q]
  float2* gM = sm.GJa;
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
  const bool one_chunk = s <= MC;   // AH and PC still hold the whole of Ahat_S and P
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
    if (!one_chunk)
      for (int e = tid; e < mc * R; e += nth) {
        AH[e] = AhS[m0 * R + e];
        PC[e] = p.P[m0 * R + e];
      }
    fill_twiddles(p, sm, TW, m0, mc, as.lo, na);
    __syncthreads();
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
    __syncthreads();
    int ir[OWN], ic[OWN];
#pragma unroll
    for (int o = 0; o < OWN; ++o) {
      const bool v = tid + o * nth < NO;
      ir[o] = v ? orow[o] : 0;
      ic[o] = v ? ocol[o] : 0;
    }
    int mm = 0;
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
  partials_A(p, sm, cta, TW, one_chunk);
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

// reduce the per-CTA partials of Ahat'_S and ||a'||^2 (this CTA's slice of the entries)
__device__ void step_reduce_A(const FrameParams& p, SM& sm, int cta, int k) {
  const int R = p.R, C = p.C, Nx = p.Nx;
  const int s = sm.misc[0];
  const int E = s * R + R;
  const Slice es = slice_of(E, C, cta);
  float2* out = p.AhS[(k + 1) & 1];
  float* nout = p.nA[(k + 1) & 1];
  for (int e = es.lo + threadIdx.x; e < es.hi; e += blockDim.x) {
    if (e < s * R) {
      out[e] = sum_partials(p.partA + e, (size_t)Nx * R, C);
    } else {
      const int r = e - s * R;
      float acc = 0.f;
      for (int c = 0; c < C; c += 4) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = c + u < C ? p.partNA[(c + u) * R + r] : 0.f;
        acc += (v[0] + v[1]) + (v[2] + v[3]);
      }
      nout[r] = acc;
    }
  }
}

// ---------------------------------------------------------------------------------
// step B: majorized B step (S2) on this CTA's rows, then partials of B^H B and P
// ---------------------------------------------------------------------------------
template <int OWN>
__device__ void step_B(const FrameParams& p, SM& sm, int cta, int k, bool last) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Nx = p.Nx, Ny = p.Ny, R = p.R, C = p.C, MC = p.MC;
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
  for (int r = tid; r < R; r += nth) {
    sm.gam[r] = p.gamma[r];
    nAs[r] = nA[r];
  }
  // MA = Ahat^H Ahat (thread-owned entries) and U[j][r] = sum_m Yt[m][j] conj(Ahat[m][r])
  float2 ma[OWN], u[OWN];
#pragma unroll
  for (int o = 0; o < OWN; ++o) ma[o] = u[o] = make_float2(0.f, 0.f);
  const int NO = nb * R;
  for (int m0 = 0; m0 < s; m0 += MC) {
    const int mc = min(MC, s - m0);
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
    for (int mm = 0; mm < mc; ++mm) {
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        cfmac(ma[o], AH[mm * R + mr[o]], AH[mm * R + mq[o]]);
        cfmac(u[o], AH[mm * R + ur[o]], YB[mm * nb + uj[o]]);
      }
    }
    __syncthreads();
  }
  // gMA[q][r] = gamma_q MA[r][q]
  float2* gMA = sm.GJa;
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
      const float2 tb = cadd(tb0, tb1);
      const float2 b = sm.B[e], b0 = sm.B0[e];
      const float2 grad = csub(cscale(b, frho), cmul(tb, cconj(sm.gam[r])));
      nbv[o].x = fmaf(-c2, grad.x, fmaf(c1, b.x, c0 * b0.x));
      nbv[o].y = fmaf(-c2, grad.y, fmaf(c1, b.y, c0 * b0.y));
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
  // partials over this CTA's rows: B'^H B' and Yt conj(B')
  partials_B<OWN>(p, sm, cta, true, true);
}

// reduce every partial of the ingest: Ahat_S, ||a||^2, B^H B, P
__device__ void step_reduce_all(const FrameParams& p, SM& sm, int cta) {
  const int R = p.R, C = p.C, Nx = p.Nx;
  const int s = sm.misc[0];
  const int E1 = s * R, E2 = E1 + R, E3 = E2 + R * R, E = E3 + s * R;
  const Slice es = slice_of(E, C, cta);
  for (int e = es.lo + threadIdx.x; e < es.hi; e += blockDim.x) {
    if (e < E1) {
      p.AhS[0][e] = sum_partials(p.partA + e, (size_t)Nx * R, C);
    } else if (e < E2) {
      const int r = e - E1;
      float acc = 0.f;
      for (int c = 0; c < C; ++c) acc += p.partNA[c * R + r];
      p.nA[0][r] = acc;
    } else if (e < E3) {
      p.MB[e - E2] = sum_partials(p.partMB + (e - E2), (size_t)R * R, C);
    } else {
      p.P[e - E3] = sum_partials(p.partP + (e - E3), (size_t)Nx * R, C);
    }
  }
}

// reduce the per-CTA partials of B^H B and P
__device__ void step_reduce_B(const FrameParams& p, SM& sm, int cta) {
  const int R = p.R, C = p.C, Nx = p.Nx;
  const int s = sm.misc[0];
  const int E = R * R + s * R;
  const Slice es = slice_of(E, C, cta);
  for (int e = es.lo + threadIdx.x; e < es.hi; e += blockDim.x) {
    const bool mb = e < R * R;
    const float2* src = mb ? p.partMB + e : p.partP + (e - R * R);
    const size_t stride = mb ? (size_t)R * R : (size_t)Nx * R;
    const float2 acc = sum_partials(src, stride, C);
    if (mb) p.MB[e] = acc;
    else p.P[e - R * R] = acc;
  }
}

// Steps [step_begin, step_end) of one frame, run by CTA `cta` of the cluster that owns it.
template <int OWN>
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
  for (int step = step_begin; step < step_end; ++step) {
    if (step > step_begin) {
      __threadfence();
      if (fused) cluster.sync();
      else __syncthreads();
    }
    if (step > 0) {
      // the frame is rejected when any CTA saw a non-finite input sample
      int bad = 0;
      for (int c = 0; c < p.C; ++c) bad |= ((volatile int*)p.status)[1 + c];
      if (bad) {
        if (step == 1 && cta == 0 && tid == 0) atomicOr(p.status, 1);
        return;
      }
    }
    if (step == 0) {
      step_ingest<OWN>(p, sm, cta);
      __syncthreads();
      continue;
    }
    if (step == 1) {
      partials_B<OWN>(p, sm, cta, false, true);
      __syncthreads();
      continue;
    }
    if (step == 2) {
      step_reduce_all(p, sm, cta);
      __syncthreads();
      continue;
    }
    const int k = (step - 3) / 4, sub = (step - 3) % 4;
    if (sub == 0) step_solve_A<OWN>(p, sm, cta, k);
    else if (sub == 1) step_reduce_A(p, sm, cta, k);
    else if (sub == 2) step_B<OWN>(p, sm, cta, k, k == p.K - 1);
    else step_reduce_B(p, sm, cta);
    __syncthreads();
  }
}

template <int OWN>
__global__ void __launch_bounds__(TTS_THREADS, 1) frame_kernel(FrameParams p, int step_begin, int step_end,
                                                               int fused) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  frame_run<OWN>(p, smem_raw, blockIdx.x, step_begin, step_end, fused);
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
    frame_run<OWN>(sp, smem_raw, rank, 0, frame_num_steps(sp.K), 1);
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
  const int Rp = (R + 15) & ~15;
  sm.Gf = base;
  float2* Glo = base + RR;
  sm.GJa = base + 2 * RR;
  sm.GJb = sm.GJa + Rp * Rp;
  sm.Pk = sm.GJb + Rp * Rp;
  sm.Tk = sm.Pk + 256;
  sm.gam = sm.Tk + 16 * Rp;
  sm.glo = sm.gam + R;
  sm.h = sm.gam + 2 * R;
  sm.rr = sm.gam + 3 * R;
  float2* hlo = sm.gam + 4 * R;
  sm.tmpv = sm.gam + 5 * R;   // refinement convergence flag
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
  ridge_solve<TTS_MAX_OWN>(sm, R, Glo, hlo, iters, 1e-28f);
  for (int e = threadIdx.x; e < R; e += blockDim.x)
    gamma[e] = make_double2((double)sm.gam[e].x + (double)sm.glo[e].x, (double)sm.gam[e].y + (double)sm.glo[e].y);
}

}  // namespace

int launch_ridge(const double2* G, const double2* h, int R, double2* gamma, cudaStream_t st) {
  const int Rp = (R + 15) & ~15;
  const int smem = (int)(sizeof(float2) * (2 * R * R + 2 * Rp * Rp + 256 + 16 * Rp + 6 * R));
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

template <int OWN>
static int launch_frame_t(const FrameParams& p, int launch_mode, cudaStream_t st) {
  static PerDevice attrs;
  int done = 0;
  if (per_device(attrs,
                 [](int, int* v) {
                   if (cudaFuncSetAttribute(frame_kernel<OWN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            227 * 1024) != cudaSuccess ||
                       cudaFuncSetAttribute(frame_kernel<OWN>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                           cudaSuccess)
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
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.C, 1, 1);
    cfg.blockDim = dim3(TTS_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, frame_kernel<OWN>, p, 0, nsteps, 1);
    if (e != cudaSuccess) return TTS_ECUDA;
  } else {
    for (int s = 0; s < nsteps; ++s) {
      frame_kernel<OWN><<<p.C, TTS_THREADS, smem, st>>>(p, s, s + 1, 0);
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
  switch (frame_own(p)) {
    case 1: return launch_frame_t<1>(p, launch_mode, st);
    case 2: return launch_frame_t<2>(p, launch_mode, st);
    case 4: return launch_frame_t<4>(p, launch_mode, st);
    default: return launch_frame_t<8>(p, launch_mode, st);
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
