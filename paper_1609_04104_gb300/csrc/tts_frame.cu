// Per-frame MM iterations of the online tensor-subspace tracker (Alg. 3 with one coil,
// S1 ridge step for gamma_t and S2 majorized factor steps, §III-A), GB300 design.
//
// Everything a frame needs is computed from small factor-sized quantities, using the
// separability of the 2D DFT with Cartesian line masks (Omega = S x [Ny]):
//   F(a b^T) = (F_Nx a)(F_Ny b)^T, F unitary and symmetric, so with
//   Ahat_S = (F_Nx A)[S,:] (|S| x R) and Yt = y_S conj(F_Ny) (|S| x Ny, once per frame):
//     Phi^H Phi = (Ahat_S^H Ahat_S) .* (B^H B)            (Gram of the masked rank-one DFTs)
//     Phi^H y   = colsum(conj(Ahat_S) .* P),  P = Yt conj(B)
//     Theta conj(B)   = conj(F_Nx)[:,S] (P - Ahat_S diag(gamma) (B^H B)^T)
//     Theta'^T conj(A) = Yt^T conj(Ahat'_S) - B diag(gamma) (Ahat'_S^H Ahat'_S)^T
// with Theta = F^{-1}(P_Omega(y - F(A diag(gamma) B^T))) the back-projected residual of
// Alg. 3 (S2). These are the same quantities as the masked 2D DFTs of the rank-one
// images and the inverse 2D DFT of the residual, computed in a different order.
//
// The frame runs as one kernel on a thread-block cluster of C CTAs. CTA c owns a slice of
// the rows of A and of B; reductions over rows go through per-CTA partial sums that one
// phase writes and the next phase reduces, each CTA reducing a slice of the entries.
// Phases are separated by cluster barriers (or run as separate launches).
#include <cooperative_groups.h>

#include "tts_internal.cuh"

namespace cg = cooperative_groups;

namespace {

struct Slice {
  int lo, hi;
};
__device__ __forceinline__ Slice slice_of(int n, int parts, int idx) {
  int per = (n + parts - 1) / parts;
  int lo = min(n, idx * per);
  int hi = min(n, lo + per);
  return {lo, hi};
}

struct Smem {
  float2* Wx;     // Nx
  float2* Wy;     // Ny
  int* rows;      // Nx
  int* misc;      // [0] = |S|, [1] = non-finite flag
  double2* G;     // R x R (lower triangle)
  double* invd;   // R
  double2* z;     // R
  double2* h;     // R
  float* fs;      // 8 float scalars of the current step
  double* ds;     // 8 double scalars of the current step
  float2* gam;    // R
  float2* gM;     // R x R  (gM[q*R + r] = gamma_q * M[r][q])
  float* red;     // TTS_THREADS scratch
  float2* fbuf;   // 2 x fft_rows x Ny
  int fft_rows;
};

__device__ Smem carve(const FrameParams& p, unsigned char* base, int fft_rows) {
  Smem s;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 15) & ~size_t(15);
    void* q = base + off;
    off += bytes;
    return q;
  };
  s.G = (double2*)take(sizeof(double2) * p.R * p.R);
  s.z = (double2*)take(sizeof(double2) * p.R);
  s.invd = (double*)take(sizeof(double) * p.R);
  s.h = (double2*)take(sizeof(double2) * p.R);
  s.fs = (float*)take(sizeof(float) * 8);
  s.ds = (double*)take(sizeof(double) * 8);
  s.Wx = (float2*)take(sizeof(float2) * p.Nx);
  s.Wy = (float2*)take(sizeof(float2) * p.Ny);
  s.gam = (float2*)take(sizeof(float2) * p.R);
  s.gM = (float2*)take(sizeof(float2) * p.R * p.R);
  s.rows = (int*)take(sizeof(int) * p.Nx);
  s.misc = (int*)take(sizeof(int) * 4);
  s.red = (float*)take(sizeof(float) * TTS_THREADS);
  s.fbuf = (float2*)take(sizeof(float2) * 2 * fft_rows * p.Ny);
  s.fft_rows = fft_rows;
  return s;
}

// ----------------------------------------------------------------------------------
// step 0: ingest the frame and form the reduced quantities of the first iteration
// ----------------------------------------------------------------------------------
__device__ void step_ingest(const FrameParams& p, Smem& sm, int cta) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int Nx = p.Nx, Ny = p.Ny, R = p.R, C = p.C;
  const int s = sm.misc[0];
  // acquired rows times conj(F_Ny): inverse row transforms of this CTA's rows of S,
  // then P[m, :] = Yt[m, :] conj(B) for those rows
  Slice ms = slice_of(s, C, cta);
  for (int m0 = ms.lo; m0 < ms.hi; m0 += sm.fft_rows) {
    const int nr = min(sm.fft_rows, ms.hi - m0);
    float2* buf = sm.fbuf;
    float2* tmp = sm.fbuf + sm.fft_rows * Ny;
    int bad = 0;
    for (int e = tid; e < nr * Ny; e += blockDim.x) {
      const int mr = e / Ny;
      const size_t src = p.full_frame ? (size_t)sm.rows[m0 + mr] * Ny + (e - mr * Ny) : (size_t)m0 * Ny + e;
      float2 v = p.yrows[src];
      if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
      buf[e] = v;
    }
    if (bad) atomicOr(&sm.misc[1], 1);
    __syncthreads();
    float2* res = fft_smem(buf, tmp, p.plan_y, nr, sm.Wy, +1, tid, blockDim.x);
    for (int e = tid; e < nr * Ny; e += blockDim.x) {
      res[e] = cscale(res[e], p.isy);
      p.Yt[(size_t)m0 * Ny + e] = res[e];
    }
    __syncthreads();
    for (int mr = warp; mr < nr; mr += nwarp) {
      const float2* yt = res + mr * Ny;
      for (int r = lane; r < R; r += 32) {
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0; j < Ny; ++j) cfma(acc, yt[j], cconj(p.B[j * R + r]));
        p.P[(size_t)(m0 + mr) * R + r] = acc;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0) p.status[1 + cta] = sm.misc[1];
  // anchors A[t-1], B[t-1] for this CTA's rows
  Slice as = slice_of(Nx, C, cta), bs = slice_of(Ny, C, cta);
  for (int e = as.lo * R + tid; e < as.hi * R; e += blockDim.x) p.A0[e] = p.A[e];
  for (int e = bs.lo * R + tid; e < bs.hi * R; e += blockDim.x) p.B0[e] = p.B[e];
  // Ahat_S = (F_Nx A)[S,:] for this CTA's rows of S
  float2* AhS = p.AhS[0];
  for (int m = ms.lo + warp; m < ms.hi; m += nwarp) {
    const int i = sm.rows[m];
    for (int r = lane; r < R; r += 32) {
      float2 acc = make_float2(0.f, 0.f);
      int idx = 0;
      for (int n = 0; n < Nx; ++n) {
        cfma(acc, sm.Wx[idx], p.A[n * R + r]);
        idx += i;
        if (idx >= Nx) idx -= Nx;
      }
      AhS[m * R + r] = cscale(acc, p.isx);
    }
  }
  // B^H B, rows q of this CTA's slice of [0, R)
  Slice qs = slice_of(R, C, cta);
  for (int q = qs.lo + warp; q < qs.hi; q += nwarp) {
    for (int r = lane; r < R; r += 32) {
      float2 acc = make_float2(0.f, 0.f);
      for (int j = 0; j < Ny; ++j) cfmac(acc, p.B[j * R + q], p.B[j * R + r]);
      p.MB[q * R + r] = acc;
    }
  }
  // ||a_r||^2 (last CTA)
  if (cta == C - 1) {
    for (int r0 = 0; r0 < R; r0 += 32) {
      const int r = r0 + lane;
      float acc = 0.f;
      if (r < R)
        for (int n = warp; n < Nx; n += nwarp) acc += cabs2(p.A[n * R + r]);
      sm.red[warp * 32 + lane] = acc;
      __syncthreads();
      if (warp == 0 && r < R) {
        float t = 0.f;
        for (int w = 0; w < nwarp; ++w) t += sm.red[w * 32 + lane];
        p.nA[0][r] = t;
      }
      __syncthreads();
    }
  }
  if (cta == 0 && tid == 0) {
    const double w = p.lf * p.sc[SC_W] + 1.0;
    p.sf[SF_W] = w;
    p.sf[SF_RHO] = p.mu / w;
    p.sf[SF_ABAR_A] = p.sc[SC_ABAR_A];
    p.sf[SF_ABAR_B] = p.sc[SC_ABAR_B];
    *p.nrows = s;
    for (int m = 0; m < s; ++m) p.rows[m] = sm.rows[m];
  }
}

// ----------------------------------------------------------------------------------
// LDL^H factorisation and solve of the R x R ridge system in FP64 (lower triangle of
// sm.G holds G on entry). On exit sm.z holds gamma.
// ----------------------------------------------------------------------------------
__device__ void ldl_solve(const FrameParams& p, Smem& sm, const double2* h) {
  const int R = p.R, tid = threadIdx.x;
  const int ntri = R * (R + 1) / 2;
  if (tid == 0) sm.invd[0] = 1.0 / sm.G[0].x;
  __syncthreads();
  for (int k = 0; k < R - 1; ++k) {
    // update G[i][j] -= G[i][k] conj(G[j][k]) / d_k for k < j <= i
    for (int e = tid; e < ntri; e += blockDim.x) {
      // e -> (i, j) with j <= i: i = floor((sqrt(8e+1)-1)/2)
      int i = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      const int j = e - i * (i + 1) / 2;
      if (j <= k) continue;
      const double2 lik = sm.G[i * R + k], ljk = sm.G[j * R + k];
      const double inv = sm.invd[k];
      double2 upd = zmul(lik, make_double2(ljk.x, -ljk.y));
      double2 g = sm.G[i * R + j];
      g.x -= upd.x * inv;
      g.y -= upd.y * inv;
      if (i == j) g.y = 0.0;
      sm.G[i * R + j] = g;
      if (i == k + 1 && j == k + 1) sm.invd[k + 1] = 1.0 / g.x;
    }
    __syncthreads();
  }
  // solve L D L^H gamma = h with L[i][k] = G[i][k] / d_k (one warp)
  if (tid < 32) {
    const int lane = tid;
    for (int i = lane; i < R; i += 32) sm.z[i] = h[i];
    __syncwarp();
    for (int k = 0; k < R; ++k) {
      const double2 zk = sm.z[k];
      for (int i = k + 1 + lane; i < R; i += 32) {
        double2 l = sm.G[i * R + k];
        double2 t = zmul(l, zk);
        sm.z[i].x -= t.x * sm.invd[k];
        sm.z[i].y -= t.y * sm.invd[k];
      }
      __syncwarp();
    }
    for (int i = lane; i < R; i += 32) {
      sm.z[i].x *= sm.invd[i];
      sm.z[i].y *= sm.invd[i];
    }
    __syncwarp();
    for (int k = R - 1; k >= 0; --k) {
      const double2 gk = sm.z[k];
      for (int i = lane; i < k; i += 32) {
        double2 l = sm.G[k * R + i];  // L[k][i] d_i
        double2 t = zmulc(l, gk);     // conj(L[k][i] d_i) gamma_k
        sm.z[i].x -= t.x * sm.invd[i];
        sm.z[i].y -= t.y * sm.invd[i];
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------------
// step "A": ridge solve for gamma (S1), then the majorized A step (S2) on this CTA's
// rows, then partial sums of Ahat'_S and ||a'_r||^2 over those rows
// ----------------------------------------------------------------------------------
__device__ void step_solve_A(const FrameParams& p, Smem& sm, int cta, int k) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int Nx = p.Nx, R = p.R, C = p.C;
  const int s = sm.misc[0];
  const float2* AhS = p.AhS[k & 1];
  // Gram of the masked rank-one DFTs and the right-hand side
  const int ntri = R * (R + 1) / 2;
  for (int e = tid; e < ntri; e += blockDim.x) {
    int i = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    const int j = e - i * (i + 1) / 2;
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 0; m < s; ++m) cfmac(acc, AhS[m * R + i], AhS[m * R + j]);
    const float2 g = cmul(acc, p.MB[i * R + j]);
    double2 gd = make_double2((double)g.x, (double)g.y);
    if (i == j) {
      gd.x += p.mu;
      gd.y = 0.0;
    }
    sm.G[i * R + j] = gd;
  }
  double2* h = sm.h;
  for (int r = tid; r < R; r += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 0; m < s; ++m) cfmac(acc, AhS[m * R + r], p.P[m * R + r]);
    h[r] = make_double2((double)acc.x, (double)acc.y);
  }
  __syncthreads();
  ldl_solve(p, sm, h);
  // gamma, alpha_A = sum |gamma_r|^2 ||b_r||^2 + rho and the step coefficients (one
  // thread: FP64 is scarce on this part)
  if (tid == 0) {
    const double rho = p.sf[SF_RHO], abar = p.sf[SF_ABAR_A];
    double alpha = rho;
    for (int r = 0; r < R; ++r) alpha += (sm.z[r].x * sm.z[r].x + sm.z[r].y * sm.z[r].y) * (double)p.MB[r * R + r].x;
    const double den = p.lf * abar + alpha;
    sm.ds[0] = alpha;
    sm.fs[0] = (float)(p.lf * abar / den);
    sm.fs[1] = (float)(alpha / den);
    sm.fs[2] = (float)(1.0 / den);
    sm.fs[3] = (float)rho;
    if (cta == 0) p.sf[SF_ALPHA_A] = alpha;
  }
  for (int r = tid; r < R; r += blockDim.x) {
    sm.gam[r] = make_float2((float)sm.z[r].x, (float)sm.z[r].y);
    if (cta == 0) {
      p.gamma_d[r] = sm.z[r];
      p.gamma[r] = sm.gam[r];
    }
  }
  __syncthreads();
  // gM[q][r] = gamma_q (B^H B)[r][q]
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int q = e / R, r = e - q * R;
    sm.gM[e] = cmul(sm.gam[q], p.MB[r * R + q]);
  }
  __syncthreads();
  // Q = P - Ahat_S diag(gamma) (B^H B)^T  (this CTA's copy)
  float2* Q = p.Q + (size_t)cta * Nx * R;
  for (int m = warp; m < s; m += nwarp) {
    for (int r = lane; r < R; r += 32) {
      float2 acc = p.P[m * R + r];
      for (int q = 0; q < R; ++q) {
        const float2 t = cmul(AhS[m * R + q], sm.gM[q * R + r]);
        acc = csub(acc, t);
      }
      Q[m * R + r] = acc;
    }
  }
  __syncthreads();
  // A step on this CTA's rows: grad = rho A - (conj(F)[:,S] Q) diag(conj gamma)
  const float c0 = sm.fs[0], c1 = sm.fs[1], c2 = sm.fs[2], frho = sm.fs[3];
  Slice as = slice_of(Nx, C, cta);
  for (int n = as.lo + warp; n < as.hi; n += nwarp) {
    for (int r = lane; r < R; r += 32) {
      float2 t = make_float2(0.f, 0.f);
      int idx = 0;
      for (int m = 0; m < s; ++m) {
        const int i = sm.rows[m];
        idx = (int)(((long long)i * n) % Nx);
        cfmac(t, sm.Wx[idx], Q[m * R + r]);
      }
      t = cscale(t, p.isx);
      const float2 a = p.A[n * R + r];
      const float2 grad = csub(cscale(a, frho), cmul(t, cconj(sm.gam[r])));
      const float2 a0 = p.A0[n * R + r];
      float2 an;
      an.x = c0 * a0.x + c1 * a.x - c2 * grad.x;
      an.y = c0 * a0.y + c1 * a.y - c2 * grad.y;
      p.A[n * R + r] = an;
    }
  }
  __syncthreads();
  // partial sums over this CTA's rows: Ahat'_S and ||a'_r||^2
  float2* part = p.partA + (size_t)cta * Nx * R;
  for (int m = warp; m < s; m += nwarp) {
    const int i = sm.rows[m];
    for (int r = lane; r < R; r += 32) {
      float2 acc = make_float2(0.f, 0.f);
      int idx = (int)(((long long)i * as.lo) % Nx);
      for (int n = as.lo; n < as.hi; ++n) {
        cfma(acc, sm.Wx[idx], p.A[n * R + r]);
        idx += i;
        if (idx >= Nx) idx -= Nx;
      }
      part[m * R + r] = cscale(acc, p.isx);
    }
  }
  if (warp == 0) {
    for (int r = lane; r < R; r += 32) {
      float acc = 0.f;
      for (int n = as.lo; n < as.hi; ++n) acc += cabs2(p.A[n * R + r]);
      p.partNA[cta * R + r] = acc;
    }
  }
}

// reduce the per-CTA partials of Ahat'_S and ||a'||^2 (this CTA's slice of entries)
__device__ void step_reduce_A(const FrameParams& p, Smem& sm, int cta, int k) {
  const int R = p.R, C = p.C, Nx = p.Nx;
  const int s = sm.misc[0];
  const int E = s * R + R;
  Slice es = slice_of(E, C, cta);
  float2* out = p.AhS[(k + 1) & 1];
  float* nout = p.nA[(k + 1) & 1];
  for (int e = es.lo + threadIdx.x; e < es.hi; e += blockDim.x) {
    if (e < s * R) {
      float2 acc = make_float2(0.f, 0.f);
      for (int c = 0; c < C; ++c) acc = cadd(acc, p.partA[(size_t)c * Nx * R + e]);
      out[e] = acc;
    } else {
      const int r = e - s * R;
      float acc = 0.f;
      for (int c = 0; c < C; ++c) acc += p.partNA[c * R + r];
      nout[r] = acc;
    }
  }
}

// ----------------------------------------------------------------------------------
// step "B": majorized B step (S2) on this CTA's rows, then partials of B^H B and P
// ----------------------------------------------------------------------------------
__device__ void step_B(const FrameParams& p, Smem& sm, int cta, int k, bool last) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int Nx = p.Nx, Ny = p.Ny, R = p.R, C = p.C;
  const int s = sm.misc[0];
  const int src = p.jacobi ? (k & 1) : ((k + 1) & 1);
  const float2* Ah = p.AhS[src];
  const float* nA = p.nA[src];
  for (int r = tid; r < R; r += blockDim.x) sm.gam[r] = p.gamma[r];
  __syncthreads();
  // gM[q][r] = gamma_q (Ahat^H Ahat)[r][q]
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int q = e / R, r = e - q * R;
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 0; m < s; ++m) cfmac(acc, Ah[m * R + r], Ah[m * R + q]);
    sm.gM[e] = cmul(sm.gam[q], acc);
  }
  if (tid == 0) {
    const double rho = p.sf[SF_RHO], abar = p.sf[SF_ABAR_B];
    double alpha = rho;
    for (int r = 0; r < R; ++r) {
      const float2 g = sm.gam[r];
      alpha += ((double)g.x * g.x + (double)g.y * g.y) * (double)nA[r];
    }
    const double den = p.lf * abar + alpha;
    sm.ds[0] = alpha;
    sm.ds[1] = abar;
    sm.fs[0] = (float)(p.lf * abar / den);
    sm.fs[1] = (float)(alpha / den);
    sm.fs[2] = (float)(1.0 / den);
    sm.fs[3] = (float)rho;
  }
  __syncthreads();
  const float c0 = sm.fs[0], c1 = sm.fs[1], c2 = sm.fs[2], frho = sm.fs[3];
  Slice bs = slice_of(Ny, C, cta);
  // one warp per row j: lane holds B[j][lane], B[j][lane+32]
  for (int j = bs.lo + warp; j < bs.hi; j += nwarp) {
    float2 b0 = lane < R ? p.B[j * R + lane] : make_float2(0.f, 0.f);
    float2 b1 = lane + 32 < R ? p.B[j * R + lane + 32] : make_float2(0.f, 0.f);
    float2 nb[2];
    const int halves = R > 32 ? 2 : 1;
    for (int h = 0; h < halves; ++h) {
      const int r = lane + 32 * h;
      float2 u = make_float2(0.f, 0.f);
      if (r < R)
        for (int m = 0; m < s; ++m) cfmac(u, Ah[m * R + r], p.Yt[(size_t)m * Ny + j]);  // Yt[m][j] conj(Ah[m][r])
      float2 tb = u;
      for (int q = 0; q < R; ++q) {
        const float2 bq = make_float2(__shfl_sync(0xffffffffu, q < 32 ? b0.x : b1.x, q & 31),
                                      __shfl_sync(0xffffffffu, q < 32 ? b0.y : b1.y, q & 31));
        if (r < R) tb = csub(tb, cmul(bq, sm.gM[q * R + r]));
      }
      const float2 b = h == 0 ? b0 : b1;
      if (r < R) {
        const float2 grad = csub(cscale(b, frho), cmul(tb, cconj(sm.gam[r])));
        const float2 bo = p.B0[j * R + r];
        nb[h].x = c0 * bo.x + c1 * b.x - c2 * grad.x;
        nb[h].y = c0 * bo.y + c1 * b.y - c2 * grad.y;
      }
    }
    __syncwarp();
    if (lane < R) p.B[j * R + lane] = nb[0];
    if (lane + 32 < R) p.B[j * R + lane + 32] = nb[1];
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
  float2* pmb = p.partMB + (size_t)cta * R * R;
  for (int q = warp; q < R; q += nwarp) {
    for (int r = lane; r < R; r += 32) {
      float2 acc = make_float2(0.f, 0.f);
      for (int j = bs.lo; j < bs.hi; ++j) cfmac(acc, p.B[j * R + q], p.B[j * R + r]);
      pmb[q * R + r] = acc;
    }
  }
  float2* pp = p.partP + (size_t)cta * Nx * R;
  for (int m = warp; m < s; m += nwarp) {
    for (int r = lane; r < R; r += 32) {
      float2 acc = make_float2(0.f, 0.f);
      for (int j = bs.lo; j < bs.hi; ++j) cfma(acc, p.Yt[(size_t)m * Ny + j], cconj(p.B[j * R + r]));
      pp[m * R + r] = acc;
    }
  }
}

// reduce the per-CTA partials of B^H B and P
__device__ void step_reduce_B(const FrameParams& p, Smem& sm, int cta) {
  const int R = p.R, C = p.C, Nx = p.Nx;
  const int s = sm.misc[0];
  const int E = R * R + s * R;
  Slice es = slice_of(E, C, cta);
  for (int e = es.lo + threadIdx.x; e < es.hi; e += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    if (e < R * R) {
      for (int c = 0; c < C; ++c) acc = cadd(acc, p.partMB[(size_t)c * R * R + e]);
      p.MB[e] = acc;
    } else {
      const int f = e - R * R;
      for (int c = 0; c < C; ++c) acc = cadd(acc, p.partP[(size_t)c * Nx * R + f]);
      p.P[f] = acc;
    }
  }
}

__global__ void __launch_bounds__(TTS_THREADS) frame_kernel(FrameParams p, int step_begin, int step_end,
                                                              int fft_rows, int fused) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem sm = carve(p, smem_raw, fft_rows);
  const int tid = threadIdx.x;
  const int cta = blockIdx.x;
  for (int e = tid; e < p.Nx; e += blockDim.x) sm.Wx[e] = p.Wx[e];
  for (int e = tid; e < p.Ny; e += blockDim.x) sm.Wy[e] = p.Wy[e];
  if (tid < 4) sm.misc[tid] = 0;
  __syncthreads();
  if (step_begin == 0) {
    // compact the line mask into the increasing list S (every CTA, warp 0)
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
    for (int e = tid; e < sm.misc[0]; e += blockDim.x) sm.rows[e] = p.rows[e];
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
      // frame rejected when any CTA saw a non-finite input sample
      int bad = 0;
      for (int c = 0; c < p.C; ++c) bad |= ((volatile int*)p.status)[1 + c];
      if (bad) {
        if (step == 1 && cta == 0 && tid == 0) atomicOr(p.status, 1);
        return;
      }
    }
    if (step == 0) {
      step_ingest(p, sm, cta);
      continue;
    }
    const int k = (step - 1) / 4, sub = (step - 1) % 4;
    if (sub == 0) step_solve_A(p, sm, cta, k);
    else if (sub == 1) step_reduce_A(p, sm, cta, k);
    else if (sub == 2) step_B(p, sm, cta, k, k == p.K - 1);
    else step_reduce_B(p, sm, cta);
    __syncthreads();
  }
}

// The ridge solve alone on a given Hermitian positive-definite system (test hook).
__global__ void __launch_bounds__(TTS_THREADS) ridge_kernel(const double2* G, const double2* h, int R, double2* gamma) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FrameParams p;
  p.R = R;
  Smem sm;
  sm.G = (double2*)smem_raw;
  sm.z = sm.G + R * R;
  sm.h = sm.z + R;
  sm.invd = (double*)(sm.h + R);
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) sm.G[e] = G[e];
  for (int e = threadIdx.x; e < R; e += blockDim.x) sm.h[e] = h[e];
  __syncthreads();
  ldl_solve(p, sm, sm.h);
  for (int e = threadIdx.x; e < R; e += blockDim.x) gamma[e] = sm.z[e];
}

}  // namespace

int launch_ridge(const double2* G, const double2* h, int R, double2* gamma, cudaStream_t st) {
  const int smem = (int)(sizeof(double2) * (R * R + 2 * R) + sizeof(double) * R);
  ridge_kernel<<<1, TTS_THREADS, smem, st>>>(G, h, R, gamma);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

int frame_smem_bytes(const FrameParams& p) {
  const int fft_rows = max(1, min((p.Nx + p.C - 1) / p.C, 4096 / p.Ny));
  size_t b = 0;
  auto add = [&](size_t bytes) { b = ((b + 15) & ~size_t(15)) + bytes; };
  add(sizeof(double2) * p.R * p.R);
  add(sizeof(double2) * p.R);
  add(sizeof(double) * p.R);
  add(sizeof(double2) * p.R);
  add(sizeof(float) * 8);
  add(sizeof(double) * 8);
  add(sizeof(float2) * p.Nx);
  add(sizeof(float2) * p.Ny);
  add(sizeof(float2) * p.R);
  add(sizeof(float2) * p.R * p.R);
  add(sizeof(int) * p.Nx);
  add(sizeof(int) * 4);
  add(sizeof(float) * TTS_THREADS);
  add(sizeof(float2) * 2 * fft_rows * p.Ny);
  return (int)b + 16;
}

int launch_frame(const FrameParams& p, int launch_mode, cudaStream_t st) {
  const int fft_rows = max(1, min((p.Nx + p.C - 1) / p.C, 4096 / p.Ny));
  const int smem = frame_smem_bytes(p);
  cudaError_t e = cudaFuncSetAttribute(frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return TTS_ECUDA;
  const int nsteps = frame_num_steps(p.K);
  if (launch_mode == TTS_LAUNCH_FUSED) {
    if (p.C > 8) {
      e = cudaFuncSetAttribute(frame_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return TTS_ECUDA;
    }
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
    e = cudaLaunchKernelEx(&cfg, frame_kernel, p, 0, nsteps, fft_rows, 1);
    if (e != cudaSuccess) return TTS_ECUDA;
  } else {
    for (int s = 0; s < nsteps; ++s) {
      frame_kernel<<<p.C, TTS_THREADS, smem, st>>>(p, s, s + 1, fft_rows, 0);
      if (cudaGetLastError() != cudaSuccess) return TTS_ECUDA;
    }
  }
  return TTS_OK;
}
