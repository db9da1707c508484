// Multi-coil tracker: Alg. 3 of the paper with C receive coils of known sensitivity
// (§IV-B, tomographic parallel MRI). Coil c sees y_c = P_Omega F(H_c .* L_t) + v. With
// coils the sensitivity-weighted rank-one images H_c .* a_r b_r^T are no longer rank
// one, so the separable shortcut of the single-coil frame kernel does not apply: each MM
// iteration transforms them explicitly.
//
// Per frame (all on the handle's stream, FP32 data, FP64 scalars and ridge system):
//   begin:   w <- lf w + 1, rho = mu / w; anchors A0 = A, B0 = B
//   per MM iteration (Gauss-Seidel gamma -> A -> B):
//     (S1)  Z[c][r] = H_c .* a_r b_r^T; batched 2D DFT; Phi rows = Z[c][r][S, :] kept
//           compact (Zs, |S| rows per image): for band-shape Nx, Ny the rows of the
//           rank-one images are generated inside the row transform and the column
//           transform stores only the rows of S
//           G = Phi^H Phi + mu I (FP32 per acquired row, FP64 across rows), h = Phi^H y;
//           gamma = G^{-1} h (FP32 Gauss-Jordan + float-float refinement, FP64 grade)
//     (S2)  E_c = P_Omega(y_c - sum_r gamma_r Z[c][r]) (zero-filled), batched inverse DFT,
//           Theta = sum_c conj(H_c) .* E_c; alpha_A = h_max sum_r |gamma_r|^2 ||b_r||^2 + rho;
//           A <- c0 A0 + c1 A - c2 (rho A - Theta conj(B) diag(conj gamma))
//           X = A diag(gamma) B^T; E'_c = P_Omega(y_c - F(H_c .* X)); Theta' likewise;
//           alpha_B with ||a_r||; B <- c0 B0 + c1 B - c2 (rho B - Theta'^T conj(A) diag(conj gamma))
//   end:     abar <- lf abar + alpha (last iteration's), frame count
#include <math.h>
#include <string.h>

#include <vector>

#include <algorithm>

#include "tts_fft_band.cuh"
#include "tts_handle.cuh"

namespace {

constexpr int kT = 256;

// Z[c * R + r] = H_c .* (a_r b_r^T)
__global__ void mc_rank1_kernel(const float2* __restrict__ H, const float2* __restrict__ A,
                                const float2* __restrict__ B, float2* __restrict__ Z, int C, int R, int Nx, int Ny) {
  const size_t NN = (size_t)Nx * Ny;
  const size_t total = (size_t)C * R * NN;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t img = e / NN, pix = e - img * NN;
    const int c = (int)(img / R), r = (int)(img - (size_t)c * R);
    const int i = (int)(pix / Ny), j = (int)(pix - (size_t)i * Ny);
    Z[e] = cmul(H[(size_t)c * NN + pix], cmul(A[i * R + r], B[j * R + r]));
  }
}

// Partial Gram and right-hand side of one acquired row (c, m): over j < Ny,
// G[q][r] += conj(Phi_q) Phi_r, h[q] += conj(Phi_q) y with Phi_r = Zs[c R + r][m][j] (the
// transformed rank-one images on the rows of S, compact). One CTA per (c, m); the R x Ny
// block of Phi staged in shared memory.
__global__ void __launch_bounds__(kT) mc_gram_kernel(const float2* __restrict__ Zs, const float2* __restrict__ y,
                                                     int C, int R, int Ny, int s, double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LD = Ny + 1;            // odd row stride: consecutive r hit distinct banks
  float2* ph = (float2*)smem_raw;   // R x LD
  float2* yr = ph + R * LD;         // Ny
  const int cm = blockIdx.x, c = cm / s, m = cm - c * s;
  for (int e = threadIdx.x; e < R * Ny; e += blockDim.x) {
    const int r = e / Ny, j = e - r * Ny;
    ph[r * LD + j] = Zs[(((size_t)c * R + r) * s + m) * Ny + j];
  }
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) yr[j] = y[((size_t)c * s + m) * Ny + j];
  __syncthreads();
  const int E = R * R + R;
  double2* out = part + (size_t)cm * E;
  // G in 2 x 2 register tiles: tile (qt, rt) holds q in {qt, qt + hR}, r in {rt, rt + hR}
  // (rows hR apart: the LD-strided loads of a warp land on distinct banks). Every output
  // sums even j and odd j in its own accumulators, in increasing j.
  const int hR = (R + 1) / 2;
  for (int tile = threadIdx.x; tile < hR * hR; tile += blockDim.x) {
    const int qt = tile / hR, rt = tile - qt * hR;
    const int q[2] = {qt, qt + hR}, r[2] = {rt, rt + hR};
    const bool qv1 = q[1] < R, rv1 = r[1] < R;
    const float2* a0 = ph + q[0] * LD;
    const float2* a1 = ph + (qv1 ? q[1] : q[0]) * LD;
    const float2* b0 = ph + r[0] * LD;
    const float2* b1 = ph + (rv1 ? r[1] : r[0]) * LD;
    float2 e0[4], e1[4];   // outputs (q0 r0, q0 r1, q1 r0, q1 r1), even / odd j
#pragma unroll
    for (int o = 0; o < 4; ++o) e0[o] = e1[o] = make_float2(0.f, 0.f);
    int j = 0;
    for (; j + 1 < Ny; j += 2) {
      const float2 x0 = a0[j], x1 = a1[j], y0 = b0[j], y1 = b1[j];
      const float2 u0 = a0[j + 1], u1 = a1[j + 1], w0 = b0[j + 1], w1 = b1[j + 1];
      cfmac(e0[0], x0, y0);
      cfmac(e1[0], u0, w0);
      cfmac(e0[1], x0, y1);
      cfmac(e1[1], u0, w1);
      cfmac(e0[2], x1, y0);
      cfmac(e1[2], u1, w0);
      cfmac(e0[3], x1, y1);
      cfmac(e1[3], u1, w1);
    }
    if (j < Ny) {
      cfmac(e0[0], a0[j], b0[j]);
      cfmac(e0[1], a0[j], b1[j]);
      cfmac(e0[2], a1[j], b0[j]);
      cfmac(e0[3], a1[j], b1[j]);
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int qq = q[o >> 1], rr = r[o & 1];
      if (qq < R && rr < R)
        out[qq * R + rr] = make_double2((double)e0[o].x + (double)e1[o].x, (double)e0[o].y + (double)e1[o].y);
    }
  }
  // h: conj(Phi_q) y
  for (int qq = threadIdx.x; qq < R; qq += blockDim.x) {
    const float2* a = ph + qq * LD;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    int j = 0;
    for (; j + 1 < Ny; j += 2) {
      cfmac(acc0, a[j], yr[j]);
      cfmac(acc1, a[j + 1], yr[j + 1]);
    }
    if (j < Ny) cfmac(acc0, a[j], yr[j]);
    out[R * R + qq] = make_double2((double)acc0.x + (double)acc1.x, (double)acc0.y + (double)acc1.y);
  }
}

// G = sum of the partials + mu I, h = sum of the partials (FP64): one warp per entry, lane l
// summing partials l, l + 32, ..., then a fixed shuffle tree (the order never changes)
__global__ void mc_gram_reduce_kernel(const double2* __restrict__ part, int nparts, int R, double mu,
                                      double2* __restrict__ G, double2* __restrict__ h) {
  const int E = R * R + R;
  const int lane = threadIdx.x & 31;
  const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (e >= E) return;   // whole warps
  double ax = 0.0, ay = 0.0;
  for (int p = lane; p < nparts; p += 32) {
    const double2 v = part[(size_t)p * E + e];
    ax += v.x;
    ay += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
  }
  if (lane == 0) {
    if (e < R * R) {
      if (e / R == e % R) ax += mu;
      G[e] = make_double2(ax, ay);
    } else {
      h[e - R * R] = make_double2(ax, ay);
    }
  }
}

// Zero-filled coil residuals: E_c[S_m][j] = y_c[m][j] - sum_r gamma_r Zs[c][r][m][j] where
// Zs holds the transformed rank-one images on the rows of S, compact (gamma from FP64),
// other rows 0. With Zx set (the refresh), the model value is Zx[c][S_m][j] instead of the
// gamma-weighted sum.
__global__ void mc_residual_kernel(const float2* __restrict__ Zf, const float2* __restrict__ Zx,
                                   const double2* __restrict__ gamma_d, const float2* __restrict__ y,
                                   const int* __restrict__ rows, const int* __restrict__ rowpos, int C, int R, int Nx,
                                   int Ny, int s, float2* __restrict__ E, float2* __restrict__ gamma_f) {
  __shared__ float2 g[TTS_MAX_R];
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double2 v = gamma_d[r];
    g[r] = make_float2((float)v.x, (float)v.y);
    if (blockIdx.x == 0 && gamma_f) gamma_f[r] = g[r];
  }
  __syncthreads();
  const size_t NN = (size_t)Nx * Ny;
  const size_t total = (size_t)C * NN;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / NN);
    const size_t pix = e - (size_t)c * NN;
    const int i = (int)(pix / Ny), j = (int)(pix - (size_t)i * Ny);
    const int m = rowpos[i];
    float2 v = make_float2(0.f, 0.f);
    if (m >= 0) {
      float2 model = make_float2(0.f, 0.f);
      if (Zx) {
        model = Zx[e];
      } else {
        for (int r = 0; r < R; ++r) cfma(model, g[r], Zf[(((size_t)c * R + r) * s + m) * Ny + j]);
      }
      v = csub(y[((size_t)c * s + m) * Ny + j], model);
    }
    E[e] = v;
  }
  (void)rows;
}

// Theta = sum_c conj(H_c) .* E_c ; or (weigh) Zx_c = H_c .* X for every coil
__global__ void mc_theta_kernel(const float2* __restrict__ H, const float2* __restrict__ E, int C, size_t NN,
                                float2* __restrict__ Theta) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < NN; p += (size_t)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < C; ++c) cfmac(acc, H[(size_t)c * NN + p], E[(size_t)c * NN + p]);
    Theta[p] = acc;
  }
}
__global__ void mc_weigh_kernel(const float2* __restrict__ H, const float2* __restrict__ X, int C, size_t NN,
                                float2* __restrict__ Zx) {
  const size_t total = (size_t)C * NN;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    Zx[e] = cmul(H[e], X[e % NN]);
}

// Frame begin / end scalars (FP64), as the single-coil frame kernel keeps them.
__global__ void mc_begin_kernel(double* sc, double* sf, double lf, double mu) {
  const double w = lf * sc[SC_W] + 1.0;
  sf[SF_W] = w;
  sf[SF_RHO] = mu / w;
  sf[SF_ABAR_A] = sc[SC_ABAR_A];
  sf[SF_ABAR_B] = sc[SC_ABAR_B];
}
__global__ void mc_end_kernel(double* sc, const double* sf, double lf, float2* gamma, const double2* gamma_d, int R) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) gamma[r] = make_float2((float)gamma_d[r].x, (float)gamma_d[r].y);
  if (threadIdx.x == 0) {
    sc[SC_W] = sf[SF_W];
    sc[SC_ABAR_A] = lf * sf[SF_ABAR_A] + sf[SF_ALPHA_A];
    sc[SC_ABAR_B] = lf * sf[SF_ABAR_B] + sf[SF_ALPHA_B];
    sc[SC_T] += 1.0;
  }
}

// MM step coefficients of one block: alpha = h_max sum_r |gamma_r|^2 ||f_r||^2 + rho over the
// other factor F (n x R); c0 = lf abar / den, c1 = alpha / den, c2 = 1 / den with
// den = lf abar + alpha; alpha to sf[slot]. One CTA.
__global__ void mc_coeff_kernel(const float2* __restrict__ F, int n, int R, const double2* __restrict__ gamma_d,
                                double hmax, double lf, double* sf, int abar_slot, int alpha_slot,
                                float* __restrict__ coef) {
  __shared__ double red[kT];
  __shared__ float g2[TTS_MAX_R];   // |gamma_r|^2 from FP64, once per r (FP64 is slow on this part)
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double2 g = gamma_d[r];
    g2[r] = (float)(g.x * g.x + g.y * g.y);
  }
  __syncthreads();
  float acc = 0.f;   // per-thread sums in FP32 (as the single-coil frame kernel), the tree in FP64
  const int total = n * R, step = blockDim.x;
  for (int base = threadIdx.x; base < total; base += 8 * step) {
    float2 v[8];   // eight loads in flight, then the sums in the same order as one at a time
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = base + u * step < total ? F[base + u * step] : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (base + u * step < total) acc = fmaf(cabs2(v[u]), g2[(base + u * step) % R], acc);
  }
  red[threadIdx.x] = (double)acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rho = sf[SF_RHO], abar = sf[abar_slot];
    const double alpha = hmax * red[0] + rho;
    const double den = lf * abar + alpha;
    sf[alpha_slot] = alpha;
    coef[0] = (float)(lf * abar / den);
    coef[1] = (float)(alpha / den);
    coef[2] = (float)(1.0 / den);
    coef[3] = (float)rho;
  }
}

// Factor step: for row p of X (n x R), T[p][r] = sum_q M(p, q) conj(F[q][r]) with
// M(p, q) = Mb[p sp + q sq] (nq terms), then X[p][r] <- c0 X0 + c1 X - c2 (rho X - T conj(gamma_r)).
// One CTA per row p; lanes over (q mod Q, r).
__global__ void __launch_bounds__(kT) mc_step_kernel(const float2* __restrict__ Mb, size_t sp, size_t sq, int nq,
                                                     const float2* __restrict__ F, int R, float2* __restrict__ X,
                                                     const float2* __restrict__ X0, const double2* __restrict__ gamma_d,
                                                     const float* __restrict__ coef) {
  __shared__ float2 red[kT];
  const int p = blockIdx.x;
  const int Q = blockDim.x / R;
  const int tid = threadIdx.x;
  const int r = tid % R, ql = tid / R;
  float2 acc = make_float2(0.f, 0.f);
  if (ql < Q)
    for (int q = ql; q < nq; q += Q) cfmac(acc, F[q * R + r], Mb[p * sp + q * sq]);   // conj(F) M
  red[tid] = acc;
  __syncthreads();
  if (tid < R) {
    float2 t = red[tid];
    for (int k = 1; k < Q; ++k) t = cadd(t, red[k * R + tid]);
    const double2 gd = gamma_d[tid];
    const float2 g = make_float2((float)gd.x, (float)gd.y);
    const float c0 = coef[0], c1 = coef[1], c2 = coef[2], rho = coef[3];
    const float2 x = X[p * R + tid], x0 = X0[p * R + tid];
    const float2 grad = csub(cscale(x, rho), cmul(t, cconj(g)));
    float2 nx;
    nx.x = fmaf(-c2, grad.x, fmaf(c1, x.x, c0 * x0.x));
    nx.y = fmaf(-c2, grad.y, fmaf(c1, x.y, c0 * x0.y));
    X[p * R + tid] = nx;
  }
}

// S (increasing) and, per line, its position in S (-1 if not acquired); one CTA.
__global__ void mc_rows_kernel(const uint8_t* __restrict__ mask, int Nx, int* rows, int* nrows, int* rowpos) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int count = 0;
    for (int base = 0; base < Nx; base += 32) {
      const int i = base + lane;
      const bool on = i < Nx && mask[i] != 0;
      const unsigned bal = __ballot_sync(0xffffffffu, on);
      const int pos = count + __popc(bal & ((1u << lane) - 1u));
      if (i < Nx) rowpos[i] = on ? pos : -1;
      if (on) rows[pos] = i;
      count += __popc(bal);
    }
    if (lane == 0) *nrows = count;
  }
}

// The acquired rows of each coil from full coil frames (C x Nx x Ny) into C x |S| x Ny.
__global__ void mc_gather_kernel(const float2* __restrict__ full, const int* __restrict__ rows, int C, int Nx,
                                 int Ny, int s, float2* __restrict__ y, int* bad) {
  const size_t total = (size_t)C * s * Ny;
  int b = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t cm = e / Ny;
    const int j = (int)(e - cm * Ny);
    const int c = (int)(cm / s), m = (int)(cm - (size_t)c * s);
    const float2 v = full[((size_t)c * Nx + rows[m]) * Ny + j];
    if (!isfinite(v.x) || !isfinite(v.y)) b = 1;
    y[e] = v;
  }
  if (b) atomicOr(bad, 1);
}

__global__ void mc_check_kernel(const float2* __restrict__ y, size_t n, int* bad) {
  int b = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 v = y[e];
    if (!isfinite(v.x) || !isfinite(v.y)) b = 1;
  }
  if (b) atomicOr(bad, 1);
}

// The rows of S of n transformed images (Nx x Ny each) into Zs, compact (|S| rows each).
__global__ void mc_compact_kernel(const float2* __restrict__ Z, const int* __restrict__ rows, int n, int Nx, int Ny,
                                  int s, float2* __restrict__ Zs) {
  const size_t total = (size_t)n * s * Ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t im = e / Ny;
    const int j = (int)(e - im * Ny);
    const size_t img = im / s;
    const int m = (int)(im - img * s);
    Zs[e] = Z[(img * Nx + rows[m]) * Ny + j];
  }
}

// (S1) for band-shape Nx and Ny (tts_fft_band.cuh): the transformed weighted rank-one images
// on the rows of S only. Row pass: image img = c R + r, row i generated as
// H_c[i][j] (a_r[i] b_r[j]) (the product of mc_rank1_kernel) and transformed into Z[img].
// Column pass: the columns of Z[img] transformed, the rows of S stored compact into Zs
// (scaled by 1 / sqrt(Nx Ny)), the others dropped. Both persistent over the bands of a group.
template <int N>
constexpr int phi_minb() {
  return fftband::Shape<N>::R == 16 ? (3 * fftband::Shape<N>::MINB) / 4 : fftband::Shape<N>::MINB;
}

template <int NY>
__global__ void __launch_bounds__(fftband::Shape<NY>::NT, phi_minb<NY>())
    mc_phi_rows_kernel(const float2* __restrict__ H, const float2* __restrict__ A, const float2* __restrict__ B, int R,
                       int Nx, int img0, int nimg, float2* __restrict__ Z, const float2* __restrict__ Wg) {
  constexpr int BAND = fftband::Shape<NY>::BAND;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = (float2*)smem_raw;
  float2* W = S + BAND * fftband::row_stride<NY>();
  for (int k = threadIdx.x; k < NY; k += blockDim.x) W[fpad(k)] = Wg[k];
  const int nb = (Nx + BAND - 1) / BAND;
  const size_t NN = (size_t)Nx * NY;
  for (int task = blockIdx.x; task < nimg * nb; task += gridDim.x) {
    __syncthreads();   // the table; the previous band's last use of S
    const int il = task / nb, band = task - il * nb;
    const int img = img0 + il, c = img / R, r = img - c * R;
    const float2* Hc = H + (size_t)c * NN;
    fftband::row_band_f<NY, false, true>(
        [=](int i, int j) { return cmul(Hc[(size_t)i * NY + j], cmul(A[i * R + r], B[j * R + r])); },
        Z + (size_t)img * NN, Nx, band * BAND, W, S);
  }
}

template <int NX>
__global__ void __launch_bounds__(fftband::Shape<NX>::NT, phi_minb<NX>())
    mc_phi_cols_kernel(const float2* __restrict__ Z, float2* __restrict__ Zs, const int* __restrict__ rowpos, int s,
                       int Ny, int img0, int nimg, const float2* __restrict__ Wg, float scale) {
  constexpr int BAND = fftband::Shape<NX>::BAND;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = (float2*)smem_raw;
  float2* W = S + BAND * fftband::row_stride<NX>();
  for (int k = threadIdx.x; k < NX; k += blockDim.x) W[fpad(k)] = Wg[k];
  const int nb = (Ny + BAND - 1) / BAND;
  const size_t NN = (size_t)NX * Ny;
  for (int task = blockIdx.x; task < nimg * nb; task += gridDim.x) {
    __syncthreads();   // the table; the previous band's last use of S
    const int il = task / nb, band = task - il * nb;
    const int img = img0 + il;
    float2* zs = Zs + (size_t)img * s * Ny;
    fftband::col_band_f<NX, false, true>(Z + (size_t)img * NN, Ny, band * BAND, W, S,
                                         [=](int k, int col, float2 v) {
                                           const int m = rowpos[k];
                                           if (m >= 0) zs[(size_t)m * Ny + col] = cscale(v, scale);
                                         });
  }
}

template <typename K>
int phi_grid(K kernel, int threads, int smem, int tasks) {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
    return 0;
  return std::min(per_sm * sms, tasks);
}

template <int NY>
int phi_rows_t(const float2* H, const float2* A, const float2* B, int R, int Nx, int img0, int nimg, float2* Z,
               const float2* Wy, cudaStream_t st) {
  constexpr int smem = fftband::smem_bytes<NY>();
  const int tasks = nimg * ((Nx + fftband::Shape<NY>::BAND - 1) / fftband::Shape<NY>::BAND);
  const int g = phi_grid(mc_phi_rows_kernel<NY>, fftband::Shape<NY>::NT, smem, tasks);
  if (g < 1) return TTS_ECUDA;
  mc_phi_rows_kernel<NY><<<g, fftband::Shape<NY>::NT, smem, st>>>(H, A, B, R, Nx, img0, nimg, Z, Wy);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

template <int NX>
int phi_cols_t(const float2* Z, float2* Zs, const int* rowpos, int s, int Ny, int img0, int nimg, const float2* Wx,
               float scale, cudaStream_t st) {
  constexpr int smem = fftband::smem_bytes<NX>();
  const int tasks = nimg * ((Ny + fftband::Shape<NX>::BAND - 1) / fftband::Shape<NX>::BAND);
  const int g = phi_grid(mc_phi_cols_kernel<NX>, fftband::Shape<NX>::NT, smem, tasks);
  if (g < 1) return TTS_ECUDA;
  mc_phi_cols_kernel<NX><<<g, fftband::Shape<NX>::NT, smem, st>>>(Z, Zs, rowpos, s, Ny, img0, nimg, Wx, scale);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

#define TTS_BAND_CASES(X) \
  X(64) X(96) X(120) X(128) X(144) X(160) X(192) X(200) X(216) X(240) X(256) X(288) X(320) X(384)

// the transformed rank-one images on the rows of S into Zs; TTS_EINVAL for other sizes
int launch_phi(const float2* H, const float2* A, const float2* B, int C, int R, int Nx, int Ny, int s,
               const int* rowpos, const float2* Wx, const float2* Wy, float2* Z, float2* Zs, cudaStream_t st) {
  if (!fftband::supported(Nx) || !fftband::supported(Ny)) return TTS_EINVAL;
  const size_t NN = (size_t)Nx * Ny;
  const int n = C * R;
  const int group = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, (40u << 20) / (NN * sizeof(float2))));
  const float scale = 1.0f / sqrtf((float)Nx * (float)Ny);
  for (int g0 = 0; g0 < n; g0 += group) {
    const int k = std::min(group, n - g0);
    int rc = TTS_EINVAL;
    switch (Ny) {
#define ROWS(N) \
  case N: rc = phi_rows_t<N>(H, A, B, R, Nx, g0, k, Z, Wy, st); break;
      TTS_BAND_CASES(ROWS)
#undef ROWS
    }
    if (rc != TTS_OK) return rc;
    rc = TTS_EINVAL;
    switch (Nx) {
#define COLS(N) \
  case N: rc = phi_cols_t<N>(Z, Zs, rowpos, s, Ny, g0, k, Wx, scale, st); break;
      TTS_BAND_CASES(COLS)
#undef COLS
    }
    if (rc != TTS_OK) return rc;
  }
  return TTS_OK;
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + kT - 1) / kT, 152 * 16); }

}  // namespace

struct MultiCoil {
  int C = 0;
  double hmax = 0.0;
  void* mem = nullptr;
  float2* H = nullptr;        // C x Nx x Ny
  float2* Z = nullptr;        // C R x Nx x Ny: weighted rank-one images, transformed in place
  float2* Zs = nullptr;       // C R x |S| x Ny: their transforms on the rows of S, compact
  float2* E = nullptr;        // C x Nx x Ny: residuals, back-projected in place; the refresh's H_c .* X
  float2* Zx = nullptr;       // C x Nx x Ny: transforms of H_c .* X
  float2* Theta = nullptr;    // Nx x Ny
  float2* X = nullptr;        // Nx x Ny
  float2* y = nullptr;        // C x |S| x Ny acquired rows
  int* rowpos = nullptr;      // Nx
  double2* part = nullptr;    // C Nx x (R^2 + R) Gram partials
  int* flag = nullptr;        // non-finite input sample seen on the device
  double2* G = nullptr;       // R x R
  double2* h = nullptr;       // R
  float* coef = nullptr;      // 4
};

namespace {
size_t up(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

int mc_attach(tts_handle* h, const float2* maps, int C, bool device) {
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny, R = h->cfg.R;
  const size_t NN = (size_t)Nx * Ny;
  std::vector<float2> hm(C * NN);
  if (device) {
    if (cudaMemcpy(hm.data(), maps, sizeof(float2) * C * NN, cudaMemcpyDeviceToHost) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "coil maps");
  } else {
    memcpy(hm.data(), maps, sizeof(float2) * C * NN);
  }
  double hmax = 0.0;
  for (size_t p = 0; p < NN; ++p) {
    double s = 0.0;
    for (int c = 0; c < C; ++c) {
      const float2 v = hm[(size_t)c * NN + p];
      if (!isfinite(v.x) || !isfinite(v.y)) return tts_fail(TTS_EINVAL, "coil maps hold NaN or Inf%s");
      s += (double)v.x * v.x + (double)v.y * v.y;
    }
    hmax = s > hmax ? s : hmax;
  }
  MultiCoil* m = h->mc ? h->mc : new MultiCoil();
  if (m->mem) cudaFree(m->mem);
  m->mem = nullptr;
  m->C = C;
  m->hmax = hmax;
  struct P {
    void** p;
    size_t b;
  };
  std::vector<P> ps = {{(void**)&m->H, sizeof(float2) * C * NN},
                       {(void**)&m->Z, sizeof(float2) * (size_t)C * R * NN},
                       {(void**)&m->Zs, sizeof(float2) * (size_t)C * R * NN},
                       {(void**)&m->E, sizeof(float2) * C * NN},
                       {(void**)&m->Zx, sizeof(float2) * C * NN},
                       {(void**)&m->Theta, sizeof(float2) * NN},
                       {(void**)&m->X, sizeof(float2) * NN},
                       {(void**)&m->y, sizeof(float2) * C * NN},
                       {(void**)&m->rowpos, sizeof(int) * Nx},
                       {(void**)&m->part, sizeof(double2) * (size_t)C * Nx * (R * R + R)},
                       {(void**)&m->G, sizeof(double2) * R * R},
                       {(void**)&m->h, sizeof(double2) * R},
                       {(void**)&m->coef, sizeof(float) * 4},
                       {(void**)&m->flag, sizeof(int)}};
  size_t total = 0;
  for (auto& q : ps) total += up(q.b);
  if (cudaMalloc(&m->mem, total) != cudaSuccess) {
    m->mem = nullptr;
    if (!h->mc) delete m;
    return tts_fail(TTS_ENOMEM, "device allocation of the multi-coil workspace failed%s");
  }
  size_t off = 0;
  for (auto& q : ps) {
    *q.p = (char*)m->mem + off;
    off += up(q.b);
  }
  h->mc = m;
  if (cudaMemcpyAsync(m->H, hm.data(), sizeof(float2) * C * NN, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return tts_cuda_fail(cudaGetLastError(), "coil maps");
  return TTS_OK;
}

void mc_detach(tts_handle* h) {
  if (!h->mc) return;
  if (h->mc->mem) cudaFree(h->mc->mem);
  delete h->mc;
  h->mc = nullptr;
}

// One frame of the multi-coil tracker. y: acquired rows C x |S| x Ny (or full coil frames
// C x Nx x Ny with TTS_FULL_FRAME), host or device; mask: Nx bytes (host or device).
int mc_push(tts_handle* h, const tts_c64* y_in, const uint8_t* mask_in, int flags) {
  MultiCoil* m = h->mc;
  FrameParams& p = h->fp;
  const int Nx = h->cfg.Nx, Ny = h->cfg.Ny, R = h->cfg.R, C = m->C, K = h->cfg.mm_iters;
  const size_t NN = (size_t)Nx * Ny;
  cudaStream_t st = h->stream;
  const bool dev = (flags & TTS_DEVICE_PTRS) != 0, full = (flags & TTS_FULL_FRAME) != 0;
  // the line set: host masks are counted here, device masks on the device
  int s = 0;
  const uint8_t* dmask = nullptr;
  std::vector<uint8_t> hmask;
  if (!mask_in) {
    if (!h->have_next) return tts_fail(TTS_ESTATE, "no mask given and none drawn yet%s");
    dmask = h->dmask_next;
    hmask.resize(Nx);
    if (cudaMemcpyAsync(hmask.data(), dmask, Nx, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "mask");
  } else if (dev) {
    dmask = mask_in;
    hmask.resize(Nx);
    if (cudaMemcpyAsync(hmask.data(), dmask, Nx, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "mask");
  } else {
    hmask.assign(mask_in, mask_in + Nx);
    if (cudaMemcpyAsync(h->dmask_push, mask_in, Nx, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "mask");
    dmask = h->dmask_push;
  }
  for (int i = 0; i < Nx; ++i) s += hmask[i] != 0;
  if (s == 0) return tts_fail(TTS_EINVAL, "the line mask selects no line%s");
  mc_rows_kernel<<<1, 32, 0, st>>>(dmask, Nx, p.rows, p.nrows, m->rowpos);
  // the acquired rows of every coil into m->y (C x |S| x Ny); device inputs are checked on
  // the device before anything is applied
  const size_t nrow_bytes = sizeof(float2) * (size_t)C * s * Ny;
  bool dev_check = true;
  if (cudaMemsetAsync(m->flag, 0, sizeof(int), st) != cudaSuccess) return tts_cuda_fail(cudaGetLastError(), "flag");
  if (full) {
    const float2* src = (const float2*)y_in;
    if (!dev) {   // host full frames: staged whole in the residual buffer, then gathered
      if (cudaMemcpyAsync(m->E, y_in, sizeof(float2) * C * NN, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return tts_cuda_fail(cudaGetLastError(), "frame");
      src = m->E;
    }
    mc_gather_kernel<<<grid_for((size_t)C * s * Ny), kT, 0, st>>>(src, p.rows, C, Nx, Ny, s, m->y, m->flag);
  } else if (dev) {
    if (cudaMemcpyAsync(m->y, y_in, nrow_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "frame");
    mc_check_kernel<<<grid_for((size_t)C * s * Ny), kT, 0, st>>>(m->y, (size_t)C * s * Ny, m->flag);
  } else {
    const float* f = (const float*)y_in;
    for (size_t e = 0; e < 2 * (size_t)C * s * Ny; ++e)
      if (!isfinite(f[e])) return tts_fail(TTS_ENONFINITE, "frame holds NaN or Inf; not applied%s");
    if (cudaMemcpyAsync(m->y, y_in, nrow_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "frame");
    dev_check = false;
  }
  if (dev_check) {
    int bad = 0;
    if (cudaMemcpyAsync(&bad, m->flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return tts_cuda_fail(cudaGetLastError(), "flag");
    if (bad) {   // skipped; reported once by tts_synchronize
      const int one = 1;
      if (cudaMemcpyAsync(p.status, &one, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return tts_cuda_fail(cudaGetLastError(), "status");
      return TTS_OK;
    }
  }
  mc_begin_kernel<<<1, 1, 0, st>>>(p.sc, p.sf, p.lf, p.mu);
  cudaMemcpyAsync(p.A0, p.A, sizeof(float2) * Nx * R, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(p.B0, p.B, sizeof(float2) * Ny * R, cudaMemcpyDeviceToDevice, st);
  const int gram_smem = (int)(sizeof(float2) * ((size_t)R * (Ny + 1) + Ny));
  if (cudaFuncSetAttribute(mc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, gram_smem) != cudaSuccess)
    return tts_cuda_fail(cudaGetLastError(), "gram attributes");
  int rc = TTS_OK;
  for (int k = 0; k < K && rc == TTS_OK; ++k) {
    // (S1)
    rc = launch_phi(m->H, p.A, p.B, C, R, Nx, Ny, s, m->rowpos, p.Wx, p.Wy, m->Z, m->Zs, st);
    if (rc == TTS_EINVAL) {   // other sizes: explicit rank-one images, batched DFT, rows of S
      mc_rank1_kernel<<<grid_for((size_t)C * R * NN), kT, 0, st>>>(m->H, p.A, p.B, m->Z, C, R, Nx, Ny);
      rc = tts_fft2d((const tts_c64*)m->Z, (tts_c64*)m->Z, C * R, Nx, Ny, 0, st);
      if (rc != TTS_OK) break;
      mc_compact_kernel<<<grid_for((size_t)C * R * s * Ny), kT, 0, st>>>(m->Z, p.rows, C * R, Nx, Ny, s, m->Zs);
    }
    if (rc != TTS_OK) break;
    mc_gram_kernel<<<C * s, kT, gram_smem, st>>>(m->Zs, m->y, C, R, Ny, s, m->part);
    mc_gram_reduce_kernel<<<((R * R + R) * 32 + kT - 1) / kT, kT, 0, st>>>(m->part, C * s, R, p.mu, m->G, m->h);
    rc = launch_ridge(m->G, m->h, R, p.gamma_d, st);
    if (rc != TTS_OK) break;
    // (S2) A block
    mc_residual_kernel<<<grid_for((size_t)C * NN), kT, 0, st>>>(m->Zs, nullptr, p.gamma_d, m->y, p.rows, m->rowpos, C,
                                                                R, Nx, Ny, s, m->E, p.gamma);
    rc = tts_fft2d((const tts_c64*)m->E, (tts_c64*)m->E, C, Nx, Ny, 1, st);
    if (rc != TTS_OK) break;
    mc_theta_kernel<<<grid_for(NN), kT, 0, st>>>(m->H, m->E, C, NN, m->Theta);
    mc_coeff_kernel<<<1, kT, 0, st>>>(p.B, Ny, R, p.gamma_d, m->hmax, p.lf, p.sf, SF_ABAR_A, SF_ALPHA_A, m->coef);
    mc_step_kernel<<<Nx, kT, 0, st>>>(m->Theta, (size_t)Ny, 1, Ny, p.B, R, p.A, p.A0, p.gamma_d, m->coef);
    // B block on the refreshed residual
    rc = launch_image(p.A, p.B, p.gamma, m->X, Nx, Ny, R, st);
    if (rc != TTS_OK) break;
    mc_weigh_kernel<<<grid_for((size_t)C * NN), kT, 0, st>>>(m->H, m->X, C, NN, m->Zx);
    rc = tts_fft2d((const tts_c64*)m->Zx, (tts_c64*)m->Zx, C, Nx, Ny, 0, st);
    if (rc != TTS_OK) break;
    mc_residual_kernel<<<grid_for((size_t)C * NN), kT, 0, st>>>(nullptr, m->Zx, p.gamma_d, m->y, p.rows, m->rowpos,
                                                                C, R, Nx, Ny, s, m->E, nullptr);
    rc = tts_fft2d((const tts_c64*)m->E, (tts_c64*)m->E, C, Nx, Ny, 1, st);
    if (rc != TTS_OK) break;
    mc_theta_kernel<<<grid_for(NN), kT, 0, st>>>(m->H, m->E, C, NN, m->Theta);
    mc_coeff_kernel<<<1, kT, 0, st>>>(p.A, Nx, R, p.gamma_d, m->hmax, p.lf, p.sf, SF_ABAR_B, SF_ALPHA_B, m->coef);
    mc_step_kernel<<<Ny, kT, 0, st>>>(m->Theta, 1, (size_t)Ny, Nx, p.A, R, p.B, p.B0, p.gamma_d, m->coef);
  }
  if (rc != TTS_OK) return tts_fail(rc, "multi-coil frame launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  mc_end_kernel<<<1, 64, 0, st>>>(p.sc, p.sf, p.lf, p.gamma, p.gamma_d, R);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return tts_cuda_fail(e, "multi-coil frame");
  h->t += 1;
  return TTS_OK;
}
