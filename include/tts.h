/*
 * tts.h - C ABI of the GB300 online tensor-subspace tracker for undersampled dynamic
 * MRI (Mardani, Giannakis, Ugurbil: "Tracking tensor subspaces with informative random
 * sampling for real-time MR imaging").
 *
 * The tracker follows Alg. 3 of the paper with one coil (single-coil model of §IV,
 * y = [F(L_t)]_{ij} + v on Omega_t), combined with the randomized line sampler of
 * Alg. 4 in the phase-encode-line form of §VI-C, run in the order of Alg. 5
 * (S0 draw lines -> S1 ridge for gamma_t -> S2 factor updates). Each frame runs
 * mm_iters alternating majorization-minimization iterations; past surrogates are
 * forgotten with factor lambda_forget.
 *
 * Conventions used by every call:
 *   - complex data are interleaved single-precision pairs (tts_c64, 8 bytes);
 *   - the image / k-space grid is Nx x Ny, row-major; Nx is the phase-encode axis
 *     (rows, index i), Ny the readout axis (columns, index j);
 *   - the DFT is unitary with DC at index 0 and no fftshift:
 *     (F_N)_{k,n} = N^{-1/2} exp(-2 pi i k n / N), F(X) = F_Nx X F_Ny;
 *   - a sampling set is a set S of phase-encode lines, Omega = S x [Ny], passed as an
 *     Nx-byte mask (nonzero = acquired); acquired rows are passed in increasing i;
 *   - factors A (Nx x R) and B (Ny x R) are row-major (A[i*R + r]).
 *
 * Memory: the caller owns every buffer it passes; the library owns all state (factors,
 * surrogate statistics, workspaces, random-number context). Unless a call says
 * otherwise, pointers are host pointers; with the TTS_DEVICE_PTRS flag they are
 * device pointers on the handle's device. Sizes are element counts.
 *
 * Errors: every call returns TTS_OK (0) or a negative TTS_E* code; tts_last_error()
 * returns a thread-local message for the last failure. A failed call leaves the
 * tracker state unchanged. There is no CPU fallback: without a usable CUDA device,
 * tts_create* fails with TTS_ECUDA.
 *
 * Synchronisation: calls are enqueued on the handle's CUDA stream. Calls that return
 * data in host memory wait for it; calls given device pointers do not.
 */
#ifndef TTS_H
#define TTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } tts_c64;

enum {
  TTS_OK = 0,
  TTS_EINVAL = -1,      /* bad argument (size, rate, mask with no line, NULL pointer) */
  TTS_ENOMEM = -2,      /* device or host allocation failed */
  TTS_ECUDA = -3,       /* CUDA runtime error, or no usable device */
  TTS_ERANGE = -4,      /* frame index that is not the most recent frame */
  TTS_ENONFINITE = -5,  /* NaN/Inf in an input frame; the frame was not applied */
  TTS_ETIMEOUT = -6,    /* a bounded device wait ran out */
  TTS_ESTATE = -7,      /* call out of order (e.g. NULL mask before any tts_next_mask) */
  TTS_EBUSY = -8        /* engine admission refused: no free slot or no arena room */
};

#define TTS_DEVICE_PTRS 1
/* tts_push_frame only: y_rows points to a whole Nx x Ny k-space frame; only the rows
 * the mask selects are read (a scanner buffer that holds the full Cartesian grid). */
#define TTS_FULL_FRAME 2
/* tts_push_frame only, host y_rows: the frame is in page-locked host memory (cudaHostAlloc,
 * cudaHostRegister or a pinned torch tensor) that the caller leaves unchanged until the
 * frame has been processed (the next synchronising call, or an event recorded on the
 * handle's stream after the call). The kernels then read the acquired rows from it in place
 * instead of the host gathering them into staging memory first, which takes that copy off
 * the path between the line draw and the frame update; a NaN or Inf is then found on the
 * device and reported by the next synchronising call (TTS_ENONFINITE), as with
 * TTS_DEVICE_PTRS. Memory that is not page-locked gives TTS_EINVAL. Ignored with the
 * tensor-core row transform and by the multi-coil tracker, which gather as without it. */
#define TTS_HOST_PINNED 4

/* Sampling policy of tts_next_mask (S0 of Alg. 5). */
enum {
  TTS_POLICY_UNIFORM = 0,      /* all non-central lines equally likely */
  TTS_POLICY_VARDENS = 1,      /* p_i proportional to d_i^vd_alpha, d_i distance from the centre line (§VI) */
  TTS_POLICY_INFORMATIVE = 2   /* leverage scores of the current subspace (§V, §VI-C) */
};

/* Order of the factor updates inside one MM iteration. */
enum {
  TTS_UPDATE_GAUSS_SEIDEL = 0, /* gamma -> A -> B with the residual refreshed after A */
  TTS_UPDATE_JACOBI = 1        /* A and B from the same iterate (Alg. 3 (S2) in parallel) */
};

/* How a frame's MM iterations are launched. */
enum {
  TTS_LAUNCH_FUSED = 0,   /* one thread-block-cluster kernel per frame, phases separated by cluster barriers */
  TTS_LAUNCH_PHASES = 1   /* one kernel launch per phase (same arithmetic, no cluster) */
};

/* The per-frame inverse DFT of the acquired rows along the readout axis (Yt = y_S conj(F_Ny),
 * the data side of the separable form of Alg. 3): in the frame kernel by a shared-memory
 * Stockham FFT in FP32 (default), or by the tensor-core matrix product of tts_dft2d_gemm
 * before it (Ny a multiple of 32 in [32, 256]; not in an engine; device frames passed to
 * tts_push_frame then 16-byte aligned, TTS_EINVAL otherwise). */
enum {
  TTS_ROWDFT_FFT = 0,
  TTS_ROWDFT_BF16X3 = 1,   /* bf16 hi + lo split operands, FP32 accumulation */
  TTS_ROWDFT_BF16 = 2      /* plain bf16 operands (does not meet the 1e-4 image bound) */
};

typedef struct tts_handle tts_handle;

/* Precision of the ridge step (S1 of Alg. 3, closed form of §III-A). The normal equations
 * (Phi^H Phi + mu I) gamma = Phi^H y are formed from the frame's FP32 operands (the rows of the
 * transformed factors and frame) with every sum accumulated in float-float arithmetic (exact
 * products, error-free additions: about 48 significant bits, FP64 grade), and solved by an FP32
 * Gauss-Jordan inverse refined against that float-float system (FP64-grade gamma). The sums over
 * the readout axis (B^H B and Yt conj(B), |S| Ny R products) are the costly part:
 * TTS_RIDGE_FF_ALL accumulates them in float-float in every MM iteration; TTS_RIDGE_FF_LAST only
 * for the last MM iteration's system, whose solution is the frame's gamma_t (the earlier MM
 * iterations' ridge steps, which only steer the FP32 factor steps, then take those two sums in
 * FP32; every other sum, the Gram product and the solve stay float-float). */
enum {
  TTS_RIDGE_FF_ALL = 0,
  TTS_RIDGE_FF_LAST = 1
};

typedef struct {
  int Nx, Ny, R;            /* grid and PARAFAC rank; 1 <= Nx, Ny <= 512 with prime factors in {2,3,5}; 1 <= R <= 64 */
  double lambda_forget;     /* forgetting factor in (0, 1] of the surrogate statistics */
  double mu;                /* Tykhonov weight (> 0): ridge of gamma, and mu / w on the factors */
  int mm_iters;             /* MM iterations per frame, >= 1 */
  int central_lines;        /* lines {-c/2 .. c/2-1} mod Nx always acquired by tts_next_mask */
  int policy;               /* TTS_POLICY_* */
  double vd_alpha;          /* exponent of TTS_POLICY_VARDENS (the paper uses -1) */
  int with_replacement;     /* 1: draw k_lines - c times with replacement (fewer lines possible) */
  int update;               /* TTS_UPDATE_* */
  int launch;               /* TTS_LAUNCH_* */
  int cluster_ctas;         /* CTAs per frame kernel, 1..16; 0 = chosen by the library */
  uint64_t init_seed;       /* seed of the default CN(0, 1/N) initial factors */
  uint32_t stream_id;       /* enters the line-draw counter so streams draw independently */
  void* cuda_stream;        /* cudaStream_t to enqueue on; NULL = a stream the handle creates */
  int row_dft;              /* TTS_ROWDFT_*: how the acquired rows are transformed each frame */
  int kspace;               /* 0: image-domain factors (Alg. 3); 1: k-space factors (Alg. 2) */
  int ridge_precision;      /* TTS_RIDGE_*: which MM iterations accumulate their readout sums in float-float */
} tts_config;

/* Fill cfg with defaults: mm_iters 1, central_lines 8, TTS_POLICY_INFORMATIVE, vd_alpha -1,
 * without replacement, Gauss-Seidel, fused launch, cluster_ctas 0, init_seed 0,
 * stream_id 0, cuda_stream NULL, row_dft TTS_ROWDFT_FFT, kspace 0.
 *
 * kspace = 1 runs the k-space interpolation tracker of Alg. 2 (§IV-A): the factors are
 * k-space factors A1 (Nx x R), A2 (Ny x R) with x^(i,j) = <a1_i, a2_j, gamma_t>, each MM
 * iteration works on the acquired rows directly (no transform in the loop), the line
 * scores are taken on the rows of A1, and tts_image returns F^{-1}(A1 diag(gamma) A2^T)
 * (the paper's image is its magnitude). Requires TTS_ROWDFT_FFT and no coil maps; not in
 * an engine. tts_get_factors / tts_set_factors then read and write A1, A2. */
void tts_config_init(tts_config* cfg, int Nx, int Ny, int R, double lambda_forget, double mu);

/* Create a tracker (problem (P2) of §III for M = 3: factors A, B of the image-domain
 * tube subspace, temporal factor gamma_t per frame). The factors start i.i.d.
 * CN(0, 1/N) from init_seed ("initialize at random", Alg. 3); the surrogate statistics
 * start at zero. On success *out owns device memory until tts_destroy. */
int tts_create(int Nx, int Ny, int R, double lambda_forget, double mu, tts_handle** out);
int tts_create_ex(const tts_config* cfg, tts_handle** out);
void tts_destroy(tts_handle* h);

/* Replace the factors (warm start, §VI; or resuming from another tracker). A is
 * Nx x R, B is Ny x R, row-major; host pointers unless TTS_DEVICE_PTRS. The
 * surrogate statistics and frame counter are left as they are. */
int tts_set_factors(tts_handle* h, const tts_c64* A, const tts_c64* B, int flags);
/* Copy the current factors out (same layouts). Waits when given host pointers. */
int tts_get_factors(tts_handle* h, tts_c64* A, tts_c64* B, int flags);
/* Surrogate statistics: abar_A, abar_B (forgotten sums of the majorization constants
 * alpha, §III-A), w (forgotten frame count), and t (frames processed). Host scalars;
 * tts_get_stats waits for queued work. */
int tts_get_stats(tts_handle* h, double* abar_A, double* abar_B, double* w, int64_t* t);
int tts_set_stats(tts_handle* h, double abar_A, double abar_B, double w, int64_t t);
/* gamma_t of the most recent frame (R values, host): the solution of the ridge step (S1)
 * of Alg. 3 in the last MM iteration. Waits. */
int tts_get_gamma(tts_handle* h, tts_c64* gamma);
/* The same gamma_t at the accuracy the ridge step solved it to (its float-float value
 * hi + lo, summed in FP64; see TTS_RIDGE_*): 2R host doubles (re, im interleaved). Waits. */
int tts_get_gamma_fp64(tts_handle* h, double* gamma);
/* Test hook: the FP32 operands of the first MM iteration's ridge step of the most recent
 * frame (the only one when mm_iters = 1), from which the separable form builds
 * Phi^H Phi = (Ahat_S^H Ahat_S) .* (B^H B) and Phi^H y = colsum(conj(Ahat_S) .* (Yt conj(B)))
 * with B = B[t-1]: Ahat_S = (F_Nx A[t-1])[S, :] (|S| x R, row-major; with kspace, the rows S of
 * A1), Yt = y_S conj(F_Ny) (|S| x Ny; with kspace, y_S), and S (increasing row indices).
 * Host buffers of at least Nx x R, Nx x Ny and Nx elements; *nrows receives |S|. Waits. */
int tts_get_ridge_operands(tts_handle* h, tts_c64* Ahat_S, tts_c64* Yt, int* rows, int* nrows);
/* The handle's configuration as it runs: cluster_ctas is the size the library chose (or
 * the engine assigned), cuda_stream the stream its work is ordered on. */
int tts_get_config(tts_handle* h, tts_config* cfg);

/* Process frame t = (frames processed so far): y_rows holds the acquired k-space rows
 * (|S| x Ny, rows in increasing i) and line_mask the Nx-byte mask of S. line_mask NULL
 * uses the mask of the last tts_next_mask (TTS_ESTATE if there is none). Runs
 * mm_iters MM iterations of Alg. 3 (S1: ridge solve for gamma_t from the masked DFTs
 * of the rank-one images; S2: majorized updates of A then B against the forgotten
 * surrogate statistics). With host pointers the frame is checked for NaN/Inf first
 * (TTS_ENONFINITE, nothing applied); with TTS_DEVICE_PTRS the check runs on the
 * device, the frame is skipped and tts_synchronize reports TTS_ENONFINITE.
 * A host mask that selects no line is refused (TTS_EINVAL); a device mask is not read on
 * the host, and one that selects no line runs the frame without data: gamma_t = 0, a zero
 * image, and both factors scaled by lf abar / (lf abar + rho), the minimiser of the
 * forgotten surrogates plus the factor penalty.
 * With TTS_FULL_FRAME, y_rows is a full Nx x Ny frame of which only the acquired rows
 * are read. Host rows are gathered (and checked) into pinned memory of the handle, which the
 * kernels read in place (mapped) or which is copied in one transfer, so y_rows may be
 * pageable and is free again when the call returns; with TTS_HOST_PINNED the kernels read
 * page-locked caller memory in place instead (see there). Asynchronous with TTS_DEVICE_PTRS
 * (the buffers must stay valid until the stream passes this work). */
int tts_push_frame(tts_handle* h, const tts_c64* y_rows, const uint8_t* line_mask, int flags);

/* Reconstructed frame X_t = A[t] diag(gamma_t) B[t]^T (Nx x Ny, row-major; the
 * image-domain counterpart of the interpolated frame of §IV-A). Only the
 * most recent frame is available: any other t gives TTS_ERANGE. With a host pointer
 * the call waits for the image. */
int tts_image(tts_handle* h, int64_t t, tts_c64* out, int flags);

/* Several receive coils (Alg. 3 with C coils, §IV-B tomographic parallel MRI): coil c sees
 * y_c = P_Omega F(H_c .* L_t) + v with known sensitivity H_c. maps: C x Nx x Ny complex64
 * (host, or device with TTS_DEVICE_PTRS), copied; C in 1..TTS_MAX_COILS; NULL or C = 0
 * returns the handle to the single-coil tracker. Afterwards tts_push_frame takes the
 * coils' acquired rows stacked, C x |S| x Ny (or C x Nx x Ny with TTS_FULL_FRAME), and
 * each MM iteration transforms the C R sensitivity-weighted rank-one images explicitly
 * (batched 2D DFTs): Phi stacks the coils' masked DFTs, Theta = sum_c conj(H_c) .*
 * F^{-1}(Xi_c), and the majoriser weights carry h_max = max_ij sum_c |H_c[i,j]|^2.
 * Requires Gauss-Seidel updates, the FFT row transform and R (Ny + 1) <= 16384; not for
 * engine streams. tts_image and tts_next_mask are unchanged; tts_save does not store the
 * maps. A multi-coil frame waits for the line count and the input check on the host. */
#define TTS_MAX_COILS 64
int tts_set_coil_maps(tts_handle* h, const tts_c64* maps, int C, int flags);

/* S0 of Alg. 5 for the next frame: draw its phase-encode lines under the handle's
 * policy (informative: scores of §V-B marginalised over readout as in §VI-C,
 * s_i = (Ny ||abar_i||^2 + R) / (R (Nx + Ny)) with abar the rows of the
 * column-normalised F_Nx A). k_lines = max(central_lines, round(rate * Nx)); the
 * central lines are always kept. The draws use Philox4x32-10 keyed by seed with the
 * counter built from (frame index, stream_id). Writes Nx bytes to line_mask_out
 * (host, or device with TTS_DEVICE_PTRS) and keeps the mask for tts_push_frame(NULL).
 * rate must lie in (0, 1]. A host line_mask_out is filled before the call returns: the call
 * waits for the draw itself (a completion word the kernel sets in mapped host memory), not for
 * the whole stream; errors of earlier work surface at the next synchronising call. A host
 * line_mask_out while the handle's stream is being captured is refused (TTS_ESTATE). */
int tts_next_mask(tts_handle* h, double rate, uint64_t seed, uint8_t* line_mask_out, int flags);

/* The line probabilities p (Nx doubles) that tts_next_mask would draw from now: the
 * marginalised scores of §V-B / §VI-C under the informative policy, the fixed policy's
 * weights otherwise. Host p waits; device p (TTS_DEVICE_PTRS) is asynchronous. */
int tts_line_probs(tts_handle* h, double* p, int flags);

/* The line draw of tts_next_mask (Alg. 4, with or without replacement as in §V-B) on
 * given probabilities p (Nx doubles, sum 1): the
 * central lines are kept; the other lines carry integer weights q_i = floor(p_i 2^52)
 * with inclusive prefix sums Q; draw d takes the Philox4x32-10 block at counter
 * (d, 1, ctr_lo, ctr_hi) under key (seed_lo, seed_hi), u = word0 | word1 << 32,
 * x = floor(u Q_total / 2^64), and selects the first line with Q > x. Without
 * replacement duplicates are rejected until k_lines lines are held or
 * 64 (k_lines - central) draws are spent, then the remaining lines are taken in
 * decreasing q (lower index first). Runs on the current device, synchronously. Pointers
 * are host pointers unless TTS_DEVICE_PTRS (then p and out are device pointers and the
 * call is asynchronous on the default stream). */
int tts_sample_lines_from_probs(const double* p, int Nx, int k_lines, int central, uint64_t seed,
                                uint64_t ctr, int with_replacement, uint8_t* out, int flags);

/* Checkpoint: the full tracker state (configuration, factors, gamma, the forgotten
 * surrogate statistics of §III-A, frame counter, last mask) as an opaque host byte string. With buf NULL
 * *len receives the size needed. tts_load restores it into a handle created with the
 * same Nx, Ny, R. */
int tts_save(tts_handle* h, void* buf, size_t* len);
int tts_load(tts_handle* h, const void* buf, size_t len);

/* Wait for the handle's queued work; returns a deferred device status once, then clears
 * it: TTS_ETIMEOUT if a bounded wait of the tensor-core row transform ran out (the frame's
 * results are invalid), TTS_ENONFINITE for a skipped frame. */
int tts_synchronize(tts_handle* h);

/* Kernel launches one tts_push_frame enqueues with the handle's settings. */
int tts_launches_per_frame(tts_handle* h);

/* The ridge step of (S1) on a given system: solves G gamma = h to FP64 accuracy with the
 * solver the frame kernel uses (§III-A: gamma = (Phi^H Phi + mu I)^{-1} Phi^H y, here
 * with G = Phi^H Phi + mu I supplied): an FP32 Gauss-Jordan inverse followed by
 * iterative refinement whose residuals are formed in float-float arithmetic. G is R x R complex128 (interleaved re, im),
 * row-major, Hermitian positive definite; only its lower triangle is read. h and gamma
 * hold R complex128 values. Host pointers; runs on the current device, synchronously. */
int tts_ridge_solve(const double* G, const double* h, int R, double* gamma);

/* Batched unitary 2D DFT (forward: F_Nx X F_Ny; inverse: conj(F_Nx) X conj(F_Ny); the
 * 2D transform in the matrix form of §IV) of `batch` row-major Nx x Ny complex images, device pointers, on `cuda_stream`
 * (NULL = default stream). in == out is allowed; any float2-aligned pointers. Nx, Ny in
 * [1, 512] with prime factors in {2, 3, 5}. Asynchronous. */
int tts_fft2d(const tts_c64* in, tts_c64* out, int batch, int Nx, int Ny, int inverse, void* cuda_stream);

/* The same unitary 2D DFT as dense complex matrix products on the tensor cores (tcgen05,
 * BF16 operands, FP32 accumulation): the paper writes the 2D transform as F_Nx X F_Ny
 * (§IV); here each of the two products multiplies the interleaved real rows by the real
 * 2N x 2N embedding of the DFT matrix. precision TTS_DFT_BF16X3 splits both operands into
 * bf16 hi + lo parts and accumulates hi*hi + hi*lo + lo*hi (relative error ~1e-5, within
 * the 1e-4 image bound); TTS_DFT_BF16 uses hi*hi only (~4e-3: plain BF16 does not meet the
 * bound). in, out, tmp: device, batch x Nx x Ny complex64, row-major; tmp (same size) holds
 * the intermediate transposes and must not alias in or out (in == out is allowed); all
 * three 16-byte aligned (TTS_EINVAL otherwise). Nx, Ny multiples of 32 in [32, 256]. dev_status: NULL, or a device int the kernel sets to 1 if
 * one of its bounded waits ran out (the results are then invalid). Asynchronous on
 * cuda_stream (NULL = default stream). */
#define TTS_DFT_BF16X3 0
#define TTS_DFT_BF16 1
int tts_dft2d_gemm(const tts_c64* in, tts_c64* out, tts_c64* tmp, int batch, int Nx, int Ny, int inverse,
                   int precision, int* dev_status, void* cuda_stream);

/* ---- Frame update without allocation ------------------------------------------------
 * The paper has no counterpart of this call; it serves callers that cannot allocate
 * device memory while they run: code whose device memory is handed out by an allocator
 * it does not control, real-time loops that were sized once and must not grow, and code
 * that cannot afford the implicit device synchronisation of cudaMalloc / cudaFree.
 *
 * It runs the same frame update as tts_push_frame on state the caller holds in device
 * memory. Every temporary lives in one fixed array of TTS_NOALLOC_SCRATCH_BYTES in
 * device memory that the library declares at file scope; every GPU that loads the
 * library holds that array until the process exits. The call allocates nothing
 * (no cudaMalloc, no cudaFree, no allocating library routine). Limits: Nx, Ny <= 256
 * with prime factors in {2,3,5}, R <= 32; larger problems return TTS_EINVAL.
 *
 * All calls on a device share the one array and it keeps the last call's contents; the
 * call re-initialises what must start at zero. Calls whose work overlaps on the GPU
 * (several host threads, or several streams) race on the array and give wrong results:
 * serialise them. The first call on a device looks up the array's device address (with
 * that device current); make that first call before any stream capture. Every call fills
 * the twiddle tables of its sizes and clears the status words in the array with one small
 * kernel of its own before the frame kernel; nothing is copied from host memory. The call
 * is asynchronous on cuda_stream (NULL = the legacy default stream). A frame with a
 * non-finite input sample is skipped on the device: A, B, gamma and stats are left as
 * they were, so stats[3] (frames processed) not advancing is how the caller sees it. */
#define TTS_NOALLOC_MAX_N 256
#define TTS_NOALLOC_MAX_R 32
#define TTS_NOALLOC_SCRATCH_BYTES (4u << 20)

typedef struct {
  int Nx, Ny, R;
  double lambda_forget, mu;
  int mm_iters;
  int update;               /* TTS_UPDATE_* */
  tts_c64* A;               /* device, Nx x R row-major, updated in place */
  tts_c64* B;               /* device, Ny x R row-major, updated in place */
  double* stats;            /* device, 4 doubles updated in place: w, abar_A, abar_B, frames
                               processed; all zero before the first frame */
  tts_c64* gamma;           /* device, R values written: gamma_t of this frame */
  const tts_c64* y_rows;    /* device: acquired rows (|S| x Ny), or the whole Nx x Ny
                               frame with TTS_FULL_FRAME */
  const uint8_t* line_mask; /* device, Nx bytes */
  int flags;                /* 0 or TTS_FULL_FRAME */
} tts_frame_args;

int tts_push_frame_noalloc(const tts_frame_args* args, void* cuda_stream);

/* ---- Many streams on one GPU: the batching and serving engine ------------------------
 * The paper tracks one cine stream at a time (Alg. 3, Alg. 5); it has no counterpart of
 * this part. An engine keeps many independent trackers (streams of any Nx, Ny, R, K,
 * lambda_forget, mu, policy and rate) resident on one GPU and advances any subset of
 * them by one frame per call, with all their work in three kernel launches (see
 * tts_engine_step). Each stream's results equal those of a handle with the same
 * tts_config and cluster_ctas run alone: the batch changes where a frame runs, not what
 * it computes.
 *
 * Memory: tts_engine_create reserves one device arena of arena_bytes; each admitted
 * stream takes tts_stream_footprint bytes of it until released. The engine owns the
 * arena, the slots' handles, a device parameter block and two pinned host copies of it.
 * All engine work is ordered on the engine's stream; calls returning host data wait
 * for it. An engine is not thread-safe: serialise calls on one engine. */
#define TTS_ENGINE_GRAPH 1          /* tts_engine_create: replay each step as a CUDA graph */
#define TTS_ENGINE_MAX_SLOTS 4096

typedef struct tts_engine tts_engine;

typedef struct {
  size_t arena_bytes;         /* size of the device arena */
  size_t arena_used;          /* bytes held by admitted streams */
  size_t arena_largest_free;  /* largest stream footprint that admission can place now */
  int active;                 /* admitted streams */
  int max_slots;
  int cluster_ctas;           /* preferred CTAs per frame (one cluster) */
  int groups;                 /* cluster sizes in use: one persistent frame launch each */
  int resident_clusters;      /* clusters those launches can keep on the GPU at once, summed */
  int64_t steps;              /* tts_engine_step calls that launched work */
} tts_engine_stats;

/* Device bytes a stream with this configuration holds in an engine arena (the same
 * workspace a handle allocates) when it runs on clusters of cfg->cluster_ctas CTAs
 * (0 = 4, the engine default); TTS_EINVAL if its layout does not fit that size. */
int tts_stream_footprint(const tts_config* cfg, size_t* bytes);

/* Create an engine on the current device. arena_bytes >= 4096; max_slots in
 * 1..TTS_ENGINE_MAX_SLOTS (at most that many streams at once); cluster_ctas in
 * {0 (= 4), 1, 2, 4, 8, 16}: the preferred number of CTAs of the cluster that runs one
 * frame (a stream whose layout does not fit takes the next larger size that fits;
 * tts_get_config shows the size a stream got); flags 0 or TTS_ENGINE_GRAPH; cuda_stream
 * NULL = a stream the engine creates. TTS_ENOMEM if the arena or the parameter block
 * cannot be allocated. */
int tts_engine_create(size_t arena_bytes, int max_slots, int cluster_ctas, int flags, void* cuda_stream,
                      tts_engine** out);
/* Waits for the engine's work, then frees everything it owns, admitted streams included. */
void tts_engine_destroy(tts_engine* e);

/* Admission: create a tracker for cfg in a free slot whose footprint fits in the arena
 * (first fit). cfg->cluster_ctas is replaced by the engine's preferred size (or the next
 * larger that fits the stream), cfg->launch and cfg->cuda_stream by the engine's; row_dft
 * must be TTS_ROWDFT_FFT (TTS_EINVAL otherwise). On success *slot is the stream's slot (0..max_slots-1). TTS_EBUSY when every
 * slot is taken or no free arena block is large enough; TTS_EINVAL for a bad cfg. Does
 * not wait for steps in flight. */
int tts_engine_admit(tts_engine* e, const tts_config* cfg, int* slot);
/* Waits for the engine's work, then frees the slot and returns its arena block. */
int tts_engine_release(tts_engine* e, int slot);
/* The tracker of a slot (owned by the engine, valid until release): tts_get_factors,
 * tts_get_stats, tts_set_factors, tts_save, tts_load ... apply to it on the engine's stream. */
int tts_engine_handle(tts_engine* e, int slot, tts_handle** h);

/* One frame for each of n distinct slots (0 <= n <= max_slots), then the image and the
 * next frame's lines of each:
 *   y_rows[k]     frame of slots[k], as for tts_push_frame (|S| x Ny acquired rows, or
 *                 Nx x Ny with TTS_FULL_FRAME), host or device per TTS_DEVICE_PTRS;
 *   line_masks    NULL, or n masks (each NULL = the mask the engine drew for the slot);
 *   rates[k]      rate in (0, 1] of the draw for the slot's next frame;
 *   seeds[k]      key of that draw.
 * For every listed slot this equals tts_push_frame, tts_image (into the engine's image
 * buffer of the slot) and tts_next_mask(rate, seed) on the slot's handle. Host frames
 * are checked and copied as tts_push_frame does, except a full host frame with a NULL
 * mask, which is copied whole and checked on the device. If any frame is refused
 * (TTS_EINVAL, TTS_ESTATE, TTS_ENONFINITE) no slot is advanced. Asynchronous; it waits
 * only for the step before last, whose host parameter copy it reuses. */
int tts_engine_step(tts_engine* e, int n, const int* slots, const tts_c64* const* y_rows,
                    const uint8_t* const* line_masks, const double* rates, const uint64_t* seeds, int flags);
/* The image (Nx x Ny) the last step computed for the slot; TTS_ERANGE before its first
 * frame. Host out waits for the engine's stream; device out is an async copy. */
int tts_engine_image(tts_engine* e, int slot, tts_c64* out, int flags);
/* The mask (Nx bytes) the last step drew for the slot's next frame; TTS_ESTATE if none. */
int tts_engine_mask(tts_engine* e, int slot, uint8_t* out, int flags);
/* Waits for the engine's stream; TTS_ENONFINITE (once) if any slot skipped a frame. */
int tts_engine_synchronize(tts_engine* e);
int tts_engine_info(tts_engine* e, tts_engine_stats* stats);

/* Autotuner of the engine's cluster size for a mix of streams: for each candidate C in
 * {1, 2, 4, 8, 16} that has a layout for every cfgs[k] (n configurations), builds a
 * temporary engine with those streams, runs two untimed steps (the first fully sampled,
 * then drawn masks) and `steps` timed steps on synthetic CN(0, 1) frames, and returns the
 * C with the least time per step in *best_C. step_ms (optional, 5 doubles) receives the
 * time per step of each candidate in that order, -1 where a candidate does not fit.
 * Fewer, larger clusters give each frame lower latency; more, smaller clusters keep more
 * frames on the GPU at once; which wins depends on the mix (streams that do not fit a
 * candidate run at their next larger size that fits, as in an engine). Synchronous; allocates the
 * temporary engines and frames on the current device and frees them before returning. */
int tts_engine_autotune(const tts_config* cfgs, int n, int steps, int* best_C, double* step_ms);

/* Autotuner of tts_fft2d's launch shape for square N x N images of the band-task sizes
 * (64, 96, 128, 144, 160, 192, 256, 288, 320, 384): times, on batch zero-filled images in
 * buffers of its own, the persistent launch at the CTAs per SM that fit and up to two fewer,
 * each with the row-ahead lag between an image's row and column tasks scaled by 0.5, 1, 1.5, 2
 * and 3 (one untimed launch, then the best of `reps`), and records the fastest shape for later
 * tts_fft2d calls of that N and direction on the current device (the library's default shape
 * until then). Outputs (each may be NULL): the best time per call in ms, its CTAs per SM and
 * lag scale. Synchronous; allocates and frees its buffers (2 x batch x N^2 complex64). */
int tts_fft2d_autotune(int N, int batch, int inverse, int reps, double* best_ms, int* per_sm, double* lag);

/* ---- Test hooks for the failure detection of the bounded device waits ----------------
 * No counterpart in the paper. Kernels that wait on other threads' arrivals (the square
 * band-task FFT's column tasks on an image's row tasks; the tensor-core DFT's MMA issuer and
 * producers on each other's mbarrier arrivals) give every wait a limit, after which they
 * record an error status and return; these hooks withhold one awaited arrival so that a test
 * can run such a wait out without faulting or hanging the GPU.
 *
 * tts_test_withheld_wait: kind 0 runs tts_fft2d's square band-task kernel (batch images of
 * N x N, N one of its sizes 64..384, forward) with the row tasks of image `index` publishing
 * nothing; kind 1 runs tts_dft2d_gemm (BF16 hi + lo, N x N, N a multiple of 32 in [32, 256];
 * tmp as there) with the bulk copy and producer arrival of K' chunk `index` (< 2N / 16) of the
 * first pass withheld. Every wait of the launch lasts at most wait_cycles SM clocks. The waits
 * for the withheld arrival run out, the kernel sets *dev_status (a device int the caller
 * zeroes first) to 1, and the outputs are invalid; the next ordinary call is unaffected.
 * Device buffers; asynchronous on cuda_stream. */
int tts_test_withheld_wait(int kind, const tts_c64* in, tts_c64* out, tts_c64* tmp, int batch, int N, int index,
                           long long wait_cycles, int* dev_status, void* cuda_stream);
/* The next tts_push_frame of a handle whose row transform runs on the tensor cores (row_dft
 * != TTS_ROWDFT_FFT) withholds K' chunk `chunk` (< 2 Ny / 16) of that transform, with every
 * wait limited to wait_cycles SM clocks: the transform gives up, the frame is skipped (the
 * factors, statistics and gamma keep their values) and tts_synchronize reports TTS_ETIMEOUT.
 * Later frames run as usual. */
int tts_test_withhold_row_transform(tts_handle* h, int chunk, long long wait_cycles);

/* Calibration (no counterpart in the paper): the device's FP32 fused multiply-add rate,
 * the denominator of the frame kernel's ALU roofline. A kernel fills every SM (the largest
 * number of 256-thread CTAs that fit) and each thread runs eight independent chains of
 * 16 x iters FMAs; one untimed launch, then `reps` launches timed with CUDA events on the
 * legacy default stream. *tflops = 2 x FMAs / best time (TFLOP/s), *ms = best time (NULL
 * allowed). Synchronous; no allocation. */
int tts_fp32_fma_rate(int iters, int reps, double* tflops, double* ms);

const char* tts_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TTS_H */
