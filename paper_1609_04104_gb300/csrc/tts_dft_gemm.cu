// The unitary 2D DFT as dense complex matrix products on the 5th-generation tensor cores
// (tcgen05), the "DFT as F_l X F_r" form of the paper's 2D transform (§IV: F(X) =
// F_Nx X F_Ny), in BF16 with FP32 accumulation, optionally with hi + lo split operands.
//
// One pass multiplies every length-N row of a batch by the DFT matrix and writes the
// result transposed per image; two passes (rows, then the rows of the transpose) give
// F_Nx X F_Ny. A complex row x (N values) times W (N x N) is the real product of the
// interleaved row [Re x0, Im x0, Re x1, ...] (K' = 2N) with the 2N x 2N real embedding
//   Bt[2j][2k] = Re W_kj, Bt[2j][2k+1] = -Im W_kj, Bt[2j+1][2k] = Im W_kj, Bt[2j+1][2k+1] = Re W_kj,
// whose output row is again interleaved (N' = 2N). Split precision writes each operand as
// hi + lo with hi = bf16(v), lo = bf16(v - hi) and accumulates hi*hi + hi*lo + lo*hi in FP32
// (the lo*lo term, ~2^-16 relative, is dropped); plain precision uses hi*hi only.
//
// Kernel: one CTA of 8 warps per 128 rows, warp-specialised on mbarriers. K' is consumed in
// chunks of 16 (one MMA K step) through four shared-memory stages:
//   - producer warp w (w < 4) fills stage w with chunks w, w + 4, ...: it loads the chunk's
//     fp32 rows (16 float4 per lane at once, so four chunks are in flight), splits them to
//     bf16 and stores them in the canonical K-major no-swizzle layout (8 x 16-byte core
//     matrices, 128 B each); its lane 0 bulk-copies the DFT-matrix chunk (pre-arranged in
//     that layout in global memory) on the stage's "full" barrier; the warp then arrives;
//   - lane 0 of warp 4 waits for a full stage, issues the tcgen05.mma instructions (M = 128,
//     N' up to 256 per accumulator, two accumulators for N' = 2N > 256) into tensor memory
//     and commits them to the stage's "empty" barrier, which lets the producer refill it;
//   - after the last commit all warps read the accumulators with tcgen05.ld (warp w owns
//     TMEM lanes 32 (w mod 4)..) and write complex outputs transposed, 256 contiguous bytes
//     per warp and output column.
// Every mbarrier wait is bounded; on timeout the CTA records an error and every role stops.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tts_async.cuh"
#include "tts_internal.cuh"

namespace {

constexpr int kRows = 128;     // rows per CTA (UMMA M)
constexpr int kKC = 16;        // K' chunk (bf16 elements) per stage: one MMA K step
constexpr int kThreads = 256;   // 8 warps: warp w and w + 4 share TMEM lanes 32 (w % 4).. in the epilogue
constexpr int kStages = 4;     // one per producer warp
constexpr int kProducers = 4;  // warps 0..3 load and split the A rows; warp w fills stage w
constexpr int kIssuer = 4;     // lane 0 of warp 4 issues the MMAs

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte offset
// (between core matrices along K) and stride byte offset (between 8-row groups), all >> 4;
// bit 46 = descriptor version 1; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N and M.
__host__ __device__ __forceinline__ uint32_t instr_desc(int n, int m) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct GemmArgs {
  const float2* x;        // rows of length N (complex), M rows in all
  float2* out;            // transposed per image: out[b][j][i]
  const uint4* bhi;       // DFT embedding, pre-arranged chunks (see dft_embedding)
  const uint4* blo;
  int M;                  // rows in all (batch * rows per image)
  int rows;               // rows per image
  int N;                  // row length (complex), K' = N' = 2N
  int nh;                 // accumulators (1, or 2 when 2N > 256)
  int split;              // 1: hi*hi + hi*lo + lo*hi; 0: hi*hi
  int* err;               // set to 1 when a wait ran out
  long long limit;        // SM clocks a bounded wait lasts (TTS_WAIT_LIMIT)
  int withhold;           // test hook: K' chunk whose copy and arrival are withheld (-1: none)
  // row mode (the acquired rows of one k-space frame): when mask is set, the rows are the
  // lines i with mask[i] != 0 (M = their number, one row per "image", so the output is
  // row-major); with full_frame, row m is x row S[m], else x row m
  const uint8_t* mask;
  int mask_n;
  int full_frame;
};

// Shared memory of one CTA (bytes): per stage A_hi, A_lo (128 x 16 bf16 = 4 KB each) and
// B_hi, B_lo (N' x 16 bf16 each); then the mbarriers and the TMEM address slot.
__host__ __device__ inline int a_bytes() { return kRows * kKC * 2; }
__host__ __device__ inline int b_bytes(int N) { return 2 * N * kKC * 2; }
__host__ __device__ inline int stage_bytes(int N) { return 2 * a_bytes() + 2 * b_bytes(N); }

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) dft_gemm_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = g.N, Np = 2 * N, NT = Np / g.nh;
  const int SB = stage_bytes(N);
  uint64_t* bars = (uint64_t*)(smem + kStages * SB);   // full[S], empty[S], done
  uint32_t* slot = (uint32_t*)(bars + 2 * kStages + 2);
  __shared__ int abort_flag;
  __shared__ int srows[TTS_MAX_N];
  __shared__ int scount;
  volatile int* abort_v = &abort_flag;
  int M = g.M;
  if (g.mask) {
    // compact the line mask into the increasing list S (warp 0)
    if (warp == 0) {
      int count = 0;
      for (int base = 0; base < g.mask_n; base += 32) {
        const int i = base + lane;
        const bool on = i < g.mask_n && g.mask[i] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) srows[count + __popc(bal & ((1u << lane) - 1u))] = i;
        count += __popc(bal);
      }
      if (lane == 0) scount = count;
    }
    __syncthreads();
    M = scount;
    if ((int)blockIdx.x * kRows >= M) return;   // uniform: the whole CTA has no rows
  }
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kStages]), done = smem_u32(&bars[2 * kStages]);
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 2);    // the producer warp, and the B copy's arrival with its bytes
      mbar_init(empty0 + 8 * s, 1);   // the MMA commit
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  const uint32_t ncols = g.nh == 1 ? 256u : 512u;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;

  const int m0 = blockIdx.x * kRows;
  const int nK = Np / kKC;
  const uint32_t idesc = instr_desc(NT, kRows);
  const uint32_t bchunk = (uint32_t)b_bytes(N);   // bytes of one K' chunk of the embedding (all N')
  if (warp < kProducers) {
    // producer warp w: chunks w, w + 4, ... into stage w (128 rows x 16 floats; a lane
    // loads 16 float4 at once, so four chunks are in flight across the producer warps)
    const int s = warp;
    unsigned char* st = smem + s * SB;
    unsigned char* ahi = st;
    unsigned char* alo = st + a_bytes();
    unsigned char* bhi = st + 2 * a_bytes();
    unsigned char* blo = bhi + b_bytes(N);
    int last = -1;   // the last use of the stage whose copy was issued
    for (int kc = s, use = 0; kc < nK; kc += kStages, ++use) {
      if (use > 0 && (*abort_v || !mbar_wait(empty0 + 8 * s, (use - 1) & 1, g.limit))) {
        abort_flag = 1;
        break;
      }
      // test hook: this chunk's arrivals never come, so the wait for it runs out
      if (kc == g.withhold) break;
      last = use;
      if (lane == 0) {
        mbar_expect_tx(full0 + 8 * s, g.split ? 2 * bchunk : bchunk);
        bulk_g2s(smem_u32(bhi), (const char*)g.bhi + (size_t)kc * bchunk, bchunk, full0 + 8 * s);
        if (g.split) bulk_g2s(smem_u32(blo), (const char*)g.blo + (size_t)kc * bchunk, bchunk, full0 + 8 * s);
      }
      float4 v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = lane + 32 * u;
        const int r = idx >> 2, q = idx & 3;
        const int m = m0 + r;
        const int src = (g.mask && g.full_frame && m < M) ? srows[m] : m;
        v[u] = m < M ? *(const float4*)((const float*)(g.x + (size_t)src * N) + kc * kKC + 4 * q)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = lane + 32 * u;
        const int r = idx >> 2, q = idx & 3;
        // byte offset: 8-row group (r / 8) x 256, core matrix along K (q / 2) x 128, row (r % 8) x 16, half (q % 2) x 8
        const int off = (r >> 3) * 256 + (q >> 1) * 128 + (r & 7) * 16 + (q & 1) * 8;
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v[u].x, v[u].y), h23 = __floats2bfloat162_rn(v[u].z, v[u].w);
        uint2 hv;
        hv.x = *(const uint32_t*)&h01;
        hv.y = *(const uint32_t*)&h23;
        *(uint2*)(ahi + off) = hv;
        if (g.split) {
          const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
          const __nv_bfloat162 l01 = __floats2bfloat162_rn(v[u].x - f01.x, v[u].y - f01.y);
          const __nv_bfloat162 l23 = __floats2bfloat162_rn(v[u].z - f23.x, v[u].w - f23.y);
          uint2 lv;
          lv.x = *(const uint32_t*)&l01;
          lv.y = *(const uint32_t*)&l23;
          *(uint2*)(alo + off) = lv;
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(full0 + 8 * s);
    }
    // the stage's last copy has landed before the CTA moves on (already so unless a wait ran
    // out: that phase then completes with the copy, the warp's own arrival being in)
    if (lane == 0 && last >= 0 && !mbar_wait(full0 + 8 * s, last & 1, g.limit)) abort_flag = 1;
  } else if (warp == kIssuer) {
    if (lane == 0) {
      for (int kc = 0; kc < nK; ++kc) {
        const int s = kc % kStages, use = kc / kStages;
        if (*abort_v || !mbar_wait(full0 + 8 * s, use & 1, g.limit)) {
          abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* st = smem + s * SB;
        const uint32_t a_hi = smem_u32(st), a_lo = a_hi + a_bytes();
        const uint32_t b_hi = a_hi + 2 * a_bytes(), b_lo = b_hi + b_bytes(N);
        const uint64_t dah = smem_desc(a_hi, 128, 256);
        const uint64_t dal = smem_desc(a_lo, 128, 256);
        for (int h = 0; h < g.nh; ++h) {
          const uint32_t boff = h * NT * kKC * 2;
          const uint64_t dbh = smem_desc(b_hi + boff, 128, 256);
          const uint32_t d = tmem + h * 256;
          umma(d, dah, dbh, idesc, kc != 0);
          if (g.split) {
            const uint64_t dbl = smem_desc(b_lo + boff, 128, 256);
            umma(d, dah, dbl, idesc, 1);
            umma(d, dal, dbh, idesc, 1);
          }
        }
        umma_commit(empty0 + 8 * s);
      }
      umma_commit(done);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
  }
  const bool fin = mbar_wait(done, 0, g.limit);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag || !fin) {
    if (tid == 0) atomicExch(g.err, 1);
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4).. (rows), 32 fp32 columns per load; the
    // warps w and w + 4 take alternate column blocks
    const int lq = warp & 3, wg = warp >> 2;
    const int r = lq * 32 + lane;
    const int m = m0 + r;
    const int b = m / g.rows, i = m - b * g.rows;
    float2* ob = g.out + (size_t)b * N * g.rows;
    for (int h = 0; h < g.nh; ++h) {
      for (int c0 = 32 * wg; c0 < NT; c0 += 64) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(lq * 32) << 16) + h * 256 + c0, v);
        if (m < M) {
          const int j0 = (h * NT + c0) >> 1;
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            ob[(size_t)(j0 + jj) * g.rows + i] = make_float2(__uint_as_float(v[2 * jj]), __uint_as_float(v[2 * jj + 1]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---- DFT-matrix embeddings, per (N, direction), cached on each device ---------------------
struct Embedding {
  int dev, N, inverse;
  uint4* hi;
  uint4* lo;
};
std::mutex g_mu;
std::vector<Embedding> g_emb;

uint16_t bf16_bits(float f) {
  // round to nearest even (finite inputs)
  uint32_t u;
  memcpy(&u, &f, 4);
  const uint32_t r = ((u >> 16) & 1u) + 0x7FFFu;
  return (uint16_t)((u + r) >> 16);
}
float bf16_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// The real 2N x 2N embedding of W = N^{-1/2} exp(-+2 pi i jk / N), as rows c (output,
// N' = 2N) and columns k' (input, K' = 2N), laid out chunk by chunk (16 columns k') in the
// canonical K-major no-swizzle layout: byte (c / 8) * 256 + (k'_in_chunk / 8) * 128 +
// (c % 8) * 16 + (k'_in_chunk % 8) * 2 within the chunk.
int embedding(int N, int inverse, const uint4** hi, const uint4** lo) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& e : g_emb)
    if (e.dev == dev && e.N == N && e.inverse == inverse) {
      *hi = e.hi;
      *lo = e.lo;
      return TTS_OK;
    }
  const int Np = 2 * N, nK = Np / kKC;
  const size_t chunk = (size_t)Np * kKC;   // bf16 elements per chunk
  std::vector<uint16_t> H(chunk * nK), L(chunk * nK);
  const double sc = 1.0 / sqrt((double)N), sgn = inverse ? 1.0 : -1.0;
  for (int c = 0; c < Np; ++c) {
    const int j = c >> 1;
    for (int kp = 0; kp < Np; ++kp) {
      const int k = kp >> 1;
      const double ang = sgn * 2.0 * M_PI * (double)(((long long)j * k) % N) / (double)N;
      const double wr = sc * cos(ang), wi = sc * sin(ang);
      double v;
      if ((c & 1) == 0) v = (kp & 1) == 0 ? wr : -wi;
      else v = (kp & 1) == 0 ? wi : wr;
      const float f = (float)v;
      const uint16_t h = bf16_bits(f);
      const uint16_t l = bf16_bits(f - bf16_float(h));
      const int kc = kp / kKC, kk = kp % kKC;
      const size_t idx = (size_t)kc * chunk + (size_t)(c >> 3) * (8 * kKC) + (kk >> 3) * 64 + (c & 7) * 8 + (kk & 7);
      H[idx] = h;
      L[idx] = l;
    }
  }
  uint4* dh = nullptr;
  uint4* dl = nullptr;
  const size_t bytes = H.size() * 2;
  if (cudaMalloc(&dh, bytes) != cudaSuccess) return TTS_ENOMEM;
  if (cudaMalloc(&dl, bytes) != cudaSuccess) {
    cudaFree(dh);
    return TTS_ENOMEM;
  }
  if (cudaMemcpy(dh, H.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dl, L.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dh);
    cudaFree(dl);
    return TTS_ECUDA;
  }
  g_emb.push_back({dev, N, inverse, dh, dl});
  *hi = dh;
  *lo = dl;
  return TTS_OK;
}

int launch_args(GemmArgs& a, int inverse, int grid, cudaStream_t st) {
  const uint4 *hi = nullptr, *lo = nullptr;
  const int rc = embedding(a.N, inverse, &hi, &lo);
  if (rc != TTS_OK) return rc;
  a.bhi = hi;
  a.blo = lo;
  a.nh = 2 * a.N > 256 ? 2 : 1;
  const int smem = std::max(kStages * stage_bytes(a.N) + 128, a.nh == 1 ? 80 * 1024 : 120 * 1024);
  if (cudaFuncSetAttribute(dft_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return TTS_ECUDA;
  dft_gemm_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

int launch_pass(const float2* x, float2* out, int batch, int rows, int N, int inverse, int split, int* err,
                cudaStream_t st, int withhold = -1, long long limit = TTS_WAIT_LIMIT) {
  const uint4 *hi = nullptr, *lo = nullptr;
  int rc = embedding(N, inverse, &hi, &lo);
  if (rc != TTS_OK) return rc;
  GemmArgs a;
  a.x = x;
  a.out = out;
  a.bhi = hi;
  a.blo = lo;
  a.M = batch * rows;
  a.rows = rows;
  a.N = N;
  a.nh = 2 * N > 256 ? 2 : 1;
  a.split = split;
  a.err = err;
  a.mask = nullptr;
  a.mask_n = 0;
  a.full_frame = 0;
  a.limit = limit;
  a.withhold = withhold;
  // TMEM holds 512 columns per SM: ask for enough shared memory that the CTAs resident on
  // one SM never need more (two CTAs of 256 columns, or one of 512), so an allocation never
  // waits on a CTA that cannot finish
  const int smem = std::max(kStages * stage_bytes(N) + 128, a.nh == 1 ? 80 * 1024 : 120 * 1024);
  if (cudaFuncSetAttribute(dft_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return TTS_ECUDA;
  const int grid = (a.M + kRows - 1) / kRows;
  dft_gemm_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? TTS_OK : TTS_ECUDA;
}

}  // namespace

// Sizes the tensor-core form supports: N a multiple of 32 in [32, 256] (K' chunks of 32,
// at most two accumulators of 256 columns).
bool dft_gemm_size_ok(int N) { return N >= 32 && N <= 256 && N % 32 == 0; }

int launch_row_dft(const float2* y, float2* yt, const uint8_t* mask, int Nx, int Ny, int full_frame, int split,
                   int* err, cudaStream_t st, int withhold, long long limit) {
  GemmArgs a;
  a.x = y;
  a.out = yt;
  a.M = Nx;      // upper bound; the kernel counts the mask's lines
  a.rows = 1;
  a.N = Ny;
  a.split = split;
  a.err = err;
  a.mask = mask;
  a.mask_n = Nx;
  a.full_frame = full_frame;
  a.limit = limit;
  a.withhold = withhold;
  return launch_args(a, 1, (Nx + kRows - 1) / kRows, st);
}

int launch_dft2d_gemm(const float2* in, float2* out, float2* tmp, int batch, int Nx, int Ny, int inverse,
                      int split, int* err, cudaStream_t st, int withhold, long long limit) {
  // rows of each image (length Ny) -> tmp holds the transposes (Ny x Nx); then the rows of
  // the transposes (length Nx) -> out holds F_Nx X F_Ny (Nx x Ny)
  int rc = launch_pass(in, tmp, batch, Nx, Ny, inverse, split, err, st, withhold, limit);
  if (rc == TTS_OK) rc = launch_pass(tmp, out, batch, Ny, Nx, inverse, split, err, st);
  return rc;
}
