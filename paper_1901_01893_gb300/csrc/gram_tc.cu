// Hankel Gram G_l = H_l^H H_l (Eqs. 8-9) on the 5th-generation tensor cores.
//
// Real form: with X = [Re H | Im H] (P x 2C), R = X^T X and
//   Re G = R[re,re] + R[im,im],   Im G = R[re,im] - R[im,re]  (= R[re,im] - R[re,im]^T).
// The columns are padded to Cp = 16*ceil(C/16), so X has 2Cp columns: Re in
// [0, Cp), Im in [Cp, 2Cp).
//
// Only R's upper triangle is needed (R is symmetric and G reads entries with
// row <= column), so one CTA computes, from one staged copy of X^T, every
// 128-row tile t of R against the columns [128 t, 2Cp): tile 0 as two MMAs of
// N = Cp, the others as one MMA of N = 2Cp - 128 t (480 TMEM columns at
// 2Cp = 288).  It covers a contiguous block of patch rows ky (split-K); its FP32
// partial goes to global memory and k_gram_tc_reduce adds the partials in FP64
// in a fixed order.  Roles (warp-specialised, 352 threads):
//   * thread 0 brings the window of patch row ky -- image rows ky..ky+r-1 of
//     every shot -- into shared memory with TMA bulk copies (two windows in
//     flight, completion counted on an mbarrier);
//   * the producer warps build each chunk of KCH patches from the window
//     (implicit im2col), split every value into BF16 pieces and write X^T (all
//     2Cp rows, every piece) into a ring of stages in the canonical K-major
//     layout;
//   * one thread of the last warp issues the piece products D_t += X1_t X1_c^T +
//     ... for every tile t (A and B are row windows of the same staged X^T) and
//     commits each stage back to its producers;
//   * four warps drain the TMEM accumulator every GTC_EPOCH chunks into the
//     CTA's FP32 partial in global memory (each thread owns one row per tile and adds
//     with fire-and-forget reductions), which bounds the error
//     that the tensor core's FP32 accumulation gathers over many chunks.
//   PREC 2 (the FP32 form): every FP32 value split into three BF16 pieces,
//                b1 = bf16(x), b2 = bf16(x - b1), b3 = bf16(x - b1 - b2), which hold
//                its 24 significant bits exactly; six products b_i b_j' with
//                i + j <= 4 (the dropped ones are below 2^-24 of the product), so
//                every product is as accurate as an FP32 multiply;
//   PREC 1 (the reduced-precision form): two pieces hi = bf16(x), lo = bf16(x - hi)
//                and three products hi hi' + hi lo' + lo hi' (~2^-16 per product).
//   A third form, a TF32 hi + lo split with three products, was measured 9x less
//   accurate than FP32 FMA (2^-22 of every operand is lost) and is not kept.
// Every wait on an mbarrier is bounded; on a timeout the kernel raises the
// plan's device error flag, lets its in-flight bulk copies and MMAs finish
// (bounded waits), frees TMEM and returns.
#include <cuda_bf16.h>

#include <cmath>

#include "common.cuh"
#include "umma.cuh"

#define GTC_PROD_WARPS 6                               // im2col producers
#define GTC_THREADS (32 * (GTC_PROD_WARPS + 4 + 1))     // + 4 drain warps + 1 MMA warp
#define GTC_MAXITER (1L << 22)

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool gtc_wait(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
  for (long it = 0; it < GTC_MAXITER; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (done) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// shared-memory layout of one CTA (bytes); the same function sizes the launch
struct GtcLayout {
  int rows_alloc;    // 128 * number of row tiles
  int wp;            // window row pitch (complex elements): N + 8 (+16), shifts consecutive rows by 8 banks
  int ext;           // periodic: the first ext (even, >= r-1) elements of a row repeated after it
  int planes;        // operand pieces staged per chunk (2 or 3)
  size_t arr_bytes;  // one piece of one staged chunk: rows_alloc x (32 * k-steps) bytes
  size_t win_elems;  // one window: Ns*r rows of wp elements
  int nst;           // ring stages (3, or 2 when three do not fit)
  size_t total;
};

// Operand pieces and MMA k-steps (32 bytes of K each) per staged chunk of each form.
__host__ __device__ constexpr int gtc_planes(int prec) { return prec == 2 ? 3 : 2; }
__host__ __device__ constexpr int gtc_ksteps(int prec) { return prec == 2 ? 1 : 2; }
// Chunks accumulated in TMEM before a drain into the FP32 partial.  Every MMA rounds the
// accumulator once, so the epoch bounds the accumulation error: 4 chunks (24 roundings)
// keep the FP32 form's Gram at FP32-FMA accuracy (5e-8 rms of sqrt(G_ii G_jj), measured;
// 16 chunks gave 4e-7); the BF16 split form's own 2^-16 products allow 16.
__host__ __device__ constexpr int gtc_epoch(int prec) { return prec == 2 ? 4 : 16; }

__host__ __device__ inline GtcLayout gtc_layout(int Ns, int N, int r, int Cp, int periodic, int prec) {
  GtcLayout L;
  L.rows_alloc = 128 * ((2 * Cp + 127) / 128);
  L.ext = periodic ? ((r - 1 + 1) & ~1) : 0;
  L.wp = N + (L.ext > 8 ? 24 : 8);
  L.planes = gtc_planes(prec);
  L.arr_bytes = (size_t)L.rows_alloc * 32 * gtc_ksteps(prec);
  L.win_elems = (size_t)Ns * r * L.wp;
  const size_t win = 2 * L.win_elems * 8;
  L.nst = (L.planes * 3 * L.arr_bytes + win <= (size_t)224 * 1024) ? 3 : 2;
  L.total = L.planes * L.nst * L.arr_bytes + win;
  return L;
}

// TMEM columns of one CTA: the row tiles' accumulators side by side, tile t holding
// the columns [128 t, 2Cp) -- sum_t (2Cp - 128 t) -- rounded up to a power of two >= 32
// (480 of 512 at 2Cp = 288).
__host__ __device__ inline int gtc_tmem_cols(int R2C) {
  const int ntile = (R2C + 127) / 128;
  const int need = ntile * R2C - 64 * ntile * (ntile - 1);
  int c = 32;
  while (c < need) c <<= 1;
  return c;
}

// This CTA: every row tile of R, patch rows ky in [ky0, ky1) (block g of nG), matrix lf.
// A chunk is KCH = 32 KSTEP / ESZ consecutive patches of one patch row (the row's
// tail zero-padded).  Producer unit = one 16-byte core-matrix row: column c of X (its
// Re and Im rows of X^T), EPC consecutive patches.
template <int PREC>
__global__ void __launch_bounds__(GTC_THREADS, 1)
    k_gram_tc(const float2* __restrict__ x, float* __restrict__ Rpart, int* __restrict__ errflag, int Ns, int N,
              int r, int C, int Cp, int nG, int P1, int periodic) {
  constexpr int ESZ = 2;                         // bytes per operand element (BF16)
  constexpr int EPC = 16 / ESZ;                  // elements per 16-byte core-matrix row
  constexpr int KSTEP = gtc_ksteps(PREC);        // MMA k-steps per staged chunk
  constexpr int NPL = gtc_planes(PREC);          // operand pieces per chunk
  constexpr int KQ = 2 * KSTEP;                  // core matrices along K per chunk
  constexpr int GTC_EPOCH = gtc_epoch(PREC);     // chunks accumulated in TMEM before a drain
  constexpr int KCH = KQ * EPC;                  // patches per chunk
  constexpr uint32_t LBO = 128;                  // next core matrix along K
  constexpr uint32_t SBO = 128 * KQ;             // next 8-row group
  constexpr int NPROD = 32 * GTC_PROD_WARPS;     // producer threads
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full_b[3], empty_b[3], accfull_b, accempty_b, win_b[2], fin_b;
  __shared__ volatile int s_abort;

  const int g = blockIdx.x, lf = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R2C = 2 * Cp;
  const GtcLayout Lo = gtc_layout(Ns, N, r, Cp, periodic, PREC);
  const int ntile = Lo.rows_alloc / 128;
  const int NST = Lo.nst;
  const size_t arr_bytes = Lo.arr_bytes;
  const int WP = Lo.wp;
  float2* win = reinterpret_cast<float2*>(gsm + NPL * NST * arr_bytes);  // [2][Ns*r][WP]
  const int ky0 = (int)((long)g * P1 / nG), ky1 = (int)((long)(g + 1) * P1 / nG);
  const int nchx = (P1 + KCH - 1) / KCH;
  const int nit = (ky1 - ky0) * nchx;
  const int nepoch = (nit + GTC_EPOCH - 1) / GTC_EPOCH;
  const int rr = r * r;
  const size_t NN = (size_t)N * N;
  const float2* xl = x + (size_t)lf * Ns * NN;
  const uint32_t win_bytes = (uint32_t)((size_t)Ns * r * (N + Lo.ext) * sizeof(float2));
  const int tmem_cols = gtc_tmem_cols(R2C);

  for (size_t e = tid; e < NPL * NST * arr_bytes / 16; e += GTC_THREADS)
    reinterpret_cast<uint4*>(gsm)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tmem_alloc(&tmem_base, tmem_cols);
  if (tid == 0) {
    for (int k = 0; k < NST; ++k) {
      mbar_init(&full_b[k], NPROD);
      mbar_init(&empty_b[k], 1);
    }
    mbar_init(&accfull_b, 1);
    mbar_init(&accempty_b, 128);
    mbar_init(&win_b[0], 1);
    mbar_init(&win_b[1], 1);
    mbar_init(&fin_b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  // window ky -> buffer b: image rows ky..ky+r-1 of every shot, one TMA bulk copy per row
  // (periodic: rows mod N, and the row's first ext elements copied again after it)
  auto load_window = [&](int ky, int b) {
    fence_async_smem();
    mbar_arrive_expect_tx(&win_b[b], win_bytes);
    for (int ip = 0; ip < Ns * r; ++ip) {
      const int i = ip / r, py = ip - i * r;
      int row = ky + py;
      if (row >= N) row -= N;
      float2* dst = win + (size_t)b * Lo.win_elems + (size_t)ip * WP;
      const float2* src = xl + (size_t)i * NN + (size_t)row * N;
      tma_bulk_g2s(dst, src, (uint32_t)(N * sizeof(float2)), &win_b[b]);
      if (Lo.ext) tma_bulk_g2s(dst + N, src, (uint32_t)(Lo.ext * sizeof(float2)), &win_b[b]);
    }
  };

  if (warp < GTC_PROD_WARPS) {
    // ---------------- producers: im2col from the staged windows into the ring ----------------
    constexpr int UPT = (144 * KQ + NPROD - 1) / NPROD;  // Cp <= 144
    int woff[UPT], kofs[UPT];
    uint32_t ore[UPT], oim[UPT];
    bool act[UPT];
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      const int u = tid + NPROD * j;
      act[j] = u < Cp * KQ;
      woff[j] = -1;
      kofs[j] = 0;
      ore[j] = oim[j] = 0;
      if (act[j]) {
        const int r8 = u & 7, kq = (u >> 3) % KQ, cg = u / (8 * KQ);
        const int c = cg * 8 + r8;
        kofs[j] = kq * EPC;
        ore[j] = umma_kmajor_off(c, kq * 16, LBO, SBO);
        oim[j] = umma_kmajor_off(Cp + c, kq * 16, LBO, SBO);
        if (c < C) {
          const int i = c / rr, p = c - i * rr;
          const int py = p / r, px = p - py * r;
          woff[j] = (i * r + py) * WP + px + kq * EPC;
        }
      }
    }
    // Thread 0 keeps two windows in flight; window w (patch row ky0 + w) goes to buffer w & 1.
    // Every producer ends each patch row at a reducing barrier, so all of them take the
    // same decision to go on or to stop, and none is left waiting at a barrier.
    int issued = 0, consumed = 0;
    if (tid == 0)
      for (; issued < 2 && ky0 + issued < ky1; ++issued) load_window(ky0 + issued, issued);
    int it = 0;
    for (int ky = ky0; ky < ky1; ++ky) {
      const int w = ky - ky0, wb = w & 1;
      bool mine = gtc_wait(&win_b[wb], (uint32_t)((w >> 1) & 1), &s_abort);
      if (mine) {
        const float2* W = win + (size_t)wb * Lo.win_elems;
        for (int cx = 0; cx < nchx; ++cx, ++it) {
          const int s = it % NST;
          if (it >= NST && !gtc_wait(&empty_b[s], (uint32_t)((it / NST - 1) & 1), &s_abort)) {
            mine = false;
            break;
          }
          unsigned char* p1 = gsm + (size_t)s * NPL * arr_bytes;  // pieces of this stage
          unsigned char* p2 = p1 + arr_bytes;
#pragma unroll
          for (int j = 0; j < UPT; ++j) {
            if (!act[j]) continue;
            const int kx0 = cx * KCH + kofs[j];  // first patch of this unit
            float re[EPC], im[EPC];
#pragma unroll
            for (int m = 0; m < EPC; ++m) {
              float2 v = cmk(0.f, 0.f);
              if (woff[j] >= 0 && kx0 + m < P1) v = W[woff[j] + cx * KCH + m];
              re[m] = v.x;
              im[m] = v.y;
            }
            __align__(16) __nv_bfloat16 ar[8], ai[8], br[8], bi[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              ar[m] = __float2bfloat16_rn(re[m]);
              ai[m] = __float2bfloat16_rn(im[m]);
              re[m] -= __bfloat162float(ar[m]);  // exact: the remainder of a round-to-nearest
              im[m] -= __bfloat162float(ai[m]);
              br[m] = __float2bfloat16_rn(re[m]);
              bi[m] = __float2bfloat16_rn(im[m]);
            }
            *reinterpret_cast<uint4*>(p1 + ore[j]) = *reinterpret_cast<const uint4*>(ar);
            *reinterpret_cast<uint4*>(p1 + oim[j]) = *reinterpret_cast<const uint4*>(ai);
            *reinterpret_cast<uint4*>(p2 + ore[j]) = *reinterpret_cast<const uint4*>(br);
            *reinterpret_cast<uint4*>(p2 + oim[j]) = *reinterpret_cast<const uint4*>(bi);
            if (PREC == 2) {
              unsigned char* p3 = p2 + arr_bytes;
              __align__(16) __nv_bfloat16 cr[8], ci[8];
#pragma unroll
              for (int m = 0; m < 8; ++m) {
                cr[m] = __float2bfloat16_rn(re[m] - __bfloat162float(br[m]));
                ci[m] = __float2bfloat16_rn(im[m] - __bfloat162float(bi[m]));
              }
              *reinterpret_cast<uint4*>(p3 + ore[j]) = *reinterpret_cast<const uint4*>(cr);
              *reinterpret_cast<uint4*>(p3 + oim[j]) = *reinterpret_cast<const uint4*>(ci);
            }
          }
          fence_async_smem();
          mbar_arrive(&full_b[s]);
        }
      }
      const bool ok = named_bar_and(1, NPROD, mine);  // also: every producer is done reading buffer wb
      if (!ok) break;
      consumed = w + 1;
      if (tid == 0 && ky0 + issued < ky1) {
        load_window(ky0 + issued, issued & 1);
        ++issued;
      }
    }
    // windows still in flight after an abort land before the CTA's shared memory is released
    if (tid == 0)
      for (int w = consumed; w < issued; ++w) mbar_wait(&win_b[w & 1], (uint32_t)((w >> 1) & 1), GTC_MAXITER);
  } else if (tid == 32 * (GTC_PROD_WARPS + 4)) {
    // ---------------- MMA issue (one thread, in a warp of its own) ----------------
    for (int it = 0; it < nit; ++it) {
      const int s = it % NST;
      if (!gtc_wait(&full_b[s], (uint32_t)((it / NST) & 1), &s_abort)) break;
      const int ep = it / GTC_EPOCH;
      if (it % GTC_EPOCH == 0 && ep > 0 && !gtc_wait(&accempty_b, (uint32_t)((ep - 1) & 1), &s_abort)) break;
      tc_fence_after();
      const uint32_t b1 = smem_u32(gsm + (size_t)s * NPL * arr_bytes), b2 = b1 + (uint32_t)arr_bytes,
                     b3 = b2 + (uint32_t)arr_bytes;
#pragma unroll
      for (int ks = 0; ks < KSTEP; ++ks) {
        const uint32_t kb = (uint32_t)ks * 2 * LBO;
        // a new epoch overwrites the accumulator
        const uint32_t acc0 = (it % GTC_EPOCH || ks) ? 1u : 0u;
        uint32_t toff = 0;  // TMEM column of tile tt's first accumulator column
        for (int tt = 0; tt < ntile; ++tt) {
          const uint32_t arow = (uint32_t)(16 * tt) * SBO;  // rows 128 tt .. of X^T
          const uint64_t a1 = umma_desc(b1 + arow + kb, LBO, SBO), a2 = umma_desc(b2 + arow + kb, LBO, SBO);
          const int w = R2C - 128 * tt;                      // columns [128 tt, 2Cp)
          const int np = (tt == 0 && w > 256) ? 2 : 1;       // N <= 256 per MMA
          const int pw = w / np;
          const uint32_t idesc = umma_idesc(1u, 128, pw);  // BF16 operands, FP32 accumulator
          for (int pc = 0; pc < np; ++pc) {
            const int c0 = 128 * tt + pc * pw;
            const uint32_t brow = (uint32_t)(c0 / 8) * SBO + kb;
            const uint64_t c1 = umma_desc(b1 + brow, LBO, SBO), c2 = umma_desc(b2 + brow, LBO, SBO);
            const uint32_t d = tmem + toff + (uint32_t)(pc * pw);
            if (PREC == 2) {  // the small products first, then the leading one
              const uint64_t a3 = umma_desc(b3 + arow + kb, LBO, SBO), c3 = umma_desc(b3 + brow, LBO, SBO);
              umma_bf16(d, a1, c3, idesc, acc0);
              umma_bf16(d, a2, c2, idesc, 1u);
              umma_bf16(d, a3, c1, idesc, 1u);
              umma_bf16(d, a1, c2, idesc, 1u);
              umma_bf16(d, a2, c1, idesc, 1u);
              umma_bf16(d, a1, c1, idesc, 1u);
            } else {
              umma_bf16(d, a1, c1, idesc, acc0);
              umma_bf16(d, a1, c2, idesc, 1u);
              umma_bf16(d, a2, c1, idesc, 1u);
            }
          }
          toff += (uint32_t)w;
        }
      }
      umma_commit(&empty_b[s]);
      if (it % GTC_EPOCH == GTC_EPOCH - 1 || it == nit - 1) umma_commit(&accfull_b);
    }
    // every MMA issued above has finished before TMEM and the ring are released
    umma_commit(&fin_b);
    mbar_wait(&fin_b, 0u, GTC_MAXITER);
  } else if (warp >= GTC_PROD_WARPS && warp < GTC_PROD_WARPS + 4) {
    // ---------------- drain: each epoch's accumulator into this CTA's FP32 partial (L2) ----------------
    const int lw = warp & 3;  // TMEM lanes 32 (warp % 4) .. +31 are this warp's
    float* Rl = Rpart + ((size_t)lf * nG + g) * R2C * R2C;
    for (int ep = 0; ep < nepoch; ++ep) {
      // warp-uniform: the TMEM loads below are .sync.aligned
      if (!__all_sync(0xffffffffu, gtc_wait(&accfull_b, (uint32_t)(ep & 1), &s_abort))) break;
      tc_fence_after();
      // the first epoch stores, later ones add without reading back (no round trip to L2)
      uint32_t toff = 0;
      for (int tt = 0; tt < ntile; ++tt) {
        const int w = R2C - 128 * tt;
        const int row = 128 * tt + 32 * lw + lane;
        if (128 * tt + 32 * lw < R2C) {  // warp-uniform: some row of this warp is in range
          float* orow = Rl + (size_t)row * R2C + 128 * tt;
          for (int c0 = 0; c0 < w; c0 += 16) {
            uint32_t dv[16];
            tmem_ld16(tmem + ((uint32_t)(32 * lw) << 16) + toff + (uint32_t)c0, dv);
            if (row < R2C) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float v0 = __uint_as_float(dv[4 * q]), v1 = __uint_as_float(dv[4 * q + 1]);
                const float v2 = __uint_as_float(dv[4 * q + 2]), v3 = __uint_as_float(dv[4 * q + 3]);
                if (ep == 0)
                  *reinterpret_cast<float4*>(orow + c0 + 4 * q) = make_float4(v0, v1, v2, v3);
                else
                  red_add_v4(orow + c0 + 4 * q, v0, v1, v2, v3);
              }
            }
          }
        }
        toff += (uint32_t)w;
      }
      tc_fence_before();
      mbar_arrive(&accempty_b);
    }
    if (nepoch == 0)
      for (int tt = 0; tt < ntile; ++tt) {
        const int row = 128 * tt + 32 * lw + lane;
        if (row < R2C)
          for (int c = 128 * tt; c < R2C; ++c) Rl[(size_t)row * R2C + c] = 0.f;
      }
  }
  __syncthreads();
  if (s_abort && tid == 0) atomicExch(errflag, SMSM_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// G[c][c'] (c <= c') = sum_g (R[c][c'] + R[Cp+c][Cp+c']) + i (R[c][Cp+c'] - R[c'][Cp+c]) in FP64,
// every entry read from R's upper triangle; G[c'][c] is written as the conjugate, so G is
// exactly Hermitian.  One CTA (32 x 8 threads) per 32 x 32 tile (c, c') on or above the
// diagonal: the three terms read along c' are coalesced, and R[c'][Cp+c] is read along c
// and transposed through shared memory.  The sum over g runs in a fixed order.
#define GRED_T 32
__global__ void __launch_bounds__(GRED_T * 8) k_gram_tc_reduce(const float* __restrict__ Rpart,
                                                               double2* __restrict__ G, int LD, int C, int Cp,
                                                               int nG) {
  __shared__ float tr[GRED_T][GRED_T + 1];
  if (blockIdx.y > blockIdx.x) return;  // tile below the diagonal (uniform per CTA)
  const int R2C = 2 * Cp;
  const int lf = blockIdx.z;
  const int c0 = blockIdx.y * GRED_T, cc0 = blockIdx.x * GRED_T;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int cc = cc0 + tx;
  double re[GRED_T / 8], im[GRED_T / 8];
#pragma unroll
  for (int k = 0; k < GRED_T / 8; ++k) re[k] = im[k] = 0.0;
  for (int g = 0; g < nG; ++g) {
    const float* R = Rpart + ((size_t)lf * nG + g) * R2C * R2C;
    for (int j = ty; j < GRED_T; j += 8) {  // tr[j][i] = R[cc0 + j][Cp + c0 + i]
      const int rj = cc0 + j, ci = c0 + tx;
      tr[j][tx] = (rj < C && ci < C) ? R[(size_t)rj * R2C + Cp + ci] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GRED_T / 8; ++k) {
      const int c = c0 + ty + 8 * k;
      if (c < C && cc < C && c <= cc) {
        re[k] += (double)R[(size_t)c * R2C + cc] + (double)R[(size_t)(Cp + c) * R2C + Cp + cc];
        im[k] += (double)R[(size_t)c * R2C + Cp + cc] - (double)tr[tx][ty + 8 * k];
      }
    }
    __syncthreads();
  }
  double2* Gl = G + (size_t)lf * C * C;
#pragma unroll
  for (int k = 0; k < GRED_T / 8; ++k) {
    const int c = c0 + ty + 8 * k;
    if (c < C && cc < C && c <= cc) {
      if (c == cc) {
        Gl[(size_t)c * C + c] = make_double2(re[k], 0.0);
      } else {
        Gl[(size_t)c * C + cc] = make_double2(re[k], im[k]);
        Gl[(size_t)cc * C + c] = make_double2(re[k], -im[k]);
      }
    }
  }
}

static int gram_tc_prec(const smsm_plan_s* P) { return P->precision == SMSM_PRECISION_BF16_SPLIT ? 1 : 2; }

static size_t gram_tc_smem_for(int C, int Ns, int r, int N, int periodic, int prec) {
  return gtc_layout(Ns, N, r, 16 * ((C + 15) / 16), periodic, prec).total;
}

// 2Cp <= 288: the row tiles' accumulators take at most 480 TMEM columns; the ring and two
// patch-row windows in shared memory
int gram_tc_supported(const smsm_plan_s* P) {
  return P->C <= 144 && gram_tc_smem_for(P->C, P->Ns, P->r, P->N, P->periodic, gram_tc_prec(P)) <= 224 * 1024;
}

int gram_tc_cp(const smsm_plan_s* P) { return 16 * ((P->C + 15) / 16); }

// blocks of patch rows per matrix (split-K): between two and four waves of CTAs over the
// 152 SMs, the count whose last wave is fullest; more blocks (down to 2 patch rows each)
// when the batch is small; the FP32 partials stay under 256 MB
int gram_tc_nG(const smsm_plan_s* P) {
  const int Cp = gram_tc_cp(P), R2C = 2 * Cp;
  const int LD = P->LD, nsm = 152;
  const int lo = (2 * nsm + LD - 1) / LD, hi = (4 * nsm + LD - 1) / LD;
  int nG = lo;
  double best = -1.0;
  for (int n = lo; n <= hi; ++n) {
    const double waves = (double)LD * n / nsm;
    const double fill = waves / std::ceil(waves);
    if (fill > best + 1e-9) {
      best = fill;
      nG = n;
    }
  }
  const int most = (P->P1 + 1) / 2;
  if (nG > most) nG = most;
  const size_t per = (size_t)LD * R2C * R2C * sizeof(float);
  int cap = (int)((size_t)256 * 1024 * 1024 / per);
  if (cap < 1) cap = 1;
  if (nG > cap) nG = cap;
  if (nG < 1) nG = 1;
  return nG;
}

// Split-K block counts the autotuner tries: one to six waves of CTAs over the 152 SMs,
// within the same bounds as the heuristic above (at least 2 patch rows per block, FP32
// partials under 256 MB).  Returns the number written to out (at most maxn), ascending.
int gram_tc_nG_candidates(const smsm_plan_s* P, int* out, int maxn) {
  const int Cp = gram_tc_cp(P), R2C = 2 * Cp;
  const int LD = P->LD, nsm = 152;
  const int most = (P->P1 + 1) / 2;
  const size_t per = (size_t)LD * R2C * R2C * sizeof(float);
  int cap = (int)((size_t)256 * 1024 * 1024 / per);
  if (cap < 1) cap = 1;
  int n = 0;
  const int heur = gram_tc_nG(P);
  const double waves[] = {1.0, 2.0, 3.0, 4.0, 6.0};
  int cand[8];
  int nc = 0;
  cand[nc++] = heur;
  for (double w : waves) cand[nc++] = (int)std::ceil(w * nsm / LD);
  for (int k = 0; k < nc; ++k) {
    int v = cand[k];
    if (v > most) v = most;
    if (v > cap) v = cap;
    if (v < 1) v = 1;
    bool dup = false;
    for (int j = 0; j < n; ++j) dup |= out[j] == v;
    if (!dup && n < maxn) out[n++] = v;
  }
  for (int a = 1; a < n; ++a)  // ascending
    for (int b = a; b > 0 && out[b] < out[b - 1]; --b) {
      const int t = out[b];
      out[b] = out[b - 1];
      out[b - 1] = t;
    }
  return n;
}

static size_t gram_tc_smem(const smsm_plan_s* P) {
  return gram_tc_smem_for(P->C, P->Ns, P->r, P->N, P->periodic, gram_tc_prec(P));
}

smsm_status gram_tc_init_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024);
  if (e != cudaSuccess) {
    smsm_set_error("cudaFuncSetAttribute (tensor-core Gram): %s", cudaGetErrorString(e));
    return SMSM_ERR_CUDA;
  }
  return SMSM_OK;
}

smsm_status launch_gram_tc(const smsm_plan_s* P, const float2* x, double2* G, cudaStream_t s) {
  const int Cp = gram_tc_cp(P);
  const int nG = P->gram_tc_nG;
  dim3 grid(nG, P->LD);
  if (P->precision == SMSM_PRECISION_BF16_SPLIT)
    k_gram_tc<1><<<grid, GTC_THREADS, gram_tc_smem(P), s>>>(x, P->Rpart, P->devflag, P->Ns, P->N, P->r, P->C, Cp,
                                                                 nG, P->P1, P->periodic);
  else
    k_gram_tc<2><<<grid, GTC_THREADS, gram_tc_smem(P), s>>>(x, P->Rpart, P->devflag, P->Ns, P->N, P->r, P->C, Cp,
                                                                 nG, P->P1, P->periodic);
  SMSM_LAUNCH_CHECK("k_gram_tc");
  const int nt = (P->C + GRED_T - 1) / GRED_T;
  k_gram_tc_reduce<<<dim3(nt, nt, P->LD), dim3(GRED_T, 8), 0, s>>>(P->Rpart, G, P->LD, P->C, Cp, nG);
  SMSM_LAUNCH_CHECK("k_gram_tc_reduce");
  return SMSM_OK;
}
