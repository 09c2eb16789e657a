// Hankel Gram G_l = H_l^H H_l (Eqs. 8-9) on the 5th-generation tensor cores.
//
// Real form: with X = [Re H | Im H] (P x 2C), R = X^T X and
//   Re G = R[re,re] + R[im,im],   Im G = R[re,im] - R[im,re]  (= R[re,im] - R[re,im]^T).
// The columns are padded to Cp = 16*ceil(C/16), so X has 2Cp columns: Re in
// [0, Cp), Im in [Cp, 2Cp).
//
// One CTA computes a 128-row tile t of R against all 2Cp columns (two MMAs of
// N = Cp) over a strided subset of the patch chunks (split-K); its FP32
// partial goes to global memory and k_gram_tc_reduce adds the partials in FP64
// in a fixed order.  Per chunk of 16 patches, the 128 threads gather the Hankel
// entries x_i[k+p] straight from the image (implicit im2col), split every value
// into hi + lo and write X^T (all 2Cp rows, hi and lo) into one of two
// shared-memory stages in the canonical K-major layout; one thread then issues
// the MMAs  D += Xh_t Xh^T + Xh_t Xl^T + Xl_t Xh^T  (the A tile is a row window
// of the same staged X^T) and commits them to the stage's mbarrier, so staging
// the next chunk overlaps the tensor-core work.  The accumulator (128 lanes x
// 2Cp FP32 columns) stays in TMEM until the epilogue reads it back.
//   precision 0: TF32 split (hi = x with the low 13 mantissa bits cleared,
//                lo = x - hi): products accurate to ~2^-21, like FP32 FMA.
//   precision 1: BF16 split (hi = bf16(x), lo = bf16(x - hi)): ~2^-16.
// Every wait on an mbarrier is bounded; on a timeout the kernel raises the
// plan's device error flag, waits (bounded) for its last MMAs, frees TMEM and
// returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "umma.cuh"

#define GTC_THREADS 288   // warps 0-3: producers; warps 4-7: accumulator drain; warp 8 lane 0: MMA issue
#define GTC_STAGES 3      // shared-memory ring of staged chunks
#define GTC_EPOCH 32      // chunks accumulated in TMEM before draining into the FP32 running sum
#define GTC_MAXITER (1L << 22)

// patches per chunk: one MMA (32 bytes along K) per chunk and pass
template <int PREC>
struct GtcCfg {
  static constexpr int ESZ = PREC == 0 ? 4 : 2;
  static constexpr int KCH = 32 / ESZ;
};

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

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)));
}

template <int PREC>
__global__ void __launch_bounds__(GTC_THREADS, 1)
    k_gram_tc(const float2* __restrict__ x, float* __restrict__ Rpart, int* __restrict__ errflag, int Ns, int N,
              int r, int C, int Cp, int nG) {
  constexpr int ESZ = GtcCfg<PREC>::ESZ;        // bytes per operand element
  constexpr int KCH = GtcCfg<PREC>::KCH;        // patches per chunk (32 bytes along K)
  constexpr int EPC = 16 / ESZ;                 // elements per 16-byte core-matrix row
  constexpr uint32_t LBO = 128;                 // next core matrix along K
  constexpr uint32_t SBO = 256;                 // next 8-row group (2 core matrices along K)
  constexpr int NPROD = 128;                    // producer threads
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full_b[GTC_STAGES], empty_b[GTC_STAGES], accfull_b, accempty_b;
  __shared__ volatile int s_abort;

  const int t = blockIdx.x, g = blockIdx.y, lf = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R2C = 2 * Cp;
  const int ntile = (R2C + 127) / 128;
  const int rows_alloc = ntile * 128;
  const size_t arr_bytes = (size_t)rows_alloc * 32;  // one of hi / lo, one chunk
  float* Ssum = reinterpret_cast<float*>(gsm + 2 * GTC_STAGES * arr_bytes);  // [128][R2C + 1] running sum
  const int sld = R2C + 1;
  const int P1 = N - r + 1, P = P1 * P1;
  const int nchunks = (P + KCH - 1) / KCH;
  const int rr = r * r;
  const size_t NN = (size_t)N * N;
  const float2* xl = x + (size_t)lf * Ns * NN;
  const bool need_h0 = Cp > 128 * t;  // columns [0, Cp) reach the upper triangle of this row tile
  const int c_begin = need_h0 ? 0 : Cp;
  const int nit = nchunks > g ? (nchunks - g + nG - 1) / nG : 0;
  const int nepoch = (nit + GTC_EPOCH - 1) / GTC_EPOCH;

  for (size_t e = tid; e < 2 * GTC_STAGES * arr_bytes / 16; e += GTC_THREADS)
    reinterpret_cast<uint4*>(gsm)[e] = make_uint4(0, 0, 0, 0);
  for (int e = tid; e < 128 * sld; e += GTC_THREADS) Ssum[e] = 0.f;
  if (warp == 0) tmem_alloc(&tmem_base, R2C > 256 ? 512 : 256);
  if (tid == 0) {
    for (int k = 0; k < GTC_STAGES; ++k) {
      mbar_init(&full_b[k], NPROD);
      mbar_init(&empty_b[k], 1);
    }
    mbar_init(&accfull_b, 1);
    mbar_init(&accempty_b, 128);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp < 4) {
    // ---------------- producers: implicit im2col into the ring ----------------
    constexpr int IPT = (144 * KCH + NPROD - 1) / NPROD;  // Cp <= 144
    int kk[IPT];
    long coff[IPT];
    uint32_t ore[IPT], oim[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const int e = tid + NPROD * j;
      kk[j] = -1;
      coff[j] = -1;
      ore[j] = oim[j] = 0;
      if (e < Cp * KCH) {
        const int r8 = e & 7;
        const int kin = (e >> 3) % EPC;
        const int kq = (e / (8 * EPC)) % (KCH / EPC);
        const int cg = e / (8 * KCH);
        const int c = cg * 8 + r8;
        kk[j] = kq * EPC + kin;
        ore[j] = umma_kmajor_off(c, kk[j] * ESZ, LBO, SBO);
        oim[j] = umma_kmajor_off(Cp + c, kk[j] * ESZ, LBO, SBO);
        if (c < C) {
          const int i = c / rr, p = c - i * rr;
          const int py = p / r, px = p - py * r;
          coff[j] = (long)i * (long)NN + (long)py * N + px;
        }
      }
    }
    auto gather = [&](int chunk, float2 (&vv)[IPT]) {
      const int q0 = chunk * KCH;
      const int ky0 = q0 / P1, kx0 = q0 - ky0 * P1;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        vv[j] = cmk(0.f, 0.f);
        if (coff[j] >= 0) {
          int kx = kx0 + kk[j], ky = ky0;
          if (kx >= P1) {
            kx -= P1;
            ++ky;
          }
          if (q0 + kk[j] < P) vv[j] = __ldg(xl + coff[j] + (size_t)ky * N + kx);
        }
      }
    };
    float2 v[IPT];
    if (nit > 0) gather(g, v);
    for (int it = 0; it < nit; ++it) {
      const int s = it % GTC_STAGES;
      if (it >= GTC_STAGES && !gtc_wait(&empty_b[s], (uint32_t)((it / GTC_STAGES - 1) & 1), &s_abort)) break;
      unsigned char* hi = gsm + (size_t)s * 2 * arr_bytes;
      unsigned char* lo = hi + arr_bytes;
#pragma unroll
      for (int j = 0; j < IPT; ++j) {
        if (kk[j] < 0) continue;
        if (PREC == 0) {
          const float hre = __uint_as_float(__float_as_uint(v[j].x) & 0xFFFFE000u);
          const float him = __uint_as_float(__float_as_uint(v[j].y) & 0xFFFFE000u);
          *reinterpret_cast<float*>(hi + ore[j]) = hre;
          *reinterpret_cast<float*>(hi + oim[j]) = him;
          *reinterpret_cast<float*>(lo + ore[j]) = v[j].x - hre;
          *reinterpret_cast<float*>(lo + oim[j]) = v[j].y - him;
        } else {
          const __nv_bfloat16 hre = __float2bfloat16_rn(v[j].x), him = __float2bfloat16_rn(v[j].y);
          *reinterpret_cast<__nv_bfloat16*>(hi + ore[j]) = hre;
          *reinterpret_cast<__nv_bfloat16*>(hi + oim[j]) = him;
          *reinterpret_cast<__nv_bfloat16*>(lo + ore[j]) = __float2bfloat16_rn(v[j].x - __bfloat162float(hre));
          *reinterpret_cast<__nv_bfloat16*>(lo + oim[j]) = __float2bfloat16_rn(v[j].y - __bfloat162float(him));
        }
      }
      fence_async_smem();
      mbar_arrive(&full_b[s]);
      if (it + 1 < nit) gather(g + (it + 1) * nG, v);
    }
  } else if (tid == 256) {
    // ---------------- MMA issue (one thread, in a warp of its own) ----------------
    const uint32_t idesc = umma_idesc(PREC == 0 ? 2u : 1u, 128, Cp);
    for (int it = 0; it < nit; ++it) {
      const int s = it % GTC_STAGES;
      if (!gtc_wait(&full_b[s], (uint32_t)((it / GTC_STAGES) & 1), &s_abort)) break;
      const int ep = it / GTC_EPOCH;
      if (it % GTC_EPOCH == 0 && ep > 0 && !gtc_wait(&accempty_b, (uint32_t)((ep - 1) & 1), &s_abort)) break;
      tc_fence_after();
      const uint32_t hb = smem_u32(gsm + (size_t)s * 2 * arr_bytes), lb = hb + (uint32_t)arr_bytes;
      const uint32_t arow = (uint32_t)(128 * t / 8) * SBO;
      const uint64_t ah = umma_desc(hb + arow, LBO, SBO), al = umma_desc(lb + arow, LBO, SBO);
      const uint32_t acc0 = (it % GTC_EPOCH) ? 1u : 0u;  // a new epoch overwrites the accumulator
      for (int h = need_h0 ? 0 : 1; h < 2; ++h) {
        const uint32_t brow = (uint32_t)(h * Cp / 8) * SBO;
        const uint64_t bh = umma_desc(hb + brow, LBO, SBO), bl = umma_desc(lb + brow, LBO, SBO);
        const uint32_t d = tmem + (uint32_t)(h * Cp);
        if (PREC == 0) {
          umma_tf32(d, ah, bh, idesc, acc0);
          umma_tf32(d, ah, bl, idesc, 1u);
          umma_tf32(d, al, bh, idesc, 1u);
        } else {
          umma_bf16(d, ah, bh, idesc, acc0);
          umma_bf16(d, ah, bl, idesc, 1u);
          umma_bf16(d, al, bh, idesc, 1u);
        }
      }
      umma_commit(&empty_b[s]);
      if (it % GTC_EPOCH == GTC_EPOCH - 1 || it == nit - 1) umma_commit(&accfull_b);
    }
  }
  if (warp >= 4 && warp < 8) {
    // ---------------- drain: each epoch's accumulator into the running sum ----------------
    const int lw = warp & 3;
    float* srow = Ssum + (size_t)(32 * lw + lane) * sld;
    for (int ep = 0; ep < nepoch; ++ep) {
      if (!gtc_wait(&accfull_b, (uint32_t)(ep & 1), &s_abort)) break;
      tc_fence_after();
      for (int c0 = c_begin; c0 < R2C; c0 += 8) {
        uint32_t dv[8];
        tmem_ld8(tmem + ((uint32_t)(32 * lw) << 16) + (uint32_t)c0, dv);
#pragma unroll
        for (int j = 0; j < 8; ++j) srow[c0 + j] += __uint_as_float(dv[j]);
      }
      tc_fence_before();
      mbar_arrive(&accempty_b);
    }
  }
  __syncthreads();
  const bool ok = !s_abort;
  if (!ok && tid == 0) atomicExch(errflag, SMSM_ERR_TIMEOUT);
  float* out = Rpart + ((size_t)lf * nG + g) * R2C * R2C;
  for (int e = tid; e < 128 * R2C; e += GTC_THREADS) {
    const int rl = e / R2C, c = e - rl * R2C;
    const int row = 128 * t + rl;
    if (row < R2C && c >= c_begin) out[(size_t)row * R2C + c] = ok ? Ssum[(size_t)rl * sld + c] : 0.f;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, R2C > 256 ? 512 : 256);
}

// G[c][c'] (c <= c') = sum_g (R[c][c'] + R[Cp+c][Cp+c']) + i (R[c][Cp+c'] - R[c'][Cp+c]) in FP64;
// the lower triangle is the conjugate, so G is exactly Hermitian.
__global__ void k_gram_tc_reduce(const float* __restrict__ Rpart, double2* __restrict__ G, int LD, int C, int Cp,
                                 int nG) {
  const int R2C = 2 * Cp;
  const size_t total = (size_t)LD * C * C;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int lf = (int)(e / ((size_t)C * C));
    const int rem = (int)(e - (size_t)lf * C * C);
    const int a = rem / C, b = rem - a * C;
    const int c = a <= b ? a : b, cc = a <= b ? b : a;
    double re = 0.0, im = 0.0;
    for (int g = 0; g < nG; ++g) {
      const float* R = Rpart + ((size_t)lf * nG + g) * R2C * R2C;
      re += (double)R[(size_t)c * R2C + cc] + (double)R[(size_t)(Cp + c) * R2C + Cp + cc];
      im += (double)R[(size_t)c * R2C + Cp + cc] - (double)R[(size_t)cc * R2C + Cp + c];
    }
    if (a > b) im = -im;
    if (a == b) im = 0.0;
    G[e] = make_double2(re, im);
  }
}

// 2Cp <= 288 TMEM columns and 3 staged chunks + the running sum in shared memory
int gram_tc_supported(const smsm_plan_s* P) { return P->C <= 144; }

int gram_tc_cp(const smsm_plan_s* P) { return 16 * ((P->C + 15) / 16); }

int gram_tc_nG(const smsm_plan_s* P) {
  const int P1 = P->P1;
  const int Cp = gram_tc_cp(P), R2C = 2 * Cp;
  const int ntile = (R2C + 127) / 128;
  // enough CTAs for two waves over 152 SMs, at most ~8k patches per partial, at least 256
  int nG = (P1 * P1 + 8191) / 8192;
  const int waves = (2 * 152 + ntile * P->LD - 1) / (ntile * P->LD);
  if (nG < waves) nG = waves;
  const int most = (P1 * P1 + 255) / 256;
  if (nG > most) nG = most;
  const size_t per = (size_t)P->LD * R2C * R2C * sizeof(float);
  int cap = (int)((size_t)256 * 1024 * 1024 / per);
  if (cap < 1) cap = 1;
  if (nG > cap) nG = cap;
  if (nG < 1) nG = 1;
  return nG;
}

static size_t gram_tc_smem(const smsm_plan_s* P) {
  const int R2C = 2 * gram_tc_cp(P);
  const int rows_alloc = 128 * ((R2C + 127) / 128);
  return 2 * GTC_STAGES * (size_t)rows_alloc * 32 + (size_t)128 * (R2C + 1) * sizeof(float);
}

smsm_status gram_tc_init_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
  if (e != cudaSuccess) {
    smsm_set_error("cudaFuncSetAttribute (tensor-core Gram): %s", cudaGetErrorString(e));
    return SMSM_ERR_CUDA;
  }
  return SMSM_OK;
}

smsm_status launch_gram_tc(const smsm_plan_s* P, const float2* x, double2* G, cudaStream_t s) {
  const int Cp = gram_tc_cp(P), R2C = 2 * Cp;
  const int ntile = (R2C + 127) / 128;
  const int nG = P->gram_tc_nG;
  dim3 grid(ntile, nG, P->LD);
  if (P->precision == SMSM_PRECISION_BF16_SPLIT)
    k_gram_tc<1><<<grid, GTC_THREADS, gram_tc_smem(P), s>>>(x, P->Rpart, P->devflag, P->Ns, P->N, P->r, P->C, Cp,
                                                                 nG);
  else
    k_gram_tc<0><<<grid, GTC_THREADS, gram_tc_smem(P), s>>>(x, P->Rpart, P->devflag, P->Ns, P->N, P->r, P->C, Cp,
                                                                 nG);
  SMSM_LAUNCH_CHECK("k_gram_tc");
  k_gram_tc_reduce<<<512, 256, 0, s>>>(P->Rpart, G, P->LD, P->C, Cp, nG);
  SMSM_LAUNCH_CHECK("k_gram_tc_reduce");
  return SMSM_OK;
}
