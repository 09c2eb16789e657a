// Column stage of (A^H A + lambda P_W) through the aliasing structure of A^H A.
//
// Every shot samples the k-space lines n = m Ns + i (m < M = N/Ns) of all
// coils, and the readout direction is fully sampled, so in the image domain
//   A^H A = S^H F_y^H Pi^H Pi F_y S        (Eqs. 1-3; Pi = CAIPI phase, slice
//                                          sum and shot mask)
// needs no transform at all.  Writing sh = N/Ldiv (the CAIPI shift of one
// slice index) and u = y + l sh, the y transform restricted to the lines of
// shot i followed by its adjoint sums exp(2 pi j m (u - u')/M) over m: it is
// M when u = u' (mod M) and 0 otherwise.  What remains couples, for each image
// column x and each class z = u mod M, the L Ns pixels (l, y) of that class:
//
//   (A^H A v)_{l,i}(y) = (1/Ns) conj(a_i^k) sum_{(l',y')} C_xz[(l,y),(l',y')] a_i^k' v_{l',i}(y'),
//
// with k = floor(u/M), a_i = exp(-2 pi j (i - N/2)/Ns) and the coil
// correlation C_xz[(l,y),(l',y')] = sum_c conj(S_{c,l}(x,y)) S_{c,l'}(x,y').
// C depends on the coil maps only, so it is formed once when they are set
// (k_alias_corr) and shared by every shot, direction and iteration.  Per
// pixel the coil loop (Nc coils x two M-point transforms) becomes L Ns complex
// multiply-adds.  The class structure needs sh to be an integer: Ldiv | N.
//
// Member a = l Ns + t of class z is the pixel y = ((z - l sh) mod M) + t M of slice l.
#include "common.cuh"
#include "fft.cuh"
#include "umma.cuh"

// corr[x][a][a'][z] = sum_c conj(S_{c,l}(x, y_a)) S_{c,l'}(x, y_a'), FP64 accumulation
// (class z fastest: the threads of a warp, consecutive pixels y, read consecutive classes)
__global__ void k_alias_corr(const float2* __restrict__ sensT, float2* __restrict__ corr, int L, int Ns, int Nc,
                             int N, int M, int sh) {
  const int B = L * Ns;
  const size_t NN = (size_t)N * N;
  const size_t total = (size_t)N * M * B * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(e % M);
    const int ap = (int)((e / M) % B);
    const int a = (int)((e / ((size_t)M * B)) % B);
    const int x = (int)(e / ((size_t)M * B * B));
    const int l = a / Ns, t = a - l * Ns, lp = ap / Ns, tp = ap - lp * Ns;
    const int y = (z - (l * sh) % M + M) % M + t * M;
    const int yp = (z - (lp * sh) % M + M) % M + tp * M;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < Nc; ++c) {
      const float2 s = sensT[(size_t)(l * Nc + c) * NN + (size_t)x * N + y];
      const float2 q = sensT[(size_t)(lp * Nc + c) * NN + (size_t)x * N + yp];
      re += (double)s.x * q.x + (double)s.y * q.y;
      im += (double)s.x * q.y - (double)s.y * q.x;
    }
    corr[e] = make_float2((float)re, (float)im);
  }
}

#define ALIAS_MAXITER (1L << 22)

// bounded wait on an mbarrier phase; false when it ran out
__device__ __forceinline__ bool alias_wait(uint64_t* mbar, uint32_t parity) {
  for (long it = 0; it < ALIAS_MAXITER; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (done) return true;
  }
  return false;
}

// One CTA per (image column x, direction): hybrid lines -> image (F_y^-1), the
// class products above plus lambda times the periodic penalty multiplier, the
// partial of Re<img, acc>, and F_y back to hybrid lines.  Thread tid < N tpy
// owns pixel row y = tid mod N of the lines b = tid / N (mod tpy); blockDim is
// N tpy rounded up to whole warps (the extra threads only help with the FFTs).
// Thread 0 starts TMA bulk copies of the column's B hybrid lines as soon as the
// CTA starts, so the HBM reads overlap the set-up.  With tpy = 1 a thread owns
// every shot of its pixel row, and (up to 5 shots) it fetches the slice's
// Ns(Ns+1)/2 multiplier entries (the Hermitian upper triangle) together, before
// the class products.
template <int L, int NS>
__global__ void __launch_bounds__(512) k_col_alias(ColArgs a, const float2* __restrict__ corr,
                                                   const float2* __restrict__ ash, int sh, int tpy) {
  constexpr int B = L * NS;
  constexpr int NPK = mult_planes(NS);
  constexpr bool PRELOAD = NPK <= 15;  // the slice's multiplier entries fit in registers (NS <= 5)
  extern __shared__ __align__(16) float2 sm[];
  __shared__ __align__(8) uint64_t bar[1];  // hybrid lines
  const int N = a.N, M = a.M;
  float2* img = sm;           // [B][N]
  float2* tmp = img + B * N;  // [B][N]
  float2* ph = tmp + B * N;   // [B][N] image times a_i^k
  float2* sTwN = ph + B * N;  // [N]
  float2* sAsh = sTwN + N;    // [NS][NS]: a_i^q, q < NS (padded to 16 bytes)
  double* red = reinterpret_cast<double*>(sAsh + ((NS * NS + 1) & ~1));  // [32]
  const int x = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t NN = (size_t)N * N;
  const size_t dir = blockIdx.y;
  const float2* __restrict__ gin = a.in + dir * (size_t)B * NN;
  float2* __restrict__ gout = a.out + dir * (size_t)B * NN;
  const float2* __restrict__ gmult = a.multT ? a.multT + dir * (size_t)L * NPK * NN : nullptr;
  double* gdot = a.dot_part ? a.dot_part + dir * SMSM_PART_MAX : nullptr;
  const bool pen = gmult != nullptr && a.lambda != 0.f;
  const uint32_t row_bytes = (uint32_t)(N * sizeof(float2));

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    mbar_arrive_expect_tx(&bar[0], (uint32_t)B * row_bytes);
    for (int b = 0; b < B; ++b) tma_bulk_g2s(img + b * N, gin + (size_t)b * NN + (size_t)x * N, row_bytes, &bar[0]);
  }
  for (int e = tid; e < N; e += nt) sTwN[e] = a.twN[e];
  for (int e = tid; e < NS * NS; e += nt) sAsh[e] = ash[e];
  const bool own = tid < N * tpy;
  const int y = tid % N, bsub = own ? tid / N : B;
  const float sy = sgn_par(y);
  // this pixel's class z, block k (mod NS) and member row in every slice
  const int t = y / M;
  int zl[L], kl[L], bs[L][L];  // (idle threads: bsub = B keeps every loop below empty)
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const int u = y + l * sh;
    zl[l] = u % M;
    kl[l] = (u / M) % NS;
  }
#pragma unroll
  for (int l = 0; l < L; ++l)
#pragma unroll
    for (int lp = 0; lp < L; ++lp) {
      int d = zl[l] - (lp * sh) % M;
      bs[l][lp] = d < 0 ? d + M : d;
    }
  __syncthreads();  // barrier initialisation visible before anyone waits on it
  // every thread agrees on the outcome of the wait, so none is left at a barrier
  if (!__syncthreads_and(alias_wait(&bar[0], 0))) {
    if (tid == 0) {
      atomicExch(a.errflag, SMSM_ERR_TIMEOUT);
      alias_wait(&bar[0], 0);  // in-flight copies land before the CTA exits
    }
    return;
  }
  // hybrid lines -> image lines (F_y^-1)
  for (int b = bsub; b < B; b += tpy) img[b * N + y] = cscale(img[b * N + y], sy);
  __syncthreads();
  {
    float2* R = fft_smem_call<true>(img, tmp, B, N, a.fN, sTwN);
    const float sc = a.sN * sy;
    for (int b = bsub; b < B; b += tpy) img[b * N + y] = cscale(R[b * N + y], sc);
  }
  __syncthreads();
#pragma unroll
  for (int l = 0; l < L; ++l) {
    int i0 = (bsub - l * NS) % tpy;
    if (i0 < 0) i0 += tpy;
    if (!own) i0 = NS;
    for (int i = i0; i < NS; i += tpy) ph[(l * NS + i) * N + y] = cmul(sAsh[i * NS + kl[l]], img[(l * NS + i) * N + y]);
  }
  __syncthreads();

  const float inv_ns = 1.f / (float)NS;
  const float2* cx = corr + (size_t)x * M * B * B;
  const size_t moff = (size_t)x * N + y;
  float dsum = 0.f;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    float2 c[B];  // row (l, t) of this pixel's class matrix, shared by every shot
    const float2* crow = cx + (size_t)(l * NS + t) * B * M + zl[l];
    if (own) {
#pragma unroll
      for (int ap = 0; ap < B; ++ap) c[ap] = __ldg(crow + (size_t)ap * M);
    }
    const float2* ml = pen ? gmult + (size_t)l * NPK * NN : nullptr;
    // output shot i of slice l: class product, plus lambda q (q = sum_j m_ij img_j)
    auto emit = [&](int i, float2 q) {
      const int b = l * NS + i;
      float2 s = cmk(0.f, 0.f);
#pragma unroll
      for (int lp = 0; lp < L; ++lp) {
        const float2* prow = ph + (lp * NS + i) * N + bs[l][lp];
#pragma unroll
        for (int tp = 0; tp < NS; ++tp) cfma(s, c[lp * NS + tp], prow[tp * M]);
      }
      float2 acc = cscale(cmulcj(sAsh[i * NS + kl[l]], s), inv_ns);
      const float2 v = img[b * N + y];
      if (pen) {
        acc.x = fmaf(a.lambda, q.x, acc.x);
        acc.y = fmaf(a.lambda, q.y, acc.y);
      }
      dsum = fmaf(v.x, acc.x, fmaf(v.y, acc.y, dsum));
      tmp[b * N + y] = cscale(acc, sy);
    };
    if (PRELOAD && tpy == 1) {
      if (own) {
        float2 mv[NPK];
        if (pen) {
#pragma unroll
          for (int k = 0; k < NPK; ++k) mv[k] = __ldg(ml + (size_t)k * NN + moff);
        }
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          float2 q = cmk(0.f, 0.f);
          if (pen) {
#pragma unroll
            for (int j = 0; j < NS; ++j) {
              const float2 m = i <= j ? mv[mult_plane(i, j, NS)] : conjf2(mv[mult_plane(j, i, NS)]);
              cfma(q, m, img[(l * NS + j) * N + y]);
            }
          }
          emit(i, q);
        }
      }
    } else {
      int i0 = (bsub - l * NS) % tpy;
      if (i0 < 0) i0 += tpy;
      if (!own) i0 = NS;
      for (int i = i0; i < NS; i += tpy) {
        float2 q = cmk(0.f, 0.f);
        if (pen) {
#pragma unroll
          for (int j = 0; j < NS; ++j) cfma(q, mult_at(ml, i, j, NS, NN, moff), img[(l * NS + j) * N + y]);
        }
        emit(i, q);
      }
    }
  }
  // partial of Re<img, acc> (Parseval: equals Re<p, q> in k-space); FP32 over this
  // thread's few pixels, FP64 from there on
  double dd = (double)dsum;
  for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
  if ((tid & 31) == 0) red[tid >> 5] = dd;
  __syncthreads();
  if (tid == 0 && gdot) {
    double s2 = 0.0;
    for (int w = 0; w < nt / 32; ++w) s2 += red[w];
    gdot[x] = s2;
  }
  float2* Rr = fft_smem_call<false>(tmp, ph, B, N, a.fN, sTwN);
  const float so = a.sN * sy;
  for (int b = bsub; b < B; b += tpy) gout[(size_t)b * NN + (size_t)x * N + y] = cscale(Rr[b * N + y], so);
}

typedef void (*ColAliasFn)(ColArgs, const float2*, const float2*, int, int);

#define CA_NS(L) {k_col_alias<L, 1>, k_col_alias<L, 2>, k_col_alias<L, 3>, k_col_alias<L, 4>, \
                  k_col_alias<L, 5>, k_col_alias<L, 6>, k_col_alias<L, 7>, k_col_alias<L, 8>}
static const ColAliasFn kColAlias[3][8] = {CA_NS(1), CA_NS(2), CA_NS(3)};
#undef CA_NS

// threads per pixel row: at least 64 threads per CTA (more threads per row measured slower:
// each one then re-reads the class rows for fewer outputs)
static int alias_tpy(int N, int B) {
  const int t = N >= 64 ? 1 : (64 + N - 1) / N;
  return t > B ? B : t;
}

static int alias_threads(int N, int B) { return (N * alias_tpy(N, B) + 31) / 32 * 32; }

static size_t alias_smem(const smsm_plan_s* P) {
  const int B = P->L * P->Ns;
  return (size_t)(3 * B * P->N + P->N + ((P->Ns * P->Ns + 1) & ~1)) * sizeof(float2) + 32 * sizeof(double);
}

size_t alias_corr_count(const smsm_plan_s* P) {
  const size_t B = (size_t)P->L * P->Ns;
  return (size_t)P->N * P->M * B * B;
}

int alias_supported(const smsm_plan_s* P) {
  if (P->N % P->Ldiv) return 0;  // CAIPI shift must be a whole number of pixels
  if (P->L < 1 || P->L > 3 || P->Ns < 1 || P->Ns > 8) return 0;
  if (alias_threads(P->N, P->L * P->Ns) > 512) return 0;
  if (alias_corr_count(P) * sizeof(float2) > (size_t)256 * 1024 * 1024) return 0;
  return alias_smem(P) <= 200 * 1024;
}

smsm_status alias_init_attrs() {
  for (int l = 0; l < 3; ++l)
    for (int n = 0; n < 8; ++n) {
      cudaError_t e = cudaFuncSetAttribute(kColAlias[l][n], cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) {
        smsm_set_error("cudaFuncSetAttribute (aliasing column stage): %s", cudaGetErrorString(e));
        return SMSM_ERR_CUDA;
      }
    }
  return SMSM_OK;
}

smsm_status launch_alias_corr(const smsm_plan_s* P, cudaStream_t s) {
  k_alias_corr<<<1024, 256, 0, s>>>(P->sensT, P->acorr, P->L, P->Ns, P->Nc, P->N, P->M, P->N / P->Ldiv);
  SMSM_LAUNCH_CHECK("k_alias_corr");
  return SMSM_OK;
}

smsm_status launch_col_alias(const smsm_plan_s* P, const ColArgs& a, cudaStream_t s) {
  const int tpy = alias_tpy(P->N, P->L * P->Ns);
  kColAlias[P->L - 1][P->Ns - 1]<<<dim3(P->N, P->D), alias_threads(P->N, P->L * P->Ns), alias_smem(P), s>>>(
      a, P->acorr, P->ash, P->N / P->Ldiv, tpy);
  SMSM_LAUNCH_CHECK("k_col_alias");
  return SMSM_OK;
}
