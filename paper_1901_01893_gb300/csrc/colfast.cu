// Fast column stage of (A^H A + lambda P_W): one warp per shot, coil loop in registers.
//
// Same mathematics as k_col<COL_NORMAL> (operators.cu): per image column x,
// for every coil c the masked, CAIPI-phased y transform of each slice-shot
// line and its adjoint (Fig. 1; Eqs. 1-3), accumulated over coils, plus the
// periodic annihilating-filter multiplier.  What changes is where the work
// happens:
//  * warp w handles shot i = w for all L slices (the CAIPI slice sum couples
//    slices, never shots), so the whole coil loop needs no __syncthreads;
//  * lane j holds pixels y = j + 32k; the shot fold y -> y mod M is then
//    lane-local for M = 32R, or an xor-shuffle sum over lanes for M in {8, 16};
//  * the M-point DFT is a local R-point DFT, a twiddle, and a 32-lane
//    radix-2 decimation-in-frequency exchange by __shfl_xor (output in
//    bit-reversed lane order); the CAIPI phase table is read in that order and
//    the inverse is the matching decimation-in-time exchange (bit-reversed in,
//    natural out), so no data is ever permuted;
//  * the per-coil accumulators live in registers for the whole coil loop.
// Only the two N-point y transforms of the slice-shot lines (before and after
// the coil loop) go through shared memory.
#include "common.cuh"
#include "fft.cuh"

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return cmk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// 32-lane (or n-lane segment) radix-2 DIF: natural order in, bit-reversed out.
// w32[k] = exp(-2 pi i k / 32).
__device__ __forceinline__ float2 lane_dif(float2 x, int lane, int n, const float2* w32) {
  for (int h = n >> 1; h >= 1; h >>= 1) {
    const float2 v = shfl_xor2(x, h);
    if (lane & h) {
      const float2 w = w32[(lane & (h - 1)) * (16 / h)];
      x = cmul(csub(v, x), w);
    } else {
      x = cadd(x, v);
    }
  }
  return x;
}

// inverse of lane_dif up to the factor n: bit-reversed in, natural out, conjugate roots
__device__ __forceinline__ float2 lane_dit_inv(float2 x, int lane, int n, const float2* w32) {
  for (int h = 1; h < n; h <<= 1) {
    const float2 v = shfl_xor2(x, h);
    const float2 w = conjf2(w32[(lane & (h - 1)) * (16 / h)]);
    if (lane & h)
      x = csub(v, cmul(x, w));
    else
      x = cadd(x, cmul(v, w));
  }
  return x;
}

template <int L, int NK, int MR>
__global__ void __launch_bounds__(256) k_col_fast(ColArgs a) {
  constexpr int N = 32 * NK;
  constexpr int RW = MR > 0 ? MR : 1;
  extern __shared__ float2 sm[];
  const int Ns = a.Ns, Nc = a.Nc, M = a.M;
  const int B = L * Ns;
  float2* img = sm;                // [B][N]
  float2* tmp = img + B * N;       // [B][N]
  float2* sTwN = tmp + B * N;      // [N]
  float2* sTs = sTwN + N;          // [Ns][N]
  float2* sCp = sTs + Ns * N;      // [L][Ns][RW][32] CAIPI table in lane order
  float2* sTwM = sCp + L * Ns * RW * 32;  // [M]
  float2* sW32 = sTwM + M;         // [32]
  double* red = reinterpret_cast<double*>(sW32 + 32);  // [Ns]
  const int x = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  const size_t NN = (size_t)N * N;
  const size_t dir = blockIdx.y;
  const float2* __restrict__ gin = a.in + dir * (size_t)B * NN;
  float2* __restrict__ gout = a.out + dir * (size_t)B * NN;
  const float2* __restrict__ gmult = a.multT ? a.multT + dir * (size_t)L * mult_planes(Ns) * NN : nullptr;
  double* gdot = a.dot_part ? a.dot_part + dir * SMSM_PART_MAX : nullptr;
  for (int e = tid; e < N; e += nt) sTwN[e] = a.twN[e];
  for (int e = tid; e < M; e += nt) sTwM[e] = a.twM[e];
  for (int e = tid; e < Ns * N; e += nt) sTs[e] = a.tw_shot[e];
  for (int e = tid; e < 32; e += nt) sW32[e] = a.twN[e * (N / 32)];  // exp(-2 pi i e/32)
  for (int e = tid; e < L * Ns * RW * 32; e += nt) {
    const int ln = e & 31;
    const int f1 = (e >> 5) % RW;
    const int li = (e >> 5) / RW;  // l * Ns + i
    int m;
    if (MR > 0) {
      m = f1 + MR * (int)(__brev((unsigned)ln) >> 27);
    } else {
      const int b = __ffs(M) - 1;  // M = 2^b <= 16
      m = (int)(__brev((unsigned)(ln & (M - 1))) >> (32 - b));
    }
    sCp[e] = a.cph[li * M + m];
  }
  // hybrid lines -> image lines (F_y^-1)
  for (int e = tid; e < B * N; e += nt) {
    const int b = e / N, ky = e - b * N;
    img[e] = cscale(gin[(size_t)b * NN + (size_t)x * N + ky], sgn_par(ky));
  }
  __syncthreads();
  {
    float2* R = fft_fixed_from<true, N, 1>(img, tmp, B, N, sTwN);
    for (int e = tid; e < B * N; e += nt) img[e] = cscale(R[e], a.sN * sgn_par(e % N));
  }
  __syncthreads();

  const int i = warp;  // this warp's shot
  float2 acc[L][NK];
  const bool pen = gmult != nullptr && a.lambda != 0.f;
#pragma unroll
  for (int l = 0; l < L; ++l)
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const int y = lane + 32 * k;
      float2 s = cmk(0.f, 0.f);
      if (pen) {
        const float2* ml = gmult + (size_t)l * mult_planes(Ns) * NN;
        for (int j = 0; j < Ns; ++j) cfma(s, mult_at(ml, i, j, Ns, NN, (size_t)x * N + y), img[(l * Ns + j) * N + y]);
        s = cscale(s, a.lambda);
      }
      acc[l][k] = s;
    }

  for (int c = 0; c < Nc; ++c) {
    float2 fw[L][RW];
    // coil multiply, shot twiddle, fold
#pragma unroll
    for (int l = 0; l < L; ++l) {
#pragma unroll
      for (int f = 0; f < RW; ++f) fw[l][f] = cmk(0.f, 0.f);
      const float2* srow = a.sensT + (size_t)(l * Nc + c) * NN + (size_t)x * N;
      const float2* irow = img + (l * Ns + i) * N;
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const int y = lane + 32 * k;
        const float2 st = cmul(__ldg(srow + y), sTs[i * N + y]);
        cfma(fw[l][MR > 0 ? k % RW : 0], st, irow[y]);
      }
    }
    if (MR == 0) {
#pragma unroll
      for (int l = 0; l < L; ++l)
        for (int h = M; h < 32; h <<= 1) fw[l][0] = cadd(fw[l][0], shfl_xor2(fw[l][0], h));
    }
    // forward M-point DFT: local R-point DFT + twiddle, then the lane exchange
#pragma unroll
    for (int l = 0; l < L; ++l) {
      if (MR > 1) {
        float2 t[RW];
#pragma unroll
        for (int f = 0; f < RW; ++f) {
          float2 s = fw[l][0];
#pragma unroll
          for (int k = 1; k < RW; ++k) cfma(s, fw[l][k], sTwM[(k * f * 32) % M]);
          t[f] = f ? cmul(s, sTwM[(lane * f) % M]) : s;
        }
#pragma unroll
        for (int f = 0; f < RW; ++f) fw[l][f] = t[f];
      }
#pragma unroll
      for (int f = 0; f < RW; ++f) fw[l][f] = lane_dif(fw[l][f], lane, MR > 0 ? 32 : M, sW32);
    }
    // CAIPI phase and slice sum (Eq. 3), then the conjugate phase back to every slice
#pragma unroll
    for (int f = 0; f < RW; ++f) {
      float2 Y = cmk(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < L; ++l) cfma(Y, sCp[((l * Ns + i) * RW + f) * 32 + lane], fw[l][f]);
#pragma unroll
      for (int l = 0; l < L; ++l) fw[l][f] = cmulcj(sCp[((l * Ns + i) * RW + f) * 32 + lane], Y);
    }
    // inverse M-point DFT
#pragma unroll
    for (int l = 0; l < L; ++l) {
#pragma unroll
      for (int f = 0; f < RW; ++f) fw[l][f] = lane_dit_inv(fw[l][f], lane, MR > 0 ? 32 : M, sW32);
      if (MR > 1) {
        float2 t[RW];
#pragma unroll
        for (int f = 0; f < RW; ++f) t[f] = f ? cmulcj(sTwM[(lane * f) % M], fw[l][f]) : fw[l][f];
#pragma unroll
        for (int k = 0; k < RW; ++k) {
          float2 s = t[0];
#pragma unroll
          for (int f = 1; f < RW; ++f) cfma(s, t[f], conjf2(sTwM[(k * f * 32) % M]));
          fw[l][k] = s;
        }
      }
    }
    // unfold, conjugate shot twiddle and coil, accumulate
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float2* srow = a.sensT + (size_t)(l * Nc + c) * NN + (size_t)x * N;
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const int y = lane + 32 * k;
        const float2 st = cmul(__ldg(srow + y), sTs[i * N + y]);
        cfmacj(acc[l][k], st, fw[l][MR > 0 ? k % RW : 0]);
      }
    }
  }

  // partial of Re<img, acc> (Parseval: equals Re<p, q> in k-space)
  double dsum = 0.0;
#pragma unroll
  for (int l = 0; l < L; ++l)
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const int y = lane + 32 * k;
      const float2 u = img[(l * Ns + i) * N + y];
      dsum += (double)u.x * acc[l][k].x + (double)u.y * acc[l][k].y;
      tmp[(l * Ns + i) * N + y] = cscale(acc[l][k], sgn_par(y));
    }
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  if (lane == 0) red[warp] = dsum;
  __syncthreads();
  if (tid == 0 && gdot) {
    double s = 0.0;
    for (int w = 0; w < Ns; ++w) s += red[w];
    gdot[x] = s;
  }
  float2* Rr = fft_fixed_from<false, N, 1>(tmp, img, B, N, sTwN);
  for (int e = tid; e < B * N; e += nt) {
    const int b = e / N, ky = e - b * N;
    gout[(size_t)b * NN + (size_t)x * N + ky] = cscale(Rr[e], a.sN * sgn_par(ky));
  }
}

typedef void (*ColFastFn)(ColArgs);

struct ColFastEntry {
  int L, NK, MR;
  ColFastFn fn;
};

#define CF(L, NK, MR) {L, NK, MR, k_col_fast<L, NK, MR>}
#define CF_L(NK, MR) CF(1, NK, MR), CF(2, NK, MR), CF(3, NK, MR)
static const ColFastEntry kColFast[] = {
    CF_L(2, 1), CF_L(2, 0),                // N = 64:  M = 32; 16, 8
    CF_L(3, 1), CF_L(3, 0),                // N = 96:  M = 32; 16
    CF_L(4, 2), CF_L(4, 1), CF_L(4, 0),    // N = 128: M = 64, 32; 16
    CF_L(6, 3), CF_L(6, 2), CF_L(6, 1),    // N = 192: M = 96, 64, 32
    CF_L(8, 4), CF_L(8, 2), CF_L(8, 1),    // N = 256: M = 128, 64, 32
};
#undef CF_L
#undef CF

static size_t colfast_smem(const smsm_plan_s* P, int RW) {
  const int B = P->L * P->Ns;
  return (size_t)(2 * B * P->N + P->N + P->Ns * P->N + P->L * P->Ns * RW * 32 + P->M + 32) * sizeof(float2) +
         (size_t)P->Ns * sizeof(double);
}

static const ColFastEntry* find_fast(const smsm_plan_s* P) {
  if (P->N % 32) return nullptr;
  const int NK = P->N / 32;
  int MR;
  if (P->M % 32 == 0)
    MR = P->M / 32;
  else if (P->M == 8 || P->M == 16)
    MR = 0;
  else
    return nullptr;
  for (const ColFastEntry& e : kColFast)
    if (e.L == P->L && e.NK == NK && e.MR == MR) return &e;
  return nullptr;
}

smsm_status colfast_init_attrs() {
  for (const ColFastEntry& e : kColFast) {
    cudaError_t err = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (err != cudaSuccess) {
      smsm_set_error("cudaFuncSetAttribute (fast column stage): %s", cudaGetErrorString(err));
      return SMSM_ERR_CUDA;
    }
  }
  return SMSM_OK;
}

smsm_status launch_col_fast(const smsm_plan_s* P, const ColArgs& a, cudaStream_t s) {
  const ColFastEntry* e = find_fast(P);
  if (!e) return SMSM_ERR_ARG;
  const size_t sm = colfast_smem(P, e->MR > 0 ? e->MR : 1);
  if (sm > 200 * 1024) return SMSM_ERR_ARG;
  e->fn<<<dim3(P->N, P->D), 32 * P->Ns, sm, s>>>(a);
  SMSM_LAUNCH_CHECK("k_col_fast");
  return SMSM_OK;
}
