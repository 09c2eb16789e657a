// SENSE / blipped-CAIPI operators of SMS-MUSSELS (Fig. 1 of the paper).
//
// Data flow.  The 2D centred DFT is split into a transform along x (rows,
// contiguous) and one along y.  Because the shot mask and the CAIPI phase act
// on k-space lines (ky) only, they commute with the x transform, so every
// per-coil step of A, A^H and A^H A runs in the "hybrid" layout [..][x][ky]
// (one contiguous line of N values per image column x):
//
//   x[l][i][ky][kx] --rowfft(inv, transposed out)--> h[l][i][x][ky]
//   h --column stage (per x line: F_y^-1, coil multiply, masked F_y with the
//        shot fold, CAIPI sum, [adjoint path], coil sum, F_y)--> h'
//   h'[l][i][x][ky] --rowfft(fwd, transposed in)--> q[l][i][ky][kx]
//
// Masked y transform of shot i.  Only lines n = m*Ns + i are kept, so with
// M = N/Ns and y = y' + t*M the centred DFT along y reduces to an M-point DFT
// of the folded line  w[y'] = sum_t tw_i[y'+tM] v[y'+tM]  with
// tw_i[y] = exp(-j 2 pi (i - N/2)(y - N/2)/N), followed by the line phase
// exp(+j 2 pi m (N/2)/M)/sqrt(N) (folded, with the CAIPI phase of Eq. 1,
// into the table cph[l][i][m]).  The coil images (201 MB at 256^2 x 32
// coils x 12 slice-shots) are never written to HBM.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"

// ---------------------------------------------------------------------------
// Tiled batch transpose: in[b][rows][cols] -> out[b][cols][rows]
// ---------------------------------------------------------------------------
__global__ void k_transpose(const float2* __restrict__ in, float2* __restrict__ out, int rows, int cols) {
  __shared__ float2 tile[32][33];
  const int b = blockIdx.z;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const float2* src = in + (size_t)b * rows * cols;
  float2* dst = out + (size_t)b * rows * cols;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = src[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[threadIdx.x][k];
  }
}

smsm_status launch_transpose(const float2* in, float2* out, int nb, int rows, int cols, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, nb), block(32, 8);
  k_transpose<<<grid, block, 0, s>>>(in, out, rows, cols);
  SMSM_LAUNCH_CHECK("k_transpose");
  return SMSM_OK;
}

// ---------------------------------------------------------------------------
// Row FFTs: centred unitary 1D DFT along the contiguous axis of length N.
// F_c v[n] = sN (-1)^n sum_y (-1)^y v[y] exp(-+ 2 pi i n y / N), sN = (-1)^(N/2)/sqrt(N).
// ---------------------------------------------------------------------------
static int pick_ty(int rows) {
  int ty = 16;
  while (ty > 1 && rows % ty) ty >>= 1;
  return ty;
}

// in[b][rows][N] -> out[b][N][rows]
template <bool INV>
__global__ void __launch_bounds__(256) k_rowfft_out_T(const float2* __restrict__ in, float2* __restrict__ out,
                                                      int rows, int TY, FftDesc d, const float2* __restrict__ tw,
                                                      float sN, int vec) {
  extern __shared__ float2 sm[];
  const int N = d.n, ld = N + 1;
  float2* b0 = sm;
  float2* b1 = sm + TY * ld;
  float2* twS = b1 + TY * ld;
  const int b = blockIdx.y, r0 = blockIdx.x * TY;
  for (int e = threadIdx.x; e < N; e += blockDim.x) twS[e] = tw[e];
  const float2* src = in + ((size_t)b * rows + r0) * N;
  // the TY rows are contiguous: two complex values per 16-byte load, all of a thread's
  // loads issued before any is used (N is even, so pairs never straddle a row)
  const float4* src4 = reinterpret_cast<const float4*>(src);
  const int n4 = vec ? TY * N / 2 : 0;
  for (int e = threadIdx.x; !vec && e < TY * N; e += blockDim.x) {
    int row = e / N, col = e - row * N;
    b0[row * ld + col] = cscale(src[e], sgn_par(col));
  }
  for (int e0 = threadIdx.x; e0 < n4; e0 += 4 * blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = e0 + k * blockDim.x;
      if (e < n4) v[k] = __ldg(src4 + e);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = e0 + k * blockDim.x;
      if (e < n4) {
        const int f = 2 * e, row = f / N, col = f - row * N;  // col even: signs +, -
        b0[row * ld + col] = cmk(v[k].x, v[k].y);
        b0[row * ld + col + 1] = cmk(-v[k].z, -v[k].w);
      }
    }
  }
  __syncthreads();
  float2* R = fft_smem<INV>(b0, b1, TY, ld, d, twS);
  float2* dst = out + (size_t)b * N * rows + r0;
  if (vec && (TY & 1) == 0 && (rows & 1) == 0) {
    // pairs of rows: 16-byte stores along each output line
    for (int e = threadIdx.x; e < TY * N / 2; e += blockDim.x) {
      const int col = e / (TY / 2), row = 2 * (e - col * (TY / 2));
      const float sc = sN * sgn_par(col);
      const float2 u = R[row * ld + col], w = R[(row + 1) * ld + col];
      *reinterpret_cast<float4*>(dst + (size_t)col * rows + row) = make_float4(sc * u.x, sc * u.y, sc * w.x, sc * w.y);
    }
  } else {
    for (int e = threadIdx.x; e < TY * N; e += blockDim.x) {
      int col = e / TY, row = e - col * TY;
      dst[(size_t)col * rows + row] = cscale(R[row * ld + col], sN * sgn_par(col));
    }
  }
}

// in[b][N][rows] -> out[b][rows][N]
template <bool INV>
__global__ void __launch_bounds__(256) k_rowfft_in_T(const float2* __restrict__ in, float2* __restrict__ out,
                                                     int rows, int TY, FftDesc d, const float2* __restrict__ tw,
                                                     float sN, int vec) {
  extern __shared__ float2 sm[];
  const int N = d.n, ld = N + 1;
  float2* b0 = sm;
  float2* b1 = sm + TY * ld;
  float2* twS = b1 + TY * ld;
  const int b = blockIdx.y, r0 = blockIdx.x * TY;
  for (int e = threadIdx.x; e < N; e += blockDim.x) twS[e] = tw[e];
  const float2* src = in + (size_t)b * N * rows + r0;
  if (vec && (TY & 1) == 0 && (rows & 1) == 0) {
    // pairs of rows of each input line: 16-byte loads, a thread's loads issued together
    const int n4 = TY * N / 2;
    for (int e0 = threadIdx.x; e0 < n4; e0 += 4 * blockDim.x) {
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + k * blockDim.x;
        if (e < n4) {
          const int col = e / (TY / 2), row = 2 * (e - col * (TY / 2));
          v[k] = __ldg(reinterpret_cast<const float4*>(src + (size_t)col * rows + row));
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + k * blockDim.x;
        if (e < n4) {
          const int col = e / (TY / 2), row = 2 * (e - col * (TY / 2));
          const float sg = sgn_par(col);
          b0[row * ld + col] = cmk(sg * v[k].x, sg * v[k].y);
          b0[(row + 1) * ld + col] = cmk(sg * v[k].z, sg * v[k].w);
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < TY * N; e += blockDim.x) {
      int col = e / TY, row = e - col * TY;
      b0[row * ld + col] = cscale(src[(size_t)col * rows + row], sgn_par(col));
    }
  }
  __syncthreads();
  float2* R = fft_smem<INV>(b0, b1, TY, ld, d, twS);
  float2* dst = out + ((size_t)b * rows + r0) * N;
  if (vec) {
    float4* dst4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < TY * N / 2; e += blockDim.x) {
      const int f = 2 * e, row = f / N, col = f - row * N;  // col even: signs +, -
      const float2 u = R[row * ld + col], w = R[row * ld + col + 1];
      dst4[e] = make_float4(sN * u.x, sN * u.y, -sN * w.x, -sN * w.y);
    }
  } else {
    for (int e = threadIdx.x; e < TY * N; e += blockDim.x) {
      int row = e / N, col = e - row * N;
      dst[e] = cscale(R[row * ld + col], sN * sgn_par(col));
    }
  }
}

// k_rowfft_out_T fused with the CG direction update of the previous step: the CTA
// forms beta = <r,r>_new / <r,r>_old from the per-CTA partials of its direction (FP64,
// fixed order), updates its rows of p in place, p = r + beta p, and transforms them.
// Buffers are the plan's own (16-byte aligned); in[b][rows][N] -> out[b][N][rows].
template <bool INV>
__global__ void __launch_bounds__(256) k_rowfft_out_T_cgp(float2* __restrict__ p, const float2* __restrict__ r,
                                                          float2* __restrict__ out, int rows, int TY, FftDesc d,
                                                          const float2* __restrict__ tw, float sN,
                                                          const double* __restrict__ rr_new,
                                                          const double* __restrict__ rr_old, int nrr, int B) {
  extern __shared__ float2 sm[];
  __shared__ double red[2];
  const int N = d.n, ld = N + 1;
  float2* b0 = sm;
  float2* b1 = sm + TY * ld;
  float2* twS = b1 + TY * ld;
  const int b = blockIdx.y, r0 = blockIdx.x * TY;
  const size_t poff = (size_t)(b / B) * SMSM_PART_MAX;
  if (threadIdx.x < 32) {  // one warp: lane-strided sums, then a fixed butterfly
    double sn = 0.0, so = 0.0;
    for (int k = threadIdx.x; k < nrr; k += 32) {
      sn += rr_new[poff + k];
      so += rr_old[poff + k];
    }
    for (int o = 16; o > 0; o >>= 1) {
      sn += __shfl_xor_sync(0xffffffffu, sn, o);
      so += __shfl_xor_sync(0xffffffffu, so, o);
    }
    if (threadIdx.x == 0) {
      red[0] = sn;
      red[1] = so;
    }
  }
  for (int e = threadIdx.x; e < N; e += blockDim.x) twS[e] = tw[e];
  __syncthreads();
  double beta = red[1] > 0.0 ? red[0] / red[1] : 0.0;
  if (!isfinite(beta)) beta = 0.0;
  const float bt = (float)beta;
  float4* p4 = reinterpret_cast<float4*>(p + ((size_t)b * rows + r0) * N);
  const float4* r4 = reinterpret_cast<const float4*>(r + ((size_t)b * rows + r0) * N);
  const int n4 = TY * N / 2;
  for (int e0 = threadIdx.x; e0 < n4; e0 += 4 * blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = e0 + k * blockDim.x;
      if (e < n4) {
        const float4 rv = __ldg(r4 + e), pv = p4[e];
        v[k] = make_float4(fmaf(bt, pv.x, rv.x), fmaf(bt, pv.y, rv.y), fmaf(bt, pv.z, rv.z), fmaf(bt, pv.w, rv.w));
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = e0 + k * blockDim.x;
      if (e < n4) {
        p4[e] = v[k];
        const int f = 2 * e, row = f / N, col = f - row * N;  // col even: signs +, -
        b0[row * ld + col] = cmk(v[k].x, v[k].y);
        b0[row * ld + col + 1] = cmk(-v[k].z, -v[k].w);
      }
    }
  }
  __syncthreads();
  float2* R = fft_smem<INV>(b0, b1, TY, ld, d, twS);
  float2* dst = out + (size_t)b * N * rows + r0;
  if ((TY & 1) == 0 && (rows & 1) == 0) {
    for (int e = threadIdx.x; e < TY * N / 2; e += blockDim.x) {
      const int col = e / (TY / 2), row = 2 * (e - col * (TY / 2));
      const float sc = sN * sgn_par(col);
      const float2 u = R[row * ld + col], w = R[(row + 1) * ld + col];
      *reinterpret_cast<float4*>(dst + (size_t)col * rows + row) = make_float4(sc * u.x, sc * u.y, sc * w.x, sc * w.y);
    }
  } else {
    for (int e = threadIdx.x; e < TY * N; e += blockDim.x) {
      int col = e / TY, row = e - col * TY;
      dst[(size_t)col * rows + row] = cscale(R[row * ld + col], sN * sgn_par(col));
    }
  }
}

static size_t rowfft_smem(int N, int TY) { return (size_t)(2 * TY * (N + 1) + N) * sizeof(float2); }

// 16-byte vector accesses when both buffers allow them (callers' buffers may be offset)
static int rowfft_vec(const void* in, const void* out) {
  return !(((uintptr_t)in | (uintptr_t)out) & 15u);
}

smsm_status launch_rowfft_out_T(const smsm_plan_s* P, const float2* in, float2* out, int nb, int rows,
                                int inverse, cudaStream_t s) {
  const int TY = pick_ty(rows);
  const int vec = rowfft_vec(in, out);
  dim3 grid(rows / TY, nb);
  size_t sm = rowfft_smem(P->N, TY);
  if (inverse)
    k_rowfft_out_T<true><<<grid, 256, sm, s>>>(in, out, rows, TY, P->fN, P->twN, P->sN, vec);
  else
    k_rowfft_out_T<false><<<grid, 256, sm, s>>>(in, out, rows, TY, P->fN, P->twN, P->sN, vec);
  SMSM_LAUNCH_CHECK("k_rowfft_out_T");
  return SMSM_OK;
}

smsm_status launch_rowfft_out_T_cgp(const smsm_plan_s* P, float2* p, const float2* r, float2* out, int nb,
                                    const double* rr_new, const double* rr_old, int nrr, cudaStream_t s) {
  const int rows = P->N;
  const int TY = pick_ty(rows);
  dim3 grid(rows / TY, nb);
  k_rowfft_out_T_cgp<true><<<grid, 256, rowfft_smem(P->N, TY), s>>>(p, r, out, rows, TY, P->fN, P->twN, P->sN,
                                                                     rr_new, rr_old, nrr, P->L * P->Ns);
  SMSM_LAUNCH_CHECK("k_rowfft_out_T_cgp");
  return SMSM_OK;
}

smsm_status launch_rowfft_in_T(const smsm_plan_s* P, const float2* in, float2* out, int nb, int rows,
                               int inverse, cudaStream_t s) {
  const int TY = pick_ty(rows);
  const int vec = rowfft_vec(in, out);
  dim3 grid(rows / TY, nb);
  size_t sm = rowfft_smem(P->N, TY);
  if (inverse)
    k_rowfft_in_T<true><<<grid, 256, sm, s>>>(in, out, rows, TY, P->fN, P->twN, P->sN, vec);
  else
    k_rowfft_in_T<false><<<grid, 256, sm, s>>>(in, out, rows, TY, P->fN, P->twN, P->sN, vec);
  SMSM_LAUNCH_CHECK("k_rowfft_in_T");
  return SMSM_OK;
}

// ---------------------------------------------------------------------------
// Column stage: one CTA per image column x.
// ---------------------------------------------------------------------------
#define COL_THREADS 256
#define SMSM_MAX_NS 8

__device__ double block_sum_double(double v, double* red) {
  // deterministic tree reduction over the block (blockDim.x a power of two <= 1024)
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

template <int MODE, bool PHASE>
__global__ void __launch_bounds__(COL_THREADS) k_col(const ColArgs a_param) {
  ColArgs a = a_param;  // per-direction offsets are applied to this copy
  extern __shared__ float2 sm[];
  __shared__ double red[COL_THREADS];
  const int L = a.L, Ns = a.Ns, N = a.N, M = a.M, Nc = a.Nc;
  const int B = L * Ns;
  float2* img = sm;          // [B][N]
  float2* acc = img + B * N; // [B][N]
  float2* fa = acc + B * N;  // [B][M]
  float2* fb = fa + B * M;   // [B][M]
  float2* sTwN = fb + B * M;
  float2* sTwM = sTwN + N;
  float2* sTs = sTwM + M;     // [Ns][N]
  float2* sCp = sTs + Ns * N; // [L][Ns][M]
  const int x = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t NN = (size_t)N * N;
  // batch: direction d has its own input, output, phase, multipliers and partials
  {
    const size_t d = blockIdx.y;
    const size_t ydir = (size_t)Ns * Nc * N * M;
    if (MODE == COL_ADJ)
      a.in += d * ydir;
    else
      a.in += d * (size_t)(PHASE ? L : B) * NN;
    if (MODE == COL_FWD)
      a.out += d * ydir;
    else
      a.out += d * (size_t)((MODE == COL_ADJ && PHASE) ? L : B) * NN;
    if (a.phaseT) a.phaseT += d * (size_t)B * NN;
    if (a.multT) a.multT += d * (size_t)L * mult_planes(Ns) * NN;
    if (a.dot_part) a.dot_part += d * SMSM_PART_MAX;
  }

  for (int e = tid; e < N; e += nt) sTwN[e] = a.twN[e];
  for (int e = tid; e < M; e += nt) sTwM[e] = a.twM[e];
  for (int e = tid; e < Ns * N; e += nt) sTs[e] = a.tw_shot[e];
  for (int e = tid; e < L * Ns * M; e += nt) sCp[e] = a.cph[e];

  if (MODE != COL_ADJ) {
    // load the hybrid lines of the input and take F_y^-1
    const int Bin = PHASE ? L : B;
    const int stride = PHASE ? Ns * N : N;
    for (int e = tid; e < Bin * N; e += nt) {
      int bi = e / N, ky = e - bi * N;
      img[bi * stride + ky] = cscale(a.in[(size_t)bi * NN + (size_t)x * N + ky], sgn_par(ky));
    }
    __syncthreads();
    float2* R = fft_smem<true>(img, acc, Bin, stride, a.fN, sTwN);
    if (PHASE) {
      for (int e = tid; e < L * N; e += nt) {
        int l = e / N, y = e - l * N;
        float2 v = cscale(R[l * stride + y], a.sN * sgn_par(y));
        for (int i = Ns - 1; i >= 0; --i)
          img[(l * Ns + i) * N + y] = cmul(v, a.phaseT[(size_t)(l * Ns + i) * NN + (size_t)x * N + y]);
      }
    } else {
      for (int e = tid; e < B * N; e += nt) {
        int y = e % N;
        img[e] = cscale(R[e], a.sN * sgn_par(y));
      }
    }
    __syncthreads();
  }

  if (MODE == COL_NORMAL || MODE == COL_PEN || MODE == COL_ADJ) {
    // accumulator init: lambda * sum_i' m_{ii'} img_i' (periodic penalty in the image domain) or 0
    const bool pen = (MODE != COL_ADJ) && a.multT != nullptr && a.lambda != 0.f;
    for (int e = tid; e < B * N; e += nt) {
      float2 s = cmk(0.f, 0.f);
      if (pen) {
        int b = e / N, y = e - b * N;
        int l = b / Ns, i = b - l * Ns;
        const float2* ml = a.multT + (size_t)l * mult_planes(Ns) * NN;
        for (int j = 0; j < Ns; ++j) cfma(s, mult_at(ml, i, j, Ns, NN, (size_t)x * N + y), img[(l * Ns + j) * N + y]);
        s = cscale(s, a.lambda);
      }
      acc[e] = s;
    }
    __syncthreads();
  }

  if (MODE != COL_PEN) {
    for (int c = 0; c < Nc; ++c) {
      float2* Ri;
      if (MODE != COL_ADJ) {
        // coil multiply + shot twiddle + fold: task (l, y')
        for (int e = tid; e < L * M; e += nt) {
          int l = e / M, yp = e - l * M;
          float2 w[SMSM_MAX_NS];
#pragma unroll
          for (int i = 0; i < SMSM_MAX_NS; ++i) w[i] = cmk(0.f, 0.f);
          const float2* srow = a.sensT + (size_t)(l * Nc + c) * NN + (size_t)x * N;
          for (int t = 0; t < Ns; ++t) {
            int y = yp + t * M;
            float2 sv = srow[y];
#pragma unroll
            for (int i = 0; i < SMSM_MAX_NS; ++i)
              if (i < Ns) cfma(w[i], cmul(sTs[i * N + y], sv), img[(l * Ns + i) * N + y]);
          }
#pragma unroll
          for (int i = 0; i < SMSM_MAX_NS; ++i)
            if (i < Ns) fa[(l * Ns + i) * M + yp] = w[i];
        }
        __syncthreads();
        float2* Rf = fft_smem<false>(fa, fb, B, M, a.fM, sTwM);
        // CAIPI phase + slice sum (Eq. 3); NORMAL: back-projection with the conjugate phase
        for (int e = tid; e < Ns * M; e += nt) {
          int i = e / M, m = e - i * M;
          float2 Y = cmk(0.f, 0.f);
          for (int l = 0; l < L; ++l) cfma(Y, sCp[(l * Ns + i) * M + m], Rf[(l * Ns + i) * M + m]);
          if (MODE == COL_FWD) {
            a.out[((size_t)(i * Nc + c) * N + x) * M + m] = Y;
          } else {
            for (int l = 0; l < L; ++l) Rf[(l * Ns + i) * M + m] = cmulcj(sCp[(l * Ns + i) * M + m], Y);
          }
        }
        __syncthreads();
        if (MODE == COL_FWD) continue;
        Ri = fft_smem<true>(Rf, Rf == fa ? fb : fa, B, M, a.fM, sTwM);
      } else {
        // adjoint: data line of (i, c) with the conjugate CAIPI phase per slice
        for (int e = tid; e < Ns * M; e += nt) {
          int i = e / M, m = e - i * M;
          float2 Y = a.in[((size_t)(i * Nc + c) * N + x) * M + m];
          for (int l = 0; l < L; ++l) fa[(l * Ns + i) * M + m] = cmulcj(sCp[(l * Ns + i) * M + m], Y);
        }
        __syncthreads();
        Ri = fft_smem<true>(fa, fb, B, M, a.fM, sTwM);
      }
      // unfold + conjugate shot twiddle + conjugate coil multiply, accumulate: task (l, y')
      for (int e = tid; e < L * M; e += nt) {
        int l = e / M, yp = e - l * M;
        const float2* srow = a.sensT + (size_t)(l * Nc + c) * NN + (size_t)x * N;
        for (int t = 0; t < Ns; ++t) {
          int y = yp + t * M;
          float2 sv = srow[y];
          for (int i = 0; i < Ns; ++i) {
            float2 g = cmulcj(sv, conjf2(sTs[i * N + y]));  // conj(S) conj(tw)
            cfma(acc[(l * Ns + i) * N + y], g, Ri[(l * Ns + i) * M + yp]);
          }
        }
      }
      __syncthreads();
    }
  }
  if (MODE == COL_FWD) return;

  int Bout = B, ostride = N;
  if (MODE == COL_ADJ && PHASE) {
    for (int e = tid; e < L * N; e += nt) {
      int l = e / N, y = e - l * N;
      float2 s = cmk(0.f, 0.f);
      for (int i = 0; i < Ns; ++i)
        cfmacj(s, a.phaseT[(size_t)(l * Ns + i) * NN + (size_t)x * N + y], acc[(l * Ns + i) * N + y]);
      acc[(l * Ns) * N + y] = s;
    }
    Bout = L;
    ostride = Ns * N;
    __syncthreads();
  }
  if ((MODE == COL_NORMAL || MODE == COL_PEN) && a.dot_part) {
    double s = 0.0;
    for (int e = tid; e < B * N; e += nt) {
      float2 u = img[e], v = acc[e];
      s += (double)u.x * v.x + (double)u.y * v.y;
    }
    s = block_sum_double(s, red);
    if (tid == 0) a.dot_part[x] = s;
  }
  // F_y of the accumulated lines
  for (int e = tid; e < Bout * N; e += nt) {
    int bo = e / N, y = e - bo * N;
    float2* p = acc + bo * ostride + y;
    *p = cscale(*p, sgn_par(y));
  }
  __syncthreads();
  float2* Rr = fft_smem<false>(acc, img, Bout, ostride, a.fN, sTwN);
  for (int e = tid; e < Bout * N; e += nt) {
    int bo = e / N, ky = e - bo * N;
    a.out[(size_t)bo * NN + (size_t)x * N + ky] = cscale(Rr[bo * ostride + ky], a.sN * sgn_par(ky));
  }
}

static size_t col_smem(const smsm_plan_s* P) {
  const int B = P->L * P->Ns;
  return (size_t)(2 * B * P->N + 2 * B * P->M + P->N + P->M + P->Ns * P->N + P->L * P->Ns * P->M) *
         sizeof(float2);
}

template <int MODE, bool PH>
static smsm_status launch_col_t(const ColArgs& a, int N, int D, size_t sm, cudaStream_t s) {
  k_col<MODE, PH><<<dim3(N, D), COL_THREADS, sm, s>>>(a);
  SMSM_LAUNCH_CHECK("k_col");
  return SMSM_OK;
}

smsm_status launch_col(const smsm_plan_s* P, int mode, int with_phase, const float2* in, float2* out,
                       const float2* phaseT, const float2* multT, float lambda, double* dot_part,
                       cudaStream_t s) {
  ColArgs a;
  a.in = in;
  a.out = out;
  a.sensT = P->sensT;
  a.phaseT = phaseT;
  a.multT = multT;
  a.twN = P->twN;
  a.twM = P->twM;
  a.tw_shot = P->tw_shot;
  a.cph = P->cph;
  a.fN = P->fN;
  a.fM = P->fM;
  a.L = P->L;
  a.Ns = P->Ns;
  a.Nc = P->Nc;
  a.N = P->N;
  a.M = P->M;
  a.sN = P->sN;
  a.lambda = lambda;
  a.dot_part = dot_part;
  a.errflag = P->devflag;
  if (mode == COL_NORMAL && !with_phase && P->alias) return launch_col_alias(P, a, s);
  if (mode == COL_NORMAL && !with_phase && !(P->flags & SMSM_FLAG_GENERIC_KERNELS)) {
    smsm_status fst = launch_col_fast(P, a, s);
    if (fst != SMSM_ERR_ARG) return fst;  // SMSM_ERR_ARG: no fast path for this geometry
  }
  size_t sm = col_smem(P);
  if (sm > 200 * 1024) {
    smsm_set_error("column stage needs %zu bytes of shared memory (> 200 KB)", sm);
    return SMSM_ERR_ARG;
  }
  switch (mode) {
    case COL_FWD:
      return with_phase ? launch_col_t<COL_FWD, true>(a, P->N, P->D, sm, s) : launch_col_t<COL_FWD, false>(a, P->N, P->D, sm, s);
    case COL_ADJ:
      return with_phase ? launch_col_t<COL_ADJ, true>(a, P->N, P->D, sm, s) : launch_col_t<COL_ADJ, false>(a, P->N, P->D, sm, s);
    case COL_NORMAL:
      return launch_col_t<COL_NORMAL, false>(a, P->N, P->D, sm, s);
    default:
      return launch_col_t<COL_PEN, false>(a, P->N, P->D, sm, s);
  }
}

size_t smsm_col_smem_bytes(const smsm_plan_s* P) { return col_smem(P); }

// Raise the dynamic shared-memory limit of every kernel that may need more
// than 48 KB.  Called once per plan, outside any stream capture.
smsm_status operators_init_attrs() {
  const int lim = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define SET_ATTR(k) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
  SET_ATTR((k_col<COL_FWD, false>));
  SET_ATTR((k_col<COL_FWD, true>));
  SET_ATTR((k_col<COL_ADJ, false>));
  SET_ATTR((k_col<COL_ADJ, true>));
  SET_ATTR((k_col<COL_NORMAL, false>));
  SET_ATTR((k_col<COL_PEN, false>));
  SET_ATTR((k_rowfft_out_T<true>));
  SET_ATTR((k_rowfft_out_T<false>));
  SET_ATTR((k_rowfft_in_T<true>));
  SET_ATTR((k_rowfft_in_T<false>));
  SET_ATTR((k_rowfft_out_T_cgp<true>));
#undef SET_ATTR
  if (e != cudaSuccess) {
    smsm_set_error("cudaFuncSetAttribute failed: %s", cudaGetErrorString(e));
    return SMSM_ERR_CUDA;
  }
  return SMSM_OK;
}
