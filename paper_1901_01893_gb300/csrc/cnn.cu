// Learned warm start: a small complex CNN trained on the GPU by these kernels.
//
// The paper has no learned component.  This network seeds the IRLS solve of
// Eq. 10: from the aliased, zero-filled image of every (slice, shot),
// a = F^-1(A^H y), it predicts a starting image x0 = a + f(a), whose k-space
// F x0 is the solve's first iterate and so also its first Gram and annihilating
// filters (Eq. 9).  f is six complex 3x3 convolutions (B -> width -> ... -> B,
// B = L*Ns) with CReLU (ReLU on the real and on the imaginary part) between them.
//
// Arithmetic: weights are held as FP32 master copies and used rounded to BF16
// (every product takes a BF16 weight); activations, products and accumulation
// are FP32.  Convolution (cross-correlation, zero padding):
//     z[o, p] = b[o] + sum_c sum_k W[o, c, k] h[c, p + k - 1].
// Gradients of the real loss are carried as G = dL/dRe + i dL/dIm:
//     dW[o, c, k] = sum_p G[o, p] conj(h[c, p + k - 1]),  db[o] = sum_p G[o, p],
//     dh[c, q]   = sum_o sum_k conj(W[o, c, k]) G[o, q - k + 1]
// -- the last is again a convolution of G, with the weights conjugated,
// transposed and their 3x3 taps reversed, so one kernel serves both.
// Loss of one sample: ||x0 - t||^2 / ||t||^2; a batch averages its samples.
// Optimiser: Adam on the master weights.  Every reduction (loss, weight
// gradients over the pixels) runs in a fixed order, so training is
// bit-reproducible.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"

#define CV_T 16     // output tile edge (pixels)
#define CV_OCB 32   // output channels per CTA
#define CV_ICB 8    // input channels staged per step
#define CV_SP 20    // staged row pitch (18 used)
#define WG_OCB 32   // weight gradient: output channels per CTA
#define WG_ICB 32   // weight gradient: input channels per CTA
#define WG_TY 8     // weight gradient pixel tile: 8 rows x 16 columns
#define WG_TX 16
#define WG_CP 181   // staged channel pitch (float2) of the weight-gradient input tile
#define WG_SPLIT 64 // pixel splits of the weight gradient (partials reduced in a fixed order)

struct smsm_cnn_s {
  int B, width, layers, H, W, maxn;
  int dev;
  std::vector<int> cin, cout;      // per layer
  std::vector<size_t> woff, boff;  // complex offsets of W_k and b_k in the parameter vector
  size_t count;                    // complex parameters
  float2 *master, *wbf, *grad, *m1, *m2;  // [count]
  float2* wt;                      // transposed-conjugated-reversed weights, largest layer
  std::vector<float2*> z;          // pre-activations per layer [maxn][cout][H][W]
  float2 *gA, *gB;                 // gradient ping-pong [maxn][width][H][W]
  float2* wpart;                   // weight-gradient partials [WG_SPLIT][max Cout*Cin*9 + Cout]
  double* lpart;                   // per-sample [2] sums (||x0 - t||^2, ||t||^2)
  int step;                        // Adam step
  size_t bytes;
};

__device__ __forceinline__ float2 crelu2(float2 v) { return cmk(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f)); }

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ---------------------------------------------------------------------------
// Convolution: out[n][o] = bias[o] + sum_c sum_k Wp[o][c][k] g(in[n][c])(p + k - 1)
//   g = CReLU when in_relu, identity otherwise; then + resid[n][o] when given, and
//   each component zeroed where that component of mask[n][o] is not > 0 when given.
// CTA: a 16 x 16 pixel tile x 32 output channels; thread: 4 consecutive pixels of a
// row x 8 output channels (32 complex accumulators).  Input channels are staged 8 at
// a time with a one-pixel halo; a thread keeps 6 pixels of an input row in registers
// and reuses them for the 3 taps along x.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cnn_conv(const float2* __restrict__ in, const float2* __restrict__ Wp,
                                                  const float2* __restrict__ bias, const float2* __restrict__ resid,
                                                  const float2* __restrict__ mask, float2* __restrict__ out, int Cin,
                                                  int Cout, int H, int W, int in_relu) {
  __shared__ __align__(16) float2 sIn[CV_ICB][CV_T + 2][CV_SP];
  __shared__ __align__(16) float2 sW[CV_ICB][9][CV_OCB];
  const int tilesx = (W + CV_T - 1) / CV_T;
  const int tx0 = (blockIdx.x % tilesx) * CV_T, ty0 = (blockIdx.x / tilesx) * CV_T;
  const int oc0 = blockIdx.y * CV_OCB, n = blockIdx.z;
  const int tid = threadIdx.x;
  const int og = tid >> 6, pg = tid & 63;
  const int py = pg >> 2, px0 = (pg & 3) * 4;
  const size_t HW = (size_t)H * W;
  const float2* inn = in + (size_t)n * Cin * HW;
  float2 acc[4][8];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[j][o] = cmk(0.f, 0.f);
  for (int ic0 = 0; ic0 < Cin; ic0 += CV_ICB) {
    for (int e = tid; e < CV_ICB * (CV_T + 2) * (CV_T + 2); e += 256) {
      const int c = e / ((CV_T + 2) * (CV_T + 2)), rem = e - c * (CV_T + 2) * (CV_T + 2);
      const int yy = rem / (CV_T + 2), xx = rem - yy * (CV_T + 2);
      const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
      float2 v = cmk(0.f, 0.f);
      if (ic0 + c < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) {
        v = inn[(size_t)(ic0 + c) * HW + (size_t)gy * W + gx];
        if (in_relu) v = crelu2(v);
      }
      sIn[c][yy][xx] = v;
    }
    for (int e = tid; e < CV_ICB * 9 * CV_OCB; e += 256) {
      const int o = e % CV_OCB, k = (e / CV_OCB) % 9, c = e / (9 * CV_OCB);
      float2 v = cmk(0.f, 0.f);
      if (oc0 + o < Cout && ic0 + c < Cin) v = Wp[((size_t)(oc0 + o) * Cin + ic0 + c) * 9 + k];
      sW[c][k][o] = v;
    }
    __syncthreads();
    const int cn = min(CV_ICB, Cin - ic0);
    for (int c = 0; c < cn; ++c) {
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        float2 h[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) h[j] = sIn[c][py + ky][px0 + j];
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const float4* wq = reinterpret_cast<const float4*>(&sW[c][ky * 3 + kx][og * 8]);
          float2 w[8];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 t = wq[q];
            w[2 * q] = cmk(t.x, t.y);
            w[2 * q + 1] = cmk(t.z, t.w);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int o = 0; o < 8; ++o) cfma(acc[j][o], w[o], h[j + kx]);
        }
      }
    }
    __syncthreads();
  }
  const int gy = ty0 + py;
  if (gy >= H) return;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int oc = oc0 + og * 8 + o;
    if (oc >= Cout) continue;
    const float2 b = bias ? bias[oc] : cmk(0.f, 0.f);
    const size_t base = ((size_t)n * Cout + oc) * HW + (size_t)gy * W;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gx = tx0 + px0 + j;
      if (gx >= W) continue;
      float2 v = cadd(acc[j][o], b);
      if (resid) v = cadd(v, resid[base + gx]);
      if (mask) {
        const float2 mk = mask[base + gx];
        v = cmk(mk.x > 0.f ? v.x : 0.f, mk.y > 0.f ? v.y : 0.f);
      }
      out[base + gx] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Weight gradient: part[s][o][c][k] = sum over split s's pixels of G[n][o][p] conj(h[n][c][p+k-1]),
// part[s][Cout*Cin*9 + o] = sum G[n][o][p] (bias), h = CReLU(in) when in_relu.
// CTA = (32 output channels, 32 input channels, split s); thread = 4 output channels x
// 1 input channel x 9 taps.  Pixel tiles (8 x 16) of all samples are dealt to the splits
// in order; a thread slides a 3 x 3 window of h along each tile row.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cnn_wgrad(const float2* __restrict__ G, const float2* __restrict__ in,
                                                   float2* __restrict__ part, int n, int Cin, int Cout, int H, int W,
                                                   int in_relu) {
  extern __shared__ __align__(16) float2 wsm[];
  float2* sG = wsm;                                 // [WG_OCB][WG_TY][WG_TX]
  float2* sH = wsm + WG_OCB * WG_TY * WG_TX;        // [WG_ICB][WG_CP] (10 x 18 used)
  const int o0 = blockIdx.x * WG_OCB, c0 = blockIdx.y * WG_ICB, sp = blockIdx.z;
  const int tid = threadIdx.x, og = tid >> 5, cl = tid & 31;
  const int tilesx = (W + WG_TX - 1) / WG_TX, tilesy = (H + WG_TY - 1) / WG_TY;
  const long ntile = (long)n * tilesx * tilesy;
  const long t0 = ntile * sp / WG_SPLIT, t1 = ntile * (sp + 1) / WG_SPLIT;
  const size_t HW = (size_t)H * W;
  float2 acc[4][9];
  float2 bacc[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    bacc[a] = cmk(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[a][k] = cmk(0.f, 0.f);
  }
  for (long t = t0; t < t1; ++t) {
    const int s = (int)(t / (tilesx * tilesy)), r = (int)(t - (long)s * tilesx * tilesy);
    const int ty0 = (r / tilesx) * WG_TY, tx0 = (r % tilesx) * WG_TX;
    for (int e = tid; e < WG_OCB * WG_TY * WG_TX; e += 256) {
      const int o = e / (WG_TY * WG_TX), rem = e - o * WG_TY * WG_TX;
      const int yy = rem / WG_TX, xx = rem - yy * WG_TX;
      const int gy = ty0 + yy, gx = tx0 + xx;
      float2 v = cmk(0.f, 0.f);
      if (o0 + o < Cout && gy < H && gx < W) v = G[((size_t)s * Cout + o0 + o) * HW + (size_t)gy * W + gx];
      sG[e] = v;
    }
    for (int e = tid; e < WG_ICB * (WG_TY + 2) * (WG_TX + 2); e += 256) {
      const int c = e / ((WG_TY + 2) * (WG_TX + 2)), rem = e - c * (WG_TY + 2) * (WG_TX + 2);
      const int yy = rem / (WG_TX + 2), xx = rem - yy * (WG_TX + 2);
      const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
      float2 v = cmk(0.f, 0.f);
      if (c0 + c < Cin && gy >= 0 && gy < H && gx >= 0 && gx < W) {
        v = in[((size_t)s * Cin + c0 + c) * HW + (size_t)gy * W + gx];
        if (in_relu) v = crelu2(v);
      }
      sH[c * WG_CP + yy * (WG_TX + 2) + xx] = v;
    }
    __syncthreads();
    const float2* hc = sH + cl * WG_CP;
    for (int yy = 0; yy < WG_TY; ++yy) {
      float2 win[3][3];  // h at rows yy..yy+2, columns xx..xx+2 of the staged tile
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        win[ky][1] = hc[(yy + ky) * (WG_TX + 2) + 0];
        win[ky][2] = hc[(yy + ky) * (WG_TX + 2) + 1];
      }
#pragma unroll 4
      for (int xx = 0; xx < WG_TX; ++xx) {
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          win[ky][0] = win[ky][1];
          win[ky][1] = win[ky][2];
          win[ky][2] = hc[(yy + ky) * (WG_TX + 2) + xx + 2];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 g = sG[((og * 4 + a) * WG_TY + yy) * WG_TX + xx];
          bacc[a] = cadd(bacc[a], g);
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) cfmacj(acc[a][ky * 3 + kx], win[ky][kx], g);
        }
      }
    }
    __syncthreads();
  }
  const size_t stride = (size_t)Cout * Cin * 9 + Cout;
  float2* ps = part + (size_t)sp * stride;
  const int c = c0 + cl;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int o = o0 + og * 4 + a;
    if (o >= Cout) continue;
    if (c < Cin)
#pragma unroll
      for (int k = 0; k < 9; ++k) ps[((size_t)o * Cin + c) * 9 + k] = acc[a][k];
    if (blockIdx.y == 0 && cl == 0) ps[(size_t)Cout * Cin * 9 + o] = bacc[a];
  }
}

// grad[i] = scale * sum_s part[s][i] in a fixed order
__global__ void k_cnn_wgrad_reduce(const float2* __restrict__ part, float2* __restrict__ grad, size_t count,
                                   float scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int s = 0; s < WG_SPLIT; ++s) {
      const float2 v = part[(size_t)s * count + i];
      re += v.x;
      im += v.y;
    }
    grad[i] = cmk((float)(re * scale), (float)(im * scale));
  }
}

// wt[c][o][k] = conj(W[o][c][8 - k]): the convolution whose output is dh
__global__ void k_cnn_wt(const float2* __restrict__ Wk, float2* __restrict__ wt, int Cin, int Cout) {
  const int total = Cout * Cin * 9;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int k = e % 9, o = (e / 9) % Cout, c = e / (9 * Cout);
    wt[e] = conjf2(Wk[((size_t)o * Cin + c) * 9 + (8 - k)]);
  }
}

// per-sample sums ||x0 - t||^2 and ||t||^2 (one CTA per sample, fixed order)
__global__ void __launch_bounds__(256) k_cnn_loss_sums(const float2* __restrict__ x0, const float2* __restrict__ t,
                                                       size_t per, double* __restrict__ sums) {
  __shared__ double r0[256], r1[256];
  const float2* a = x0 + (size_t)blockIdx.x * per;
  const float2* b = t + (size_t)blockIdx.x * per;
  double s0 = 0.0, s1 = 0.0;
  for (size_t e = threadIdx.x; e < per; e += 256) {
    const float2 u = a[e], v = b[e];
    const float dx = u.x - v.x, dy = u.y - v.y;
    s0 += (double)(dx * dx + dy * dy);
    s1 += (double)(v.x * v.x + v.y * v.y);
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[2 * blockIdx.x] = r0[0];
    sums[2 * blockIdx.x + 1] = r1[0];
  }
}

// G = 2 (x0 - t) / ||t||^2 of each sample (the gradient of its loss)
__global__ void k_cnn_loss_grad(const float2* __restrict__ x0, const float2* __restrict__ t, size_t per,
                                const double* __restrict__ sums, float2* __restrict__ G) {
  const size_t total = per * gridDim.y;
  const int n = blockIdx.y;
  const float sc = (float)(2.0 / sums[2 * n + 1]);
  (void)total;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < per; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = (size_t)n * per + e;
    const float2 u = x0[i], v = t[i];
    G[i] = cmk(sc * (u.x - v.x), sc * (u.y - v.y));
  }
}

// Adam on the FP32 master weights; the BF16-rounded copy is what the convolutions use
__global__ void k_cnn_adam(float2* __restrict__ master, float2* __restrict__ wbf, const float2* __restrict__ grad,
                           float2* __restrict__ m1, float2* __restrict__ m2, size_t count, float lr, float c1,
                           float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 g = grad[i];
    float2 m = m1[i], v = m2[i], w = master[i];
    m = cmk(b1 * m.x + (1.f - b1) * g.x, b1 * m.y + (1.f - b1) * g.y);
    v = cmk(b2 * v.x + (1.f - b2) * g.x * g.x, b2 * v.y + (1.f - b2) * g.y * g.y);
    w.x -= lr * (m.x / c1) / (sqrtf(v.x / c2) + eps);
    w.y -= lr * (m.y / c1) / (sqrtf(v.y / c2) + eps);
    m1[i] = m;
    m2[i] = v;
    master[i] = w;
    wbf[i] = cmk(bf16r(w.x), bf16r(w.y));
  }
}

__global__ void k_cnn_round(const float2* __restrict__ master, float2* __restrict__ wbf, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 w = master[i];
    wbf[i] = cmk(bf16r(w.x), bf16r(w.y));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t wgrad_smem() { return (size_t)(WG_OCB * WG_TY * WG_TX + WG_ICB * WG_CP) * sizeof(float2); }

static smsm_status conv(const float2* in, const float2* Wp, const float2* bias, const float2* resid, const float2* mask,
                        float2* out, int n, int Cin, int Cout, int H, int W, int in_relu, cudaStream_t s) {
  const int tiles = ((W + CV_T - 1) / CV_T) * ((H + CV_T - 1) / CV_T);
  dim3 grid(tiles, (Cout + CV_OCB - 1) / CV_OCB, n);
  k_cnn_conv<<<grid, 256, 0, s>>>(in, Wp, bias, resid, mask, out, Cin, Cout, H, W, in_relu);
  SMSM_LAUNCH_CHECK("k_cnn_conv");
  return SMSM_OK;
}

static void cnn_free(smsm_cnn_s* c) {
  if (!c) return;
  void* ptrs[] = {c->master, c->wbf, c->grad, c->m1, c->m2, c->wt, c->gA, c->gB, c->wpart, c->lpart};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (float2* p : c->z)
    if (p) cudaFree(p);
  delete c;
}

template <typename T>
static smsm_status calloc_dev(smsm_cnn_s* c, T** p, size_t count) {
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    smsm_set_error("smsm_cnn_create: cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return SMSM_ERR_NOMEM;
  }
  c->bytes += bytes;
  e = cudaMemset(*p, 0, bytes);
  if (e != cudaSuccess) {
    smsm_set_error("smsm_cnn_create: %s", cudaGetErrorString(e));
    return SMSM_ERR_CUDA;
  }
  return SMSM_OK;
}

extern "C" smsm_status smsm_cnn_create(smsm_cnn_t* out, int channels, int width, int layers, int height, int wdt,
                                       int max_batch) {
  if (!out) {
    smsm_set_error("smsm_cnn_create: out is NULL");
    return SMSM_ERR_ARG;
  }
  *out = nullptr;
  if (channels < 1 || channels > 256 || width < 1 || width > 256 || layers < 1 || layers > 32 || height < 1 ||
      wdt < 1 || height > 4096 || wdt > 4096 || max_batch < 1 || max_batch > 4096) {
    smsm_set_error("smsm_cnn_create: need channels, width in [1, 256], layers in [1, 32], image sides in "
                   "[1, 4096], max_batch in [1, 4096]");
    return SMSM_ERR_ARG;
  }
  smsm_cnn_s* c = new smsm_cnn_s();
  c->B = channels;
  c->width = width;
  c->layers = layers;
  c->H = height;
  c->W = wdt;
  c->maxn = max_batch;
  cudaGetDevice(&c->dev);
  size_t off = 0, maxw = 0;
  for (int k = 0; k < layers; ++k) {
    const int ci = k == 0 ? channels : width, co = k + 1 == layers ? channels : width;
    c->cin.push_back(ci);
    c->cout.push_back(co);
    c->woff.push_back(off);
    off += (size_t)co * ci * 9;
    c->boff.push_back(off);
    off += co;
    maxw = maxw > (size_t)co * ci * 9 + co ? maxw : (size_t)co * ci * 9 + co;
  }
  c->count = off;
  const size_t HW = (size_t)height * wdt;
  const int wmax = width > channels ? width : channels;
  smsm_status st = SMSM_OK;
  if (!st) st = calloc_dev(c, &c->master, off);
  if (!st) st = calloc_dev(c, &c->wbf, off);
  if (!st) st = calloc_dev(c, &c->grad, off);
  if (!st) st = calloc_dev(c, &c->m1, off);
  if (!st) st = calloc_dev(c, &c->m2, off);
  if (!st) st = calloc_dev(c, &c->wt, maxw);
  c->z.assign(layers, nullptr);
  for (int k = 0; k < layers && !st; ++k) st = calloc_dev(c, &c->z[k], (size_t)max_batch * c->cout[k] * HW);
  if (!st) st = calloc_dev(c, &c->gA, (size_t)max_batch * wmax * HW);
  if (!st) st = calloc_dev(c, &c->gB, (size_t)max_batch * wmax * HW);
  if (!st) st = calloc_dev(c, &c->wpart, (size_t)WG_SPLIT * maxw);
  if (!st) st = calloc_dev(c, &c->lpart, (size_t)2 * max_batch);
  if (!st) {
    cudaError_t e = cudaFuncSetAttribute(k_cnn_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem());
    if (e != cudaSuccess) {
      smsm_set_error("smsm_cnn_create: %s", cudaGetErrorString(e));
      st = SMSM_ERR_CUDA;
    }
  }
  if (st) {
    cnn_free(c);
    return st;
  }
  *out = c;
  return SMSM_OK;
}

smsm_status cnn_shape(const smsm_cnn_s* c, int* B, int* H, int* W, int* maxn) {
  *B = c->B;
  *H = c->H;
  *W = c->W;
  *maxn = c->maxn;
  return SMSM_OK;
}

extern "C" smsm_status smsm_cnn_destroy(smsm_cnn_t cnn) {
  cnn_free(cnn);
  return SMSM_OK;
}

extern "C" size_t smsm_cnn_param_count(smsm_cnn_t cnn) { return cnn ? cnn->count : 0; }

static smsm_status check_cnn(smsm_cnn_t cnn, const char* fn, int n) {
  if (!cnn) {
    smsm_set_error("%s: cnn is NULL", fn);
    return SMSM_ERR_ARG;
  }
  if (n < 0 || n > cnn->maxn) {
    smsm_set_error("%s: batch %d outside [0, %d]", fn, n, cnn->maxn);
    return SMSM_ERR_ARG;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != cnn->dev) {
    smsm_set_error("%s: the network lives on device %d, the current device is %d", fn, cnn->dev, dev);
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

static bool al16(const void* p) { return p && ((uintptr_t)p & 15u) == 0; }

extern "C" smsm_status smsm_cnn_set_params(smsm_cnn_t cnn, const void* params, void* stream) {
  smsm_status st;
  if ((st = check_cnn(cnn, "smsm_cnn_set_params", 0))) return st;
  if (!al16(params)) {
    smsm_set_error("smsm_cnn_set_params: params must be a 16-byte aligned device pointer");
    return SMSM_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SMSM_CUDA_TRY(cudaMemcpyAsync(cnn->master, params, cnn->count * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  SMSM_CUDA_TRY(cudaMemsetAsync(cnn->m1, 0, cnn->count * sizeof(float2), s));
  SMSM_CUDA_TRY(cudaMemsetAsync(cnn->m2, 0, cnn->count * sizeof(float2), s));
  cnn->step = 0;
  k_cnn_round<<<256, 256, 0, s>>>(cnn->master, cnn->wbf, cnn->count);
  SMSM_LAUNCH_CHECK("k_cnn_round");
  return SMSM_OK;
}

extern "C" smsm_status smsm_cnn_get_params(smsm_cnn_t cnn, void* params, void* stream) {
  smsm_status st;
  if ((st = check_cnn(cnn, "smsm_cnn_get_params", 0))) return st;
  if (!al16(params)) {
    smsm_set_error("smsm_cnn_get_params: params must be a 16-byte aligned device pointer");
    return SMSM_ERR_ARG;
  }
  SMSM_CUDA_TRY(cudaMemcpyAsync(params, cnn->master, cnn->count * sizeof(float2), cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
  return SMSM_OK;
}

// forward through every layer, keeping the pre-activations in z; x0 = a + z_last
static smsm_status cnn_forward(smsm_cnn_s* c, const float2* a, float2* x0, int n, cudaStream_t s) {
  smsm_status st;
  const float2* h = a;
  for (int k = 0; k < c->layers; ++k) {
    const bool last = k + 1 == c->layers;
    float2* o = last ? x0 : c->z[k];
    if ((st = conv(h, c->wbf + c->woff[k], c->wbf + c->boff[k], last ? a : nullptr, nullptr, o, n, c->cin[k],
                   c->cout[k], c->H, c->W, k > 0, s)))
      return st;
    h = c->z[k];
  }
  return SMSM_OK;
}

extern "C" smsm_status smsm_cnn_forward(smsm_cnn_t cnn, const void* a, void* x0, int n, void* stream) {
  smsm_status st;
  if ((st = check_cnn(cnn, "smsm_cnn_forward", n))) return st;
  if (!al16(a) || !al16(x0) || a == x0) {
    smsm_set_error("smsm_cnn_forward: a and x0 must be distinct 16-byte aligned device pointers");
    return SMSM_ERR_ARG;
  }
  if (n == 0) return SMSM_OK;
  return cnn_forward(cnn, (const float2*)a, (float2*)x0, n, (cudaStream_t)stream);
}

// loss (mean over the batch) and its gradients into cnn->grad; x0 lands in z[last]
static smsm_status cnn_backward(smsm_cnn_s* c, const float2* a, const float2* t, int n, double* loss,
                                cudaStream_t s) {
  smsm_status st;
  const int Lk = c->layers;
  const size_t HW = (size_t)c->H * c->W, per = (size_t)c->B * HW;
  float2* x0 = c->z[Lk - 1];
  if ((st = cnn_forward(c, a, x0, n, s))) return st;
  k_cnn_loss_sums<<<n, 256, 0, s>>>(x0, t, per, c->lpart);
  SMSM_LAUNCH_CHECK("k_cnn_loss_sums");
  float2* G = c->gA;
  float2* Gn = c->gB;
  k_cnn_loss_grad<<<dim3(64, n), 256, 0, s>>>(x0, t, per, c->lpart, G);
  SMSM_LAUNCH_CHECK("k_cnn_loss_grad");
  for (int k = Lk - 1; k >= 0; --k) {
    const int ci = c->cin[k], co = c->cout[k];
    const float2* h = k == 0 ? a : c->z[k - 1];
    dim3 gw((co + WG_OCB - 1) / WG_OCB, (ci + WG_ICB - 1) / WG_ICB, WG_SPLIT);
    k_cnn_wgrad<<<gw, 256, wgrad_smem(), s>>>(G, h, c->wpart, n, ci, co, c->H, c->W, k > 0);
    SMSM_LAUNCH_CHECK("k_cnn_wgrad");
    const size_t cnt = (size_t)co * ci * 9 + co;  // W_k and b_k are contiguous
    k_cnn_wgrad_reduce<<<(int)((cnt + 255) / 256), 256, 0, s>>>(c->wpart, c->grad + c->woff[k], cnt, 1.f / n);
    SMSM_LAUNCH_CHECK("k_cnn_wgrad_reduce");
    if (k > 0) {
      k_cnn_wt<<<(int)(((size_t)co * ci * 9 + 255) / 256), 256, 0, s>>>(c->wbf + c->woff[k], c->wt, ci, co);
      SMSM_LAUNCH_CHECK("k_cnn_wt");
      // dh_{k} = conv(G, wt); times the CReLU mask of z_{k-1}: the gradient of z_{k-1}
      if ((st = conv(G, c->wt, nullptr, nullptr, c->z[k - 1], Gn, n, co, ci, c->H, c->W, 0, s))) return st;
      float2* tmp = G;
      G = Gn;
      Gn = tmp;
    }
  }
  if (loss) {
    std::vector<double> h(2 * (size_t)n);
    SMSM_CUDA_TRY(cudaMemcpyAsync(h.data(), c->lpart, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    SMSM_CUDA_TRY(cudaStreamSynchronize(s));
    double L = 0.0;
    for (int i = 0; i < n; ++i) L += h[2 * i] / h[2 * i + 1];
    *loss = L / n;
  }
  return SMSM_OK;
}

static smsm_status check_train_args(smsm_cnn_t cnn, const char* fn, const void* a, const void* t, int n) {
  smsm_status st;
  if ((st = check_cnn(cnn, fn, n))) return st;
  if (n < 1 || !al16(a) || !al16(t)) {
    smsm_set_error("%s: need n >= 1 and 16-byte aligned device pointers a, t", fn);
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

extern "C" smsm_status smsm_cnn_gradients(smsm_cnn_t cnn, const void* a, const void* t, int n, void* grad,
                                          double* loss, void* stream) {
  smsm_status st;
  if ((st = check_train_args(cnn, "smsm_cnn_gradients", a, t, n))) return st;
  if (!al16(grad)) {
    smsm_set_error("smsm_cnn_gradients: grad must be a 16-byte aligned device pointer");
    return SMSM_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = cnn_backward(cnn, (const float2*)a, (const float2*)t, n, loss, s))) return st;
  SMSM_CUDA_TRY(cudaMemcpyAsync(grad, cnn->grad, cnn->count * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  return SMSM_OK;
}

extern "C" smsm_status smsm_cnn_train_step(smsm_cnn_t cnn, const void* a, const void* t, int n, float lr,
                                           double* loss, void* stream) {
  smsm_status st;
  if ((st = check_train_args(cnn, "smsm_cnn_train_step", a, t, n))) return st;
  if (!(lr > 0.f)) {
    smsm_set_error("smsm_cnn_train_step: learning rate must be > 0");
    return SMSM_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = cnn_backward(cnn, (const float2*)a, (const float2*)t, n, loss, s))) return st;
  cnn->step += 1;
  const float c1 = 1.f - powf(0.9f, (float)cnn->step), c2 = 1.f - powf(0.999f, (float)cnn->step);
  k_cnn_adam<<<512, 256, 0, s>>>(cnn->master, cnn->wbf, cnn->grad, cnn->m1, cnn->m2, cnn->count, lr, c1, c2);
  SMSM_LAUNCH_CHECK("k_cnn_adam");
  return SMSM_OK;
}
