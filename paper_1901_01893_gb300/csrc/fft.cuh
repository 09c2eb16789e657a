// Shared-memory batched FFT (mixed radix 2/3/4, Stockham autosort).
//
// Each pass with radix R over a length-n transform reads element j + r*n/R,
// applies the twiddle w^(r*k*n/(s*R)) (k = j mod s, s = product of the
// earlier radices, w = exp(-2 pi i/n)), does an R-point DFT, and writes
// element (j/s)*s*R + k + r*s of the other buffer.  After all passes the
// result is in natural order; no bit reversal is needed.  The twiddle table
// holds exp(-2 pi i k/n), k < n, computed on the host in FP64.
#pragma once
#include "common.cuh"

template <bool INV>
__device__ __forceinline__ float2 tw_get(const float2* tw, int idx) {
  float2 w = tw[idx];
  return INV ? conjf2(w) : w;
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
  // forward: X1 = a0 - i a1 - a2 + i a3 ; inverse swaps the sign of i
  float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
  // -i * d13 = (d13.y, -d13.x)
  float2 rot = INV ? cmk(-d13.y, d13.x) : cmk(d13.y, -d13.x);
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, rot);
  v[3] = csub(d02, rot);
}

// 8-point DFT in registers, natural order in and out: two 4-point DFTs of the even and odd
// elements, the odd ones turned by w8^k (w8 = exp(-+ 2 pi i / 8)), then one radix-2 step
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float h = 0.707106781186547524f;  // sqrt(1/2)
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // forward: w8 = h (1 - i), w8^2 = -i, w8^3 = h (-1 - i); inverse: their conjugates
  const float2 o1 = INV ? cmk(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                        : cmk(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
  const float2 o2 = INV ? cmk(-o[2].y, o[2].x) : cmk(o[2].y, -o[2].x);
  const float2 o3 = INV ? cmk(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                        : cmk(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  // X1 = a0 - t1/2 -+ i (sqrt3/2) t2, X2 = a0 - t1/2 +- i (sqrt3/2) t2, t1 = a1+a2, t2 = a1-a2
  const float h3 = 0.866025403784438647f;
  float2 t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
  float2 m = cmk(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  // -i * h3 * t2 = (h3 t2.y, -h3 t2.x)
  float2 j = INV ? cmk(-h3 * t2.y, h3 * t2.x) : cmk(h3 * t2.y, -h3 * t2.x);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, j);
  v[2] = csub(m, j);
}

// One radix-R pass (R in {2, 3, 4, 8}) of the Stockham FFT described above, with
// the transform length N, R and the product S of the earlier radices fixed at
// compile time (so every index division is by a constant); then the next pass.
// Radices are taken in the order 8, ..., 8, 4, 2, 3, ..., 3: fewer passes through
// shared memory than the runtime descriptor's 4, ..., 4, 2, 3, ..., 3 (used only for
// the lengths without a fixed chain).
template <bool INV, int N, int S>
__device__ __forceinline__ float2* fft_fixed_from(float2* src, float2* dst, int nbatch, int bstride,
                                                  const float2* tw) {
  if constexpr (S == N) {
    return src;
  } else {
    constexpr int REM = N / S;
    constexpr int R = (REM % 8 == 0) ? 8 : ((REM % 4 == 0) ? 4 : ((REM % 2 == 0) ? 2 : 3));
    constexpr int nR = N / R;
    constexpr int tstep = N / (S * R);
    const int ntask = nbatch * nR;
    for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
      const int bb = t / nR;
      const int j = t - bb * nR;
      const float2* Sp = src + bb * bstride;
      float2* Dp = dst + bb * bstride;
      const int k = j % S;
      const int base = (j - k) * R + k;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = Sp[j + r * nR];
      if (S > 1 && k) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_get<INV>(tw, r * k * tstep));
      }
      if constexpr (R == 8)
        dft8<INV>(v);
      else if constexpr (R == 4)
        dft4<INV>(v);
      else if constexpr (R == 2)
        dft2<INV>(v);
      else
        dft3<INV>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) Dp[base + r * S] = v[r];
    }
    __syncthreads();
    return fft_fixed_from<INV, N, S * R>(dst, src, nbatch, bstride, tw);
  }
}

// Batched FFT of `nbatch` transforms of length d.n; transform b starts at
// a + b*bstride (and b + b*bstride for the ping-pong buffer).  All threads
// of the block take part; the routine ends with __syncthreads() after every
// pass and returns the buffer that holds the result.  Unnormalised.  The
// common lengths run a compile-time pass chain.
template <bool INV>
__device__ float2* fft_smem(float2* a, float2* b, int nbatch, int bstride, const FftDesc& d,
                            const float2* tw) {
  switch (d.n) {
    case 64: return fft_fixed_from<INV, 64, 1>(a, b, nbatch, bstride, tw);
    case 96: return fft_fixed_from<INV, 96, 1>(a, b, nbatch, bstride, tw);
    case 128: return fft_fixed_from<INV, 128, 1>(a, b, nbatch, bstride, tw);
    case 192: return fft_fixed_from<INV, 192, 1>(a, b, nbatch, bstride, tw);
    case 256: return fft_fixed_from<INV, 256, 1>(a, b, nbatch, bstride, tw);
    default: break;
  }
  const int n = d.n;
  int s = 1;
  float2* src = a;
  float2* dst = b;
  for (int ps = 0; ps < d.np; ++ps) {
    const unsigned rc = (d.code >> (2 * ps)) & 3u;
    const int R = rc == 2u ? 4 : (rc == 1u ? 3 : 2);
    const int nR = n / R;
    const int tstep = n / (s * R);
    const int ntask = nbatch * nR;
    for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
      const int bb = t / nR;
      const int j = t - bb * nR;
      const float2* S = src + bb * bstride;
      float2* D = dst + bb * bstride;
      const int k = j % s;
      const int base = (j - k) * R + k;
      float2 v[4];
      if (R == 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = S[j + r * nR];
        if (k) {
#pragma unroll
          for (int r = 1; r < 4; ++r) v[r] = cmul(v[r], tw_get<INV>(tw, r * k * tstep));
        }
        dft4<INV>(v);
#pragma unroll
        for (int r = 0; r < 4; ++r) D[base + r * s] = v[r];
      } else if (R == 2) {
        v[0] = S[j];
        v[1] = S[j + nR];
        if (k) v[1] = cmul(v[1], tw_get<INV>(tw, k * tstep));
        dft2<INV>(v);
        D[base] = v[0];
        D[base + s] = v[1];
      } else {  // R == 3
#pragma unroll
        for (int r = 0; r < 3; ++r) v[r] = S[j + r * nR];
        if (k) {
          v[1] = cmul(v[1], tw_get<INV>(tw, k * tstep));
          v[2] = cmul(v[2], tw_get<INV>(tw, 2 * k * tstep));
        }
        dft3<INV>(v);
#pragma unroll
        for (int r = 0; r < 3; ++r) D[base + r * s] = v[r];
      }
    }
    __syncthreads();
    float2* t = src;
    src = dst;
    dst = t;
    s *= R;
  }
  return src;
}

// fft_smem as an out-of-line call: kernels instantiated many times over other
// template parameters share one copy of every pass chain
template <bool INV>
__device__ __noinline__ float2* fft_smem_call(float2* a, float2* b, int nbatch, int bstride, const FftDesc& d,
                                              const float2* tw) {
  return fft_smem<INV>(a, b, nbatch, bstride, d, tw);
}

// (-1)^n as a float
__device__ __forceinline__ float sgn_par(int n) { return (n & 1) ? -1.f : 1.f; }
