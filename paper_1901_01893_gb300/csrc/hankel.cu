// Hankel-structured kernels of SMS-MUSSELS (Eqs. 8-10 of the paper).
//
//  * Gram  G_l = H_l^H H_l,  G[(i,p),(i',q)] = sum_{k in V} conj(x_i[k+p]) x_i'[k+q],
//    V = [0, N-r]^2 (VALID patches, the (N1-r+1)(N2-r+1) rows of Eq. 8).  The
//    Hankel matrix is never formed: each CTA stages a (16+r-1)^2 window of
//    every shot in shared memory and gathers the patch entries from it.
//  * Penalty  P_W(x)_l = H_l^*(H_l(x_l) W_l).  For an output pixel n whose
//    patches are all valid (n in [r-1, N-r]^2) it is the multichannel
//    correlation  sum_i' sum_d wt_ii'[d] x_i'[n+d],  wt_ii'[d] = sum_{q-p=d}
//    W[(i',q),(i,p)].  Periodically extended, that correlation is diagonal in
//    the image domain: out_img_i = sum_i' m_ii' img_i' with
//    m_ii'[y] = sum_d wt_ii'[d] exp(-j 2 pi d.(y - N/2)/N).  The column stage
//    applies m (see operators.cu); k_band then replaces the periodic value
//    by the exact one on the border band (pixels within r-1 of an edge), using
//    per-position "class" filters that only sum the valid patches.
#include "common.cuh"

// ---------------------------------------------------------------------------
// Gram
// ---------------------------------------------------------------------------
#define GT 48   // output tile edge (rows/cols of G per CTA)
#define GCH 16  // patch-origin chunk edge

__global__ void __launch_bounds__(256) k_gram_part(const float2* __restrict__ x, double2* __restrict__ part, int Ns,
                                                   int N, int r, int C, int P1, int nkx, int tside) {
  extern __shared__ float2 xs[];
  const int TW = GCH + r - 1;  // window edge
  const int l = blockIdx.z;
  int t = blockIdx.y, ta = 0;
  while (t >= tside - ta) {
    t -= tside - ta;
    ++ta;
  }
  const int tb = ta + t;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int rr = r * r;
  int offR[3], offC[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    int rho = ta * GT + ty + 16 * u;
    int kap = tb * GT + tx + 16 * u;
    if (rho >= C) rho = 0;
    if (kap >= C) kap = 0;
    int i = rho / rr, p = rho - i * rr;
    offR[u] = i * TW * TW + (p / r) * TW + (p % r);
    i = kap / rr;
    p = kap - i * rr;
    offC[u] = i * TW * TW + (p / r) * TW + (p % r);
  }
  double2 accd[3][3];
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 3; ++v) accd[u][v] = make_double2(0.0, 0.0);

  const int kx0 = blockIdx.x * GCH;
  const int nkxv = min(GCH, P1 - kx0);
  const float2* xl = x + (size_t)l * Ns * N * N;
  for (int ky0 = 0; ky0 < P1; ky0 += GCH) {
    const int nkyv = min(GCH, P1 - ky0);
    __syncthreads();
    for (int e = threadIdx.x; e < Ns * TW * TW; e += blockDim.x) {
      int i = e / (TW * TW), rem = e - i * TW * TW;
      int yy = rem / TW, xx = rem - yy * TW;
      int gy = ky0 + yy, gx = kx0 + xx;
      xs[e] = (gy < N && gx < N) ? xl[((size_t)i * N + gy) * N + gx] : cmk(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) acc[u][v] = cmk(0.f, 0.f);
    for (int py = 0; py < nkyv; ++py) {
      for (int px = 0; px < nkxv; ++px) {
        const int base = py * TW + px;
        float2 A[3], Bv[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) A[u] = xs[base + offR[u]];
#pragma unroll
        for (int v = 0; v < 3; ++v) Bv[v] = xs[base + offC[v]];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int v = 0; v < 3; ++v) cfmacj(acc[u][v], A[u], Bv[v]);
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        accd[u][v].x += acc[u][v].x;
        accd[u][v].y += acc[u][v].y;
      }
  }
  double2* out = part + ((size_t)l * nkx + blockIdx.x) * C * C;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    int rho = ta * GT + ty + 16 * u;
    if (rho >= C) continue;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      int kap = tb * GT + tx + 16 * v;
      if (kap < C) out[(size_t)rho * C + kap] = accd[u][v];
    }
  }
}

// G[rho][kap] = sum over chunks (fixed order, FP64); the lower triangle is the
// conjugate of the upper one, so G is exactly Hermitian with a real diagonal.
__global__ void k_gram_reduce(const double2* __restrict__ part, double2* __restrict__ G, int L, int C, int nkx) {
  const size_t total = (size_t)L * C * C;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int l = (int)(e / ((size_t)C * C));
    int rem = (int)(e - (size_t)l * C * C);
    int rho = rem / C, kap = rem - rho * C;
    int a = rho <= kap ? rho : kap, b = rho <= kap ? kap : rho;
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < nkx; ++k) {
      double2 v = part[(((size_t)l * nkx + k) * C + a) * C + b];
      sx += v.x;
      sy += v.y;
    }
    if (rho > kap) sy = -sy;
    if (rho == kap) sy = 0.0;
    G[e] = make_double2(sx, sy);
  }
}

smsm_status launch_gram(const smsm_plan_s* P, const float2* x, double2* G, cudaStream_t s) {
  const int tside = (P->C + GT - 1) / GT;
  const int ntile = tside * (tside + 1) / 2;
  const int nkx = P->gram_nkx;
  const int TW = GCH + P->r - 1;
  size_t sm = (size_t)P->Ns * TW * TW * sizeof(float2);
  dim3 grid(nkx, ntile, P->LD);
  k_gram_part<<<grid, 256, sm, s>>>(x, P->Gpart, P->Ns, P->N, P->r, P->C, P->P1, nkx, tside);
  SMSM_LAUNCH_CHECK("k_gram_part");
  k_gram_reduce<<<256, 256, 0, s>>>(P->Gpart, G, P->LD, P->C, nkx);
  SMSM_LAUNCH_CHECK("k_gram_reduce");
  return SMSM_OK;
}

// ---------------------------------------------------------------------------
// Filters from W.
//   class c in [0, R2) per axis, R2 = 2r-1: c < r-1 -> pixel c from the low
//   edge; c == r-1 -> interior; c > r-1 -> pixel N-r + (c-(r-1)) near the
//   high edge.  Valid patch offsets p in [max(0, c-(r-1)), min(r-1, c)].
//   wcls[l][cy*R2+cx][i][i'][d], wper[l][i][i'][d] (= the interior class),
//   d = (dy + r-1)*R2 + (dx + r-1).
// ---------------------------------------------------------------------------
__global__ void k_filters(const float2* __restrict__ W, float2* __restrict__ wcls, float2* __restrict__ wper, int Ns,
                          int r, int C) {
  const int R2 = 2 * r - 1;
  const int cls = blockIdx.x;  // 0..R2*R2 (last = periodic copy)
  const int ij = blockIdx.y;
  const int l = blockIdx.z;
  const int i = ij / Ns, j = ij - i * Ns;
  const bool per = (cls == R2 * R2);
  const int cy = per ? r - 1 : cls / R2, cx = per ? r - 1 : cls % R2;
  const int ly = max(0, cy - (r - 1)), hy = min(r - 1, cy);
  const int lx = max(0, cx - (r - 1)), hx = min(r - 1, cx);
  const float2* Wl = W + (size_t)l * C * C;
  const int rr = r * r;
  for (int d = threadIdx.x; d < R2 * R2; d += blockDim.x) {
    const int dy = d / R2 - (r - 1), dx = d % R2 - (r - 1);
    float2 s = cmk(0.f, 0.f);
    for (int py = ly; py <= hy; ++py) {
      const int qy = py + dy;
      if (qy < 0 || qy >= r) continue;
      for (int px = lx; px <= hx; ++px) {
        const int qx = px + dx;
        if (qx < 0 || qx >= r) continue;
        s = cadd(s, Wl[(size_t)(j * rr + qy * r + qx) * C + (i * rr + py * r + px)]);
      }
    }
    if (per)
      wper[((size_t)(l * Ns + i) * Ns + j) * R2 * R2 + d] = s;
    else
      wcls[(((size_t)l * R2 * R2 + cls) * Ns * Ns + ij) * R2 * R2 + d] = s;
  }
}

// multT[l][i][i'][x][y] = sum_dy E[dy][y] sum_dx wt[dy][dx] E[dx][x],  E[d][n] = exp(-j 2 pi (d-(r-1)) (n - N/2)/N)
#define MULT_XB 8
__global__ void __launch_bounds__(256) k_mult(const float2* __restrict__ wper, const float2* __restrict__ E,
                                              float2* __restrict__ multT, int Ns, int N, int r) {
  const int R2 = 2 * r - 1;
  __shared__ float2 wt[23 * 23];
  __shared__ float2 T[23][MULT_XB];
  const int x0 = blockIdx.x * MULT_XB;
  const int ij = blockIdx.y, l = blockIdx.z;
  const size_t fb = ((size_t)l * Ns * Ns + ij);
  for (int e = threadIdx.x; e < R2 * R2; e += blockDim.x) wt[e] = wper[fb * R2 * R2 + e];
  __syncthreads();
  for (int e = threadIdx.x; e < R2 * MULT_XB; e += blockDim.x) {
    int dy = e / MULT_XB, xl = e - dy * MULT_XB;
    float2 s = cmk(0.f, 0.f);
    if (x0 + xl < N)
      for (int dx = 0; dx < R2; ++dx) cfma(s, wt[dy * R2 + dx], E[(size_t)dx * N + x0 + xl]);
    T[dy][xl] = s;
  }
  __syncthreads();
  float2* out = multT + fb * (size_t)N * N;
  for (int e = threadIdx.x; e < MULT_XB * N; e += blockDim.x) {
    int xl = e / N, y = e - xl * N;
    if (x0 + xl >= N) continue;
    float2 s = cmk(0.f, 0.f);
    for (int dy = 0; dy < R2; ++dy) cfma(s, E[(size_t)dy * N + y], T[dy][xl]);
    out[(size_t)(x0 + xl) * N + y] = s;
  }
}

__global__ void k_c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = cmk((float)in[e].x, (float)in[e].y);
}

smsm_status launch_w_from_c128(const smsm_plan_s* P, const double2* W64, float2* W, cudaStream_t s) {
  k_c128_to_c64<<<128, 256, 0, s>>>(W64, W, (size_t)P->LD * P->C * P->C);
  SMSM_LAUNCH_CHECK("k_c128_to_c64");
  return SMSM_OK;
}

smsm_status launch_filters(const smsm_plan_s* P, const float2* W, cudaStream_t s) {
  const int R2 = P->R2;
  dim3 g1(R2 * R2 + 1, P->Ns * P->Ns, P->LD);
  k_filters<<<g1, 128, 0, s>>>(W, P->wcls, P->wper, P->Ns, P->r, P->C);
  SMSM_LAUNCH_CHECK("k_filters");
  dim3 g2((P->N + MULT_XB - 1) / MULT_XB, P->Ns * P->Ns, P->LD);
  k_mult<<<g2, 256, 0, s>>>(P->wper, P->Etab, P->multT, P->Ns, P->N, P->r);
  SMSM_LAUNCH_CHECK("k_mult");
  return SMSM_OK;
}

// ---------------------------------------------------------------------------
// Border band: out[n] += scale * (P_valid(x)[n] - P_periodic(x)[n]) for the
// pixels within r-1 of an edge; optional partial of Re<x, scale*corr>.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void band_pixel(int b, int N, int r, int& ny, int& nx) {
  const int w = r - 1;
  const int top = 2 * w * N;
  if (b < top) {
    int row = b / N;
    nx = b - row * N;
    ny = row < w ? row : N - w + (row - w);
  } else {
    int b2 = b - top;
    int row = b2 / (2 * w), c = b2 - row * (2 * w);
    ny = w + row;
    nx = c < w ? c : N - w + (c - w);
  }
}

__device__ __forceinline__ int pix_class(int n, int N, int r) {
  if (n < r - 1) return n;
  if (n <= N - r) return r - 1;
  return r - 1 + (n - (N - r));
}

__global__ void __launch_bounds__(256) k_band(const float2* __restrict__ x, float2* __restrict__ out,
                                              const float2* __restrict__ wper, const float2* __restrict__ wcls,
                                              int L, int Ns, int N, int r, int nband, float scale,
                                              double* __restrict__ dot_part) {
  __shared__ double red[256];
  const int R2 = 2 * r - 1;
  const int total = L * nband * Ns;  // per direction
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double dsum = 0.0;
  if (idx < total) {
    const int i = idx % Ns;
    const int t = idx / Ns;
    const int bp = t % nband, l = blockIdx.y * L + t / nband;  // flat (direction, slice)
    int ny, nx;
    band_pixel(bp, N, r, ny, nx);
    const int cls = pix_class(ny, N, r) * R2 + pix_class(nx, N, r);
    float2 corr = cmk(0.f, 0.f);
    for (int j = 0; j < Ns; ++j) {
      const float2* wc = wcls + (((size_t)l * R2 * R2 + cls) * Ns * Ns + i * Ns + j) * R2 * R2;
      const float2* wp = wper + ((size_t)(l * Ns + i) * Ns + j) * R2 * R2;
      const float2* xj = x + (size_t)(l * Ns + j) * N * N;
      for (int dy = 0; dy < R2; ++dy) {
        int yy = ny + dy - (r - 1);
        bool iny = (yy >= 0 && yy < N);
        int yw = yy < 0 ? yy + N : (yy >= N ? yy - N : yy);
        for (int dx = 0; dx < R2; ++dx) {
          int xx = nx + dx - (r - 1);
          bool inx = (xx >= 0 && xx < N);
          int xw = xx < 0 ? xx + N : (xx >= N ? xx - N : xx);
          float2 v = xj[(size_t)yw * N + xw];
          const int d = dy * R2 + dx;
          float2 w = wp[d];
          if (iny && inx) w = csub(w, wc[d]);
          // corr -= (wper - wcls) v  on in-range taps, corr -= wper v on wrapped taps
          corr.x -= w.x * v.x - w.y * v.y;
          corr.y -= w.x * v.y + w.y * v.x;
        }
      }
    }
    corr = cscale(corr, scale);
    const size_t o = (size_t)(l * Ns + i) * N * N + (size_t)ny * N + nx;
    out[o] = cadd(out[o], corr);
    if (dot_part) {
      float2 xv = x[o];
      dsum = (double)xv.x * corr.x + (double)xv.y * corr.y;
    }
  }
  if (dot_part) {
    red[threadIdx.x] = dsum;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) dot_part[(size_t)blockIdx.y * SMSM_PART_MAX + blockIdx.x] = red[0];
  }
}

int band_blocks(const smsm_plan_s* P) { return (P->L * P->nband * P->Ns + 255) / 256; }

smsm_status launch_band(const smsm_plan_s* P, const float2* x, float2* out, float scale, double* dot_part,
                        cudaStream_t s) {
  const int nb = band_blocks(P);
  if (nb <= 0) return SMSM_OK;
  k_band<<<dim3(nb, P->D), 256, 0, s>>>(x, out, P->wper, P->wcls, P->L, P->Ns, P->N, P->r, P->nband, scale,
                                        dot_part);
  SMSM_LAUNCH_CHECK("k_band");
  return SMSM_OK;
}
