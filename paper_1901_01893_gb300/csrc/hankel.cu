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
                                                   int N, int r, int C, int P1, int nkx, int tside, int periodic) {
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
      if (periodic) {  // origins over all of [0, N)^2, indices mod N
        gy %= N;
        gx %= N;
      }
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
  if (P->gram_tc) return launch_gram_tc(P, x, G, s);
  const int tside = (P->C + GT - 1) / GT;
  const int ntile = tside * (tside + 1) / 2;
  const int nkx = P->gram_nkx;
  const int TW = GCH + P->r - 1;
  size_t sm = (size_t)P->Ns * TW * TW * sizeof(float2);
  dim3 grid(nkx, ntile, P->LD);
  k_gram_part<<<grid, 256, sm, s>>>(x, P->Gpart, P->Ns, P->N, P->r, P->C, P->P1, nkx, tside, P->periodic);
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
//   wper[l][i][i'][d]: periodic (interior) filter, d = (dy + r-1)*R2 + (dx + r-1).
//   dcls[l][cls][i'][d][i]: the border correction taps of class cls,
//     (tap in range ? class filter : 0) - periodic filter, applied to the
//     periodically wrapped x:  corr_i[n] = sum_{i',d} dcls * x_i'[(n + d) mod N].
//   A tap (dy, dx) is in range for class (cy, cx) when the pixel plus the tap
//   stays inside [0, N): dy >= -cy for low classes, dy <= 2r-2-cy for high ones.
// ---------------------------------------------------------------------------
// One CTA per (input shot j, matrix l): the rows (j, q) of W_l are staged in
// shared memory (row stride C+1); thread (d, i) forms, for its tap d and output
// shot i, the r x r array A[p] = W[(j, p+d), (i, p)] (0 where p+d leaves the
// support) and every class sum from running sums.  The valid-patch range of a
// class is a prefix [0, c] or a suffix [c-r+1, r-1] of p along each axis, so
// accumulating rows from the top (prefix classes) or from the bottom (suffix
// classes) and, within the rows accumulated so far, column prefix and suffix
// sums gives each class sum as one lookup.  The periodic filter is the full sum.
#define FILT_MAXR 12
__device__ __forceinline__ float2 filt_a(const float2* wi, int ldw, int r, int dy, int dx, int py, int px) {
  const int qy = py + dy, qx = px + dx;
  return (qy >= 0 && qy < r && qx >= 0 && qx < r) ? wi[(qy * r + qx) * ldw + py * r + px] : cmk(0.f, 0.f);
}

__global__ void __launch_bounds__(256) k_filters(const float2* __restrict__ W, float2* __restrict__ dcls,
                                                 float2* __restrict__ wper, int Ns, int r, int C, int classes) {
  extern __shared__ float2 sW[];  // [r*r (q)][C + 1]
  const int R2 = 2 * r - 1, RR = R2 * R2;
  const int j = blockIdx.x;
  const int l = blockIdx.y;
  const int rr = r * r;
  const int ldw = C + 1;
  const float2* Wl = W + (size_t)l * C * C + (size_t)j * rr * C;
  for (int e = threadIdx.x; e < rr * C; e += blockDim.x) {
    const int q = e / C, c = e - q * C;
    sW[q * ldw + c] = Wl[e];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < RR * Ns; t += blockDim.x) {
    const int i = t % Ns, d = t / Ns;
    const int dy = d / R2 - (r - 1), dx = d % R2 - (r - 1);
    const float2* wi = sW + i * rr;
    // periodic filter: the sum over every p
    float2 sp = cmk(0.f, 0.f);
    for (int py = 0; py < r; ++py)
      for (int px = 0; px < r; ++px) sp = cadd(sp, filt_a(wi, ldw, r, dy, dx, py, px));
    wper[((size_t)(l * Ns + i) * Ns + j) * RR + d] = sp;
    if (!classes) continue;  // periodic patches: no border band, no class taps
    float2* out = dcls + ((size_t)l * RR * Ns + j) * RR * Ns + (size_t)d * Ns + i;  // + cls * Ns * RR * Ns
    const size_t cstride = (size_t)Ns * RR * Ns;
    // pass 0: rows 0..cy (classes cy <= r-1); pass 1: rows cy-r+1..r-1 (classes cy >= r-1)
    for (int pass = 0; pass < 2; ++pass) {
      float2 cpre[FILT_MAXR], csuf[FILT_MAXR];  // column prefix / suffix sums over the rows so far
#pragma unroll
      for (int k = 0; k < FILT_MAXR; ++k) cpre[k] = csuf[k] = cmk(0.f, 0.f);
      for (int step = 0; step < r; ++step) {
        const int py = pass == 0 ? step : r - 1 - step;
        float2 run = cmk(0.f, 0.f);
#pragma unroll
        for (int px = 0; px < FILT_MAXR; ++px)
          if (px < r) {
            run = cadd(run, filt_a(wi, ldw, r, dy, dx, py, px));
            cpre[px] = cadd(cpre[px], run);
          }
        run = cmk(0.f, 0.f);
#pragma unroll
        for (int k = FILT_MAXR - 1; k >= 0; --k)
          if (k < r) {
            run = cadd(run, filt_a(wi, ldw, r, dy, dx, py, k));
            csuf[k] = cadd(csuf[k], run);
          }
        // rows so far: [0, step] (pass 0: class cy = step) or [r-1-step, r-1] (pass 1:
        // class cy = 2r-2-step, whose valid rows are [cy-r+1, r-1])
        const int cy = pass == 0 ? step : 2 * r - 2 - step;
        if (pass == 1 && step == r - 1) continue;  // cy = r-1 (all rows) came out of pass 0
        const bool iny = (cy < r - 1) ? (dy >= -cy) : (cy > r - 1 ? dy <= 2 * r - 2 - cy : true);
#pragma unroll
        for (int cx = 0; cx < 2 * FILT_MAXR - 1; ++cx)
          if (cx < R2) {
            // columns [0, cx] (cx <= r-1) or [cx-r+1, r-1] (cx >= r-1)
            const float2 sc = cx <= r - 1 ? cpre[cx < FILT_MAXR ? cx : 0] : csuf[cx - r + 1 < FILT_MAXR ? cx - r + 1 : 0];
            const bool inx = (cx < r - 1) ? (dx >= -cx) : (cx > r - 1 ? dx <= 2 * r - 2 - cx : true);
            out[(size_t)(cy * R2 + cx) * cstride] = (iny && inx) ? csub(sc, sp) : cscale(sp, -1.f);
          }
      }
    }
  }
}

static size_t filters_smem(const smsm_plan_s* P) { return (size_t)P->r * P->r * (P->C + 1) * sizeof(float2); }

// multT[l][pk(i,i')][x][y] = sum_dy E[dy][y] sum_dx wt_ii'[dy][dx] E[dx][x],  E[d][n] = exp(-j 2 pi (d-(r-1)) (n - N/2)/N),
// for i <= i' only (the multiplier is Hermitian in the shot pair); the diagonal planes are real.
#define MULT_XB 8
__global__ void __launch_bounds__(256) k_mult(const float2* __restrict__ wper, const float2* __restrict__ E,
                                              float2* __restrict__ multT, int Ns, int N, int r) {
  const int R2 = 2 * r - 1;
  __shared__ float2 wt[23 * 23];
  __shared__ float2 T[23][MULT_XB];
  const int x0 = blockIdx.x * MULT_XB;
  const int pk = blockIdx.y, l = blockIdx.z;
  int i = 0;
  while (mult_plane(i + 1, i + 1, Ns) <= pk) ++i;
  const int j = i + (pk - mult_plane(i, i, Ns));
  const size_t fb = (size_t)l * Ns * Ns + (size_t)i * Ns + j;
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
  float2* out = multT + ((size_t)l * mult_planes(Ns) + pk) * N * N;
  for (int e = threadIdx.x; e < MULT_XB * N; e += blockDim.x) {
    int xl = e / N, y = e - xl * N;
    if (x0 + xl >= N) continue;
    float2 s = cmk(0.f, 0.f);
    for (int dy = 0; dy < R2; ++dy) cfma(s, E[(size_t)dy * N + y], T[dy][xl]);
    if (i == j) s.y = 0.f;
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
  k_filters<<<dim3(P->Ns, P->LD), 256, filters_smem(P), s>>>(W, P->wcls, P->wper, P->Ns, P->r, P->C,
                                                              !P->periodic);  // wcls holds the class taps dcls
  SMSM_LAUNCH_CHECK("k_filters");
  dim3 g2((P->N + MULT_XB - 1) / MULT_XB, mult_planes(P->Ns), P->LD);
  k_mult<<<g2, 256, 0, s>>>(P->wper, P->Etab, P->multT, P->Ns, P->N, P->r);
  SMSM_LAUNCH_CHECK("k_mult");
  return SMSM_OK;
}

// ---------------------------------------------------------------------------
// Border band: out[n] += scale * (P_valid(x)[n] - P_periodic(x)[n]) for the
// pixels within r-1 of an edge, with the per-class taps dcls; optional
// partials of Re<x, scale*corr>.
// The band is four strips -- top (rows 0..r-2) and bottom (rows N-r+1..N-1),
// left and right (columns 0..r-2, N-r+1..N-1), each over the interior range
// [r-1, N-r] of the other coordinate -- plus the four (r-1) x (r-1) corners.
// Every pixel of a strip line has the same class, so k_band stages the line's
// taps once per CTA; the corner pixels each have their own class and are
// summed by k_band_corner.
// ---------------------------------------------------------------------------
#define BAND_P 2                  // pixels per thread
#define BAND_TX (32 * BAND_P)     // pixels per strip line per CTA

// One CTA = one chunk of BAND_TX pixels of one line of one strip; warp j sums
// the taps of input shot j for every output shot; the NS partials of each
// (pixel, output shot) are then added in a fixed order (deterministic).  The
// line's window of x (2r-1 lines across, BAND_TX + 2r-2 along, periodically
// wrapped) is staged in shared memory as [shot][across][along] for both
// orientations, and so are the line's taps [j][d][i] (read as broadcasts); both
// with asynchronous copies, all in flight at once.  Lane q owns the pixels
// q + 32 p (p < BAND_P), so the window reads of a warp are consecutive.
template <int NS>
__global__ void __launch_bounds__(32 * NS) k_band(const float2* __restrict__ x, float2* __restrict__ out,
                                                  const float2* __restrict__ dcls, int L, int N, int r, float scale,
                                                  double* __restrict__ dot_part) {
  extern __shared__ __align__(16) float2 bsm[];
  __shared__ double red[8];
  const int R2 = 2 * r - 1, w = r - 1;
  const int strip = blockIdx.y;  // 0 top, 1 bottom, 2 left, 3 right
  const int lf = blockIdx.z;     // flat (direction, slice)
  const int d = lf / L, l = lf - d * L;
  const int horiz = strip < 2;
  const int lo = (strip == 0 || strip == 2);
  const int nchunk = (N - 2 * w + BAND_TX - 1) / BAND_TX;
  const int line = blockIdx.x / nchunk, chunk = blockIdx.x - line * nchunk;
  const int tid = threadIdx.x, j = tid >> 5, lane = tid & 31;
  const int nt = blockDim.x;
  const int Wl = BAND_TX + R2 - 1;
  const int start = w + chunk * BAND_TX;  // first pixel along the line
  const int limit = N - w;
  const int fixed = (lo ? 0 : N - w) + line;
  const size_t NN = (size_t)N * N;
  const float2* xl = x + (size_t)lf * NS * NN;
  const int ntap = NS * R2 * R2 * NS;  // taps of one class
  const int cfix = lo ? line : r + line;  // class along the fixed coordinate
  const int clsline = horiz ? cfix * R2 + (r - 1) : (r - 1) * R2 + cfix;
  const float2* tl = dcls + ((size_t)lf * R2 * R2 + clsline) * ntap;
  float2* tsm = bsm;                               // [NS (j)][R2*R2][NS (i)]
  float2* xs = tsm + ((ntap + 1) & ~1);            // [NS][R2][Wl]
  float2* part = xs;                               // [NS (j)][BAND_TX][NS (i)], after the window is used
  for (int e = tid; e < ntap; e += nt) cp_async8(tsm + e, tl + e);
  // window rows (shot jj, across aa): one warp per row, lanes along the line.  Along the
  // line only [start - w, min(start + BAND_TX, limit) + w) is read by kept pixels: all of
  // it inside the image (the rest of the row is never written and only feeds discarded
  // pixels); across the line the window wraps periodically.
  const int Wv = min(Wl, limit - start + 2 * w);
  for (int row = j; row < NS * R2; row += nt >> 5) {
    const int jj = row / R2, aa = row - jj * R2;
    float2* dst = xs + (size_t)row * Wl;
    if (horiz) {
      int gy = fixed + aa - w;
      gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
      const float2* src = xl + (size_t)jj * NN + (size_t)gy * N + (start - w);
      for (int u = lane; u < Wv; u += 32) cp_async8(dst + u, src + u);
    } else {
      int gx = fixed + aa - w;
      gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
      const float2* src = xl + (size_t)jj * NN + (size_t)(start - w) * N + gx;
      for (int u = lane; u < Wv; u += 32) cp_async8(dst + u, src + (size_t)u * N);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  float2 acc[BAND_P][NS];
#pragma unroll
  for (int p = 0; p < BAND_P; ++p)
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[p][i] = cmk(0.f, 0.f);
  {
    const float2* taps = tsm + (size_t)j * R2 * R2 * NS;
    // tap (aa, bb) of the line is d = aa R2 + bb (horizontal strips) or bb R2 + aa
    const int tstep = (horiz ? 1 : R2) * NS;
    for (int aa = 0; aa < R2; ++aa) {
      const float2* xr = xs + ((size_t)j * R2 + aa) * Wl + lane;
      const float2* tp0 = taps + (size_t)(horiz ? aa * R2 : aa) * NS;
#pragma unroll 4
      for (int bb = 0; bb < R2; ++bb) {
        const float2* tp = tp0 + bb * tstep;
        float2 tv[NS];
        if (NS % 2 == 0 && (ntap % 2 == 0)) {
#pragma unroll
          for (int i = 0; i + 1 < NS; i += 2) {
            const float4 t4 = *reinterpret_cast<const float4*>(tp + i);
            tv[i] = cmk(t4.x, t4.y);
            tv[i + 1] = cmk(t4.z, t4.w);
          }
        } else {
#pragma unroll
          for (int i = 0; i < NS; ++i) tv[i] = tp[i];
        }
#pragma unroll
        for (int p = 0; p < BAND_P; ++p) {
          const float2 xv = xr[32 * p + bb];
#pragma unroll
          for (int i = 0; i < NS; ++i) cfma(acc[p][i], tv[i], xv);
        }
      }
    }
  }
  __syncthreads();  // the window is no longer read: part takes its place
#pragma unroll
  for (int p = 0; p < BAND_P; ++p)
#pragma unroll
    for (int i = 0; i < NS; ++i) part[((size_t)j * BAND_TX + lane + 32 * p) * NS + i] = acc[p][i];
  __syncthreads();
  double dsum = 0.0;
  for (int t = tid; t < BAND_TX * NS; t += nt) {
    const int pu = t / NS, i = t - pu * NS;
    const int pos = start + pu;
    if (pos >= limit) continue;
    float2 sacc = part[(size_t)pu * NS + i];
    for (int jj = 1; jj < NS; ++jj) sacc = cadd(sacc, part[((size_t)jj * BAND_TX + pu) * NS + i]);
    const int ny = horiz ? fixed : pos, nx = horiz ? pos : fixed;
    const size_t o = ((size_t)lf * NS + i) * NN + (size_t)ny * N + nx;
    const float2 c = cscale(sacc, scale);
    out[o] = cadd(out[o], c);
    if (dot_part) {
      const float2 xv = xl[(size_t)i * NN + (size_t)ny * N + nx];
      dsum += (double)xv.x * c.x + (double)xv.y * c.y;
    }
  }
  if (dot_part) {
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lane == 0) red[j] = dsum;
    __syncthreads();
    if (tid == 0) {
      double sacc = 0.0;
      for (int k = 0; k < (nt >> 5); ++k) sacc += red[k];
      dot_part[(size_t)d * SMSM_PART_MAX + ((size_t)l * 4 + strip) * gridDim.x + blockIdx.x] = sacc;
    }
  }
}

// One CTA per (corner pixel, corner, flat (direction, slice)): every corner
// pixel has its own class, so the CTA stages that class's taps [j][d][i] and the
// pixel's R2 x R2 window of every shot (periodically wrapped) with asynchronous
// copies, all in flight at once.  Thread (i, j, c) sums the taps d = c (mod nc)
// of input shot j for output shot i; the partials of output shot i are then
// added in a fixed order.
#define BAND_CORNER_THREADS 128
__global__ void __launch_bounds__(BAND_CORNER_THREADS) k_band_corner(const float2* __restrict__ x,
                                                                     float2* __restrict__ out,
                                                                     const float2* __restrict__ dcls, int L, int Ns,
                                                                     int N, int r, float scale,
                                                                     double* __restrict__ dot_part, int part_base) {
  extern __shared__ __align__(16) float2 csm[];
  const int R2 = 2 * r - 1, w = r - 1, RR = R2 * R2;
  const int pix = blockIdx.x;     // py * w + px
  const int corner = blockIdx.y;  // bit 0: right, bit 1: bottom
  const int lf = blockIdx.z;
  const int d = lf / L, l = lf - d * L;
  const int py = pix / w, px = pix - py * w;
  const int ny = ((corner & 2) ? N - w : 0) + py, nx = ((corner & 1) ? N - w : 0) + px;
  const int cy = (corner & 2) ? r + py : py, cx = (corner & 1) ? r + px : px;
  const size_t NN = (size_t)N * N;
  const float2* xl = x + (size_t)lf * Ns * NN;
  const int ntap = Ns * RR * Ns;
  const int tid = threadIdx.x, nt = blockDim.x;
  float2* tsm = csm;                     // [Ns (j)][RR][Ns (i)]
  float2* xw = tsm + ntap;               // [Ns][R2][R2]: pixel (ny + aa - w, nx + bb - w)
  float2* part = xw + (size_t)Ns * RR;   // [Ns (i)][Ns (j) * nc]
  const float2* ct = dcls + ((size_t)lf * RR + cy * R2 + cx) * ntap;
  for (int e = tid; e < ntap; e += nt) cp_async8(tsm + e, ct + e);
  for (int e = tid; e < Ns * RR; e += nt) {
    const int jj = e / RR, rem = e - jj * RR;
    const int aa = rem / R2, bb = rem - aa * R2;
    int gy = ny + aa - w, gx = nx + bb - w;
    gy = gy < 0 ? gy + N : (gy >= N ? gy - N : gy);
    gx = gx < 0 ? gx + N : (gx >= N ? gx - N : gx);
    cp_async8(xw + e, xl + (size_t)jj * NN + (size_t)gy * N + gx);
  }
  cp_async_wait_all();
  __syncthreads();
  const int npair = Ns * Ns;
  const int nc = nt / npair > 0 ? nt / npair : 1;  // tap subsets per (i, j)
  for (int t = tid; t < npair * nc; t += nt) {
    const int i = t % Ns, jj = (t / Ns) % Ns, c = t / npair;
    const float2* tp = tsm + (size_t)jj * RR * Ns + i;
    const float2* xr = xw + (size_t)jj * RR;
    float2 s = cmk(0.f, 0.f);
    for (int dd = c; dd < RR; dd += nc) cfma(s, tp[(size_t)dd * Ns], xr[dd]);
    part[(size_t)i * Ns * nc + jj * nc + c] = s;
  }
  __syncthreads();
  if (tid < 32) {
    double dsum = 0.0;
    for (int i = tid; i < Ns; i += 32) {
      float2 sacc = cmk(0.f, 0.f);
      for (int k = 0; k < Ns * nc; ++k) sacc = cadd(sacc, part[(size_t)i * Ns * nc + k]);
      const size_t o = ((size_t)lf * Ns + i) * NN + (size_t)ny * N + nx;
      const float2 cc = cscale(sacc, scale);
      out[o] = cadd(out[o], cc);
      if (dot_part) {
        const float2 xv = xl[(size_t)i * NN + (size_t)ny * N + nx];
        dsum += (double)xv.x * cc.x + (double)xv.y * cc.y;
      }
    }
    if (dot_part) {
      for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      if (tid == 0) dot_part[(size_t)d * SMSM_PART_MAX + part_base + ((size_t)l * 4 + corner) * w * w + pix] = dsum;
    }
  }
}

static size_t band_corner_smem(const smsm_plan_s* P) {
  const size_t R2 = P->R2, Ns = P->Ns;
  const size_t npair = Ns * Ns, nc = BAND_CORNER_THREADS / npair > 0 ? BAND_CORNER_THREADS / npair : 1;
  return (Ns * R2 * R2 * Ns + Ns * R2 * R2 + npair * nc) * sizeof(float2);
}

static int band_chunks(const smsm_plan_s* P) {
  return (P->r - 1) * ((P->N - 2 * (P->r - 1) + BAND_TX - 1) / BAND_TX);
}

// partial sums per direction written by k_band and k_band_corner
int band_blocks(const smsm_plan_s* P) {
  return (P->r > 1 && !P->periodic) ? P->L * 4 * band_chunks(P) + P->L * 4 * (P->r - 1) * (P->r - 1) : 0;
}

static size_t band_smem(const smsm_plan_s* P) {
  const int R2 = P->R2, Ns = P->Ns;
  const size_t ntap = (size_t)Ns * R2 * R2 * Ns;
  const size_t win = (size_t)Ns * R2 * (BAND_TX + R2 - 1), part = (size_t)Ns * BAND_TX * Ns;
  return (((ntap + 1) & ~(size_t)1) + (win > part ? win : part)) * sizeof(float2);
}

typedef void (*BandFn)(const float2*, float2*, const float2*, int, int, int, float, double*);
static BandFn band_fn(const smsm_plan_s* P) {
  switch (P->Ns) {
    case 1: return k_band<1>;
    case 2: return k_band<2>;
    case 3: return k_band<3>;
    case 4: return k_band<4>;
    case 5: return k_band<5>;
    case 6: return k_band<6>;
    case 7: return k_band<7>;
    default: return k_band<8>;
  }
}

smsm_status band_init_attrs(const smsm_plan_s* P) {
  cudaError_t e = cudaFuncSetAttribute(band_fn(P), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_band_corner, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_filters, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess || band_smem(P) > 200 * 1024 || band_corner_smem(P) > 200 * 1024 ||
      filters_smem(P) > 200 * 1024) {
    smsm_set_error("border-band kernel needs %zu bytes of shared memory", band_smem(P));
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

smsm_status launch_band(const smsm_plan_s* P, const float2* x, float2* out, float scale, double* dot_part,
                        cudaStream_t s) {
  if (P->r <= 1 || P->periodic) {  // filter 1 or periodic patches: the periodic value is exact
    if (dot_part) SMSM_CUDA_TRY(cudaMemsetAsync(dot_part, 0, sizeof(double) * SMSM_PART_MAX * P->D, s));
    return SMSM_OK;
  }
  dim3 grid(band_chunks(P), 4, P->LD);
  band_fn(P)<<<grid, 32 * P->Ns, band_smem(P), s>>>(x, out, P->wcls, P->L, P->N, P->r, scale, dot_part);
  SMSM_LAUNCH_CHECK("k_band");
  // corner pixels: disjoint from the strips, so the two kernels may run in either order
  k_band_corner<<<dim3((P->r - 1) * (P->r - 1), 4, P->LD), BAND_CORNER_THREADS, band_corner_smem(P), s>>>(
      x, out, P->wcls, P->L, P->Ns, P->N, P->r, scale, dot_part, P->L * 4 * band_chunks(P));
  SMSM_LAUNCH_CHECK("k_band_corner");
  return SMSM_OK;
}
