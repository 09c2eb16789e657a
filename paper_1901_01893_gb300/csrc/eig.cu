// Eigen-decomposition of the per-slice Gram G_l and the weight update.
//
// The low-rank penalty of Eq. 10 is handled by iteratively reweighted least
// squares: W_l = V diag((s + eps)^(-1/2)) V^H (nuclear-norm majoriser) or the
// projector onto the C - rank smallest eigenvectors (a fixed common rank, the
// Methods' choice of "the same rank for every slice").  The eigenvectors of
// the annihilation relation's null space (Eq. 9) are the annihilating filters.
//
// Eigensolver: two-sided cyclic Jacobi for Hermitian matrices, G held in shared
// memory, parallel round-robin ordering (C/2 disjoint rotations per round, all 2x2
// blocks updated at once).  Each matrix takes a cluster of two CTAs: the second
// holds V in its shared memory and applies every round's rotations to it while the
// first goes on with the next round.
//
// Precision: the Gram arrives in FP64 and is rounded once to FP32 on load; rotations
// are FP32.  What decides the accuracy of W is not the arithmetic width of the
// rotations but two things around them:
//  * no rotation is skipped because it is small next to the largest eigenvalue:
//    W = (G + eps I)^(-1/2) is largest on the smallest eigenvalues (down to eps_min),
//    so off-diagonal entries far below s_max still move W there (an entry delta left
//    in place changes W by about delta / (2 eps) relative).  The only absolute floor
//    is 1e-12 of the largest diagonal entry, which stops rounding noise between
//    exactly zero eigenvalues from churning;
//  * V stays orthonormal: the rotations of one eigen step (and the warm starts from
//    the previous V) would otherwise add their rounding to V's orthogonality from
//    one outer iteration to the next.  After every eigen step V is re-orthonormalised
//    by a Newton-Schulz step V <- V (3I - V^H V)/2, which squares the error.
// A sweep cap that ends the Jacobi with rotations still pending is reported
// (SMSM_ERR_EIG_UNCONVERGED in the solve's status) instead of passing silently.
#include <math.h>

#include "common.cuh"
#include "jacobi.cuh"
#include "umma.cuh"


__device__ __forceinline__ bool is_ident(float4 J) { return J.y == 0.f && J.z == 1.f && J.w == 0.f; }

// Rotation k of a round acts on the pair (p_k, q_k) with
// J = [[c, s], [-s e, c e]],  e = exp(-i phi) = (er, ei), phi = arg(G_pq).
// G lives in shared memory with row stride Cp+1 (odd, so column walks hit
// distinct banks).  Each round: C/2 threads compute the rotations of the
// round-robin pairs (p_k, q_k) into shared tables; then every 2x2 block
// (k1 <= k2) is transformed as J_k1^H B J_k2, its mirror (k2, k1) written as
// the conjugate transpose (G stays exactly Hermitian), and the diagonal blocks
// are set to their analytic result diag(a - t|b|, d + t|b|).  The blocks of
// the triangle k1 <= k2 < n (n = Cp/2, rounded up to even) are dealt out
// evenly: rows k and n-1-k of the triangle together hold n+1 blocks, so the
// triangle is an (n/2) x (n+1) rectangle of block indices.
// warm != 0: start from Gw = V_prev^H G V_prev (symmetrised on load).

#define JAC_BLK 4  // blocks per thread: (Cp/2 rounded to even)/2 * (that + 1) <= 4 * 992 for Cp <= 168

// block bi of the folded triangle -> (k1, k2), k1 <= k2 < n (n even)
__device__ __forceinline__ void tri_block(int bi, int n, float inv_n1, int& k1, int& k2) {
  int fr = __float2int_rz(((float)bi + 0.5f) * inv_n1);
  int c = bi - fr * (n + 1);
  if (c < 0) {
    --fr;
    c += n + 1;
  } else if (c > n) {
    ++fr;
    c -= n + 1;
  }
  if (c < n - fr) {
    k1 = fr;
    k2 = fr + c;
  } else {
    k1 = n - 1 - fr;
    k2 = k1 + (c - (n - fr));
  }
}

// The eigen step runs as a cluster of two CTAs per matrix.  Rank 0 holds G and runs
// the Jacobi rounds; rank 1 holds V (the previous eigenvectors, or I) and applies
// each round's rotations to it as they come, so V never leaves the chip and no log
// of rotations is written.  Rank 0 sends round m's rotations into rank 1's shared
// memory (buffer m & 1) and arrives on rank 1's `full` mbarrier; rank 1 applies them
// and arrives on rank 0's `empty` mbarrier, which rank 0 waits for before it reuses
// the buffer.  The sending is the last warp's only job: the other 31 warps update G's
// blocks meanwhile, so the latency of the remote stores and of the release stays off the
// round's critical path.  A message with header -1 ends the exchange.  Every wait is bounded:
// on a timeout the waiting side raises the device error flag (SMSM_ERR_TIMEOUT) and
// goes on, and both CTAs meet at a final cluster barrier, so neither leaves while the
// other may still touch its shared memory.
#define JAC_VS 3  // pair slots per lane of the V-CTA: Cp/2 <= 32 JAC_VS (Cp <= 192)

// shared-memory layout (bytes), the same in both CTAs: region A holds G (rank 0) or V
// (rank 1), both with row stride Cp + 1; region B holds rank 0's rotation, p and q
// tables or rank 1's two message buffers of Cp/2 rotations.
__host__ __device__ inline size_t jac_region_a(int Cp) { return (((size_t)Cp * (Cp + 1) * 8) + 15) & ~(size_t)15; }
__host__ __device__ inline size_t jac_smem_bytes(int Cp) { return jac_region_a(Cp) + (size_t)(Cp / 2) * 32; }

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(1024)
    k_jacobi(const double2* __restrict__ G, const float2* __restrict__ Gw, float* __restrict__ eig,
             float2* __restrict__ V, int warmv, int* __restrict__ sweeps_out, int C, int Cp, int max_sweeps, float tol,
             float floor_rel, SolverState* st, int L, int* __restrict__ errflag) {
  extern __shared__ __align__(16) unsigned char jsm[];
  __shared__ __align__(8) uint64_t full_b[2], empty_b[2];
  __shared__ int hdr[2];
  __shared__ float dmax;
  const uint32_t rank = cl_rank();
  const int l = blockIdx.x >> 1, tid = threadIdx.x, nt = blockDim.x;
  const int ld = Cp + 1;
  const int half = Cp / 2;
  float2* g = reinterpret_cast<float2*>(jsm);                          // rank 0: G;  rank 1: V
  unsigned char* regb = jsm + jac_region_a(Cp);
  float4* rbuf = reinterpret_cast<float4*>(regb);                      // rank 1: [2][half]
  if (tid == 0) {
    mbar_init(&full_b[0], 32);  // one arrival per lane of rank 0's sender warp
    mbar_init(&full_b[1], 32);
    mbar_init(&empty_b[0], 1);
    mbar_init(&empty_b[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  cl_sync();  // every mbarrier is initialised before the other CTA may arrive on it

  if (rank == 1) {
    // ---------------- V: apply every round's rotations as they arrive ----------------
    float2* Vl = V + (size_t)l * C * C;
    for (int e = tid; e < C * Cp; e += nt) {
      const int t = e / Cp, j = e - t * Cp;
      float2 v = cmk(0.f, 0.f);
      if (j < C) v = warmv ? Vl[(size_t)t * C + j] : cmk(j == t ? 1.f : 0.f, 0.f);
      g[t * ld + j] = v;
    }
    __syncthreads();
    // lane j applies the pairs k = j + 32 u of every round to the rows t = warp + 32 v;
    // the pairs' round-robin indices advance by one (mod Cp - 1) from round to round
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int mm = Cp - 1;
    int ia[JAC_VS], ib[JAC_VS];
    bool ok = true;
    int last = -1;
    for (long m = 0;; ++m) {
      const int b = (int)(m & 1);
      if (ok && !cl_wait(&full_b[b], (uint32_t)((m >> 1) & 1))) {
        ok = false;
        if (tid == 0) atomicExch(errflag, SMSM_ERR_TIMEOUT);
      }
      if (!__syncthreads_and(ok)) break;
      const int round = hdr[b];
      if (round < 0) break;
#pragma unroll
      for (int u = 0; u < JAC_VS; ++u) {
        const int k = lane + 32 * u;
        if (round == 0 || round != last + 1) {  // a new sweep starts over from round 0
          ia[u] = (k + round) % mm;
          ib[u] = (mm - k % mm + round) % mm;
        } else {
          ia[u] = ia[u] + 1 == mm ? 0 : ia[u] + 1;
          ib[u] = ib[u] + 1 == mm ? 0 : ib[u] + 1;
        }
      }
      last = round;
      const float4* R = rbuf + b * half;
#pragma unroll
      for (int u = 0; u < JAC_VS; ++u) {
        const int k = lane + 32 * u;
        if (k >= half) continue;
        const float4 J = R[k];
        if (is_ident(J)) continue;
        int pa, pb;
        if (k == 0) {
          pa = 0;
          pb = 1 + round;
        } else {
          pa = 1 + ia[u];
          pb = 1 + ib[u];
        }
        const int p = min(pa, pb), q = max(pa, pb);
        const float2 e = cmk(J.z, J.w);
        for (int t = warp; t < C; t += nw) {
          float2* row = g + t * ld;
          const float2 vp = row[p], evq = cmul(e, row[q]);
          row[p] = cmk(J.x * vp.x - J.y * evq.x, J.x * vp.y - J.y * evq.y);
          row[q] = cmk(J.y * vp.x + J.x * evq.x, J.y * vp.y + J.x * evq.y);
        }
      }
      __syncthreads();  // every thread is done with buffer b (and with this round's rows)
      if (tid == 0) cl_arrive(cl_map(&empty_b[b], 0), 1);
    }
    __syncthreads();
    for (int e = tid; e < C * C; e += nt) {
      const int t = e / C, j = e - t * C;
      Vl[e] = g[t * ld + j];
    }
    __syncthreads();
    cl_sync();  // rank 0 has sent its last message: nothing touches this CTA any more
    return;
  }

  // ---------------- rank 0: Jacobi rounds on G ----------------
  const int nh = (half + 1) & ~1;  // triangle edge rounded up to even (virtual pair skipped)
  const int nblk = (nh / 2) * (nh + 1);
  const float inv_n1 = 1.f / (float)(nh + 1);
  float4* rot = reinterpret_cast<float4*>(regb);
  int2* rpq = reinterpret_cast<int2*>(rot + half);  // (p, q) of every pair of the round
  const uint32_t r_buf = cl_map(rbuf, 1), r_hdr = cl_map(hdr, 1);
  const uint32_t r_full0 = cl_map(&full_b[0], 1), r_full1 = cl_map(&full_b[1], 1);
  long msg = 0;  // messages sent to rank 1 (counted by the sender warp)
  bool link = true;
  const int nbt = nt - 32;  // threads with blocks of G; the last warp sends
  const int lane = tid & 31;
  // send round `round` (or -1: the end) from the rotation table: the sender warp's lanes
  // write it (lane k the rotations k, k + 32, ...) and each arrives once; the end message
  // is lane 0's alone (one arrival counting for all 32)
  auto send = [&](int round) {
    const int b = (int)(msg & 1);
    if (msg >= 2 && link && !cl_wait(&empty_b[b], (uint32_t)(((msg >> 1) - 1) & 1))) {
      link = false;
      atomicExch(errflag, SMSM_ERR_TIMEOUT);
    }
    if (round >= 0) {
      for (int k = lane; k < half; k += 32) cl_st_v4(r_buf + (uint32_t)((b * half + k) * sizeof(float4)), rot[k]);
      if (lane == 0) cl_st_s32(r_hdr + (uint32_t)(b * sizeof(int)), round);
      cl_arrive(b ? r_full1 : r_full0, 1);
    } else if (lane == 0) {
      cl_st_s32(r_hdr + (uint32_t)(b * sizeof(int)), -1);
      cl_arrive(b ? r_full1 : r_full0, 32);
    }
    ++msg;
  };
  const double2* Gl = G + (size_t)l * C * C;
  const float2* Gwl = Gw ? Gw + (size_t)l * C * C : nullptr;
  for (int e = tid; e < Cp * Cp; e += nt) {
    const int a = e / Cp, b = e - a * Cp;
    float2 v = cmk(0.f, 0.f);
    if (a < C && b < C) {
      if (Gwl) {
        const float2 u = Gwl[(size_t)a * C + b], w = Gwl[(size_t)b * C + a];
        v = cmk(0.5f * (u.x + w.x), 0.5f * (u.y - w.y));
        if (a == b) v.y = 0.f;
      } else {
        v = cmk((float)Gl[(size_t)a * C + b].x, (float)Gl[(size_t)a * C + b].y);
      }
    }
    g[a * ld + b] = v;
  }
  if (tid == 0) dmax = 0.f;
  __syncthreads();
  if (tid < Cp) atomicMax(reinterpret_cast<int*>(&dmax), __float_as_int(fmaxf(g[tid * ld + tid].x, 0.f)));
  __syncthreads();
  // absolute floor of the rotation test (given relative to the largest diagonal entry)
  const float floor_abs = floor_rel * dmax;
  // this thread's blocks of the folded triangle, the same in every round
  int kb1[JAC_BLK], kb2[JAC_BLK];
#pragma unroll
  for (int m = 0; m < JAC_BLK; ++m) {
    const int bi = tid + m * nbt;
    kb1[m] = kb2[m] = -1;
    if (tid < nbt && bi < nblk) {
      tri_block(bi, nh, inv_n1, kb1[m], kb2[m]);
      if (kb2[m] >= half) kb1[m] = -1;  // virtual pair of an odd half
    }
  }
  int sw = 0;
  int pending = 1;  // the last sweep (or the direct test after it) found a pair to rotate
  for (; sw < max_sweeps; ++sw) {
    int rotated = 0;  // this thread set a non-identity rotation during the sweep
    // this thread's pair of the round-robin (tid < half): both indices advance by one
    // (mod Cp - 1, over 1..Cp-1) from round to round, index 0 stays with pair 0
    int pa = 0, pb = 0;
    if (tid < half) jpair(0, tid, Cp, pa, pb);
    for (int round = 0; round < Cp - 1; ++round) {
      if (tid < half) {
        const int p = min(pa, pb), q = max(pa, pb);
        rpq[tid] = make_int2(p, q);
        const float a = g[p * ld + p].x, d = g[q * ld + q].x;
        const float2 b = g[p * ld + q];
        const float babs = hypotf(b.x, b.y);
        float4 J = make_float4(1.f, 0.f, 1.f, 0.f);
        if (babs > floor_abs && babs > tol * sqrtf(fabsf(a * d))) {
          // one correctly rounded reciprocal and one reciprocal square root instead of
          // four divisions
          const float ib = __frcp_rn(babs);
          const float theta = 0.5f * (d - a) * ib;
          const float t = copysignf(__frcp_rn(fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f))), theta);
          const float c = __frsqrt_rn(fmaf(t, t, 1.f));
          J = make_float4(c, t * c, b.x * ib, -b.y * ib);
          rotated = 1;
        }
        rot[tid] = J;
        pb = pb == Cp - 1 ? 1 : pb + 1;
        if (tid > 0) pa = pa == Cp - 1 ? 1 : pa + 1;
      }
      __syncthreads();
      if (tid >= nbt) send(round);  // the sender warp, while the others update G
#pragma unroll
      for (int m = 0; m < JAC_BLK; ++m) {
        const int k1 = kb1[m], k2 = kb2[m];
        if (k1 < 0) continue;
        const float4 J1 = rot[k1];
        const bool id1 = is_ident(J1);
        const int2 pq1 = rpq[k1];
        const int p1 = pq1.x, q1 = pq1.y;
        if (k2 == k1) {
          if (id1) continue;
          const float a = g[p1 * ld + p1].x, d = g[q1 * ld + q1].x;
          const float2 b = g[p1 * ld + q1];
          const float tb = (J1.y / J1.x) * hypotf(b.x, b.y);
          g[p1 * ld + p1] = cmk(a - tb, 0.f);
          g[q1 * ld + q1] = cmk(d + tb, 0.f);
          g[p1 * ld + q1] = cmk(0.f, 0.f);
          g[q1 * ld + p1] = cmk(0.f, 0.f);
          continue;
        }
        const float4 J2 = rot[k2];
        if (id1 && is_ident(J2)) continue;
        const int2 pq2 = rpq[k2];
        const int p2 = pq2.x, q2 = pq2.y;
        const float2 B00 = g[p1 * ld + p2], B01 = g[p1 * ld + q2];
        // row q1 times conj(e1)
        const float2 e1c = cmk(J1.z, -J1.w);
        const float2 B10 = cmul(e1c, g[q1 * ld + p2]), B11 = cmul(e1c, g[q1 * ld + q2]);
        // T = J1^H B : row0 = c B0 - s B1', row1 = s B0 + c B1'
        const float c1 = J1.x, s1 = J1.y;
        const float2 T00 = cmk(c1 * B00.x - s1 * B10.x, c1 * B00.y - s1 * B10.y);
        const float2 T01 = cmk(c1 * B01.x - s1 * B11.x, c1 * B01.y - s1 * B11.y);
        const float2 T10 = cmk(s1 * B00.x + c1 * B10.x, s1 * B00.y + c1 * B10.y);
        const float2 T11 = cmk(s1 * B01.x + c1 * B11.x, s1 * B01.y + c1 * B11.y);
        // O = T J2 : col0 = c T0 - s T1', col1 = s T0 + c T1', T1' = e2 T1
        const float2 e2 = cmk(J2.z, J2.w);
        const float2 U01 = cmul(T01, e2), U11 = cmul(T11, e2);
        const float c2 = J2.x, s2 = J2.y;
        const float2 O00 = cmk(c2 * T00.x - s2 * U01.x, c2 * T00.y - s2 * U01.y);
        const float2 O10 = cmk(c2 * T10.x - s2 * U11.x, c2 * T10.y - s2 * U11.y);
        const float2 O01 = cmk(s2 * T00.x + c2 * U01.x, s2 * T00.y + c2 * U01.y);
        const float2 O11 = cmk(s2 * T10.x + c2 * U11.x, s2 * T10.y + c2 * U11.y);
        g[p1 * ld + p2] = O00;
        g[p1 * ld + q2] = O01;
        g[q1 * ld + p2] = O10;
        g[q1 * ld + q2] = O11;
        g[p2 * ld + p1] = conjf2(O00);
        g[q2 * ld + p1] = conjf2(O01);
        g[p2 * ld + q1] = conjf2(O10);
        g[q2 * ld + q1] = conjf2(O11);
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) {
      pending = 0;
      break;
    }
    // A sweep that sets no rotation changes nothing, and it sets none exactly when no
    // pair passes the rotation test on the current matrix: test every pair directly
    // (same arithmetic as the rotation step) instead of running that sweep.
    int need = 0;
    for (int e = tid; e < Cp * Cp && !need; e += nt) {
      const int p = e / Cp, q = e - p * Cp;
      if (p >= q) continue;
      const float2 b = g[p * ld + q];
      const float babs = hypotf(b.x, b.y);
      need = babs > floor_abs && babs > tol * sqrtf(fabsf(g[p * ld + p].x * g[q * ld + q].x));
    }
    if (!__syncthreads_or(need)) {
      ++sw;
      pending = 0;
      break;
    }
  }
  // sweep cap reached with a pair still above the rotation test: report it (unless an
  // earlier error of this problem is already recorded)
  if (pending && tid == 0 && st) atomicCAS(&st[l / L].status, 0, (int)SMSM_ERR_EIG_UNCONVERGED);
  for (int j = tid; j < Cp; j += nt) eig[(size_t)l * Cp + j] = g[j * ld + j].x;
  if (tid == 0) sweeps_out[l] = sw;
  __syncthreads();  // rank 1 reads the last rounds' buffers until it sees the end message
  if (tid >= nbt) send(-1);
  __syncthreads();
  cl_sync();
}

// The small complex GEMMs of the eigen step, C x C per matrix, FP32 accumulation:
//   SG_GV:  T  = G V            (G in FP64, rounded on load; the warm start's first product)
//   SG_VHT: Gw = V^H T          (the warm start's second product)
//   SG_VHV: M  = V^H V          (Newton-Schulz, step 0)
//   SG_NS:  V' = V (3I - M) / 2 (Newton-Schulz, step 1)
//   SG_W:   W  = V diag(f) V^H, f_j = (max(s_j, 0) + eps)^(-1/2) (IRLS) or
//           [s_j among the C - rank smallest] (NULLSPACE)
// A CTA computes a 32 x 32 output tile, each thread 2 x 2 entries (rows ty, ty + 16, columns
// tx, tx + 16), over k-steps of 16 staged in shared memory; every operand tile is loaded
// along its contiguous index.
#define SG_T 32
#define SG_K 16
enum { SG_GV = 0, SG_VHT = 1, SG_VHV = 2, SG_NS = 3, SG_W = 4 };

template <int OP>
__global__ void __launch_bounds__(256) k_cgemm(const double2* __restrict__ G, const float2* __restrict__ X,
                                               const float2* __restrict__ Y, float2* __restrict__ out, int C,
                                               const float* __restrict__ eig, const SolverState* __restrict__ st,
                                               int Cp, int mode, int rank, int L) {
  __shared__ float2 As[SG_T][SG_K + 1];
  __shared__ float2 Bs[SG_K][SG_T + 1];
  __shared__ float f[OP == SG_W ? SMSM_MAX_C : 1];
  const int l = blockIdx.z;  // flat (direction, slice)
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int a0 = blockIdx.y * SG_T, b0 = blockIdx.x * SG_T;
  const size_t off = (size_t)l * C * C;
  const float2* Xl = X + off;
  if constexpr (OP == SG_W) {
    const float* s = eig + (size_t)l * Cp;
    const double eps = st[l / L].eps;
    for (int j = tid; j < C; j += blockDim.x) {
      if (mode == SMSM_MODE_NULLSPACE) {
        int rk = 0;
        const float sj = s[j];
        for (int k = 0; k < C; ++k) rk += (s[k] < sj) || (s[k] == sj && k < j);
        f[j] = rk < C - rank ? 1.f : 0.f;
      } else {
        f[j] = (float)(1.0 / sqrt(fmax((double)s[j], 0.0) + eps));
      }
    }
    __syncthreads();
  }
  // A is read along k (row-contiguous) except for V^H, read along a
  constexpr bool a_rows = !(OP == SG_VHT || OP == SG_VHV);
  // B is read along b except for conj(V)^T of the weights, read along k
  constexpr bool b_rows = OP != SG_W;
  float2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = cmk(0.f, 0.f);
  for (int k0 = 0; k0 < C; k0 += SG_K) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int t = tid + 256 * it;
      const int al = a_rows ? t / SG_K : t % SG_T, kl = a_rows ? t % SG_K : t / SG_T;
      const int a = a0 + al, k = k0 + kl;
      float2 v = cmk(0.f, 0.f);
      if (a < C && k < C) {
        if constexpr (OP == SG_GV) {
          const double2 g = G[off + (size_t)a * C + k];
          v = cmk((float)g.x, (float)g.y);
        } else if constexpr (OP == SG_VHT || OP == SG_VHV) {
          v = conjf2(Xl[(size_t)k * C + a]);
        } else if constexpr (OP == SG_NS) {
          v = Xl[(size_t)a * C + k];
        } else {
          v = cscale(Xl[(size_t)a * C + k], f[k]);
        }
      }
      As[al][kl] = v;
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int t = tid + 256 * it;
      const int bl = b_rows ? t % SG_T : t / SG_K, kl = b_rows ? t / SG_T : t % SG_K;
      const int b = b0 + bl, k = k0 + kl;
      float2 v = cmk(0.f, 0.f);
      if (b < C && k < C) {
        if constexpr (OP == SG_GV || OP == SG_VHV) {
          v = Xl[(size_t)k * C + b];
        } else if constexpr (OP == SG_VHT) {
          v = Y[off + (size_t)k * C + b];
        } else if constexpr (OP == SG_NS) {
          const float2 m = Y[off + (size_t)k * C + b];
          v = cmk(((k == b ? 3.f : 0.f) - m.x) * 0.5f, -0.5f * m.y);
        } else {
          v = conjf2(Xl[(size_t)b * C + k]);
        }
      }
      Bs[kl][bl] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SG_K; ++k) {
      const float2 x0 = As[ty][k], x1 = As[ty + 16][k];
      const float2 y0 = Bs[k][tx], y1 = Bs[k][tx + 16];
      cfma(acc[0][0], x0, y0);
      cfma(acc[0][1], x0, y1);
      cfma(acc[1][0], x1, y0);
      cfma(acc[1][1], x1, y1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < C && b < C) out[off + (size_t)a * C + b] = acc[i][j];
    }
}

template <int OP>
static smsm_status launch_cgemm(const smsm_plan_s* P, const double2* G, const float2* X, const float2* Y,
                                float2* out, const smsm_params* prm, cudaStream_t s) {
  const int C = P->C;
  const dim3 grid((C + SG_T - 1) / SG_T, (C + SG_T - 1) / SG_T, P->LD);
  k_cgemm<OP><<<grid, 256, 0, s>>>(G, X, Y, out, C, P->eig, P->st, P->Cp, prm ? prm->mode : 0, prm ? prm->rank : 0,
                                   P->L);
  SMSM_LAUNCH_CHECK("k_cgemm");
  return SMSM_OK;
}

// eps schedule and report, one CTA per direction d: eps_1 = eps0_rel * (largest
// eigenvalue over d's slices), then eps_k = max(eps_{k-1}/eta, eps_min).
__global__ void k_eps(const float* __restrict__ eig, const int* __restrict__ sweeps, SolverState* st, DevReport* rep,
                      int L, int C, int Cp, int outer, double eps0_rel, double eta, double eps_min_rel) {
  __shared__ float mx[256];
  const int d = blockIdx.x;
  float m = 0.f;
  for (int e = threadIdx.x; e < L * C; e += blockDim.x) {
    int l = e / C, j = e - l * C;
    m = fmaxf(m, eig[(size_t)(d * L + l) * Cp + j]);
  }
  mx[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) mx[threadIdx.x] = fmaxf(mx[threadIdx.x], mx[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    SolverState* sd = st + d;
    if (outer == 0) {
      sd->eps0 = eps0_rel * (double)mx[0];
      sd->eps = sd->eps0;
      sd->eps_min = eps_min_rel * sd->eps0;
    } else {
      sd->eps = fmax(sd->eps / eta, sd->eps_min);
    }
    if (d == 0 && outer < SMSM_MAX_OUTER) {  // the report follows direction 0
      int smax = 0;
      for (int l = 0; l < L; ++l) smax = max(smax, sweeps[l]);
      rep->eps[outer] = sd->eps;
      rep->sweeps[outer] = smax;
    }
  }
}

// the two-CTA solver holds all of G in one CTA's shared memory (C up to 168)
bool eig_pair_supported(int Cp) {
  const int nh = (Cp / 2 + 1) & ~1;
  return (nh / 2) * (nh + 1) <= JAC_BLK * (1024 - 32) && Cp / 2 <= 32 * JAC_VS && jac_smem_bytes(Cp) <= 227 * 1024;
}

smsm_status eig_init_attrs(const smsm_plan_s* P) {
  if (P->eig_cluster) return eig_cluster_init_attrs(P->C);
  const int Cp = P->Cp;
  if (!eig_pair_supported(Cp)) {
    smsm_set_error("Jacobi kernel: C = %d is above the two-CTA solver's limit", Cp);
    return SMSM_ERR_ARG;
  }
  // the attribute belongs to the kernel, not to the plan: set the most any plan uses, so a
  // plan made later with a smaller C does not shrink it under an earlier plan's launches
  const size_t sm = jac_smem_bytes(Cp);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jac_smem_bytes(168));
  if (e != cudaSuccess) {
    smsm_set_error("Jacobi kernel cannot get %zu bytes of shared memory: %s", sm, cudaGetErrorString(e));
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

size_t eig_jacobi_smem(int Cp) { return jac_smem_bytes(Cp); }

smsm_status launch_eig_weights(const smsm_plan_s* P, const double2* G, int outer, const smsm_params* prm,
                               cudaStream_t s, Timer* T) {
  const int Cp = P->Cp, C = P->C;
  int msw = prm->max_sweeps > 0 ? prm->max_sweeps : SMSM_MAX_SWEEPS;
  if (msw > SMSM_MAX_SWEEPS) msw = SMSM_MAX_SWEEPS;
  // warm start from the previous outer iteration's eigenvectors (same solve)
  const int warm = (outer > 0 && !prm->eig_cold) ? 1 : 0;
  if (T) T->begin(SMSM_STAGE_EIG);
  smsm_status sg;
  if (P->eig_cluster) {
    // one-sided Jacobi on A = G V_prev (the congruence's first product) or on G itself
    if (warm && (sg = launch_cgemm<SG_GV>(P, G, P->V, nullptr, P->Gw, prm, s))) return sg;
    const float tol = prm->eig_tol > 0.f ? prm->eig_tol : 2e-6f;
    smsm_status st = launch_eig_cluster(P, G, warm ? P->Gw : nullptr, msw, tol, 1e-12f, s);
    if (st) return st;
  } else {
  if (warm) {
    if ((sg = launch_cgemm<SG_GV>(P, G, P->V, nullptr, P->Gw, prm, s))) return sg;
    if ((sg = launch_cgemm<SG_VHT>(P, nullptr, P->V, P->Gw, P->Gw2, prm, s))) return sg;
  }
  // absolute floor of the rotation test, relative to the largest diagonal entry: far below
  // every eigenvalue W resolves (the weight changes by about delta / (2 eps) for an
  // off-diagonal entry delta left in place, so delta must stay many orders below eps_min);
  // it only stops the churning of rounding noise between exactly zero eigenvalues
  const double frel = 1e-12;
  // two CTAs per matrix: the Jacobi rounds on G and, beside them, V times every rotation
  k_jacobi<<<2 * P->LD, 1024, jac_smem_bytes(Cp), s>>>(G, warm ? P->Gw2 : nullptr, P->eig, P->V, warm, P->sweeps, C,
                                                        Cp, msw, prm->eig_tol > 0.f ? prm->eig_tol : 1e-6f,
                                                        (float)frel, P->st, P->L, P->devflag);
  SMSM_LAUNCH_CHECK("k_jacobi");
  }
  if (T) T->end(SMSM_STAGE_EIG);
  if (T) T->begin(SMSM_STAGE_VAPPLY);
  if ((sg = launch_cgemm<SG_VHV>(P, nullptr, P->V, nullptr, P->Gw, prm, s))) return sg;
  if ((sg = launch_cgemm<SG_NS>(P, nullptr, P->V, P->Gw, P->Gw2, prm, s))) return sg;
  SMSM_CUDA_TRY(cudaMemcpyAsync(P->V, P->Gw2, sizeof(float2) * (size_t)P->LD * C * C, cudaMemcpyDeviceToDevice, s));
  if (T) T->end(SMSM_STAGE_VAPPLY);
  if (T) T->begin(SMSM_STAGE_WEIGHTS);
  k_eps<<<P->D, 256, 0, s>>>(P->eig, P->sweeps, P->st, P->rep, P->L, C, Cp, outer, prm->eps0_rel, prm->eta,
                             prm->eps_min_rel);
  SMSM_LAUNCH_CHECK("k_eps");
  if ((sg = launch_cgemm<SG_W>(P, nullptr, P->V, nullptr, P->Wf, prm, s))) return sg;
  if (T) T->end(SMSM_STAGE_WEIGHTS);
  return SMSM_OK;
}
