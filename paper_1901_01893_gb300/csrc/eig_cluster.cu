// Eigen step for the large Grams (C = Ns r^2 up to 320, e.g. 8 shots with a 6x6 filter):
// one-sided block Jacobi on a cluster of eight CTAs per matrix.
//
// The Gram G_l of Eq. 9 is Hermitian positive semi-definite, so its eigenvectors are
// the right singular vectors of G_l itself.  One-sided (Hestenes) Jacobi finds them by
// rotating pairs of columns of A = G V (and the same columns of V) until all columns
// of A are mutually orthogonal; then A = V diag(s) and s_j = v_j^H a_j.  The 2x2
// problem of a pair is the Gram of its two columns, [[|a_p|^2, a_p^H a_q], [., |a_q|^2]],
// diagonalised by the same complex rotation as in the two-sided solver.  The starting
// point is the previous outer iteration's V (A = G V_prev, made by the congruence
// kernel's first product) or V = I, A = G.
//
// Why one-sided here: a 288 x 288 complex matrix is 664 KB, three times a CTA's shared
// memory, and a rotation only ever touches two columns.  The columns of A and V are
// dealt out in 16 blocks of w columns, two blocks per CTA (all C rows of each), so
// every pair rotation is local to one CTA:
//  * each sweep first rotates the pairs inside every block (w - 1 rounds of w/2 pairs
//    per block, both blocks of a CTA at once: w pairs per round, one warp per pair);
//  * then 15 block rounds of a round-robin tournament over the 16 blocks: in each, a
//    CTA rotates every pair (one column from each of its two blocks) in w rounds of w
//    disjoint pairs, and the blocks then move one position around the tournament
//    circle (block 0 stays) through distributed shared memory.  After 15 moves every
//    block is home again and every pair of columns has met exactly once.
// A block move copies both blocks of a CTA (A and V columns) from the neighbours'
// shared memory in chunks held in registers: every CTA reads chunk c of its sources,
// the cluster meets at a barrier, every CTA writes chunk c into its own slots.  Chunks
// are taken at the same offsets in both slots, so a read never sees data written in
// the same move.  All waits are hardware cluster barriers that every thread of every
// CTA reaches the same number of times (the loop trip counts are the same in every
// CTA and the end of the sweeps is decided by a vote all CTAs read after one barrier);
// no flag is spun on.
//
// Accuracy: the column sums are FP32 per lane over C/32 rows, then a butterfly over
// the warp (the same value in every lane, so every decision is warp-uniform); their
// relative error is a few 1e-7, below the rotation test's 2e-6.  A is scaled on load by
// a power of two that brings the largest diagonal entry of G to [0.5, 1) so that the
// squared column norms stay far inside the FP32 range.
#include <math.h>

#include "common.cuh"
#include "jacobi.cuh"

#define OSJ_R 8            // CTAs per cluster (the portable maximum)
#define OSJ_NB (2 * OSJ_R) // column blocks

// block width (even, so that a block's round-robin pairs up all its columns)
__host__ __device__ inline int osj_w(int C) {
  const int w = (C + OSJ_NB - 1) / OSJ_NB;
  return w + (w & 1);
}
// row groups of 32 (one lane per row of each group)
__host__ __device__ inline int osj_kr(int C) { return (C + 31) / 32; }
// two slots x (A and V) x w columns x 32 KR rows
__host__ __device__ inline size_t osj_smem(int C) { return (size_t)4 * osj_w(C) * 32 * osj_kr(C) * sizeof(float2); }

// Rotate columns p, q of A and V so that a_p^H a_q = 0 (when the pair passes the test).
// One warp; lane j holds rows j + 32 k.  Returns 1 if a rotation was applied.
template <int KR>
__device__ __forceinline__ int osj_pair(float2* __restrict__ Ap, float2* __restrict__ Aq, float2* __restrict__ Vp,
                                        float2* __restrict__ Vq, int lane, float tol, float floor_abs) {
  float2 ap[KR], aq[KR];
  float sa = 0.f, sb = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    ap[k] = Ap[lane + 32 * k];
    aq[k] = Aq[lane + 32 * k];
    sa = fmaf(ap[k].x, ap[k].x, fmaf(ap[k].y, ap[k].y, sa));
    sb = fmaf(aq[k].x, aq[k].x, fmaf(aq[k].y, aq[k].y, sb));
    gr = fmaf(ap[k].x, aq[k].x, fmaf(ap[k].y, aq[k].y, gr));   // Re conj(a_p) a_q
    gi = fmaf(ap[k].x, aq[k].y, fmaf(-ap[k].y, aq[k].x, gi));  // Im conj(a_p) a_q
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, m);
    sb += __shfl_xor_sync(0xffffffffu, sb, m);
    gr += __shfl_xor_sync(0xffffffffu, gr, m);
    gi += __shfl_xor_sync(0xffffffffu, gi, m);
  }
  const float babs = hypotf(gr, gi);
  if (!(babs > floor_abs && babs > tol * sqrtf(sa * sb))) return 0;
  // J = [[c, s], [-s e, c e]], e = exp(-i arg(a_p^H a_q)): new a_p = c a_p - s e a_q,
  // new a_q = s a_p + c e a_q, t = s / c the smaller root of t^2 + 2 theta t - 1 = 0
  const float theta = (sb - sa) / (2.f * babs);
  const float t = fabsf(theta) > 1e10f ? 0.5f / theta
                                       : (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
  const float c = 1.f / sqrtf(t * t + 1.f), s = t * c;
  const float2 e = cmk(gr / babs, -gi / babs);
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const float2 evq = cmul(e, aq[k]);
    Ap[lane + 32 * k] = cmk(c * ap[k].x - s * evq.x, c * ap[k].y - s * evq.y);
    Aq[lane + 32 * k] = cmk(s * ap[k].x + c * evq.x, s * ap[k].y + c * evq.y);
  }
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const float2 vp = Vp[lane + 32 * k], evq = cmul(e, Vq[lane + 32 * k]);
    Vp[lane + 32 * k] = cmk(c * vp.x - s * evq.x, c * vp.y - s * evq.y);
    Vq[lane + 32 * k] = cmk(s * vp.x + c * evq.x, s * vp.y + c * evq.y);
  }
  return 1;
}

// One move of the tournament: the block at circle position i >= 1 goes to position
// i + 1 (15 -> 1), position 0 stays.  CTA k holds positions k (slot 0) and 15 - k
// (slot 1), so slot 0 of CTA k >= 2 comes from slot 0 of CTA k - 1, slot 0 of CTA 1
// from slot 1 of CTA 0, slot 1 of CTA k <= 6 from slot 1 of CTA k + 1, and slot 1 of
// CTA 7 from its own slot 0.
__device__ __forceinline__ void osj_move(float2* sm, int F4, uint32_t rank, int tid, int nt) {
  int src_cta[2], src_slot[2];
  src_cta[0] = rank <= 1 ? 0 : (int)rank - 1;  // (rank 0 keeps its slot 0: no source)
  src_slot[0] = rank == 1 ? 1 : 0;
  src_cta[1] = rank == OSJ_R - 1 ? OSJ_R - 1 : (int)rank + 1;
  src_slot[1] = rank == OSJ_R - 1 ? 0 : 1;
  const bool keep0 = rank == 0;  // position 0 never moves
  uint32_t src[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) src[s] = cl_map(sm, (uint32_t)src_cta[s]) + (uint32_t)(src_slot[s] * F4 * 16);
  float4* dst = reinterpret_cast<float4*>(sm);
  cl_sync();  // every CTA is done rotating its columns
  for (int o0 = 0; o0 < F4; o0 += 3 * nt) {
    float4 buf[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int o = o0 + j * nt + tid;
        if (o < F4 && !(s == 0 && keep0)) buf[s][j] = cl_ld_v4(src[s] + (uint32_t)o * 16u);
      }
    cl_sync();  // chunk read everywhere before anyone overwrites it
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int o = o0 + j * nt + tid;
        if (o < F4 && !(s == 0 && keep0)) dst[s * F4 + o] = buf[s][j];
      }
  }
  __syncthreads();
}

template <int KR>
__global__ void __cluster_dims__(OSJ_R, 1, 1) __launch_bounds__(640, 1)
    k_jacobi_os(const double2* __restrict__ G, const float2* __restrict__ T, float* __restrict__ eig,
                float2* __restrict__ V, int* __restrict__ sweeps_out, int C, int Cp, int max_sweeps, float tol,
                float floor_rel, SolverState* st, int L) {
  extern __shared__ __align__(16) float2 osm[];
  __shared__ int vote[OSJ_R];
  __shared__ float dmax_s;
  constexpr int Cr = 32 * KR;
  const int w = osj_w(C), hw = w / 2;
  const uint32_t rank = cl_rank();
  const int l = blockIdx.x / OSJ_R;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  const int blk0 = (int)rank, blk1 = OSJ_NB - 1 - (int)rank;  // home blocks of slots 0 and 1
  // slot s: A columns c at osm + (2 w s + c) Cr, V columns at osm + (2 w s + w + c) Cr
#define OSJ_A(s, c) (osm + (size_t)(2 * w * (s) + (c)) * Cr)
#define OSJ_V(s, c) (osm + (size_t)(2 * w * (s) + w + (c)) * Cr)
  cl_sync();  // every CTA of the cluster is running before any touches another's memory

  const double2* Gl = G + (size_t)l * C * C;
  if (tid == 0) dmax_s = 0.f;
  __syncthreads();
  for (int j = tid; j < C; j += nt)
    atomicMax(reinterpret_cast<int*>(&dmax_s), __float_as_int(fmaxf((float)Gl[(size_t)j * C + j].x, 0.f)));
  __syncthreads();
  int ex = 0;
  if (dmax_s > 0.f) frexpf(dmax_s, &ex);
  const float scale = ldexpf(1.f, -ex), inv_scale = ldexpf(1.f, ex);
  // A squared column norms are ~ s^2: the absolute floor of the pair test is floor_rel^2
  // of the squared largest diagonal entry (below 1 after scaling)
  const float floor_abs = floor_rel * floor_rel;

  const float2* Tl = T ? T + (size_t)l * C * C : nullptr;
  float2* Vl = V + (size_t)l * C * C;
  for (int e = tid; e < 2 * Cr * w; e += nt) {
    const int s = e / (Cr * w), rem = e - s * Cr * w;
    const int t = rem / w, c = rem - t * w;
    const int j = (s ? blk1 : blk0) * w + c;
    float2 a = cmk(0.f, 0.f), v = cmk(0.f, 0.f);
    if (t < C && j < C) {
      if (Tl) {
        a = Tl[(size_t)t * C + j];
        v = Vl[(size_t)t * C + j];
      } else {
        const double2 g = Gl[(size_t)t * C + j];
        a = cmk((float)g.x, (float)g.y);
        v = cmk(t == j ? 1.f : 0.f, 0.f);
      }
    }
    OSJ_A(s, c)[t] = cscale(a, scale);
    OSJ_V(s, c)[t] = v;
  }
  __syncthreads();

  const int F4 = w * Cr;  // float4 per slot (A and V columns)
  int sw = 0, pending = 1;
  while (sw < max_sweeps) {
    int rotated = 0;
    // pairs inside each block: both slots at once, one warp per pair
    for (int rd = 0; rd < w - 1; ++rd) {
      if (warp < w) {
        const int s = warp / hw, k = warp - s * hw;
        int p, q;
        jpair(rd, k, w, p, q);
        rotated |= osj_pair<KR>(OSJ_A(s, p), OSJ_A(s, q), OSJ_V(s, p), OSJ_V(s, q), lane, tol, floor_abs);
      }
      __syncthreads();
    }
    // pairs across blocks: 15 tournament rounds, each w rounds of w disjoint pairs
    for (int br = 0; br < OSJ_NB - 1; ++br) {
      for (int t = 0; t < w; ++t) {
        if (warp < w) {
          const int q = warp + t < w ? warp + t : warp + t - w;
          rotated |= osj_pair<KR>(OSJ_A(0, warp), OSJ_A(1, q), OSJ_V(0, warp), OSJ_V(1, q), lane, tol, floor_abs);
        }
        __syncthreads();
      }
      osj_move(osm, F4, rank, tid, nt);
    }
    ++sw;
    // cluster vote: did any CTA rotate during this sweep?
    const int any = __syncthreads_or(rotated);
    if (tid < OSJ_R) cl_st_s32(cl_map(&vote[rank], (uint32_t)tid), any);
    cl_sync();
    int tot = 0;
#pragma unroll
    for (int k = 0; k < OSJ_R; ++k) tot |= vote[k];
    if (!tot) {
      pending = 0;
      break;
    }
  }
  if (pending && rank == 0 && tid == 0 && st) atomicCAS(&st[l / L].status, 0, (int)SMSM_ERR_EIG_UNCONVERGED);
  if (rank == 0 && tid == 0) sweeps_out[l] = sw;
  // eigenvalue s_j = Re(v_j^H a_j) / |v_j|^2 (a_j = G v_j), undoing the load scale.  The
  // rotations are unitary only to rounding, so a column of V drifts in length over the
  // sweeps (by some 1e-5); A's column drifts with it, and the quotient does not see it.
  for (int cc = warp; cc < 2 * w; cc += nw) {
    const int s = cc / w, c = cc - s * w;
    const int j = (s ? blk1 : blk0) * w + c;
    const float2* a = OSJ_A(s, c);
    const float2* v = OSJ_V(s, c);
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const float2 av = a[lane + 32 * k], vv = v[lane + 32 * k];
      num = fmaf(vv.x, av.x, fmaf(vv.y, av.y, num));
      den = fmaf(vv.x, vv.x, fmaf(vv.y, vv.y, den));
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, m);
      den += __shfl_xor_sync(0xffffffffu, den, m);
    }
    if (lane == 0 && j < Cp) eig[(size_t)l * Cp + j] = (j < C && den > 0.f) ? num / den * inv_scale : 0.f;
  }
  for (int e = tid; e < 2 * Cr * w; e += nt) {
    const int s = e / (Cr * w), rem = e - s * Cr * w;
    const int t = rem / w, c = rem - t * w;
    const int j = (s ? blk1 : blk0) * w + c;
    if (t < C && j < C) Vl[(size_t)t * C + j] = OSJ_V(s, c)[t];
  }
#undef OSJ_A
#undef OSJ_V
  cl_sync();  // no CTA leaves while another may still address its shared memory
}

typedef void (*OsjFn)(const double2*, const float2*, float*, float2*, int*, int, int, int, float, float,
                      SolverState*, int);

static OsjFn osj_fn(int C) {
  switch (osj_kr(C)) {
    case 3: return k_jacobi_os<3>;
    case 4: return k_jacobi_os<4>;
    case 5: return k_jacobi_os<5>;
    case 6: return k_jacobi_os<6>;
    case 7: return k_jacobi_os<7>;
    case 8: return k_jacobi_os<8>;
    case 9: return k_jacobi_os<9>;
    case 10: return k_jacobi_os<10>;
    default: return nullptr;
  }
}

bool eig_cluster_supported(int C) { return C >= 65 && C <= SMSM_MAX_C && osj_smem(C) <= 227 * 1024; }

smsm_status eig_cluster_init_attrs(int C) {
  OsjFn fn = eig_cluster_supported(C) ? osj_fn(C) : nullptr;
  if (!fn) {
    smsm_set_error("cluster eigensolver: C = %d outside [65, %d]", C, SMSM_MAX_C);
    return SMSM_ERR_ARG;
  }
  // per kernel, not per plan: the most any C of this instance (same C/32 rounded up) uses
  const int cmax = 32 * osj_kr(C) < SMSM_MAX_C ? 32 * osj_kr(C) : SMSM_MAX_C;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osj_smem(cmax));
  if (e != cudaSuccess) {
    smsm_set_error("cluster eigensolver cannot get %zu bytes of shared memory: %s", osj_smem(C),
                   cudaGetErrorString(e));
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

smsm_status launch_eig_cluster(const smsm_plan_s* P, const double2* G, const float2* T, int max_sweeps, float tol,
                               float floor_rel, cudaStream_t s) {
  OsjFn fn = osj_fn(P->C);
  if (!fn) return SMSM_ERR_ARG;
  fn<<<OSJ_R * P->LD, 32 * osj_w(P->C), osj_smem(P->C), s>>>(G, T, P->eig, P->V, P->sweeps, P->C, P->Cp, max_sweeps,
                                                             tol, floor_rel, P->st, P->L);
  SMSM_LAUNCH_CHECK("k_jacobi_os");
  return SMSM_OK;
}
