// Eigen-decomposition of the per-slice Gram G_l and the weight update.
//
// The low-rank penalty of Eq. 10 is handled by iteratively reweighted least
// squares: W_l = V diag((s + eps)^(-1/2)) V^H (nuclear-norm majoriser) or the
// projector onto the C - rank smallest eigenvectors (a fixed common rank, the
// Methods' choice of "the same rank for every slice").  The eigenvectors of
// the annihilation relation's null space (Eq. 9) are the annihilating filters.
//
// Eigensolver: two-sided cyclic Jacobi for Hermitian matrices, one CTA per
// slice, G held in shared memory, parallel round-robin ordering (C/2
// disjoint rotations per round, all 2x2 blocks updated at once).  The
// rotations of every round are logged, and a second kernel replays them on
// the rows of V (independent rows, spread over many CTAs), so V never has to
// share the CTA's shared memory with G.
//
// Precision: FP32 storage and rotations.  The Gram itself is only
// FP32-accurate (its inputs are FP32), and a Jacobi sweep is backward stable
// to u*||G||, so an FP64 eigensolver would not make W more accurate -- while
// FP64 on this part runs at about 1/60 of the FP32 rate.
#include <math.h>

#include "common.cuh"

__device__ __forceinline__ void jpair(int round, int k, int Cp, int& p, int& q) {
  const int m = Cp - 1;
  int a, b;
  if (k == 0) {
    a = 0;
    b = 1 + (round % m);
  } else {
    a = 1 + ((k + round) % m);
    b = 1 + ((m - k + round) % m);
  }
  p = min(a, b);
  q = max(a, b);
}

__device__ __forceinline__ bool is_ident(float4 J) { return J.y == 0.f && J.z == 1.f && J.w == 0.f; }

// J = [[c, s], [-s e, c e]],  e = exp(-i phi) = (er, ei), phi = arg(G_pq)
__global__ void __launch_bounds__(1024) k_jacobi(const double2* __restrict__ G, float* __restrict__ eig,
                                                 float4* __restrict__ rlog, int* __restrict__ sweeps_out, int C,
                                                 int Cp, int max_sweeps, float tol) {
  extern __shared__ float2 g[];
  float4* rot = reinterpret_cast<float4*>(g + (size_t)Cp * Cp);
  __shared__ int nrot;
  __shared__ float dmax;
  const int l = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const double2* Gl = G + (size_t)l * C * C;
  for (int e = tid; e < Cp * Cp; e += nt) {
    int a = e / Cp, b = e - a * Cp;
    g[e] = (a < C && b < C) ? cmk((float)Gl[(size_t)a * C + b].x, (float)Gl[(size_t)a * C + b].y) : cmk(0.f, 0.f);
  }
  if (tid == 0) dmax = 0.f;
  __syncthreads();
  if (tid < Cp) atomicMax(reinterpret_cast<int*>(&dmax), __float_as_int(fmaxf(g[tid * Cp + tid].x, 0.f)));
  __syncthreads();
  // rotations below this absolute size only churn rounding noise
  const float floor_abs = 1e-7f * dmax;
  const int half = Cp / 2;
  int sw = 0;
  for (; sw < max_sweeps; ++sw) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int round = 0; round < Cp - 1; ++round) {
      if (tid < half) {
        int p, q;
        jpair(round, tid, Cp, p, q);
        const float a = g[p * Cp + p].x, d = g[q * Cp + q].x;
        const float2 b = g[p * Cp + q];
        const float babs = hypotf(b.x, b.y);
        float4 J = make_float4(1.f, 0.f, 1.f, 0.f);
        if (babs > floor_abs && babs > tol * sqrtf(fabsf(a * d))) {
          const float theta = (d - a) / (2.f * babs);
          const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
          const float c = 1.f / sqrtf(t * t + 1.f);
          J = make_float4(c, t * c, b.x / babs, -b.y / babs);
          atomicAdd(&nrot, 1);
        }
        rot[tid] = J;
        rlog[(((size_t)l * SMSM_MAX_SWEEPS + sw) * (Cp - 1) + round) * half + tid] = J;
      }
      __syncthreads();
      for (int blk = tid; blk < half * half; blk += nt) {
        const int k1 = blk / half, k2 = blk - k1 * half;
        const float4 J1 = rot[k1], J2 = rot[k2];
        if (is_ident(J1) && is_ident(J2)) continue;
        int p1, q1, p2, q2;
        jpair(round, k1, Cp, p1, q1);
        jpair(round, k2, Cp, p2, q2);
        float2 B00 = g[p1 * Cp + p2], B01 = g[p1 * Cp + q2];
        float2 B10 = g[q1 * Cp + p2], B11 = g[q1 * Cp + q2];
        // T = J1^H B : row0 = c B0 - s conj(e1) B1 ; row1 = s B0 + c conj(e1) B1
        const float2 e1c = cmk(J1.z, -J1.w);
        float2 T00 = csub(cscale(B00, J1.x), cscale(cmul(e1c, B10), J1.y));
        float2 T01 = csub(cscale(B01, J1.x), cscale(cmul(e1c, B11), J1.y));
        float2 T10 = cadd(cscale(B00, J1.y), cscale(cmul(e1c, B10), J1.x));
        float2 T11 = cadd(cscale(B01, J1.y), cscale(cmul(e1c, B11), J1.x));
        // O = T J2 : col0 = c T0 - s e2 T1 ; col1 = s T0 + c e2 T1
        const float2 e2 = cmk(J2.z, J2.w);
        float2 O00 = csub(cscale(T00, J2.x), cscale(cmul(T01, e2), J2.y));
        float2 O10 = csub(cscale(T10, J2.x), cscale(cmul(T11, e2), J2.y));
        float2 O01 = cadd(cscale(T00, J2.y), cscale(cmul(T01, e2), J2.x));
        float2 O11 = cadd(cscale(T10, J2.y), cscale(cmul(T11, e2), J2.x));
        if (k1 == k2) {
          O01 = cmk(0.f, 0.f);
          O10 = cmk(0.f, 0.f);
          O00.y = 0.f;
          O11.y = 0.f;
        }
        g[p1 * Cp + p2] = O00;
        g[p1 * Cp + q2] = O01;
        g[q1 * Cp + p2] = O10;
        g[q1 * Cp + q2] = O11;
      }
      __syncthreads();
    }
    const bool done = (nrot == 0);
    __syncthreads();
    if (done) break;
  }
  for (int j = tid; j < Cp; j += nt) eig[(size_t)l * Cp + j] = g[j * Cp + j].x;
  if (tid == 0) sweeps_out[l] = sw;
}

// V = product of the logged rotations; one warp per row of V.
__global__ void __launch_bounds__(256) k_vapply(const float4* __restrict__ rlog, const int* __restrict__ sweeps,
                                                float2* __restrict__ V, int C, int Cp) {
  extern __shared__ float2 rows[];
  const int l = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y * 8 + w;
  if (t >= C) return;
  float2* row = rows + w * Cp;
  for (int j = lane; j < Cp; j += 32) row[j] = cmk(j == t ? 1.f : 0.f, 0.f);
  __syncwarp();
  const int nsw = sweeps[l];
  const int half = Cp / 2;
  for (int sw = 0; sw < nsw; ++sw) {
    for (int round = 0; round < Cp - 1; ++round) {
      const float4* lg = rlog + (((size_t)l * SMSM_MAX_SWEEPS + sw) * (Cp - 1) + round) * half;
      for (int k = lane; k < half; k += 32) {
        const float4 J = lg[k];
        if (is_ident(J)) continue;
        int p, q;
        jpair(round, k, Cp, p, q);
        const float2 vp = row[p], vq = row[q];
        const float2 evq = cmul(cmk(J.z, J.w), vq);
        row[p] = csub(cscale(vp, J.x), cscale(evq, J.y));
        row[q] = cadd(cscale(vp, J.y), cscale(evq, J.x));
      }
      __syncwarp();
    }
  }
  float2* Vr = V + ((size_t)l * C + t) * C;
  for (int j = lane; j < C; j += 32) Vr[j] = row[j];
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

// W[a][b] = sum_j V[a][j] f_j conj(V[b][j])
__global__ void __launch_bounds__(256) k_weights(const float2* __restrict__ V, const float* __restrict__ eig,
                                                 const SolverState* __restrict__ st, float2* __restrict__ W, int C,
                                                 int Cp, int mode, int rank, int L) {
  __shared__ float f[SMSM_MAX_C];
  __shared__ float2 Va[16][SMSM_MAX_C];
  const int l = blockIdx.x, a0 = blockIdx.y * 16;
  const float* s = eig + (size_t)l * Cp;
  const double eps = st[l / L].eps;  // l is the flat (direction, slice) index
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    if (mode == SMSM_MODE_NULLSPACE) {
      int rk = 0;
      const float sj = s[j];
      for (int k = 0; k < C; ++k) rk += (s[k] < sj) || (s[k] == sj && k < j);
      f[j] = rk < C - rank ? 1.f : 0.f;
    } else {
      f[j] = (float)(1.0 / sqrt(fmax((double)s[j], 0.0) + eps));
    }
  }
  const float2* Vl = V + (size_t)l * C * C;
  for (int e = threadIdx.x; e < 16 * C; e += blockDim.x) {
    int ar = e / C, j = e - ar * C;
    Va[ar][j] = (a0 + ar < C) ? Vl[(size_t)(a0 + ar) * C + j] : cmk(0.f, 0.f);
  }
  __syncthreads();
  const int ar = threadIdx.x >> 4;
  const int a = a0 + ar;
  if (a >= C) return;
  for (int b = threadIdx.x & 15; b < C; b += 16) {
    const float2* Vb = Vl + (size_t)b * C;
    float2 acc = cmk(0.f, 0.f);
    for (int j = 0; j < C; ++j) {
      float2 va = cscale(Va[ar][j], f[j]);
      float2 vb = Vb[j];
      // va * conj(vb)
      acc.x += va.x * vb.x + va.y * vb.y;
      acc.y += va.y * vb.x - va.x * vb.y;
    }
    W[((size_t)l * C + a) * C + b] = acc;
  }
}

static size_t jacobi_smem(int Cp) { return (size_t)Cp * Cp * sizeof(float2) + (size_t)(Cp / 2) * sizeof(float4); }

smsm_status eig_init_attrs(int Cp) {
  size_t sm = jacobi_smem(Cp);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) {
    smsm_set_error("Jacobi kernel cannot get %zu bytes of shared memory: %s", sm, cudaGetErrorString(e));
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

size_t eig_jacobi_smem(int Cp) { return jacobi_smem(Cp); }

smsm_status launch_eig_weights(const smsm_plan_s* P, const double2* G, int outer, const smsm_params* prm,
                               cudaStream_t s, Timer* T) {
  const int Cp = P->Cp;
  int msw = prm->max_sweeps > 0 ? prm->max_sweeps : 15;
  if (msw > SMSM_MAX_SWEEPS) msw = SMSM_MAX_SWEEPS;
  if (T) T->begin(SMSM_STAGE_EIG);
  k_jacobi<<<P->LD, 1024, jacobi_smem(Cp), s>>>(G, P->eig, P->rotlog, P->sweeps, P->C, Cp, msw, 1e-6f);
  SMSM_LAUNCH_CHECK("k_jacobi");
  if (T) T->end(SMSM_STAGE_EIG);
  if (T) T->begin(SMSM_STAGE_VAPPLY);
  dim3 gv(P->LD, (P->C + 7) / 8);
  k_vapply<<<gv, 256, (size_t)8 * Cp * sizeof(float2), s>>>(P->rotlog, P->sweeps, P->V, P->C, Cp);
  SMSM_LAUNCH_CHECK("k_vapply");
  if (T) T->end(SMSM_STAGE_VAPPLY);
  if (T) T->begin(SMSM_STAGE_WEIGHTS);
  k_eps<<<P->D, 256, 0, s>>>(P->eig, P->sweeps, P->st, P->rep, P->L, P->C, Cp, outer, prm->eps0_rel, prm->eta,
                          prm->eps_min_rel);
  SMSM_LAUNCH_CHECK("k_eps");
  dim3 gw(P->LD, (P->C + 15) / 16);
  k_weights<<<gw, 256, 0, s>>>(P->V, P->eig, P->st, P->Wf, P->C, Cp, prm->mode, prm->rank, P->L);
  SMSM_LAUNCH_CHECK("k_weights");
  if (T) T->end(SMSM_STAGE_WEIGHTS);
  return SMSM_OK;
}
