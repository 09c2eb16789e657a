// Shared definitions of the SMS-MUSSELS CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/smsm.h"

// ----------------------------------------------------------------------------
// complex64 helpers (float2 = re, im)
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 conjf2(float2 a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulcj(float2 a, float2 b) {
  return cmk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmacj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// asynchronous 8-byte global -> shared copy (completes at cp_async_wait_all)
// Periodic penalty multiplier m_ii'[x][y] of one (direction, slice).  It is
// Hermitian in the shot pair (wt_ii'[d] = conj(wt_i'i[-d]) because W is), so only
// the upper triangle i <= i' is stored, in Ns(Ns+1)/2 planes [pk][x][y] with
// pk = i Ns - i(i-1)/2 + (i' - i); the lower entries are the conjugates.
__host__ __device__ constexpr int mult_planes(int Ns) { return Ns * (Ns + 1) / 2; }
__host__ __device__ constexpr int mult_plane(int i, int j, int Ns) { return i * Ns - i * (i - 1) / 2 + (j - i); }
// m_ij at offset off of a plane; m points at the slice's first plane
__device__ __forceinline__ float2 mult_at(const float2* __restrict__ m, int i, int j, int Ns, size_t NN, size_t off) {
  if (i <= j) return __ldg(m + (size_t)mult_plane(i, j, Ns) * NN + off);
  const float2 v = __ldg(m + (size_t)mult_plane(j, i, Ns) * NN + off);
  return cmk(v.x, -v.y);
}

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// ----------------------------------------------------------------------------
// FFT descriptor: length n = prod(rad[0..np)), radices in {2, 3, 4}.
// ----------------------------------------------------------------------------
struct FftDesc {
  int n;
  int np;
  unsigned code;  // radix of pass p in bits [2p, 2p+2): 0 -> 2, 1 -> 3, 2 -> 4 (no indexed param access)
  int rad[12];
};

// ----------------------------------------------------------------------------
// Device-side solver state (one per plan).
// ----------------------------------------------------------------------------
struct SolverState {
  double eps;      // current eps_k
  double eps0;     // eps_1
  double eps_min;  // eps_min_rel * eps_1
  int status;      // smsm_status set by device checks
  int pad;
};

struct DevReport {
  double eps[SMSM_MAX_OUTER];
  double rr_start[SMSM_MAX_OUTER];
  double rr_end[SMSM_MAX_OUTER];
  int sweeps[SMSM_MAX_OUTER];
};

// Maximum sizes of this build.
#define SMSM_MAX_C 320
#define SMSM_MAX_N 512
#define SMSM_MAX_SWEEPS 30
#define SMSM_PART_MAX 8192  // capacity of each partial-sum array (doubles)

struct smsm_plan_s {
  int L, Ns, Nc, N, r, C, Cp /* C rounded up to even */, M, Ldiv, P1 /* origins per axis: N-r+1, or N if periodic */,
      R2 /* 2r-1 */;
  int D;   // batch: independent problems (diffusion directions) sharing geometry and coil maps
  int flags;      // smsm_opts.flags
  int precision;  // smsm_opts.precision
  int periodic;   // smsm_opts.boundary == PERIODIC: patch origins over all of [0, N)^2, mod N
  int gram_tc;    // 1: tensor-core Gram
  int gram_tc_nG; // split-K partials of the tensor-core Gram (the autotuner may change it)
  int gram_nG_max; // split-K partials the Rpart buffer holds
  int tuned_lanes; // lanes chosen by the autotuner (0: none; used when params->lanes == 0)
  int eig_cluster; // 1: eigen step by one-sided block Jacobi on an 8-CTA cluster (C > 168, or asked for)
  float* Rpart;   // [LD][nG][2Cp][2Cp] tensor-core Gram partials
  int alias;      // 1: column stage of A^H A through the per-class coil correlations
  float2* acorr;  // [N(x)][L Ns][L Ns][M(class)] coil correlations of the aliasing classes
  float2* ash;    // [Ns][Ns]: exp(-2 pi j (i - N/2) q / Ns)
  int* devflag;   // device error flag raised by bounded waits (SMSM_ERR_TIMEOUT)
  int LD;  // D * L: number of (direction, slice) Hankel matrices
  int nvb; // CTAs per direction of the CG vector kernels (fixed at plan creation)
  int nband;  // pixels within r-1 of an edge
  int dev;
  FftDesc fN, fM;
  float sN;   // (-1)^(N/2)/sqrt(N)
  // tables (device)
  float2 *twN, *twM, *tw_shot, *cph, *Etab;
  // coil maps, transposed [L][Nc][x][y]
  float2* sensT;
  int has_sens;
  // work buffers
  float2 *hA, *hB;   // [L][Ns][N][N]
  float2* yh;        // [Ns][Nc][N][M] (x-major)
  float2* phaseT;    // [L][Ns][N][N] (x-major)
  float2 *xs, *bv, *rv, *pv, *qv;  // solver vectors [L][Ns][N][N]
  float2* ybuf;      // [Ns][Nc][M][N]
  double2* G64;      // [L][C][C]
  double2* Gpart;    // [L][nkx][C][C]
  int gram_nkx;
  float* eig;        // [L][Cp]
  int* sweeps;       // [L]
  float2 *V, *Wf;    // [LD][C][C]
  float2 *Gw, *Gw2;  // [LD][C][C] warm-start congruence V^H G V (and its half product)
  float2* wper;      // [L][Ns][Ns][R2*R2]
  float2* wcls;      // [LD][R2*R2 classes][Ns (i')][R2*R2 taps][Ns (i)] border correction taps
  float2* multT;     // [L][Ns(Ns+1)/2][N(x)][N(y)]: upper triangle of the Hermitian shot coupling
  double *part_pq_col, *part_pq_band, *part_rr;  // partial sums [D][PART]; part_rr: [2 banks][D][PART]
  SolverState* st;   // [D]
  DevReport* rep;
  size_t bytes;
  // graph cache for smsm_reconstruct: the captured solve and its instantiation
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  unsigned graph_gen;  // bumped whenever the captured solve is dropped (group launches re-check it)
  cudaStream_t cap_stream;
  cudaStream_t lane_s[SMSM_MAX_LANES];  // capture streams of lanes 1.. (lane 0 captures on cap_stream)
  cudaEvent_t lane_ev[2 * SMSM_MAX_LANES + 1];  // fork, per-lane join and eigen-step events
  smsm_params gparams;
  int has_graph;
  int graph_kernels;
  cudaEvent_t ev0, ev1;
  void* tpool;  // TimingPool (solver.cu): events bracketing timed stages
};

// ----------------------------------------------------------------------------
// error reporting (host)
// ----------------------------------------------------------------------------
void smsm_set_error(const char* fmt, ...);

#define SMSM_CUDA_TRY(call)                                                          \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      smsm_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                     __LINE__);                                                      \
      return SMSM_ERR_CUDA;                                                          \
    }                                                                                \
  } while (0)

#define SMSM_LAUNCH_CHECK(what)                                                        \
  do {                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess) {                                                           \
      smsm_set_error("launch of %s failed: %s", what, cudaGetErrorString(e_));         \
      return SMSM_ERR_CUDA;                                                            \
    }                                                                                  \
  } while (0)

// ----------------------------------------------------------------------------
// stage timing (host)
// ----------------------------------------------------------------------------
// Events bracketing the launches of the timed stages (smsm_params.timing).
// Recorded as external event nodes of the captured graph, so every replay
// re-records them on the device.
struct TimingPool {
  std::vector<cudaEvent_t> ev;  // 2 per bracket
  std::vector<int> stage;       // stage of bracket k
  size_t used = 0;              // brackets in the current graph
};

struct Timer {
  TimingPool* tp;
  int mask;
  cudaStream_t s;
  cudaError_t err = cudaSuccess;
  bool on(int stage) const { return tp && ((mask >> stage) & 1); }
  void begin(int stage) {
    if (!on(stage) || err != cudaSuccess) return;
    const size_t k = tp->used;
    while (tp->ev.size() < 2 * (k + 1)) {
      cudaEvent_t e;
      err = cudaEventCreate(&e);
      if (err != cudaSuccess) return;
      tp->ev.push_back(e);
    }
    if (tp->stage.size() < k + 1) tp->stage.resize(k + 1);
    tp->stage[k] = stage;
    err = cudaEventRecordWithFlags(tp->ev[2 * k], s, cudaEventRecordExternal);
  }
  void end(int stage) {
    if (!on(stage) || err != cudaSuccess) return;
    const size_t k = tp->used;
    err = cudaEventRecordWithFlags(tp->ev[2 * k + 1], s, cudaEventRecordExternal);
    tp->used = k + 1;
  }
};

// ----------------------------------------------------------------------------
// launchers implemented in the .cu files (all enqueue on `s`, return status)
// ----------------------------------------------------------------------------
// operators.cu
smsm_status launch_transpose(const float2* in, float2* out, int nb, int rows, int cols, cudaStream_t s);
smsm_status launch_rowfft_out_T(const smsm_plan_s* P, const float2* in, float2* out, int nb, int rows,
                                int inverse, cudaStream_t s);
smsm_status launch_rowfft_in_T(const smsm_plan_s* P, const float2* in, float2* out, int nb, int rows,
                               int inverse, cudaStream_t s);
// inverse row FFT of p (N rows per image) with the CG update p = r + beta p fused in
smsm_status launch_rowfft_out_T_cgp(const smsm_plan_s* P, float2* p, const float2* r, float2* out, int nb,
                                    const double* rr_new, const double* rr_old, int nrr, cudaStream_t s);
enum ColMode { COL_FWD = 0, COL_ADJ = 1, COL_NORMAL = 2, COL_PEN = 3 };
// Column-stage arguments (operators.cu, colfast.cu)
struct ColArgs {
  const float2* in;  // (offset per direction inside the kernel)
  float2* out;
  const float2* sensT;   // [L][Nc][x][y]
  const float2* phaseT;  // [L][Ns][x][y]
  const float2* multT;   // [L][Ns(Ns+1)/2][x][y] (upper triangle, see mult_at)
  const float2* twN;
  const float2* twM;
  const float2* tw_shot;  // [Ns][N]
  const float2* cph;      // [L][Ns][M]
  FftDesc fN, fM;
  int L, Ns, Nc, N, M;
  float sN, lambda;
  double* dot_part;  // [N] per-CTA partial of Re<img, acc> (nullable)
  int* errflag;      // device error flag (bounded waits that ran out)
};

// colfast.cu: warp-shuffle column stage of (A^H A + lambda P_W); returns SMSM_ERR_ARG when the
// geometry has no fast path (the caller then uses the generic kernel)
smsm_status launch_col_fast(const smsm_plan_s* P, const ColArgs& a, cudaStream_t s);
smsm_status colfast_init_attrs();

smsm_status launch_col(const smsm_plan_s* P, int mode, int with_phase, const float2* in, float2* out,
                       const float2* phaseT, const float2* multT, float lambda, double* dot_part,
                       cudaStream_t s);
// colalias.cu: column stage of (A^H A + lambda P_W) through the aliasing classes
int alias_supported(const smsm_plan_s* P);
size_t alias_corr_count(const smsm_plan_s* P);
smsm_status alias_init_attrs();
smsm_status launch_alias_corr(const smsm_plan_s* P, cudaStream_t s);
smsm_status launch_col_alias(const smsm_plan_s* P, const ColArgs& a, cudaStream_t s);
// hankel.cu
smsm_status launch_gram(const smsm_plan_s* P, const float2* x, double2* G, cudaStream_t s);
// gram_tc.cu
int gram_tc_supported(const smsm_plan_s* P);
int gram_tc_cp(const smsm_plan_s* P);
int gram_tc_nG(const smsm_plan_s* P);
int gram_tc_nG_candidates(const smsm_plan_s* P, int* out, int maxn);
smsm_status gram_tc_init_attrs();
smsm_status launch_gram_tc(const smsm_plan_s* P, const float2* x, double2* G, cudaStream_t s);
smsm_status launch_filters(const smsm_plan_s* P, const float2* W, cudaStream_t s);
smsm_status launch_band(const smsm_plan_s* P, const float2* x, float2* out, float scale, double* dot_part,
                        cudaStream_t s);
smsm_status launch_w_from_c128(const smsm_plan_s* P, const double2* W64, float2* W, cudaStream_t s);
// eig.cu
void solver_drop_graph(smsm_plan_s* P);
void solver_forget_plan(smsm_plan_s* P);
smsm_status launch_eig_weights(const smsm_plan_s* P, const double2* G, int outer, const smsm_params* prm,
                               cudaStream_t s, Timer* T);
smsm_status eig_init_attrs(const smsm_plan_s* P);
size_t eig_jacobi_smem(int Cp);
bool eig_pair_supported(int Cp);
bool eig_cluster_supported(int C);
smsm_status eig_cluster_init_attrs(int C);
smsm_status launch_eig_cluster(const smsm_plan_s* P, const double2* G, const float2* T, int max_sweeps, float tol,
                               float floor_rel, cudaStream_t s);
smsm_status operators_init_attrs();
size_t smsm_col_smem_bytes(const smsm_plan_s* P);
int band_blocks(const smsm_plan_s* P);
smsm_status band_init_attrs(const smsm_plan_s* P);
// cnn.cu
smsm_status cnn_shape(const smsm_cnn_s* c, int* B, int* H, int* W, int* maxn);
// solver.cu
int vec_blocks(const smsm_plan_s* P);
smsm_status solver_reconstruct(smsm_plan_s* P, const void* y, void* x, const smsm_params* prm,
                               smsm_report* report, cudaStream_t s);
smsm_status solver_autotune(smsm_plan_s* P, const void* y, const smsm_params* prm, smsm_tune_report* out,
                            cudaStream_t s);
int tune_cache_lookup(const smsm_plan_s* P, int* nG, int* lanes);
void solver_free_timing(smsm_plan_s* P);
smsm_status solver_reconstruct_groups(int n, smsm_plan_s* const* plans, const void* const* ys, void* const* xs,
                                      const smsm_params* prm, smsm_report* reports, cudaStream_t s);
smsm_status solver_sense(smsm_plan_s* P, const void* y, const void* phase, void* x, int J, smsm_report* report,
                         cudaStream_t s);
smsm_status apply_normal_pen(smsm_plan_s* P, const float2* v, float2* q, float lambda, int with_dots,
                             cudaStream_t s);
