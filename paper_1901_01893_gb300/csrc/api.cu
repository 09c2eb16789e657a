// C ABI of the SMS-MUSSELS library: plan construction (host FP64 tables,
// device workspace) and the entry points declared in include/smsm.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

void smsm_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* smsm_last_error(void) { return g_err; }

extern "C" void smsm_default_params(smsm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->lambda = 1e-2;
  p->eps0_rel = 1e-2;
  p->eta = 1.5;
  p->eps_min_rel = 1e-2;
  p->outer_iters = 10;
  p->cg_iters = 10;
  p->mode = SMSM_MODE_IRLS;
  p->rank = 0;
  p->warm = 0;
  p->max_sweeps = SMSM_MAX_SWEEPS;
}

// ---------------------------------------------------------------------------
// host tables (FP64, rounded once to FP32)
// ---------------------------------------------------------------------------
static bool factor_radix(int n, FftDesc* d) {
  d->n = n;
  d->np = 0;
  int m = n;
  while (m % 4 == 0 && d->np < 12) {
    d->rad[d->np++] = 4;
    m /= 4;
  }
  while (m % 2 == 0 && d->np < 12) {
    d->rad[d->np++] = 2;
    m /= 2;
  }
  while (m % 3 == 0 && d->np < 12) {
    d->rad[d->np++] = 3;
    m /= 3;
  }
  d->code = 0;
  for (int p = 0; p < d->np; ++p) d->code |= (unsigned)(d->rad[p] == 4 ? 2 : (d->rad[p] == 3 ? 1 : 0)) << (2 * p);
  return m == 1 && n >= 2;
}

// exp(-j 2 pi num / den) with num reduced exactly modulo den first
static float2 expi_frac(long long num, long long den) {
  long long r = num % den;
  if (r < 0) r += den;
  const double a = -2.0 * M_PI * (double)r / (double)den;
  return make_float2((float)cos(a), (float)sin(a));
}

template <typename T>
static smsm_status dalloc(smsm_plan_s* P, T** p, size_t count) {
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    smsm_set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return SMSM_ERR_NOMEM;
  }
  P->bytes += bytes;
  return SMSM_OK;
}

template <typename T>
static smsm_status upload(T* d, const std::vector<T>& h) {
  SMSM_CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SMSM_OK;
}

static void free_plan(smsm_plan_s* P) {
  if (!P) return;
  void* ptrs[] = {P->twN,  P->twM,  P->tw_shot, P->cph,  P->Etab,  P->sensT, P->hA,   P->hB,
                  P->yh,   P->phaseT, P->xs,    P->bv,   P->rv,    P->pv,    P->qv,   P->ybuf,
                  P->G64,  P->Gpart, P->eig,    P->sweeps, P->V,   P->Wf,   P->wper, P->Gw, P->Gw2,
                  P->wcls, P->multT, P->part_pq_col, P->part_pq_band, P->part_rr, P->st, P->rep,
                  P->Rpart, P->devflag, P->acorr, P->ash};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  solver_forget_plan(P);
  solver_drop_graph(P);
  solver_free_timing(P);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  for (int k = 0; k < SMSM_MAX_LANES; ++k)
    if (P->lane_s[k]) cudaStreamDestroy(P->lane_s[k]);
  for (int k = 0; k < 2 * SMSM_MAX_LANES + 1; ++k)
    if (P->lane_ev[k]) cudaEventDestroy(P->lane_ev[k]);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  free(P);
}

extern "C" smsm_status smsm_plan(smsm_plan_t* out, int mb, int shots, int coils, int nx, int ny, int filter,
                                 const smsm_opts* opts) {
  if (!out) {
    smsm_set_error("smsm_plan: out is NULL");
    return SMSM_ERR_ARG;
  }
  *out = nullptr;
  const int N = nx;
  if (mb < 1 || shots < 1 || coils < 1 || nx != ny || N < 16 || N > SMSM_MAX_N || (N & 1) || N % shots) {
    smsm_set_error("smsm_plan: need mb, shots, coils >= 1, nx == ny even in [16, %d], ny %% shots == 0 "
                   "(got mb=%d shots=%d coils=%d nx=%d ny=%d)", SMSM_MAX_N, mb, shots, coils, nx, ny);
    return SMSM_ERR_ARG;
  }
  if (shots > 8) {
    smsm_set_error("smsm_plan: at most 8 shots in this build (got %d)", shots);
    return SMSM_ERR_ARG;
  }
  const int M = N / shots;
  FftDesc fN, fM;
  if (!factor_radix(N, &fN) || !factor_radix(M, &fM)) {
    smsm_set_error("smsm_plan: N=%d and N/shots=%d must be of the form 2^a 3^b (and N/shots >= 2)", N, M);
    return SMSM_ERR_ARG;
  }
  const int r = filter;
  if (r < 1 || r > 12 || 2 * r > N) {
    smsm_set_error("smsm_plan: filter must be in [1, min(12, N/2)] (got %d)", r);
    return SMSM_ERR_ARG;
  }
  const int C = shots * r * r;
  const int Cp = C + (C & 1);
  const int flags = opts ? opts->flags : 0;
  const int eig_cluster = !eig_pair_supported(Cp) || (flags & SMSM_FLAG_CLUSTER_EIG);
  if (C > SMSM_MAX_C || (eig_cluster && !eig_cluster_supported(C))) {
    smsm_set_error("smsm_plan: shots*filter^2 = %d is outside the eigensolver's range (at most %d; at least 65 "
                   "with SMSM_FLAG_CLUSTER_EIG)", C, SMSM_MAX_C);
    return SMSM_ERR_ARG;
  }
  const int caipi_div = (opts && opts->caipi_div > 0) ? opts->caipi_div : mb;
  const int D = (opts && opts->batch > 0) ? opts->batch : 1;
  if (D > 4096) {
    smsm_set_error("smsm_plan: batch must be in [1, 4096] (got %d)", D);
    return SMSM_ERR_ARG;
  }

  smsm_plan_s* P = (smsm_plan_s*)calloc(1, sizeof(smsm_plan_s));
  if (!P) {
    smsm_set_error("smsm_plan: host allocation failed");
    return SMSM_ERR_NOMEM;
  }
  P->L = mb;
  P->Ns = shots;
  P->Nc = coils;
  P->N = N;
  P->r = r;
  P->C = C;
  P->Cp = Cp;
  P->M = M;
  P->Ldiv = caipi_div;
  P->D = D;
  P->LD = D * mb;
  P->flags = flags;
  P->eig_cluster = eig_cluster;
  P->precision = opts ? opts->precision : SMSM_PRECISION_FP32;
  if (P->precision != SMSM_PRECISION_FP32 && P->precision != SMSM_PRECISION_BF16_SPLIT) {
    free(P);
    smsm_set_error("smsm_plan: unknown precision %d", opts->precision);
    return SMSM_ERR_ARG;
  }
  const int boundary = opts ? opts->boundary : SMSM_BOUNDARY_VALID;
  if (boundary != SMSM_BOUNDARY_VALID && boundary != SMSM_BOUNDARY_PERIODIC) {
    free(P);
    smsm_set_error("smsm_plan: unknown boundary %d", boundary);
    return SMSM_ERR_ARG;
  }
  P->periodic = boundary == SMSM_BOUNDARY_PERIODIC;
  P->gram_tc = gram_tc_supported(P) && !(P->flags & SMSM_FLAG_GENERIC_KERNELS);
  if (P->precision == SMSM_PRECISION_BF16_SPLIT && !gram_tc_supported(P)) {
    free(P);
    smsm_set_error("smsm_plan: the BF16 split form needs C = shots*filter^2 <= 144");
    return SMSM_ERR_ARG;
  }
  if (P->precision == SMSM_PRECISION_BF16_SPLIT) P->gram_tc = 1;
  P->alias = !(P->flags & (SMSM_FLAG_GENERIC_KERNELS | SMSM_FLAG_PER_COIL_NORMAL)) && alias_supported(P);
  P->P1 = P->periodic ? N : N - r + 1;
  P->R2 = 2 * r - 1;
  P->fN = fN;
  P->fM = fM;
  P->sN = (float)(((N / 2) % 2 ? -1.0 : 1.0) / sqrt((double)N));
  const int inner = N - 2 * (r - 1);
  P->nband = P->periodic ? 0 : N * N - (inner > 0 ? inner * inner : 0);
  P->gram_nkx = (P->P1 + 15) / 16;
  cudaGetDevice(&P->dev);

  smsm_status st = SMSM_OK;
  const size_t NN = (size_t)N * N;
  const size_t nvec = (size_t)D * mb * shots * NN;  // one batch of unknowns
  const size_t LD = (size_t)D * mb;
  const size_t nyv = (size_t)D * shots * coils * M * N;
  const int R2 = P->R2;
#define A(ptr, cnt) \
  if (!st) st = dalloc(P, &P->ptr, (size_t)(cnt))
  A(twN, N);
  A(twM, M);
  A(tw_shot, (size_t)shots * N);
  A(cph, (size_t)mb * shots * M);
  A(Etab, (size_t)R2 * N);
  A(sensT, (size_t)mb * coils * NN);
  A(hA, nvec);
  A(hB, nvec);
  A(yh, nyv);
  A(phaseT, nvec);
  A(xs, nvec);
  A(bv, nvec);
  A(rv, nvec);
  A(pv, nvec);
  A(qv, nvec);
  A(ybuf, nyv);
  A(G64, LD * C * C);
  A(Gpart, LD * P->gram_nkx * C * C);
  A(eig, LD * Cp);
  A(sweeps, LD);
  A(V, LD * C * C);
  A(Wf, LD * C * C);
  A(Gw, LD * C * C);
  A(Gw2, LD * C * C);
  A(wper, LD * shots * shots * R2 * R2);
  A(wcls, LD * R2 * R2 * shots * shots * R2 * R2);
  A(multT, LD * mult_planes(shots) * NN);
  A(part_pq_col, (size_t)D * SMSM_PART_MAX);
  A(part_pq_band, (size_t)D * SMSM_PART_MAX);
  A(part_rr, (size_t)2 * D * SMSM_PART_MAX);
  A(st, D);
  if (P->gram_tc) {
    P->gram_tc_nG = gram_tc_nG(P);
    int cand[8];
    const int nc = gram_tc_nG_candidates(P, cand, 8);
    P->gram_nG_max = P->gram_tc_nG;
    for (int k = 0; k < nc; ++k) P->gram_nG_max = cand[k] > P->gram_nG_max ? cand[k] : P->gram_nG_max;
    int tnG = 0, tl = 0;
    if (tune_cache_lookup(P, &tnG, &tl)) {  // an earlier plan of this shape was tuned
      if (tnG > 0 && tnG <= P->gram_nG_max) P->gram_tc_nG = tnG;
      P->tuned_lanes = tl;
    }
    const size_t R2C = 2 * (size_t)gram_tc_cp(P);
    A(Rpart, LD * P->gram_nG_max * R2C * R2C);
  } else {
    int tnG = 0, tl = 0;
    if (tune_cache_lookup(P, &tnG, &tl)) P->tuned_lanes = tl;
  }
  if (P->alias) {
    A(acorr, alias_corr_count(P));
    A(ash, (size_t)shots * shots);
  }
  A(devflag, 1);
  A(rep, SMSM_MAX_LANES);  // one report record per lane; lane 0's is the one returned
#undef A
  if (st) {
    free_plan(P);
    return st;
  }
  P->nvb = vec_blocks(P);  // fixed for the plan: lanes (sub-batches) reduce in the same order
  if (band_blocks(P) > SMSM_PART_MAX || vec_blocks(P) > SMSM_PART_MAX) {
    free_plan(P);
    smsm_set_error("smsm_plan: problem too large for the partial-sum buffers");
    return SMSM_ERR_ARG;
  }
  // tables
  {
    std::vector<float2> h(N);
    for (int k = 0; k < N; ++k) h[k] = expi_frac(k, N);
    st = upload(P->twN, h);
  }
  if (!st) {
    std::vector<float2> h(M);
    for (int k = 0; k < M; ++k) h[k] = expi_frac(k, M);
    st = upload(P->twM, h);
  }
  if (!st) {
    // tw_i[y] = exp(-j 2 pi (i - N/2)(y - N/2)/N)
    std::vector<float2> h((size_t)shots * N);
    for (int i = 0; i < shots; ++i)
      for (int y = 0; y < N; ++y) h[(size_t)i * N + y] = expi_frac((long long)(i - N / 2) * (y - N / 2), N);
    st = upload(P->tw_shot, h);
  }
  if (!st) {
    // cph[l][i][m] = exp(-j 2 pi l (m Ns + i - N/2)/Ldiv) * exp(+j 2 pi m (N/2)/M) / sqrt(N)
    std::vector<float2> h((size_t)mb * shots * M);
    for (int l = 0; l < mb; ++l)
      for (int i = 0; i < shots; ++i)
        for (int m = 0; m < M; ++m) {
          const long long n = (long long)m * shots + i - N / 2;
          long long a = ((long long)l * n) % caipi_div;
          if (a < 0) a += caipi_div;
          long long b = ((long long)m * (N / 2)) % M;
          const double ang = -2.0 * M_PI * (double)a / caipi_div + 2.0 * M_PI * (double)b / M;
          const double sc = 1.0 / sqrt((double)N);
          h[((size_t)l * shots + i) * M + m] = make_float2((float)(cos(ang) * sc), (float)(sin(ang) * sc));
        }
    st = upload(P->cph, h);
  }
  if (!st) {
    // E[d][n] = exp(-j 2 pi (d - (r-1)) (n - N/2)/N)
    std::vector<float2> h((size_t)R2 * N);
    for (int d = 0; d < R2; ++d)
      for (int n = 0; n < N; ++n) h[(size_t)d * N + n] = expi_frac((long long)(d - (r - 1)) * (n - N / 2), N);
    st = upload(P->Etab, h);
  }
  if (!st && P->alias) {
    // ash[i][q] = exp(-j 2 pi (i - N/2) q / Ns)
    std::vector<float2> h((size_t)shots * shots);
    for (int i = 0; i < shots; ++i)
      for (int q = 0; q < shots; ++q) h[(size_t)i * shots + q] = expi_frac((long long)(i - N / 2) * q, shots);
    st = upload(P->ash, h);
  }
  if (!st) st = operators_init_attrs();
  if (!st) st = colfast_init_attrs();
  if (!st) st = alias_init_attrs();
  if (!st) st = band_init_attrs(P);
  if (!st) st = gram_tc_init_attrs();
  if (!st) {
    cudaError_t e = cudaMemset(P->devflag, 0, sizeof(int));
    if (e != cudaSuccess) {
      smsm_set_error("smsm_plan: %s", cudaGetErrorString(e));
      st = SMSM_ERR_CUDA;
    }
  }
  if (!st) st = eig_init_attrs(P);
  if (!st && smsm_col_smem_bytes(P) > 200 * 1024) {
    smsm_set_error("smsm_plan: column stage would need %zu bytes of shared memory", smsm_col_smem_bytes(P));
    st = SMSM_ERR_ARG;
  }
  if (!st) {
    cudaError_t e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    for (int k = 1; k < SMSM_MAX_LANES && e == cudaSuccess; ++k)
      e = cudaStreamCreateWithFlags(&P->lane_s[k], cudaStreamNonBlocking);
    for (int k = 0; k < 2 * SMSM_MAX_LANES + 1 && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&P->lane_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&P->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&P->ev1);
    if (e == cudaSuccess) e = cudaMemset(P->part_pq_band, 0, sizeof(double) * SMSM_PART_MAX * D);
    if (e != cudaSuccess) {
      smsm_set_error("smsm_plan: %s", cudaGetErrorString(e));
      st = SMSM_ERR_CUDA;
    }
  }
  if (st) {
    free_plan(P);
    return st;
  }
  *out = P;
  return SMSM_OK;
}

extern "C" smsm_status smsm_plan_destroy(smsm_plan_t plan) {
  if (plan) {
    cudaDeviceSynchronize();
    free_plan(plan);
  }
  return SMSM_OK;
}

extern "C" size_t smsm_plan_workspace_bytes(smsm_plan_t plan) { return plan ? plan->bytes : 0; }

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static smsm_status check_ptr(const char* fn, const char* name, const void* p) {
  if (!p) {
    smsm_set_error("%s: %s is NULL", fn, name);
    return SMSM_ERR_ARG;
  }
  if (!aligned16(p)) {
    smsm_set_error("%s: %s is not 16-byte aligned", fn, name);
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

#define CHECK_PTR(fn, p)                               \
  do {                                                 \
    smsm_status s_ = check_ptr(fn, #p, p);             \
    if (s_) return s_;                                 \
  } while (0)

#define CHECK_PLAN(fn)                                 \
  do {                                                 \
    if (!plan) {                                       \
      smsm_set_error("%s: plan is NULL", fn);          \
      return SMSM_ERR_ARG;                             \
    }                                                  \
  } while (0)

static cudaStream_t S(void* s) { return (cudaStream_t)s; }

extern "C" smsm_status smsm_plan_set_sens(smsm_plan_t plan, const void* sens, void* stream) {
  CHECK_PLAN("smsm_plan_set_sens");
  CHECK_PTR("smsm_plan_set_sens", sens);
  smsm_status st = launch_transpose((const float2*)sens, plan->sensT, plan->L * plan->Nc, plan->N, plan->N, S(stream));
  if (!st && plan->alias) st = launch_alias_corr(plan, S(stream));
  if (!st) plan->has_sens = 1;
  return st;
}

static smsm_status need_sens(smsm_plan_t plan, const char* fn) {
  if (!plan->has_sens) {
    smsm_set_error("%s: coil sensitivities not set (call smsm_plan_set_sens first)", fn);
    return SMSM_ERR_STATE;
  }
  return SMSM_OK;
}

extern "C" smsm_status smsm_forward(smsm_plan_t plan, const void* x, const void* phase, void* y, void* stream) {
  CHECK_PLAN("smsm_forward");
  CHECK_PTR("smsm_forward", x);
  CHECK_PTR("smsm_forward", y);
  if (phase) CHECK_PTR("smsm_forward", phase);
  smsm_status st;
  if ((st = need_sens(plan, "smsm_forward"))) return st;
  const int L = plan->L, Ns = plan->Ns, N = plan->N, D = plan->D;
  cudaStream_t s = S(stream);
  if (phase && (st = launch_transpose((const float2*)phase, plan->phaseT, D * L * Ns, N, N, s))) return st;
  if ((st = launch_rowfft_out_T(plan, (const float2*)x, plan->hA, D * (phase ? L : L * Ns), N, 1, s))) return st;
  if ((st = launch_col(plan, COL_FWD, phase != nullptr, plan->hA, plan->yh, plan->phaseT, nullptr, 0.f, nullptr, s)))
    return st;
  return launch_rowfft_in_T(plan, plan->yh, (float2*)y, D * Ns * plan->Nc, plan->M, 0, s);
}

extern "C" smsm_status smsm_adjoint(smsm_plan_t plan, const void* y, const void* phase, void* x, void* stream) {
  CHECK_PLAN("smsm_adjoint");
  CHECK_PTR("smsm_adjoint", y);
  CHECK_PTR("smsm_adjoint", x);
  if (phase) CHECK_PTR("smsm_adjoint", phase);
  smsm_status st;
  if ((st = need_sens(plan, "smsm_adjoint"))) return st;
  const int L = plan->L, Ns = plan->Ns, N = plan->N, D = plan->D;
  cudaStream_t s = S(stream);
  if ((st = launch_rowfft_out_T(plan, (const float2*)y, plan->yh, D * Ns * plan->Nc, plan->M, 1, s))) return st;
  if (phase && (st = launch_transpose((const float2*)phase, plan->phaseT, D * L * Ns, N, N, s))) return st;
  if ((st = launch_col(plan, COL_ADJ, phase != nullptr, plan->yh, plan->hB, plan->phaseT, nullptr, 0.f, nullptr, s)))
    return st;
  return launch_rowfft_in_T(plan, plan->hB, (float2*)x, D * (phase ? L : L * Ns), N, 0, s);
}

extern "C" smsm_status smsm_hankel_gram(smsm_plan_t plan, const void* x, void* G, void* stream) {
  CHECK_PLAN("smsm_hankel_gram");
  CHECK_PTR("smsm_hankel_gram", x);
  CHECK_PTR("smsm_hankel_gram", G);
  if ((uintptr_t)x & 15u) {
    smsm_set_error("smsm_hankel_gram: x must be 16-byte aligned");
    return SMSM_ERR_ARG;
  }
  return launch_gram(plan, (const float2*)x, (double2*)G, S(stream));
}

extern "C" smsm_status smsm_apply_filters(smsm_plan_t plan, const void* W, const void* x, void* out, void* stream) {
  CHECK_PLAN("smsm_apply_filters");
  CHECK_PTR("smsm_apply_filters", W);
  CHECK_PTR("smsm_apply_filters", x);
  CHECK_PTR("smsm_apply_filters", out);
  if (x == out) {
    smsm_set_error("smsm_apply_filters: x and out must not alias");
    return SMSM_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  smsm_status st;
  const int B = plan->D * plan->L * plan->Ns;
  if ((st = launch_w_from_c128(plan, (const double2*)W, plan->Wf, s))) return st;
  if ((st = launch_filters(plan, plan->Wf, s))) return st;
  if ((st = launch_rowfft_out_T(plan, (const float2*)x, plan->hA, B, plan->N, 1, s))) return st;
  if ((st = launch_col(plan, COL_PEN, 0, plan->hA, plan->hB, nullptr, plan->multT, 1.f, nullptr, s))) return st;
  if ((st = launch_rowfft_in_T(plan, plan->hB, (float2*)out, B, plan->N, 0, s))) return st;
  return launch_band(plan, (const float2*)x, (float2*)out, 1.f, nullptr, s);
}

extern "C" smsm_status smsm_fft2c(smsm_plan_t plan, const void* in, void* out, int count, int inverse, void* stream) {
  CHECK_PLAN("smsm_fft2c");
  CHECK_PTR("smsm_fft2c", in);
  CHECK_PTR("smsm_fft2c", out);
  if (count < 0) {
    smsm_set_error("smsm_fft2c: count < 0");
    return SMSM_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  const int chunk = plan->D * plan->L * plan->Ns;
  const size_t NN = (size_t)plan->N * plan->N;
  smsm_status st;
  for (int b0 = 0; b0 < count; b0 += chunk) {
    const int nb = count - b0 < chunk ? count - b0 : chunk;
    const float2* src = (const float2*)in + (size_t)b0 * NN;
    float2* dst = (float2*)out + (size_t)b0 * NN;
    if ((st = launch_rowfft_out_T(plan, src, plan->hA, nb, plan->N, inverse != 0, s))) return st;
    if ((st = launch_rowfft_out_T(plan, plan->hA, dst, nb, plan->N, inverse != 0, s))) return st;
  }
  return SMSM_OK;
}

extern "C" smsm_status smsm_plan_device_status(smsm_plan_t plan, void* stream) {
  CHECK_PLAN("smsm_plan_device_status");
  int flag = 0;
  SMSM_CUDA_TRY(cudaMemcpyAsync(&flag, plan->devflag, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
  SMSM_CUDA_TRY(cudaStreamSynchronize(S(stream)));
  if (flag) {
    smsm_set_error("a kernel gave up a bounded wait (device status %d)", flag);
    return (smsm_status)flag;
  }
  return SMSM_OK;
}

// parameters of a solve on `plan`: defaults for NULL, then the range checks
static smsm_status solve_params(smsm_plan_t plan, const smsm_params* params, smsm_params* p, const char* fn) {
  if (params)
    *p = *params;
  else
    smsm_default_params(p);
  if (p->outer_iters < 0 || p->outer_iters > SMSM_MAX_OUTER || p->cg_iters < 0 || p->eta < 1.0 ||
      !(p->lambda >= 0.0) || !(p->eps0_rel > 0.0) || !(p->eps_min_rel > 0.0) ||
      (p->mode != SMSM_MODE_IRLS && p->mode != SMSM_MODE_NULLSPACE) ||
      (p->mode == SMSM_MODE_NULLSPACE && (p->rank <= 0 || p->rank >= plan->C)) || p->lanes < 0 ||
      p->lanes > SMSM_MAX_LANES || !(p->eig_tol >= 0.f && p->eig_tol < 1.f)) {
    smsm_set_error("%s: invalid parameters (K in [0,%d], J >= 0, eta >= 1, lambda >= 0, "
                   "eps0_rel, eps_min_rel > 0, NULLSPACE rank in (0, C), lanes in [0, %d], eig_tol in [0, 1))", fn,
                   SMSM_MAX_OUTER, SMSM_MAX_LANES);
    return SMSM_ERR_ARG;
  }
  return SMSM_OK;
}

extern "C" smsm_status smsm_reconstruct(smsm_plan_t plan, const void* y, void* x, const smsm_params* params,
                                        smsm_report* report, void* stream) {
  CHECK_PLAN("smsm_reconstruct");
  CHECK_PTR("smsm_reconstruct", y);
  CHECK_PTR("smsm_reconstruct", x);
  smsm_status st;
  if ((st = need_sens(plan, "smsm_reconstruct"))) return st;
  smsm_params p;
  if ((st = solve_params(plan, params, &p, "smsm_reconstruct"))) return st;
  return solver_reconstruct(plan, y, x, &p, report, S(stream));
}

extern "C" smsm_status smsm_reconstruct_groups(int n, smsm_plan_t const* plans, const void* const* ys,
                                               void* const* xs, const smsm_params* params, smsm_report* reports,
                                               void* stream) {
  if (n < 1 || !plans || !ys || !xs) {
    smsm_set_error("smsm_reconstruct_groups: n >= 1 and the plans, ys and xs arrays are required");
    return SMSM_ERR_ARG;
  }
  smsm_status st;
  smsm_params p;
  int dev = -1;
  cudaGetDevice(&dev);
  for (int k = 0; k < n; ++k) {
    smsm_plan_t plan = plans[k];
    CHECK_PLAN("smsm_reconstruct_groups");
    if (plan->dev != dev) {
      smsm_set_error("smsm_reconstruct_groups: plan %d was made on device %d, the current device is %d", k,
                     plan->dev, dev);
      return SMSM_ERR_ARG;
    }
    CHECK_PTR("smsm_reconstruct_groups", ys[k]);
    CHECK_PTR("smsm_reconstruct_groups", xs[k]);
    if ((st = need_sens(plan, "smsm_reconstruct_groups"))) return st;
    if ((st = solve_params(plan, params, &p, "smsm_reconstruct_groups"))) return st;
    for (int j = 0; j < k; ++j)
      if (plans[j] == plan) {
        smsm_set_error("smsm_reconstruct_groups: plan %d appears twice (a plan holds one group's buffers)", k);
        return SMSM_ERR_ARG;
      }
  }
  return solver_reconstruct_groups(n, plans, ys, xs, &p, reports, S(stream));
}

extern "C" smsm_status smsm_sense(smsm_plan_t plan, const void* y, const void* phase, void* x, int cg_iters,
                                  smsm_report* report, void* stream) {
  CHECK_PLAN("smsm_sense");
  CHECK_PTR("smsm_sense", y);
  CHECK_PTR("smsm_sense", x);
  if (phase) CHECK_PTR("smsm_sense", phase);
  smsm_status st;
  if ((st = need_sens(plan, "smsm_sense"))) return st;
  if (cg_iters < 0) {
    smsm_set_error("smsm_sense: cg_iters must be >= 0");
    return SMSM_ERR_ARG;
  }
  return solver_sense(plan, y, phase, x, cg_iters, report, S(stream));
}

// x_out = F(cnn(F^-1(x_in))) for the plan's batch; the plan's work vectors hold a and x0
extern "C" smsm_status smsm_learned_start(smsm_plan_t plan, smsm_cnn_t cnn, const void* x_in, void* x_out,
                                          void* stream) {
  CHECK_PLAN("smsm_learned_start");
  CHECK_PTR("smsm_learned_start", x_in);
  CHECK_PTR("smsm_learned_start", x_out);
  int B = 0, H = 0, W = 0, maxn = 0;
  if (!cnn || cnn_shape(cnn, &B, &H, &W, &maxn) || B != plan->L * plan->Ns || H != plan->N || W != plan->N ||
      maxn < plan->D) {
    smsm_set_error("smsm_learned_start: the network must take L*Ns = %d channels of %d x %d images and batches "
                   "of %d", plan->L * plan->Ns, plan->N, plan->N, plan->D);
    return SMSM_ERR_ARG;
  }
  smsm_status st;
  const int count = plan->D * plan->L * plan->Ns;
  if ((st = smsm_fft2c(plan, x_in, plan->bv, count, 1, stream))) return st;
  if ((st = smsm_cnn_forward(cnn, plan->bv, plan->pv, plan->D, stream))) return st;
  return smsm_fft2c(plan, plan->pv, x_out, count, 0, stream);
}

extern "C" smsm_status smsm_autotune(smsm_plan_t plan, const void* y, const smsm_params* params,
                                     smsm_tune_report* report, void* stream) {
  CHECK_PLAN("smsm_autotune");
  CHECK_PTR("smsm_autotune", y);
  smsm_status st;
  if ((st = need_sens(plan, "smsm_autotune"))) return st;
  smsm_params p;
  if ((st = solve_params(plan, params, &p, "smsm_autotune"))) return st;
  return solver_autotune(plan, y, &p, report, S(stream));
}
