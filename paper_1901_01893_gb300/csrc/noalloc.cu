// smsm_hankel_gram_noalloc: the Hankel Gram without any device allocation.
//
// Who needs this: callers that must not allocate GPU memory at all -- for
// example code running inside a host framework that owns every device
// allocation through its own pool (so a stray cudaMalloc would fragment or
// overrun it), or a real-time path that may not block on the allocator.
// smsm_plan() allocates its workspace with cudaMalloc, so those callers
// cannot create a plan.  This entry point needs no plan: the caller passes
// the input and the output, and the only scratch (the per-chunk partial
// sums of the Gram) lives in one fixed-size array that is part of the
// library image itself.
//
// Costs and limits:
//  * Every GPU that loads the library's device code holds
//    SMSM_NOALLOC_SCRATCH_BYTES (8 MiB) for this array until the process
//    exits.  With lazy module loading (the CUDA default) the device code,
//    and with it the array, is loaded on the first call of this entry point
//    or the first launch of any kernel of the library on that device.
//  * C = shots*filter^2 is at most 320.
//  * A geometry whose partial sums need more than that is rejected with
//    SMSM_ERR_ARG (the requirement is ceil((N-filter+1)/16) * C^2 * 16 bytes
//    per slice, C = shots*filter^2; slices are processed one after another).
//  * Every call on a device shares the one array.  Calls that overlap on the
//    GPU (different streams, or different host threads) race on it and give
//    wrong results; serialise them.  The kernels overwrite every scratch
//    entry before reading it, so nothing needs clearing between calls and
//    the array may hold any earlier call's contents.
//  * Every call looks the array's device address up (cudaGetSymbolAddress,
//    with the caller's device current), so the address stays right after a
//    context is torn down and created again (cudaDeviceReset), when the
//    module may load at another address.  The first call on a device can
//    load the library's device code; make it once at set-up, before any
//    stream capture begins on that device.
#include "common.cuh"

#define SMSM_NOALLOC_SCRATCH_BYTES (8u << 20)

// The scratch array.  In host code this name is only a host-side stand-in,
// never a device address: host code must use the pointer obtained below.
static __device__ __align__(256) double2 g_gram_scratch[SMSM_NOALLOC_SCRATCH_BYTES / sizeof(double2)];

// Gram kernels (hankel.cu)
__global__ void k_gram_part(const float2* __restrict__ x, double2* __restrict__ part, int Ns, int N, int r, int C,
                            int P1, int nkx, int tside, int periodic);
__global__ void k_gram_reduce(const double2* __restrict__ part, double2* __restrict__ G, int L, int C, int nkx);

// Device address of the scratch array in the current context.  Looked up on every call
// (a host-side table lookup in the runtime): no cached pointer can outlive a context.
static smsm_status scratch_for_current_device(double2** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
  if (e != cudaSuccess || !p) {
    int dev = -1;
    cudaGetDevice(&dev);
    smsm_set_error("smsm_hankel_gram_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                   cudaGetErrorString(e));
    return SMSM_ERR_CUDA;
  }
  *out = (double2*)p;
  return SMSM_OK;
}

extern "C" smsm_status smsm_hankel_gram_noalloc(const void* x, void* G, int mb, int shots, int n, int filter,
                                                void* stream) {
  if (!x || !G || ((uintptr_t)x & 15u) || ((uintptr_t)G & 15u)) {
    smsm_set_error("smsm_hankel_gram_noalloc: x and G must be non-NULL, 16-byte aligned device pointers");
    return SMSM_ERR_ARG;
  }
  const int N = n, r = filter;
  if (mb < 1 || shots < 1 || shots > 8 || N < 16 || N > SMSM_MAX_N || r < 1 || r > 12 || 2 * r > N) {
    smsm_set_error("smsm_hankel_gram_noalloc: need mb >= 1, 1 <= shots <= 8, 16 <= n <= %d, "
                   "1 <= filter <= min(12, n/2) (got mb=%d shots=%d n=%d filter=%d)",
                   SMSM_MAX_N, mb, shots, n, filter);
    return SMSM_ERR_ARG;
  }
  const int C = shots * r * r;
  const int P1 = N - r + 1;
  const int nkx = (P1 + 15) / 16;
  const size_t need = (size_t)nkx * C * C * sizeof(double2);
  if (C > SMSM_MAX_C) {
    smsm_set_error("smsm_hankel_gram_noalloc: C = shots*filter^2 = %d is above %d", C, SMSM_MAX_C);
    return SMSM_ERR_ARG;
  }
  if (need > SMSM_NOALLOC_SCRATCH_BYTES) {
    smsm_set_error("smsm_hankel_gram_noalloc: this geometry needs %zu bytes of scratch, above the fixed "
                   "%u bytes (C = shots*filter^2 = %d)", need, SMSM_NOALLOC_SCRATCH_BYTES, C);
    return SMSM_ERR_ARG;
  }
  double2* scratch = nullptr;
  smsm_status st = scratch_for_current_device(&scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int GT = 48, GCH = 16;
  const int tside = (C + GT - 1) / GT;
  const int ntile = tside * (tside + 1) / 2;
  const int TW = GCH + r - 1;
  const size_t sm = (size_t)shots * TW * TW * sizeof(float2);
  const size_t NN = (size_t)N * N;
  for (int l = 0; l < mb; ++l) {
    const float2* xl = (const float2*)x + (size_t)l * shots * NN;
    double2* Gl = (double2*)G + (size_t)l * C * C;
    k_gram_part<<<dim3(nkx, ntile, 1), 256, sm, s>>>(xl, scratch, shots, N, r, C, P1, nkx, tside, 0);
    SMSM_LAUNCH_CHECK("k_gram_part (no-alloc)");
    k_gram_reduce<<<128, 256, 0, s>>>(scratch, Gl, 1, C, nkx);
    SMSM_LAUNCH_CHECK("k_gram_reduce (no-alloc)");
  }
  return SMSM_OK;
}
