// pgvimp_noalloc.cu -- marginal recovery without any device allocation.
//
// Some callers cannot allocate device memory at all: code running while a
// stream is being captured into a CUDA graph (cudaMalloc is not capturable and
// can synchronise the device), runtimes that hand a component a fixed memory
// budget and forbid growth, and hosts that manage every device byte through
// their own pool and reject foreign allocations.  For them this file provides
// one entry point that computes the block marginals of a block-tridiagonal
// precision into caller-provided buffers, with its per-state scratch in a
// file-scope device array instead of allocated memory.
//
// The array is a static module variable: every GPU that loads this library
// holds kNoallocScratchBytes for it until the process exits.  All calls share
// it and it keeps the last call's contents (the sweep writes every scratch
// element before reading it, so nothing needs clearing); two calls that
// overlap on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
#include <cuda.h>   // driver types only; the two driver calls are reached through cudart
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "pgvimp_device.cuh"

namespace pgv {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr size_t kNoallocScratchDoubles = kNoallocScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

// Resolved addresses, one per (device, CUDA context).  A module variable
// lives in a context: after cudaDeviceReset, or under another context made
// current on the same device, the library is loaded again at another address,
// so an address is reused only while the context it was resolved in is the
// current one.  Contexts are told apart by their process-unique id.
struct NoallocEntry {
  int dev;
  unsigned long long ctx_id;
  double* ptr;
};
constexpr int kMaxEntries = 4 * kMaxDevices;
std::mutex g_noalloc_mu;
NoallocEntry g_noalloc_cache[kMaxEntries];
int g_noalloc_used = 0;
int g_noalloc_next = 0;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the context current on the calling thread (cuCtxGetCurrent,
// cuCtxGetId, reached through cudaGetDriverEntryPointByVersion so that the
// library needs no link to the driver library).
pgvimp_status current_ctx_id(unsigned long long* id);

// Per-state scratch: packed C_i^-1 (padded to an even count) and W_i.
template <int n>
__host__ __device__ constexpr size_t noalloc_stride() {
  return (size_t)(n * (n + 1) / 2 + ((n * (n + 1) / 2) & 1)) + (size_t)n * n;
}

// Forward elimination (pivots C_i, W_i = Lambda_{i+1,i} C_i^-1) and backward
// selected inverse Sigma_i = C_i^-1 + W_i^T Sigma_{i+1} W_i,
// Sigma_{i+1,i} = -Sigma_{i+1} W_i, in FP64; log det from the pivots.
template <int n>
__global__ void k_marginals_noalloc(const double* __restrict__ Ld, const double* __restrict__ Lo,
                                    double* __restrict__ Sd, double* __restrict__ So, double* __restrict__ logdet,
                                    double* __restrict__ scratch, int N) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  constexpr int nn = n * n, np = n * (n + 1) / 2;
  constexpr size_t SS = noalloc_stride<n>();
  constexpr int oW = np + (np & 1);
  double S[np];
  for (int e = 0; e < np; ++e) S[e] = 0.0;
  LogDetAcc<double> ld;
  ld.init();
  bool ok = true;
  for (int i = 0; i <= N; ++i) {
    double C[np], Ci[np];
    ld_sym<n, double>(Ld + (size_t)i * nn, C);
    for (int e = 0; e < np; ++e) C[e] -= S[e];
    chol_inverse<n, double>(C, Ci, ld, ok);
    double* sp = scratch + (size_t)i * SS;
    st_packed<n, double>(sp, Ci);
    if (i < N) {
      double E[nn], W[nn];
      ld_blk<n, double>(Lo + (size_t)i * nn, E);
      mul_full_sym<n, double>(E, Ci, W);
      mul_nt_packed<n, double>(W, E, S);
      st_blk<n, double>(sp + oW, W);
    }
  }
  *logdet = ok ? ld.log_value() : NAN;
  if (!ok) return;
  double Sn[np];
  ld_packed<n, double>(scratch + (size_t)N * SS, Sn);
  st_sym<n, double>(Sd + (size_t)N * nn, Sn);
  for (int i = N - 1; i >= 0; --i) {
    const double* sp = scratch + (size_t)i * SS;
    double Ci[np], W[nn], T[nn], Si[np];
    ld_packed<n, double>(sp, Ci);
    ld_blk<n, double>(sp + oW, W);
    mul_sym_full<n, double>(Sn, W, T);
    add_tn_packed<n, double>(Ci, W, T, Si);
    for (int e = 0; e < nn; ++e) T[e] = -T[e];
    st_blk<n, double>(So + (size_t)i * nn, T);
    st_sym<n, double>(Sd + (size_t)i * nn, Si);
    for (int e = 0; e < np; ++e) Sn[e] = Si[e];
  }
}

pgvimp_status noalloc_fail(pgvimp_status st, const std::string& m) {
  set_thread_error(m);   // reported by pgvimp_last_error(NULL)
  return st;
}

pgvimp_status current_ctx_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return noalloc_fail(PGVIMP_ECUDA, "the driver's context queries are not available");
    get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
    get_id = reinterpret_cast<PfnCtxGetId>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return noalloc_fail(PGVIMP_ECUDA, "cuCtxGetCurrent failed");
  if (!ctx) {
    // no context yet on this thread: cudaSetDevice makes the device's primary
    // context current (it allocates nothing)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return noalloc_fail(PGVIMP_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return noalloc_fail(PGVIMP_ECUDA, "no current CUDA context");
  }
  if (get_id(ctx, id) != CUDA_SUCCESS) return noalloc_fail(PGVIMP_ECUDA, "cuCtxGetId failed");
  return PGVIMP_OK;
}

// Device address of the scratch array in the current device's current
// context, resolved once per (device, context) with that device current
// (host code must not use the symbol itself as an address).
pgvimp_status noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(PGVIMP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(PGVIMP_EINVAL, "device index out of range");
  unsigned long long id = 0;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  pgvimp_status st = current_ctx_id(&id);
  if (st != PGVIMP_OK) return st;
  for (int k = 0; k < g_noalloc_used; ++k)
    if (g_noalloc_cache[k].dev == dev && g_noalloc_cache[k].ctx_id == id) {
      *out = g_noalloc_cache[k].ptr;
      return PGVIMP_OK;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return noalloc_fail(PGVIMP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  NoallocEntry& slot = g_noalloc_cache[g_noalloc_used < kMaxEntries ? g_noalloc_used++ : g_noalloc_next];
  if (g_noalloc_used == kMaxEntries) g_noalloc_next = (g_noalloc_next + 1) % kMaxEntries;
  slot.dev = dev;
  slot.ctx_id = id;
  slot.ptr = static_cast<double*>(p);
  *out = slot.ptr;
  return PGVIMP_OK;
}

template <int n>
size_t noalloc_need(int N) {
  return (size_t)(N + 1) * noalloc_stride<n>();
}

}  // namespace
}  // namespace pgv

using namespace pgv;

extern "C" pgvimp_status pgvimp_marginals_noalloc(int n, int N, const double* Ld, const double* Lo, double* Sd,
                                                  double* So, double* logdet, void* stream) {
  if (N < 1) return noalloc_fail(PGVIMP_EINVAL, "N must be >= 1");
  if (!Ld || !Lo || !Sd || !So || !logdet) return noalloc_fail(PGVIMP_EINVAL, "NULL buffer");
  const uintptr_t mis = reinterpret_cast<uintptr_t>(Ld) | reinterpret_cast<uintptr_t>(Lo) |
                        reinterpret_cast<uintptr_t>(Sd) | reinterpret_cast<uintptr_t>(So);
  if (mis & 15) return noalloc_fail(PGVIMP_EINVAL, "block buffers must be 16-byte aligned");
  size_t need;
  switch (n) {
    case 4: need = noalloc_need<4>(N); break;
    case 6: need = noalloc_need<6>(N); break;
    case 14: need = noalloc_need<14>(N); break;
    default: return noalloc_fail(PGVIMP_EINVAL, "state dimension n must be one of 4, 6, 14");
  }
  if (need > kNoallocScratchDoubles)
    return noalloc_fail(PGVIMP_EINVAL, "N too large for the fixed scratch: needs " + std::to_string(need * 8) +
                                           " bytes, the limit is " + std::to_string(kNoallocScratchBytes) + " bytes");
  double* scratch = nullptr;
  pgvimp_status st = noalloc_scratch(&scratch);
  if (st != PGVIMP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (n) {
    case 4: k_marginals_noalloc<4><<<1, 32, 0, s>>>(Ld, Lo, Sd, So, logdet, scratch, N); break;
    case 6: k_marginals_noalloc<6><<<1, 32, 0, s>>>(Ld, Lo, Sd, So, logdet, scratch, N); break;
    case 14: k_marginals_noalloc<14><<<1, 32, 0, s>>>(Ld, Lo, Sd, So, logdet, scratch, N); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(PGVIMP_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return PGVIMP_OK;
}
