// hsma_pair_sum_static: the direct pair sum (the near-field / check-point /
// far-field kernel of the evaluation) for callers that cannot allocate
// device memory.
//
// Who needs it: engines that hand out all device memory from their own pool
// and forbid raw cudaMalloc/cudaFree (an allocation behind the pool's back
// breaks its accounting), plug-ins that run inside such an engine, and
// real-time loops that must not pay for an allocation or the synchronisation
// that cudaFree implies.  Such a caller passes its inputs and outputs as
// device pointers; the kernel's scratch (the converted targets and sources
// and the per-chunk partial sums) lives in one file-scope __device__ array of
// fixed size instead of memory from cudaMalloc.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/hsma.h"
#include "api_internal.hpp"
#include "internal.hpp"

namespace hsma {

// 64 MiB per GPU that loads the library, held until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  void* ptr = nullptr;
  unsigned long long ctx_id = 0;   // context the address belongs to
};
ScratchAddr g_scratch[kMaxDevices];

// Unique id of the current CUDA context (0 if the driver cannot tell).  A
// device reset or a new primary context loads the module again, possibly at
// another address, so the cached address is keyed by the context's id.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetIdFn)f;
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array for the current device and context,
// looked up with cudaGetSymbolAddress the first time (per device, and again
// after the device's context has been replaced).  Host code may not use
// g_static_scratch itself: on the host that name is only a stand-in.
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchAddr& c = g_scratch[dev];
  if (!c.ptr || c.ctx_id != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    c.ptr = p;
    c.ctx_id = ctx;
  }
  *out = c.ptr;
  return cudaSuccess;
}

// True when p is device memory of the current device (or managed memory).
bool on_current_device(const void* p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

__global__ void k_convert(const double* __restrict__ tgt, int n_tgt, const double* __restrict__ src,
                          int n_src, int precision, float4* t32, float4* s32, double4_32a* t64,
                          double4_32a* s64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_tgt) {
    const double x = tgt[3 * (size_t)i], y = tgt[3 * (size_t)i + 1], z = tgt[3 * (size_t)i + 2];
    if (precision) t32[i] = make_float4((float)x, (float)y, (float)z, 0.f);
    else t64[i] = make_double4_32a(x, y, z, 0.0);
  }
  if (i < n_src) {
    const double* s = src + 4 * (size_t)i;
    if (precision) s32[i] = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[3]);
    else s64[i] = make_double4_32a(s[0], s[1], s[2], s[3]);
  }
}

// out[4 t + c] = sum over chunks of part[(chunk * 4 + c) * n_tgt + t].  A block
// takes 32 targets; its 8 warps sum every 8th chunk (lanes over targets, so
// the reads are coalesced), then warp 0 adds the 8 partial sums in warp
// order.  The order is fixed, so the result does not depend on the launch.
constexpr int kCombineWarps = 8;
__global__ void __launch_bounds__(32 * kCombineWarps) k_combine(const double* __restrict__ part, int n_chunks,
                                                                int n_tgt, double* __restrict__ out) {
  __shared__ double sh[kCombineWarps][4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (t < n_tgt) {
    for (int ch = w; ch < n_chunks; ch += kCombineWarps) {
#pragma unroll
      for (int c = 0; c < 4; ++c) s[c] += part[((size_t)ch * 4 + c) * n_tgt + t];
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) sh[w][c][lane] = s[c];
  __syncthreads();
  if (w == 0 && t < n_tgt) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < kCombineWarps; ++k) v += sh[k][c][lane];
      out[4 * (size_t)t + c] = v;
    }
  }
}

}  // namespace
}  // namespace hsma

using namespace hsma;

extern "C" int hsma_pair_sum_static(const double* targets, int64_t n_tgt, const double* sources,
                                    int64_t n_src, double* out, int precision, void* stream) {
  if (!targets || !sources || !out || n_tgt < 1 || n_src < 1 || (precision != 0 && precision != 1))
    return HSMA_ERR_ARG;
  // Size check first, with one chunk (the smallest footprint), before any CUDA call.
  const size_t item = precision ? 16 : 32;
  const size_t fixed = round256((size_t)n_tgt * item) + round256((size_t)n_src * item);
  const size_t per_chunk = round256((size_t)4 * n_tgt * 8);
  if (n_tgt > (1 << 30) || n_src > (1 << 30) || fixed + per_chunk > kStaticScratchBytes)
    return HSMA_ERR_ARG;   // beyond the 64 MiB static scratch
  if (!on_current_device(targets) || !on_current_device(sources) || !on_current_device(out))
    return HSMA_ERR_ARG;   // host memory or another GPU's memory: not reachable as scratch-free device input
  void* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HSMA_ERR_CUDA;
  }
  const int tpt = 12;  // packed FP32x2 pair kernel
  const int tile = pair_tile_targets(precision, tpt);
  const int slots = pair_slots(precision, tpt);
  const int tiles = (int)((n_tgt + tile - 1) / tile);
  int chunks = choose_chunks(tiles, slots, (double)n_src, precision ? 256 : 128);
  const int max_chunks = (int)((kStaticScratchBytes - fixed) / per_chunk);
  if (chunks > max_chunks) chunks = max_chunks;
  unsigned char* p = (unsigned char*)base;
  void* tgt = p;
  void* src = p + round256((size_t)n_tgt * item);
  double* part = (double*)(p + fixed);
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)(n_tgt > n_src ? n_tgt : n_src);
  k_convert<<<(n + 255) / 256, 256, 0, s>>>(targets, (int)n_tgt, sources, (int)n_src, precision,
                                            (float4*)tgt, (float4*)src, (double4_32a*)tgt,
                                            (double4_32a*)src);
  PairArgs a;
  a.tgt = tgt;
  a.n_tgt = (int)n_tgt;
  a.src = src;
  a.n_src = (int)n_src;
  a.sc = nullptr;
  a.n_diag = 0;
  a.n_tiles = tiles;
  a.n_chunks = chunks;
  a.part = part;
  a.ld = (int)n_tgt;
  const long items = (long)tiles * chunks;
  e = launch_pair(precision, tpt, a, (int)(items < slots ? items : slots), s);
  if (e == cudaSuccess) {
    k_combine<<<(int)((n_tgt + 31) / 32), 32 * kCombineWarps, 0, s>>>(part, chunks, (int)n_tgt, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HSMA_ERR_CUDA;
  }
  return HSMA_OK;
}
