// hsma_pair_sum_static: the direct pair sum (the near-field / check-point /
// far-field kernel of the evaluation) for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs while CUDA stream capture is active in global
// mode (cudaMalloc is not allowed then), engines that hand out all device
// memory from their own pool and forbid raw cudaMalloc/cudaFree, and
// real-time loops that must not pay for an allocation.  Such a caller passes
// its inputs and outputs as device pointers; the kernel's scratch (the
// converted targets and sources and the per-chunk partial sums) lives in one
// file-scope __device__ array of fixed size instead of memory from
// cudaMalloc.
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
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  Host code may
// not use g_static_scratch itself: on the host that name is only a stand-in.
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
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

__global__ void k_combine(const double* __restrict__ part, int n_chunks, int n_tgt, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tgt) return;
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int ch = 0; ch < n_chunks; ++ch) s += part[((size_t)ch * 4 + c) * n_tgt + t];
    out[4 * (size_t)t + c] = s;
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
    k_combine<<<(int)((n_tgt + 255) / 256), 256, 0, s>>>(part, chunks, (int)n_tgt, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HSMA_ERR_CUDA;
  }
  return HSMA_OK;
}
