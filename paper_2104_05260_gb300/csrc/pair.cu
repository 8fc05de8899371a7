// Direct pair sums of one HSMA evaluation (Sec. 2.2 of the paper), sm_103a:
// targets x sources -> phi and grad phi.  The near field (Sec. 2.2, first and
// last steps), the check-point sums (Sec. 2.2, Eq. 6) and the far field of the
// surface charges all run through these kernels.
//
// FP32 pair arithmetic (rsqrt on the MUFU pipe) with TwoSum-compensated
// float-float accumulation per target, or an FP64 twin.  Sources are staged
// through shared memory and broadcast to every thread; each CTA walks
// (target tile, source chunk) items of a static schedule, and every item
// writes its own FP64 partial, so the result does not depend on which CTA
// ran it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "internal.hpp"

namespace hsma {

// ------------------------------------------------------------------ pair sums
#ifndef HSMA_PAIR_UNROLL
#define HSMA_PAIR_UNROLL 8     // images per unrolled step of the FP32 inner loops
#endif
constexpr int kUnroll = HSMA_PAIR_UNROLL;
constexpr int kPairThreads = 256;
constexpr int kTile32 = 256;   // images per shared-memory tile (FP32 path)
constexpr int kAccBytes2 = 8 * 4 * kPairThreads * 4;   // (hi, lo) x 4 components x 4 targets
constexpr int kTile64 = 128;   // images per tile (FP64 path)
constexpr float kFar = 1.0e18f;

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  // Knuth TwoSum: hi + v = s + err exactly; err is carried in lo
  const float s = hi + v;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += err;
}

// Section-1 index range holding the own images of the ions in the target
// tile [t0, t0 + tt) (images are emitted source-major, so it is contiguous).
__device__ __forceinline__ void own_range(const PairArgs& a, int t0, int tt, int* lo, int* hi) {
  *lo = 0;
  *hi = 0;
  if (!a.ioff || t0 >= a.n_diag) return;
  const int tl = min(t0 + tt, a.n_diag) - 1;
  *lo = a.ioff[t0];
  *hi = a.ioff[tl] + a.icnt[tl];
}

// (tile, chunk) of a work item: tile-major with a fused reduction (a tile's
// chunks run close together, so its partials are still in L2 when the last
// one sums them), chunk-major otherwise.
__device__ __forceinline__ void item_tile_chunk(const PairArgs& a, int item, int* tile, int* chunk) {
  if (a.red) {
    *tile = item / a.n_chunks;
    *chunk = item - *tile * a.n_chunks;
  } else {
    *tile = item % a.n_tiles;
    *chunk = item / a.n_tiles;
  }
}

// After a CTA has written its (tile, chunk) partials: count the chunk in, and
// if it was the tile's last, sum the tile's partials over the chunks into
// red.  Per target and component the order is that of k_reduce_chunks: eight
// running sums s_k over the chunks ch = k (mod 8) in increasing order, then
// ((s0 + s4) + (s2 + s6)) + ((s1 + s5) + (s3 + s7)); so the result is bitwise
// the same as the separate reduction, whichever CTA finishes last.  A warp
// takes 4 targets at a time with 8 lanes each (lane = 8 * target + k); the
// final sums use shuffles within each group of 8.  The partials of other
// CTAs are read through L2 (ld.cg).  Called by every thread of the CTA.
__device__ void fused_reduce(const PairArgs& a, int tile, int tile_targets) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket + tile, 1) == a.n_chunks - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int t0 = tile * tile_targets;
  const int t1 = min(a.n_tgt, t0 + tile_targets);
  const size_t ld = (size_t)a.ld;
  const int lane = threadIdx.x & 31, k = lane & 7;
  const int first = 4 * (threadIdx.x >> 5) + (lane >> 3);    // target slot of this lane's group
  const int groups = 4 * (blockDim.x >> 5);
  for (int tb = t0; tb < t1; tb += groups) {
    const int t = tb + first;
    const bool live = t < t1;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    if (live) {
      const double* p = a.part + t;
      int ch = k;
      for (; ch + 24 < a.n_chunks; ch += 32) {   // four chunks per step, loads first
        double v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < 4; ++c) v[u][c] = __ldcg(p + ((size_t)(ch + 8 * u) * 4 + c) * ld);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < 4; ++c) s[c] += v[u][c];
      }
      for (; ch < a.n_chunks; ch += 8)
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] += __ldcg(p + ((size_t)ch * 4 + c) * ld);
    }
    // s_k += s_{k+4}; s_k += s_{k+2}; s_0 += s_1 (as the separate reduction)
#pragma unroll
    for (int w = 4; w > 0; w >>= 1)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double o = __shfl_down_sync(0xffffffffu, s[c], w, 8);
        if (k < w) s[c] += o;
      }
    if (live && k == 0)
#pragma unroll
      for (int c = 0; c < 4; ++c) a.red[(size_t)c * ld + t] = s[c];
  }
  // The tile's partials are dead now: drop their lines from L2 without
  // writing them back (discard.global.L2), so that partials that were summed
  // while still in L2 never reach DRAM.  Only lines wholly inside this tile's
  // target range: the boundary lines are shared with the neighbouring tiles,
  // whose partials may still be pending.
  __syncthreads();   // every thread of the CTA has read its partials
  const int lines = tile_targets / 16;   // 128-byte lines per row of tile_targets doubles
  const int rows = 4 * a.n_chunks;
  for (int idx = threadIdx.x; idx < rows * lines; idx += blockDim.x) {
    const int row = idx / lines, line = idx - row * lines;
    const uintptr_t r0 = (uintptr_t)(a.part + (size_t)row * ld + t0);
    const uintptr_t r1 = (uintptr_t)(a.part + (size_t)row * ld + t1);
    const uintptr_t p = ((r0 + 127) & ~(uintptr_t)127) + 128 * (uintptr_t)line;
    if (p + 128 <= r1) asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
  }
  if (threadIdx.x == 0) a.ticket[tile] = 0;
}

// The item loop of the pair kernels: a static round-robin schedule, or, with
// a.queue, items taken from a counter (the last CTA to find it empty resets
// it).  body(item) must be called by every thread of the CTA.
template <class Body>
__device__ __forceinline__ void for_each_item(const PairArgs& a, Body&& body) {
  const int items = a.n_tiles * a.n_chunks;
  if (!a.queue) {
    for (int item = blockIdx.x; item < items; item += gridDim.x) body(item);
    return;
  }
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= items) break;
    body(item);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.queue + 1, 1) == (int)gridDim.x - 1) {
      a.queue[0] = 0;
      a.queue[1] = 0;
    }
  }
}

template <int TPT>
__device__ __forceinline__ void pair_item_f32(const PairArgs& a, int item, float4* sh) {
  const float4* __restrict__ tgt = (const float4*)a.tgt;
  const float4* __restrict__ src = (const float4*)a.src;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile32 - 1) / kTile32 * kTile32;
  {
    int tile, chunk;
    item_tile_chunk(a, item, &tile, &chunk);
    const int t0 = tile * kPairThreads * TPT;
    float tx[TPT], ty[TPT], tz[TPT];
    float hp[TPT], lp[TPT], hx[TPT], lx[TPT], hy[TPT], ly[TPT], hz[TPT], lz[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int t = t0 + threadIdx.x + k * kPairThreads;
      const float4 v = (t < a.n_tgt) ? tgt[t] : make_float4(kFar, kFar, kFar, 0.f);
      tx[k] = v.x; ty[k] = v.y; tz[k] = v.z;
      hp[k] = lp[k] = hx[k] = lx[k] = hy[k] = ly[k] = hz[k] = lz[k] = 0.f;
    }
    int so[TPT], sc[TPT];   // own section-1 image range of each ion target
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int t = t0 + threadIdx.x + k * kPairThreads;
      const bool ion = a.ioff && t < a.n_diag;
      so[k] = ion ? a.ioff[t] : 0;
      sc[k] = ion ? a.icnt[t] : 0;
    }
    int lo1 = 0, hi1 = 0;
    own_range(a, t0, kPairThreads * TPT, &lo1, &hi1);
    const int s0 = chunk * per;
    const int s1 = min(ns, s0 + per);
    for (int sb = s0; sb < s1; sb += kTile32) {
      const int n = min(kTile32, s1 - sb);
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += kPairThreads) sh[i] = src[sb + i];
      __syncthreads();
      float p[TPT], gx[TPT], gy[TPT], gz[TPT];
#pragma unroll
      for (int k = 0; k < TPT; ++k) p[k] = gx[k] = gy[k] = gz[k] = 0.f;
      const bool diag = ((sb < a.n_diag) && (t0 < a.n_diag) && (sb < t0 + kPairThreads * TPT) && (t0 < sb + n)) ||
                        (sb < hi1 && lo1 < sb + n);
      if (!diag) {
#pragma unroll kUnroll
        for (int i = 0; i < n; ++i) {
          const float4 s = sh[i];
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const float dx = s.x - tx[k], dy = s.y - ty[k], dz = s.z - tz[k];
            float r2 = dx * dx;
            r2 = fmaf(dy, dy, r2);
            r2 = fmaf(dz, dz, r2);
            const float inv = rsqrtf(r2);
            const float qi = s.w * inv;
            p[k] += qi;
            const float q3 = qi * (inv * inv);
            gx[k] = fmaf(q3, dx, gx[k]);
            gy[k] = fmaf(q3, dy, gy[k]);
            gz[k] = fmaf(q3, dz, gz[k]);
          }
        }
      } else {
        for (int i = 0; i < n; ++i) {
          const float4 s = sh[i];
          const int sidx = sb + i;
#pragma unroll
          for (int k = 0; k < TPT; ++k) {
            const int t = t0 + threadIdx.x + k * kPairThreads;
            const float dx = s.x - tx[k], dy = s.y - ty[k], dz = s.z - tz[k];
            float r2 = dx * dx;
            r2 = fmaf(dy, dy, r2);
            r2 = fmaf(dz, dz, r2);
            // an ion (t < n_diag) skips its identity image and, on the FP32
            // path, its own shifted images (added in FP64 by k_prep_emit)
            const bool own = (sidx == t && t < a.n_diag) || (unsigned)(sidx - so[k]) < (unsigned)sc[k];
            const float inv = own ? 0.f : rsqrtf(r2);
            const float qi = s.w * inv;
            p[k] += qi;
            const float q3 = qi * (inv * inv);
            gx[k] = fmaf(q3, dx, gx[k]);
            gy[k] = fmaf(q3, dy, gy[k]);
            gz[k] = fmaf(q3, dz, gz[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < TPT; ++k) {
        two_sum_add(hp[k], lp[k], p[k]);
        two_sum_add(hx[k], lx[k], gx[k]);
        two_sum_add(hy[k], ly[k], gy[k]);
        two_sum_add(hz[k], lz[k], gz[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int t = t0 + threadIdx.x + k * kPairThreads;
      if (t < a.n_tgt) {
        double* o = a.part + (size_t)chunk * 4 * a.ld + t;
        o[0] = (double)hp[k] + (double)lp[k];
        o[(size_t)a.ld] = (double)hx[k] + (double)lx[k];
        o[2 * (size_t)a.ld] = (double)hy[k] + (double)ly[k];
        o[3 * (size_t)a.ld] = (double)hz[k] + (double)lz[k];
      }
    }
    if (a.red) fused_reduce(a, tile, kPairThreads * TPT);
  }
}

template <int TPT>
__global__ void __launch_bounds__(kPairThreads) k_pair_f32(PairArgs a) {
  __shared__ float4 sh[kTile32];
  for_each_item(a, [&](int item) { pair_item_f32<TPT>(a, item, sh); });
}

// Packed FP32x2 variant: the same per-pair arithmetic on two targets at once
// with Blackwell's paired FP32 instructions (FADD2/FMUL2/FFMA2), so one issued
// instruction does the work of two.  Each thread holds 2*NP targets as NP
// pairs; a shared-memory image is stored twice over, (x, x, y, y) and
// (z, z, q, q), so every operand is already a pair.
template <int NP>
__device__ __forceinline__ void pair_item_f32x2(const PairArgs& a, int item, float4* sh) {
  const float4* __restrict__ tgt = (const float4*)a.tgt;
  const float4* __restrict__ src = (const float4*)a.src;
  constexpr int TPT = 2 * NP;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile32 - 1) / kTile32 * kTile32;
  {
    int tile, chunk;
    item_tile_chunk(a, item, &tile, &chunk);
    const int t0 = tile * kPairThreads * TPT;
    // pair k holds targets t0 + tid + (2k)*256 and t0 + tid + (2k+1)*256, negated
    float2 nx[NP], ny[NP], nz[NP];
    float hp[TPT], lp[TPT], hx[TPT], lx[TPT], hy[TPT], ly[TPT], hz[TPT], lz[TPT];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
      const int tb = ta + kPairThreads;
      const float4 va = (ta < a.n_tgt) ? tgt[ta] : make_float4(kFar, kFar, kFar, 0.f);
      const float4 vb = (tb < a.n_tgt) ? tgt[tb] : make_float4(kFar, kFar, kFar, 0.f);
      nx[k] = make_float2(-va.x, -vb.x);
      ny[k] = make_float2(-va.y, -vb.y);
      nz[k] = make_float2(-va.z, -vb.z);
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) hp[k] = lp[k] = hx[k] = lx[k] = hy[k] = ly[k] = hz[k] = lz[k] = 0.f;
    int so[TPT], sc[TPT];   // own section-1 image range of each ion target
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int t = t0 + threadIdx.x + k * kPairThreads;
      const bool ion = a.ioff && t < a.n_diag;
      so[k] = ion ? a.ioff[t] : 0;
      sc[k] = ion ? a.icnt[t] : 0;
    }
    int lo1 = 0, hi1 = 0;
    own_range(a, t0, kPairThreads * TPT, &lo1, &hi1);
    const int s0 = chunk * per;
    const int s1 = min(ns, s0 + per);
    for (int sb = s0; sb < s1; sb += kTile32) {
      const int n = min(kTile32, s1 - sb);
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += kPairThreads) {
        const float4 v = src[sb + i];
        sh[2 * i] = make_float4(v.x, v.x, v.y, v.y);
        sh[2 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
      }
      __syncthreads();
      float2 p[NP], gx[NP], gy[NP], gz[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) p[k] = gx[k] = gy[k] = gz[k] = make_float2(0.f, 0.f);
      const bool diag = ((sb < a.n_diag) && (t0 < a.n_diag) && (sb < t0 + kPairThreads * TPT) && (t0 < sb + n)) ||
                        (sb < hi1 && lo1 < sb + n);
      if (!diag) {
#pragma unroll kUnroll
        for (int i = 0; i < n; ++i) {
          const float4 A = sh[2 * i], B = sh[2 * i + 1];
          const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
          const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            const float2 dx = __fadd2_rn(sx, nx[k]);
            const float2 dy = __fadd2_rn(sy, ny[k]);
            const float2 dz = __fadd2_rn(sz, nz[k]);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            const float2 qi = __fmul2_rn(sq, inv);
            p[k] = __fadd2_rn(p[k], qi);
            const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
            gx[k] = __ffma2_rn(q3, dx, gx[k]);
            gy[k] = __ffma2_rn(q3, dy, gy[k]);
            gz[k] = __ffma2_rn(q3, dz, gz[k]);
          }
        }
      } else {
        for (int i = 0; i < n; ++i) {
          const float4 A = sh[2 * i], B = sh[2 * i + 1];
          const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
          const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
          const int sidx = sb + i;
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
            const int tb = ta + kPairThreads;
            const float2 dx = __fadd2_rn(sx, nx[k]);
            const float2 dy = __fadd2_rn(sy, ny[k]);
            const float2 dz = __fadd2_rn(sz, nz[k]);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            // an ion skips its identity image and its own shifted images
            const bool owna = (sidx == ta && ta < a.n_diag) || (unsigned)(sidx - so[2 * k]) < (unsigned)sc[2 * k];
            const bool ownb = (sidx == tb && tb < a.n_diag) || (unsigned)(sidx - so[2 * k + 1]) < (unsigned)sc[2 * k + 1];
            const float2 inv = make_float2(owna ? 0.f : rsqrtf(r2.x), ownb ? 0.f : rsqrtf(r2.y));
            const float2 qi = __fmul2_rn(sq, inv);
            p[k] = __fadd2_rn(p[k], qi);
            const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
            gx[k] = __ffma2_rn(q3, dx, gx[k]);
            gy[k] = __ffma2_rn(q3, dy, gy[k]);
            gz[k] = __ffma2_rn(q3, dz, gz[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        two_sum_add(hp[2 * k], lp[2 * k], p[k].x);
        two_sum_add(hp[2 * k + 1], lp[2 * k + 1], p[k].y);
        two_sum_add(hx[2 * k], lx[2 * k], gx[k].x);
        two_sum_add(hx[2 * k + 1], lx[2 * k + 1], gx[k].y);
        two_sum_add(hy[2 * k], ly[2 * k], gy[k].x);
        two_sum_add(hy[2 * k + 1], ly[2 * k + 1], gy[k].y);
        two_sum_add(hz[2 * k], lz[2 * k], gz[k].x);
        two_sum_add(hz[2 * k + 1], lz[2 * k + 1], gz[k].y);
      }
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      const int t = t0 + threadIdx.x + k * kPairThreads;
      if (t < a.n_tgt) {
        double* o = a.part + (size_t)chunk * 4 * a.ld + t;
        o[0] = (double)hp[k] + (double)lp[k];
        o[(size_t)a.ld] = (double)hx[k] + (double)lx[k];
        o[2 * (size_t)a.ld] = (double)hy[k] + (double)ly[k];
        o[3 * (size_t)a.ld] = (double)hz[k] + (double)lz[k];
      }
    }
    if (a.red) fused_reduce(a, tile, kPairThreads * TPT);
  }
}

// Low-register variant of the packed kernel: the compensated (hi, lo) sums
// of every target live in shared memory (one column per thread, so the
// accesses are conflict-free) and the own-image ranges are read only in the
// rare guarded tiles, which lets more CTAs share an SM.
// TwoSum of v into the (hi, lo) pair of target slot `slot`, component comp.
__device__ __forceinline__ void smem_two_sum(float* acc, int slot, int comp, float v) {
  float* hp = acc + ((8 * slot + 2 * comp) * kPairThreads + threadIdx.x);
  float hi = hp[0], lo = hp[kPairThreads];
  two_sum_add(hi, lo, v);
  hp[0] = hi;
  hp[kPairThreads] = lo;
}

template <int NP>
__device__ __forceinline__ void pair_item_f32x2s(const PairArgs& a, int item, float4* sh, float* acc) {
  const float4* __restrict__ tgt = (const float4*)a.tgt;
  const float4* __restrict__ src = (const float4*)a.src;
  constexpr int TPT = 2 * NP;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile32 - 1) / kTile32 * kTile32;
  int tile, chunk;
  item_tile_chunk(a, item, &tile, &chunk);
  const int t0 = tile * kPairThreads * TPT;
  float2 nx[NP], ny[NP], nz[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
    const int tb = ta + kPairThreads;
    const float4 va = (ta < a.n_tgt) ? tgt[ta] : make_float4(kFar, kFar, kFar, 0.f);
    const float4 vb = (tb < a.n_tgt) ? tgt[tb] : make_float4(kFar, kFar, kFar, 0.f);
    nx[k] = make_float2(-va.x, -vb.x);
    ny[k] = make_float2(-va.y, -vb.y);
    nz[k] = make_float2(-va.z, -vb.z);
  }
  // acc[(8*k + c) * kPairThreads + tid]: c = 2*component + (0 hi, 1 lo), target slot k
#pragma unroll
  for (int r = 0; r < 8 * TPT; ++r) acc[r * kPairThreads + threadIdx.x] = 0.f;
  int lo1 = 0, hi1 = 0;
  own_range(a, t0, kPairThreads * TPT, &lo1, &hi1);
  const int s0 = chunk * per;
  const int s1 = min(ns, s0 + per);
  for (int sb = s0; sb < s1; sb += kTile32) {
    const int n = min(kTile32, s1 - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kPairThreads) {
      const float4 v = src[sb + i];
      sh[2 * i] = make_float4(v.x, v.x, v.y, v.y);
      sh[2 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
    }
    __syncthreads();
    float2 p[NP], gx[NP], gy[NP], gz[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) p[k] = gx[k] = gy[k] = gz[k] = make_float2(0.f, 0.f);
    const bool diag = ((sb < a.n_diag) && (t0 < a.n_diag) && (sb < t0 + kPairThreads * TPT) && (t0 < sb + n)) ||
                      (sb < hi1 && lo1 < sb + n);
    if (!diag) {
#pragma unroll kUnroll
      for (int i = 0; i < n; ++i) {
        const float4 A = sh[2 * i], B = sh[2 * i + 1];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const float2 dx = __fadd2_rn(sx, nx[k]);
          const float2 dy = __fadd2_rn(sy, ny[k]);
          const float2 dz = __fadd2_rn(sz, nz[k]);
          float2 r2 = __fmul2_rn(dx, dx);
          r2 = __ffma2_rn(dy, dy, r2);
          r2 = __ffma2_rn(dz, dz, r2);
          const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
          const float2 qi = __fmul2_rn(sq, inv);
          p[k] = __fadd2_rn(p[k], qi);
          const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
          gx[k] = __ffma2_rn(q3, dx, gx[k]);
          gy[k] = __ffma2_rn(q3, dy, gy[k]);
          gz[k] = __ffma2_rn(q3, dz, gz[k]);
        }
      }
    } else {
      for (int i = 0; i < n; ++i) {
        const float4 A = sh[2 * i], B = sh[2 * i + 1];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
        const int sidx = sb + i;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
          const int tb = ta + kPairThreads;
          const bool ia = a.ioff && ta < a.n_diag, ib = a.ioff && tb < a.n_diag;
          const int soa = ia ? a.ioff[ta] : 0, sca = ia ? a.icnt[ta] : 0;
          const int sob = ib ? a.ioff[tb] : 0, scb = ib ? a.icnt[tb] : 0;
          const float2 dx = __fadd2_rn(sx, nx[k]);
          const float2 dy = __fadd2_rn(sy, ny[k]);
          const float2 dz = __fadd2_rn(sz, nz[k]);
          float2 r2 = __fmul2_rn(dx, dx);
          r2 = __ffma2_rn(dy, dy, r2);
          r2 = __ffma2_rn(dz, dz, r2);
          // an ion skips its identity image and its own shifted images
          const bool owna = (sidx == ta && ta < a.n_diag) || (unsigned)(sidx - soa) < (unsigned)sca;
          const bool ownb = (sidx == tb && tb < a.n_diag) || (unsigned)(sidx - sob) < (unsigned)scb;
          const float2 inv = make_float2(owna ? 0.f : rsqrtf(r2.x), ownb ? 0.f : rsqrtf(r2.y));
          const float2 qi = __fmul2_rn(sq, inv);
          p[k] = __fadd2_rn(p[k], qi);
          const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
          gx[k] = __ffma2_rn(q3, dx, gx[k]);
          gy[k] = __ffma2_rn(q3, dy, gy[k]);
          gz[k] = __ffma2_rn(q3, dz, gz[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      smem_two_sum(acc, 2 * k, 0, p[k].x);
      smem_two_sum(acc, 2 * k + 1, 0, p[k].y);
      smem_two_sum(acc, 2 * k, 1, gx[k].x);
      smem_two_sum(acc, 2 * k + 1, 1, gx[k].y);
      smem_two_sum(acc, 2 * k, 2, gy[k].x);
      smem_two_sum(acc, 2 * k + 1, 2, gy[k].y);
      smem_two_sum(acc, 2 * k, 3, gz[k].x);
      smem_two_sum(acc, 2 * k + 1, 3, gz[k].y);
    }
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int t = t0 + threadIdx.x + k * kPairThreads;
    if (t < a.n_tgt) {
      double* o = a.part + (size_t)chunk * 4 * a.ld + t;
#pragma unroll
      for (int comp = 0; comp < 4; ++comp) {
        const float* hp = acc + ((8 * k + 2 * comp) * kPairThreads + threadIdx.x);
        o[comp * (size_t)a.ld] = (double)hp[0] + (double)hp[kPairThreads];
      }
    }
  }
  if (a.red) fused_reduce(a, tile, kPairThreads * TPT);
}

// Exact-difference variant (precision 2): each coordinate is carried as an
// FP32 pair hi + lo (lo = x - (float)x, written by the prep in FP64), and the
// difference of a source and a target is (hi_s - hi_t) + (lo_s - lo_t).  For
// close pairs hi_s - hi_t is exact, so the difference has FP32 relative
// accuracy however large the coordinates; the rest of the arithmetic is that
// of k_pair_f32x2.  A null lo array stands for zeros (surface charges).
template <int NP>
__device__ __forceinline__ void pair_item_f32x2x(const PairArgs& a, int item, float4* sh) {
  const float4* __restrict__ tgt = (const float4*)a.tgt;
  const float4* __restrict__ src = (const float4*)a.src;
  constexpr int TPT = 2 * NP;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile32 - 1) / kTile32 * kTile32;
  int tile, chunk;
  item_tile_chunk(a, item, &tile, &chunk);
  const int t0 = tile * kPairThreads * TPT;
  float2 nx[NP], ny[NP], nz[NP], mx[NP], my[NP], mz[NP];   // -hi, -lo of the targets
  float hp[TPT], lp[TPT], hx[TPT], lx[TPT], hy[TPT], ly[TPT], hz[TPT], lz[TPT];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
    const int tb = ta + kPairThreads;
    const float4 va = (ta < a.n_tgt) ? tgt[ta] : make_float4(kFar, kFar, kFar, 0.f);
    const float4 vb = (tb < a.n_tgt) ? tgt[tb] : make_float4(kFar, kFar, kFar, 0.f);
    const float4 la = (a.tgt_lo && ta < a.n_tgt) ? a.tgt_lo[ta] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 lb = (a.tgt_lo && tb < a.n_tgt) ? a.tgt_lo[tb] : make_float4(0.f, 0.f, 0.f, 0.f);
    nx[k] = make_float2(-va.x, -vb.x);
    ny[k] = make_float2(-va.y, -vb.y);
    nz[k] = make_float2(-va.z, -vb.z);
    mx[k] = make_float2(-la.x, -lb.x);
    my[k] = make_float2(-la.y, -lb.y);
    mz[k] = make_float2(-la.z, -lb.z);
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k) hp[k] = lp[k] = hx[k] = lx[k] = hy[k] = ly[k] = hz[k] = lz[k] = 0.f;
  int so[TPT], sc[TPT];   // own section-1 image range of each ion target
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int t = t0 + threadIdx.x + k * kPairThreads;
    const bool ion = a.ioff && t < a.n_diag;
    so[k] = ion ? a.ioff[t] : 0;
    sc[k] = ion ? a.icnt[t] : 0;
  }
  int lo1 = 0, hi1 = 0;
  own_range(a, t0, kPairThreads * TPT, &lo1, &hi1);
  const int s0 = chunk * per;
  const int s1 = min(ns, s0 + per);
  for (int sb = s0; sb < s1; sb += kTile32) {
    const int n = min(kTile32, s1 - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kPairThreads) {
      const float4 v = src[sb + i];
      const float4 l = a.src_lo ? a.src_lo[sb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      sh[4 * i] = make_float4(v.x, v.x, v.y, v.y);
      sh[4 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
      sh[4 * i + 2] = make_float4(l.x, l.x, l.y, l.y);
      sh[4 * i + 3] = make_float4(l.z, l.z, 0.f, 0.f);
    }
    __syncthreads();
    float2 p[NP], gx[NP], gy[NP], gz[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) p[k] = gx[k] = gy[k] = gz[k] = make_float2(0.f, 0.f);
    // tiles that hold no identity or own image of these targets skip the checks
    const bool diag = ((sb < a.n_diag) && (t0 < a.n_diag) && (sb < t0 + kPairThreads * TPT) && (t0 < sb + n)) ||
                      (sb < hi1 && lo1 < sb + n);
    if (!diag) {
#pragma unroll kUnroll
      for (int i = 0; i < n; ++i) {
        const float4 A = sh[4 * i], B = sh[4 * i + 1], Cl = sh[4 * i + 2], Dl = sh[4 * i + 3];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
        const float2 tx = make_float2(Cl.x, Cl.y), ty = make_float2(Cl.z, Cl.w), tz = make_float2(Dl.x, Dl.y);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const float2 dx = __fadd2_rn(__fadd2_rn(sx, nx[k]), __fadd2_rn(tx, mx[k]));
          const float2 dy = __fadd2_rn(__fadd2_rn(sy, ny[k]), __fadd2_rn(ty, my[k]));
          const float2 dz = __fadd2_rn(__fadd2_rn(sz, nz[k]), __fadd2_rn(tz, mz[k]));
          float2 r2 = __fmul2_rn(dx, dx);
          r2 = __ffma2_rn(dy, dy, r2);
          r2 = __ffma2_rn(dz, dz, r2);
          const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
          const float2 qi = __fmul2_rn(sq, inv);
          p[k] = __fadd2_rn(p[k], qi);
          const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
          gx[k] = __ffma2_rn(q3, dx, gx[k]);
          gy[k] = __ffma2_rn(q3, dy, gy[k]);
          gz[k] = __ffma2_rn(q3, dz, gz[k]);
        }
      }
    } else
    for (int i = 0; i < n; ++i) {
      const float4 A = sh[4 * i], B = sh[4 * i + 1], Cl = sh[4 * i + 2], Dl = sh[4 * i + 3];
      const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
      const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
      const float2 tx = make_float2(Cl.x, Cl.y), ty = make_float2(Cl.z, Cl.w), tz = make_float2(Dl.x, Dl.y);
      const int sidx = sb + i;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
        const int tb = ta + kPairThreads;
        const float2 dx = __fadd2_rn(__fadd2_rn(sx, nx[k]), __fadd2_rn(tx, mx[k]));
        const float2 dy = __fadd2_rn(__fadd2_rn(sy, ny[k]), __fadd2_rn(ty, my[k]));
        const float2 dz = __fadd2_rn(__fadd2_rn(sz, nz[k]), __fadd2_rn(tz, mz[k]));
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        // an ion skips its identity image and its own shifted images
        const bool owna = (sidx == ta && ta < a.n_diag) || (unsigned)(sidx - so[2 * k]) < (unsigned)sc[2 * k];
        const bool ownb = (sidx == tb && tb < a.n_diag) || (unsigned)(sidx - so[2 * k + 1]) < (unsigned)sc[2 * k + 1];
        const float2 inv = make_float2(owna ? 0.f : rsqrtf(r2.x), ownb ? 0.f : rsqrtf(r2.y));
        const float2 qi = __fmul2_rn(sq, inv);
        p[k] = __fadd2_rn(p[k], qi);
        const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
        gx[k] = __ffma2_rn(q3, dx, gx[k]);
        gy[k] = __ffma2_rn(q3, dy, gy[k]);
        gz[k] = __ffma2_rn(q3, dz, gz[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      two_sum_add(hp[2 * k], lp[2 * k], p[k].x);
      two_sum_add(hp[2 * k + 1], lp[2 * k + 1], p[k].y);
      two_sum_add(hx[2 * k], lx[2 * k], gx[k].x);
      two_sum_add(hx[2 * k + 1], lx[2 * k + 1], gx[k].y);
      two_sum_add(hy[2 * k], ly[2 * k], gy[k].x);
      two_sum_add(hy[2 * k + 1], ly[2 * k + 1], gy[k].y);
      two_sum_add(hz[2 * k], lz[2 * k], gz[k].x);
      two_sum_add(hz[2 * k + 1], lz[2 * k + 1], gz[k].y);
    }
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int t = t0 + threadIdx.x + k * kPairThreads;
    if (t < a.n_tgt) {
      double* o = a.part + (size_t)chunk * 4 * a.ld + t;
      o[0] = (double)hp[k] + (double)lp[k];
      o[(size_t)a.ld] = (double)hx[k] + (double)lx[k];
      o[2 * (size_t)a.ld] = (double)hy[k] + (double)ly[k];
      o[3 * (size_t)a.ld] = (double)hz[k] + (double)lz[k];
    }
  }
  if (a.red) fused_reduce(a, tile, kPairThreads * TPT);
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads) k_pair_f32x2x(PairArgs a) {
  __shared__ float4 sh[4 * kTile32];
  for_each_item(a, [&](int item) { pair_item_f32x2x<NP>(a, item, sh); });
}

// Exact differences (as in pair_item_f32x2x) with the compensated sums in
// shared memory (as in pair_item_f32x2s), for a lower register count.
template <int NP>
__device__ __forceinline__ void pair_item_f32x2xs(const PairArgs& a, int item, float4* sh, float* acc) {
  const float4* __restrict__ tgt = (const float4*)a.tgt;
  const float4* __restrict__ src = (const float4*)a.src;
  constexpr int TPT = 2 * NP;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile32 - 1) / kTile32 * kTile32;
  int tile, chunk;
  item_tile_chunk(a, item, &tile, &chunk);
  const int t0 = tile * kPairThreads * TPT;
  float2 nx[NP], ny[NP], nz[NP], mx[NP], my[NP], mz[NP];   // -hi, -lo of the targets
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
    const int tb = ta + kPairThreads;
    const float4 va = (ta < a.n_tgt) ? tgt[ta] : make_float4(kFar, kFar, kFar, 0.f);
    const float4 vb = (tb < a.n_tgt) ? tgt[tb] : make_float4(kFar, kFar, kFar, 0.f);
    const float4 la = (a.tgt_lo && ta < a.n_tgt) ? a.tgt_lo[ta] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 lb = (a.tgt_lo && tb < a.n_tgt) ? a.tgt_lo[tb] : make_float4(0.f, 0.f, 0.f, 0.f);
    nx[k] = make_float2(-va.x, -vb.x);
    ny[k] = make_float2(-va.y, -vb.y);
    nz[k] = make_float2(-va.z, -vb.z);
    mx[k] = make_float2(-la.x, -lb.x);
    my[k] = make_float2(-la.y, -lb.y);
    mz[k] = make_float2(-la.z, -lb.z);
  }
  // acc[(8*k + c) * kPairThreads + tid]: c = 2*component + (0 hi, 1 lo), target slot k
#pragma unroll
  for (int r = 0; r < 8 * TPT; ++r) acc[r * kPairThreads + threadIdx.x] = 0.f;
  int lo1 = 0, hi1 = 0;
  own_range(a, t0, kPairThreads * TPT, &lo1, &hi1);
  const int s0 = chunk * per;
  const int s1 = min(ns, s0 + per);
  for (int sb = s0; sb < s1; sb += kTile32) {
    const int n = min(kTile32, s1 - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kPairThreads) {
      const float4 v = src[sb + i];
      const float4 l = a.src_lo ? a.src_lo[sb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      sh[4 * i] = make_float4(v.x, v.x, v.y, v.y);
      sh[4 * i + 1] = make_float4(v.z, v.z, v.w, v.w);
      sh[4 * i + 2] = make_float4(l.x, l.x, l.y, l.y);
      sh[4 * i + 3] = make_float4(l.z, l.z, 0.f, 0.f);
    }
    __syncthreads();
    float2 p[NP], gx[NP], gy[NP], gz[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) p[k] = gx[k] = gy[k] = gz[k] = make_float2(0.f, 0.f);
    const bool diag = ((sb < a.n_diag) && (t0 < a.n_diag) && (sb < t0 + kPairThreads * TPT) && (t0 < sb + n)) ||
                      (sb < hi1 && lo1 < sb + n);
    if (!diag) {
#pragma unroll kUnroll
      for (int i = 0; i < n; ++i) {
        const float4 A = sh[4 * i], B = sh[4 * i + 1], Cl = sh[4 * i + 2], Dl = sh[4 * i + 3];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
        const float2 tx = make_float2(Cl.x, Cl.y), ty = make_float2(Cl.z, Cl.w), tz = make_float2(Dl.x, Dl.y);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const float2 dx = __fadd2_rn(__fadd2_rn(sx, nx[k]), __fadd2_rn(tx, mx[k]));
          const float2 dy = __fadd2_rn(__fadd2_rn(sy, ny[k]), __fadd2_rn(ty, my[k]));
          const float2 dz = __fadd2_rn(__fadd2_rn(sz, nz[k]), __fadd2_rn(tz, mz[k]));
          float2 r2 = __fmul2_rn(dx, dx);
          r2 = __ffma2_rn(dy, dy, r2);
          r2 = __ffma2_rn(dz, dz, r2);
          const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
          const float2 qi = __fmul2_rn(sq, inv);
          p[k] = __fadd2_rn(p[k], qi);
          const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
          gx[k] = __ffma2_rn(q3, dx, gx[k]);
          gy[k] = __ffma2_rn(q3, dy, gy[k]);
          gz[k] = __ffma2_rn(q3, dz, gz[k]);
        }
      }
    } else {
      for (int i = 0; i < n; ++i) {
        const float4 A = sh[4 * i], B = sh[4 * i + 1], Cl = sh[4 * i + 2], Dl = sh[4 * i + 3];
        const float2 sx = make_float2(A.x, A.y), sy = make_float2(A.z, A.w);
        const float2 sz = make_float2(B.x, B.y), sq = make_float2(B.z, B.w);
        const float2 tx = make_float2(Cl.x, Cl.y), ty = make_float2(Cl.z, Cl.w), tz = make_float2(Dl.x, Dl.y);
        const int sidx = sb + i;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const int ta = t0 + threadIdx.x + (2 * k) * kPairThreads;
          const int tb = ta + kPairThreads;
          const bool ia = a.ioff && ta < a.n_diag, ib = a.ioff && tb < a.n_diag;
          const int soa = ia ? a.ioff[ta] : 0, sca = ia ? a.icnt[ta] : 0;
          const int sob = ib ? a.ioff[tb] : 0, scb = ib ? a.icnt[tb] : 0;
          const float2 dx = __fadd2_rn(__fadd2_rn(sx, nx[k]), __fadd2_rn(tx, mx[k]));
          const float2 dy = __fadd2_rn(__fadd2_rn(sy, ny[k]), __fadd2_rn(ty, my[k]));
          const float2 dz = __fadd2_rn(__fadd2_rn(sz, nz[k]), __fadd2_rn(tz, mz[k]));
          float2 r2 = __fmul2_rn(dx, dx);
          r2 = __ffma2_rn(dy, dy, r2);
          r2 = __ffma2_rn(dz, dz, r2);
          // an ion skips its identity image and its own shifted images
          const bool owna = (sidx == ta && ta < a.n_diag) || (unsigned)(sidx - soa) < (unsigned)sca;
          const bool ownb = (sidx == tb && tb < a.n_diag) || (unsigned)(sidx - sob) < (unsigned)scb;
          const float2 inv = make_float2(owna ? 0.f : rsqrtf(r2.x), ownb ? 0.f : rsqrtf(r2.y));
          const float2 qi = __fmul2_rn(sq, inv);
          p[k] = __fadd2_rn(p[k], qi);
          const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
          gx[k] = __ffma2_rn(q3, dx, gx[k]);
          gy[k] = __ffma2_rn(q3, dy, gy[k]);
          gz[k] = __ffma2_rn(q3, dz, gz[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      smem_two_sum(acc, 2 * k, 0, p[k].x);
      smem_two_sum(acc, 2 * k + 1, 0, p[k].y);
      smem_two_sum(acc, 2 * k, 1, gx[k].x);
      smem_two_sum(acc, 2 * k + 1, 1, gx[k].y);
      smem_two_sum(acc, 2 * k, 2, gy[k].x);
      smem_two_sum(acc, 2 * k + 1, 2, gy[k].y);
      smem_two_sum(acc, 2 * k, 3, gz[k].x);
      smem_two_sum(acc, 2 * k + 1, 3, gz[k].y);
    }
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    const int t = t0 + threadIdx.x + k * kPairThreads;
    if (t < a.n_tgt) {
      double* o = a.part + (size_t)chunk * 4 * a.ld + t;
#pragma unroll
      for (int comp = 0; comp < 4; ++comp) {
        const float* hp = acc + ((8 * k + 2 * comp) * kPairThreads + threadIdx.x);
        o[comp * (size_t)a.ld] = (double)hp[0] + (double)hp[kPairThreads];
      }
    }
  }
  if (a.red) fused_reduce(a, tile, kPairThreads * TPT);
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads, 3) k_pair_f32x2xs(PairArgs a) {
  __shared__ float4 sh[4 * kTile32];
  extern __shared__ float acc[];   // 8 * 2NP * kPairThreads floats
  for_each_item(a, [&](int item) { pair_item_f32x2xs<NP>(a, item, sh, acc); });
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads, 3) k_pair_f32x2s(PairArgs a) {
  __shared__ float4 sh[2 * kTile32];
  extern __shared__ float acc[];   // 8 * 2NP * kPairThreads floats
  for_each_item(a, [&](int item) { pair_item_f32x2s<NP>(a, item, sh, acc); });
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads) k_pair_f32x2(PairArgs a) {
  __shared__ float4 sh[2 * kTile32];
  for_each_item(a, [&](int item) { pair_item_f32x2<NP>(a, item, sh); });
}

// Ragged launch over several independent pair sums (requests of the serving
// loop): item i belongs to the descriptor d with start[d] <= i < start[d+1].
// Each item writes only its own descriptor's partials, so every request's
// result is the same whatever else shares the launch.  Items are taken in
// a static round-robin, or from the counter queue[0] when queue is not null
// (queue[1] counts CTAs that found it empty; the last resets both).
// Variants, by the pair-kernel code of the items (descriptors must be planned
// with that code's tile): 12 = packed, 2 targets per thread (512-target
// tiles, more items for small requests); 24 = packed, 4 targets, sums in
// shared memory (1024-target tiles, the single-instance kernel of large N);
// 32 and 44 = the exact-difference versions of the two (precision 2).
template <int V>
__device__ __forceinline__ void ragged_item(const PairArgs& a, int item, float4* sh, float* acc) {
  if (V == 12) pair_item_f32x2<1>(a, item, sh);
  else if (V == 24) pair_item_f32x2s<2>(a, item, sh, acc);
  else if (V == 32) pair_item_f32x2x<1>(a, item, sh);
  else pair_item_f32x2xs<2>(a, item, sh, acc);
}

template <int V>
__global__ void __launch_bounds__(kPairThreads, (V == 12 || V == 32) ? 4 : 3)
    k_pair_ragged(const PairArgs* __restrict__ descs, const int* __restrict__ start, int n_desc,
                  int* __restrict__ queue) {
  __shared__ float4 sh[(V == 12 || V == 24) ? 2 * kTile32 : 4 * kTile32];
  extern __shared__ float acc[];   // V = 24, 44: 8 * 4 * kPairThreads floats
  const int total = start[n_desc];
  __shared__ int s_item;
  int next = blockIdx.x;
  for (;;) {
    int item = next;
    if (queue) {
      __syncthreads();
      if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
      __syncthreads();
      item = s_item;
    }
    if (item >= total) break;
    int d = 0;
    while (d + 1 < n_desc && start[d + 1] <= item) ++d;
    const PairArgs a = descs[d];
    ragged_item<V>(a, item - start[d], sh, acc);
    next += gridDim.x;
  }
  if (queue && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
      queue[0] = 0;
      queue[1] = 0;
    }
  }
}

static bool ragged_code_ok(int precision, int v) {
  return precision == 2 ? (v == 32 || v == 44) : (v == 12 || v == 24);
}

int pair_ragged_variant(int precision) { return precision == 2 ? 32 : 12; }

static const void* ragged_fn(int v) {
  switch (v) {
    case 24: return (const void*)k_pair_ragged<24>;
    case 32: return (const void*)k_pair_ragged<32>;
    case 44: return (const void*)k_pair_ragged<44>;
    default: return (const void*)k_pair_ragged<12>;
  }
}

static size_t ragged_smem(int v) { return (v == 24 || v == 44) ? kAccBytes2 : 0; }

cudaError_t launch_pair_ragged(int precision, int variant, const PairArgs* descs, const int* start, int n_desc,
                               int grid, int* queue, cudaStream_t s) {
  if (grid < 1) grid = 1;
  if (!ragged_code_ok(precision, variant)) return cudaErrorInvalidValue;
  const size_t smem = ragged_smem(variant);
  if (smem) cudaFuncSetAttribute(ragged_fn(variant), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  switch (variant) {
    case 24: k_pair_ragged<24><<<grid, kPairThreads, smem, s>>>(descs, start, n_desc, queue); break;
    case 32: k_pair_ragged<32><<<grid, kPairThreads, smem, s>>>(descs, start, n_desc, queue); break;
    case 44: k_pair_ragged<44><<<grid, kPairThreads, smem, s>>>(descs, start, n_desc, queue); break;
    default: k_pair_ragged<12><<<grid, kPairThreads, smem, s>>>(descs, start, n_desc, queue); break;
  }
  return cudaGetLastError();
}

int pair_ragged_slots(int precision, int variant) {
  if (!ragged_code_ok(precision, variant)) variant = pair_ragged_variant(precision);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ragged_smem(variant);
  if (smem) cudaFuncSetAttribute(ragged_fn(variant), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ragged_fn(variant), kPairThreads, smem);
  return sms * (per < 1 ? 1 : per);
}

bool pair_ragged_code_ok(int precision, int variant) { return ragged_code_ok(precision, variant); }

__device__ __forceinline__ void pair_item_f64(const PairArgs& a, int item, double4_32a* sh) {
  const double4_32a* __restrict__ tgt = (const double4_32a*)a.tgt;
  const double4_32a* __restrict__ src = (const double4_32a*)a.src;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile64 - 1) / kTile64 * kTile64;
  int tile, chunk;
  item_tile_chunk(a, item, &tile, &chunk);
  const int t = tile * kPairThreads + threadIdx.x;
  const double4_32a tv = (t < a.n_tgt) ? tgt[t] : make_double4_32a(1e18, 1e18, 1e18, 0.0);
  double p = 0, gx = 0, gy = 0, gz = 0;
  const int s0 = chunk * per;
  const int s1 = min(ns, s0 + per);
  const int t0 = tile * kPairThreads;
  for (int sb = s0; sb < s1; sb += kTile64) {
    const int n = min(kTile64, s1 - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kPairThreads) sh[i] = src[sb + i];
    __syncthreads();
    const bool diag = (sb < a.n_diag) && (t0 < a.n_diag) && (sb < t0 + kPairThreads) && (t0 < sb + n);
    for (int i = 0; i < n; ++i) {
      const double4_32a s = sh[i];
      const double dx = s.x - tv.x, dy = s.y - tv.y, dz = s.z - tv.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      double inv = rsqrt(r2);
      if (diag && sb + i == t && t < a.n_diag) inv = 0.0;
      const double qi = s.w * inv;
      p += qi;
      const double q3 = qi * inv * inv;
      gx += q3 * dx;
      gy += q3 * dy;
      gz += q3 * dz;
    }
  }
  if (t < a.n_tgt) {
    double* o = a.part + (size_t)chunk * 4 * a.ld + t;
    o[0] = p;
    o[(size_t)a.ld] = gx;
    o[2 * (size_t)a.ld] = gy;
    o[3 * (size_t)a.ld] = gz;
  }
  if (a.red) fused_reduce(a, tile, kPairThreads);
}

__global__ void __launch_bounds__(kPairThreads) k_pair_f64(PairArgs a) {
  __shared__ double4_32a sh[kTile64];
  for_each_item(a, [&](int item) { pair_item_f64(a, item, sh); });
}

// Kernel variants of the FP32 path, by code: 1, 2, 4 = scalar FP32 with that
// many targets per thread; 12, 14 = packed FP32x2 with 2 or 4 targets;
// 24 = packed, 4 targets, compensated sums in shared memory; 32, 34 = packed
// exact differences with 2 or 4 targets; 44 = exact differences, 4 targets,
// compensated sums in shared memory.
int pair_tile_targets(int precision, int tpt) {
  if (precision == 0) return kPairThreads;
  return kPairThreads * (tpt > 40 ? tpt - 40 : tpt > 30 ? tpt - 30 : tpt > 20 ? tpt - 20 : tpt > 10 ? tpt - 10 : tpt);
}

static const void* pair_fn(int precision, int tpt) {
  if (precision == 0) return (const void*)k_pair_f64;
  switch (tpt) {
    case 1: return (const void*)k_pair_f32<1>;
    case 2: return (const void*)k_pair_f32<2>;
    case 12: return (const void*)k_pair_f32x2<1>;
    case 14: return (const void*)k_pair_f32x2<2>;
    case 24: return (const void*)k_pair_f32x2s<2>;
    case 32: return (const void*)k_pair_f32x2x<1>;
    case 34: return (const void*)k_pair_f32x2x<2>;
    case 44: return (const void*)k_pair_f32x2xs<2>;
    default: return (const void*)k_pair_f32<4>;
  }
}

// The variants with compensated sums in dynamic shared memory use 48 KB or
// more in all (static + dynamic): allow it, once per device.
static void allow_pair_smem() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  const unsigned long long bit = 1ull << dev;
  if (done.load() & bit) return;
  cudaFuncSetAttribute((const void*)k_pair_f32x2s<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAccBytes2);
  cudaFuncSetAttribute((const void*)k_pair_f32x2xs<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAccBytes2);
  cudaGetLastError();
  done.fetch_or(bit);
}

int pair_slots(int precision, int tpt) {
  allow_pair_smem();
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pair_fn(precision, tpt), kPairThreads,
                                                (tpt == 24 || tpt == 44) ? kAccBytes2 : 0);
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t launch_pair(int precision, int tpt, PairArgs a, int grid, cudaStream_t s) {
  if (grid < 1) grid = 1;
  allow_pair_smem();
  if (precision == 0) k_pair_f64<<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 1) k_pair_f32<1><<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 2) k_pair_f32<2><<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 12) k_pair_f32x2<1><<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 14) k_pair_f32x2<2><<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 24) k_pair_f32x2s<2><<<grid, kPairThreads, kAccBytes2, s>>>(a);
  else if (tpt == 32) k_pair_f32x2x<1><<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 34) k_pair_f32x2x<2><<<grid, kPairThreads, 0, s>>>(a);
  else if (tpt == 44) k_pair_f32x2xs<2><<<grid, kPairThreads, kAccBytes2, s>>>(a);
  else k_pair_f32<4><<<grid, kPairThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hsma
