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

template <int TPT>
__global__ void __launch_bounds__(kPairThreads) k_pair_f32(PairArgs a) {
  __shared__ float4 sh[kTile32];
  const float4* __restrict__ tgt = (const float4*)a.tgt;
  const float4* __restrict__ src = (const float4*)a.src;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile32 - 1) / kTile32 * kTile32;
  const int items = a.n_tiles * a.n_chunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
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
  }
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
    const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
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
  const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
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
  const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
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
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads) k_pair_f32x2x(PairArgs a) {
  __shared__ float4 sh[4 * kTile32];
  const int items = a.n_tiles * a.n_chunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) pair_item_f32x2x<NP>(a, item, sh);
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
  const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
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
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads, 3) k_pair_f32x2xs(PairArgs a) {
  __shared__ float4 sh[4 * kTile32];
  extern __shared__ float acc[];   // 8 * 2NP * kPairThreads floats
  const int items = a.n_tiles * a.n_chunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) pair_item_f32x2xs<NP>(a, item, sh, acc);
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads, 3) k_pair_f32x2s(PairArgs a) {
  __shared__ float4 sh[2 * kTile32];
  extern __shared__ float acc[];   // 8 * 2NP * kPairThreads floats
  const int items = a.n_tiles * a.n_chunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) pair_item_f32x2s<NP>(a, item, sh, acc);
}

template <int NP>
__global__ void __launch_bounds__(kPairThreads) k_pair_f32x2(PairArgs a) {
  __shared__ float4 sh[2 * kTile32];
  const int items = a.n_tiles * a.n_chunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) pair_item_f32x2<NP>(a, item, sh);
}

// Ragged launch over several independent pair sums (requests of the serving
// loop): item i belongs to the descriptor d with start[d] <= i < start[d+1].
// Each item writes only its own descriptor's partials, so every request's
// result is the same whatever else shares the launch.
// Ragged launches run the packed kernel with 2 targets per thread (code 12):
// its 512-target tiles give small requests more items than the 4-target
// variants, which keeps served latency down.  Descriptors must be planned
// with that tile size.
__global__ void __launch_bounds__(kPairThreads, 4) k_pair_ragged(const PairArgs* __restrict__ descs,
                                                                const int* __restrict__ start,
                                                                int n_desc) {
  __shared__ float4 sh[2 * kTile32];
  const int total = start[n_desc];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int d = 0;
    while (d + 1 < n_desc && start[d + 1] <= item) ++d;
    const PairArgs a = descs[d];
    pair_item_f32x2<1>(a, item - start[d], sh);
  }
}

// The same ragged launch for precision 2 (exact differences), 512-target tiles.
__global__ void __launch_bounds__(kPairThreads, 4) k_pair_ragged_x(const PairArgs* __restrict__ descs,
                                                                  const int* __restrict__ start,
                                                                  int n_desc) {
  __shared__ float4 sh[4 * kTile32];
  const int total = start[n_desc];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int d = 0;
    while (d + 1 < n_desc && start[d + 1] <= item) ++d;
    const PairArgs a = descs[d];
    pair_item_f32x2x<1>(a, item - start[d], sh);
  }
}

int pair_ragged_variant(int precision) { return precision == 2 ? 32 : 12; }

cudaError_t launch_pair_ragged(int precision, const PairArgs* descs, const int* start, int n_desc, int grid,
                               cudaStream_t s) {
  if (grid < 1) grid = 1;
  if (precision == 2) k_pair_ragged_x<<<grid, kPairThreads, 0, s>>>(descs, start, n_desc);
  else k_pair_ragged<<<grid, kPairThreads, 0, s>>>(descs, start, n_desc);
  return cudaGetLastError();
}

int pair_ragged_slots(int precision) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (precision == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair_ragged_x, kPairThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair_ragged, kPairThreads, 0);
  return sms * (per < 1 ? 1 : per);
}

__global__ void __launch_bounds__(kPairThreads) k_pair_f64(PairArgs a) {
  __shared__ double4_32a sh[kTile64];
  const double4_32a* __restrict__ tgt = (const double4_32a*)a.tgt;
  const double4_32a* __restrict__ src = (const double4_32a*)a.src;
  const int ns = a.sc ? a.sc->Ns : a.n_src;
  int per = (ns + a.n_chunks - 1) / a.n_chunks;
  per = (per + kTile64 - 1) / kTile64 * kTile64;
  const int items = a.n_tiles * a.n_chunks;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
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
  }
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

int pair_slots(int precision, int tpt) {
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
