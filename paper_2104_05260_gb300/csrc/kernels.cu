// Device kernels of one HSMA evaluation (Sec. 2.2 of the paper), sm_103a.
//
//  prep   wrap/centre in FP64, sphere membership of every image in FP64
//         (|x|^2 < R_s^2 in the order ((x*x + y*y) + z*z), never contracted
//         into FMAs, so the decision is the one the FP64 reference makes),
//         neutrality sums, and a deterministic compaction of the images in B
//         into one list: section 0 holds the identity image of every source
//         in source order, section 1 the other images, source-major.
//  pair   generic direct sum targets x sources -> phi and grad phi.  The near
//         field (Sec. 2.2, first and last steps), the check-point sums
//         (Sec. 2.2, Eq. 6) and the far field of the surface charges all run
//         through it.  FP32 pair arithmetic (rsqrt on the MUFU pipe) with
//         TwoSum-compensated float-float accumulation per target, or an FP64
//         twin.  Sources are staged through shared memory and broadcast to
//         every thread; each CTA walks (target tile, source chunk) items of a
//         static schedule, and every item writes its own FP64 partial, so the
//         result does not depend on which CTA ran it.
//  fit    FP64: combine the check-point partials in fixed order, A = P v,
//         Q = W A (the least-squares solve and the surface map of Sec. 2.2).
//  assemble  Phi_i, F_i = -q_i grad Phi_i, E = 1/2 sum q_i Phi_i (Sec. 3.1),
//         with fixed-order tree reductions (no floating-point atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.hpp"

namespace hsma {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double wrap_centre(double x, double L) {
  // (x - L*floor(x/L)) - L/2, each operation rounded separately
  const double f = floor(__ddiv_rn(x, L));
  return __dsub_rn(__dsub_rn(x, __dmul_rn(L, f)), 0.5 * L);
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  // fixed-order tree over the block's threads (deterministic)
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

template <int NT>
__device__ __forceinline__ int block_excl_scan_i(int v, int* sh, int* total) {
  // Hillis-Steele inclusive scan in shared memory, then shift
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < NT; off <<= 1) {
    const int t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  const int incl = sh[threadIdx.x];
  *total = sh[NT - 1];
  __syncthreads();
  return incl - v;
}

// ------------------------------------------------------------------ prep
// One warp per ion, one lane per image shift: every FP64 sphere test is its
// own short chain (FP64 latency is long on this part), and a warp ballot
// compacts the images of an ion in shift order.
constexpr int kPrepThreads = 256;
constexpr int kIonsPerBlock = kPrepThreads / 32;

int prep_blocks(int N, int n_check) {
  const int a = (N + kIonsPerBlock - 1) / kIonsPerBlock;
  const int b = (n_check + kPrepThreads - 1) / kPrepThreads;
  return a > b ? a : b;
}

// Image of the box-centred source (xc, yc, zc) under shift s, and whether it
// lies inside B: |p|^2 < R_s^2 with every operation rounded separately.
__device__ __forceinline__ bool image_in_B(const PrepArgs& a, int s, double xc, double yc, double zc,
                                           double* px, double* py, double* pz) {
  const double* sh = a.shifts + 5 * s;
  *px = __dadd_rn(xc, sh[0]);
  *py = __dadd_rn(yc, sh[1]);
  *pz = __dadd_rn(__dmul_rn(sh[2], zc), sh[3]);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(*px, *px), __dmul_rn(*py, *py)), __dmul_rn(*pz, *pz));
  return r2 < a.Rs2;
}

// Box-centred FP64 position of ion j for the whole warp: lane d < 3 wraps
// coordinate d (one FP64 division each) and the warp shares the results.
__device__ __forceinline__ void centre_ion(const PrepArgs& a, int j, double* xc, double* yc, double* zc) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  if (lane < 3) {
    const double u = a.x[3 * (size_t)j + lane];
    if (lane < 2 || a.dims == 3) {
      v = wrap_centre(u, a.L[lane]);
    } else {
      if (!(u > 0.0 && u < a.L[2])) atomicOr(&a.sc->flags, FLAG_OUT_OF_SLAB);
      v = __dsub_rn(u, 0.5 * a.L[2]);
    }
  }
  *xc = __shfl_sync(0xffffffffu, v, 0);
  *yc = __shfl_sync(0xffffffffu, v, 1);
  *zc = __shfl_sync(0xffffffffu, v, 2);
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_count(PrepArgs a) {
  __shared__ int sc_cnt[kIonsPerBlock];
  __shared__ double sc_q[kIonsPerBlock], sc_aq[kIonsPerBlock];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kIonsPerBlock + w;
  int c = 0;
  double qj = 0.0;
  if (j < a.N) {
    double xc, yc, zc;
    centre_ion(a, j, &xc, &yc, &zc);
    if (lane == 0) {
      a.xc[3 * (size_t)j] = xc;
      a.xc[3 * (size_t)j + 1] = yc;
      a.xc[3 * (size_t)j + 2] = zc;
    }
    for (int s0 = 1, g = 0; s0 < a.n_shift; s0 += 32, ++g) {
      const int s = s0 + lane;
      double px, py, pz;
      const bool in = s < a.n_shift && image_in_B(a, s, xc, yc, zc, &px, &py, &pz);
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (lane == 0) a.mask[(size_t)j * a.mwords + g] = m;
      c += __popc(m);
    }
    if (lane == 0) a.cnt[j] = c;
    qj = a.q[j];
  }
  if (lane == 0) {
    sc_cnt[w] = c;
    sc_q[w] = qj;
    sc_aq[w] = fabs(qj);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tc = 0;
    double tq = 0.0, taq = 0.0;
    for (int k = 0; k < kIonsPerBlock; ++k) {   // fixed order
      tc += sc_cnt[k];
      tq += sc_q[k];
      taq += sc_aq[k];
    }
    a.blk[blockIdx.x] = tc;
    a.blk_q[blockIdx.x] = tq;
    a.blk_aq[blockIdx.x] = taq;
  }
}

constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_prep_scan(PrepArgs a, int nblk) {
  __shared__ double shd[kScanThreads];
  __shared__ int shi[kScanThreads];
  const int per = (nblk + kScanThreads - 1) / kScanThreads;
  const int b0 = threadIdx.x * per;
  const int b1 = min(nblk, b0 + per);
  int c = 0;
  double q = 0.0, aq = 0.0;
  for (int b = b0; b < b1; ++b) {
    c += a.blk[b];
    q += a.blk_q[b];
    aq += a.blk_aq[b];
  }
  int tot;
  int off = block_excl_scan_i<kScanThreads>(c, shi, &tot);
  const double sq = block_sum_d<kScanThreads>(q, shd);
  const double saq = block_sum_d<kScanThreads>(aq, shd);
  for (int b = b0; b < b1; ++b) {
    const int v = a.blk[b];
    a.blk[b] = off;
    off += v;
  }
  if (threadIdx.x == 0) {
    a.sc->Ns = a.N + tot;
    a.sc->qsum = sq;
    a.sc->qabs = saq;
    a.sc->qcorr = sq / (double)a.N;
    if (fabs(sq) > 1e-10 * saq) atomicOr(&a.sc->flags, FLAG_NOT_NEUTRAL);
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_emit(PrepArgs a) {
  __shared__ int sh_off[kIonsPerBlock];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kIonsPerBlock + w;
  if (threadIdx.x == 0) {
    int o = a.blk[blockIdx.x];
    for (int k = 0; k < kIonsPerBlock; ++k) {   // exclusive prefix over the block's ions
      const int jj = blockIdx.x * kIonsPerBlock + k;
      sh_off[k] = o;
      o += (jj < a.N) ? a.cnt[jj] : 0;
    }
  }
  __syncthreads();
  if (j < a.N) {
    int o = a.N + sh_off[w];
    if (a.ioff && lane == 0) a.ioff[j] = o;
    const double xc = a.xc[3 * (size_t)j], yc = a.xc[3 * (size_t)j + 1], zc = a.xc[3 * (size_t)j + 2];
    const double qj = a.q[j] - a.sc->qcorr;
    if (lane == 0) {
      if (a.src32) {
        a.src32[j] = make_float4((float)xc, (float)yc, (float)zc, (float)qj);
        a.tgt32[j] = make_float4((float)xc, (float)yc, (float)zc, 0.f);
      }
      if (a.src64) {
        a.src64[j] = make_double4_32a(xc, yc, zc, qj);
        a.tgt64[j] = make_double4_32a(xc, yc, zc, 0.0);
      }
    }
    // own-image sums in FP64 (FP32 path): the ion's interaction with its own
    // shifted images, which the FP32 pair kernel skips
    double sp = 0.0, sgx = 0.0, sgy = 0.0, sgz = 0.0;
    for (int s0 = 1, g = 0; s0 < a.n_shift; s0 += 32, ++g) {
      const int s = s0 + lane;
      const unsigned m = a.mask[(size_t)j * a.mwords + g];   // decided in FP64 by k_prep_count
      if ((m >> lane) & 1u) {
        const double* sh = a.shifts + 5 * s;
        const double px = __dadd_rn(xc, sh[0]);
        const double py = __dadd_rn(yc, sh[1]);
        const double pz = __dadd_rn(__dmul_rn(sh[2], zc), sh[3]);
        const int k = o + __popc(m & ((1u << lane) - 1u));
        const double qs = sh[4] * qj;
        if (a.src32) a.src32[k] = make_float4((float)px, (float)py, (float)pz, (float)qs);
        if (a.src64) a.src64[k] = make_double4_32a(px, py, pz, qs);
        if (a.self) {
          const double dx = px - xc, dy = py - yc, dz = pz - zc;
          const double inv = rsqrt(dx * dx + dy * dy + dz * dz);
          const double qi = qs * inv;
          const double q3 = qi * inv * inv;
          sp += qi;
          sgx += q3 * dx;
          sgy += q3 * dy;
          sgz += q3 * dz;
        }
      }
      o += __popc(m);
    }
    if (a.self) {
      for (int off = 16; off > 0; off >>= 1) {   // fixed-order warp sum
        sp += __shfl_xor_sync(0xffffffffu, sp, off);
        sgx += __shfl_xor_sync(0xffffffffu, sgx, off);
        sgy += __shfl_xor_sync(0xffffffffu, sgy, off);
        sgz += __shfl_xor_sync(0xffffffffu, sgz, off);
      }
      if (lane == 0) {
        a.self[j] = sp;
        a.self[(size_t)a.N + j] = sgx;
        a.self[2 * (size_t)a.N + j] = sgy;
        a.self[3 * (size_t)a.N + j] = sgz;
      }
    }
  }
  const int t = blockIdx.x * kPrepThreads + threadIdx.x;
  if (t < a.n_check) {
    const double* cp = a.check_pts + 3 * (size_t)t;
    const double c0 = a.cscale * cp[0], c1 = a.cscale * cp[1], c2 = a.cscale * cp[2];
    if (a.tgt32) a.tgt32[a.N + t] = make_float4((float)c0, (float)c1, (float)c2, 0.f);
    if (a.tgt64) a.tgt64[a.N + t] = make_double4_32a(c0, c1, c2, 0.0);
  }
}

cudaError_t launch_prep(const PrepArgs& a, int nblk, cudaStream_t s) {
  (void)nblk;
  const int nb = (a.N + kIonsPerBlock - 1) / kIonsPerBlock;
  k_prep_count<<<nb, kPrepThreads, 0, s>>>(a);
  k_prep_scan<<<1, kScanThreads, 0, s>>>(a, nb);
  k_prep_emit<<<prep_blocks(a.N, a.n_check), kPrepThreads, 0, s>>>(a);
  return cudaGetLastError();
}

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

int pair_ragged_variant() { return 12; }

cudaError_t launch_pair_ragged(const PairArgs* descs, const int* start, int n_desc, int grid,
                               cudaStream_t s) {
  if (grid < 1) grid = 1;
  k_pair_ragged<<<grid, kPairThreads, 0, s>>>(descs, start, n_desc);
  return cudaGetLastError();
}

int pair_ragged_slots() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair_ragged, kPairThreads, 0);
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
// 24 = packed, 4 targets, compensated sums in shared memory.
int pair_tile_targets(int precision, int tpt) {
  if (precision == 0) return kPairThreads;
  return kPairThreads * (tpt > 20 ? tpt - 20 : tpt > 10 ? tpt - 10 : tpt);
}

static const void* pair_fn(int precision, int tpt) {
  if (precision == 0) return (const void*)k_pair_f64;
  switch (tpt) {
    case 1: return (const void*)k_pair_f32<1>;
    case 2: return (const void*)k_pair_f32<2>;
    case 12: return (const void*)k_pair_f32x2<1>;
    case 14: return (const void*)k_pair_f32x2<2>;
    case 24: return (const void*)k_pair_f32x2s<2>;
    default: return (const void*)k_pair_f32<4>;
  }
}

int pair_slots(int precision, int tpt) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pair_fn(precision, tpt), kPairThreads,
                                                tpt == 24 ? kAccBytes2 : 0);
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
  else k_pair_f32<4><<<grid, kPairThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ fit + map
constexpr int kFitThreads = 256;

__global__ void k_check_combine(const double* part, int n_chunks, int ld, int N, int n_check,
                                int dims, double* v, double* cphi, double* cdz) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_check) return;
  double p = 0.0, d = 0.0;
  for (int ch = 0; ch < n_chunks; ++ch) {
    p += part[((size_t)ch * 4 + 0) * ld + N + c];
    d += part[((size_t)ch * 4 + 3) * ld + N + c];
  }
  v[c] = p;
  if (dims == 2) v[n_check + c] = d;
  cphi[c] = p;
  cdz[c] = d;
}

__global__ void __launch_bounds__(kFitThreads) k_gemv_rows(const double* P, int nv, const double* v, double* A) {
  __shared__ double sh[kFitThreads];
  const double* row = P + (size_t)blockIdx.x * nv;
  double s = 0.0;
  for (int k = threadIdx.x; k < nv; k += kFitThreads) s += row[k] * v[k];
  s = block_sum_d<kFitThreads>(s, sh);
  if (threadIdx.x == 0) A[blockIdx.x] = s;
}

__global__ void k_surface(const double* W, int M, int nA, const double* A, const double* ysurf,
                          double scale, double* Q, float4* s32, double4_32a* s64) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  const double* w = W + (size_t)m * nA;
  for (int r = 0; r < nA; ++r) s += w[r] * A[r];
  s *= scale;   // W and the surface points of a geometry built for a box scaled by 1/scale
  Q[m] = s;
  const double x = scale * ysurf[3 * m], y = scale * ysurf[3 * m + 1], z = scale * ysurf[3 * m + 2];
  if (s32) s32[m] = make_float4((float)x, (float)y, (float)z, (float)s);
  if (s64) s64[m] = make_double4_32a(x, y, z, s);
}

cudaError_t launch_fit(int dims, const double* part, int n_chunks, int ld, int N, int n_check,
                       const double* P, int nA, int nv, const double* W, int M,
                       const double* ysurf, double scale, double* v, double* A, double* cphi,
                       double* cdz, double* Q, float4* s32, double4_32a* s64, cudaStream_t s) {
  k_check_combine<<<(n_check + 255) / 256, 256, 0, s>>>(part, n_chunks, ld, N, n_check, dims, v, cphi, cdz);
  k_gemv_rows<<<nA, kFitThreads, 0, s>>>(P, nv, v, A);
  k_surface<<<(M + 127) / 128, 128, 0, s>>>(W, M, nA, A, ysurf, scale, Q, s32, s64);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ assembly
constexpr int kAsmThreads = 256;

__global__ void __launch_bounds__(kAsmThreads) k_assemble(const double* part, int n_chunks, int ld,
                                                          const double* fpart, int f_chunks, int fld,
                                                          const double* self, const double* q, int N,
                                                          double pref,
                                                          const DevScalars* sc, double* forces,
                                                          double* pot, double* grad, double* blk_e) {
  __shared__ double sh[kAsmThreads];
  const int i = blockIdx.x * kAsmThreads + threadIdx.x;
  double e = 0.0;
  if (i < N) {
    double g[4] = {0, 0, 0, 0};
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int ch = 0; ch < n_chunks; ++ch) s += part[((size_t)ch * 4 + c) * ld + i];
      double f = 0.0;
      for (int ch = 0; ch < f_chunks; ++ch) f += fpart[((size_t)ch * 4 + c) * fld + i];
      if (self) s += self[(size_t)c * N + i];
      g[c] = s + f;
    }
    const double qi = q[i] - sc->qcorr;
    if (forces) {
      forces[3 * (size_t)i] = -pref * qi * g[1];
      forces[3 * (size_t)i + 1] = -pref * qi * g[2];
      forces[3 * (size_t)i + 2] = -pref * qi * g[3];
    }
    if (pot) pot[i] = pref * g[0];
    if (grad) {
      grad[3 * (size_t)i] = g[1];
      grad[3 * (size_t)i + 1] = g[2];
      grad[3 * (size_t)i + 2] = g[3];
    }
    e = qi * g[0];
  }
  e = block_sum_d<kAsmThreads>(e, sh);
  if (threadIdx.x == 0) blk_e[blockIdx.x] = e;
}

__global__ void __launch_bounds__(kScanThreads) k_energy(const double* blk_e, int nblk, double pref, DevScalars* sc) {
  __shared__ double sh[kScanThreads];
  const int per = (nblk + kScanThreads - 1) / kScanThreads;
  const int b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
  double s = 0.0;
  for (int b = b0; b < b1; ++b) s += blk_e[b];
  s = block_sum_d<kScanThreads>(s, sh);
  if (threadIdx.x == 0) sc->energy = 0.5 * pref * s;
}

cudaError_t launch_assemble(const double* part, int n_chunks, int ld, const double* fpart,
                            int f_chunks, int fld, const double* self, const double* q, int N,
                            double pref, DevScalars* sc, double* forces, double* pot, double* grad,
                            double* blk_e, cudaStream_t s) {
  const int nblk = (N + kAsmThreads - 1) / kAsmThreads;
  k_assemble<<<nblk, kAsmThreads, 0, s>>>(part, n_chunks, ld, fpart, f_chunks, fld, self, q, N, pref,
                                          sc, forces, pot, grad, blk_e);
  k_energy<<<1, kScanThreads, 0, s>>>(blk_e, nblk, pref, sc);
  return cudaGetLastError();
}


}  // namespace hsma
