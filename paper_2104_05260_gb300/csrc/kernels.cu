// Device kernels of one HSMA evaluation (Sec. 2.2 of the paper), sm_103a.
//
//  prep   wrap/centre in FP64, sphere membership of every image in FP64
//         (|x|^2 < R_s^2 in the order ((x*x + y*y) + z*z), never contracted
//         into FMAs, so the decision is the one the FP64 reference makes),
//         neutrality sums, and a deterministic compaction of the images in B
//         into one list: section 0 holds the identity image of every source
//         in source order, section 1 the other images, source-major.
//  pair   the direct pair sums live in pair.cu.
//  fit    FP64: combine the check-point partials in fixed order, A = P v,
//         Q = W A (the least-squares solve and the surface map of Sec. 2.2).
//  series the far field as the fitted series itself (optional; Eq. 5).
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

// Box-centred FP64 coordinate d of ion j (one thread per coordinate, so a
// block's wraps share a few warp instructions of the narrow FP64 pipe).
__device__ __forceinline__ double centre_coord(const PrepArgs& a, int j, int d) {
  const double u = a.x[3 * (size_t)j + d];
  if (d < 2 || a.dims == 3) return wrap_centre(u, a.L[d]);
  if (!(u > 0.0 && u < a.L[2])) atomicOr(&a.sc->flags, FLAG_OUT_OF_SLAB);
  return __dsub_rn(u, 0.5 * a.L[2]);
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_count(PrepArgs a) {
  __shared__ int sc_cnt[kIonsPerBlock];
  __shared__ double sc_q[kIonsPerBlock], sc_aq[kIonsPerBlock];
  __shared__ double sh_xc[3 * kIonsPerBlock];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kIonsPerBlock + w;
  if (threadIdx.x < 3 * kIonsPerBlock) {
    const int jj = blockIdx.x * kIonsPerBlock + threadIdx.x / 3;
    if (jj < a.N) sh_xc[threadIdx.x] = centre_coord(a, jj, threadIdx.x % 3);
  }
  __syncthreads();
  int c = 0;
  double qj = 0.0;
  if (j < a.N) {
    const double xc = sh_xc[3 * w], yc = sh_xc[3 * w + 1], zc = sh_xc[3 * w + 2];
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

// Own-image terms of the shifts that do not reflect (zs = 1): the image
// lies exactly (sx, sy, zo) from its ion, so 1/|d| and d/|d|^3 depend on the
// shift alone and are formed once per block (FP64).
constexpr int kSelfTable = 256;

// One thread per ion: its identity entry, then its images in B in shift
// order (the mask bits k_prep_count set in FP64), then its own-image sums in
// FP64, added serially in shift order.  A thread per ion rather than a lane
// per shift: only about a fifth of the shifts put an image in B, and GB300's
// FP64 pipe charges a warp instruction a full pass whatever its active lanes.
// Thread t also writes check point t.
// One warp per block: the FP64 pipe is the limit, so small N still spreads
// over many SMs.
constexpr int kEmitThreads = 32;

__global__ void __launch_bounds__(kEmitThreads) k_prep_emit(PrepArgs a) {
  __shared__ double sh_self[4][kSelfTable];
  if (a.self)
    for (int t = threadIdx.x + 1; t < min(a.n_shift, kSelfTable); t += kEmitThreads) {
      const double* sh = a.shifts + 5 * t;
      if (sh[2] == 1.0) {
        const double dx = sh[0], dy = sh[1], dz = sh[3];
        const double inv = rsqrt(dx * dx + dy * dy + dz * dz);
        const double inv3 = inv * inv * inv;
        sh_self[0][t] = inv;
        sh_self[1][t] = inv3 * dx;
        sh_self[2][t] = inv3 * dy;
        sh_self[3][t] = inv3 * dz;
      }
    }
  __syncthreads();
  const int j = blockIdx.x * kEmitThreads + threadIdx.x;
  if (j < a.N) {
    // blk holds the exclusive image offset of each group of kIonsPerBlock ions
    int o = a.N + a.blk[j / kIonsPerBlock];
    for (int i = j - j % kIonsPerBlock; i < j; ++i) o += a.cnt[i];
    if (a.ioff) a.ioff[j] = o;
    const double xc = a.xc[3 * (size_t)j], yc = a.xc[3 * (size_t)j + 1], zc = a.xc[3 * (size_t)j + 2];
    const double qj = a.q[j] - a.sc->qcorr;
    if (a.src32) {
      a.src32[j] = make_float4((float)xc, (float)yc, (float)zc, (float)qj);
      a.tgt32[j] = make_float4((float)xc, (float)yc, (float)zc, 0.f);
    }
    if (a.src32lo) {
      const float4 lo = make_float4((float)(xc - (double)(float)xc), (float)(yc - (double)(float)yc),
                                    (float)(zc - (double)(float)zc), 0.f);
      a.src32lo[j] = lo;
      a.tgt32lo[j] = lo;
    }
    if (a.src64) {
      a.src64[j] = make_double4_32a(xc, yc, zc, qj);
      a.tgt64[j] = make_double4_32a(xc, yc, zc, 0.0);
    }
    // own-image sums in FP64 (FP32 path): the ion's interaction with its own
    // shifted images, which the FP32 pair kernel skips
    double sp = 0.0, sgx = 0.0, sgy = 0.0, sgz = 0.0;
    for (int g = 0; g < a.mwords; ++g) {
      unsigned m = a.mask[(size_t)j * a.mwords + g];   // decided in FP64 by k_prep_count
      while (m) {
        const int s = 32 * g + __ffs(m);   // bit b stands for shift b + 1
        m &= m - 1u;
        const double* sh = a.shifts + 5 * s;
        const double px = __dadd_rn(xc, sh[0]);
        const double py = __dadd_rn(yc, sh[1]);
        const double pz = __dadd_rn(__dmul_rn(sh[2], zc), sh[3]);
        const int k = o++;
        if (a.img_shift) a.img_shift[k - a.N] = s;
        const double qs = sh[4] * qj;
        if (a.src32) a.src32[k] = make_float4((float)px, (float)py, (float)pz, (float)qs);
        if (a.src32lo)
          a.src32lo[k] = make_float4((float)(px - (double)(float)px), (float)(py - (double)(float)py),
                                     (float)(pz - (double)(float)pz), 0.f);
        if (a.src64) a.src64[k] = make_double4_32a(px, py, pz, qs);
        if (a.self) {
          if (sh[2] == 1.0 && s < kSelfTable) {
            sp += qs * sh_self[0][s];
            sgx += qs * sh_self[1][s];
            sgy += qs * sh_self[2][s];
            sgz += qs * sh_self[3][s];
          } else {
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
      }
    }
    if (a.self) {
      a.self[j] = sp;
      a.self[(size_t)a.N + j] = sgx;
      a.self[2 * (size_t)a.N + j] = sgy;
      a.self[3 * (size_t)a.N + j] = sgz;
    }
  }
  if (j < a.n_check) {
    const double* cp = a.check_pts + 3 * (size_t)j;
    const double c0 = a.cscale * cp[0], c1 = a.cscale * cp[1], c2 = a.cscale * cp[2];
    if (a.tgt32) a.tgt32[a.N + j] = make_float4((float)c0, (float)c1, (float)c2, 0.f);
    if (a.tgt32lo)
      a.tgt32lo[a.N + j] = make_float4((float)(c0 - (double)(float)c0), (float)(c1 - (double)(float)c1),
                                       (float)(c2 - (double)(float)c2), 0.f);
    if (a.tgt64) a.tgt64[a.N + j] = make_double4_32a(c0, c1, c2, 0.0);
  }
}

cudaError_t launch_prep(const PrepArgs& a, int nblk, cudaStream_t s) {
  (void)nblk;
  const int nb = (a.N + kIonsPerBlock - 1) / kIonsPerBlock;
  k_prep_count<<<nb, kPrepThreads, 0, s>>>(a);
  k_prep_scan<<<1, kScanThreads, 0, s>>>(a, nb);
  const int ne = a.N > a.n_check ? a.N : a.n_check;
  k_prep_emit<<<(ne + kEmitThreads - 1) / kEmitThreads, kEmitThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ fit + map
constexpr int kFitThreads = 256;

// v = [Phi_B at the check points ; (2D) dPhi_B/dz there ; (gradient rows)
// dx, dy, dz Phi_B at the first n_grad check points (monitoring points and
// their wraps), component-major].
__global__ void k_check_combine(const double* part, int n_chunks, int ld, int N, int n_check,
                                int dims, int n_grad, double* v, double* cphi, double* cdz) {
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
  if (c < n_grad) {
    double gx = 0.0, gy = 0.0;
    for (int ch = 0; ch < n_chunks; ++ch) {
      gx += part[((size_t)ch * 4 + 1) * ld + N + c];
      gy += part[((size_t)ch * 4 + 2) * ld + N + c];
    }
    double* vg = v + (dims == 2 ? 2 * n_check : n_check);
    vg[c] = gx;
    vg[n_grad + c] = gy;
    vg[2 * n_grad + c] = d;
  }
}

__global__ void __launch_bounds__(kFitThreads) k_gemv_rows(const double* P, int nv, const double* v, double* A) {
  __shared__ double sh[kFitThreads];
  const double* row = P + (size_t)blockIdx.x * nv;
  double s = 0.0;
  for (int k = threadIdx.x; k < nv; k += kFitThreads) s += row[k] * v[k];
  s = block_sum_d<kFitThreads>(s, sh);
  if (threadIdx.x == 0) A[blockIdx.x] = s;
}

// Q = W A, one warp per surface point: the lanes read the row of W
// coalesced (every 32nd coefficient each) and a fixed butterfly adds them.
__global__ void __launch_bounds__(256) k_surface(const double* __restrict__ W, int M, int nA,
                                                 const double* __restrict__ A, const double* __restrict__ ysurf,
                                                 double scale, double* Q, float4* s32, double4_32a* s64) {
  const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (m >= M) return;   // uniform per warp
  const double* w = W + (size_t)m * nA;
  double s = 0.0;
  for (int r = lane; r < nA; r += 32) s += w[r] * A[r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  s *= scale;   // W and the surface points of a geometry built for a box scaled by 1/scale
  Q[m] = s;
  const double x = scale * ysurf[3 * m], y = scale * ysurf[3 * m + 1], z = scale * ysurf[3 * m + 2];
  if (s32) s32[m] = make_float4((float)x, (float)y, (float)z, (float)s);
  if (s64) s64[m] = make_double4_32a(x, y, z, s);
}

cudaError_t launch_fit(int dims, const double* part, int n_chunks, int ld, int N, int n_check,
                       int n_grad, const double* P, int nA, int nv, const double* W, int M,
                       const double* ysurf, double scale, double* v, double* A, double* cphi,
                       double* cdz, double* Q, float4* s32, double4_32a* s64, cudaStream_t s) {
  k_check_combine<<<(n_check + 255) / 256, 256, 0, s>>>(part, n_chunks, ld, N, n_check, dims, n_grad, v,
                                                        cphi, cdz);
  k_gemv_rows<<<nA, kFitThreads, 0, s>>>(P, nv, v, A);
  k_surface<<<(int)(((size_t)M * 32 + 255) / 256), 256, 0, s>>>(W, M, nA, A, ysurf, scale, Q, s32, s64);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ far field as a series
// The fitted truncated series of Sec. 2.2, Eq. 5 evaluated directly at each
// ion (an alternative to the surface charges): phi = sum_{n>=1} A_nm S_nm,
// S_nm the real orthonormal solid harmonics in coordinates scaled by 1/R_c,
// written as polynomials: (x + iy)^m = C_m + i S_m and
// V_n^m(z, r^2) = r^(n-m) d^m P_n/dt^m (t = z/r) from the three-term
// recursion.  The gradient carries dV/dz at fixed r^2, dV/d(r^2) and the x, y
// derivatives of C_m, S_m along the same recursions.  norm[n*(p+1) + m] holds
// c_n0 for m = 0 and sqrt(2) c_nm (2m-1)!! for m > 0.
template <typename T, typename TV>
__global__ void __launch_bounds__(256) k_far_series(const TV* __restrict__ tgt, int N, const double* __restrict__ A,
                                                    const double* __restrict__ norm, int p, double inv_rc,
                                                    double* __restrict__ out) {
  // per block: the coefficient pairs (A_n,m c, A_n,-m c) for 0 <= m <= n <= p in
  // the working precision, then 1/k for k = 1..p (the recursion's divisor)
  extern __shared__ __align__(16) unsigned char far_smem[];
  T* coef = reinterpret_cast<T*>(far_smem);
  const int P1 = p + 1;
  T* recip = coef + 2 * P1 * P1;
  for (int e = threadIdx.x; e < P1 * P1; e += blockDim.x) {
    const int n = e / P1, m = e - n * P1;
    T ac = 0, as = 0;
    if (n >= 1 && m <= n) {
      const int base = n * n + n - 1;           // coefficient index of (n, 0)
      const double c = norm[e];
      ac = (T)(A[base + m] * c);
      as = m ? (T)(A[base - m] * c) : (T)0;
    }
    coef[2 * e] = ac;
    coef[2 * e + 1] = as;
  }
  for (int k = threadIdx.x; k <= p; k += blockDim.x) recip[k] = k ? (T)1 / (T)k : (T)0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const TV t = tgt[i];
  const T s = (T)inv_rc;
  const T x = (T)t.x * s, y = (T)t.y * s, z = (T)t.z * s;
  const T r2 = x * x + y * y + z * z;
  T phi = 0, gx = 0, gy = 0, gz = 0;
  T C = 1, S = 0, Cx = 0, Cy = 0, Sx = 0, Sy = 0;
  for (int m = 0; m <= p; ++m) {
    // V_n^m / (2m-1)!!: the recursion is linear, so the double factorial
    // lives in the host-side table (keeps FP32 in range for large p)
    T v1 = 1, vz1 = 0, vr1 = 0;       // V_{n-1}
    T v2 = 0, vz2 = 0, vr2 = 0;       // V_{n-2}
    for (int n = m; n <= p; ++n) {
      T v, vz, vr;
      if (n == m) {
        v = v1; vz = vz1; vr = vr1;
      } else {
        if (n == m + 1) {
          const T a = (T)(2 * m + 1);
          v = a * z * v1;
          vz = a * (v1 + z * vz1);
          vr = a * z * vr1;
        } else {
          const T a = (T)(2 * n - 1), b = (T)(n + m - 1), inv = recip[n - m];
          v = (a * z * v1 - b * r2 * v2) * inv;
          vz = (a * (v1 + z * vz1) - b * r2 * vz2) * inv;
          vr = (a * z * vr1 - b * (v2 + r2 * vr2)) * inv;
        }
        v2 = v1; vz2 = vz1; vr2 = vr1;
        v1 = v; vz1 = vz; vr1 = vr;
      }
      if (n >= 1) {
        // grad V = (2x dV/dr2, 2y dV/dr2, dV/dz + 2z dV/dr2)
        const T Vx = 2 * x * vr, Vy = 2 * y * vr, Vz = vz + 2 * z * vr;
        const T ac = coef[2 * (n * P1 + m)], as = coef[2 * (n * P1 + m) + 1];
        const T w = ac * C + as * S;                // combined azimuthal factor
        const T wx = ac * Cx + as * Sx, wy = ac * Cy + as * Sy;
        phi += v * w;
        gx += Vx * w + v * wx;
        gy += Vy * w + v * wy;
        gz += Vz * w;
      }
    }
    // (x + iy)^(m+1) and its x, y derivatives
    const T nC = x * C - y * S, nS = x * S + y * C;
    const T nCx = C + x * Cx - y * Sx, nSx = S + x * Sx + y * Cx;
    const T nCy = x * Cy - S - y * Sy, nSy = x * Sy + C + y * Cy;
    C = nC; S = nS; Cx = nCx; Sx = nSx; Cy = nCy; Sy = nSy;
  }
  out[i] = (double)phi;
  out[(size_t)N + i] = (double)gx * inv_rc;
  out[2 * (size_t)N + i] = (double)gy * inv_rc;
  out[3 * (size_t)N + i] = (double)gz * inv_rc;
}

cudaError_t launch_far_series(int precision, const void* tgt, int N, const double* A, const double* norm,
                              int p, double inv_rc, double* out, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int grid = (N + 255) / 256;
  const size_t P1 = (size_t)p + 1;
  const size_t smem = (2 * P1 * P1 + P1) * (precision ? sizeof(float) : sizeof(double));
  if (precision)
    k_far_series<float, float4><<<grid, 256, smem, s>>>((const float4*)tgt, N, A, norm, p, inv_rc, out);
  else
    k_far_series<double, double4_32a><<<grid, 256, smem, s>>>((const double4_32a*)tgt, N, A, norm, p, inv_rc,
                                                              out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ chunk partials
// Sum the per-chunk FP64 partials of a pair launch, part[(ch*4 + c)*ld + r],
// into one row set out[c*ld + r] (the layout of a single chunk).  A block
// takes 32 targets; its 8 lanes per target sum the chunks ch = lane (mod 8)
// in increasing order, then a fixed tree adds the 8 lane sums, so the result
// does not depend on the launch.  Reads are coalesced along the targets.
constexpr int kRedTargets = 32, kRedLanes = 8;

__global__ void __launch_bounds__(kRedTargets * kRedLanes) k_reduce_chunks(const double* __restrict__ part,
                                                                           int n_chunks, int ld, int n_rows,
                                                                           double* __restrict__ out) {
  __shared__ double sh[kRedLanes][4][kRedTargets];
  const int tx = threadIdx.x % kRedTargets, ty = threadIdx.x / kRedTargets;
  const int r = blockIdx.x * kRedTargets + tx;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (r < n_rows)
    for (int ch = ty; ch < n_chunks; ch += kRedLanes)
      for (int c = 0; c < 4; ++c) acc[c] += part[((size_t)ch * 4 + c) * ld + r];
  for (int c = 0; c < 4; ++c) sh[ty][c][tx] = acc[c];
  __syncthreads();
  for (int w = kRedLanes / 2; w > 0; w >>= 1) {
    if (ty < w)
      for (int c = 0; c < 4; ++c) sh[ty][c][tx] += sh[ty + w][c][tx];
    __syncthreads();
  }
  if (ty == 0 && r < n_rows)
    for (int c = 0; c < 4; ++c) out[(size_t)c * ld + r] = sh[0][c][tx];
}

cudaError_t launch_reduce_chunks(const double* part, int n_chunks, int ld, int n_rows, double* out,
                                 cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  k_reduce_chunks<<<(n_rows + kRedTargets - 1) / kRedTargets, kRedTargets * kRedLanes, 0, s>>>(
      part, n_chunks, ld, n_rows, out);
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
