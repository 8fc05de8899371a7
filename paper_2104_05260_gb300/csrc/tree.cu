// Tree evaluation of the near-field and check-point sums (the O(N) path the
// paper takes with an FMM library, Sec. 2.2 last step): the images in B are
// binned into a uniform octree over the cube [-R_s, R_s]^3 with leaves at
// level L, cells carry multipole expansions of order P, and every target sums
//   - the multipoles of the cells in its FMM interaction lists (children of
//     its parent's neighbours that are not its own neighbours), level by
//     level (multipole-to-particle), and
//   - the sources of its neighbourhood directly (FP32 pairs),
// which covers every source exactly once.  Two layouts of the finest level:
//   - leaf multipoles: lists at levels 2..L, direct pairs with the 27
//     neighbouring leaves of the target's own leaf;
//   - direct leaf level (for sparse leaves): lists at levels 2..L-1, direct
//     pairs with every leaf of the 27 neighbours of the target's cell G of
//     level L-1 (the 6 x 6 x 6 leaves around G), the same set for all of G's
//     targets.  The expansion uses the real
// orthonormal solid harmonics of the fit (Eq. 5) and the addition theorem
//   1/|x - s| = sum_n 4 pi/(2n+1) sum_m R_nm(s - c) I_nm(x - c),
// R_nm = r^n Y_nm, I_nm = r^(-n-1) Y_nm, in coordinates scaled by the cell
// width.  Both are polynomials in x, y, z (and 1/r^2 for I) evaluated by
// three-term recursions; norm[n*(P+1) + m] folds in the normalisation and
// (2m-1)!! as in the series far field.
//
// Binning uses atomic slots followed by a per-bin sort by index, and every
// sum has a fixed order, so the result is deterministic.  All arithmetic of
// the expansions is FP32 with FP64 sums across levels; the identity image of
// an ion is skipped and its other own images among the direct pairs are
// summed in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.hpp"

namespace hsma {

constexpr int kTreeThreads = 128;    // targets per M2P/P2P pass
constexpr int kBatch = 8;            // interaction cells staged per barrier
constexpr int kMaxOrder = 14;   // orders 4, 6, ..., 14 are compiled

__device__ __forceinline__ int spread3(int v) {
  // interleave the low 10 bits of v with two zero bits between each
  unsigned x = (unsigned)v & 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return (int)x;
}

__device__ __forceinline__ int morton(int ix, int iy, int iz) {
  return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

__device__ __forceinline__ int cell_coord(float x, float origin, float inv_w, int n) {
  int c = (int)floorf((x - origin) * inv_w);
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// ---------------------------------------------------------------- binning
__global__ void k_tree_bin(const float4* __restrict__ pts, int n_fixed, const DevScalars* sc, TreeArgs t,
                           int* __restrict__ key, int* __restrict__ count) {
  const int n = sc ? sc->Ns : n_fixed;
  const int nside = 1 << t.L;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 p = pts[i];
    const int k = morton(cell_coord(p.x, -t.Rs, t.inv_wL, nside), cell_coord(p.y, -t.Rs, t.inv_wL, nside),
                         cell_coord(p.z, -t.Rs, t.inv_wL, nside));
    key[i] = k;
    atomicAdd(&count[k], 1);
  }
}

// exclusive scan of count[0..n) into start[0..n], one block: warp w takes a
// contiguous range and reads it 32 entries at a time (coalesced), with warp
// shuffles for the running prefix; a second pass writes the offsets
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

__global__ void __launch_bounds__(1024) k_tree_scan(const int* __restrict__ count, int n, int* __restrict__ start) {
  __shared__ int wsum[32];
  __shared__ int total;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_warp = ((n + 31) / 32 + 31) / 32 * 32;
  const int b0 = min(n, warp * per_warp), b1 = min(n, b0 + per_warp);
  int s = 0;
  for (int b = b0 + lane; b < b1; b += 32) s += count[b];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane == 0) wsum[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const int v = wsum[lane];
    const int incl = warp_incl_scan(v, lane);
    wsum[lane] = incl - v;
    if (lane == 31) total = incl;
  }
  __syncthreads();
  int carry = wsum[warp];
  for (int b = b0; b < b1; b += 32) {
    const int i = b + lane;
    const int v = i < b1 ? count[i] : 0;
    const int incl = warp_incl_scan(v, lane);
    if (i < b1) start[i] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (threadIdx.x == 0) start[n] = total;
}

__global__ void k_tree_fill(int n_fixed, const DevScalars* sc, const int* __restrict__ key,
                            const int* __restrict__ start, int* __restrict__ cursor, int* __restrict__ order) {
  const int n = sc ? sc->Ns : n_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = key[i];
    order[start[k] + atomicAdd(&cursor[k], 1)] = i;
  }
}

// each bin's entries in increasing index order (deterministic sums): one
// warp per bin; the entries (distinct indices) are ranked by counting the
// smaller ones, up to kSortPer per lane in registers, then written in place.
// Larger bins (never seen at the planned leaf sizes) fall back to an
// insertion sort by one lane.
constexpr int kSortPer = 8;

__global__ void k_tree_sort_bins(const int* __restrict__ start, int n_bins, int* __restrict__ order) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < n_bins; b += warps) {
    int* l = order + start[b];
    const int n = start[b + 1] - start[b];
    if (n <= 1) continue;
    if (n <= 32 * kSortPer) {
      int v[kSortPer], rank[kSortPer];
#pragma unroll
      for (int t = 0; t < kSortPer; ++t) {
        const int i = t * 32 + lane;
        v[t] = i < n ? l[i] : 0x7fffffff;
        rank[t] = 0;
      }
#pragma unroll
      for (int t2 = 0; t2 < kSortPer; ++t2) {
        if (t2 * 32 >= n) break;
        for (int j = 0; j < 32; ++j) {
          const int o = __shfl_sync(0xffffffffu, v[t2], j);
#pragma unroll
          for (int t = 0; t < kSortPer; ++t) rank[t] += (o < v[t]) ? 1 : 0;
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kSortPer; ++t)
        if (t * 32 + lane < n) l[rank[t]] = v[t];
      __syncwarp();
    } else if (lane == 0) {
      for (int k = 1; k < n; ++k) {
        const int x = l[k];
        int j = k - 1;
        while (j >= 0 && l[j] > x) {
          l[j + 1] = l[j];
          --j;
        }
        l[j + 1] = x;
      }
    }
    __syncwarp();
  }
}

// sources in bin order (positions and charges), for the P2M and P2P loops
__global__ void k_tree_gather(const float4* __restrict__ src, const int* __restrict__ order, int n_fixed,
                              const DevScalars* sc, float4* __restrict__ out) {
  const int n = sc ? sc->Ns : n_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = src[order[i]];
}

// ---------------------------------------------------------------- P2M
// One block per item (a cell of level il >= l: a contiguous range of leaves
// in Morton order), its sources expanded about the centre of its level-l
// ancestor.  Each lane takes one source and walks all (n, m) by the regular
// recursions (P a compile-time constant).  The terms come out in a fixed
// production order j (chain m = 0..P; n = m..P; cos then sin); each group of
// 32 is written row-wise into a padded 32 x 33 tile of the warp's shared
// memory and read back column-wise, so lane L sums term 32 g + L over the
// warp's 32 sources in lane order.  The warps' rows are added in warp order
// in FP64.  part[item * nc + k], k = n^2 + n +- m.
constexpr int kP2mThreads = 128;

// production index -> harmonic index k
template <int P>
__device__ __forceinline__ int p2m_term(int j) {
  int m = 0, left = j;
  while (true) {
    const int len = m == 0 ? P + 1 : 2 * (P - m + 1);
    if (left < len) break;
    left -= len;
    ++m;
  }
  if (m == 0) return left * left + left;
  const int n = m + left / 2;
  return n * n + n + ((left & 1) ? -m : m);
}

template <int P>
__global__ void __launch_bounds__(kP2mThreads) k_tree_p2m(TreeArgs t, int l, int il, const float4* __restrict__ srcs,
                                                          const int* __restrict__ leaf_start,
                                                          double* __restrict__ part) {
  constexpr int nc = (P + 1) * (P + 1);
  constexpr int ng = (nc + 31) / 32;    // groups of 32 terms; lane L owns term 32 g + L
  constexpr int kWarps = kP2mThreads / 32;
  __shared__ float acc[kWarps][ng * 32];
  __shared__ float tile[kWarps][32 * 33];
  const int item = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* tw = tile[warp];
  const int shift = 3 * (t.L - il);
  const int s0 = leaf_start[item << shift], s1 = leaf_start[(item + 1) << shift];
  for (int g = 0; g < ng; ++g) acc[warp][g * 32 + lane] = 0.0f;
  if (s1 > s0) {
    int ix, iy, iz;
    {
      const int code = item >> (3 * (il - l));
      ix = iy = iz = 0;
      for (int b = 0; b < l; ++b) {
        ix |= ((code >> (3 * b)) & 1) << b;
        iy |= ((code >> (3 * b + 1)) & 1) << b;
        iz |= ((code >> (3 * b + 2)) & 1) << b;
      }
    }
    const float w = t.D / (float)(1 << l), inv_w = 1.0f / w;
    const float cx = -t.Rs + (ix + 0.5f) * w, cy = -t.Rs + (iy + 0.5f) * w, cz = -t.Rs + (iz + 0.5f) * w;
    for (int sb = s0 + warp * 32; sb < s1; sb += kP2mThreads) {
      const int si = sb + lane;
      float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);   // lanes past the end carry q = 0
      if (si < s1) pt = srcs[si];
      const float x = (pt.x - cx) * inv_w, y = (pt.y - cy) * inv_w, z = (pt.z - cz) * inv_w;
      const float r2 = x * x + y * y + z * z;
      float C = pt.w, S = 0.0f;   // q (x + iy)^m
      int j = 0;                  // production index
#pragma unroll
      for (int m = 0; m <= P; ++m) {
        float v1 = 1.0f, v2 = 0.0f;
#pragma unroll
        for (int n = m; n <= P; ++n) {
          if (n == m + 1) {
            v2 = v1;
            v1 = (float)(2 * m + 1) * z * v1;
          } else if (n > m + 1) {
            const float v = ((float)(2 * n - 1) / (float)(n - m)) * z * v1 - ((float)(n + m - 1) / (float)(n - m)) * r2 * v2;
            v2 = v1;
            v1 = v;
          }
#pragma unroll
          for (int cs = 0; cs < (m > 0 ? 2 : 1); ++cs) {
            tw[lane * 33 + (j & 31)] = v1 * (cs == 0 ? C : S);
            if ((j & 31) == 31 || j == nc - 1) {
              __syncwarp();
              float sum = 0.0f;
#pragma unroll 8
              for (int r = 0; r < 32; ++r) sum += tw[r * 33 + lane];
              if ((j & ~31) + lane < nc) acc[warp][(j & ~31) + lane] += sum;
              __syncwarp();
            }
            ++j;
          }
        }
        const float nC = x * C - y * S;
        S = x * S + y * C;
        C = nC;
      }
    }
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < nc; jj += kP2mThreads) {
    double sum = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; ++w2) sum += (double)acc[w2][jj];
    const int k = p2m_term<P>(jj);
    part[(size_t)item * nc + k] = sum * (double)t.fac[k];
  }
}

// Multipoles are stored in rows n = 0..P of 2n + 2 floats starting at
// n (n + 1): the cos coefficient of m = 0, one unused slot, then the (cos,
// sin) pair of each m = 1..n, so that the evaluation reads a pair with one
// 8-byte load.  Slot of the harmonic index k = n^2 + n +- m:
__device__ __forceinline__ int paired_slot(int k) {
  int n = (int)sqrtf((float)k);
  while ((n + 1) * (n + 1) <= k) ++n;
  while (n * n > k) --n;
  const int off = k - n * n - n;   // +m (cos) or -m (sin)
  const int m = off < 0 ? -off : off;
  return n * (n + 1) + (m == 0 ? 0 : 2 * m + (off < 0 ? 1 : 0));
}

// M[cell][paired_slot(k)] = sum over the cell's items (contiguous in Morton
// order) of part[.][k]; ncp = (P + 1)(P + 2) floats a cell
__global__ void k_tree_m_reduce(const double* __restrict__ part, int items_per_cell, int n_cells, int nc, int ncp,
                                float* __restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cells * nc) return;
  const int c = i / nc, k = i - c * nc;
  double s = 0.0;
  for (int j = 0; j < items_per_cell; ++j) s += part[((size_t)c * items_per_cell + j) * nc + k];
  M[(size_t)c * ncp + paired_slot(k)] = (float)s;
}

// ---------------------------------------------------------------- M2P + P2P
// One warp per work item: up to 32 targets of one cell G of level L-1 (in
// index order within each leaf) and one part of their lists.  For levels
// l < L the interaction list depends only on G's ancestor, so each listed
// cell's multipole is staged once in shared memory for the warp's targets.
// With leaf multipoles, the leaf-level list is the children of G's
// neighbours, a lane skipping the leaves adjacent to its own, and direct
// pairs come from the 4 x 4 x 4 leaves around G, each lane taking those
// adjacent to its own leaf; with a direct leaf level the direct pairs are the
// 6 x 6 x 6 leaves around G for every lane.  Tiles whose index range holds no
// identity or own image of any lane's target are summed two sources at a
// time with paired FP32 instructions.
//
// Multipoles hold 4 pi/(2n+1) norm^2 sum q V'T, so the evaluation multiplies
// by the irregular polynomial U'T alone; 1/(n-m) comes from a table.
template <int P, int PL>
__device__ __forceinline__ void m2p_accumulate(const float* __restrict__ Mc, float x, float y, float z, bool full,
                                               float* phi, float* gx, float* gy, float* gz) {
  // The terms n <= P when full, else n <= PL (PL <= P).  One code body serves
  // both orders, so that warps at different orders share the instruction
  // cache: the terms n > PL are the tail of each m-chain (m <= PL) and the
  // whole chains m > PL, each skipped by one test of full, not one per term.
  // P is a compile-time constant: both loops unroll and the recursion
  // coefficients fold.  A term is u(r^2, z) (C_m Mc + S_m Ms) with
  // C_m + i S_m = (x + iy)^m, so its gradient is
  //   2 (x, y, z) du/dr^2 (...) + (0, 0, du/dz|r^2) (...) + u (d/dx, d/dy)(...),
  // and d/dx (x + iy)^m = m (x + iy)^(m-1), d/dy = i m (x + iy)^(m-1).
  // Along each m-chain the terms are summed against Mc and Ms separately and
  // the powers of x + iy are applied once per chain.
  // The chain variable is v_n = U_n / K_nm with K_nm = prod_{k=m+1..n}
  // (2k-1)/(k-m), which makes the z-term coefficient of the three-term
  // recursion 1:  v_n = z rho v_(n-1) - c_nm rho v_(n-2),
  // c_nm = (n+m-1)(n-m-1) / ((2n-1)(2n-3)).  K_nm is folded into the stored
  // multipoles (the fac table), so the sums below see U_n M_nm unchanged.
  const float r2 = x * x + y * y + z * z;
  const float rho = 1.0f / r2;
  const float rinv = rsqrtf(r2);
  const float zr = z * rho;
  float C = 1.0f, S = 0.0f, C1 = 0.0f, S1 = 0.0f;   // (x + iy)^m and (x + iy)^(m-1)
  float um = rinv;   // r^-(2m+1) for m = 0
  float p = 0.f, sq = 0.f, sz = 0.f, sx = 0.f, sy = 0.f;
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    if (m == PL + 1 && !full) break;
    float u1 = um, z1 = 0.0f, q1 = -((float)m + 0.5f) * rho * um;   // v, dv/dz, dv/d(r^2)
    float u2 = 0.0f, z2 = 0.0f, q2 = 0.0f;
    float uc = 0.f, us = 0.f, qc = 0.f, qs = 0.f, zc = 0.f, zs = 0.f;
#pragma unroll
    for (int n = m; n <= P; ++n) {
      if (m <= PL && n == PL + 1 && !full) break;
      float u, uz, uq;
      if (n == m) {
        u = u1; uz = z1; uq = q1;
      } else {
        if (n == m + 1) {
          u = zr * u1;
          uz = rho * u1;                 // dv_m/dz = 0
          uq = zr * q1 - rho * u;
        } else {
          const float b = ((float)((n + m - 1) * (n - m - 1)) / (float)((2 * n - 1) * (2 * n - 3))) * rho;
          u = zr * u1 - b * u2;
          uz = rho * (u1 + z * z1) - b * z2;
          uq = zr * q1 - b * q2 - rho * u;
        }
        u2 = u1; z2 = z1; q2 = q1;
        u1 = u; z1 = uz; q1 = uq;
      }
      const int row = n * (n + 1);   // paired layout (see k_tree_m_reduce)
      if (m == 0) {
        const float ac = Mc[row];
        uc += u * ac;
        qc += uq * ac;
        zc += uz * ac;
      } else {
        const float2 a = *reinterpret_cast<const float2*>(Mc + row + 2 * m);
        uc += u * a.x;
        qc += uq * a.x;
        zc += uz * a.x;
        us += u * a.y;
        qs += uq * a.y;
        zs += uz * a.y;
      }
    }
    if (m == 0) {
      p += uc;
      sq += qc;
      sz += zc;
    } else {
      p += C * uc + S * us;
      sq += C * qc + S * qs;
      sz += C * zc + S * zs;
      sx += (float)m * (C1 * uc + S1 * us);
      sy += (float)m * (C1 * us - S1 * uc);
    }
    C1 = C; S1 = S;
    const float nC = x * C - y * S, nS = x * S + y * C;
    C = nC; S = nS;
    um *= rho;
  }
  *phi += p;
  *gx += 2.0f * x * sq + sx;
  *gy += 2.0f * y * sq + sy;
  *gz += 2.0f * z * sq + sz;
}

__device__ __forceinline__ void morton_decode(int code, int bits, int* x, int* y, int* z) {
  int ix = 0, iy = 0, iz = 0;
  for (int b = 0; b < bits; ++b) {
    ix |= ((code >> (3 * b)) & 1) << b;
    iy |= ((code >> (3 * b + 1)) & 1) << b;
    iz |= ((code >> (3 * b + 2)) & 1) << b;
  }
  *x = ix;
  *y = iy;
  *z = iz;
}

// Work items of the evaluation: a task is up to 32 consecutive targets of one
// cell G of level L-1 (task_start[G] .. task_start[G+1]); each task is split
// into S parts, part s taking every S-th batch of each level's interaction
// list and every S-th of the candidate leaves for direct pairs (4x4x4 around
// G's children, or the 6x6x6 of the direct leaf level).  An item (task, part) is
// computed the same way whichever warp takes it, and writes its own partial
// out[(s*4 + c)*ld + t]; the parts are summed afterwards in fixed order.
__global__ void k_tree_tasks(const int* __restrict__ tgt_start, int n_cells, int* __restrict__ count) {
  const int G = blockIdx.x * blockDim.x + threadIdx.x;
  if (G < n_cells) count[G] = (tgt_start[(G + 1) << 3] - tgt_start[G << 3] + 31) >> 5;
}

// What the direct pairs need to sum an ion's own images in FP64: an ion
// close to a dielectric interface has its own reflection 2d away, where
// rounding the coordinates to FP32 would spoil a large term.
struct OwnImages {
  const DevScalars* sc;
  const double* xc;
  const double* q;
  const double* shifts;
  const int* ioff;
  const int* icnt;
  const int* img_shift;
};

// Resident blocks of the evaluation kernel per SM: 6 (80 registers a thread)
// up to order 10; the higher orders need more registers and keep 5.  Six
// blocks measured 2 % faster than 5 at P = 10; 7 and 8 (72 and 64 registers)
// were slower.
constexpr int tree_eval_blocks(int P) { return P <= 10 ? 6 : 5; }

template <int P, bool COUNT>
__global__ void __launch_bounds__(kTreeThreads, tree_eval_blocks(P)) k_tree_eval(TreeArgs t, const float4* __restrict__ tgt,
                                                               int n_ions, const int* __restrict__ tgt_start,
                                                               const int* __restrict__ tgt_order,
                                                               const float4* __restrict__ srcs,
                                                               const int* __restrict__ src_order,
                                                               const int* __restrict__ leaf_start,
                                                               const float* __restrict__ M,
                                                               const int* __restrict__ task_start, int n_cells,
                                                               int S, int* __restrict__ queue,
                                                               double* __restrict__ out, int ld, OwnImages own,
                                                               unsigned long long* __restrict__ work) {
  // Persistent warps, no block barriers: each warp takes the next item from
  // the queue, compacts each level's list itself and stages multipoles in its
  // own slice of shared memory.
  extern __shared__ __align__(16) float tree_smem[];
  constexpr int nc = (P + 1) * (P + 2);   // floats a cell (paired layout)
  constexpr int nc4 = (nc + 3) & ~3;
  constexpr int kWarps = kTreeThreads / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sM = tree_smem + (size_t)warp * kBatch * nc4;                        // kBatch multipoles
  float4* stile = reinterpret_cast<float4*>(tree_smem + (size_t)kWarps * kBatch * nc4) + warp * 32;
  float* tx = reinterpret_cast<float*>(stile);   // the warp's direct-pair tile: x, y, z, q arrays
  float* ty = tx + 32;
  float* tz = tx + 64;
  float* tq = tx + 96;
  int* sid = reinterpret_cast<int*>(reinterpret_cast<float4*>(tree_smem + (size_t)kWarps * kBatch * nc4) +
                                    kTreeThreads) + warp * 32;
  int* slist = sid + (kTreeThreads - warp * 32) + warp * 216;                  // compacted list, 216 per warp
  const int nsideL = 1 << t.L;
  const int n_items = S * task_start[n_cells];
  unsigned long long n_m2p = 0, n_dir = 0, n_m2p_low = 0;   // counting instance only
  // far cells of the levels above the leaf level: order PL (see TreeArgs)
  constexpr int PL = P >= 8 ? P - 4 : P;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(queue, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const int task = item / S, part = item - task * S;
    // G: the last cell whose first task is <= task
    int lo = 0, hi = n_cells;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (task_start[mid] <= task) lo = mid;
      else hi = mid - 1;
    }
    const int G = lo;                              // cell of level L-1
    const int t0 = tgt_start[G << 3], t1 = tgt_start[(G + 1) << 3];
    const int base = t0 + (task - task_start[G]) * 32;
    int gx0, gy0, gz0;
    morton_decode(G, t.L - 1, &gx0, &gy0, &gz0);
    const int slot = base + lane;
    const bool active = slot < t1;
    const int ti = active ? tgt_order[slot] : tgt_order[t0];
    const float4 p = tgt[ti];
    // this target's leaf (the first leaf of G whose range holds the slot);
    // only the leaf-multipole layout needs it
    int lx = 0, ly = 0, lz = 0;
    if (!t.direct_leaf) {
      int leaf = G << 3;
      while (leaf < ((G + 1) << 3) - 1 && tgt_start[leaf + 1] <= slot) ++leaf;
      morton_decode(leaf, t.L, &lx, &ly, &lz);
    }
    double phi = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    const int l_top = t.direct_leaf ? t.L - 1 : t.L;
    for (int l = 2; l <= l_top; ++l) {
      // the reference cell: G's ancestor at l < L; at l = L the lists of all
      // eight leaves together (children of G's neighbours)
      const int sh = (t.L - 1) - l;
      const int cx = l < t.L ? gx0 >> sh : gx0, cy = l < t.L ? gy0 >> sh : gy0, cz = l < t.L ? gz0 >> sh : gz0;
      const int px = l < t.L ? cx >> 1 : gx0, py = l < t.L ? cy >> 1 : gy0, pz = l < t.L ? cz >> 1 : gz0;
      const int nside = 1 << l;
      const float w = t.D / (float)nside, inv_w = 1.0f / w;
      const int lshift = 3 * (t.L - l);
      // the list's non-empty cells, compacted in candidate order (warp ballot)
      int n_list = 0;
      for (int r = 0; r < 216; r += 32) {
        const int j = r + lane;
        bool ok = false;
        int code = 0;
        if (j < 216) {
          const int ox = 2 * (px + (j % 3) - 1) + ((j / 27) & 1);
          const int oy = 2 * (py + ((j / 3) % 3) - 1) + ((j / 54) & 1);
          const int oz = 2 * (pz + ((j / 9) % 3) - 1) + ((j / 108) & 1);
          ok = !(ox < 0 || oy < 0 || oz < 0 || ox >= nside || oy >= nside || oz >= nside);
          if (ok && l < t.L && abs(ox - cx) <= 1 && abs(oy - cy) <= 1 && abs(oz - cz) <= 1) ok = false;
          if (ok) {
            code = morton(ox, oy, oz);
            ok = leaf_start[(code + 1) << lshift] != leaf_start[code << lshift];
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) slist[n_list + __popc(bal & ((1u << lane) - 1u))] = code;
        n_list += __popc(bal);
      }
      __syncwarp();
      float fp = 0.0f, fx = 0.0f, fy = 0.0f, fz = 0.0f;
      for (int b0 = part * kBatch; b0 < n_list; b0 += S * kBatch) {
        const int nb = min(kBatch, n_list - b0);
        __syncwarp();
        for (int k = lane; k < nb * nc4; k += 32) {
          const int c = k / nc4, kk = k - c * nc4;
          sM[k] = kk < nc ? M[t.moff[l] + (size_t)slist[b0 + c] * nc + kk] : 0.0f;
        }
        __syncwarp();
        if (active)
          for (int c = 0; c < nb; ++c) {
            int ox, oy, oz;
            morton_decode(slist[b0 + c], l, &ox, &oy, &oz);
            if (l == t.L && abs(ox - lx) <= 1 && abs(oy - ly) <= 1 && abs(oz - lz) <= 1) continue;
            const float dx = (p.x - (-t.Rs + (ox + 0.5f) * w)) * inv_w;
            const float dy = (p.y - (-t.Rs + (oy + 0.5f) * w)) * inv_w;
            const float dz = (p.z - (-t.Rs + (oz + 0.5f) * w)) * inv_w;
            // the same cell for every lane (levels above the leaf level are
            // listed for G's ancestor), so the choice does not diverge
            const int ex = ox - cx, ey = oy - cy, ez = oz - cz;
            const bool far = PL < P && t.far_d2 > 0 && l < t.L && ex * ex + ey * ey + ez * ez >= t.far_d2;
            if (COUNT) {
              if (far) ++n_m2p_low;
              else ++n_m2p;
            }
            m2p_accumulate<P, PL>(sM + c * nc4, dx, dy, dz, !far, &fp, &fx, &fy, &fz);
          }
      }
      phi += (double)fp * (double)inv_w;
      gx += (double)fx * (double)(inv_w * inv_w);
      gy += (double)fy * (double)(inv_w * inv_w);
      gz += (double)fz * (double)(inv_w * inv_w);
    }
    // direct pairs (FP32 pairs, FP64 sums per leaf): the 4 x 4 x 4 leaves
    // around G, each target its own 27; or, with a direct leaf level, the
    // 6 x 6 x 6 leaves around G, all of them for every target.  The identity
    // image of an ion is skipped and its other own images are summed in FP64
    // from the shift table (the same terms as the prep's own-image sums).
    const bool ion = active && ti < n_ions;
    const int own0 = ion ? own.ioff[ti] : 0, own_n = ion ? own.icnt[ti] : 0;
    const int span = t.direct_leaf ? 6 : 4, lo_off = t.direct_leaf ? -2 : -1;
    for (int jl = part; jl < span * span * span; jl += S) {
      const int ox = 2 * gx0 + lo_off + jl % span, oy = 2 * gy0 + lo_off + (jl / span) % span;
      const int oz = 2 * gz0 + lo_off + jl / (span * span);
      if (ox < 0 || oy < 0 || oz < 0 || ox >= nsideL || oy >= nsideL || oz >= nsideL) continue;
      const int code = morton(ox, oy, oz);
      const int s0 = leaf_start[code], s1 = leaf_start[code + 1];
      if (s1 <= s0) continue;
      const bool take =
          active && (t.direct_leaf || (abs(ox - lx) <= 1 && abs(oy - ly) <= 1 && abs(oz - lz) <= 1));
      if (!__any_sync(0xffffffffu, take)) continue;
      float fp = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
      float2 fp2 = make_float2(0.f, 0.f), fx2 = fp2, fy2 = fp2, fz2 = fp2;
      for (int sb = s0; sb < s1; sb += 32) {
        // the warp's tile as x, y, z, q arrays; slots past the leaf's end hold
        // a far, uncharged source
        __syncwarp();
        float4 v = make_float4(1e18f, 1e18f, 1e18f, 0.f);
        int id = -1;
        if (sb + lane < s1) {
          v = srcs[sb + lane];
          id = src_order[sb + lane];
        }
        tx[lane] = v.x;
        ty[lane] = v.y;
        tz[lane] = v.z;
        tq[lane] = v.w;
        sid[lane] = id;
        __syncwarp();
        const int nb = min(32, s1 - sb);
        // a leaf's sources are in increasing index order, so the tile holds
        // neither the target's identity image nor an own image of it when
        // both lie outside [sid[0], sid[nb-1]]: then pairs go two at a time
        const int lo = sid[0], hi = sid[nb - 1];
        const bool clean =
            !ion || ((ti < lo || ti > hi) && (own_n == 0 || own0 + own_n <= lo || own0 > hi));
        if (__all_sync(0xffffffffu, clean)) {
          if (take) {
            if (COUNT) n_dir += nb;
            const float2 npx = make_float2(-p.x, -p.x), npy = make_float2(-p.y, -p.y);
            const float2 npz = make_float2(-p.z, -p.z);
            for (int k = 0; k < nb; k += 2) {   // an odd tile ends on a padding slot
              const float2 dx = __fadd2_rn(*reinterpret_cast<const float2*>(tx + k), npx);
              const float2 dy = __fadd2_rn(*reinterpret_cast<const float2*>(ty + k), npy);
              const float2 dz = __fadd2_rn(*reinterpret_cast<const float2*>(tz + k), npz);
              float2 r2 = __fmul2_rn(dx, dx);
              r2 = __ffma2_rn(dy, dy, r2);
              r2 = __ffma2_rn(dz, dz, r2);
              const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
              const float2 qi = __fmul2_rn(*reinterpret_cast<const float2*>(tq + k), inv);
              fp2 = __fadd2_rn(fp2, qi);
              const float2 q3 = __fmul2_rn(qi, __fmul2_rn(inv, inv));
              fx2 = __ffma2_rn(q3, dx, fx2);
              fy2 = __ffma2_rn(q3, dy, fy2);
              fz2 = __ffma2_rn(q3, dz, fz2);
            }
          }
          continue;
        }
        if (take)
          for (int k = 0; k < nb; ++k) {
            const int sidx = sid[k];
            if (ion && (sidx == ti || (unsigned)(sidx - own0) < (unsigned)own_n)) {
              if (sidx != ti) {
                const double* sh = own.shifts + 5 * own.img_shift[sidx - n_ions];
                const double xi = own.xc[3 * (size_t)ti], yi = own.xc[3 * (size_t)ti + 1];
                const double zi = own.xc[3 * (size_t)ti + 2];
                const double ddx = __dadd_rn(xi, sh[0]) - xi, ddy = __dadd_rn(yi, sh[1]) - yi;
                const double ddz = __dadd_rn(__dmul_rn(sh[2], zi), sh[3]) - zi;
                const double qs = sh[4] * (own.q[ti] - own.sc->qcorr);
                const double inv = rsqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                const double qi = qs * inv, q3 = qi * inv * inv;
                phi += qi;
                gx += q3 * ddx;
                gy += q3 * ddy;
                gz += q3 * ddz;
              }
              continue;
            }
            if (COUNT) ++n_dir;
            const float dx = tx[k] - p.x, dy = ty[k] - p.y, dz = tz[k] - p.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float ri = rsqrtf(r2);
            const float qr = tq[k] * ri;
            const float qr3 = qr * ri * ri;
            fp += qr;
            fx += qr3 * dx;
            fy += qr3 * dy;
            fz += qr3 * dz;
          }
      }
      phi += fp + (fp2.x + fp2.y);
      gx += fx + (fx2.x + fx2.y);
      gy += fy + (fy2.x + fy2.y);
      gz += fz + (fz2.x + fz2.y);
    }
    if (active) {
      // as the pair kernels: phi and its gradient with respect to the target
      double* o = out + (size_t)part * 4 * ld;
      o[ti] = phi;
      o[(size_t)ld + ti] = gx;
      o[2 * (size_t)ld + ti] = gy;
      o[3 * (size_t)ld + ti] = gz;
    }
  }
  if (COUNT) {
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
      n_m2p += __shfl_down_sync(0xffffffffu, n_m2p, w);
      n_dir += __shfl_down_sync(0xffffffffu, n_dir, w);
      n_m2p_low += __shfl_down_sync(0xffffffffu, n_m2p_low, w);
    }
    if (lane == 0) {
      atomicAdd(work, n_m2p);
      atomicAdd(work + 1, n_dir);
      atomicAdd(work + 2, n_m2p_low);
    }
  }
}

int tree_paired_floats(int P) { return (P + 1) * (P + 2); }

size_t tree_eval_smem(int P) {
  const int nc4 = ((P + 1) * (P + 2) + 3) & ~3;
  const int warps = kTreeThreads / 32;
  return (size_t)warps * kBatch * nc4 * 4 + kTreeThreads * 16 + kTreeThreads * 4 + (size_t)warps * 216 * 4;
}

int tree_max_order() { return kMaxOrder; }

int tree_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 1;
  }
  return sms;
}

cudaError_t launch_tree(const TreeLaunch& T, cudaStream_t s) {
  const TreeArgs& t = T.t;
  const int nleaf = 1 << (3 * t.L);
  const int nc = (t.P + 1) * (t.P + 1);
  const int grid = 4 * 152;
  cudaError_t e = cudaMemsetAsync(T.src_count, 0, (size_t)nleaf * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(T.src_cursor, 0, (size_t)nleaf * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(T.tgt_count, 0, (size_t)nleaf * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(T.tgt_cursor, 0, (size_t)nleaf * 4, s);
  if (e != cudaSuccess) return e;
  // sources (count on the device) and targets into leaves
  k_tree_bin<<<grid, 256, 0, s>>>(T.src, 0, T.sc, t, T.src_key, T.src_count);
  k_tree_bin<<<grid, 256, 0, s>>>(T.tgt, T.n_tgt, nullptr, t, T.tgt_key, T.tgt_count);
  k_tree_scan<<<1, 1024, 0, s>>>(T.src_count, nleaf, T.src_start);
  k_tree_scan<<<1, 1024, 0, s>>>(T.tgt_count, nleaf, T.tgt_start);
  k_tree_fill<<<grid, 256, 0, s>>>(0, T.sc, T.src_key, T.src_start, T.src_cursor, T.src_order);
  k_tree_fill<<<grid, 256, 0, s>>>(T.n_tgt, nullptr, T.tgt_key, T.tgt_start, T.tgt_cursor, T.tgt_order);
  k_tree_sort_bins<<<grid, 256, 0, s>>>(T.src_start, nleaf, T.src_order);
  k_tree_sort_bins<<<grid, 256, 0, s>>>(T.tgt_start, nleaf, T.tgt_order);
  k_tree_gather<<<grid, 256, 0, s>>>(T.src, T.src_order, 0, T.sc, T.src_sorted);
  // multipoles, level by level (not the leaf level when it is summed
  // directly): items are cells of level il = max(l, L - 1)
  for (int l = 2; l <= (t.direct_leaf ? t.L - 1 : t.L); ++l) {
    const int il = l >= t.L - 1 ? l : t.L - 1;
    const int items = 1 << (3 * il);
#define HSMA_TREE_P2M(PP) k_tree_p2m<PP><<<items, kP2mThreads, 0, s>>>(t, l, il, T.src_sorted, T.src_start, T.part)
    switch (t.P) {
      case 4: HSMA_TREE_P2M(4); break;
      case 6: HSMA_TREE_P2M(6); break;
      case 8: HSMA_TREE_P2M(8); break;
      case 10: HSMA_TREE_P2M(10); break;
      case 12: HSMA_TREE_P2M(12); break;
      case 14: HSMA_TREE_P2M(14); break;
      default: return cudaErrorInvalidValue;
    }
#undef HSMA_TREE_P2M
    const int cells = 1 << (3 * l);
    const int per = items / cells;
    k_tree_m_reduce<<<(cells * nc + 255) / 256, 256, 0, s>>>(T.part, per, cells, nc, tree_paired_floats(t.P),
                                                              T.M + t.moff[l]);
  }
  // tasks per cell of level L-1 (the cursors are free again after the fills)
  const int n_cells = nleaf / 8;
  int* task_count = T.src_cursor;
  int* task_start = T.tgt_cursor;
  int* queue = T.tgt_count;
  k_tree_tasks<<<(n_cells + 255) / 256, 256, 0, s>>>(T.tgt_start, n_cells, task_count);
  k_tree_scan<<<1, 1024, 0, s>>>(task_count, n_cells, task_start);
  e = cudaMemsetAsync(queue, 0, 4, s);
  if (e != cudaSuccess) return e;
  const OwnImages own{T.sc, T.xc, T.q, T.shifts, T.ioff, T.icnt, T.img_shift};
  const size_t sm = tree_eval_smem(t.P);
  const int eval_grid = tree_eval_blocks(t.P) * tree_sm_count();
  if (T.eval_ev[0]) cudaEventRecord(T.eval_ev[0], s);
#define HSMA_TREE_EVAL(PP)                                                                                  \
  if (T.work)                                                                                                \
    k_tree_eval<PP, true><<<eval_grid, kTreeThreads, sm, s>>>(t, T.tgt, T.n_ions, T.tgt_start, T.tgt_order, \
                                                              T.src_sorted, T.src_order, T.src_start, T.M,    \
                                                              task_start, n_cells, T.parts, queue,            \
                                                              T.out_parts, T.ld, own, T.work);                \
  else                                                                                                       \
    k_tree_eval<PP, false><<<eval_grid, kTreeThreads, sm, s>>>(t, T.tgt, T.n_ions, T.tgt_start, T.tgt_order, \
                                                               T.src_sorted, T.src_order, T.src_start, T.M,    \
                                                               task_start, n_cells, T.parts, queue,            \
                                                               T.out_parts, T.ld, own, nullptr)
  switch (t.P) {
    case 4: HSMA_TREE_EVAL(4); break;
    case 6: HSMA_TREE_EVAL(6); break;
    case 8: HSMA_TREE_EVAL(8); break;
    case 10: HSMA_TREE_EVAL(10); break;
    case 12: HSMA_TREE_EVAL(12); break;
    case 14: HSMA_TREE_EVAL(14); break;
    default: return cudaErrorInvalidValue;
  }
#undef HSMA_TREE_EVAL
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (T.eval_ev[1]) cudaEventRecord(T.eval_ev[1], s);
  return launch_reduce_chunks(T.out_parts, T.parts, T.ld, T.n_tgt, T.out, s);
}

}  // namespace hsma
