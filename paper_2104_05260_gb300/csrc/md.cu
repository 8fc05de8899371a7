// Device kernels of the MD loop around the electrostatics (the validation
// workload of Sec. 4.1): velocity-Verlet kicks and drift, a cell list for the
// shifted-truncated LJ repulsion, its forces, the Nose-Hoover thermostat
// (symmetric Trotter splitting, chain length one) and an RDF histogram.
// All reductions are fixed-order trees, and each cell's particles are sorted
// by index before use, so a run is bitwise reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include "md_internal.hpp"

namespace hsma {

constexpr int kMdThreads = 256;

__device__ __forceinline__ double md_block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kMdThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int md_cell_of(double x, double inv_w, int n) {
  int c = (int)(x * inv_w);
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// v = s v + (dt/2) F / m;  x += dt v;  wrap into [0, L) and count images
__global__ void __launch_bounds__(kMdThreads) k_md_kick_drift(MdArgs a) {
  const int i = blockIdx.x * kMdThreads + threadIdx.x;
  if (i >= a.N) return;
  const double s = a.sc->vscale;
  for (int d = 0; d < 3; ++d) {
    const size_t k = 3 * (size_t)i + d;
    double v = a.v[k] * s + a.half_dt_m * (a.f_lj[k] + a.f_c[k]);
    double x = a.x[k] + a.dt * v;
    const double L = a.L[d];
    if (a.slab && d == 2) {
      // confined by the walls: no wrap; leaving (0, Lz) is an error
      if (!(x > 0.0 && x < L)) atomicOr(&a.sc->flags, MD_FLAG_LEFT_SLAB);
      a.v[k] = v;
      a.x[k] = x;
      continue;
    }
    double w = floor(x / L);
    x -= w * L;
    // the quotient can round across an integer: bring x back into [0, L)
    if (x >= L) {
      x -= L;
      w += 1.0;
    } else if (x < 0.0) {
      x += L;
      w -= 1.0;
      if (x >= L) {
        x = 0.0;
        w += 1.0;
      }
    }
    a.v[k] = v;
    a.x[k] = x;
    a.img[k] += (int)w;
  }
}

// cell list: slot by atomic counter, then each cell sorted by particle index
__global__ void __launch_bounds__(kMdThreads) k_md_cell_fill(MdArgs a) {
  const int i = blockIdx.x * kMdThreads + threadIdx.x;
  if (i >= a.N) return;
  const int cx = md_cell_of(a.x[3 * (size_t)i], a.inv_w[0], a.nc[0]);
  const int cy = md_cell_of(a.x[3 * (size_t)i + 1], a.inv_w[1], a.nc[1]);
  const int cz = md_cell_of(a.x[3 * (size_t)i + 2], a.inv_w[2], a.nc[2]);
  const int c = (cz * a.nc[1] + cy) * a.nc[0] + cx;
  const int slot = atomicAdd(&a.cell_count[c], 1);
  if (slot < a.cap) a.cell_list[(size_t)c * a.cap + slot] = i;
  else atomicOr(&a.sc->flags, MD_FLAG_CELL_OVERFLOW);
}

__global__ void __launch_bounds__(kMdThreads) k_md_cell_sort(MdArgs a, int n_cells) {
  const int c = blockIdx.x * kMdThreads + threadIdx.x;
  if (c >= n_cells) return;
  const int n = min(a.cell_count[c], a.cap);
  int* l = a.cell_list + (size_t)c * a.cap;
  for (int k = 1; k < n; ++k) {
    const int v = l[k];
    int j = k - 1;
    while (j >= 0 && l[j] > v) {
      l[j + 1] = l[j];
      --j;
    }
    l[j + 1] = v;
  }
}

// shifted-truncated LJ repulsion: one warp per particle, lane k < 27 takes
// neighbour cell k (fixed order), the periodic shift of that cell applied
// explicitly (cells are at least r_c wide and at least 3 a side, so the
// shifted copy is the minimum image); lane sums are added by a fixed
// butterfly.  Per-block energy partials hold half of each pair's energy.
constexpr int kLjWarps = kMdThreads / 32;

__global__ void __launch_bounds__(kMdThreads) k_md_lj(MdArgs a) {
  __shared__ double sh[kMdThreads];
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kLjWarps + (threadIdx.x >> 5);
  double fx = 0.0, fy = 0.0, fz = 0.0, u = 0.0;
  if (i < a.N && lane < 27) {
    const double xi = a.x[3 * (size_t)i], yi = a.x[3 * (size_t)i + 1], zi = a.x[3 * (size_t)i + 2];
    const int c0[3] = {md_cell_of(xi, a.inv_w[0], a.nc[0]), md_cell_of(yi, a.inv_w[1], a.nc[1]),
                       md_cell_of(zi, a.inv_w[2], a.nc[2])};
    const int off[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
    int cc[3];
    double shift[3];
    bool none = false;
    for (int d = 0; d < 3; ++d) {
      cc[d] = c0[d] + off[d];
      shift[d] = 0.0;
      if (a.slab && d == 2) {
        none = cc[d] < 0 || cc[d] >= a.nc[d];   // no cell beyond a wall
        continue;
      }
      if (cc[d] < 0) {
        cc[d] += a.nc[d];
        shift[d] = -a.L[d];
      } else if (cc[d] >= a.nc[d]) {
        cc[d] -= a.nc[d];
        shift[d] = a.L[d];
      }
    }
    const int c = none ? 0 : (cc[2] * a.nc[1] + cc[1]) * a.nc[0] + cc[0];
    const int n = none ? 0 : min(a.cell_count[c], a.cap);
    const int* l = a.cell_list + (size_t)c * a.cap;
    for (int k = 0; k < n; ++k) {
      const int j = l[k];
      if (j == i) continue;
      const double dx = (a.x[3 * (size_t)j] + shift[0]) - xi;
      const double dy = (a.x[3 * (size_t)j + 1] + shift[1]) - yi;
      const double dz = (a.x[3 * (size_t)j + 2] + shift[2]) - zi;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < a.rc2) {
        const double s2 = a.sigma2 / r2;
        const double s6 = s2 * s2 * s2;
        u += 0.5 * (4.0 * a.eps * (s6 * s6 - s6) + a.eps);
        const double f = 24.0 * a.eps * (2.0 * s6 * s6 - s6) / r2;   // force on i is -f d
        fx -= f * dx;
        fy -= f * dy;
        fz -= f * dz;
      }
    }
    if (a.slab && lane == 0) {
      // the two walls: distance d, force along the wall normal
      const double dd[2] = {zi, a.L[2] - zi}, sgn[2] = {1.0, -1.0};
      for (int wv = 0; wv < 2; ++wv)
        if (dd[wv] < a.wall_rc) {
          const double s2 = a.wall_sigma * a.wall_sigma / (dd[wv] * dd[wv]);
          const double s6 = s2 * s2 * s2;
          u += 4.0 * a.wall_eps * (s6 * s6 - s6) + a.wall_eps;
          fz += sgn[wv] * 24.0 * a.wall_eps * (2.0 * s6 * s6 - s6) / dd[wv];
        }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
    u += __shfl_xor_sync(0xffffffffu, u, o);
  }
  if (lane == 0 && i < a.N) {
    a.f_lj[3 * (size_t)i] = fx;
    a.f_lj[3 * (size_t)i + 1] = fy;
    a.f_lj[3 * (size_t)i + 2] = fz;
  }
  // one energy value per warp (lane 0), the rest zero, then the block tree
  u = (lane == 0) ? u : 0.0;
  u = md_block_sum(u, sh);
  if (threadIdx.x == 0) a.blk_u[blockIdx.x] = u;
}

// v += (dt/2) F / m; per-block kinetic-energy partials
__global__ void __launch_bounds__(kMdThreads) k_md_kick(MdArgs a) {
  __shared__ double sh[kMdThreads];
  const int i = blockIdx.x * kMdThreads + threadIdx.x;
  double k2 = 0.0;
  if (i < a.N) {
    for (int d = 0; d < 3; ++d) {
      const size_t k = 3 * (size_t)i + d;
      const double v = a.v[k] + a.half_dt_m * (a.f_lj[k] + a.f_c[k]);
      a.v[k] = v;
      k2 += v * v;
    }
  }
  k2 = md_block_sum(k2, sh);
  if (threadIdx.x == 0) a.blk_k[blockIdx.x] = k2;
}

// the sum of v^2 as it stands (before the first step)
__global__ void __launch_bounds__(kMdThreads) k_md_ke(MdArgs a) {
  __shared__ double sh[kMdThreads];
  const int i = blockIdx.x * kMdThreads + threadIdx.x;
  double k2 = 0.0;
  if (i < a.N)
    for (int d = 0; d < 3; ++d) k2 += a.v[3 * (size_t)i + d] * a.v[3 * (size_t)i + d];
  k2 = md_block_sum(k2, sh);
  if (threadIdx.x == 0) a.blk_k[blockIdx.x] = k2;
}

// Thermostat half step of length dt/2 on the kinetic energy K (returns the
// velocity scale, updates xi, eta and K).
__device__ double nh_half(MdScalars* sc, const MdArgs& a, double* K) {
  const double h = 0.5 * a.dt;
  sc->xi += (2.0 * *K - a.g_kT) / a.Q * (0.5 * h);
  const double f = exp(-sc->xi * h);
  sc->eta += sc->xi * h;
  *K *= f * f;
  sc->xi += (2.0 * *K - a.g_kT) / a.Q * (0.5 * h);
  return f;
}

// One block: totals in fixed order, thermostat, thermo row.
//  mode 0: end of a step (end-of-step half, record, start-of-next half)
//  mode 1: start of a run (the start-of-step half only)
__global__ void __launch_bounds__(kMdThreads) k_md_finish(MdArgs a, int nblk_k, int nblk_u, int mode) {
  __shared__ double sh[kMdThreads];
  double k2 = 0.0, u = 0.0;
  {
    const int per = (nblk_k + kMdThreads - 1) / kMdThreads;
    const int b0 = threadIdx.x * per, b1 = min(nblk_k, b0 + per);
    for (int b = b0; b < b1; ++b) k2 += a.blk_k[b];
  }
  {
    const int per = (nblk_u + kMdThreads - 1) / kMdThreads;
    const int b0 = threadIdx.x * per, b1 = min(nblk_u, b0 + per);
    for (int b = b0; b < b1; ++b) u += a.blk_u[b];
  }
  k2 = md_block_sum(k2, sh);
  u = md_block_sum(u, sh);
  if (threadIdx.x != 0) return;
  MdScalars* sc = a.sc;
  double K = 0.5 * a.mass * k2;
  double s = 1.0;
  if (mode == 0) {
    if (a.thermostat) s = nh_half(sc, a, &K);
    sc->vscale_end = s;   // the physical velocities of this step are v * s
    const double uc = a.coul_energy ? *a.coul_energy : 0.0;
    const long long row = sc->step;
    if (row < a.thermo_cap) {
      double* t = a.thermo + (size_t)row * MD_THERMO_COLS;
      t[0] = K;
      t[1] = u;
      t[2] = uc;
      t[3] = sc->xi;
      t[4] = sc->eta;
      t[5] = K + u + uc + (a.thermostat ? 0.5 * a.Q * sc->xi * sc->xi + a.g_kT * sc->eta : 0.0);
    }
    sc->step = row + 1;
    sc->last_K = K;
    sc->last_U = u + uc;
  }
  if (a.thermostat) s *= nh_half(sc, a, &K);
  sc->vscale = s;
}

// RDF pair counts: hist[kind * bins + b], kind 0 = (+, -), 1 = (+, +),
// 2 = (-, -); all pairs i < j, minimum image
// Pair counts for the RDF: one warp per particle i, its lanes over j > i.
// The minimum image multiplies by 1/L (a division per pair is a long
// sequence on the FP64 pipe); the quotient can differ from dx / L in its
// last bit only where it rounds at a half-integer, i.e. |dx| near L/2, and
// such a pair lies at r >= L/2 >= rdf_rmax either way, so the counts are
// those of the division.  Counts go to a per-block histogram in shared
// memory when it fits (kRdfSmemBins bins), then once per bin to the global
// one; integer sums, so the order does not matter.
constexpr int kRdfSmemBins = 4096;

__global__ void __launch_bounds__(kMdThreads) k_md_rdf(MdArgs a) {
  extern __shared__ unsigned int rdf_local[];   // 3 x rdf_bins when local
  const bool local = a.rdf_bins <= kRdfSmemBins;
  if (local) {
    for (int k = threadIdx.x; k < 3 * a.rdf_bins; k += blockDim.x) rdf_local[k] = 0u;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kLjWarps + (threadIdx.x >> 5);
  const double qi = i < a.N ? a.q[i] : 0.0;
  if (qi != 0.0) {
    const double xi = a.x[3 * (size_t)i], yi = a.x[3 * (size_t)i + 1], zi = a.x[3 * (size_t)i + 2];
    const double rmax2 = a.rdf_rmax * a.rdf_rmax;
    const double scale = a.rdf_bins / a.rdf_rmax;
    const double ix = 1.0 / a.L[0], iy = 1.0 / a.L[1], iz = 1.0 / a.L[2];
    for (int j = i + 1 + lane; j < a.N; j += 32) {
      const double qj = a.q[j];
      if (qj == 0.0) continue;
      double dx = a.x[3 * (size_t)j] - xi, dy = a.x[3 * (size_t)j + 1] - yi, dz = a.x[3 * (size_t)j + 2] - zi;
      dx -= a.L[0] * rint(dx * ix);
      dy -= a.L[1] * rint(dy * iy);
      if (!a.slab) dz -= a.L[2] * rint(dz * iz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rmax2) {
        const int b = min(a.rdf_bins - 1, (int)(sqrt(r2) * scale));
        const int kind = (qi > 0.0) != (qj > 0.0) ? 0 : (qi > 0.0 ? 1 : 2);
        if (local) atomicAdd(&rdf_local[kind * a.rdf_bins + b], 1u);
        else atomicAdd(&a.rdf[kind * a.rdf_bins + b], 1ULL);
      }
    }
  }
  if (local) {
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * a.rdf_bins; k += blockDim.x)
      if (rdf_local[k]) atomicAdd(&a.rdf[k], (unsigned long long)rdf_local[k]);
  }
}

__global__ void k_md_rdf_count(MdArgs a) { a.sc->rdf_samples += 1; }

// ion density across the slab: counts of cations and anions in zhist_bins
// bins over (0, Lz)
__global__ void __launch_bounds__(kMdThreads) k_md_zhist(MdArgs a) {
  const int i = blockIdx.x * kMdThreads + threadIdx.x;
  if (i >= a.N) return;
  const double qi = a.q[i];
  if (qi == 0.0) return;
  int b = (int)(a.x[3 * (size_t)i + 2] / a.L[2] * a.zhist_bins);
  b = b < 0 ? 0 : (b >= a.zhist_bins ? a.zhist_bins - 1 : b);
  atomicAdd(&a.zhist[(qi > 0.0 ? 0 : 1) * a.zhist_bins + b], 1ULL);
}

static int blocks(int n) { return (n + kMdThreads - 1) / kMdThreads; }

cudaError_t md_launch_kick_drift(const MdArgs& a, cudaStream_t s) {
  k_md_kick_drift<<<blocks(a.N), kMdThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t md_launch_lj(const MdArgs& a, int n_cells, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.cell_count, 0, (size_t)n_cells * sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_md_cell_fill<<<blocks(a.N), kMdThreads, 0, s>>>(a);
  k_md_cell_sort<<<blocks(n_cells), kMdThreads, 0, s>>>(a, n_cells);
  k_md_lj<<<(a.N + kLjWarps - 1) / kLjWarps, kMdThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t md_launch_kick_finish(const MdArgs& a, cudaStream_t s) {
  k_md_kick<<<blocks(a.N), kMdThreads, 0, s>>>(a);
  k_md_finish<<<1, kMdThreads, 0, s>>>(a, blocks(a.N), (a.N + kLjWarps - 1) / kLjWarps, 0);
  return cudaGetLastError();
}

cudaError_t md_launch_start(const MdArgs& a, cudaStream_t s) {
  k_md_ke<<<blocks(a.N), kMdThreads, 0, s>>>(a);
  k_md_finish<<<1, kMdThreads, 0, s>>>(a, blocks(a.N), 0, 1);
  return cudaGetLastError();
}

cudaError_t md_launch_rdf(const MdArgs& a, cudaStream_t s) {
  const size_t smem = a.rdf_bins <= kRdfSmemBins ? (size_t)3 * a.rdf_bins * sizeof(unsigned int) : 0;
  k_md_rdf<<<(a.N + kLjWarps - 1) / kLjWarps, kMdThreads, smem, s>>>(a);
  if (a.slab) k_md_zhist<<<blocks(a.N), kMdThreads, 0, s>>>(a);
  k_md_rdf_count<<<1, 1, 0, s>>>(a);
  return cudaGetLastError();
}

int md_blocks(int N) { return blocks(N); }
int md_lj_blocks(int N) { return (N + kLjWarps - 1) / kLjWarps; }

}  // namespace hsma
