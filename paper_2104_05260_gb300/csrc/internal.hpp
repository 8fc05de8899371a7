// Declarations shared by the host API (api.cpp, serve.cpp) and the device
// kernels (kernels.cu).  Everything here is internal to libhsma.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hsma {

// Per-evaluation scalars that live on the device, so the whole evaluation can
// be enqueued without a host round trip.
struct DevScalars {
  double qsum, qabs, qcorr;  // sum q, sum |q|, neutral residual per ion
  double energy;             // 1/2 pref sum q_i Phi_i
  int Ns;                    // images in B (identity section + compacted rest)
  int flags;                 // FLAG_* bits
};

enum { FLAG_NOT_NEUTRAL = 1, FLAG_OUT_OF_SLAB = 2, FLAG_TIMEOUT = 4 };

// Inputs of the three prep kernels (wrap/centre, sphere membership, images).
struct PrepArgs {
  const double* x;       // N*3, API coordinates
  const double* q;       // N
  int N;
  int dims;
  double L[3];
  double Rs2;
  const double* shifts;  // n_shift*5 (sx, sy, zs, zo, f); identity first
  int n_shift;
  const double* check_pts;  // n_check*3 (box-centred), multiplied by cscale
  int n_check;
  double cscale;
  double* xc;            // N*3 box-centred FP64 positions
  int* cnt;              // N: non-identity images of each source inside B
  int* blk;              // per-block image counts -> exclusive offsets
  double* blk_q;
  double* blk_aq;
  DevScalars* sc;
  float4* src32;         // images (x, y, z, q): FP32 path, or NULL
  double4_32a* src64;        // images: FP64 path, or NULL
  float4* tgt32;         // targets: N particles then n_check check points
  double4_32a* tgt64;
  float4* src32lo;       // x - (float)x of the images (exact-difference path), or NULL
  float4* tgt32lo;       // the same for the targets, or NULL
  int* ioff;             // N: first section-1 image of each ion, or NULL
  unsigned* mask;        // N x mwords: bit s-1 set when shift s puts the ion's image in B
  int mwords;            // ceil((n_shift - 1) / 32)
  double* self;          // 4 x N: FP64 sums over each ion's own images, or NULL
  int* img_shift;        // Ns - N: shift index of each section-1 image, or NULL
};

// One generic pair-sum launch: targets x sources -> per-chunk partial sums of
// (phi, dphi/dx, dphi/dy, dphi/dz) in FP64, part[(chunk*4 + c)*ld + t].
struct PairArgs {
  const void* tgt;       // float4* or double4_32a*
  int n_tgt;
  const void* src;       // float4* or double4_32a* (x, y, z, q)
  int n_src;             // used when sc == NULL
  const DevScalars* sc;  // when not NULL, the source count is sc->Ns
  int n_diag;            // target t and source t (t < n_diag) are the same ion
  int n_tiles;           // target tiles
  int n_chunks;          // source chunks per target tile
  double* part;
  int ld;
  // FP32 path: ion t (t < n_diag) also skips its own section-1 images
  // [ioff[t], ioff[t] + icnt[t]); those terms are added in FP64 elsewhere.
  const int* ioff = nullptr;
  const int* icnt = nullptr;
  // exact-difference variants: the FP32 rounding remainders x - (float)x of
  // the sources and targets (null = zero), so that x_s - x_t is formed as
  // (hi_s - hi_t) + (lo_s - lo_t)
  const float4* src_lo = nullptr;
  const float4* tgt_lo = nullptr;
  // Fused chunk reduction (red != NULL): items are numbered tile-major, and
  // the CTA that completes the last chunk of a target tile sums that tile's
  // partials over the chunks, in the fixed order of k_reduce_chunks, into
  // red[c*ld + t].  ticket holds one counter per tile, zero between launches
  // (the reducing CTA sets it back).
  double* red = nullptr;
  int* ticket = nullptr;
  // Dynamic schedule (queue != NULL): CTAs take items from the counter
  // queue[0]; queue[1] counts CTAs that found the queue empty, and the last
  // of them sets both back to zero for the next launch.
  int* queue = nullptr;
};

struct PairPlan {
  int tpt;               // targets per thread (FP32 path)
  int threads;           // threads per CTA
  int n_tiles, n_chunks, grid;
};

// Plans and launches; all return cudaError_t of the launch.
int pair_tile_targets(int precision, int tpt);
cudaError_t launch_prep(const PrepArgs& a, int nblk, cudaStream_t s);
int prep_blocks(int N, int n_check);   // blocks of the prep kernels (8 ions each)
cudaError_t launch_pair(int precision, int tpt, PairArgs a, int grid, cudaStream_t s);
int pair_slots(int precision, int tpt);   // resident CTAs on the whole GPU
// One launch over several packed-FP32 pair sums (descs and start in device
// memory; start has n_desc + 1 entries, start[n_desc] = total items).
cudaError_t launch_pair_ragged(int precision, int variant, const PairArgs* descs, const int* start, int n_desc,
                               int grid, int* queue, cudaStream_t s);
int pair_ragged_slots(int precision, int variant);
int pair_ragged_variant(int precision);   // default kernel code of the ragged launch (plan tiles with it)
bool pair_ragged_code_ok(int precision, int variant);
// Far field as the fitted series itself (no surface charges): out[c*N + i],
// c = phi, grad; norm[n*(p+1) + m] = c_n0 (m = 0), sqrt(2) c_nm (2m-1)!! (m > 0)
// with c_nm the orthonormal harmonic normalisation; A as the fit writes it.
cudaError_t launch_far_series(int precision, const void* tgt, int N, const double* A, const double* norm,
                              int p, double inv_rc, double* out, cudaStream_t s);
// scale multiplies W and ysurf (a geometry built for the box divided by scale)
// Tree evaluation of the near-field and check-point sums (tree.cu).
struct TreeArgs {
  int L, P;              // leaf level (8^L leaves), expansion order
  float Rs, D, inv_wL;   // root cube [-Rs, Rs]^3 of side D (Rs: its half-width); 1 / leaf width
  int moff[8];           // offset (floats) of level l's multipoles in M
  const float* norm;     // (P+1)^2: c_n0, sqrt(2) c_nm (2m-1)!! at n*(P+1) + m
  const float* fac;      // (P+1)^2: 4 pi/(2n+1) * norm^2 at k = n^2 + n + m
  int direct_leaf;       // 1: the leaf level is summed directly (no leaf multipoles)
  // Above the leaf level, a listed cell whose centre lies at least
  // sqrt(far_d2) cell widths from the target's cell is evaluated to order
  // P - 4 instead of P (P >= 8); 0 = every cell to order P.
  int far_d2;
};
struct TreeLaunch {
  TreeArgs t;
  const float4* src;     // images in B (x, y, z, q), count sc->Ns
  const DevScalars* sc;
  const float4* tgt;     // targets: ions (n_ions) then check points (n_tgt total)
  int n_tgt, n_ions;
  int *src_key, *src_count, *src_start, *src_cursor, *src_order;   // leaves: 8^L (+1)
  int *tgt_key, *tgt_count, *tgt_start, *tgt_cursor, *tgt_order;
  float4* src_sorted;    // images in leaf order
  double* part;          // 8^L * (P+1)^2 P2M partials
  float* M;              // multipoles of levels 2..L
  double* out;           // out[c*ld + t], c = phi, grad (one chunk's layout)
  int ld;
  int parts;             // items per task of the evaluation (each a partial sum)
  double* out_parts;     // parts * 4 * ld partials, summed into out in part order
  // own images of the ion targets, summed in FP64 by the direct pairs
  const double* xc;      // n_ions*3 box-centred FP64 positions
  const double* q;       // n_ions charges (neutral residual: sc->qcorr)
  const double* shifts;  // n_shift*5 (sx, sy, zs, zo, f)
  const int* ioff;       // n_ions: first section-1 image of each ion
  const int* icnt;       // n_ions: its number of section-1 images
  const int* img_shift;  // section-1 image (index - n_ions) -> shift index
  // when not NULL, the evaluation runs its counting instance, which adds to
  // work[0] the multipole evaluations (M2P) to order P, to work[1] the FP32
  // direct pairs it sums and to work[2] the M2P to the lower order of far
  // cells (the algorithmic work behind the tree's roofline)
  unsigned long long* work = nullptr;
  // when not NULL, recorded just before and after the evaluation kernel
  cudaEvent_t eval_ev[2] = {nullptr, nullptr};
};
cudaError_t launch_tree(const TreeLaunch& T, cudaStream_t s);
size_t tree_eval_smem(int P);
// floats of one cell's multipole in the evaluation's paired layout
int tree_paired_floats(int P);
int tree_max_order();
int tree_sm_count();

// Sum a pair launch's per-chunk partials (rows 0..n_rows of leading
// dimension ld) into out[c*ld + r], the layout of a single chunk; fixed order.
cudaError_t launch_reduce_chunks(const double* part, int n_chunks, int ld, int n_rows, double* out,
                                 cudaStream_t s);
// n_grad: check points (2 N_m, monitoring points then wraps) whose gradients
// also enter v for the gradient-periodicity rows; 0 without them.
cudaError_t launch_fit(int dims, const double* part, int n_chunks, int ld, int N, int n_check,
                       int n_grad, const double* P, int nA, int nv, const double* W, int M,
                       const double* ysurf, double scale, double* v, double* A, double* cphi,
                       double* cdz, double* Q, float4* s32, double4_32a* s64, cudaStream_t s);
cudaError_t launch_assemble(const double* part, int n_chunks, int ld, const double* fpart,
                            int f_chunks, int fld, const double* self, const double* q, int N,
                            double pref, DevScalars* sc, double* forces, double* pot, double* grad,
                            double* blk_e, cudaStream_t s);


}  // namespace hsma
