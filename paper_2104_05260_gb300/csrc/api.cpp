// C ABI of libhsma.so: handles, options, the evaluation pipeline (Sec. 2.2 of
// the paper, in launch order) and diagnostics.  See include/hsma.h.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/hsma.h"
#include "api_internal.hpp"
#include "geometry.hpp"
#include "internal.hpp"

using hsma::DevBuf;

namespace hsma {

// Guard bands (a bounds check that needs no sanitizer): every device buffer
// is allocated kGuardBytes longer than asked and the tail is filled with
// kGuardByte.  The live buffers are kept in a process-wide table; a buffer's
// tail is compared with the pattern when it is freed and, for all live
// buffers, when the info key "guard_violations" is read.  A kernel that wrote
// past the end of its buffer shows up as a changed tail.
namespace {
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
std::mutex g_guard_mu;
std::map<void*, size_t>& guard_table() {
  static std::map<void*, size_t>* t = new std::map<void*, size_t>();   // outlives static destructors
  return *t;
}
int64_t g_guard_bad_freed = 0;

// 1 if the tail of the buffer at p (n bytes asked) differs from the pattern
int guard_changed(void* p, size_t n) {
  unsigned char buf[kGuardBytes];
  if (cudaMemcpy(buf, (char*)p + n, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return 0;   // no context left (process exit): nothing to compare
  }
  for (size_t i = 0; i < kGuardBytes; ++i)
    if (buf[i] != kGuardByte) return 1;
  return 0;
}
}  // namespace

int DevBuf::ensure(size_t bytes) {
  if (bytes <= n) return 0;
  // a buffer that has to grow grows by half again at least, so that a run of
  // slowly increasing sizes (serving slots) reallocates, and waits for the
  // device, only a few times
  if (n > 0) bytes = std::max(bytes, n + n / 2);
  release();
  if (bytes == 0) return 0;
  if (cudaMalloc(&p, bytes + kGuardBytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return -1;
  }
  if (cudaMemset((char*)p + bytes, kGuardByte, kGuardBytes) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    p = nullptr;
    return -1;
  }
  n = bytes;
  std::lock_guard<std::mutex> lk(g_guard_mu);
  guard_table()[p] = n;
  return 0;
}

void DevBuf::release() {
  if (p) {
    // the buffer's last users may still be running on a non-blocking stream
    if (cudaDeviceSynchronize() != cudaSuccess) cudaGetLastError();
    const int bad = guard_changed(p, n);
    {
      std::lock_guard<std::mutex> lk(g_guard_mu);
      guard_table().erase(p);
      g_guard_bad_freed += bad;
    }
    cudaFree(p);
  }
  p = nullptr;
  n = 0;
}

// Buffers, live or freed, whose guard band has been written.
int64_t guard_violations() {
  if (cudaDeviceSynchronize() != cudaSuccess) cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_guard_mu);
  int64_t bad = g_guard_bad_freed;
  for (const auto& e : guard_table()) bad += guard_changed(e.first, e.second);
  return bad;
}

// Write one byte into (value 1) or restore (value 0) the guard band of the
// buffer at p, n bytes long: it lies inside the allocation, so this is an
// ordinary in-bounds write.  It exists so that a test can see the check work.
int guard_selftest(void* p, size_t n, int value) {
  if (!p) return -1;
  if (cudaMemset((char*)p + n, value ? 0x00 : kGuardByte, 1) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Expected number of images in B, for planning only (the exact count is made
// on the device).  3D: sphere volume over cell volume.  2D: per image layer,
// the sphere's cross-section area at the layer centre over the cell area.
double estimate_images(const Geometry& g, int64_t N) {
  const double* L = g.par.box;
  const double kPi = 3.14159265358979323846;
  if (!g.par.sphere_mask) return (double)N * (double)g.shifts.size();
  if (g.par.dims == 3) {
    const double r = 4.0 * kPi / 3.0 * g.Rs * g.Rs * g.Rs / (L[0] * L[1] * L[2]);
    return (double)N * std::min<double>((double)g.shifts.size(), std::max(1.0, r));
  }
  double tot = 0;
  std::vector<double> zc;
  for (const Shift& s : g.shifts)
    if (s.sx == 0 && s.sy == 0) zc.push_back(s.zo);
  for (double z : zc) tot += std::max(0.0, kPi * (g.Rs2 - z * z) / (L[0] * L[1]));
  return (double)N * std::max(1.0, tot);
}

// Source chunks per target tile: the schedule has tiles*chunks equal-cost
// items spread over `slots` resident CTAs; pick the count that fills the last
// wave best while keeping chunks long enough to amortise their partials.
int choose_chunks(int tiles, int slots, double n_src, int min_len) {
  int best = 1;
  double best_eff = -1;
  for (int S = 1; S <= 512; ++S) {
    if (S > 1 && n_src / S < min_len) break;
    const long items = (long)tiles * S;
    const long waves = (items + slots - 1) / slots;
    const double eff = (double)items / (double)(waves * slots);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = S;
    }
  }
  return best;
}

}  // namespace hsma

using namespace hsma;

static int fail(hsma_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

static int cuda_fail(hsma_ctx* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(h, e == cudaErrorMemoryAllocation ? HSMA_ERR_NOMEM : HSMA_ERR_CUDA, m);
}

hsma_ctx::~hsma_ctx() {
  for (DevBuf* b : {&d_shifts, &d_check, &d_P, &d_W, &d_ysurf, &d_v, &d_A, &d_cphi, &d_cdz, &d_Q,
                    &d_s32, &d_s64, &d_x, &d_q, &d_xc, &d_cnt, &d_blk, &d_blkq, &d_blkaq, &d_src32,
                    &d_src64, &d_tgt32, &d_tgt64, &d_part, &d_fpart, &d_forces, &d_pot, &d_grad, &d_ticket, &d_twork,
                    &d_blke, &d_sc, &d_ioff, &d_self, &d_mask, &d_norm, &d_red1, &d_red2, &d_tkey_s,
                    &d_tcnt_s, &d_tstart_s, &d_tcur_s, &d_tord_s, &d_tkey_t, &d_tcnt_t, &d_tstart_t, &d_tcur_t,
                    &d_tord_t, &d_tsrc, &d_tpart, &d_tM, &d_tnorm, &d_tfac, &d_src32lo, &d_tgt32lo,
                    &d_imgshift})
    b->release();
  if (gexec) cudaGraphExecDestroy(gexec);
  if (h_sc) cudaFreeHost(h_sc);
  for (int i = 0; i < hsma_ctx::kEvents; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  for (cudaEvent_t e : tree_ev)
    if (e) cudaEventDestroy(e);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

int hsma_ctx_init(hsma_ctx* h) {
  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
  h->own_stream = true;
  e = cudaMallocHost((void**)&h->h_sc, sizeof(DevScalars));
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMallocHost");
  for (int i = 0; i < hsma_ctx::kEvents; ++i) {
    e = cudaEventCreate(&h->ev[i]);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
  }
  if (h->d_sc.ensure(sizeof(DevScalars))) return fail(h, HSMA_ERR_NOMEM, "device scalars");
  return HSMA_OK;
}

// Build and upload the geometry if an option changed since the last build.
int ensure_geometry(hsma_ctx* h) {
  if (!h->geo_dirty) return HSMA_OK;
  std::string err;
  int rc = build_geometry(h->gp, &h->geo, &err);
  if (rc) return fail(h, rc, err);
  const Geometry& g = h->geo;
  std::vector<double> sh(g.shifts.size() * 5);
  for (size_t i = 0; i < g.shifts.size(); ++i) {
    sh[5 * i] = g.shifts[i].sx;
    sh[5 * i + 1] = g.shifts[i].sy;
    sh[5 * i + 2] = g.shifts[i].zs;
    sh[5 * i + 3] = g.shifts[i].zo;
    sh[5 * i + 4] = g.shifts[i].f;
  }
  // normalisation table of the direct series far field (k_far_series)
  const int p = g.par.p;
  std::vector<double> norm((size_t)(p + 1) * (p + 1), 0.0);
  for (int n = 0; n <= p; ++n)
    for (int m = 0; m <= n; ++m) {
      double ratio = 1.0;  // (n-m)!/(n+m)!
      for (int k = n - m + 1; k <= n + m; ++k) ratio /= k;
      double c = std::sqrt((2 * n + 1) / (4.0 * 3.14159265358979323846) * ratio);
      if (m > 0) {
        c *= std::sqrt(2.0);
        for (int k = 2 * m - 1; k > 1; k -= 2) c *= k;
      }
      norm[(size_t)n * (p + 1) + m] = c;
    }
  struct Up { DevBuf* b; const void* src; size_t bytes; };
  const Up ups[] = {
      {&h->d_norm, norm.data(), norm.size() * 8},
      {&h->d_shifts, sh.data(), sh.size() * 8},
      {&h->d_check, g.check_pts.data(), g.check_pts.size() * 8},
      {&h->d_P, g.P.data(), g.P.size() * 8},
      {&h->d_W, g.W.data(), g.W.size() * 8},
      {&h->d_ysurf, g.ysurf.data(), g.ysurf.size() * 8},
  };
  for (const Up& u : ups) {
    if (u.b->ensure(u.bytes)) return fail(h, HSMA_ERR_NOMEM, "geometry upload");
    cudaError_t e = cudaMemcpyAsync(u.b->p, u.src, u.bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "geometry upload");
  }
  const size_t M = g.par.M;
  if (h->d_v.ensure((size_t)g.nv * 8) || h->d_A.ensure((size_t)g.nA * 8) ||
      h->d_cphi.ensure((size_t)g.n_check * 8) || h->d_cdz.ensure((size_t)g.n_check * 8) ||
      h->d_Q.ensure(M * 8) || h->d_s32.ensure(M * 16) || h->d_s64.ensure(M * 32))
    return fail(h, HSMA_ERR_NOMEM, "geometry buffers");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "geometry upload");
  h->geo_dirty = false;
  h->plan_N = -1;
  h->tuned_N = -1;
  h->tuned_chunks = 0;
  return HSMA_OK;
}

void drop_graph(hsma_ctx* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  h->graph_N = -1;
}

// Tree plan: leaf level from the expected image count (about 32 images per
// occupied leaf; the sphere fills 52 % of the root cube), buffers, the
// normalisation tables of the expansion.
static int plan_tree(hsma_ctx* h, size_t n, size_t nt, size_t simg) {
  const Geometry& g = h->geo;
  const int P = h->tree_order;
  // images fill the sphere B (52 % of its cube) or, unmasked, the whole cube
  const double per_leaf = h->ns_est / (32.0 * (g.par.sphere_mask ? 0.52 : 1.0));
  int L = (int)std::floor(std::log(std::max(per_leaf, 1.0)) / std::log(8.0));
  if (h->tree_leaf_level > 0) L = h->tree_leaf_level;
  L = std::max(2, std::min(6, L));
  const size_t nleaf = (size_t)1 << (3 * L);
  const int nc = (P + 1) * (P + 1);
  // root cube: the sphere B, or, for the unmasked near set, every image of
  // the shift table (sources must lie inside their cells for the expansions)
  double half = g.Rs;
  if (!g.par.sphere_mask) {
    half = 0.0;
    for (const Shift& sh : g.shifts) {
      half = std::max(half, std::fabs(sh.sx) + 0.5 * g.par.box[0]);
      half = std::max(half, std::fabs(sh.sy) + 0.5 * g.par.box[1]);
      half = std::max(half, std::fabs(sh.zo) + 0.5 * g.par.box[2]);
    }
    half *= 1.0 + 1e-6;
  }
  TreeArgs& t = h->tree_args;
  t.L = L;
  t.P = P;
  // the finest level summed directly when its leaves are sparse: about 48
  // images per occupied leaf or fewer (measured at 35 and 92 images a leaf:
  // direct 3.9 ms against 4.4 ms; leaf multipoles 10.4 ms against 12.0 ms).
  // The images fill the sphere B, in 2D only within the z-extent of the image
  // layers (a slab of half-thickness hz through it), or, unmasked, the cube.
  double frac = 1.0;
  if (g.par.sphere_mask) {
    double hz = half;
    if (g.par.dims == 2) {
      double zmax = 0.0;
      for (const Shift& sh : g.shifts) zmax = std::max(zmax, std::fabs(sh.zo) + 0.5 * g.par.box[2]);
      hz = std::min(half, zmax);
    }
    frac = 3.14159265358979323846 * (2.0 * hz * half * half - 2.0 * hz * hz * hz / 3.0) / (8.0 * half * half * half);
  }
  const double occupied = h->ns_est / (frac * (double)((size_t)1 << (3 * L)));
  t.direct_leaf = h->tree_leaf_mode == 1 ? 1 : h->tree_leaf_mode == 2 ? 0 : (occupied <= 48.0 ? 1 : 0);
  // listed cells at least sqrt(8) cell widths from the target's cell: order
  // P - 4.  A cell of half-diagonal 0.866 w seen from anywhere in a cell at
  // centre distance D converges with ratio 0.866 / (D - 0.866); the nearest
  // listed cells (D = 2) give 0.764, whose P + 1 = 11th power is 0.05, and
  // D = sqrt(8) gives 0.441, whose 7th power is 0.003: the truncation bound
  // of every far cell stays well below that of the nearest cells
  t.far_d2 = h->tree_far_order ? 8 : 0;
  t.Rs = (float)half;
  t.D = (float)(2.0 * half);
  t.inv_wL = (float)((double)(1 << L) / (2.0 * half));
  size_t off = 0;
  for (int l = 0; l < 8; ++l) {
    t.moff[l] = (int)off;
    if (l >= 2 && l <= L) off += ((size_t)1 << (3 * l)) * tree_paired_floats(P);
  }
  std::vector<float> norm(nc), fac(nc);
  for (int nn = 0; nn <= P; ++nn)
    for (int m = 0; m <= nn; ++m) {
      double ratio = 1.0;
      for (int k = nn - m + 1; k <= nn + m; ++k) ratio /= k;
      double c = std::sqrt((2 * nn + 1) / (4.0 * 3.14159265358979323846) * ratio);
      if (m > 0) {
        c *= std::sqrt(2.0);
        for (int k = 2 * m - 1; k > 1; k -= 2) c *= k;
      }
      norm[nn * (P + 1) + m] = (float)c;
      // the evaluation has no norm; its recursion variable is U_nm / K_nm with
      // K_nm = prod_{k=m+1..nn} (2k-1)/(k-m), so the stored multipole carries K_nm
      double K = 1.0;
      for (int k = m + 1; k <= nn; ++k) K *= (2.0 * k - 1.0) / (double)(k - m);
      const double f = 4.0 * 3.14159265358979323846 / (2 * nn + 1) * c * c * K;
      fac[nn * nn + nn + m] = (float)f;
      fac[nn * nn + nn - m] = (float)f;
    }
  const bool bad = h->d_tkey_s.ensure(simg * 4) || h->d_tord_s.ensure(simg * 4) || h->d_tsrc.ensure(simg * 16) ||
                   h->d_imgshift.ensure(simg * 4) ||
                   h->d_tcnt_s.ensure(nleaf * 4) || h->d_tcur_s.ensure(nleaf * 4) ||
                   h->d_tstart_s.ensure((nleaf + 1) * 4) || h->d_tkey_t.ensure(nt * 4) ||
                   h->d_tord_t.ensure(nt * 4) || h->d_tcnt_t.ensure(nleaf * 4) || h->d_tcur_t.ensure(nleaf * 4) ||
                   h->d_tstart_t.ensure((nleaf + 1) * 4) || h->d_tpart.ensure(std::max(nleaf * nc, (size_t)h->tree_parts * 4 * nt) * 8) ||
                   h->d_tM.ensure(off * 4) || h->d_tnorm.ensure((size_t)nc * 4) || h->d_tfac.ensure((size_t)nc * 4);
  if (bad) return fail(h, HSMA_ERR_NOMEM, "tree buffers");
  cudaError_t e = cudaMemcpy(h->d_tnorm.p, norm.data(), (size_t)nc * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tfac.p, fac.data(), (size_t)nc * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "tree tables");
  t.norm = (const float*)h->d_tnorm.p;
  t.fac = (const float*)h->d_tfac.p;
  h->tree_L = L;
  (void)n;
  return HSMA_OK;
}

static int launch_near_tree(hsma_ctx* h, int64_t N) {
  TreeLaunch T;
  T.t = h->tree_args;
  T.src = (const float4*)h->d_src32.p;
  T.sc = (const DevScalars*)h->d_sc.p;
  T.tgt = (const float4*)h->d_tgt32.p;
  T.n_tgt = h->n_tgt1;
  T.n_ions = (int)N;
  T.src_key = (int*)h->d_tkey_s.p;
  T.src_count = (int*)h->d_tcnt_s.p;
  T.src_start = (int*)h->d_tstart_s.p;
  T.src_cursor = (int*)h->d_tcur_s.p;
  T.src_order = (int*)h->d_tord_s.p;
  T.tgt_key = (int*)h->d_tkey_t.p;
  T.tgt_count = (int*)h->d_tcnt_t.p;
  T.tgt_start = (int*)h->d_tstart_t.p;
  T.tgt_cursor = (int*)h->d_tcur_t.p;
  T.tgt_order = (int*)h->d_tord_t.p;
  T.src_sorted = (float4*)h->d_tsrc.p;
  T.part = (double*)h->d_tpart.p;
  T.M = (float*)h->d_tM.p;
  T.out = (double*)h->d_red1.p;
  T.ld = h->n_tgt1;
  T.parts = h->tree_parts;
  T.out_parts = (double*)h->d_tpart.p;     // the P2M partials are consumed before the evaluation
  T.xc = (const double*)h->d_xc.p;
  T.q = (const double*)h->d_q.p;
  T.shifts = (const double*)h->d_shifts.p;
  T.ioff = (const int*)h->d_ioff.p;
  T.icnt = (const int*)h->d_cnt.p;
  T.img_shift = (const int*)h->d_imgshift.p;
  if (h->tree_count && h->d_twork.p) {   // allocated when the option is set (this may run under capture)
    if (cudaMemsetAsync(h->d_twork.p, 0, 3 * sizeof(unsigned long long), h->stream) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, HSMA_ERR_CUDA, "tree work counters");
    }
    T.work = (unsigned long long*)h->d_twork.p;
  }
  if (h->timing) {
    for (cudaEvent_t& ev : h->tree_ev)
      if (!ev && cudaEventCreate(&ev) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, HSMA_ERR_CUDA, "tree timing events");
      }
    T.eval_ev[0] = h->tree_ev[0];
    T.eval_ev[1] = h->tree_ev[1];
  }
  cudaError_t e = launch_tree(T, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "tree launch");
  return HSMA_OK;
}

int mask_words(const Geometry& g) { return std::max<int>(1, ((int)g.shifts.size() - 1 + 31) / 32); }

// Pair-kernel variant code for the handle's precision: FP64 has one; the
// exact-difference path (precision 2) runs the hi/lo variants 32, 34 or 44.
static int eff_tpt(const hsma_ctx* h) {
  if (h->precision == 0) return 1;
  if (h->precision == 2) return (h->tpt == 32 || h->tpt == 34 || h->tpt == 44) ? h->tpt : 34;
  return h->tpt;
}

// Whether a pair launch sums its own chunk partials (option fused_reduce).
// In the fused form one CTA sums a tile's partials after its last chunk: about
// n_chunks x tile_targets / 1024 us of L2 round trips that a short launch
// cannot hide (the last tiles' sums form its tail), while the separate
// reduction spreads the same reads over the whole GPU.  With the default
// (1) the launch fuses when that estimate is under a tenth of the launch's
// pair time at the kernel's rate (pairs x 13 FP32 operations at about
// 30e12 a second): at N = 3,000 with 108 chunks the fused form made an
// MD step 30 % slower, at N >= 1e5 it saves DRAM traffic for a few tenths
// of a percent of time.  Both forms give bitwise the same sums.
static bool use_fused(const hsma_ctx* h, int n_chunks, int tile_targets, double pairs) {
  if (h->fused_reduce != 1) return h->fused_reduce == 2;
  const double reduce_us = (double)n_chunks * tile_targets / 1024.0;
  const double launch_us = pairs * 13.0 / 30e12 * 1e6;
  return reduce_us < 0.1 * launch_us;
}

// Launch plan and buffers for N particles.
int ensure_plan(hsma_ctx* h, int64_t N) {
  if (h->plan_N == N) return HSMA_OK;
  const Geometry& g = h->geo;
  // image and target indices are 32-bit on the device: every image of the
  // shift table (the most B can hold) and every target must stay below 2^31
  if ((double)N * (double)g.shifts.size() + (double)g.n_check >= 2147483647.0)
    return fail(h, HSMA_ERR_ARG, "N = " + std::to_string(N) + " times " + std::to_string(g.shifts.size()) +
                                     " image shifts exceeds the 32-bit index range");
  const int prec = h->precision;
  const int tpt = eff_tpt(h);
  const int tile = pair_tile_targets(prec, tpt);
  const int slots = pair_slots(prec, tpt);
  h->n_tgt1 = (int)N + g.n_check;
  h->tiles1 = (h->n_tgt1 + tile - 1) / tile;
  h->ns_est = estimate_images(g, N);
  h->chunks1 = h->chunks_opt > 0 ? h->chunks_opt
                                  : choose_chunks(h->tiles1, slots, h->ns_est, prec == 0 ? 128 : 256);
  if (h->tuned_chunks > 0 && h->tuned_N == N) h->chunks1 = h->tuned_chunks;
  h->grid1 = (int)std::min<long>((long)h->tiles1 * h->chunks1, slots);
  h->tiles2 = ((int)N + tile - 1) / tile;
  h->chunks2 = choose_chunks(h->tiles2, slots, g.par.M, 128);
  h->grid2 = (int)std::min<long>((long)h->tiles2 * h->chunks2, slots);
  h->slots = slots;
  h->fuse1 = use_fused(h, h->chunks1, tile, (double)h->n_tgt1 * (double)h->ns_est);
  h->fuse2 = use_fused(h, h->chunks2, tile, (double)N * (double)g.par.M);
  const size_t n = (size_t)N, nt = (size_t)h->n_tgt1;
  const size_t nblk = (size_t)prep_blocks((int)n, g.n_check) + (n + 255) / 256;
  const size_t simg = n * g.shifts.size();  // upper bound on images in B
  if (h->d_mask.ensure(n * 4 * (size_t)mask_words(g))) return fail(h, HSMA_ERR_NOMEM, "mask buffer");
  bool bad = h->d_x.ensure(n * 24) || h->d_q.ensure(n * 8) || h->d_xc.ensure(n * 24) ||
             h->d_cnt.ensure(n * 4) || h->d_blk.ensure(nblk * 4) || h->d_blkq.ensure(nblk * 8) ||
             h->d_blkaq.ensure(nblk * 8) || h->d_forces.ensure(n * 24) || h->d_pot.ensure(n * 8) ||
             h->d_grad.ensure(n * 24) || h->d_blke.ensure(nblk * 8) ||
             h->d_part.ensure((size_t)std::max(h->chunks1, h->part_chunks_min) * 4 * nt * 8) ||
             h->d_fpart.ensure((size_t)h->chunks2 * 4 * n * 8) || h->d_red1.ensure(4 * nt * 8) ||
             h->d_red2.ensure(4 * n * 8);
  if (prec == 0)
    bad = bad || h->d_src64.ensure(simg * 32) || h->d_tgt64.ensure(nt * 32);
  else
    bad = bad || h->d_src32.ensure(simg * 16) || h->d_tgt32.ensure(nt * 16) ||
          h->d_ioff.ensure(n * 4) || h->d_self.ensure(n * 32);
  if (prec == 2) bad = bad || h->d_src32lo.ensure(simg * 16) || h->d_tgt32lo.ensure(nt * 16);
  // tile counters of the fused reduction, for the smallest tile any variant
  // uses (256 targets), then the two launches' queue counters; all zero
  // between launches
  h->ticket_far = (int)(nt / 256 + 1);
  h->ticket_queue = h->ticket_far + (int)(n / 256 + 1);
  const size_t nticket = (size_t)h->ticket_queue + 4;
  if (h->fused_reduce || h->dynamic_schedule) {
    bad = bad || h->d_ticket.ensure(nticket * 4);
    if (!bad && cudaMemsetAsync(h->d_ticket.p, 0, nticket * 4, h->stream) != cudaSuccess) {
      cudaGetLastError();
      bad = true;
    }
  }
  if (bad) return fail(h, HSMA_ERR_NOMEM, "device buffers for N = " + std::to_string(N));
  if (h->near_tree) {
    if (prec != 1) return fail(h, HSMA_ERR_ARG, "near_tree needs precision 1 (FP32 pair arithmetic)");
    int rc = plan_tree(h, n, nt, simg);
    if (rc) return rc;
  }
  h->plan_N = N;
  h->plan_gen++;
  drop_graph(h);
  return HSMA_OK;
}

// Geometry arrays on the device: the handle's own, or a shared unit-box
// geometry (serving) that the kernels scale by h->gscale.
static const double* geo_P(hsma_ctx* h) { return h->ext_P ? h->ext_P : (const double*)h->d_P.p; }
static const double* geo_W(hsma_ctx* h) { return h->ext_W ? h->ext_W : (const double*)h->d_W.p; }
static const double* geo_Y(hsma_ctx* h) { return h->ext_Y ? h->ext_Y : (const double*)h->d_ysurf.p; }
static const double* geo_C(hsma_ctx* h) { return h->ext_C ? h->ext_C : (const double*)h->d_check.p; }

// Stage 1: wrap/centre, sphere membership, image list, check-point targets
// (and on the FP32 path each ion's own images in FP64).
int stage_prep(hsma_ctx* h, int64_t N) {
  const Geometry& g = h->geo;
  const int prec = h->precision;
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->d_sc.p, 0, sizeof(DevScalars), s);
  PrepArgs a;
  a.x = (const double*)h->d_x.p;
  a.q = (const double*)h->d_q.p;
  a.N = (int)N;
  a.dims = g.par.dims;
  for (int d = 0; d < 3; ++d) a.L[d] = g.par.box[d];
  // unmasked near set: every image of the table passes r2 < +inf
  a.Rs2 = g.par.sphere_mask ? g.Rs2 : HUGE_VAL;
  a.shifts = (const double*)h->d_shifts.p;
  a.n_shift = (int)g.shifts.size();
  a.check_pts = geo_C(h);
  a.n_check = g.n_check;
  a.cscale = h->gscale;
  a.xc = (double*)h->d_xc.p;
  a.cnt = (int*)h->d_cnt.p;
  a.blk = (int*)h->d_blk.p;
  a.blk_q = (double*)h->d_blkq.p;
  a.blk_aq = (double*)h->d_blkaq.p;
  a.sc = (DevScalars*)h->d_sc.p;
  a.src32 = prec ? (float4*)h->d_src32.p : nullptr;
  a.tgt32 = prec ? (float4*)h->d_tgt32.p : nullptr;
  a.src32lo = prec == 2 ? (float4*)h->d_src32lo.p : nullptr;
  a.tgt32lo = prec == 2 ? (float4*)h->d_tgt32lo.p : nullptr;
  a.src64 = prec ? nullptr : (double4_32a*)h->d_src64.p;
  a.tgt64 = prec ? nullptr : (double4_32a*)h->d_tgt64.p;
  a.ioff = prec ? (int*)h->d_ioff.p : nullptr;
  a.mask = (unsigned*)h->d_mask.p;
  a.mwords = mask_words(g);
  // FP32 path: each ion's own shifted images are summed in FP64 by the prep
  // kernels and skipped by the FP32 pair kernel
  a.self = prec ? (double*)h->d_self.p : nullptr;
  // the tree sums an ion's own images in FP64 from their shift indices
  a.img_shift = (prec && h->near_tree) ? (int*)h->d_imgshift.p : nullptr;
  const int nblk = (int)((N + 255) / 256);
  cudaError_t e = launch_prep(a, nblk, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "prep launch");
  return HSMA_OK;
}

// Stage 2 arguments: near field + check points (targets: ions then check
// points; sources: the images in B, counted on the device).
PairArgs near_args(hsma_ctx* h, int64_t N) {
  const int prec = h->precision;
  PairArgs p1;
  p1.tgt = prec ? (const void*)h->d_tgt32.p : (const void*)h->d_tgt64.p;
  p1.n_tgt = h->n_tgt1;
  p1.src = prec ? (const void*)h->d_src32.p : (const void*)h->d_src64.p;
  p1.n_src = 0;
  p1.sc = (const DevScalars*)h->d_sc.p;
  p1.n_diag = (int)N;
  p1.n_tiles = h->tiles1;
  p1.n_chunks = h->chunks1;
  p1.part = (double*)h->d_part.p;
  p1.ld = h->n_tgt1;
  p1.ioff = prec ? (const int*)h->d_ioff.p : nullptr;
  p1.icnt = prec ? (const int*)h->d_cnt.p : nullptr;
  p1.src_lo = prec == 2 ? (const float4*)h->d_src32lo.p : nullptr;
  p1.tgt_lo = prec == 2 ? (const float4*)h->d_tgt32lo.p : nullptr;
  if (h->fuse1) {
    p1.red = (double*)h->d_red1.p;
    p1.ticket = (int*)h->d_ticket.p;
  }
  if (h->dynamic_schedule) p1.queue = (int*)h->d_ticket.p + h->ticket_queue;
  return p1;
}

// Stage 3: combine the check-point partials, A = P v, Q = W A (FP64).
int stage_fit(hsma_ctx* h, int64_t N) {
  const Geometry& g = h->geo;
  const int prec = h->precision;
  // the near/check partials summed over chunks once; the fit and the
  // assembly read the single row set
  cudaError_t e = cudaSuccess;
  if (!h->near_tree && !h->fuse1)   // the tree and the fused launch write one row set
    e = launch_reduce_chunks((const double*)h->d_part.p, h->chunks1, h->n_tgt1, h->n_tgt1,
                             (double*)h->d_red1.p, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "chunk reduction");
  e = launch_fit(g.par.dims, (const double*)h->d_red1.p, 1, h->n_tgt1, (int)N,
                             g.n_check, g.par.grad_rows ? 2 * g.n_mon : 0, geo_P(h), g.nA, g.nv, geo_W(h), g.par.M, geo_Y(h), h->gscale,
                             (double*)h->d_v.p, (double*)h->d_A.p, (double*)h->d_cphi.p,
                             (double*)h->d_cdz.p, (double*)h->d_Q.p,
                             prec ? (float4*)h->d_s32.p : nullptr,
                             prec ? nullptr : (double4_32a*)h->d_s64.p, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "fit launch");
  return HSMA_OK;
}

// Stage 4 arguments: far field (targets: ions; sources: surface charges).
PairArgs far_args(hsma_ctx* h, int64_t N) {
  const int prec = h->precision;
  PairArgs p2;
  p2.tgt = prec ? (const void*)h->d_tgt32.p : (const void*)h->d_tgt64.p;
  p2.n_tgt = (int)N;
  p2.src = prec ? (const void*)h->d_s32.p : (const void*)h->d_s64.p;
  p2.n_src = h->geo.par.M;
  p2.sc = nullptr;
  p2.n_diag = 0;
  p2.n_tiles = h->tiles2;
  p2.n_chunks = h->chunks2;
  p2.part = (double*)h->d_fpart.p;
  p2.ld = (int)N;
  p2.tgt_lo = prec == 2 ? (const float4*)h->d_tgt32lo.p : nullptr;   // surface charges: no lo part
  if (h->fuse2) {
    p2.red = (double*)h->d_red2.p;
    p2.ticket = (int*)h->d_ticket.p + h->ticket_far;
  }
  if (h->dynamic_schedule) p2.queue = (int*)h->d_ticket.p + h->ticket_queue + 2;
  return p2;
}

// Stage 5: potentials, forces, energy; scalars back to pinned host memory.
int stage_assemble(hsma_ctx* h, int64_t N, double* forces_dev, double* pot_dev) {
  const int prec = h->precision;
  // the far field's single row set: the series writes it, the fused launch
  // sums its chunks itself, one chunk needs no sum
  const bool far_one = h->far_series || (!h->fuse2 && h->chunks2 == 1);
  const bool far_sum = !h->far_series && !h->fuse2 && h->chunks2 > 1;
  cudaError_t e = cudaSuccess;
  if (far_sum)
    e = launch_reduce_chunks((const double*)h->d_fpart.p, h->chunks2, (int)N, (int)N, (double*)h->d_red2.p,
                             h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "chunk reduction");
  e = launch_assemble((const double*)h->d_red1.p, 1, h->n_tgt1,
                                  (const double*)(far_one ? h->d_fpart.p : h->d_red2.p), 1, (int)N,
                                  (prec && !h->near_tree) ? (const double*)h->d_self.p : nullptr,
                                  (const double*)h->d_q.p, (int)N, h->pref, (DevScalars*)h->d_sc.p,
                                  forces_dev, pot_dev, (double*)h->d_grad.p, (double*)h->d_blke.p,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_sc, h->d_sc.p, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble launch");
  return HSMA_OK;
}

// Enqueue one evaluation on h->stream; inputs already in d_x, d_q.
int enqueue_eval(hsma_ctx* h, int64_t N, double* forces_dev, double* pot_dev) {
  const int prec = h->precision;
  const int tpt = eff_tpt(h);
  cudaStream_t s = h->stream;
  const bool tm = h->timing != 0;
  if (tm) cudaEventRecord(h->ev[0], s);
  int rc = stage_prep(h, N);
  if (rc) return rc;
  if (tm) cudaEventRecord(h->ev[1], s);
  cudaError_t e = cudaSuccess;
  if (h->near_tree) {
    rc = launch_near_tree(h, N);
    if (rc) return rc;
  } else {
    e = launch_pair(prec, tpt, near_args(h, N), h->grid1, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "near/check launch");
  }
  if (tm) cudaEventRecord(h->ev[2], s);
  rc = stage_fit(h, N);
  if (rc) return rc;
  if (tm) cudaEventRecord(h->ev[3], s);
  if (h->far_series)
    e = launch_far_series(prec, prec ? (const void*)h->d_tgt32.p : (const void*)h->d_tgt64.p, (int)N,
                          (const double*)h->d_A.p, (const double*)h->d_norm.p, h->geo.par.p,
                          1.0 / (h->geo.Rc * h->gscale), (double*)h->d_fpart.p, s);
  else
    e = launch_pair(prec, tpt, far_args(h, N), h->grid2, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "far launch");
  if (tm) cudaEventRecord(h->ev[4], s);
  rc = stage_assemble(h, N, forces_dev, pot_dev);
  if (rc) return rc;
  if (tm) cudaEventRecord(h->ev[5], s);
  // kernels this pipeline launches: prep 3; near 1 and its chunk reduction
  // 1 (none when the launch sums its own chunks), or the tree's 9 binning kernels, 2 per multipole level (2..L, or
  // 2..L-1 with a direct leaf level), task count and scan, evaluation and
  // part reduction; fit 3; far 1; far reduction 1 (not with one far chunk);
  // assembly 2
  const bool far_sum = !h->far_series && !h->fuse2 && h->chunks2 > 1;
  const int m_levels = h->near_tree ? std::max(0, h->tree_L - 1 - h->tree_args.direct_leaf) : 0;
  h->kernels_per_eval =
      3 + (h->near_tree ? 13 + 2 * m_levels : (h->fuse1 ? 1 : 2)) + 3 + 1 + (far_sum ? 1 : 0) + 2;
  return HSMA_OK;
}

int finish_eval(hsma_ctx* h, double* energy) {
  const DevScalars& r = *h->h_sc;
  h->last_Ns = r.Ns;
  if (h->timing) {
    float t;
    const int pairs[6][2] = {{0, 5}, {0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}};
    for (int i = 0; i < 6; ++i) {
      if (cudaEventElapsedTime(&t, h->ev[pairs[i][0]], h->ev[pairs[i][1]]) != cudaSuccess) {
        cudaGetLastError();
        t = -1.f;
      }
      h->times[i] = t;
    }
    float tt = 0.f;
    if (h->near_tree && h->tree_ev[0] && cudaEventElapsedTime(&tt, h->tree_ev[0], h->tree_ev[1]) == cudaSuccess)
      h->t_tree_eval = tt;
    else
      cudaGetLastError();
  }
  if (h->tree_count && h->near_tree && h->d_twork.p) {
    unsigned long long w[3] = {0, 0, 0};
    if (cudaMemcpy(w, h->d_twork.p, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) cudaGetLastError();
    for (int i = 0; i < 3; ++i) h->tree_work[i] = (double)w[i];
  }
  if (r.flags & FLAG_OUT_OF_SLAB) return fail(h, HSMA_ERR_OUT_OF_SLAB, "some z outside (0, Lz)");
  if (r.flags & FLAG_NOT_NEUTRAL) return fail(h, HSMA_ERR_NOT_NEUTRAL, "system not neutral");
  if (r.flags & FLAG_TIMEOUT) return fail(h, HSMA_ERR_TIMEOUT, "device wait timed out");
  if (!std::isfinite(r.energy))
    return fail(h, HSMA_ERR_NUMERIC, "energy is not finite (a position or charge is not finite)");
  if (energy) *energy = r.energy;
  return HSMA_OK;
}

// Process-wide cache of tuned near/check launches: (dims, precision, N bucket,
// check-point bucket) -> (kernel variant, source chunks).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune;

// Time the near/check launch for each candidate (kernel variant x chunk
// count) on the real input and keep the fastest.  Inputs are in d_x, d_q.
static int tune_near(hsma_ctx* h, int64_t N) {
  const Geometry& g = h->geo;
  const int prec = h->precision;
  // keyed by N, the check-point count and the expected images per target
  // (which the sphere radius and the mask set), each in quarter-octave buckets
  const auto key = std::make_tuple(g.par.dims, prec, (int)std::lround(4.0 * std::log2((double)N)),
                                   (int)std::lround(4.0 * std::log2((double)g.n_check + 1.0)),
                                   (int)std::lround(4.0 * std::log2(h->ns_est / (double)N + 1.0)));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      if (prec) h->tpt = it->second.first;   // (the cache key holds the precision)
      h->tuned_chunks = std::max(1, it->second.second);
      h->tuned_N = N;
      h->plan_N = -1;
      return ensure_plan(h, N);
    }
  }
  std::vector<int> tpts = prec == 2 ? std::vector<int>{32, 34, 44}
                         : prec ? std::vector<int>{12, 14, 24, 1} : std::vector<int>{1};
  struct Cand { int tpt, chunks; float ms; };
  std::vector<Cand> cands;
  int maxc = 1;
  for (int tpt : tpts) {
    const int tile = pair_tile_targets(prec, tpt);
    const int tiles = (h->n_tgt1 + tile - 1) / tile;
    const int s0 = choose_chunks(tiles, pair_slots(prec, tpt), h->ns_est, prec == 0 ? 128 : 256);
    for (int c : {s0, std::max(1, s0 / 2), 2 * s0, 4 * s0}) {
      bool dup = false;
      for (const Cand& k : cands) dup |= (k.tpt == tpt && k.chunks == c);
      if (!dup) cands.push_back({tpt, c, 0.f});
      maxc = std::max(maxc, c);
    }
  }
  h->part_chunks_min = maxc;
  h->plan_N = -1;
  int rc = ensure_plan(h, N);
  if (rc) return rc;
  rc = stage_prep(h, N);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  for (size_t ci = 0; ci <= cands.size(); ++ci) {
    Cand& c = cands[ci == 0 ? 0 : ci - 1];       // the first launch is an untimed warm-up
    PairArgs a = near_args(h, N);
    const int tile = pair_tile_targets(prec, c.tpt);
    a.n_tiles = (h->n_tgt1 + tile - 1) / tile;
    a.n_chunks = c.chunks;
    // each candidate with the reduction form it would run with
    const bool fused = use_fused(h, c.chunks, tile, (double)h->n_tgt1 * (double)h->ns_est);
    a.red = fused ? (double*)h->d_red1.p : nullptr;
    a.ticket = fused ? (int*)h->d_ticket.p : nullptr;
    const int grid = (int)std::min<long>((long)a.n_tiles * a.n_chunks, pair_slots(prec, c.tpt));
    // timed with the chunk reduction that consumes its partials: more
    // chunks fill the GPU at small N but cost partial traffic
    cudaEventRecord(h->ev[0], s);
    cudaError_t e = launch_pair(prec, prec ? c.tpt : 1, a, grid, s);
    if (e == cudaSuccess && !fused)
      e = launch_reduce_chunks(a.part, a.n_chunks, a.ld, h->n_tgt1, (double*)h->d_red1.p, s);
    cudaEventRecord(h->ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->ev[1]);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    if (ci > 0) cudaEventElapsedTime(&c.ms, h->ev[0], h->ev[1]);
  }
  // The fastest plan, except that plans within 2 % of it (the spread of one
  // timed launch) are ranked by a fixed preference, so that runs settle on
  // the same plan: the shared-memory-sum variants first, then the packed 2-
  // and 4-target ones, then the scalar one; at equal variant the chunk count
  // of the heuristic, then fewer chunks.
  float fastest = cands[0].ms;
  for (const Cand& c : cands) fastest = std::min(fastest, c.ms);
  auto rank = [&](int tpt) {
    static const int order[] = {24, 44, 12, 34, 14, 32, 1};
    for (int i = 0; i < 7; ++i)
      if (order[i] == tpt) return i;
    return 7;
  };
  const Cand* best = nullptr;
  for (const Cand& c : cands) {
    if (c.ms > 1.02f * fastest) continue;
    if (!best) {
      best = &c;
      continue;
    }
    const int rc = rank(c.tpt), rb = rank(best->tpt);
    if (rc != rb) {
      if (rc < rb) best = &c;
      continue;
    }
    const int tile = pair_tile_targets(prec, c.tpt);
    const int s0 = choose_chunks((h->n_tgt1 + tile - 1) / tile, pair_slots(prec, c.tpt), h->ns_est,
                                 prec == 0 ? 128 : 256);
    const bool c_is_s0 = c.chunks == s0, b_is_s0 = best->chunks == s0;
    if (c_is_s0 != b_is_s0 ? c_is_s0 : c.chunks < best->chunks) best = &c;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {best->tpt, best->chunks};
  }
  if (prec) h->tpt = best->tpt;
  h->tuned_chunks = best->chunks;
  h->tuned_N = N;
  h->plan_N = -1;
  return ensure_plan(h, N);
}

static int eval_impl(hsma_ctx* h, const double* x, const double* q, int64_t N, double* energy,
                     double* forces, double* potential) {
  if (!h) return HSMA_ERR_ARG;
  if (h->is_server) return fail(h, HSMA_ERR_ARG, "handle is a server; use hsma_submit");
  if (!x || !q || !energy) return fail(h, HSMA_ERR_ARG, "NULL x, q or energy");
  if (N < 1 || N > (int64_t)1 << 28) return fail(h, HSMA_ERR_ARG, "N out of range");
  int rc = ensure_geometry(h);
  if (rc) return rc;
  rc = ensure_plan(h, N);
  if (rc) return rc;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemcpyAsync(h->d_x.p, x, (size_t)N * 24, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q.p, q, (size_t)N * 8, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "input copy");
  if (h->autotune && h->chunks_opt == 0 && h->tuned_N != N && !h->near_tree) {
    rc = tune_near(h, N);
    if (rc) return rc;
  }
  const bool fdev = forces && is_device_ptr(forces);
  const bool pdev = potential && is_device_ptr(potential);
  // per-phase timing records events between the launches, so it runs unrolled
  const bool graph = h->use_graphs != 0 && h->timing == 0;
  double* fout = (graph || !fdev) ? (double*)h->d_forces.p : forces;
  double* pout = (graph || !pdev) ? (double*)h->d_pot.p : potential;
  if (graph) {
    if (!h->gexec || h->graph_N != N) {
      drop_graph(h);
      cudaGraph_t gr = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
      rc = enqueue_eval(h, N, fout, pout);
      e = cudaStreamEndCapture(s, &gr);
      if (rc) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        h->gexec = nullptr;
        return cuda_fail(h, e, "graph instantiate");
      }
      h->graph_N = N;
    }
    e = cudaGraphLaunch(h->gexec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
  } else {
    rc = enqueue_eval(h, N, fout, pout);
    if (rc) return rc;
  }
  if (forces && fout != forces) {
    e = cudaMemcpyAsync(forces, fout, (size_t)N * 24, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "force copy");
  }
  if (potential && pout != potential) {
    e = cudaMemcpyAsync(potential, pout, (size_t)N * 8, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "potential copy");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "evaluation");
  h->last_N = N;
  return finish_eval(h, energy);
}

// ---------------------------------------------------------------------------
extern "C" {

int hsma_create(const double box[3], int dims, int p, int M, double gamma_top, double gamma_bot,
                hsma_t* out) {
  if (!out || !box) return HSMA_ERR_ARG;
  *out = nullptr;
  if (dims != 2 && dims != 3) return HSMA_ERR_ARG;
  if (p < 1 || p > 40 || M < (p + 1) * (p + 1) || !geometry_size_ok(p, M, 2 * (p + 1) * (p + 1)))
    return HSMA_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0) || !std::isfinite(box[d])) return HSMA_ERR_ARG;
  if (dims == 2 && (!(std::fabs(gamma_top) <= 1) || !(std::fabs(gamma_bot) <= 1))) return HSMA_ERR_ARG;
  hsma_ctx* h = new (std::nothrow) hsma_ctx();
  if (!h) return HSMA_ERR_NOMEM;
  h->gp.dims = dims;
  for (int d = 0; d < 3; ++d) h->gp.box[d] = box[d];
  h->gp.p = p;
  h->gp.M = M;
  h->gp.lam = (dims == 3) ? 1.3 : 1.6;
  h->gp.n_monitor = 2 * (p + 1) * (p + 1);
  h->gp.gtop = (dims == 2) ? gamma_top : 0.0;
  h->gp.gbot = (dims == 2) ? gamma_bot : 0.0;
  h->gp.G = 80;
  int rc = hsma_ctx_init(h);
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return HSMA_OK;
}

int hsma_set_option(hsma_t h, const char* key, double v) {
  if (!h || !key) return HSMA_ERR_ARG;
  const std::string k(key);
  if (h->is_server) return server_set_option(h, k, v);
  if (k == "lambda") {
    if (!(v > 1.0) || !std::isfinite(v)) return fail(h, HSMA_ERR_ARG, "lambda must be > 1");
    h->gp.lam = v;
    h->geo_dirty = true;
  } else if (k == "n_monitor") {
    const int p = h->gp.p;
    if (!(v >= (p + 1) * (p + 1)) || v > 1e6) return fail(h, HSMA_ERR_ARG, "n_monitor must be >= (p+1)^2");
    h->gp.n_monitor = (int)v;
    h->geo_dirty = true;
  } else if (k == "precision") {
    if (v != 0 && v != 1 && v != 2) return fail(h, HSMA_ERR_ARG, "precision must be 0, 1 or 2");
    h->precision = (int)v;
    if (v == 1 && h->tpt >= 30) h->tpt = 12;   // back from the exact-difference variants
    h->tuned_N = -1;
    h->tuned_chunks = 0;
    h->plan_N = -1;
  } else if (k == "dtn_grid") {
    if (!(v >= 4) || v > 1024) return fail(h, HSMA_ERR_ARG, "dtn_grid must be in [4, 1024]");
    h->gp.G = (int)v;
    h->geo_dirty = true;
  } else if (k == "coulomb_prefactor") {
    if (!std::isfinite(v)) return fail(h, HSMA_ERR_ARG, "prefactor must be finite");
    h->pref = v;
    drop_graph(h);
  } else if (k == "timing") {
    h->timing = (v != 0);
    drop_graph(h);
  } else if (k == "sphere_mask") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "sphere_mask must be 0 or 1");
    h->gp.sphere_mask = (int)v;
    h->geo_dirty = true;
  } else if (k == "grad_rows") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "grad_rows must be 0 or 1");
    h->gp.grad_rows = (int)v;
    h->geo_dirty = true;
  } else if (k == "grad_weight") {
    if (!(v > 0) || !std::isfinite(v)) return fail(h, HSMA_ERR_ARG, "grad_weight must be > 0");
    h->gp.grad_weight = v;
    h->geo_dirty = true;
  } else if (k == "surface_rule") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "surface_rule must be 0 or 1");
    if (v == 1 && fibonacci_before(h->gp.M) == 0)
      return fail(h, HSMA_ERR_ARG, "surface_rule 1 needs M to be a Fibonacci number >= 13");
    h->gp.surface_rule = (int)v;
    h->geo_dirty = true;
  } else if (k == "guard_selftest") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "guard_selftest must be 0 or 1");
    if (guard_selftest(h->d_x.p, h->d_x.n, (int)v))
      return fail(h, HSMA_ERR_ARG, "guard_selftest needs an evaluation first");
  } else if (k == "near_tree") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "near_tree must be 0 or 1");
    h->near_tree = (int)v;
    h->plan_N = -1;
  } else if (k == "tree_order") {
    if (!(v >= 4) || v > tree_max_order() || std::fmod(v, 2.0) != 0.0)
      return fail(h, HSMA_ERR_ARG, "tree_order must be one of 4, 6, 8, 10, 12, 14");
    h->tree_order = (int)v;
    h->plan_N = -1;
  } else if (k == "tree_parts") {
    if (!(v >= 1) || v > 8 || std::floor(v) != v) return fail(h, HSMA_ERR_ARG, "tree_parts must be in [1, 8]");
    h->tree_parts = (int)v;
    h->plan_N = -1;
  } else if (k == "tree_leaf_mode") {
    if (v != 0 && v != 1 && v != 2) return fail(h, HSMA_ERR_ARG, "tree_leaf_mode must be 0, 1 or 2");
    h->tree_leaf_mode = (int)v;
    h->plan_N = -1;
  } else if (k == "tree_leaf_level") {
    if (!(v >= 0) || v > 6 || v == 1) return fail(h, HSMA_ERR_ARG, "tree_leaf_level must be 0 (automatic) or in [2, 6]");
    h->tree_leaf_level = (int)v;
    h->plan_N = -1;
  } else if (k == "far_field") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "far_field must be 0 (surface charges) or 1 (series)");
    h->far_series = (int)v;
    drop_graph(h);
  } else if (k == "graphs") {
    h->use_graphs = (v != 0);
    drop_graph(h);
  } else if (k == "tree_far_order") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "tree_far_order must be 0 or 1");
    h->tree_far_order = (int)v;
    h->plan_N = -1;
  } else if (k == "tree_count") {
    if (v != 0 && v != 1) return fail(h, HSMA_ERR_ARG, "tree_count must be 0 or 1");
    if (v == 1 && h->d_twork.ensure(3 * sizeof(unsigned long long)))
      return fail(h, HSMA_ERR_NOMEM, "tree work counters");
    h->tree_count = (int)v;
    drop_graph(h);
  } else if (k == "fused_reduce" || k == "dynamic_schedule") {
    if (v != 0 && v != 1 && !(v == 2 && k == "fused_reduce"))
      return fail(h, HSMA_ERR_ARG, k == "fused_reduce" ? "fused_reduce must be 0, 1 or 2" : k + " must be 0 or 1");
    (k == "fused_reduce" ? h->fused_reduce : h->dynamic_schedule) = (int)v;
    h->tuned_N = -1;
    h->tuned_chunks = 0;
    h->plan_N = -1;
    drop_graph(h);
  } else if (k == "autotune") {
    h->autotune = (v != 0);
    h->tuned_N = -1;
    h->tuned_chunks = 0;
    h->plan_N = -1;
  } else if (k == "chunks") {
    if (!(v >= 0) || v > 4096) return fail(h, HSMA_ERR_ARG, "chunks must be in [0, 4096]");
    h->chunks_opt = (int)v;
    h->tuned_N = -1;
    h->tuned_chunks = 0;
    h->plan_N = -1;
  } else if (k == "targets_per_thread") {
    if (v != 1 && v != 2 && v != 4 && v != 12 && v != 14 && v != 24 && v != 32 && v != 34 && v != 44)
      return fail(h, HSMA_ERR_ARG,
                  "targets_per_thread must be 1, 2, 4 (scalar), 12, 14, 24 (packed) or 32, 34, 44 (exact differences)");
    h->tpt = (int)v;
    h->autotune = 0;          // an explicit kernel choice turns tuning off
    h->tuned_N = -1;
    h->tuned_chunks = 0;
    h->plan_N = -1;
  } else {
    return fail(h, HSMA_ERR_ARG, "unknown option " + k);
  }
  return HSMA_OK;
}

int hsma_set_stream(hsma_t h, void* stream) {
  if (!h) return HSMA_ERR_ARG;
  if (stream) {
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->own_stream = false;
    h->stream = (cudaStream_t)stream;
  } else if (!h->own_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
    h->own_stream = true;
  }
  return HSMA_OK;
}

int hsma_eval(hsma_t h, const double* x, const double* q, int64_t N, double* energy, double* forces) {
  return eval_impl(h, x, q, N, energy, forces, nullptr);
}

int hsma_eval_ex(hsma_t h, const double* x, const double* q, int64_t N, double* energy,
                 double* forces, double* potential) {
  return eval_impl(h, x, q, N, energy, forces, potential);
}

int hsma_get_info(hsma_t h, const char* key, double* value) {
  if (!h || !key || !value) return HSMA_ERR_ARG;
  const std::string k(key);
  if (h->is_server) {
    if (server_get_info(h, k, value) != HSMA_OK) return fail(h, HSMA_ERR_ARG, "unknown server info key " + k);
    return HSMA_OK;
  }
  if (!h->is_server && (k == "Rc" || k == "Rs" || k == "n_shifts" || k == "n_check" || k == "rank")) {
    int rc = ensure_geometry(h);
    if (rc) return rc;
  }
  const Geometry& g = h->geo;
  if (k == "Rc") *value = g.Rc;
  else if (k == "Rs") *value = g.Rs;
  else if (k == "n_shifts") *value = (double)g.shifts.size();
  else if (k == "n_check") *value = g.n_check;
  else if (k == "rank") *value = g.rank;
  else if (k == "Ns") *value = h->last_Ns;
  else if (k == "t_total_ms") *value = h->times[0];
  else if (k == "t_prep_ms") *value = h->times[1];
  else if (k == "t_near_ms") *value = h->times[2];
  else if (k == "t_fit_ms") *value = h->times[3];
  else if (k == "t_far_ms") *value = h->times[4];
  else if (k == "t_assemble_ms") *value = h->times[5];
  else if (k == "chunks") *value = h->chunks1;
  else if (k == "kernel") *value = h->precision ? eff_tpt(h) : 0;
  else if (k == "far_chunks") *value = h->far_series ? 1 : h->chunks2;
  else if (k == "far_field") *value = h->far_series;
  else if (k == "tree_levels") *value = h->near_tree ? h->tree_L : 0;
  else if (k == "tree_direct_leaf") *value = h->near_tree ? h->tree_args.direct_leaf : 0;
  else if (k == "kernels_per_eval") *value = h->kernels_per_eval;
  else if (k == "t_tree_eval_ms") *value = h->t_tree_eval;
  else if (k == "tree_m2p") *value = h->tree_work[0];
  else if (k == "tree_m2p_low") *value = h->tree_work[2];
  else if (k == "tree_far_order") *value = h->tree_far_order;
  else if (k == "tree_direct_pairs") *value = h->tree_work[1];
  else if (k == "fused_reduce") *value = h->fused_reduce;
  else if (k == "fused_near") *value = h->fuse1;
  else if (k == "fused_far") *value = h->fuse2;
  else if (k == "dynamic_schedule") *value = h->dynamic_schedule;
  else if (k == "guard_violations") *value = (double)guard_violations();
  else if (k == "grid") *value = h->grid1;
  else if (k == "slots") *value = h->slots;
  else if (k == "tile_targets") *value = pair_tile_targets(h->precision, eff_tpt(h));
  else return fail(h, HSMA_ERR_ARG, "unknown info key " + k);
  return HSMA_OK;
}

int hsma_get_array(hsma_t h, const char* name, double* out, int64_t n) {
  if (!h || !name || !out) return HSMA_ERR_ARG;
  const std::string k(name);
  const Geometry& g = h->geo;
  if (h->geo_dirty) return fail(h, HSMA_ERR_ARG, "no evaluation yet");
  const void* src = nullptr;
  int64_t len = 0;
  bool host = false;
  if (k == "check_points") { src = g.check_pts.data(); len = g.n_check * 3; host = true; }
  else if (k == "surface_points") { src = g.ysurf.data(); len = (int64_t)g.par.M * 3; host = true; }
  else if (k == "check_phi") { src = h->d_cphi.p; len = g.n_check; }
  else if (k == "check_dz") { src = h->d_cdz.p; len = g.n_check; }
  else if (k == "coeffs") { src = h->d_A.p; len = g.nA; }
  else if (k == "surface_q") { src = h->d_Q.p; len = g.par.M; }
  else if (k == "grad") { src = h->d_grad.p; len = h->last_N * 3; }
  else return fail(h, HSMA_ERR_ARG, "unknown array " + k);
  if (n < len) return fail(h, HSMA_ERR_ARG, "output too small for " + k);
  if (host) {
    std::memcpy(out, src, (size_t)len * 8);
    return HSMA_OK;
  }
  cudaError_t e = cudaMemcpy(out, src, (size_t)len * 8, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(h, e, "array copy");
  return HSMA_OK;
}

void hsma_destroy(hsma_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  server_shutdown(h);
  delete h;
}

const char* hsma_last_error(hsma_t h) {
  if (!h) return "NULL handle";
  return h->err.c_str();
}

}  // extern "C"

extern "C" int hsma_geometry_array(const double box[3], int dims, int p, int M, double gamma_top,
                                   double gamma_bot, double lam, int n_monitor, int G,
                                   double grad_weight, int surface_rule, const char* name, double* out,
                                   int64_t n) {
  if (!box || !name || !out) return HSMA_ERR_ARG;
  if (dims != 2 && dims != 3) return HSMA_ERR_ARG;
  GeoParams gp;
  gp.dims = dims;
  for (int d = 0; d < 3; ++d) gp.box[d] = box[d];
  gp.p = p;
  gp.M = M;
  gp.lam = lam > 0 ? lam : (dims == 3 ? 1.3 : 1.6);
  gp.n_monitor = n_monitor > 0 ? n_monitor : 2 * (p + 1) * (p + 1);
  gp.gtop = dims == 2 ? gamma_top : 0.0;
  gp.gbot = dims == 2 ? gamma_bot : 0.0;
  gp.G = G > 0 ? G : 80;
  gp.grad_rows = grad_weight > 0 ? 1 : 0;
  if (grad_weight > 0) gp.grad_weight = grad_weight;
  gp.surface_rule = surface_rule;
  Geometry g;
  std::string err;
  const int rc = build_geometry(gp, &g, &err);
  if (rc) return rc;
  const std::string k(name);
  std::vector<double> v;
  if (k == "T") {
    if ((int64_t)M * g.nv > n) return HSMA_ERR_ARG;
    v.assign((size_t)M * g.nv, 0.0);
    for (int m = 0; m < M; ++m)
      for (int r = 0; r < g.nA; ++r) {
        const double w = g.W[(size_t)m * g.nA + r];
        const double* prow = &g.P[(size_t)r * g.nv];
        double* o = &v[(size_t)m * g.nv];
        for (int c = 0; c < g.nv; ++c) o[c] += w * prow[c];
      }
  } else if (k == "check_points") {
    v = g.check_pts;
  } else if (k == "surface_points") {
    v = g.ysurf;
  } else if (k == "shifts") {
    for (const Shift& s : g.shifts) v.insert(v.end(), {s.sx, s.sy, s.zs, s.zo, s.f});
  } else if (k == "sizes") {
    v = {(double)g.n_check, (double)g.nv, (double)g.nA, (double)g.rank, (double)g.shifts.size(),
         g.Rc, g.Rs, g.Rs2};
  } else {
    return HSMA_ERR_ARG;
  }
  if ((int64_t)v.size() > n) return HSMA_ERR_ARG;
  std::memcpy(out, v.data(), v.size() * 8);
  return HSMA_OK;
}
