// The handle behind hsma_t and the helpers the API and the request loop share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "geometry.hpp"
#include "internal.hpp"

namespace hsma {

// A device allocation that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  int ensure(size_t bytes);   // 0 or -1 (allocation failed)
  void release();
};

struct Server;  // request loop state (serve.cpp)

bool is_device_ptr(const void* ptr);
int64_t guard_violations();
int guard_selftest(void* p, size_t n, int value);
double estimate_images(const Geometry& g, int64_t N);
int choose_chunks(int tiles, int slots, double n_src, int min_len);

}  // namespace hsma

struct hsma_ctx {
  static constexpr int kEvents = 6;
  bool is_server = false;
  hsma::GeoParams gp;
  int precision = 1;
  double pref = 1.0;
  int timing = 0;
  int chunks_opt = 0;
  int tpt = 12;  // packed FP32x2 pair kernel, 2 targets per thread
  bool geo_dirty = true;
  hsma::Geometry geo;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // geometry-sized device buffers
  hsma::DevBuf d_shifts, d_check, d_P, d_W, d_ysurf, d_v, d_A, d_cphi, d_cdz, d_Q, d_s32, d_s64, d_norm;
  // N-sized device buffers
  hsma::DevBuf d_x, d_q, d_xc, d_cnt, d_blk, d_blkq, d_blkaq, d_src32, d_src64, d_tgt32, d_tgt64,
      d_part, d_fpart, d_forces, d_pot, d_grad, d_blke, d_sc, d_ioff, d_self, d_mask,
      d_red1, d_red2,  // chunk-reduced partials of the near/check and far launches
      d_src32lo, d_tgt32lo,  // FP32 rounding remainders of images and targets (precision 2)
      d_imgshift;            // shift index of each section-1 image (tree evaluation)
  hsma::DevScalars* h_sc = nullptr;  // pinned
  cudaEvent_t ev[kEvents] = {};
  double times[6] = {0, 0, 0, 0, 0, 0};
  // plan for plan_N particles
  int64_t plan_N = -1;
  int n_tgt1 = 0, tiles1 = 0, chunks1 = 1, grid1 = 1;
  int tiles2 = 0, chunks2 = 1, grid2 = 1, slots = 1;
  double ns_est = 0;
  int64_t last_N = 0;
  int last_Ns = 0;
  hsma::Server* srv = nullptr;
  // shared geometry arrays (serving): used instead of d_P, d_W, d_ysurf,
  // d_check when set; check points, W and surface points are scaled by gscale
  const double* ext_P = nullptr;
  const double* ext_W = nullptr;
  const double* ext_Y = nullptr;
  const double* ext_C = nullptr;
  double gscale = 1.0;
  // CUDA graph of the per-evaluation pipeline (prep .. assembly), valid for
  // graph_N particles under the current plan and options
  int use_graphs = 1;
  int far_series = 0;  // far field: 0 surface charges (Eq. 8), 1 the fitted series (Eq. 5)
  // tree evaluation of the near-field and check-point sums (tree.cu)
  int near_tree = 0;
  int tree_order = 10;
  int tree_L = 0;
  int tree_leaf_level = 0;   // 0: from the expected image count
  int tree_parts = 4;        // work items per 32-target task of the tree evaluation
  int tree_leaf_mode = 0;    // 0: by leaf occupancy, 1: direct leaf level, 2: leaf multipoles
  int kernels_per_eval = 0;  // kernel launches of the last enqueued evaluation
  uint64_t plan_gen = 0;     // incremented whenever the plan or its buffers change
  hsma::DevBuf d_tkey_s, d_tcnt_s, d_tstart_s, d_tcur_s, d_tord_s, d_tkey_t, d_tcnt_t, d_tstart_t, d_tcur_t,
      d_tord_t, d_tsrc, d_tpart, d_tM, d_tnorm, d_tfac;
  hsma::TreeArgs tree_args = {};
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_N = -1;
  // autotuning of the near/check launch (kernel variant, source chunks)
  int autotune = 1;
  int64_t tuned_N = -1;
  int tuned_chunks = 0;
  int part_chunks_min = 0;   // d_part holds at least this many chunks
  // pair launches: chunk partials summed inside the launch by the last CTA of
  // each tile (fused_reduce: 0 never, 1 where it pays, 2 always), items taken
  // from a counter (dynamic_schedule); fuse1 / fuse2: the choice for the
  // near/check and the far launch of the current plan
  int fused_reduce = 1;
  int dynamic_schedule = 1;
  bool fuse1 = false, fuse2 = false;
  // tree evaluation work counts (option tree_count): M2P evaluations and FP32
  // direct pairs of the last evaluation
  int tree_count = 0;
  hsma::DevBuf d_twork;
  double tree_work[3] = {0, 0, 0};
  int tree_far_order = 1;    // far cells above the leaf level to order P - 4 (P >= 8)
  cudaEvent_t tree_ev[2] = {nullptr, nullptr};   // around the tree evaluation kernel (timing mode)
  double t_tree_eval = 0;
  hsma::DevBuf d_ticket;     // per-tile counters of both launches, then two queues
  int ticket_far = 0;        // offset of the far launch's counters in d_ticket
  int ticket_queue = 0;      // offset of the two queue pairs in d_ticket
  ~hsma_ctx();
};

int hsma_ctx_init(hsma_ctx* h);
int ensure_geometry(hsma_ctx* h);
int ensure_plan(hsma_ctx* h, int64_t N);
int enqueue_eval(hsma_ctx* h, int64_t N, double* forces_dev, double* pot_dev);
int stage_prep(hsma_ctx* h, int64_t N);
hsma::PairArgs near_args(hsma_ctx* h, int64_t N);
int stage_fit(hsma_ctx* h, int64_t N);
hsma::PairArgs far_args(hsma_ctx* h, int64_t N);
int stage_assemble(hsma_ctx* h, int64_t N, double* forces_dev, double* pot_dev);
void drop_graph(hsma_ctx* h);
int mask_words(const hsma::Geometry& g);
int finish_eval(hsma_ctx* h, double* energy);
void server_shutdown(hsma_ctx* h);
int server_set_option(hsma_ctx* h, const std::string& key, double v);
int server_get_info(hsma_ctx* h, const std::string& key, double* v);
