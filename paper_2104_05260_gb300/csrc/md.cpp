// The MD loop of the validation workload (Sec. 4.1) on the device: each step
// is one CUDA graph replay holding the velocity-Verlet kicks and drift, the
// cell list and LJ forces (md.cu), and the HSMA electrostatics of the handle
// the loop was created with (api.cpp's per-evaluation pipeline, captured into
// the same graph).  Nothing returns to the host between steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hsma.h"
#include "api_internal.hpp"
#include "md_internal.hpp"

using hsma::DevBuf;
using hsma::MdArgs;
using hsma::MdScalars;

struct hsma_md {
  hsma_ctx* h = nullptr;
  int64_t N = 0;
  double L[3] = {0, 0, 0};
  double mass = 1, dt = 0.01, kT = 1, tdamp = 0, sigma = 1, eps = 1;
  int cap = 8;
  int n_cells = 0;
  int nc[3] = {0, 0, 0};
  DevBuf x, v, img, q, f_lj, f_c, blk_k, blk_u, sc, thermo, cells, rdf, zhist;
  int slab = 0;
  double wall_sigma = 0.5, wall_eps = 1.0;
  int zhist_bins = 100;
  long long thermo_cap = 0;
  int rdf_bins = 200;
  double rdf_rmax = 5.0;
  int rdf_every = 0;
  cudaGraphExec_t g_step = nullptr, g_rdf = nullptr;
  uint64_t plan_gen = 0;   // the electrostatics plan the loop was set up with
  std::string err;
  ~hsma_md();
};

hsma_md::~hsma_md() {
  if (g_step) cudaGraphExecDestroy(g_step);
  if (g_rdf) cudaGraphExecDestroy(g_rdf);
  for (DevBuf* b : {&x, &v, &img, &q, &f_lj, &f_c, &blk_k, &blk_u, &sc, &thermo, &cells, &rdf, &zhist})
    b->release();
}

static int md_fail(hsma_md* m, int code, const std::string& msg) {
  m->err = msg;
  return code;
}

static int md_cuda_fail(hsma_md* m, cudaError_t e, const char* where) {
  cudaGetLastError();
  return md_fail(m, e == cudaErrorMemoryAllocation ? HSMA_ERR_NOMEM : HSMA_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

static MdArgs md_args(hsma_md* m) {
  MdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.N = (int)m->N;
  for (int d = 0; d < 3; ++d) {
    a.L[d] = m->L[d];
    a.nc[d] = m->nc[d];
    a.inv_w[d] = m->nc[d] / m->L[d];
  }
  a.x = (double*)m->x.p;
  a.v = (double*)m->v.p;
  a.img = (int*)m->img.p;
  a.q = (const double*)m->q.p;
  a.f_lj = (double*)m->f_lj.p;
  a.f_c = (const double*)m->f_c.p;
  a.coul_energy = &((const hsma::DevScalars*)m->h->d_sc.p)->energy;
  a.blk_k = (double*)m->blk_k.p;
  a.blk_u = (double*)m->blk_u.p;
  a.sc = (MdScalars*)m->sc.p;
  a.thermo = (double*)m->thermo.p;
  a.thermo_cap = m->thermo_cap;
  a.cap = m->cap;
  a.cell_count = (int*)m->cells.p;
  a.cell_list = (int*)m->cells.p + m->n_cells;
  a.dt = m->dt;
  a.mass = m->mass;
  a.half_dt_m = 0.5 * m->dt / m->mass;
  a.sigma2 = m->sigma * m->sigma;
  a.eps = m->eps;
  const double rc = std::pow(2.0, 1.0 / 6.0) * m->sigma;
  a.rc2 = rc * rc;
  a.thermostat = m->tdamp > 0 ? 1 : 0;
  const double g = 3.0 * (double)m->N - 3.0;
  a.g_kT = g * m->kT;
  a.Q = g * m->kT * m->tdamp * m->tdamp;
  a.rdf = (unsigned long long*)m->rdf.p;
  a.rdf_bins = m->rdf_bins;
  a.rdf_rmax = m->rdf_rmax;
  a.slab = m->slab;
  a.wall_sigma = m->wall_sigma;
  a.wall_eps = m->wall_eps;
  a.wall_rc = std::pow(2.0, 1.0 / 6.0) * m->wall_sigma;
  a.zhist = (unsigned long long*)m->zhist.p;
  a.zhist_bins = m->zhist_bins;
  return a;
}

// Forces at the current positions: LJ (cell list) and Coulomb (HSMA).
static int enqueue_forces(hsma_md* m, const MdArgs& a) {
  hsma_ctx* h = m->h;
  cudaStream_t s = h->stream;
  cudaError_t e = hsma::md_launch_lj(a, m->n_cells, s);
  if (e != cudaSuccess) return md_cuda_fail(m, e, "LJ forces");
  e = cudaMemcpyAsync(h->d_x.p, m->x.p, (size_t)m->N * 24, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q.p, m->q.p, (size_t)m->N * 8, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return md_cuda_fail(m, e, "electrostatics input");
  const int rc = enqueue_eval(h, m->N, (double*)m->f_c.p, nullptr);
  if (rc) return md_fail(m, rc, std::string("electrostatics: ") + h->err);
  return HSMA_OK;
}

static int capture(hsma_md* m, bool with_rdf, cudaGraphExec_t* out) {
  cudaStream_t s = m->h->stream;
  const MdArgs a = md_args(m);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return md_cuda_fail(m, e, "graph capture");
  int rc = HSMA_OK;
  e = hsma::md_launch_kick_drift(a, s);
  if (e == cudaSuccess) rc = enqueue_forces(m, a);
  if (e == cudaSuccess && rc == HSMA_OK) e = hsma::md_launch_kick_finish(a, s);
  if (e == cudaSuccess && rc == HSMA_OK && with_rdf) e = hsma::md_launch_rdf(a, s);
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (rc || e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    return md_cuda_fail(m, e != cudaSuccess ? e : e2, "MD step capture");
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return md_cuda_fail(m, e, "MD graph instantiate");
  }
  return HSMA_OK;
}

static int ensure_thermo(hsma_md* m, long long rows) {
  if (rows <= m->thermo_cap) return HSMA_OK;
  if (m->thermo.ensure((size_t)rows * hsma::MD_THERMO_COLS * 8)) return md_fail(m, HSMA_ERR_NOMEM, "thermo buffer");
  m->thermo_cap = rows;
  // the graphs hold the old capacity and pointer
  if (m->g_step) cudaGraphExecDestroy(m->g_step);
  if (m->g_rdf) cudaGraphExecDestroy(m->g_rdf);
  m->g_step = m->g_rdf = nullptr;
  return HSMA_OK;
}

extern "C" {

int hsma_md_create(hsma_t h, const double* x, const double* v, const double* q, int64_t N, double mass,
                   double dt, double kT, double tdamp, double lj_sigma, double lj_eps, hsma_md_t* out) {
  if (!out) return HSMA_ERR_ARG;
  *out = nullptr;
  if (!h || h->is_server || !x || !v || !q) return HSMA_ERR_ARG;
  if (N < 2 || N > (int64_t)1 << 24) return HSMA_ERR_ARG;
  if (!(mass > 0) || !(dt > 0) || !(kT > 0) || !(lj_sigma > 0) || !(lj_eps >= 0) || !std::isfinite(tdamp))
    return HSMA_ERR_ARG;
  hsma_md* m = new (std::nothrow) hsma_md();
  if (!m) return HSMA_ERR_NOMEM;
  m->h = h;
  m->N = N;
  m->mass = mass;
  m->dt = dt;
  m->kT = kT;
  m->tdamp = tdamp > 0 ? tdamp : 0.0;
  m->sigma = lj_sigma;
  m->eps = lj_eps;
  m->slab = h->gp.dims == 2 ? 1 : 0;
  const double rc = std::pow(2.0, 1.0 / 6.0) * lj_sigma;
  for (int d = 0; d < 3; ++d) {
    m->L[d] = h->gp.box[d];
    m->nc[d] = std::max(1, (int)std::floor(m->L[d] / rc));
    // the 27-cell neighbour scheme needs 3 cells a side in periodic directions
    if (m->nc[d] < 3 && !(m->slab && d == 2)) {
      delete m;
      return HSMA_ERR_ARG;
    }
  }
  m->n_cells = m->nc[0] * m->nc[1] * m->nc[2];
  // one evaluation through the public path builds the geometry, the plan and
  // the tuning for N (and checks neutrality)
  std::vector<double> xh((size_t)N * 3), qh((size_t)N), vh((size_t)N * 3);
  cudaError_t e = cudaMemcpy(xh.data(), x, xh.size() * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(qh.data(), q, qh.size() * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(vh.data(), v, vh.size() * 8, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return HSMA_ERR_ARG;
  }
  double e0;
  int rc0 = hsma_eval(h, xh.data(), qh.data(), N, &e0, nullptr);
  if (rc0) {
    delete m;
    return rc0;
  }
  // wrap into [0, L) on the host with the kernel's rule, image counters from it
  std::vector<int> img((size_t)N * 3, 0);
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) {
      double& c = xh[3 * i + d];
      const double L = m->L[d];
      if (m->slab && d == 2) continue;   // z stays inside (0, Lz): checked by the evaluation
      double w = std::floor(c / L);
      c -= w * L;
      if (c >= L) {
        c -= L;
        w += 1.0;
      } else if (c < 0.0) {
        c += L;
        w -= 1.0;
        if (c >= L) {
          c = 0.0;
          w += 1.0;
        }
      }
      img[3 * i + d] = (int)w;
    }
  const size_t n3 = (size_t)N * 3;
  const int nb = hsma::md_blocks((int)N);
  if (m->x.ensure(n3 * 8) || m->v.ensure(n3 * 8) || m->img.ensure(n3 * 4) || m->q.ensure((size_t)N * 8) ||
      m->f_lj.ensure(n3 * 8) || m->f_c.ensure(n3 * 8) || m->blk_k.ensure((size_t)nb * 8) ||
      m->blk_u.ensure((size_t)hsma::md_lj_blocks((int)N) * 8) || m->sc.ensure(sizeof(MdScalars)) ||
      m->cells.ensure((size_t)m->n_cells * (1 + m->cap) * 4) || m->rdf.ensure((size_t)3 * m->rdf_bins * 8) ||
      m->zhist.ensure((size_t)2 * m->zhist_bins * 8) ||
      ensure_thermo(m, 1)) {
    delete m;
    return HSMA_ERR_NOMEM;
  }
  cudaStream_t s = h->stream;
  MdScalars init;
  std::memset(&init, 0, sizeof(init));
  init.vscale = 1.0;
  init.vscale_end = 1.0;
  e = cudaMemcpyAsync(m->x.p, xh.data(), n3 * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->v.p, vh.data(), n3 * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->img.p, img.data(), n3 * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->q.p, qh.data(), (size_t)N * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->sc.p, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->rdf.p, 0, (size_t)3 * m->rdf_bins * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->zhist.p, 0, (size_t)2 * m->zhist_bins * 8, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return HSMA_ERR_CUDA;
  }
  // forces at the start and the first thermostat half step
  const MdArgs a = md_args(m);
  int frc = enqueue_forces(m, a);
  if (frc == HSMA_OK) {
    e = hsma::md_launch_start(a, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) frc = HSMA_ERR_CUDA;
  }
  if (frc) {
    cudaGetLastError();
    delete m;
    return frc;
  }
  m->plan_gen = h->plan_gen;
  *out = m;
  return HSMA_OK;
}

int hsma_md_set_option(hsma_md_t m, const char* key, double v) {
  if (!m || !key) return HSMA_ERR_ARG;
  const std::string k(key);
  if (k == "rdf_every") {
    if (!(v >= 0) || v > 1e9) return md_fail(m, HSMA_ERR_ARG, "rdf_every must be >= 0");
    m->rdf_every = (int)v;
    return HSMA_OK;
  }
  if (k == "rdf_bins" || k == "rdf_rmax") {
    if (k == "rdf_bins") {
      if (!(v >= 1) || v > 100000) return md_fail(m, HSMA_ERR_ARG, "rdf_bins must be in [1, 1e5]");
      m->rdf_bins = (int)v;
      if (m->rdf.ensure((size_t)3 * m->rdf_bins * 8)) return md_fail(m, HSMA_ERR_NOMEM, "rdf buffer");
    } else {
      if (!(v > 0) || !(v <= 0.5 * std::fmin(m->L[0], std::fmin(m->L[1], m->L[2]))))
        return md_fail(m, HSMA_ERR_ARG, "rdf_rmax must be in (0, L/2]");
      m->rdf_rmax = v;
    }
    cudaError_t e = cudaMemsetAsync(m->rdf.p, 0, (size_t)3 * m->rdf_bins * 8, m->h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->zhist.p, 0, (size_t)2 * m->zhist_bins * 8, m->h->stream);
    MdScalars* d = (MdScalars*)m->sc.p;
    if (e == cudaSuccess) e = cudaMemsetAsync(&d->rdf_samples, 0, sizeof(long long), m->h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->h->stream);
    if (e != cudaSuccess) return md_cuda_fail(m, e, "rdf reset");
    if (m->g_rdf) cudaGraphExecDestroy(m->g_rdf);
    m->g_rdf = nullptr;
    return HSMA_OK;
  }
  if (k == "wall_sigma" || k == "wall_eps") {
    if (!m->slab) return md_fail(m, HSMA_ERR_ARG, k + " applies to slabs (dims 2) only");
    if (!(v > 0) || !std::isfinite(v)) return md_fail(m, HSMA_ERR_ARG, k + " must be > 0");
    if (k == "wall_sigma") m->wall_sigma = v;
    else m->wall_eps = v;
    if (m->g_step) cudaGraphExecDestroy(m->g_step);
    if (m->g_rdf) cudaGraphExecDestroy(m->g_rdf);
    m->g_step = m->g_rdf = nullptr;
    // the forces of the current positions change with the walls
    const MdArgs a = md_args(m);
    int rc = enqueue_forces(m, a);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(m->h->stream);
    if (e != cudaSuccess) return md_cuda_fail(m, e, "wall forces");
    return HSMA_OK;
  }
  if (k == "zhist_bins") {
    if (!(v >= 1) || v > 100000) return md_fail(m, HSMA_ERR_ARG, "zhist_bins must be in [1, 1e5]");
    m->zhist_bins = (int)v;
    if (m->zhist.ensure((size_t)2 * m->zhist_bins * 8)) return md_fail(m, HSMA_ERR_NOMEM, "zhist buffer");
    cudaError_t e = cudaMemsetAsync(m->zhist.p, 0, (size_t)2 * m->zhist_bins * 8, m->h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->h->stream);
    if (e != cudaSuccess) return md_cuda_fail(m, e, "zhist reset");
    if (m->g_rdf) cudaGraphExecDestroy(m->g_rdf);
    m->g_rdf = nullptr;
    return HSMA_OK;
  }
  if (k == "cell_capacity") {
    if (!(v >= 1) || v > 1024) return md_fail(m, HSMA_ERR_ARG, "cell_capacity must be in [1, 1024]");
    m->cap = (int)v;
    if (m->cells.ensure((size_t)m->n_cells * (1 + m->cap) * 4)) return md_fail(m, HSMA_ERR_NOMEM, "cells");
    if (m->g_step) cudaGraphExecDestroy(m->g_step);
    if (m->g_rdf) cudaGraphExecDestroy(m->g_rdf);
    m->g_step = m->g_rdf = nullptr;
    return HSMA_OK;
  }
  return md_fail(m, HSMA_ERR_ARG, "unknown option " + k);
}

int hsma_md_run(hsma_md_t m, int64_t steps, double* thermo) {
  if (!m) return HSMA_ERR_ARG;
  if (steps < 0 || steps > (int64_t)1 << 40) return md_fail(m, HSMA_ERR_ARG, "steps out of range");
  hsma_ctx* h = m->h;
  if (h->timing) return md_fail(m, HSMA_ERR_ARG, "the electrostatics handle has timing on");
  if (h->geo_dirty || h->plan_N != m->N || h->plan_gen != m->plan_gen)
    return md_fail(m, HSMA_ERR_ARG, "the electrostatics handle was re-planned or changed");
  int rc = ensure_thermo(m, std::max<long long>(1, steps));
  if (rc) return rc;
  if (!m->g_step && (rc = capture(m, false, &m->g_step))) return rc;
  if (m->rdf_every > 0 && !m->g_rdf && (rc = capture(m, true, &m->g_rdf))) return rc;
  cudaStream_t s = h->stream;
  MdScalars* d = (MdScalars*)m->sc.p;
  cudaError_t e = cudaMemsetAsync(&d->step, 0, sizeof(long long), s);
  for (int64_t k = 0; k < steps && e == cudaSuccess; ++k) {
    const bool rdf = m->rdf_every > 0 && (k + 1) % m->rdf_every == 0;
    e = cudaGraphLaunch(rdf ? m->g_rdf : m->g_step, s);
  }
  MdScalars hs;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, m->sc.p, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && thermo && steps > 0)
    e = cudaMemcpyAsync(thermo, m->thermo.p, (size_t)steps * hsma::MD_THERMO_COLS * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return md_cuda_fail(m, e, "MD run");
  if (hs.flags & hsma::MD_FLAG_CELL_OVERFLOW)
    return md_fail(m, HSMA_ERR_ARG, "a cell held more particles than cell_capacity");
  if (hs.flags & hsma::MD_FLAG_LEFT_SLAB)
    return md_fail(m, HSMA_ERR_OUT_OF_SLAB, "an ion left the slab (0, Lz)");
  const hsma::DevScalars& r = *h->h_sc;
  if (r.flags & hsma::FLAG_NOT_NEUTRAL) return md_fail(m, HSMA_ERR_NOT_NEUTRAL, "system not neutral");
  if (r.flags & hsma::FLAG_OUT_OF_SLAB) return md_fail(m, HSMA_ERR_OUT_OF_SLAB, "an ion left the slab (0, Lz)");
  return HSMA_OK;
}

int hsma_md_get(hsma_md_t m, const char* name, double* out, int64_t n) {
  if (!m || !name || !out) return HSMA_ERR_ARG;
  const std::string k(name);
  const int64_t N = m->N;
  cudaStream_t s = m->h->stream;
  MdScalars hs;
  cudaError_t e = cudaMemcpyAsync(&hs, m->sc.p, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return md_cuda_fail(m, e, "MD state");
  if (k == "x" || k == "v" || k == "x_unwrapped" || k == "forces") {
    if (n < 3 * N) return md_fail(m, HSMA_ERR_ARG, "output too small");
    std::vector<double> a((size_t)N * 3), b;
    const void* src = k == "v" ? m->v.p : (k == "forces" ? m->f_lj.p : m->x.p);
    e = cudaMemcpy(a.data(), src, a.size() * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && k == "forces") {
      b.resize(a.size());
      e = cudaMemcpy(b.data(), m->f_c.p, b.size() * 8, cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < a.size(); ++i) a[i] += b[i];
    }
    if (e == cudaSuccess && k == "x_unwrapped") {
      std::vector<int> img(a.size());
      e = cudaMemcpy(img.data(), m->img.p, img.size() * 4, cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < a.size(); ++i) a[i] += img[i] * m->L[i % 3];
    }
    if (e != cudaSuccess) return md_cuda_fail(m, e, "MD copy");
    if (k == "v")
      for (double& c : a) c *= hs.vscale_end;
    std::memcpy(out, a.data(), a.size() * 8);
    return HSMA_OK;
  }
  if (k == "rdf") {
    const int64_t len = 3 * (int64_t)m->rdf_bins;
    if (n < len) return md_fail(m, HSMA_ERR_ARG, "output too small");
    std::vector<unsigned long long> c((size_t)len);
    e = cudaMemcpy(c.data(), m->rdf.p, c.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return md_cuda_fail(m, e, "MD copy");
    for (int64_t i = 0; i < len; ++i) out[i] = (double)c[i];
    return HSMA_OK;
  }
  if (k == "zhist") {
    const int64_t len = 2 * (int64_t)m->zhist_bins;
    if (n < len) return md_fail(m, HSMA_ERR_ARG, "output too small");
    std::vector<unsigned long long> c((size_t)len);
    e = cudaMemcpy(c.data(), m->zhist.p, c.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return md_cuda_fail(m, e, "MD copy");
    for (int64_t i = 0; i < len; ++i) out[i] = (double)c[i];
    return HSMA_OK;
  }
  if (k == "state") {
    if (n < 6) return md_fail(m, HSMA_ERR_ARG, "output too small");
    out[0] = hs.xi;
    out[1] = hs.eta;
    out[2] = hs.last_K;
    out[3] = hs.last_U;
    out[4] = (double)hs.rdf_samples;
    out[5] = hs.vscale_end;
    return HSMA_OK;
  }
  return md_fail(m, HSMA_ERR_ARG, "unknown array " + k);
}

const char* hsma_md_last_error(hsma_md_t m) { return m ? m->err.c_str() : "null MD handle"; }

void hsma_md_destroy(hsma_md_t m) {
  if (!m) return;
  if (m->h && m->h->stream) cudaStreamSynchronize(m->h->stream);
  delete m;
}

}  // extern "C"
