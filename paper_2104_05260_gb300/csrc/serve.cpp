// Request loop for independent HSMA3D evaluations (hsma_submit / hsma_poll):
// continuous batching on one GPU.
//
// Requests queue in arrival order.  Each step of the loop retires finished
// batches, then admits queued requests while a slot, the device-memory budget
// and a batch buffer are free, and enqueues the admitted ones as one batch:
// per-request prep kernels, ONE ragged launch of the pair kernel over the
// near-field and check-point items of every request in the batch, the
// per-request FP64 fits, ONE ragged launch over their far-field items, and
// the per-request assembly and copies back.  Batches run back to back on the
// server's stream while the host keeps admitting, so requests that arrive
// while others are on the GPU join the next batch.
//
// Each request's work decomposition (target tiles, source chunks) and its
// partial-sum buffers depend only on that request, and every partial is
// combined in a fixed order, so a request's result is bitwise the same alone
// or in any mix.
//
// Geometry: everything that depends on the box only through its scale (the
// fit operator, the surface map, the check and surface points) is built once
// per (box shape, p, M) for the box divided by Lx and scaled on the device;
// the sphere radius and the image shifts are built from the actual box with
// the same FP64 operations as hsma_create's path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hsma.h"
#include "api_internal.hpp"

namespace hsma {

struct Request {
  uint64_t ticket;
  int64_t N;
  double box[3];
  int p, M;
  double* hx = nullptr;    // pinned copies of the inputs, then the forces
  double* hq = nullptr;
  double* hf = nullptr;
  double energy = 0;
  int status = HSMA_PENDING;
  std::string err;         // why the request failed (status < 0)
  size_t bytes = 0;
  int slot = -1;
};

struct UnitGeo {
  Geometry g;                       // built for (1, Ly/Lx, Lz/Lx)
  DevBuf d_P, d_W, d_Y, d_C;
};

constexpr int kBatchBufs = 8;

struct BatchBuf {
  PairArgs* h_desc = nullptr;       // pinned: near descriptors, then far
  int* h_start = nullptr;           // pinned: near starts, then far starts
  DevBuf d_desc, d_start;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request*> reqs;
};

struct Slot {
  hsma_ctx* ctx = nullptr;
  Request* req = nullptr;
  const UnitGeo* geo = nullptr;
  double box[3] = {0, 0, 0};
  double* h_shifts = nullptr;   // pinned staging of the shift table (no stream sync on upload)
  size_t h_shifts_n = 0;        // its capacity in doubles
};

struct Server {
  int precision = 1;
  double budget = 0;
  double in_use = 0;
  uint64_t next_ticket = 1;
  cudaStream_t stream = nullptr;
  int ragged_slots = 1;
  std::vector<Slot> slots;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  std::map<std::tuple<double, double, int, int>, std::unique_ptr<UnitGeo>> geos;
  BatchBuf bufs[kBatchBufs];
  // host-side fault injection (tests): the request with this ticket fails as
  // if a CUDA call had failed while it was being bound to a slot
  uint64_t inject_fail_ticket = 0;
};

static void free_request(Request* r) {
  if (r->hx) cudaFreeHost(r->hx);
  if (r->hq) cudaFreeHost(r->hq);
  if (r->hf) cudaFreeHost(r->hf);
  delete r;
}

// Device bytes one request holds in its slot (an upper bound for admission):
// inputs and per-ion arrays, images in B, targets, partial sums, outputs.
static size_t request_bytes(int64_t N, const double box[3], int p, int M, int precision) {
  const double ns = 27.0 * (double)N;   // every image of the 27 cells, the most B can hold
  const double img = precision == 1 ? 16.0 : 32.0;   // FP32 (x, y, z, q); FP64 or hi + lo
  const double nck = 4.0 * (p + 1) * (p + 1);
  const double chunks = 64.0;   // generous bound on source chunks per tile
  return (size_t)(ns * img + (N + nck) * (img + 32.0 * chunks) + N * 200.0 + (double)M * 64);
}

static const UnitGeo* unit_geometry(Server* s, const Request* r, std::string* err) {
  const double ry = r->box[1] / r->box[0], rz = r->box[2] / r->box[0];
  auto key = std::make_tuple(ry, rz, r->p, r->M);
  auto it = s->geos.find(key);
  if (it != s->geos.end()) return it->second.get();
  std::unique_ptr<UnitGeo> u(new UnitGeo());
  GeoParams gp;
  gp.dims = 3;
  gp.box[0] = 1.0;
  gp.box[1] = ry;
  gp.box[2] = rz;
  gp.p = r->p;
  gp.M = r->M;
  gp.lam = 1.3;
  gp.n_monitor = 2 * (r->p + 1) * (r->p + 1);
  if (build_geometry(gp, &u->g, err) != HSMA_OK) return nullptr;
  const Geometry& g = u->g;
  struct Up { DevBuf* b; const std::vector<double>* v; };
  const Up ups[] = {{&u->d_P, &g.P}, {&u->d_W, &g.W}, {&u->d_Y, &g.ysurf}, {&u->d_C, &g.check_pts}};
  for (const Up& up : ups) {
    if (up.b->ensure(up.v->size() * 8) ||
        cudaMemcpy(up.b->p, up.v->data(), up.v->size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      *err = "geometry upload failed";
      return nullptr;
    }
  }
  const UnitGeo* out = u.get();
  s->geos[key] = std::move(u);
  return out;
}

// Point a slot's handle at a request: geometry view for its box, buffers for N.
static int bind_request(Server* s, Slot& sl, Request* r, std::string* err) {
  const UnitGeo* ug = unit_geometry(s, r, err);
  if (!ug) return HSMA_ERR_NUMERIC;
  hsma_ctx* h = sl.ctx;
  const bool same = sl.geo == ug && sl.box[0] == r->box[0] && sl.box[1] == r->box[1] &&
                    sl.box[2] == r->box[2];
  if (!same) {
    const Geometry& u = ug->g;
    Geometry& g = h->geo;
    g.par = u.par;
    for (int d = 0; d < 3; ++d) g.par.box[d] = r->box[d];
    sphere_radius(g.par.box, g.par.lam, &g.Rc, &g.Rs, &g.Rs2);
    build_shifts(g.par, g.Rs, &g.shifts);
    g.n_mon = u.n_mon;
    g.n_check = u.n_check;
    g.nv = u.nv;
    g.nA = u.nA;
    g.rank = u.rank;
    // the slot's previous request has retired, so its pinned staging buffer
    // is no longer read by a pending copy
    const size_t nsh = g.shifts.size() * 5;
    if (sl.h_shifts_n < nsh) {
      if (sl.h_shifts) cudaFreeHost(sl.h_shifts);
      sl.h_shifts = nullptr;
      sl.h_shifts_n = 0;
      if (cudaMallocHost((void**)&sl.h_shifts, nsh * 8) != cudaSuccess) {
        cudaGetLastError();
        sl.h_shifts = nullptr;
        *err = "pinned shift buffer";
        return HSMA_ERR_NOMEM;
      }
      sl.h_shifts_n = nsh;
    }
    double* sh = sl.h_shifts;
    for (size_t i = 0; i < g.shifts.size(); ++i) {
      sh[5 * i] = g.shifts[i].sx;
      sh[5 * i + 1] = g.shifts[i].sy;
      sh[5 * i + 2] = g.shifts[i].zs;
      sh[5 * i + 3] = g.shifts[i].zo;
      sh[5 * i + 4] = g.shifts[i].f;
    }
    const size_t M = g.par.M;
    if (h->d_shifts.ensure(nsh * 8) || h->d_v.ensure((size_t)g.nv * 8) ||
        h->d_A.ensure((size_t)g.nA * 8) || h->d_cphi.ensure((size_t)g.n_check * 8) ||
        h->d_cdz.ensure((size_t)g.n_check * 8) || h->d_Q.ensure(M * 8) ||
        h->d_s32.ensure(M * 16) || h->d_s64.ensure(M * 32)) {
      *err = "slot buffers";
      return HSMA_ERR_NOMEM;
    }
    // ordered on the server stream after any earlier batch that used them
    if (cudaMemcpyAsync(h->d_shifts.p, sh, nsh * 8, cudaMemcpyHostToDevice, h->stream) !=
        cudaSuccess) {
      cudaGetLastError();
      *err = "shift upload";
      return HSMA_ERR_CUDA;
    }
    h->ext_P = (const double*)ug->d_P.p;
    h->ext_W = (const double*)ug->d_W.p;
    h->ext_Y = (const double*)ug->d_Y.p;
    h->ext_C = (const double*)ug->d_C.p;
    h->gscale = r->box[0];
    h->geo_dirty = false;
    h->plan_N = -1;
    sl.geo = ug;
    for (int d = 0; d < 3; ++d) sl.box[d] = r->box[d];
  }
  int rc = ensure_plan(h, r->N);
  if (rc) *err = h->err;
  return rc;
}

static void retire(Server* s) {
  for (BatchBuf& bb : s->bufs) {
    if (!bb.busy) continue;
    cudaError_t q = cudaEventQuery(bb.done);
    if (q == cudaErrorNotReady) continue;
    for (Request* r : bb.reqs) {
      Slot& sl = s->slots[r->slot];
      if (q != cudaSuccess) {
        r->status = HSMA_ERR_CUDA;
        r->err = cudaGetErrorString(q);
      } else {
        r->status = finish_eval(sl.ctx, &r->energy);
        if (r->status != HSMA_OK) r->err = sl.ctx->err;
      }
      s->in_use -= (double)r->bytes;
      sl.req = nullptr;
    }
    if (q != cudaSuccess) cudaGetLastError();
    bb.reqs.clear();
    bb.busy = false;
  }
}

static int launch_batch(Server* s, BatchBuf& bb) {
  cudaStream_t st = s->stream;
  const int n = (int)bb.reqs.size();
  for (Request* r : bb.reqs) {
    hsma_ctx* h = s->slots[r->slot].ctx;
    cudaError_t e = cudaMemcpyAsync(h->d_x.p, r->hx, (size_t)r->N * 24, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q.p, r->hq, (size_t)r->N * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return HSMA_ERR_CUDA;
    int rc = stage_prep(h, r->N);
    if (rc) return rc;
  }
  for (int phase = 0; phase < 2; ++phase) {
    if (phase == 1)
      for (Request* r : bb.reqs) {
        int rc = stage_fit(s->slots[r->slot].ctx, r->N);
        if (rc) return rc;
      }
    if (s->precision >= 1) {
      PairArgs* d = bb.h_desc + phase * (int)s->slots.size();
      int* start = bb.h_start + phase * ((int)s->slots.size() + 1);
      int items = 0;
      for (int k = 0; k < n; ++k) {
        Request* r = bb.reqs[k];
        hsma_ctx* h = s->slots[r->slot].ctx;
        d[k] = phase == 0 ? near_args(h, r->N) : far_args(h, r->N);
        start[k] = items;
        items += d[k].n_tiles * d[k].n_chunks;
      }
      start[n] = items;
      PairArgs* dd = (PairArgs*)bb.d_desc.p + phase * (int)s->slots.size();
      int* ds = (int*)bb.d_start.p + phase * ((int)s->slots.size() + 1);
      cudaError_t e = cudaMemcpyAsync(dd, d, sizeof(PairArgs) * n, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ds, start, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = launch_pair_ragged(s->precision, dd, ds, n, std::min(items, s->ragged_slots), st);
      if (e != cudaSuccess) return HSMA_ERR_CUDA;
    } else {
      for (Request* r : bb.reqs) {
        hsma_ctx* h = s->slots[r->slot].ctx;
        cudaError_t e = phase == 0 ? launch_pair(0, 1, near_args(h, r->N), h->grid1, st)
                                   : launch_pair(0, 1, far_args(h, r->N), h->grid2, st);
        if (e != cudaSuccess) return HSMA_ERR_CUDA;
      }
    }
  }
  for (Request* r : bb.reqs) {
    hsma_ctx* h = s->slots[r->slot].ctx;
    int rc = stage_assemble(h, r->N, (double*)h->d_forces.p, (double*)h->d_pot.p);
    if (rc) return rc;
    if (cudaMemcpyAsync(r->hf, h->d_forces.p, (size_t)r->N * 24, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return HSMA_ERR_CUDA;
  }
  if (cudaEventRecord(bb.done, st) != cudaSuccess) return HSMA_ERR_CUDA;
  bb.busy = true;
  return HSMA_OK;
}

static int step(Server* s) {
  retire(s);
  BatchBuf* bb = nullptr;
  for (BatchBuf& b : s->bufs)
    if (!b.busy) { bb = &b; break; }
  if (bb) {
    // admit in arrival order while a slot and the budget allow
    while (!s->queue.empty()) {
      Request* r = s->queue.front();
      int free_slot = -1;
      for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].req) { free_slot = (int)i; break; }
      if (free_slot < 0 || s->in_use + (double)r->bytes > s->budget) break;
      s->queue.pop_front();
      std::string err;
      Slot& sl = s->slots[free_slot];
      int rc = bind_request(s, sl, r, &err);
      if (rc == HSMA_OK && r->ticket == s->inject_fail_ticket) {
        rc = HSMA_ERR_CUDA;
        err = "injected failure";
      }
      if (rc != HSMA_OK) {
        r->status = rc;
        r->err = err;
        continue;
      }
      sl.req = r;
      r->slot = free_slot;
      s->in_use += (double)r->bytes;
      bb->reqs.push_back(r);
    }
    if (!bb->reqs.empty()) {
      int rc = launch_batch(s, *bb);
      if (rc != HSMA_OK) {
        // the batch could not be enqueued: fail its requests, free their slots
        cudaStreamSynchronize(s->stream);
        cudaGetLastError();
        for (Request* r : bb->reqs) {
          r->status = rc;
          r->err = "the batch launch failed";
          s->in_use -= (double)r->bytes;
          s->slots[r->slot].req = nullptr;
        }
        bb->reqs.clear();
      }
    }
  }
  int active = (int)s->queue.size();
  for (Slot& sl : s->slots) active += sl.req ? 1 : 0;
  return active;
}

}  // namespace hsma

using namespace hsma;

int server_set_option(hsma_ctx* h, const std::string& key, double v) {
  if (!h->srv) return HSMA_ERR_ARG;
  if (key == "inject_fail_ticket" && v >= 0) {
    h->srv->inject_fail_ticket = (uint64_t)v;
    return HSMA_OK;
  }
  h->err = "unknown server option " + key;
  return HSMA_ERR_ARG;
}

void server_shutdown(hsma_ctx* h) {
  if (!h->srv) return;
  Server* s = h->srv;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (Slot& sl : s->slots) {
    delete sl.ctx;
    if (sl.h_shifts) cudaFreeHost(sl.h_shifts);
  }
  for (BatchBuf& bb : s->bufs) {
    if (bb.h_desc) cudaFreeHost(bb.h_desc);
    if (bb.h_start) cudaFreeHost(bb.h_start);
    bb.d_desc.release();
    bb.d_start.release();
    if (bb.done) cudaEventDestroy(bb.done);
  }
  for (auto& kv : s->geos) {
    kv.second->d_P.release();
    kv.second->d_W.release();
    kv.second->d_Y.release();
    kv.second->d_C.release();
  }
  for (auto& kv : s->all) free_request(kv.second);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  h->srv = nullptr;
}

extern "C" {

int hsma_server_create(int slots, double budget_bytes, int precision, hsma_t* out) {
  if (!out) return HSMA_ERR_ARG;
  *out = nullptr;
  if (slots < 1 || slots > 64 || !(budget_bytes > 0) || precision < 0 || precision > 2)
    return HSMA_ERR_ARG;
  hsma_ctx* h = new (std::nothrow) hsma_ctx();
  if (!h) return HSMA_ERR_NOMEM;
  h->is_server = true;
  Server* s = new Server();
  h->srv = s;
  s->precision = precision;
  s->budget = budget_bytes;
  int rc = HSMA_OK;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) rc = HSMA_ERR_CUDA;
  if (rc == HSMA_OK) s->ragged_slots = pair_ragged_slots(precision);
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    if (rc != HSMA_OK) break;
    sl.ctx = new hsma_ctx();
    sl.ctx->precision = precision;
    sl.ctx->autotune = 0;                      // a request's plan depends only on the request
    if (precision) sl.ctx->tpt = pair_ragged_variant(precision);
    rc = hsma_ctx_init(sl.ctx);
    if (rc == HSMA_OK) {
      cudaStreamDestroy(sl.ctx->stream);
      sl.ctx->stream = s->stream;      // every slot works on the server's stream
      sl.ctx->own_stream = false;
    }
  }
  for (BatchBuf& bb : s->bufs) {
    if (rc != HSMA_OK) break;
    if (cudaMallocHost((void**)&bb.h_desc, sizeof(PairArgs) * 2 * slots) != cudaSuccess ||
        cudaMallocHost((void**)&bb.h_start, sizeof(int) * 2 * (slots + 1)) != cudaSuccess ||
        bb.d_desc.ensure(sizeof(PairArgs) * 2 * slots) || bb.d_start.ensure(sizeof(int) * 2 * (slots + 1)) ||
        cudaEventCreateWithFlags(&bb.done, cudaEventDisableTiming) != cudaSuccess)
      rc = HSMA_ERR_NOMEM;
  }
  if (rc != HSMA_OK) {
    cudaGetLastError();
    server_shutdown(h);
    delete h;
    return rc;
  }
  *out = h;
  return HSMA_OK;
}

int hsma_submit(hsma_t server, const double* x, const double* q, int64_t N, const double box[3],
                int p, int M, uint64_t* ticket) {
  if (!server || !server->srv) return HSMA_ERR_ARG;
  hsma_ctx* h = server;
  Server* s = h->srv;
  if (!x || !q || !box || !ticket || N < 1 || N > (int64_t)1 << 28) {
    h->err = "bad submit arguments";
    return HSMA_ERR_ARG;
  }
  if (p < 1 || p > 40 || M < (p + 1) * (p + 1) || !geometry_size_ok(p, M, 2 * (p + 1) * (p + 1))) {
    h->err = "need 1 <= p <= 40 and (p+1)^2 <= M <= 2^31 / (p+1)^2";
    return HSMA_ERR_ARG;
  }
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0) || !std::isfinite(box[d])) {
      h->err = "box lengths must be > 0";
      return HSMA_ERR_ARG;
    }
  Request* r = new Request();
  r->N = N;
  for (int d = 0; d < 3; ++d) r->box[d] = box[d];
  r->p = p;
  r->M = M;
  r->bytes = request_bytes(N, box, p, M, s->precision);
  if ((double)r->bytes > s->budget) {
    delete r;
    h->err = "request exceeds the memory budget";
    return HSMA_ERR_BUDGET;
  }
  if (cudaMallocHost((void**)&r->hx, (size_t)N * 24) != cudaSuccess ||
      cudaMallocHost((void**)&r->hq, (size_t)N * 8) != cudaSuccess ||
      cudaMallocHost((void**)&r->hf, (size_t)N * 24) != cudaSuccess) {
    cudaGetLastError();
    free_request(r);
    h->err = "pinned host allocation failed";
    return HSMA_ERR_NOMEM;
  }
  if (cudaMemcpy(r->hx, x, (size_t)N * 24, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(r->hq, q, (size_t)N * 8, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    free_request(r);
    h->err = "input copy failed";
    return HSMA_ERR_CUDA;
  }
  double qs = 0, qa = 0;
  for (int64_t i = 0; i < N; ++i) {
    qs += r->hq[i];
    qa += std::fabs(r->hq[i]);
  }
  if (std::fabs(qs) > 1e-10 * qa) {
    free_request(r);
    h->err = "system not neutral";
    return HSMA_ERR_NOT_NEUTRAL;
  }
  r->ticket = s->next_ticket++;
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  step(s);
  return HSMA_OK;
}

int hsma_poll(hsma_t server, uint64_t ticket, double* energy, double* forces) {
  if (!server || !server->srv) return HSMA_ERR_ARG;
  Server* s = server->srv;
  auto it = s->all.find(ticket);
  if (it == s->all.end()) {
    server->err = "unknown ticket";
    return HSMA_ERR_ARG;
  }
  step(s);
  Request* r = it->second;
  if (r->status == HSMA_PENDING) return HSMA_PENDING;
  const int st = r->status;
  if (st == HSMA_OK) {
    if (energy) *energy = r->energy;
    if (forces) {
      cudaError_t e = cudaMemcpy(forces, r->hf, (size_t)r->N * 24, cudaMemcpyDefault);
      if (e != cudaSuccess) {
        cudaGetLastError();
        server->err = "result copy failed";
        return HSMA_ERR_CUDA;
      }
    }
  } else {
    server->err = r->err;
  }
  s->all.erase(it);
  free_request(r);
  return st;
}

int hsma_server_step(hsma_t server) {
  if (!server || !server->srv) return HSMA_ERR_ARG;
  return step(server->srv);
}

}  // extern "C"
