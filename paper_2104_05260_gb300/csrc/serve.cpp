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
  cudaEvent_t start = nullptr;      // recorded before the batch's first operation
  cudaEvent_t phase_ev[2] = {nullptr, nullptr};   // after the near and the far ragged launch
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
  cudaEvent_t ev = nullptr;     // joins the slot's stream into the server stream
  cudaStream_t own_stream = nullptr;   // the slot context's own stream
};

// Pinned host buffers, reused: requests take their input and result buffers
// from here and give them back when polled.  cudaMallocHost / cudaFreeHost
// are slow and freeing synchronises with the device, which would drain the
// batches in flight at every poll; the pool keeps both off the request path.
// Buffers are kept per power-of-two size class until the server is destroyed.
struct PinnedPool {
  std::map<size_t, std::vector<void*>> free_;
  std::vector<void*> all_;
  static size_t size_class(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
  }
  void* get(size_t bytes) {
    const size_t c = size_class(bytes);
    std::vector<void*>& v = free_[c];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    all_.push_back(p);
    return p;
  }
  void put(void* p, size_t bytes) {
    if (p) free_[size_class(bytes)].push_back(p);
  }
  void release() {
    for (void* p : all_) cudaFreeHost(p);
    all_.clear();
    free_.clear();
  }
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
  PinnedPool pinned;
  // counters: batches enqueued, and how many earlier batches were still on
  // the GPU when the last one was enqueued
  uint64_t batches = 0;
  int inflight_at_last = 0;
  double gpu_ms = 0;   // summed span (first to last operation) of the retired batches
  // the ragged pair launch: kernel code of its items (slots plan their tiles
  // with it) and, when dynamic, a counter pair per launch (near, far)
  int ragged_variant = 12;
  int ragged_dynamic = 1;
  int slot_streams = 1;   // each slot's small kernels on a stream of its own
  int max_batch = 0;      // requests per batch at most (0: every free slot)
  DevBuf d_queue;
};

static void free_request(Server* s, Request* r) {
  s->pinned.put(r->hx, (size_t)r->N * 24);
  s->pinned.put(r->hq, (size_t)r->N * 8);
  s->pinned.put(r->hf, (size_t)r->N * 24);
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
    float ms = 0.f;
    if (q == cudaSuccess && cudaEventElapsedTime(&ms, bb.start, bb.done) == cudaSuccess) s->gpu_ms += ms;
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

// Enqueue one batch.  Each request's own small kernels (prep, fit,
// assembly) and copies run on its slot's stream, so those of different
// requests overlap on the GPU; the two ragged pair launches run on the server
// stream.  Events join the streams: the server stream waits for every slot
// before each ragged launch, the slots wait for that launch before their next
// stage, and the batch's done event follows every slot's last copy.  A slot's
// first stage (input copies, prep) waits for nothing: the slot's buffers
// belong to its request alone, so with several batches in flight (option
// max_batch) a batch's prep runs while an earlier batch is still on the GPU.
// With slot streams off (option slot_streams = 0) everything runs on the
// server stream in this order.
static int launch_batch(Server* s, BatchBuf& bb) {
  cudaStream_t st = s->stream;
  const int n = (int)bb.reqs.size();
  if (cudaEventRecord(bb.start, st) != cudaSuccess) return HSMA_ERR_CUDA;
  auto slot_of = [&](Request* r) -> Slot& { return s->slots[r->slot]; };
  // the slot streams wait for ev (recorded on the server stream)
  auto fan_out = [&](cudaEvent_t ev) -> bool {
    if (!s->slot_streams) return true;
    for (Request* r : bb.reqs)
      if (cudaStreamWaitEvent(slot_of(r).ctx->stream, ev, 0) != cudaSuccess) return false;
    return true;
  };
  // the server stream waits for every slot stream's work so far
  auto fan_in = [&]() -> bool {
    if (!s->slot_streams) return true;
    for (Request* r : bb.reqs) {
      Slot& sl = slot_of(r);
      if (cudaEventRecord(sl.ev, sl.ctx->stream) != cudaSuccess ||
          cudaStreamWaitEvent(st, sl.ev, 0) != cudaSuccess)
        return false;
    }
    return true;
  };
  for (Request* r : bb.reqs) {
    hsma_ctx* h = slot_of(r).ctx;
    cudaError_t e = cudaMemcpyAsync(h->d_x.p, r->hx, (size_t)r->N * 24, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->d_q.p, r->hq, (size_t)r->N * 8, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return HSMA_ERR_CUDA;
    int rc = stage_prep(h, r->N);
    if (rc) return rc;
  }
  for (int phase = 0; phase < 2; ++phase) {
    if (phase == 1)
      for (Request* r : bb.reqs) {
        int rc = stage_fit(slot_of(r).ctx, r->N);
        if (rc) return rc;
      }
    if (s->precision >= 1) {
      if (!fan_in()) return HSMA_ERR_CUDA;
      PairArgs* d = bb.h_desc + phase * (int)s->slots.size();
      int* start = bb.h_start + phase * ((int)s->slots.size() + 1);
      int items = 0;
      for (int k = 0; k < n; ++k) {
        Request* r = bb.reqs[k];
        hsma_ctx* h = slot_of(r).ctx;
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
        e = launch_pair_ragged(s->precision, s->ragged_variant, dd, ds, n, std::min(items, s->ragged_slots),
                               s->ragged_dynamic ? (int*)s->d_queue.p + 2 * phase : nullptr, st);
      if (e == cudaSuccess) e = cudaEventRecord(bb.phase_ev[phase], st);
      if (e != cudaSuccess || !fan_out(bb.phase_ev[phase])) return HSMA_ERR_CUDA;
    } else {
      // FP64: one launch per request, on its slot stream
      for (Request* r : bb.reqs) {
        hsma_ctx* h = slot_of(r).ctx;
        cudaError_t e = phase == 0 ? launch_pair(0, 1, near_args(h, r->N), h->grid1, h->stream)
                                   : launch_pair(0, 1, far_args(h, r->N), h->grid2, h->stream);
        if (e != cudaSuccess) return HSMA_ERR_CUDA;
      }
    }
  }
  for (Request* r : bb.reqs) {
    hsma_ctx* h = slot_of(r).ctx;
    int rc = stage_assemble(h, r->N, (double*)h->d_forces.p, (double*)h->d_pot.p);
    if (rc) return rc;
    if (cudaMemcpyAsync(r->hf, h->d_forces.p, (size_t)r->N * 24, cudaMemcpyDeviceToHost, h->stream) !=
        cudaSuccess)
      return HSMA_ERR_CUDA;
  }
  if (!fan_in()) return HSMA_ERR_CUDA;
  if (cudaEventRecord(bb.done, st) != cudaSuccess) return HSMA_ERR_CUDA;
  int inflight = 0;
  for (const BatchBuf& b : s->bufs) inflight += b.busy ? 1 : 0;
  s->inflight_at_last = inflight;
  s->batches++;
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
    while (!s->queue.empty() && (s->max_batch <= 0 || (int)bb->reqs.size() < s->max_batch)) {
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
        cudaDeviceSynchronize();
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

int server_get_info(hsma_ctx* h, const std::string& key, double* v) {
  if (!h->srv) return HSMA_ERR_ARG;
  if (key == "batches") *v = (double)h->srv->batches;
  else if (key == "inflight_at_last_batch") *v = h->srv->inflight_at_last;
  else if (key == "queued") *v = (double)h->srv->queue.size();
  else if (key == "gpu_ms") *v = h->srv->gpu_ms;
  else if (key == "ragged_variant") *v = h->srv->ragged_variant;
  else if (key == "ragged_dynamic") *v = h->srv->ragged_dynamic;
  else if (key == "slot_streams") *v = h->srv->slot_streams;
  else if (key == "max_batch") *v = h->srv->max_batch;
  else return HSMA_ERR_ARG;
  return HSMA_OK;
}

int server_set_option(hsma_ctx* h, const std::string& key, double v) {
  if (!h->srv) return HSMA_ERR_ARG;
  Server* s = h->srv;
  if (key == "inject_fail_ticket" && v >= 0) {
    s->inject_fail_ticket = (uint64_t)v;
    return HSMA_OK;
  }
  if (key == "max_batch") {
    // takes effect at the next batch; requests already admitted keep theirs
    if (v < 0 || v != (int)v) {
      h->err = "max_batch must be an integer >= 0";
      return HSMA_ERR_ARG;
    }
    s->max_batch = (int)v;
    return HSMA_OK;
  }
  if (key == "ragged_variant" || key == "ragged_dynamic" || key == "slot_streams") {
    // only while no request is in the server (slots plan with the variant)
    bool idle = s->queue.empty();
    for (const Slot& sl : s->slots) idle = idle && !sl.req;
    if (!idle) {
      h->err = key + " can be changed only while the server holds no request";
      return HSMA_ERR_ARG;
    }
    if (key == "ragged_dynamic" || key == "slot_streams") {
      if (v != 0 && v != 1) {
        h->err = key + " must be 0 or 1";
        return HSMA_ERR_ARG;
      }
      if (key == "ragged_dynamic") {
        s->ragged_dynamic = (int)v;
        return HSMA_OK;
      }
      // every slot context works on its own stream, or on the server's
      s->slot_streams = (int)v;
      for (Slot& sl : s->slots) sl.ctx->stream = v ? sl.own_stream : s->stream;
      return HSMA_OK;
    }
    if (s->precision == 0 || !pair_ragged_code_ok(s->precision, (int)v) || v != (int)v) {
      h->err = "ragged_variant must be 12 or 24 (precision 1), 32 or 44 (precision 2)";
      return HSMA_ERR_ARG;
    }
    s->ragged_variant = (int)v;
    s->ragged_slots = pair_ragged_slots(s->precision, s->ragged_variant);
    for (Slot& sl : s->slots) {
      sl.ctx->tpt = s->ragged_variant;
      sl.ctx->plan_N = -1;
    }
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
    if (sl.own_stream) cudaStreamSynchronize(sl.own_stream);
    if (sl.ctx) sl.ctx->stream = sl.own_stream;   // the context destroys its own stream
    delete sl.ctx;
    if (sl.h_shifts) cudaFreeHost(sl.h_shifts);
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
  for (BatchBuf& bb : s->bufs) {
    if (bb.h_desc) cudaFreeHost(bb.h_desc);
    if (bb.h_start) cudaFreeHost(bb.h_start);
    bb.d_desc.release();
    bb.d_start.release();
    if (bb.done) cudaEventDestroy(bb.done);
    if (bb.start) cudaEventDestroy(bb.start);
    for (cudaEvent_t& e : bb.phase_ev)
      if (e) cudaEventDestroy(e);
  }
  for (auto& kv : s->geos) {
    kv.second->d_P.release();
    kv.second->d_W.release();
    kv.second->d_Y.release();
    kv.second->d_C.release();
  }
  for (auto& kv : s->all) free_request(s, kv.second);
  s->pinned.release();
  s->d_queue.release();
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
  if (precision) s->ragged_variant = pair_ragged_variant(precision);
  if (rc == HSMA_OK) s->ragged_slots = pair_ragged_slots(precision, s->ragged_variant);
  if (rc == HSMA_OK && (s->d_queue.ensure(4 * sizeof(int)) ||
                        cudaMemset(s->d_queue.p, 0, 4 * sizeof(int)) != cudaSuccess))
    rc = HSMA_ERR_NOMEM;
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    if (rc != HSMA_OK) break;
    sl.ctx = new hsma_ctx();
    sl.ctx->precision = precision;
    sl.ctx->autotune = 0;                      // a request's plan depends only on the request
    sl.ctx->fused_reduce = 0;                  // ragged launches leave the chunk sums to k_reduce_chunks
    sl.ctx->dynamic_schedule = 0;
    if (precision) sl.ctx->tpt = s->ragged_variant;
    rc = hsma_ctx_init(sl.ctx);   // the slot's context owns a non-blocking stream
    if (rc == HSMA_OK && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess)
      rc = HSMA_ERR_CUDA;
    if (rc == HSMA_OK) sl.own_stream = sl.ctx->stream;
  }
  for (BatchBuf& bb : s->bufs) {
    if (rc != HSMA_OK) break;
    if (cudaMallocHost((void**)&bb.h_desc, sizeof(PairArgs) * 2 * slots) != cudaSuccess ||
        cudaMallocHost((void**)&bb.h_start, sizeof(int) * 2 * (slots + 1)) != cudaSuccess ||
        bb.d_desc.ensure(sizeof(PairArgs) * 2 * slots) || bb.d_start.ensure(sizeof(int) * 2 * (slots + 1)) ||
        cudaEventCreate(&bb.done) != cudaSuccess || cudaEventCreate(&bb.start) != cudaSuccess ||
        cudaEventCreateWithFlags(&bb.phase_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bb.phase_ev[1], cudaEventDisableTiming) != cudaSuccess)
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
  r->hx = (double*)s->pinned.get((size_t)N * 24);
  r->hq = (double*)s->pinned.get((size_t)N * 8);
  r->hf = (double*)s->pinned.get((size_t)N * 24);
  if (!r->hx || !r->hq || !r->hf) {
    free_request(s, r);
    h->err = "pinned host allocation failed";
    return HSMA_ERR_NOMEM;
  }
  // host inputs are copied on the host; device inputs through the driver
  if (!is_device_ptr(x) && !is_device_ptr(q)) {
    std::memcpy(r->hx, x, (size_t)N * 24);
    std::memcpy(r->hq, q, (size_t)N * 8);
  } else if (cudaMemcpy(r->hx, x, (size_t)N * 24, cudaMemcpyDefault) != cudaSuccess ||
             cudaMemcpy(r->hq, q, (size_t)N * 8, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    free_request(s, r);
    h->err = "input copy failed";
    return HSMA_ERR_CUDA;
  }
  double qs = 0, qa = 0;
  for (int64_t i = 0; i < N; ++i) {
    qs += r->hq[i];
    qa += std::fabs(r->hq[i]);
  }
  if (std::fabs(qs) > 1e-10 * qa) {
    free_request(s, r);
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
      if (!is_device_ptr(forces)) {
        std::memcpy(forces, r->hf, (size_t)r->N * 24);
      } else if (cudaMemcpy(forces, r->hf, (size_t)r->N * 24, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        server->err = "result copy failed";
        return HSMA_ERR_CUDA;
      }
    }
  } else {
    server->err = r->err;
  }
  s->all.erase(it);
  free_request(s, r);
  return st;
}

int hsma_server_step(hsma_t server) {
  if (!server || !server->srv) return HSMA_ERR_ARG;
  return step(server->srv);
}

}  // extern "C"
