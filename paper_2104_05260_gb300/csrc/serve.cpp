// Request loop for independent HSMA3D evaluations (hsma_submit / hsma_poll).
//
// Requests are admitted in arrival order while a slot and enough of the
// device-memory budget are free; each admitted request runs the evaluation
// pipeline on its slot's own stream, so requests that arrive while others are
// on the GPU overlap with them.  A request's launch plan depends only on its
// own N and geometry, so its result does not depend on what else is running.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/hsma.h"
#include "api_internal.hpp"

namespace hsma {

struct Request {
  uint64_t ticket;
  int64_t N;
  double box[3];
  int p, M;
  double* hx = nullptr;    // pinned copies of the inputs, then the results
  double* hq = nullptr;
  double* hf = nullptr;
  double energy = 0;
  int status = HSMA_PENDING;
  size_t bytes = 0;
  int slot = -1;
};

struct Slot {
  hsma_ctx* ctx = nullptr;
  Request* req = nullptr;
  cudaEvent_t done = nullptr;
};

struct Server {
  int precision = 1;
  double budget = 0;
  double in_use = 0;
  uint64_t next_ticket = 1;
  std::vector<Slot> slots;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
};

static void free_request(Request* r) {
  if (r->hx) cudaFreeHost(r->hx);
  if (r->hq) cudaFreeHost(r->hq);
  if (r->hf) cudaFreeHost(r->hf);
  delete r;
}

// Device bytes one request holds (FP32 path): inputs, images, targets,
// partials and outputs; an upper bound used for admission.
static size_t request_bytes(int64_t N, const double box[3], int p, int M, int precision) {
  GeoParams gp;
  for (int d = 0; d < 3; ++d) gp.box[d] = box[d];
  double Rc, Rs, Rs2;
  sphere_radius(box, 1.3, &Rc, &Rs, &Rs2);
  const double V = box[0] * box[1] * box[2];
  const double ns = std::min(27.0, 1.2 * 4.18879 * Rs * Rs * Rs / V + 1.0) * (double)N;
  const int nm = 2 * (p + 1) * (p + 1);
  const double img = precision ? 16.0 : 32.0;
  const double per_n = 24 + 8 + 24 + 4 + 24 + 8 + 24;
  return (size_t)(ns * img + (N + 2 * nm) * (img + 8.0 * 4 * 16) + N * (per_n + 8.0 * 4 * 16) +
                  (double)M * 64 + 4.0 * M * (p + 1) * (p + 1) * 8);
}

static int start_request(Server* s, int si, Request* r, std::string* err) {
  Slot& sl = s->slots[si];
  hsma_ctx* h = sl.ctx;
  if (h->gp.box[0] != r->box[0] || h->gp.box[1] != r->box[1] || h->gp.box[2] != r->box[2] ||
      h->gp.p != r->p || h->gp.M != r->M) {
    for (int d = 0; d < 3; ++d) h->gp.box[d] = r->box[d];
    h->gp.p = r->p;
    h->gp.M = r->M;
    h->gp.n_monitor = 2 * (r->p + 1) * (r->p + 1);
    h->geo_dirty = true;
  }
  int rc = ensure_geometry(h);
  if (rc == HSMA_OK) rc = ensure_plan(h, r->N);
  if (rc != HSMA_OK) {
    *err = h->err;
    return rc;
  }
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemcpyAsync(h->d_x.p, r->hx, (size_t)r->N * 24, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q.p, r->hq, (size_t)r->N * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return HSMA_ERR_CUDA;
  }
  rc = enqueue_eval(h, r->N, (double*)h->d_forces.p, (double*)h->d_pot.p);
  if (rc != HSMA_OK) {
    *err = h->err;
    return rc;
  }
  e = cudaMemcpyAsync(r->hf, h->d_forces.p, (size_t)r->N * 24, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return HSMA_ERR_CUDA;
  }
  sl.req = r;
  r->slot = si;
  return HSMA_OK;
}

static int step(Server* s) {
  // retire finished requests
  for (Slot& sl : s->slots) {
    if (!sl.req) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    Request* r = sl.req;
    if (q != cudaSuccess) {
      cudaGetLastError();
      r->status = HSMA_ERR_CUDA;
    } else {
      r->status = finish_eval(sl.ctx, &r->energy);
    }
    s->in_use -= (double)r->bytes;
    sl.req = nullptr;
  }
  // admit in arrival order
  while (!s->queue.empty()) {
    Request* r = s->queue.front();
    int free_slot = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
      if (!s->slots[i].req) { free_slot = (int)i; break; }
    if (free_slot < 0 || s->in_use + (double)r->bytes > s->budget) break;
    s->queue.pop_front();
    std::string err;
    int rc = start_request(s, free_slot, r, &err);
    if (rc != HSMA_OK) {
      r->status = rc;
      continue;
    }
    s->in_use += (double)r->bytes;
  }
  int active = (int)s->queue.size();
  for (Slot& sl : s->slots) active += sl.req ? 1 : 0;
  return active;
}

}  // namespace hsma

using namespace hsma;

void server_shutdown(hsma_ctx* h) {
  if (!h->srv) return;
  Server* s = h->srv;
  for (Slot& sl : s->slots) {
    if (sl.ctx) {
      if (sl.ctx->stream) cudaStreamSynchronize(sl.ctx->stream);
      delete sl.ctx;
    }
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (auto& kv : s->all) free_request(kv.second);
  delete s;
  h->srv = nullptr;
}

extern "C" {

int hsma_server_create(int slots, double budget_bytes, int precision, hsma_t* out) {
  if (!out) return HSMA_ERR_ARG;
  *out = nullptr;
  if (slots < 1 || slots > 256 || !(budget_bytes > 0) || (precision != 0 && precision != 1))
    return HSMA_ERR_ARG;
  hsma_ctx* h = new (std::nothrow) hsma_ctx();
  if (!h) return HSMA_ERR_NOMEM;
  h->is_server = true;
  Server* s = new Server();
  h->srv = s;
  s->precision = precision;
  s->budget = budget_bytes;
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    sl.ctx = new hsma_ctx();
    sl.ctx->precision = precision;
    int rc = hsma_ctx_init(sl.ctx);
    if (rc == HSMA_OK && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
      rc = HSMA_ERR_CUDA;
    if (rc != HSMA_OK) {
      server_shutdown(h);
      delete h;
      return rc;
    }
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
  if (p < 1 || p > 40 || M < (p + 1) * (p + 1)) {
    h->err = "need p >= 1 and M >= (p+1)^2";
    return HSMA_ERR_ARG;
  }
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0)) {
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
