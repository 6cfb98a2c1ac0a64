// Request server: continuous batching of independent Ising solves on one GPU.
//
// A worker thread owns `max_active` slots, each a context with its own
// stream. It loops: (1) admits queued requests in arrival order while a slot
// is free and the estimated device footprint of the admitted set stays within
// the budget, and sets them up (upload, pruning, session); (2) for every
// admitted request whose previous chunk has completed (an event on its
// stream, polled without blocking), either queues `chunk_steps` more
// domain-selection steps or, when its steps are done, finishes it (final
// energy pass, best of restarts, reconstruction, full-instance energy) and
// releases its memory and slot. Slots progress independently, so a small
// request never waits for a large one's chunk, and requests arriving at any
// time are admitted as soon as a slot and memory free up.
// With ISING_SERVER_PACK, the dense tensor-core requests that are ready in a
// round are grouped by kind (operand type, energy mode, tile width) and each
// group advances its chunk as one pack (ising_pack: one launch per step for
// all of them, on the server's own stream); a group's pack is kept, with its
// captured step graph, while the group stays the same.
#include "ds_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

using namespace ising;

namespace ising {
int prune_device(ising_ctx* ctx, const DevInstance& I, int flags, ising_prune_result** out);
int pack_advance(ising_pack* pk, int64_t steps);
}

namespace {

struct Request {
  uint64_t id = 0;
  // owned host copy of the instance
  std::vector<unsigned char> J, h;
  std::vector<int64_t> indptr;
  std::vector<int32_t> indices;
  ising_instance inst{};
  ising_ds_params p{};
  int prune_flags = 0;
  size_t footprint = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int slot = -1;
  // running state
  DevInstance I;
  ising_prune_result* pr = nullptr;
  ising_ds* ds = nullptr;
  int64_t nG = 0;
  bool started = false;
  cudaEvent_t ev = nullptr;  // completion of the request's last queued chunk
  bool in_flight = false;
  // result
  int status = ISING_OK;
  bool done = false;
  std::vector<int8_t> spins;
  double energy = 0.0;
  ising_ds_stats stats{};
};

// Device bytes a request holds while admitted (instance copy, pruning work,
// operands, state, spins, partials, bests), estimated from its shape.
size_t estimate_footprint(const ising_instance* in, const ising_ds_params* p) {
  const double n = (double)in->n, B = (double)p->restarts;
  const double ld = n + 16.0;
  const double jsz = (double)dtype_size(in->j_dtype);
  double bytes;
  if (in->layout == ISING_LAYOUT_DENSE) {
    bytes = n * n * jsz * 2.0          // uploaded instance and the reduced copy
            + n * ld * 2.0 * 2.0       // operand planes (at most two 16-bit)
            + B * ld * (12.0 + 3.0 * 2.0);  // theta, m, v and three spin slots
  } else {
    const double nnz = (double)in->nnz;
    bytes = nnz * (jsz + 4.0) * 2.0 + n * 16.0 * 2.0 + nnz * 8.0  // instance, reduced, folds
            + ((B + 127.0) / 128.0 * 128.0) * n * (12.0 + 3.0 / 8.0);
  }
  bytes += B * (n + 16.0) + B * 64.0;           // best spins, per-restart scalars
  bytes += 2.0 * B * (4.0 * (n / 128.0 + 1.0)) * 20.0;  // energy partials
  bytes += 4.0 * 1024.0 * 1024.0;               // small buffers
  return (size_t)bytes;
}

}  // namespace

struct ising_server {
  ising_ctx* parent = nullptr;
  ising_server_cfg cfg{};
  std::vector<std::unique_ptr<ising_ctx>> slots;
  std::vector<bool> slot_busy;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;       // work arrived / stop
  std::condition_variable done_cv;  // a request finished
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  size_t used = 0;
  bool stop = false;
  uint64_t next_id = 1;
  // packed advancement (ISING_SERVER_PACK): the server's stream, and the
  // pack of each current group of requests (keyed by its members' ids)
  std::unique_ptr<ising_ctx> pack_ctx;
  std::map<std::vector<uint64_t>, ising_pack*> packs;
  std::chrono::steady_clock::time_point t0;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Pruning and session set-up of an admitted request on its slot's stream.
int start_request(ising_server* srv, Request* r) {
  ising_ctx* ctx = srv->slots[r->slot].get();
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  ISING_TRY(upload_instance(ctx, &r->inst, &r->I));
  ISING_TRY(prune_device(ctx, r->I, r->prune_flags, &r->pr));
  ising_prune_info(r->pr, &r->nG, nullptr, nullptr, nullptr, nullptr);
  if (r->nG > 0) {
    ising_instance red;
    ising_prune_reduced(r->pr, &red);
    ising_ds_params p = r->p;
    p.flags |= ISING_DS_STREAMING;  // no grid barrier across concurrent requests
    ISING_TRY(ds_create_impl(ctx, &red, &p, &r->ds, false));
  }
  ISING_CUDA(ctx, cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
  r->started = true;
  return ISING_OK;
}

// Final pass and result of a request whose steps are done.
int finish_request(ising_server* srv, Request* r) {
  ising_ctx* ctx = srv->slots[r->slot].get();
  DevMem sG, full, E;
  ISING_TRY(dev_alloc(ctx, sG, std::max<int64_t>(r->nG, 1)));
  ISING_TRY(dev_alloc(ctx, full, r->inst.n));
  ISING_TRY(dev_alloc(ctx, E, 8));
  if (r->ds) {
    double eg = 0.0;
    ISING_TRY(ising_ds_finish(r->ds));
    ISING_TRY(ising_ds_result(r->ds, sG.as<int8_t>(), &eg, &r->stats, ISING_MEM_DEVICE));
  }
  ISING_TRY(ising_reconstruct(ctx, r->pr, sG.as<int8_t>(), full.as<int8_t>(), ISING_MEM_DEVICE));
  ISING_TRY(energy_device(ctx, r->I, full.as<int8_t>(), 1, E.as<double>(), nullptr, nullptr));
  r->spins.resize(r->inst.n);
  ISING_CUDA(ctx, cudaMemcpyAsync(r->spins.data(), full.p, r->inst.n, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaMemcpyAsync(&r->energy, E.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

void release_request(ising_server* srv, Request* r) {
  if (r->ds) ising_ds_destroy(r->ds);
  r->ds = nullptr;
  if (r->pr) ising_prune_free(r->pr);
  r->pr = nullptr;
  r->I = DevInstance();
  r->J.clear();
  r->J.shrink_to_fit();
  r->h.clear();
  r->indptr.clear();
  r->indices.clear();
  if (r->slot >= 0) cudaStreamSynchronize(srv->slots[r->slot]->stream);
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
}

void worker_loop(ising_server* srv) {
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    // 1. admission, in arrival order
    std::vector<Request*> admitted;
    while (!srv->queue.empty() && (int)srv->active.size() < srv->cfg.max_active) {
      Request* r = srv->queue.front();
      if (srv->used + r->footprint > srv->cfg.budget_bytes) break;
      srv->queue.pop_front();
      int slot = 0;
      while (srv->slot_busy[slot]) ++slot;
      srv->slot_busy[slot] = true;
      r->slot = slot;
      r->t_admit = srv->now_ms();
      srv->used += r->footprint;
      srv->active.push_back(r);
      admitted.push_back(r);
    }
    if (srv->active.empty()) {
      if (srv->stop && srv->queue.empty()) break;
      srv->cv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    std::vector<Request*> act = srv->active;
    const int64_t chunk = srv->cfg.chunk_steps;
    lk.unlock();
    for (Request* r : admitted) {
      int rc = start_request(srv, r);
      if (rc != ISING_OK) {
        r->status = rc;
        r->started = false;
      }
    }
    // 2. every request whose last chunk has completed: next chunk, or finish
    bool progressed = !admitted.empty();
    std::vector<Request*> finished;
    std::map<uint64_t, std::vector<Request*>> groups;  // packable requests by kind
    for (Request* r : act) {
      if (r->in_flight) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        r->in_flight = false;
        if (q != cudaSuccess) r->status = ISING_ECUDA;
        if (r->status == ISING_OK && r->ds) {
          int rc = ds_conv_check(r->ds);  // convergence rule: have all restarts stopped?
          if (rc != ISING_OK) r->status = rc;
        }
      }
      progressed = true;
      const bool steps_done =
          r->status != ISING_OK || !r->ds || r->ds->t >= r->ds->T || r->ds->conv_all;
      if (!steps_done) {
        if (srv->pack_ctx && tc_packable(r->ds)) {
          groups[tc_pack_key(r->ds)].push_back(r);
          continue;
        }
        const int64_t todo = std::min<int64_t>(chunk, r->ds->T - r->ds->t);
        int rc = ds_advance(r->ds, todo);
        if (rc == ISING_OK && cudaEventRecord(r->ev, srv->slots[r->slot]->stream) != cudaSuccess)
          rc = ISING_ECUDA;
        if (rc != ISING_OK) r->status = rc;
        else r->in_flight = true;
        continue;
      }
      if (r->status == ISING_OK) {
        int rc = finish_request(srv, r);
        if (rc != ISING_OK) r->status = rc;
      }
      release_request(srv, r);
      r->t_done = srv->now_ms();
      finished.push_back(r);
    }
    // 3. each group of ready dense tensor-core requests of one kind: one
    // packed chunk (their chunks end together, at the group's smallest
    // remaining step count)
    for (auto& kv : groups) {
      std::vector<Request*>& grp = kv.second;
      std::vector<uint64_t> ids;
      for (Request* r : grp) ids.push_back(r->id);
      int64_t todo = chunk;
      for (Request* r : grp) todo = std::min<int64_t>(todo, r->ds->T - r->ds->t);
      int rc = ISING_OK;
      ising_pack* pk = nullptr;
      auto it = srv->packs.find(ids);
      if (it != srv->packs.end()) {
        pk = it->second;
      } else {
        std::vector<ising_ds*> ds;
        for (Request* r : grp) ds.push_back(r->ds);
        rc = ising_pack_create(srv->pack_ctx.get(), ds.data(), (int32_t)ds.size(), &pk);
        if (rc == ISING_OK) srv->packs[ids] = pk;
      }
      if (rc == ISING_OK) rc = pack_advance(pk, todo);
      for (Request* r : grp) {
        int rr = rc;
        if (rr == ISING_OK && cudaEventRecord(r->ev, srv->pack_ctx->stream) != cudaSuccess)
          rr = ISING_ECUDA;
        if (rr != ISING_OK) r->status = rr;
        else r->in_flight = true;
      }
    }
    // packs whose group no longer exists (a member finished, or the group
    // changed): their launches are complete (every member was ready)
    for (auto it = srv->packs.begin(); it != srv->packs.end();) {
      bool live = false;
      for (auto& kv : groups) {
        std::vector<uint64_t> ids;
        for (Request* r : kv.second) ids.push_back(r->id);
        if (ids == it->first) live = true;
      }
      bool in_flight = false;
      for (Request* r : act)
        if (r->in_flight && std::find(it->first.begin(), it->first.end(), r->id) != it->first.end())
          in_flight = true;
      if (!live && !in_flight) {
        ising_pack_destroy(it->second);
        it = srv->packs.erase(it);
      } else {
        ++it;
      }
    }
    lk.lock();
    for (Request* r : finished) {
      srv->slot_busy[r->slot] = false;
      srv->used -= r->footprint;
      r->done = true;
      for (size_t k = 0; k < srv->active.size(); ++k)
        if (srv->active[k] == r) {
          srv->active.erase(srv->active.begin() + k);
          break;
        }
    }
    if (!finished.empty()) srv->done_cv.notify_all();
    // nothing completed: wait a little (new submissions wake the worker)
    if (!progressed) srv->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

void fill_result(const Request* r, ising_result* res) {
  res->status = r->status;
  res->done = r->done ? 1 : 0;
  res->n = r->inst.n;
  res->best_energy = r->energy;
  res->best_restart = r->stats.best_restart;
  res->best_step = r->stats.best_step;
  res->footprint = (int64_t)r->footprint;
  res->t_submit_ms = r->t_submit;
  res->t_admit_ms = r->t_admit;
  res->t_done_ms = r->t_done;
}

int copy_in(ising_ctx* ctx, void* dst, const void* src, size_t bytes, int mem) {
  if (!bytes) return ISING_OK;
  if (mem == ISING_MEM_HOST) {
    memcpy(dst, src, bytes);
    return ISING_OK;
  }
  ISING_CUDA(ctx, cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  return ISING_OK;
}

}  // namespace

extern "C" int ising_server_create(ising_ctx* ctx, const ising_server_cfg* cfg,
                                   ising_server** out) {
  if (!ctx) return ISING_EINVAL;
  if (!cfg || !out) return fail(ctx, ISING_EINVAL, "cfg and out are required");
  if (cfg->max_active < 1 || cfg->max_active > 256 || cfg->chunk_steps < 1 ||
      (cfg->flags & ~ISING_SERVER_PACK) != 0)
    return fail(ctx, ISING_EINVAL, "bad server configuration");
  *out = nullptr;
  auto srv = new ising_server();
  srv->parent = ctx;
  srv->cfg = *cfg;
  srv->t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < cfg->max_active; ++k) {
    auto c = std::make_unique<ising_ctx>();
    c->device = ctx->device;
    c->sm_count = ctx->sm_count;
    c->smem_optin = ctx->smem_optin;
    cudaSetDevice(ctx->device);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& s : srv->slots) cudaStreamDestroy(s->stream);
      delete srv;
      return fail(ctx, ISING_ECUDA, "stream creation failed");
    }
    srv->slots.push_back(std::move(c));
  }
  srv->slot_busy.assign(cfg->max_active, false);
  if (cfg->flags & ISING_SERVER_PACK) {
    auto c = std::make_unique<ising_ctx>();
    c->device = ctx->device;
    c->sm_count = ctx->sm_count;
    c->smem_optin = ctx->smem_optin;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& s : srv->slots) cudaStreamDestroy(s->stream);
      delete srv;
      return fail(ctx, ISING_ECUDA, "stream creation failed");
    }
    srv->pack_ctx = std::move(c);
  }
  srv->worker = std::thread(worker_loop, srv);
  *out = srv;
  return ISING_OK;
}

extern "C" int ising_server_submit(ising_server* srv, const ising_instance* inst,
                                   const ising_ds_params* p, int prune_flags, uint64_t* req_id) {
  if (!srv) return ISING_EINVAL;
  ising_ctx* ctx = srv->parent;
  if (!inst || !p || !req_id) return fail(ctx, ISING_EINVAL, "inst, p and req_id are required");
  if (inst->n < 1 || (inst->layout != ISING_LAYOUT_DENSE && inst->layout != ISING_LAYOUT_CSR) ||
      dtype_size(inst->j_dtype) == 0 || !inst->J ||
      (inst->mem != ISING_MEM_HOST && inst->mem != ISING_MEM_DEVICE))
    return fail(ctx, ISING_EINVAL, "bad instance");
  if (inst->layout == ISING_LAYOUT_CSR && (!inst->indptr || (inst->nnz > 0 && !inst->indices)))
    return fail(ctx, ISING_EINVAL, "CSR instance needs indptr and indices");
  if (p->restarts < 1 || p->steps < 0) return fail(ctx, ISING_EINVAL, "bad parameters");
  auto r = std::make_unique<Request>();
  r->footprint = estimate_footprint(inst, p);
  if (r->footprint > srv->cfg.budget_bytes)
    return fail(ctx, ISING_EBUSY, "request footprint %zu exceeds the budget", r->footprint);
  const int64_t n = inst->n;
  const size_t jsz = dtype_size(inst->j_dtype);
  const size_t jcount = inst->layout == ISING_LAYOUT_DENSE ? (size_t)n * n : (size_t)inst->nnz;
  r->J.resize(jcount * jsz);
  ISING_TRY(copy_in(ctx, r->J.data(), inst->J, jcount * jsz, inst->mem));
  if (inst->layout == ISING_LAYOUT_CSR) {
    r->indptr.resize(n + 1);
    r->indices.resize(inst->nnz);
    ISING_TRY(copy_in(ctx, r->indptr.data(), inst->indptr, (n + 1) * 8, inst->mem));
    ISING_TRY(copy_in(ctx, r->indices.data(), inst->indices, inst->nnz * 4, inst->mem));
  }
  if (inst->h) {
    const size_t hb = (size_t)n * dtype_size(inst->h_dtype);
    r->h.resize(hb);
    ISING_TRY(copy_in(ctx, r->h.data(), inst->h, hb, inst->mem));
  }
  r->inst = *inst;
  r->inst.mem = ISING_MEM_HOST;
  r->inst.J = r->J.data();
  r->inst.indptr = inst->layout == ISING_LAYOUT_CSR ? r->indptr.data() : nullptr;
  r->inst.indices = inst->layout == ISING_LAYOUT_CSR ? r->indices.data() : nullptr;
  r->inst.h = inst->h ? r->h.data() : nullptr;
  r->p = *p;
  r->prune_flags = prune_flags;
  std::lock_guard<std::mutex> g(srv->mu);
  if (srv->stop) return fail(ctx, ISING_EINVAL, "server is stopping");
  r->id = srv->next_id++;
  r->t_submit = srv->now_ms();
  *req_id = r->id;
  srv->queue.push_back(r.get());
  srv->all[r->id] = std::move(r);
  srv->cv.notify_all();
  return ISING_OK;
}

extern "C" int ising_server_poll(ising_server* srv, uint64_t req_id, ising_result* res,
                                 int8_t* spins) {
  if (!srv || !res) return ISING_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->all.find(req_id);
  if (it == srv->all.end()) return fail(srv->parent, ISING_EINVAL, "unknown request id");
  const Request* r = it->second.get();
  fill_result(r, res);
  if (r->done && spins && r->status == ISING_OK) memcpy(spins, r->spins.data(), r->spins.size());
  return ISING_OK;
}

extern "C" int ising_server_wait(ising_server* srv, uint64_t req_id, double timeout_s,
                                 ising_result* res, int8_t* spins) {
  if (!srv || !res) return ISING_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->all.find(req_id);
  if (it == srv->all.end()) return fail(srv->parent, ISING_EINVAL, "unknown request id");
  Request* r = it->second.get();
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s));
  while (!r->done) {
    if (srv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
      return fail(srv->parent, ISING_ETIMEOUT, "request %llu not done in time",
                  (unsigned long long)req_id);
  }
  fill_result(r, res);
  if (spins && r->status == ISING_OK) memcpy(spins, r->spins.data(), r->spins.size());
  return ISING_OK;
}

extern "C" int ising_server_release(ising_server* srv, uint64_t req_id) {
  if (!srv) return ISING_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->all.find(req_id);
  if (it == srv->all.end()) return fail(srv->parent, ISING_EINVAL, "unknown request id");
  if (!it->second->done) return fail(srv->parent, ISING_EINVAL, "request not done");
  srv->all.erase(it);
  return ISING_OK;
}

extern "C" int ising_server_destroy(ising_server* srv) {
  if (!srv) return ISING_OK;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();
  for (auto& kv : srv->packs) ising_pack_destroy(kv.second);
  srv->packs.clear();
  if (srv->pack_ctx) {
    cudaStreamSynchronize(srv->pack_ctx->stream);
    cudaStreamDestroy(srv->pack_ctx->stream);
  }
  for (auto& s : srv->slots) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  delete srv;
  return ISING_OK;
}
