// Request server: continuous batching of independent Ising solves on one GPU.
//
// A worker thread owns `max_active` slots, each a context with its own
// stream. It loops: (1) admits queued requests in arrival order while a slot
// is free and the estimated device footprint of the admitted set stays within
// the budget, and hands their set-up (upload, pruning, session) to a helper
// thread; (2) for every set-up request whose previous chunk has completed (an
// event on its stream, polled without blocking), either queues `chunk_steps`
// more domain-selection steps or, when its steps are done, hands it to a
// helper that finishes it (final energy pass, best of restarts,
// reconstruction, full-instance energy) and releases its memory and slot.
// Slots progress independently, so a small request never waits for a large
// one's chunk, requests arriving at any time are admitted as soon as a slot
// and memory free up, and set-up and finishing (host work and
// synchronisations of a request's own stream) do not hold up the chunks of
// the others.
// With ISING_SERVER_PACK, the dense tensor-core requests that are ready in a
// round are grouped by kind (operand type, energy mode) and each group
// advances its chunk as one pack (ising_pack: one launch per step for all of
// them, on one of the server's pack streams, which packs take in turn so
// that different groups' chunks overlap); a group's pack is kept, with its
// captured step graph, while the group stays the same.
#include "ds_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
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
  bool has_target = false;  // time-to-target query
  double target = 0.0;
  bool reached = false;
  std::atomic<bool> cancel{false};  // set by ising_server_cancel
  bool cancelled = false;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int slot = -1;
  int phase = 0;  // kQueued, kSettingUp, kReady, kFinishing, kDone
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
  std::string error;  // the failure's message
  bool done = false;
  std::vector<int8_t> spins;
  double energy = 0.0;
  ising_ds_stats stats{};
};

enum Phase { kQueued = 0, kSettingUp, kReady, kFinishing, kDone };

constexpr int kPackStreams = 4;  // streams the server's packs take in turn

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
  std::vector<std::thread> helpers;
  std::mutex mu;
  std::condition_variable cv;       // work arrived / a request is ready / stop
  std::condition_variable done_cv;  // a request finished
  std::condition_variable task_cv;  // set-up or finishing for the helpers
  std::deque<Request*> tasks;
  bool helpers_stop = false;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  size_t used = 0;
  bool stop = false;
  uint64_t next_id = 1;
  // packed advancement (ISING_SERVER_PACK): the server's pack streams, and
  // the pack of each current group of requests (keyed by its members' ids)
  // with the stream it runs on; packs take the streams in turn, so the
  // chunks of different groups overlap on the device (a pack of a few small
  // requests holds only a few SMs)
  std::vector<std::unique_ptr<ising_ctx>> pack_ctxs;
  int next_pack_ctx = 0;
  struct PackSlot {
    ising_pack* pk;
    ising_ctx* ctx;
  };
  std::map<std::vector<uint64_t>, PackSlot> packs;
  std::chrono::steady_clock::time_point t0;
  ising_server_stats st{};  // guarded by mu

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t).count();
}

// Pruning and session set-up of an admitted request on its slot's stream;
// `ms` receives the upload, pruning and session times.
int start_request(ising_server* srv, Request* r, double ms[3]) {
  ising_ctx* ctx = srv->slots[r->slot].get();
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  auto t = Clock::now();
  ISING_TRY(upload_instance(ctx, &r->inst, &r->I));
  ms[0] = ms_since(t);
  t = Clock::now();
  ISING_TRY(prune_device(ctx, r->I, r->prune_flags, &r->pr));
  ising_prune_info(r->pr, &r->nG, nullptr, nullptr, nullptr, nullptr);
  ms[1] = ms_since(t);
  t = Clock::now();
  if (r->nG > 0) {
    ising_instance red;
    ising_prune_reduced(r->pr, &red);
    ising_ds_params p = r->p;
    // no grid barrier across concurrent requests: the streaming form, except
    // where the small resident form applies (n <= 128, without the
    // convergence rule or the relaxed product: each CTA holds all of J and
    // its restarts, no grid barrier), which runs a whole chunk in one launch
    const bool small = red.n <= 128 && !(p.flags & (ISING_DS_CONVERGE | ISING_DS_RELAXED));
    if (!small) p.flags |= ISING_DS_STREAMING;
    ISING_TRY(ds_create_impl(ctx, &red, &p, &r->ds, false));
  }
  ISING_CUDA(ctx, cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
  ms[2] = ms_since(t);
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
    ISING_TRY(ising_ds_finish(r->ds));
    ISING_TRY(ising_ds_result(r->ds, sG.as<int8_t>(), nullptr, &r->stats, ISING_MEM_DEVICE));
  }
  ISING_TRY(ising_reconstruct(ctx, r->pr, sG.as<int8_t>(), full.as<int8_t>(), ISING_MEM_DEVICE));
  ISING_TRY(energy_device(ctx, r->I, full.as<int8_t>(), 1, E.as<double>(), nullptr, nullptr));
  r->spins.resize(r->inst.n);
  ISING_CUDA(ctx, cudaMemcpyAsync(r->spins.data(), full.p, r->inst.n, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaMemcpyAsync(&r->energy, E.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

// Time-to-target check: the full-instance energy of the best spins so far
// (as finish_request would report them, without the final pass).
int check_target(ising_server* srv, Request* r, bool* hit) {
  ising_ctx* ctx = srv->slots[r->slot].get();
  DevMem sG, full, E;
  ISING_TRY(dev_alloc(ctx, sG, std::max<int64_t>(r->nG, 1)));
  ISING_TRY(dev_alloc(ctx, full, r->inst.n));
  ISING_TRY(dev_alloc(ctx, E, 8));
  ISING_TRY(ising_ds_result(r->ds, sG.as<int8_t>(), nullptr, nullptr, ISING_MEM_DEVICE));
  ISING_TRY(ising_reconstruct(ctx, r->pr, sG.as<int8_t>(), full.as<int8_t>(), ISING_MEM_DEVICE));
  ISING_TRY(energy_device(ctx, r->I, full.as<int8_t>(), 1, E.as<double>(), nullptr, nullptr));
  double e = 0.0;
  ISING_CUDA(ctx, cudaMemcpyAsync(&e, E.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *hit = e <= r->target;
  return ISING_OK;
}

// Records a request's failure with the message of the context that saw it.
void set_failed(Request* r, int rc, const ising_ctx* ctx) {
  if (r->status != ISING_OK) return;  // keep the first
  r->status = rc;
  r->error = ctx ? ctx->err : std::string("a CUDA call failed");
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

// Helper threads: the set-up of admitted requests and the finishing of
// requests whose steps are done run here, so the worker keeps queueing chunks
// meanwhile. A request is handed from thread to thread by its phase, under
// the server's lock, so one thread at a time works on it.
void helper_loop(ising_server* srv) {
  cudaSetDevice(srv->parent->device);  // (as in worker_loop)
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    srv->task_cv.wait(lk, [&] { return srv->helpers_stop || !srv->tasks.empty(); });
    if (srv->tasks.empty()) break;  // stopping, nothing left
    Request* r = srv->tasks.front();
    srv->tasks.pop_front();
    const bool setup = r->phase == kSettingUp;
    lk.unlock();
    const auto t0 = Clock::now();
    double release_ms = 0.0;
    ising_ctx* sctx = srv->slots[r->slot].get();
    double part[3] = {0.0, 0.0, 0.0};
    if (setup) {
      int rc = start_request(srv, r, part);
      if (rc != ISING_OK) {
        set_failed(r, rc, sctx);
        r->started = false;
      }
    } else {
      if (r->status == ISING_OK) {
        int rc = finish_request(srv, r);
        if (rc != ISING_OK) set_failed(r, rc, sctx);
        // a target met by the steps of the last chunk or the final pass
        else if (r->has_target && r->energy <= r->target) r->reached = true;
      }
      const auto t1 = Clock::now();
      release_request(srv, r);
      release_ms = ms_since(t1);
    }
    const double ms = ms_since(t0);
    lk.lock();
    if (setup) {
      srv->st.setup_ms += ms;
      srv->st.setup_upload_ms += part[0];
      srv->st.setup_prune_ms += part[1];
      srv->st.setup_session_ms += part[2];
      r->phase = kReady;
    } else {
      srv->st.finish_ms += ms - release_ms;
      srv->st.release_ms += release_ms;
      srv->st.completed += 1;
      r->t_done = srv->now_ms();
      r->phase = kDone;
      r->done = true;
      srv->slot_busy[r->slot] = false;
      srv->used -= r->footprint;
      for (size_t k = 0; k < srv->active.size(); ++k)
        if (srv->active[k] == r) {
          srv->active.erase(srv->active.begin() + k);
          break;
        }
      srv->done_cv.notify_all();
    }
    srv->cv.notify_all();  // a request is ready, or a slot and memory are free
  }
}

void worker_loop(ising_server* srv) {
  // the thread's current device (and context: some launches first encode
  // tensor maps through the driver, which needs one)
  cudaSetDevice(srv->parent->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    // 1. admission, in arrival order; the set-up runs on a helper thread
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
      r->phase = kSettingUp;
      srv->active.push_back(r);
      srv->tasks.push_back(r);
      srv->task_cv.notify_one();
    }
    if (srv->active.empty()) {
      if (srv->stop && srv->queue.empty()) break;
      const auto tw = Clock::now();
      srv->cv.wait_for(lk, std::chrono::milliseconds(5));
      srv->st.idle_ms += ms_since(tw);
      continue;
    }
    std::vector<Request*> act;
    for (Request* r : srv->active)
      if (r->phase == kReady) act.push_back(r);
    const int64_t chunk = srv->cfg.chunk_steps;
    lk.unlock();
    ising_server_stats rs{};  // this round's share, merged under the lock
    auto tp = Clock::now();
    // 2. every ready request whose last chunk has completed: next chunk, or
    // (its steps done, its target met or a failure) hand it to a helper
    bool progressed = false;
    std::vector<Request*> finishing;
    std::map<uint64_t, std::vector<Request*>> groups;  // packable requests by kind
    for (Request* r : act) {
      if (r->in_flight) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        r->in_flight = false;
        ising_ctx* sctx = srv->slots[r->slot].get();
        if (q != cudaSuccess) {
          fail(sctx, ISING_ECUDA, "a chunk of steps failed: %s", cudaGetErrorString(q));
          set_failed(r, ISING_ECUDA, sctx);
        }
        tp = Clock::now();
        if (r->status == ISING_OK && r->ds) {
          int rc = ds_conv_check(r->ds);  // convergence rule: have all restarts stopped?
          if (rc != ISING_OK) set_failed(r, rc, sctx);
        }
        if (r->status == ISING_OK && r->ds && r->has_target && r->ds->t < r->ds->T) {
          bool hit = false;
          int rc = check_target(srv, r, &hit);
          rs.target_checks += 1;
          if (rc != ISING_OK) {
            set_failed(r, rc, sctx);
          } else if (hit) {
            r->reached = true;
            r->ds->T = r->ds->t;  // finish without the remaining steps
          }
        }
        rs.check_ms += ms_since(tp);
      }
      progressed = true;
      if (r->cancel.load() && r->ds && r->ds->t < r->ds->T) {
        r->cancelled = true;
        r->ds->T = r->ds->t;  // finish with the steps run so far
      }
      const bool steps_done =
          r->status != ISING_OK || !r->ds || r->ds->t >= r->ds->T || r->ds->conv_all;
      if (!steps_done) {
        if (!srv->pack_ctxs.empty() && tc_packable(r->ds)) {
          groups[tc_pack_key(r->ds)].push_back(r);
          continue;
        }
        const int64_t todo = std::min<int64_t>(chunk, r->ds->T - r->ds->t);
        tp = Clock::now();
        ising_ctx* sctx = srv->slots[r->slot].get();
        int rc = ds_advance(r->ds, todo);
        if (rc == ISING_OK) {
          const cudaError_t e = cudaEventRecord(r->ev, sctx->stream);
          if (e != cudaSuccess)
            rc = fail(sctx, ISING_ECUDA, "cudaEventRecord failed: %s", cudaGetErrorString(e));
        }
        rs.advance_ms += ms_since(tp);
        rs.chunks += 1;
        if (rc != ISING_OK) set_failed(r, rc, sctx);
        else r->in_flight = true;
        continue;
      }
      finishing.push_back(r);
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
      ising_ctx* pctx = nullptr;
      tp = Clock::now();
      auto it = srv->packs.find(ids);
      if (it != srv->packs.end()) {
        pk = it->second.pk;
        pctx = it->second.ctx;
      } else {
        std::vector<ising_ds*> ds;
        for (Request* r : grp) ds.push_back(r->ds);
        pctx = srv->pack_ctxs[srv->next_pack_ctx].get();
        srv->next_pack_ctx = (srv->next_pack_ctx + 1) % (int)srv->pack_ctxs.size();
        rc = ising_pack_create(pctx, ds.data(), (int32_t)ds.size(), &pk);
        if (rc == ISING_OK) srv->packs[ids] = {pk, pctx};
        rs.packs_created += 1;
        rs.pack_create_ms += ms_since(tp);
      }
      if (rc == ISING_OK) rc = pack_advance(pk, todo);
      rs.advance_ms += ms_since(tp);
      rs.pack_chunks += 1;
      for (Request* r : grp) {
        int rr = rc;
        if (rr == ISING_OK) {
          const cudaError_t e = cudaEventRecord(r->ev, pctx->stream);
          if (e != cudaSuccess)
            rr = fail(pctx, ISING_ECUDA, "cudaEventRecord failed: %s", cudaGetErrorString(e));
        }
        if (rr != ISING_OK) set_failed(r, rr, pctx);
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
        ising_pack_destroy(it->second.pk);
        it = srv->packs.erase(it);
      } else {
        ++it;
      }
    }
    lk.lock();
    rs.rounds = progressed ? 1 : 0;
    ising_server_stats& t = srv->st;
    t.rounds += rs.rounds;
    t.chunks += rs.chunks;
    t.pack_chunks += rs.pack_chunks;
    t.packs_created += rs.packs_created;
    t.target_checks += rs.target_checks;
    t.advance_ms += rs.advance_ms;
    t.pack_create_ms += rs.pack_create_ms;
    t.check_ms += rs.check_ms;
    for (Request* r : finishing) {
      r->phase = kFinishing;
      srv->tasks.push_back(r);
    }
    if (!finishing.empty()) srv->task_cv.notify_all();
    // nothing completed: wait a little (submissions and helpers wake the worker)
    if (!progressed) {
      const auto tw = Clock::now();
      srv->cv.wait_for(lk, std::chrono::microseconds(50));
      srv->st.idle_ms += ms_since(tw);
    }
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
  res->steps_done = r->stats.steps_done;
  res->reached = r->reached ? 1 : 0;
  res->cancelled = r->cancelled ? 1 : 0;
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
      cfg->helper_threads < 0 || cfg->helper_threads > 16 ||
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
    for (int k = 0; k < kPackStreams; ++k) {
      auto c = std::make_unique<ising_ctx>();
      c->device = ctx->device;
      c->sm_count = ctx->sm_count;
      c->smem_optin = ctx->smem_optin;
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        for (auto& s : srv->slots) cudaStreamDestroy(s->stream);
        for (auto& s : srv->pack_ctxs) cudaStreamDestroy(s->stream);
        delete srv;
        return fail(ctx, ISING_ECUDA, "stream creation failed");
      }
      srv->pack_ctxs.push_back(std::move(c));
    }
  }
  const int helpers = cfg->helper_threads > 0 ? cfg->helper_threads : 2;
  for (int k = 0; k < helpers; ++k) srv->helpers.emplace_back(helper_loop, srv);
  srv->worker = std::thread(worker_loop, srv);
  *out = srv;
  return ISING_OK;
}

namespace {

int submit_impl(ising_server* srv, const ising_instance* inst, const ising_ds_params* p,
                int prune_flags, const double* target, uint64_t* req_id) {
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
  if (target) {
    r->has_target = true;
    r->target = *target;
  }
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

}  // namespace

extern "C" int ising_server_submit(ising_server* srv, const ising_instance* inst,
                                   const ising_ds_params* p, int prune_flags, uint64_t* req_id) {
  return submit_impl(srv, inst, p, prune_flags, nullptr, req_id);
}

extern "C" int ising_server_submit_target(ising_server* srv, const ising_instance* inst,
                                          const ising_ds_params* p, int prune_flags,
                                          double target_energy, uint64_t* req_id) {
  if (srv && std::isnan(target_energy))
    return fail(srv->parent, ISING_EINVAL, "target energy is NaN");
  return submit_impl(srv, inst, p, prune_flags, &target_energy, req_id);
}

extern "C" int ising_server_cancel(ising_server* srv, uint64_t req_id) {
  if (!srv) return ISING_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->all.find(req_id);
  if (it == srv->all.end()) return fail(srv->parent, ISING_EINVAL, "unknown request id");
  Request* r = it->second.get();
  if (r->done) return ISING_OK;
  if (r->phase == kQueued) {
    // not admitted yet: dropped, done at once without a result
    for (size_t k = 0; k < srv->queue.size(); ++k)
      if (srv->queue[k] == r) {
        srv->queue.erase(srv->queue.begin() + k);
        break;
      }
    r->cancelled = true;
    r->energy = std::nan("");
    r->t_admit = r->t_done = srv->now_ms();
    r->phase = kDone;
    r->done = true;
    srv->done_cv.notify_all();
    return ISING_OK;
  }
  r->cancel.store(true);
  srv->cv.notify_all();
  return ISING_OK;
}

extern "C" int ising_server_error(ising_server* srv, uint64_t req_id, char* buf, int64_t len) {
  if (!srv) return ISING_EINVAL;
  if (!buf || len < 1) return fail(srv->parent, ISING_EINVAL, "buf and len >= 1 are required");
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->all.find(req_id);
  if (it == srv->all.end()) return fail(srv->parent, ISING_EINVAL, "unknown request id");
  const Request* r = it->second.get();
  const std::string msg = r->done ? r->error : std::string();
  const size_t k = std::min<size_t>(msg.size(), (size_t)(len - 1));
  memcpy(buf, msg.data(), k);
  buf[k] = 0;
  return ISING_OK;
}

extern "C" int ising_server_stats_get(ising_server* srv, ising_server_stats* out) {
  if (!srv) return ISING_EINVAL;
  if (!out) return fail(srv->parent, ISING_EINVAL, "out is required");
  std::lock_guard<std::mutex> g(srv->mu);
  *out = srv->st;
  out->elapsed_ms = srv->now_ms();
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
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->helpers_stop = true;
    srv->task_cv.notify_all();
  }
  for (auto& h : srv->helpers)
    if (h.joinable()) h.join();
  for (auto& kv : srv->packs) ising_pack_destroy(kv.second.pk);
  srv->packs.clear();
  for (auto& c : srv->pack_ctxs) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  for (auto& s : srv->slots) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  delete srv;
  return ISING_OK;
}
