// Batching: several domain-selection sessions (Sec. III-B), of different
// sizes and restart counts, advanced together. One step of every member is
// one persistent tensor-core launch over the concatenation of the members'
// tiles, whose epilogue warps also track every member's previous step (with
// the convergence rule: a tracking launch over all their restarts after each
// step instead); each member keeps its own device step counter, from which
// the launches pick its spin and partial slots, so the launches are the same
// for every step whatever the members' progress and the step loop is
// replayed from a CUDA graph.
// A small instance that would leave most SMs idle alone shares the SMs with
// the other members instead (the restarts of Sec. IV-C, across instances).
#include "ds_internal.cuh"

#include <algorithm>
#include <vector>

using namespace ising;

struct ising_pack {
  ising_ctx* ctx = nullptr;
  std::vector<ising_ds*> members;
  uint64_t key = 0;
  int bn = 128;     // restart-tile width of every member's tiles
  int spin_kind = 0;
  int tiles = 0;
  int64_t restarts = 0;
  DevMem entries;   // PackEntry[count]
  DevMem start;     // int[count + 1] tile offsets
  DevMem targs;     // TrackArgs[count]
  DevMem rstart;    // int64[count + 1] restart offsets
  DevMem words;     // [0] track block counter, [1] error word
  cudaGraphExec_t graph = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev = nullptr;
  bool launched = false;  // the kernels have run once outside capture
  int64_t advances = 0;   // pack_advance calls so far
  // the step launches track every member's previous step (no member uses
  // the convergence rule); each pack_advance then ends with one tracking
  // launch for the last step
  bool fold = false;
};

namespace {

constexpr int64_t kPackGraphSteps = 25;

// The pack's restart-tile width: a persistent CTA per SM takes the tiles in
// waves, so a step costs about (waves) x (the time of one tile), and a
// tile's time grows with its width (its epilogue over 128 x bn elements, and
// its products): the width with the least waves x bn is taken (padding of
// the members' restart counts included in the tile counts), the wider one
// on a tie.
int pack_width(const ising_ctx* ctx, ising_ds* const* s, int count) {
  const int widths[4] = {256, 224, 128, 64};
  int pick = 0;
  int64_t best = -1;
  for (int w = 0; w < 4; ++w) {
    int64_t tiles = 0;
    for (int k = 0; k < count; ++k)
      tiles += (int64_t)ceil_div_i(s[k]->n, 128) * ceil_div_i(s[k]->B, widths[w]);
    const int64_t cost = (tiles + ctx->sm_count - 1) / ctx->sm_count * widths[w];
    if (best < 0 || cost < best) {
      best = cost;
      pick = w;
    }
  }
  return widths[pick];
}

int pack_step(ising_pack* pk) {
  ising_ctx* ctx = pk->ctx;
  int* err = reinterpret_cast<int*>(pk->words.as<unsigned long long>() + 1);
  PackFold f;
  if (pk->fold) {
    f.trk = pk->targs.as<TrackArgs>();
    f.rstart = pk->rstart.as<int64_t>();
    f.done = pk->words.as<unsigned long long>();
  }
  ISING_TRY(tc_pack_launch(ctx, pk->key, pk->bn, pk->entries.p, pk->start.as<int>(),
                           (int)pk->members.size(), pk->tiles, err, f));
  if (pk->fold) return ISING_OK;
  return track_pack(ctx, pk->spin_kind, pk->targs.as<TrackArgs>(), pk->rstart.as<int64_t>(),
                    (int)pk->members.size(), pk->restarts, pk->words.as<unsigned long long>());
}

// Captures kPackGraphSteps steps on a private stream.
int pack_graph(ising_pack* pk) {
  ising_ctx* ctx = pk->ctx;
  ISING_CUDA(ctx, cudaStreamCreateWithFlags(&pk->gstream, cudaStreamNonBlocking));
  cudaStream_t saved = ctx->stream;
  ctx->stream = pk->gstream;
  cudaGraph_t g = nullptr;
  int rc = ISING_OK;
  cudaError_t e = cudaStreamBeginCapture(pk->gstream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int64_t s = 0; s < kPackGraphSteps && rc == ISING_OK; ++s) rc = pack_step(pk);
    e = cudaStreamEndCapture(pk->gstream, &g);
  }
  ctx->stream = saved;
  if (rc != ISING_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, ISING_ECUDA, "pack graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&pk->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    pk->graph = nullptr;
    return fail(ctx, ISING_ECUDA, "pack graph instantiation failed: %s", cudaGetErrorString(e));
  }
  return ISING_OK;
}

// Orders the pack's stream after the work already queued on every member's
// own stream (set-up, earlier steps).
int wait_for_members(ising_pack* pk) {
  for (ising_ds* ds : pk->members) {
    if (ds->ctx->stream == pk->ctx->stream) continue;
    ISING_CUDA(pk->ctx, cudaEventRecord(pk->ev, ds->ctx->stream));
    ISING_CUDA(pk->ctx, cudaStreamWaitEvent(pk->ctx->stream, pk->ev, 0));
  }
  return ISING_OK;
}

// Orders every member's stream after the pack's work so far.
int members_wait(ising_pack* pk) {
  ISING_CUDA(pk->ctx, cudaEventRecord(pk->ev, pk->ctx->stream));
  for (ising_ds* ds : pk->members)
    if (ds->ctx->stream != pk->ctx->stream)
      ISING_CUDA(pk->ctx, cudaStreamWaitEvent(ds->ctx->stream, pk->ev, 0));
  return ISING_OK;
}

}  // namespace

namespace ising {

// Queues `steps` steps of every member on the pack's stream (no wait).
int pack_advance(ising_pack* pk, int64_t steps) {
  ising_ctx* ctx = pk->ctx;
  for (ising_ds* ds : pk->members)
    if (ds->finished || steps > ds->T - ds->t)
      return fail(ctx, ISING_EINVAL, "pack: a member has fewer than %lld steps left",
                  (long long)steps);
  ISING_TRY(wait_for_members(pk));
  int64_t s = 0;
  // the first steps run outside capture (the kernels' attributes are set
  // on their first launch), then graph replays, then single steps; the
  // graph is captured once the pack is advanced a second time (a pack that
  // lives for one call does not pay for a capture)
  const bool replay = pk->advances > 0;
  while (s < steps) {
    if (replay && pk->launched && steps - s >= kPackGraphSteps) {
      if (!pk->graph) ISING_TRY(pack_graph(pk));
      ISING_CUDA(ctx, cudaEventRecord(pk->ev, ctx->stream));
      ISING_CUDA(ctx, cudaStreamWaitEvent(pk->gstream, pk->ev, 0));
      ISING_CUDA(ctx, cudaGraphLaunch(pk->graph, pk->gstream));
      ISING_CUDA(ctx, cudaEventRecord(pk->ev, pk->gstream));
      ISING_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, pk->ev, 0));
      s += kPackGraphSteps;
    } else {
      ISING_TRY(pack_step(pk));
      s += 1;
      pk->launched = true;
    }
  }
  // the last step's tracking (its launch tracked only its predecessor)
  if (pk->fold && steps > 0)
    ISING_TRY(track_pack(ctx, pk->spin_kind, pk->targs.as<TrackArgs>(), pk->rstart.as<int64_t>(),
                         (int)pk->members.size(), pk->restarts, pk->words.as<unsigned long long>(),
                         true));
  for (ising_ds* ds : pk->members) ds->t += steps;
  pk->advances += 1;
  return members_wait(pk);
}

// Whether a bounded wait of a packed launch gave up (synchronises).
int pack_error(ising_pack* pk) {
  int e = 0;
  ISING_CUDA(pk->ctx, cudaMemcpyAsync(&e, pk->words.as<unsigned long long>() + 1, 4,
                                      cudaMemcpyDeviceToHost, pk->ctx->stream));
  ISING_CUDA(pk->ctx, cudaStreamSynchronize(pk->ctx->stream));
  if (e) return fail(pk->ctx, ISING_ETIMEOUT, "packed step: a bounded wait gave up (role %d)", e);
  return ISING_OK;
}

}  // namespace ising

extern "C" int ising_pack_create(ising_ctx* ctx, ising_ds* const* sessions, int32_t count,
                                 ising_pack** out) {
  if (!ctx) return ISING_EINVAL;
  if (!out || !sessions || count < 1 || count > 4096)
    return fail(ctx, ISING_EINVAL, "pack: 1 to 4096 sessions are required");
  *out = nullptr;
  uint64_t key = 0;
  for (int k = 0; k < count; ++k) {
    ising_ds* ds = sessions[k];
    if (!ds || !tc_packable(ds))
      return fail(ctx, ISING_ENOTSUP,
                  "pack: member %d is not a tensor-core session in the streaming form "
                  "(create it with ISING_DS_STREAMING, rounded product)", k);
    if (ds->ctx->device != ctx->device) return fail(ctx, ISING_EINVAL, "pack: members on another device");
    for (int j = 0; j < k; ++j)
      if (sessions[j] == ds) return fail(ctx, ISING_EINVAL, "pack: session %d appears twice", k);
    const uint64_t kk = tc_pack_key(ds);
    if (k == 0) key = kk;
    else if (kk != key)
      return fail(ctx, ISING_EINVAL, "pack: members differ in operand type, energy mode or J planes (member %d)", k);
  }
  auto pk = new ising_pack();
  pk->ctx = ctx;
  // members by size, largest first: their tiles then come in decreasing cost
  // (K = n), which the packed launch's wave-by-wave tile order spreads evenly
  pk->members.assign(sessions, sessions + count);
  std::stable_sort(pk->members.begin(), pk->members.end(),
                   [](const ising_ds* a, const ising_ds* b) { return a->n > b->n; });
  pk->key = key;
  pk->bn = pack_width(ctx, sessions, count);
  pk->spin_kind = sessions[0]->spin_kind;
  pk->fold = true;
  for (int k = 0; k < count; ++k)
    if (sessions[k]->conv.p) pk->fold = false;  // retired tiles read the tracked counts
  int rc = [&]() -> int {
    ISING_CUDA(ctx, cudaEventCreateWithFlags(&pk->ev, cudaEventDisableTiming));
    const size_t eb = tc_pack_entry_bytes();
    std::vector<unsigned char> ent(eb * count);
    std::vector<int> start(count + 1, 0);
    std::vector<TrackArgs> targs(count);
    std::vector<int64_t> rstart(count + 1, 0);
    for (int k = 0; k < count; ++k) {
      ising_ds* ds = pk->members[k];
      // one tile width for all: the results do not depend on it
      ISING_TRY(tc_set_bn(ds, pk->bn));
      ISING_TRY(tc_pack_entry(ds, ent.data() + eb * k));
      start[k + 1] = start[k] + ceil_div_i(ds->n, 128) * ceil_div_i(ds->B, pk->bn);
      targs[k] = track_args(ds);
      rstart[k + 1] = rstart[k] + ds->B;
    }
    pk->tiles = start[count];
    pk->restarts = rstart[count];
    ISING_TRY(dev_alloc(ctx, pk->entries, ent.size()));
    ISING_TRY(dev_alloc(ctx, pk->start, start.size() * sizeof(int)));
    ISING_TRY(dev_alloc(ctx, pk->targs, targs.size() * sizeof(TrackArgs)));
    ISING_TRY(dev_alloc(ctx, pk->rstart, rstart.size() * sizeof(int64_t)));
    ISING_TRY(dev_alloc(ctx, pk->words, 16));
    // the tables travel as kernel parameters: nothing here waits for the
    // stream's earlier work (other packs' steps on a shared stream)
    ISING_TRY(upload_async(ctx, pk->entries.p, ent.data(), ent.size()));
    ISING_TRY(upload_async(ctx, pk->start.p, start.data(), start.size() * sizeof(int)));
    ISING_TRY(upload_async(ctx, pk->targs.p, targs.data(), targs.size() * sizeof(TrackArgs)));
    ISING_TRY(upload_async(ctx, pk->rstart.p, rstart.data(), rstart.size() * sizeof(int64_t)));
    ISING_CUDA(ctx, cudaMemsetAsync(pk->words.p, 0, 16, ctx->stream));
    return ISING_OK;
  }();
  if (rc != ISING_OK) {
    ising_pack_destroy(pk);
    return rc;
  }
  *out = pk;
  return ISING_OK;
}

extern "C" int ising_pack_run(ising_pack* pk, int64_t steps) {
  if (!pk) return ISING_EINVAL;
  if (steps < 0) return fail(pk->ctx, ISING_EINVAL, "steps must be >= 0");
  if (steps == 0) return ISING_OK;
  NvtxRange range("ising_pack_run");
  ISING_TRY(pack_advance(pk, steps));
  return pack_error(pk);
}

// Nothing waits here: the pack's buffers are freed in stream order after its
// launches, and a stream or event destroyed with work pending is released
// once that work completes.
extern "C" int ising_pack_destroy(ising_pack* pk) {
  if (!pk) return ISING_OK;
  if (pk->graph) cudaGraphExecDestroy(pk->graph);
  if (pk->gstream) cudaStreamDestroy(pk->gstream);
  if (pk->ev) cudaEventDestroy(pk->ev);
  delete pk;
  return ISING_OK;
}
