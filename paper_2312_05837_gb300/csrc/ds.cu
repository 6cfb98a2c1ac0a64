// Domain selection (Sec. III-B): session management shared by every path,
// initialisation theta = asin(x0), best tracking per restart (K4 part 1),
// best-of-restarts reduction (K4 part 2) and the public C ABI calls.
#include "ds_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <fstream>
#include <limits>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

using namespace ising;

namespace ising {
namespace {

// asin(x) to FP32 accuracy from a double x: directly for |x| <= 1/2, else by
// asin(x) = pi/2 - 2 asin(sqrt((1 - |x|) / 2)) with 1 - |x| formed exactly in
// FP64 (the direct form loses accuracy near |x| = 1 where its slope blows up).
// The sign of x is kept (x0 is 0 or at least 2^-52 in magnitude).
__device__ __forceinline__ float asin_of(double x) {
  const double ax = fabs(x);
  float r;
  if (ax <= 0.5) {
    r = asinf((float)ax);
  } else {
    const float y = (float)((1.0 - ax) * 0.5);
    r = 1.57079632679489662f - 2.0f * asinf(sqrtf(y));
  }
  return x < 0.0 ? -r : r;
}

// theta_0 = asin(x0), x0 = SplitMix64(seed, (b << 32) | i) mapped to [-1, 1);
// m = v = 0; S_1 = sgn+(x0). Dense state is [Bp][ld] restart-major, sparse
// state [n][Bp].
template <int KIND>
__global__ void init_kernel(int64_t n, int64_t Bp, int64_t ld, bool spin_major, uint64_t seed,
                            float* __restrict__ theta, float* __restrict__ m,
                            float* __restrict__ v, void* __restrict__ spins) {
  const int64_t total = spin_major ? n * Bp : Bp * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b, i;
    if (spin_major) { i = e / Bp; b = e - i * Bp; } else { b = e / ld; i = e - b * ld; }
    float th = 0.0f;
    bool pos = true;
    bool pad = i >= n;
    if (!pad) {
      uint64_t z = splitmix64(seed, ((uint64_t)b << 32) | (uint64_t)i);
      double x0 = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
      th = asin_of(x0);
      pos = x0 >= 0.0;
    }
    theta[e] = th;
    m[e] = 0.0f;
    v[e] = 0.0f;
    if (KIND == kSpinF32) {
      static_cast<float*>(spins)[e] = pad ? 0.0f : (pos ? 1.0f : -1.0f);
    } else if (KIND == kSpinBF16) {
      static_cast<__nv_bfloat16*>(spins)[e] = __float2bfloat16(pad ? 0.0f : (pos ? 1.0f : -1.0f));
    } else if (KIND == kSpinF16) {
      // FP16: +1 = 0x3C00, -1 = 0xBC00
      static_cast<uint16_t*>(spins)[e] = pad ? 0 : (pos ? 0x3C00 : 0xBC00);
    } else if (KIND == kSpinE4M3) {
      // E4M3: +1 = 0x38, -1 = 0xB8, 0 = 0x00
      static_cast<uint8_t*>(spins)[e] = pad ? 0 : (pos ? 0x38 : 0xB8);
    }
  }
}

// Bit-packed spins for the sparse path: word w of spin i holds restarts
// 32w .. 32w+31, bit set = +1.
__global__ void init_bits_kernel(int64_t n, int64_t Bp, uint64_t seed,
                                 uint32_t* __restrict__ bits) {
  const int64_t words = Bp / 32;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * words;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / words, w = e - i * words;
    uint32_t word = 0;
    for (int r = 0; r < 32; ++r) {
      uint64_t b = (uint64_t)(w * 32 + r);
      uint64_t z = splitmix64(seed, (b << 32) | (uint64_t)i);
      double x0 = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
      if (x0 >= 0.0) word |= 1u << r;
    }
    bits[e] = word;
  }
}

template <int KIND>
__device__ __forceinline__ int8_t spin_at(const void* spins, int64_t n, int64_t Bp, int64_t ld,
                                          int64_t b, int64_t i) {
  if (KIND == kSpinF32) return static_cast<const float*>(spins)[b * ld + i] > 0.0f ? 1 : -1;
  if (KIND == kSpinBF16 || KIND == kSpinF16)  // +-1 in either 16-bit type: the sign bit
    return (static_cast<const uint16_t*>(spins)[b * ld + i] & 0x8000u) ? -1 : 1;
  if (KIND == kSpinE4M3) return static_cast<const uint8_t*>(spins)[b * ld + i] == 0x38 ? 1 : -1;
  const uint32_t w = static_cast<const uint32_t*>(spins)[i * (Bp / 32) + (b >> 5)];
  return (w >> (b & 31)) & 1u ? 1 : -1;
}

// Best tracking for step t = counters[0] + 1 of one session, one warp per
// restart; the last block advances the step counter and records t as
// tracked (counters[2]). With A.flush, the step the counter names (already
// advanced by a step launch that tracks its predecessor) is tracked unless
// counters[2] says it has been, and only counters[2] changes.
template <int KIND>
__global__ void __launch_bounds__(256) track_kernel(const TrackArgs A) {
  const long long t = A.counters[0] + (A.flush ? 0 : 1);
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  if (t >= 1 && t > A.counters[2])
    for (int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); b < A.B;
         b += warps)
      track_restart<KIND>(A, t, b, lane);
  __shared__ bool last;
  __syncthreads();
  __threadfence();
  if (threadIdx.x == 0) {
    unsigned long long prev = atomicAdd(reinterpret_cast<unsigned long long*>(&A.counters[1]), 1ull);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    // (every block has read counters[0] and [2] by now)
    A.counters[0] = t;
    if (t > A.counters[2]) A.counters[2] = t;
    A.counters[1] = 0;
    __threadfence();
  }
}

// Best tracking of every member of a pack, each at its own step t =
// counters[0] + 1: member e owns the restarts [rstart[e], rstart[e + 1]) of
// the launch, one warp per restart; the last block advances every member's
// step counter (`done` counts finished blocks and is reset). With `flush`,
// each member at t = counters[0], the counters left alone.
template <int KIND>
__global__ void __launch_bounds__(256) track_pack_kernel(const TrackArgs* __restrict__ M,
                                                         const int64_t* __restrict__ rstart,
                                                         int count, unsigned long long* done,
                                                         bool flush) {
  const int lane = threadIdx.x & 31;
  const int64_t total = rstart[count];
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < total;
       g += warps) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rstart[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const TrackArgs& A = M[lo];
    const long long t = A.counters[0] + (flush ? 0 : 1);
    if (t >= 1 && t > A.counters[2]) track_restart<KIND>(A, t, g - rstart[lo], lane);
  }
  __shared__ bool last;
  __syncthreads();
  __threadfence();
  if (threadIdx.x == 0) last = atomicAdd(done, 1ull) == gridDim.x - 1;
  __syncthreads();
  if (last) {
    // (every block has read the counters by now) each member's tracked step
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
      long long* c = M[e].counters;
      const long long t = c[0] + (flush ? 0 : 1);
      c[0] = t;
      if (t > c[2]) c[2] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *done = 0;
      __threadfence();
    }
  }
}

// Copy of S_t into best_s for the restarts that improved at step t, for the
// bit-packed spins of the sparse path (the flags come from track_kernel). A
// warp task is one spin word column w (restarts 32w .. 32w + 31) over 32
// consecutive spins: a lane loads the word of its spin and writes bit r of it
// to row 32w + r of best_s for every improved r, so each store of the warp
// covers 32 consecutive bytes of one row.
__global__ void __launch_bounds__(256) track_bits_copy_kernel(
    int64_t n, int64_t B, int64_t words, const uint32_t* __restrict__ bits,
    const uint8_t* __restrict__ improved, int8_t* __restrict__ best_s, int64_t bs_ld) {
  const int lane = threadIdx.x & 31;
  const int64_t chunks = (n + 31) / 32;
  const int64_t tasks = chunks * words;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < tasks;
       task += nwarps) {
    const int64_t w = task / chunks;
    const int64_t i = (task - w * chunks) * 32 + lane;
    const int64_t b = w * 32 + lane;
    const unsigned int mask = __ballot_sync(0xffffffffu, b < B && improved[b] != 0);
    if (!mask) continue;
    if (i >= n) continue;
    const uint32_t word = bits[i * words + w];
    for (unsigned int m = mask; m; m &= m - 1) {
      const int r = __ffs(m) - 1;
      best_s[(w * 32 + r) * bs_ld + i] = ((word >> r) & 1u) ? 1 : -1;
    }
  }
}

template <int KIND>
__global__ void export_spins_kernel(int64_t n, int64_t B, int64_t Bp, int64_t ld,
                                    const void* __restrict__ spins, int8_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < B * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / n, i = e - b * n;
    out[e] = spin_at<KIND>(spins, n, Bp, ld, b, i);
  }
}

// [n][Bp] <-> [B][n] transposes for the sparse path's state.
__global__ void spin_major_to_restart_major(int64_t n, int64_t B, int64_t Bp,
                                            const float* __restrict__ in, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < B * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / n, i = e - b * n;
    out[e] = in[i * Bp + b];
  }
}

__global__ void restart_major_to_spin_major(int64_t n, int64_t B, int64_t Bp,
                                            const float* __restrict__ in, float* __restrict__ out,
                                            bool wrap) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < B * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / n, i = e - b * n;
    float x = in[e];
    out[i * Bp + b] = wrap ? wrap_angle(x) : x;
  }
}

__global__ void wrap_rows_kernel(int64_t n, int64_t B, int64_t ld, float* __restrict__ th) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < B * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / n, i = e - b * n;
    th[b * ld + i] = wrap_angle(th[b * ld + i]);
  }
}

// Spins from theta (restart-major dense state) into a spin slot.
template <int KIND>
__global__ void spins_from_theta_dense(int64_t n, int64_t Bp, int64_t ld,
                                       const float* __restrict__ th, void* __restrict__ spins) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Bp * ld;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % ld;
    bool pad = i >= n;
    bool pos = sin_nonneg(th[e]);
    if (KIND == kSpinF32) static_cast<float*>(spins)[e] = pad ? 0.f : (pos ? 1.f : -1.f);
    if (KIND == kSpinBF16)
      static_cast<__nv_bfloat16*>(spins)[e] = __float2bfloat16(pad ? 0.f : (pos ? 1.f : -1.f));
    if (KIND == kSpinF16) static_cast<uint16_t*>(spins)[e] = pad ? 0 : (pos ? 0x3C00 : 0xBC00);
    if (KIND == kSpinE4M3) static_cast<uint8_t*>(spins)[e] = pad ? 0 : (pos ? 0x38 : 0xB8);
  }
}

// Relaxed spins x = sin(theta) of the state (any layout; `ld` > 0 marks the
// restart-major dense layout, whose padding columns i >= n stay 0) as FP32
// or in the tensor cores' 16-bit type (kind 1 BF16, 2 FP16; 0 FP32).
__global__ void x_from_theta(int64_t count, int64_t n, int64_t ld, int kind,
                             const float* __restrict__ th, void* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool pad = ld > 0 && e % ld >= n;
    const float v = pad ? 0.f : sin_proj(th[e]);
    if (kind == 1) static_cast<__nv_bfloat16*>(x)[e] = __float2bfloat16(v);
    else if (kind == 2) static_cast<__half*>(x)[e] = __float2half_rn(v);
    else static_cast<float*>(x)[e] = v;
  }
}

__global__ void spins_from_theta_bits(int64_t n, int64_t Bp, const float* __restrict__ th,
                                      uint32_t* __restrict__ bits) {
  const int64_t words = Bp / 32;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * words;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / words, w = e - i * words;
    uint32_t word = 0;
    for (int r = 0; r < 32; ++r)
      if (sin_nonneg(th[i * Bp + w * 32 + r])) word |= 1u << r;
    bits[e] = word;
  }
}

__global__ void fill_double(double* p, int64_t count, double x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = x;
}

// K4: lowest (energy, restart) over B restarts; one block, fixed reduction tree.
__global__ void __launch_bounds__(1024) argmin_kernel(int64_t B, const double* __restrict__ E,
                                                      long long* __restrict__ out) {
  __shared__ double se[1024];
  __shared__ long long sb[1024];
  double be = INFINITY;
  long long bb = -1;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
    double e = E[b];
    if (bb < 0 || e < be) { be = e; bb = b; }
  }
  se[threadIdx.x] = be;
  sb[threadIdx.x] = bb;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double e2 = se[threadIdx.x + s];
      long long b2 = sb[threadIdx.x + s];
      if (b2 >= 0 && (sb[threadIdx.x] < 0 || e2 < se[threadIdx.x] ||
                      (e2 == se[threadIdx.x] && b2 < sb[threadIdx.x]))) {
        se[threadIdx.x] = e2;
        sb[threadIdx.x] = b2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sb[0];
}

int grid1d(ising_ctx* ctx, int64_t work) {
  int64_t g = (work + 255) / 256;
  int64_t cap = (int64_t)std::max(ctx->sm_count, 1) * 16;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

int check_params(ising_ctx* ctx, const ising_ds_params* p) {
  if (!p) return fail(ctx, ISING_EINVAL, "params is NULL");
  if (p->restarts < 1 || p->restarts > (1 << 20))
    return fail(ctx, ISING_EINVAL, "restarts must be in [1, 2^20]");
  if (p->steps < 0) return fail(ctx, ISING_EINVAL, "steps must be >= 0");
  if (!std::isfinite(p->lr) || p->lr < 0) return fail(ctx, ISING_EINVAL, "lr must be finite and >= 0");
  if (!std::isfinite(p->mu) || p->mu < 0) return fail(ctx, ISING_EINVAL, "mu must be finite and >= 0");
  if (!(p->beta1 >= 0 && p->beta1 < 1) || !(p->beta2 >= 0 && p->beta2 < 1))
    return fail(ctx, ISING_EINVAL, "beta1 and beta2 must lie in [0, 1)");
  if (!(p->eps > 0) || !std::isfinite(p->eps)) return fail(ctx, ISING_EINVAL, "eps must be > 0");
  if (p->flags & ~(ISING_DS_PROFILE | ISING_DS_STREAMING | ISING_DS_NO_AUTOTUNE |
                   ISING_DS_CONVERGE | ISING_DS_RELAXED))
    return fail(ctx, ISING_EINVAL, "unknown flags");
  if (p->precision < ISING_PREC_AUTO || p->precision > ISING_PREC_FP8)
    return fail(ctx, ISING_EINVAL, "unknown precision %d", p->precision);
  return ISING_OK;
}

}  // namespace

TrackArgs track_args(const ising_ds* ds) {
  TrackArgs A;
  A.n = ds->n;
  A.B = ds->B;
  A.Bp = ds->Bp;
  A.ld = ds->ld;
  A.mtiles = ds->mtiles;
  A.int_mode = ds->int_energy;
  A.cq = ds->inst.cq;
  A.chs = ds->inst.ch * std::ldexp(1.0, -ds->h_shift);
  for (int k = 0; k < 2; ++k) {
    A.qpart[k] = ds->qpart[k].as<long long>();
    A.hpart[k] = ds->hpart[k].as<long long>();
    A.epart[k] = ds->epart[k].as<float>();
  }
  for (int k = 0; k < 3; ++k) A.spins[k] = ds->spins[k].p;
  A.best_E = ds->best_E.as<double>();
  A.best_t = ds->best_t.as<long long>();
  A.best_s = ds->best_s.as<int8_t>();
  A.last_E = ds->last_E.as<double>();
  A.counters = ds->counters.as<long long>();
  A.bs_ld = ds->bs_ld;
  A.improved = ds->improved.as<uint8_t>();
  A.T = ds->T;
  const bool conv = ds->conv.p != nullptr;
  A.conv_ring = conv ? ds->conv_ring() : nullptr;
  A.conv_init = conv ? ds->conv_init() : nullptr;
  A.conv_step = conv ? ds->conv_step() : nullptr;
  A.conv_count = conv ? ds->conv_count() : nullptr;
  A.live32 = conv ? ds->live.as<int>() : nullptr;
  A.inline_bits = false;
  A.flush = false;
  return A;
}

// Bit-packed spins up to this many per restart are copied by the tracking
// warps themselves (one launch less per step for small instances).
constexpr int64_t kInlineBitsMaxN = 4096;

int track_step(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  const int slot = (int)((ds->t + 1) % 3);
  int grid = (int)std::min<int64_t>((ds->B + 7) / 8, (int64_t)ctx->sm_count * 4);
  const TrackArgs A = track_args(ds);
  switch (ds->spin_kind) {
    case kSpinF32: track_kernel<kSpinF32><<<grid, 256, 0, ctx->stream>>>(A); break;
    case kSpinBF16:
    case kSpinF16: track_kernel<kSpinBF16><<<grid, 256, 0, ctx->stream>>>(A); break;  // sign bits
    case kSpinE4M3: track_kernel<kSpinE4M3><<<grid, 256, 0, ctx->stream>>>(A); break;
    default: {
      if (ds->n <= kInlineBitsMaxN) {
        // small instances: each improved restart's spins copied by its warp
        TrackArgs Ai = A;
        Ai.inline_bits = true;
        track_kernel<kSpinBits><<<grid, 256, 0, ctx->stream>>>(Ai);
        break;
      }
      track_kernel<kSpinBits><<<grid, 256, 0, ctx->stream>>>(A);
      const int64_t words = ds->Bp / 32;
      const int64_t tasks = (ds->n + 31) / 32 * words;
      const int cgrid = (int)std::max<int64_t>(
          1, std::min<int64_t>((tasks + 7) / 8, (int64_t)ctx->sm_count * 8));
      track_bits_copy_kernel<<<cgrid, 256, 0, ctx->stream>>>(
          ds->n, ds->B, words, ds->spins[slot].as<uint32_t>(), ds->improved.as<uint8_t>(),
          ds->best_s.as<int8_t>(), ds->bs_ld);
      break;
    }
  }
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

int track_flush(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  const int grid = (int)std::min<int64_t>((ds->B + 7) / 8, (int64_t)ctx->sm_count * 4);
  TrackArgs A = track_args(ds);
  A.flush = true;
  switch (ds->spin_kind) {
    case kSpinE4M3: track_kernel<kSpinE4M3><<<grid, 256, 0, ctx->stream>>>(A); break;
    case kSpinBF16:
    case kSpinF16: track_kernel<kSpinBF16><<<grid, 256, 0, ctx->stream>>>(A); break;
    default: return fail(ctx, ISING_EINVAL, "tracking flush: spin kind %d", ds->spin_kind);
  }
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

int track_pack(ising_ctx* ctx, int spin_kind, const TrackArgs* members, const int64_t* rstart,
               int count, int64_t total_restarts, unsigned long long* done, bool flush) {
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((total_restarts + 7) / 8, (int64_t)ctx->sm_count * 4));
  switch (spin_kind) {
    case kSpinE4M3:
      track_pack_kernel<kSpinE4M3><<<grid, 256, 0, ctx->stream>>>(members, rstart, count, done, flush);
      break;
    case kSpinBF16:
    case kSpinF16:
      track_pack_kernel<kSpinBF16><<<grid, 256, 0, ctx->stream>>>(members, rstart, count, done, flush);
      break;
    default: return fail(ctx, ISING_ENOTSUP, "packed tracking: dense spin slots only");
  }
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

int export_spins_int8(ising_ds* ds, int slot, int8_t* out) {
  ising_ctx* ctx = ds->ctx;
  int g = grid1d(ctx, ds->B * ds->n);
  const void* sp = ds->spins[slot].p;
  switch (ds->spin_kind) {
    case kSpinF32: export_spins_kernel<kSpinF32><<<g, 256, 0, ctx->stream>>>(ds->n, ds->B, ds->Bp, ds->ld, sp, out); break;
    case kSpinBF16:
    case kSpinF16: export_spins_kernel<kSpinBF16><<<g, 256, 0, ctx->stream>>>(ds->n, ds->B, ds->Bp, ds->ld, sp, out); break;
    case kSpinE4M3: export_spins_kernel<kSpinE4M3><<<g, 256, 0, ctx->stream>>>(ds->n, ds->B, ds->Bp, ds->ld, sp, out); break;
    default: export_spins_kernel<kSpinBits><<<g, 256, 0, ctx->stream>>>(ds->n, ds->B, ds->Bp, ds->ld, sp, out); break;
  }
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

namespace {

// x = sin(theta) of the current state into relaxed slot `slot`.
int derive_x(ising_ds* ds, int slot) {
  ising_ctx* ctx = ds->ctx;
  const bool dense = ds->path != ISING_PATH_SPARSE;
  const int64_t count = dense ? ds->Bp * ds->ld : ds->n * ds->Bp;
  x_from_theta<<<grid1d(ctx, count), 256, 0, ctx->stream>>>(
      count, ds->n, dense ? ds->ld : 0,
      ds->path == ISING_PATH_TC ? (ds->spin_kind == kSpinF16 ? 2 : 1) : 0, ds->theta.as<float>(),
      ds->xbuf[slot].p);
  ISING_CUDA(ctx, cudaGetLastError());
  return ISING_OK;
}

int init_state(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  const bool spin_major = ds->path == ISING_PATH_SPARSE;
  const int64_t elems = spin_major ? ds->n * ds->Bp : ds->Bp * ds->ld;
  ISING_TRY(dev_alloc(ctx, ds->theta, elems * 4));
  ISING_TRY(dev_alloc(ctx, ds->m, elems * 4));
  ISING_TRY(dev_alloc(ctx, ds->v, elems * 4));
  size_t spin_bytes;
  switch (ds->spin_kind) {
    case kSpinF32: spin_bytes = elems * 4; break;
    case kSpinBF16:
    case kSpinF16: spin_bytes = elems * 2; break;
    case kSpinE4M3: spin_bytes = elems; break;
    default: spin_bytes = ds->n * (ds->Bp / 32) * 4; break;
  }
  for (auto& s : ds->spins) {
    ISING_TRY(dev_alloc(ctx, s, spin_bytes));
    ISING_CUDA(ctx, cudaMemsetAsync(s.p, 0, spin_bytes, ctx->stream));
  }
  const int slot1 = 1;  // S_1 lives in spins[1 % 3]
  int g = grid1d(ctx, elems);
  float* th = ds->theta.as<float>();
  float* mm = ds->m.as<float>();
  float* vv = ds->v.as<float>();
  void* s1 = ds->spins[slot1].p;
  uint64_t seed = ds->p.seed;
  switch (ds->spin_kind) {
    case kSpinF32: init_kernel<kSpinF32><<<g, 256, 0, ctx->stream>>>(ds->n, ds->Bp, ds->ld, false, seed, th, mm, vv, s1); break;
    case kSpinBF16: init_kernel<kSpinBF16><<<g, 256, 0, ctx->stream>>>(ds->n, ds->Bp, ds->ld, false, seed, th, mm, vv, s1); break;
    case kSpinF16: init_kernel<kSpinF16><<<g, 256, 0, ctx->stream>>>(ds->n, ds->Bp, ds->ld, false, seed, th, mm, vv, s1); break;
    case kSpinE4M3: init_kernel<kSpinE4M3><<<g, 256, 0, ctx->stream>>>(ds->n, ds->Bp, ds->ld, false, seed, th, mm, vv, s1); break;
    default:
      init_kernel<kSpinBits><<<g, 256, 0, ctx->stream>>>(ds->n, ds->Bp, ds->ld, true, seed, th, mm, vv, nullptr);
      init_bits_kernel<<<grid1d(ctx, ds->n * ds->Bp / 32), 256, 0, ctx->stream>>>(
          ds->n, ds->Bp, seed, ds->spins[slot1].as<uint32_t>());
      break;
  }
  ISING_CUDA(ctx, cudaGetLastError());
  if (ds->relaxed()) {
    const size_t xb = (size_t)elems * (ds->path == ISING_PATH_TC ? 2 : 4);
    for (auto& x : ds->xbuf) {
      ISING_TRY(dev_alloc(ctx, x, xb));
      ISING_CUDA(ctx, cudaMemsetAsync(x.p, 0, xb, ctx->stream));
    }
    ISING_TRY(derive_x(ds, 1));  // x_1 = sin(theta_0)
  }
  return ISING_OK;
}

int common_alloc(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  const int64_t B = ds->B, n = ds->n;
  for (int s = 0; s < 2; ++s) {
    ISING_TRY(dev_alloc(ctx, ds->qpart[s], (size_t)ds->mtiles * ds->Bp * 8));
    ISING_TRY(dev_alloc(ctx, ds->hpart[s], (size_t)ds->mtiles * ds->Bp * 8));
    ISING_TRY(dev_alloc(ctx, ds->epart[s], (size_t)ds->mtiles * ds->Bp * 4));
    ISING_CUDA(ctx, cudaMemsetAsync(ds->hpart[s].p, 0, ds->hpart[s].bytes, ctx->stream));
  }
  ISING_TRY(dev_alloc(ctx, ds->best_E, B * 8));
  ISING_TRY(dev_alloc(ctx, ds->best_t, B * 8));
  ds->bs_ld = (n + 15) / 16 * 16;
  ISING_TRY(dev_alloc(ctx, ds->best_s, (size_t)B * ds->bs_ld));
  ISING_TRY(dev_alloc(ctx, ds->last_E, B * 8));
  ISING_TRY(dev_alloc(ctx, ds->improved, B));
  if (ds->p.flags & ISING_DS_CONVERGE) {
    ISING_TRY(dev_alloc(ctx, ds->conv, (size_t)(7 * B + 1) * 8));
    ISING_CUDA(ctx, cudaMemsetAsync(ds->conv.p, 0, ds->conv.bytes, ctx->stream));
    const int64_t nb = (B + 31) / 32;
    std::vector<int> live(nb);
    for (int64_t k = 0; k < nb; ++k) live[k] = (int)std::min<int64_t>(32, B - 32 * k);
    ISING_TRY(dev_alloc(ctx, ds->live, nb * 4));
    ISING_TRY(upload_async(ctx, ds->live.p, live.data(), nb * 4));
  }
  ISING_TRY(dev_alloc(ctx, ds->work, 8));
  ISING_CUDA(ctx, cudaMemsetAsync(ds->work.p, 0, 8, ctx->stream));
  ISING_TRY(dev_alloc(ctx, ds->counters, 32));
  ISING_TRY(dev_alloc(ctx, ds->scratch, 64));
  fill_double<<<grid1d(ctx, B), 256, 0, ctx->stream>>>(ds->best_E.as<double>(), B, INFINITY);
  fill_double<<<grid1d(ctx, B), 256, 0, ctx->stream>>>(ds->last_E.as<double>(), B, INFINITY);
  ISING_CUDA(ctx, cudaGetLastError());
  ISING_CUDA(ctx, cudaMemsetAsync(ds->best_t.p, 0, B * 8, ctx->stream));
  ISING_CUDA(ctx, cudaMemsetAsync(ds->best_s.p, 0, (size_t)B * ds->bs_ld, ctx->stream));
  ISING_CUDA(ctx, cudaMemsetAsync(ds->counters.p, 0, 32, ctx->stream));
  // Adam bias corrections for t = 0 .. T + 1 (entry 0 unused)
  std::vector<float> bias((size_t)(ds->T + 2) * 2);
  for (int64_t t = 1; t <= ds->T + 1; ++t) {
    bias[2 * t] = (float)(1.0 / (1.0 - std::pow(ds->p.beta1, (double)t)));
    bias[2 * t + 1] = (float)(1.0 / (1.0 - std::pow(ds->p.beta2, (double)t)));
  }
  bias[0] = bias[1] = 1.0f;
  ISING_TRY(dev_alloc(ctx, ds->bias, bias.size() * 4));
  return upload_async(ctx, ds->bias.p, bias.data(), bias.size() * 4);
}

int setup_field(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  const int64_t n = ds->n;
  ISING_TRY(dev_alloc(ctx, ds->hf, n * 4));
  ISING_TRY(dev_alloc(ctx, ds->hint, n * 4));
  ISING_CUDA(ctx, cudaMemsetAsync(ds->hf.p, 0, n * 4, ctx->stream));
  ISING_CUDA(ctx, cudaMemsetAsync(ds->hint.p, 0, n * 4, ctx->stream));
  if (!ds->inst.has_h) return ISING_OK;
  std::vector<double> h(n);
  size_t es = dtype_size(ds->inst.h_dtype);
  std::vector<unsigned char> raw(n * es);
  ISING_CUDA(ctx, cudaMemcpyAsync(raw.data(), ds->inst.h.p, n * es, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int64_t i = 0; i < n; ++i) {
    switch (ds->inst.h_dtype) {
      case ISING_F64: h[i] = reinterpret_cast<double*>(raw.data())[i]; break;
      case ISING_F32: h[i] = reinterpret_cast<float*>(raw.data())[i]; break;
      default: h[i] = reinterpret_cast<int32_t*>(raw.data())[i]; break;
    }
  }
  std::vector<float> hf(n);
  std::vector<int32_t> hi(n);
  for (int64_t i = 0; i < n; ++i) {
    hf[i] = (float)h[i];
    hi[i] = ds->int_energy ? (int32_t)std::llrint(std::ldexp(h[i], ds->h_shift)) : 0;
  }
  ISING_TRY(upload_async(ctx, ds->hf.p, hf.data(), n * 4));
  return upload_async(ctx, ds->hint.p, hi.data(), n * 4);
}

int path_step_raw(ising_ds* ds, bool update) {
  if (update && ds->relaxed()) {
    // relaxed product: the sparse kernel gathers both spin forms at once; the
    // dense paths take the energies of the rounded spins in a pass of their own
    switch (ds->path) {
      case ISING_PATH_SPARSE: return sparse_step(ds, kModeRelaxed, nullptr);
      case ISING_PATH_PLAIN:
        ISING_TRY(plain_step(ds, kModeEnergy, nullptr));
        return plain_step(ds, kModeRelaxed, nullptr);
      default:
        ISING_TRY(tc_step(ds, kModeEnergy, nullptr));
        return tc_step(ds, kModeRelaxed, nullptr);
    }
  }
  const int mode = update ? kModeUpdate : kModeEnergy;
  switch (ds->path) {
    case ISING_PATH_PLAIN: return plain_step(ds, mode, nullptr);
    case ISING_PATH_SPARSE: return sparse_step(ds, mode, nullptr);
    default: return tc_step(ds, mode, nullptr);
  }
}

// One step kernel; with ISING_DS_PROFILE its device time is measured by a
// pair of events on the launching stream.
int path_step(ising_ds* ds, bool update) {
  if (!(ds->p.flags & ISING_DS_PROFILE)) return path_step_raw(ds, update);
  ising_ctx* ctx = ds->ctx;
  if (!ds->kev[0]) {
    ISING_CUDA(ctx, cudaEventCreate(&ds->kev[0]));
    ISING_CUDA(ctx, cudaEventCreate(&ds->kev[1]));
  }
  ISING_CUDA(ctx, cudaEventRecord(ds->kev[0], ctx->stream));
  ISING_TRY(path_step_raw(ds, update));
  ISING_CUDA(ctx, cudaEventRecord(ds->kev[1], ctx->stream));
  ISING_CUDA(ctx, cudaEventSynchronize(ds->kev[1]));
  float ms = 0.f;
  ISING_CUDA(ctx, cudaEventElapsedTime(&ms, ds->kev[0], ds->kev[1]));
  ds->kernel_ms += ms;
  ds->kernel_launches += 1;
  return ISING_OK;
}

int copy_out(ising_ctx* ctx, void* dst, const void* src, size_t bytes, int mem) {
  if (bytes == 0) return ISING_OK;
  ISING_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes,
                                  mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost
                                                        : cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  return ISING_OK;
}

// Overall best: K4 on the per-restart bests. With non-integer energies the
// tracked values are FP32-accurate, so every restart within a margin of the
// minimum is re-evaluated in FP64 (K3) and the lowest (energy, restart) of
// those re-evaluated values wins.
int select_best(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  argmin_kernel<<<1, 1024, 0, ctx->stream>>>(ds->B, ds->best_E.as<double>(),
                                             ds->scratch.as<long long>());
  ISING_CUDA(ctx, cudaGetLastError());
  long long bidx = -1;
  ISING_CUDA(ctx, cudaMemcpyAsync(&bidx, ds->scratch.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> bestE(ds->B), lastE(ds->B);
  ISING_CUDA(ctx, cudaMemcpyAsync(bestE.data(), ds->best_E.p, ds->B * 8, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaMemcpyAsync(lastE.data(), ds->last_E.p, ds->B * 8, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (bidx < 0) return fail(ctx, ISING_ECUDA, "best-of-restarts reduction found no restart");
  // the paper's literal output: best of the final spins
  ds->last_best_restart = 0;
  for (int64_t b = 1; b < ds->B; ++b)
    if (lastE[b] < lastE[ds->last_best_restart]) ds->last_best_restart = b;
  ds->last_best_energy = lastE[ds->last_best_restart];
  if (ds->int_energy) {
    ds->best_restart = bidx;
    ds->best_energy = bestE[bidx];
    return ISING_OK;
  }
  const double emin = bestE[bidx];
  const double margin = 1e-4 * std::fabs(emin) + 1e-9;
  std::vector<int64_t> cand;
  for (int64_t b = 0; b < ds->B; ++b)
    if (bestE[b] <= emin + margin) cand.push_back(b);
  std::sort(cand.begin(), cand.end(), [&](int64_t a, int64_t b) {
    return bestE[a] < bestE[b] || (bestE[a] == bestE[b] && a < b);
  });
  if (cand.size() > 64) cand.resize(64);
  DevMem rows, E;
  ISING_TRY(dev_alloc(ctx, rows, cand.size() * ds->n));
  ISING_TRY(dev_alloc(ctx, E, cand.size() * 8));
  for (size_t c = 0; c < cand.size(); ++c)
    ISING_CUDA(ctx, cudaMemcpyAsync(rows.as<int8_t>() + c * ds->n, ds->best_s.as<int8_t>() + cand[c] * ds->bs_ld,
                                    ds->n, cudaMemcpyDeviceToDevice, ctx->stream));
  ISING_TRY(energy_device(ctx, ds->inst, rows.as<int8_t>(), (int64_t)cand.size(), E.as<double>(),
                          nullptr, nullptr));
  std::vector<double> ex(cand.size());
  ISING_CUDA(ctx, cudaMemcpyAsync(ex.data(), E.p, cand.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  size_t w = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (ex[c] < ex[w] || (ex[c] == ex[w] && cand[c] < cand[w])) w = c;
  ds->best_restart = cand[w];
  ds->best_energy = ex[w];
  return ISING_OK;
}

}  // namespace
}  // namespace ising

// ------------------------------------------------------------------ C ABI

namespace ising {
int ds_create_impl(ising_ctx* ctx, const ising_instance* inst, const ising_ds_params* p,
                   ising_ds** out, bool validate);
}

extern "C" int ising_ds_create(ising_ctx* ctx, const ising_instance* inst,
                               const ising_ds_params* p, ising_ds** out) {
  return ising::ds_create_impl(ctx, inst, p, out, true);
}

int ising::ds_create_impl(ising_ctx* ctx, const ising_instance* inst, const ising_ds_params* p,
                          ising_ds** out, bool validate) {
  if (!ctx) return ISING_EINVAL;
  if (!out) return fail(ctx, ISING_EINVAL, "out is NULL");
  *out = nullptr;
  ISING_TRY(check_params(ctx, p));
  ISING_CUDA(ctx, cudaSetDevice(ctx->device));
  auto ds = new ising_ds();
  ds->ctx = ctx;
  ds->p = *p;
  int rc = [&]() -> int {
    ISING_TRY(upload_instance(ctx, inst, &ds->inst, validate));
    ds->n = ds->inst.n;
    ds->B = p->restarts;
    ds->T = p->steps;
    const DevInstance& I = ds->inst;
    // exact integer energies when every G = J s fits a float exactly
    ds->int_energy = I.j_integer && I.j_absmax * (double)ds->n < 4194304.0 && I.h_dyadic;
    ds->h_shift = I.h_shift;
    ds->k = StepConsts{(float)I.cq, (float)I.ch, (float)p->mu, (float)p->lr,
                       (float)p->beta1, (float)p->beta2, (float)p->eps,
                       (float)(1.0 - p->beta1), (float)(1.0 - p->beta2)};
    int prec = p->precision;
    if (I.layout == ISING_LAYOUT_CSR) {
      if (prec != ISING_PREC_AUTO && prec != ISING_PREC_FP32_PLAIN)
        return fail(ctx, ISING_ENOTSUP, "CSR instances run the sparse FP32/int path only");
      ds->path = ISING_PATH_SPARSE;
      ds->prec = ISING_PREC_FP32_PLAIN;
    } else if (prec == ISING_PREC_FP32_PLAIN) {
      ds->path = ISING_PATH_PLAIN;
      ds->prec = prec;
    } else {
      ds->path = ISING_PATH_TC;
      ds->prec = prec;  // AUTO is resolved by the tensor-core set-up
    }
    switch (ds->path) {
      case ISING_PATH_PLAIN: ISING_TRY(plain_setup(ds)); break;
      case ISING_PATH_SPARSE: ISING_TRY(sparse_setup(ds)); break;
      default: ISING_TRY(tc_setup(ds)); break;
    }
    ISING_TRY(setup_field(ds));
    ISING_TRY(common_alloc(ds));
    ISING_TRY(init_state(ds));
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ISING_OK;
  }();
  if (rc != ISING_OK) {
    ising_ds_destroy(ds);
    return rc;
  }
  *out = ds;
  return ISING_OK;
}

namespace ising {
namespace {

constexpr int64_t kGraphSteps = 48;  // a multiple of the launch period 6

// Whether the update launches of this session track the step before theirs
// (the streaming tensor-core form without the convergence rule or the
// relaxed product): a step then takes one launch instead of two, and the
// last step of each run is tracked by a flush launch. The session's
// counters[2] names the latest tracked step, so no launch tracks a step
// twice, nor a step whose energies were never computed (an imported one).
bool fold_ok(ising_ds* ds) {
  return ds->path == ISING_PATH_TC && !tc_is_resident(ds) && !ds->relaxed() && !ds->conv.p;
}

// Captures kGraphSteps steps (step kernel + tracking) into a graph on a
// private stream; the host step counter is restored afterwards because
// capture does not execute anything.
int build_graph(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  ISING_CUDA(ctx, cudaStreamCreateWithFlags(&ds->gstream, cudaStreamNonBlocking));
  ISING_CUDA(ctx, cudaEventCreateWithFlags(&ds->gev[0], cudaEventDisableTiming));
  ISING_CUDA(ctx, cudaEventCreateWithFlags(&ds->gev[1], cudaEventDisableTiming));
  cudaStream_t saved = ctx->stream;
  const int64_t t0 = ds->t;
  ctx->stream = ds->gstream;
  cudaGraph_t g = nullptr;
  int rc = ISING_OK;
  const bool fold = fold_ok(ds);
  cudaError_t e = cudaStreamBeginCapture(ds->gstream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int64_t s = 0; s < kGraphSteps && rc == ISING_OK; ++s) {
      ds->fold_track = fold;
      rc = path_step_raw(ds, true);
      ds->fold_track = false;
      if (rc == ISING_OK && !fold) rc = track_step(ds);
      ds->t += 1;
    }
    e = cudaStreamEndCapture(ds->gstream, &g);
  }
  ds->t = t0;
  ctx->stream = saved;
  if (rc != ISING_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, ISING_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ds->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ds->graph = nullptr;
    return fail(ctx, ISING_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  return ISING_OK;
}

// kGraphSteps steps by one graph launch, ordered after prior work on the
// context's stream and before later work on it.
int replay_graph(ising_ds* ds) {
  ising_ctx* ctx = ds->ctx;
  ISING_CUDA(ctx, cudaEventRecord(ds->gev[0], ctx->stream));
  ISING_CUDA(ctx, cudaStreamWaitEvent(ds->gstream, ds->gev[0], 0));
  ISING_CUDA(ctx, cudaGraphLaunch(ds->graph, ds->gstream));
  ISING_CUDA(ctx, cudaEventRecord(ds->gev[1], ds->gstream));
  ISING_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ds->gev[1], 0));
  ds->t += kGraphSteps;
  return ISING_OK;
}

}  // namespace
}  // namespace ising

namespace ising {
namespace {

// Launch-shape autotuner: the chosen sparse slice width per problem shape,
// kept for the process and optionally in the file named by ISING_TUNE_CACHE.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const ising_ds* ds) {
  std::ostringstream k;
  k << "sparse n=" << ds->n << " nnz=" << ds->inst.nnz << " Bp=" << ds->Bp
    << " i8=" << ds->sp_int8 << " ie=" << ds->int_energy;
  return k.str();
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("ISING_TUNE_CACHE");
  if (!path) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t bar = line.rfind('|');
    if (bar == std::string::npos) continue;
    g_tune[line.substr(0, bar)] = std::atoi(line.c_str() + bar + 1);
  }
}

void tune_store_locked(const std::string& key, int v) {
  g_tune[key] = v;
  const char* path = std::getenv("ISING_TUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << "|" << v << "\n";
}

// Times one real step with each candidate shape (twice, alternating) and keeps
// the fastest; returns the number of steps it ran.
int autotune_sparse(ising_ds* ds, int64_t budget, int64_t* done) {
  *done = 0;
  ds->tuned = true;
  if ((ds->p.flags & ISING_DS_NO_AUTOTUNE) || (ds->Bp / 128) % 2 != 0) return ISING_OK;
  const std::string key = tune_key(ds);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      ds->sp_q = it->second;
      return ISING_OK;
    }
  }
  if (budget < 5) return ISING_OK;
  ising_ctx* ctx = ds->ctx;
  cudaEvent_t ev[5];
  for (auto& e : ev) ISING_CUDA(ctx, cudaEventCreate(&e));
  // one untimed step warms the caches, then shapes 1, 2, 2, 1 (balanced order)
  const int order[5] = {1, 1, 2, 2, 1};
  int rc = ISING_OK;
  for (int k = 0; k < 5 && rc == ISING_OK; ++k) {
    if (k >= 1) cudaEventRecord(ev[k - 1], ctx->stream);
    ds->sp_q = order[k];
    rc = sparse_step(ds, kModeUpdate, nullptr);
    if (rc == ISING_OK) rc = track_step(ds);
    ds->t += 1;
    *done += 1;
  }
  if (rc == ISING_OK) cudaEventRecord(ev[4], ctx->stream);
  float t[4] = {0, 0, 0, 0};
  if (rc == ISING_OK) {
    cudaEventSynchronize(ev[4]);
    for (int k = 0; k < 4; ++k) cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]);
    ds->sp_q = (t[0] + t[3] <= t[1] + t[2]) ? 1 : 2;
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_store_locked(key, ds->sp_q);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

std::string dense_key(const ising_ds* ds) {
  std::ostringstream k;
  k << "dense n=" << ds->n << " B=" << ds->B << " spins=" << ds->spin_kind << " planes=" << ds->planes
    << " ie=" << ds->int_energy;
  return k.str();
}

// Tensor-core streaming form: one untimed step, then each candidate tile
// width for one timed step in the order c0 .. c(k-1), c(k-1) .. c0 (every
// candidate sees early and late positions), the fastest total kept.
int autotune_dense(ising_ds* ds, int64_t budget, int64_t* done) {
  *done = 0;
  ds->tuned = true;
  int cand[8];
  const int nc = tc_bn_candidates(ds, cand);
  if ((ds->p.flags & ISING_DS_NO_AUTOTUNE) || nc <= 1) return ISING_OK;
  const std::string key = dense_key(ds);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return tc_set_bn(ds, it->second);
  }
  if (budget < 1 + 2 * nc) return ISING_OK;
  ising_ctx* ctx = ds->ctx;
  cudaEvent_t ev[17];
  for (int k = 0; k <= 2 * nc; ++k) ISING_CUDA(ctx, cudaEventCreate(&ev[k]));
  int rc = ISING_OK;
  for (int k = 0; k <= 2 * nc && rc == ISING_OK; ++k) {
    if (k >= 1) {
      const int c = k - 1 < nc ? cand[k - 1] : cand[2 * nc - k];
      rc = tc_set_bn(ds, c);
      if (rc == ISING_OK) cudaEventRecord(ev[k - 1], ctx->stream);
    }
    if (rc == ISING_OK) rc = path_step(ds, true);
    if (rc == ISING_OK) rc = track_step(ds);
    ds->t += 1;
    *done += 1;
  }
  if (rc == ISING_OK) cudaEventRecord(ev[2 * nc], ctx->stream);
  if (rc == ISING_OK) {
    cudaEventSynchronize(ev[2 * nc]);
    float best = 0.f;
    int pick = cand[0];
    for (int c = 0; c < nc; ++c) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ev[c], ev[c + 1]);
      cudaEventElapsedTime(&b, ev[2 * nc - 1 - c], ev[2 * nc - c]);
      if (c == 0 || a + b < best) {
        best = a + b;
        pick = cand[c];
      }
    }
    rc = tc_set_bn(ds, pick);
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_store_locked(key, pick);
  }
  for (int k = 0; k <= 2 * nc; ++k) cudaEventDestroy(ev[k]);
  return rc;
}

}  // namespace
}  // namespace ising

// Queues up to `todo` steps on the session's stream without waiting for them:
// one cooperative launch in the resident form, otherwise the autotuner's
// first steps, then graph replays of kGraphSteps steps and single steps.
int ising::ds_advance(ising_ds* ds, int64_t todo) {
  if (ds->path == ISING_PATH_TC && tc_is_resident(ds)) {
    ISING_TRY(tc_run_resident(ds, todo));
    ds->t += todo;
    ds->work_host += todo * ds->B;
    if (ds->p.flags & ISING_DS_PROFILE) ds->kernel_launches += todo;
    return ISING_OK;
  }
  int64_t s0 = 0;
  if (ds->path == ISING_PATH_SPARSE && !ds->tuned) ISING_TRY(autotune_sparse(ds, todo, &s0));
  if (ds->path == ISING_PATH_TC && !ds->tuned) ISING_TRY(autotune_dense(ds, todo, &s0));
  const bool use_graph = !(ds->p.flags & ISING_DS_PROFILE) && todo >= 2 * kGraphSteps;
  const bool fold = fold_ok(ds);
  for (int64_t s = s0; s < todo;) {
    // (t > 0: the kernels have run once outside capture, which sets their attributes)
    if (use_graph && ds->t > 0 && ds->t % 6 == 0 && todo - s >= kGraphSteps) {
      if (!ds->graph) ISING_TRY(build_graph(ds));
      ISING_TRY(replay_graph(ds));
      s += kGraphSteps;
    } else {
      ds->fold_track = fold;
      const int rc = path_step(ds, true);
      ds->fold_track = false;
      ISING_TRY(rc);
      if (!fold) ISING_TRY(track_step(ds));
      ds->t += 1;
      s += 1;
    }
  }
  // the last step's tracking (its launch tracked only its predecessor)
  if (fold && todo > s0) ISING_TRY(track_flush(ds));
  return ISING_OK;
}

// With the convergence rule: whether every restart has stopped (reads the
// device count; synchronises the stream).
int ising::ds_conv_check(ising_ds* ds) {
  if (!ds->conv.p || ds->conv_all) return ISING_OK;
  unsigned long long c = 0;
  ISING_CUDA(ds->ctx, cudaMemcpyAsync(&c, ds->conv_count(), 8, cudaMemcpyDeviceToHost, ds->ctx->stream));
  ISING_CUDA(ds->ctx, cudaStreamSynchronize(ds->ctx->stream));
  if ((int64_t)c >= ds->B) ds->conv_all = true;
  return ISING_OK;
}

namespace {
constexpr int64_t kConvChunk = 48;  // steps between checks of the convergence count

// ds_advance, in chunks with a check of the convergence count after each
// when the rule is on; stops once every restart has stopped.
int advance_checked(ising_ds* ds, int64_t todo) {
  if (!ds->conv.p) return ds_advance(ds, todo);
  while (todo > 0 && !ds->conv_all) {
    const int64_t k = std::min(todo, kConvChunk);
    ISING_TRY(ds_advance(ds, k));
    todo -= k;
    ISING_TRY(ds_conv_check(ds));
  }
  return ISING_OK;
}
}  // namespace

extern "C" int ising_ds_run(ising_ds* ds, int64_t steps) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (steps < 0) return fail(ctx, ISING_EINVAL, "steps must be >= 0");
  if (ds->finished) return fail(ctx, ISING_EINVAL, "session already finished");
  int64_t todo = std::min(steps, ds->T - ds->t);
  if (todo <= 0 || ds->conv_all) return ISING_OK;
  NvtxRange range("ising_ds_run");
  cudaEvent_t e0, e1;
  ISING_CUDA(ctx, cudaEventCreate(&e0));
  ISING_CUDA(ctx, cudaEventCreate(&e1));
  ISING_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
  int rc = advance_checked(ds, todo);
  if (rc != ISING_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  ISING_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
  ISING_CUDA(ctx, cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  ds->device_ms += ms;
  if (ds->path == ISING_PATH_TC && tc_is_resident(ds) && (ds->p.flags & ISING_DS_PROFILE))
    ds->kernel_ms += ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ISING_CUDA(ctx, cudaGetLastError());
  if (ds->path == ISING_PATH_TC) ISING_TRY(tc_error(ds));
  return ISING_OK;
}

extern "C" int ising_ds_finish(ising_ds* ds) {
  if (!ds) return ISING_EINVAL;
  if (ds->finished) return ISING_OK;
  ising_ctx* ctx = ds->ctx;
  ISING_TRY(ising_ds_run(ds, ds->T - ds->t));
  NvtxRange range("ising_ds_finish");
  // energy of S_{T+1}: the step kernels in energy-only mode, then tracking
  // (nothing to evaluate once every restart has stopped)
  if (!ds->conv_all) {
    ISING_TRY(path_step(ds, false));
    ISING_TRY(track_step(ds));
  }
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ds->path == ISING_PATH_TC) ISING_TRY(tc_error(ds));
  ISING_TRY(select_best(ds));
  ds->finished = true;
  return ISING_OK;
}

extern "C" int ising_ds_export_state(ising_ds* ds, float* theta, float* m, float* v,
                                     int8_t* spins, int64_t* t, int mem) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  const int64_t n = ds->n, B = ds->B;
  cudaMemcpyKind kind = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  float* outs[3] = {theta, m, v};
  const DevMem* srcs[3] = {&ds->theta, &ds->m, &ds->v};
  DevMem tmp;
  for (int a = 0; a < 3; ++a) {
    if (!outs[a]) continue;
    if (ds->path == ISING_PATH_SPARSE) {
      if (!tmp.p) ISING_TRY(dev_alloc(ctx, tmp, (size_t)B * n * 4));
      spin_major_to_restart_major<<<grid1d(ctx, B * n), 256, 0, ctx->stream>>>(
          n, B, ds->Bp, srcs[a]->as<float>(), tmp.as<float>());
      ISING_CUDA(ctx, cudaGetLastError());
      ISING_CUDA(ctx, cudaMemcpyAsync(outs[a], tmp.p, (size_t)B * n * 4, kind, ctx->stream));
      ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    } else {
      ISING_CUDA(ctx, cudaMemcpy2DAsync(outs[a], n * 4, srcs[a]->p, ds->ld * 4, n * 4, B, kind,
                                        ctx->stream));
    }
  }
  if (spins) {
    DevMem s8;
    ISING_TRY(dev_alloc(ctx, s8, (size_t)B * n));
    ISING_TRY(export_spins_int8(ds, (int)((ds->t + 1) % 3), s8.as<int8_t>()));
    ISING_CUDA(ctx, cudaMemcpyAsync(spins, s8.p, (size_t)B * n,
                                    mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost
                                                          : cudaMemcpyDeviceToDevice,
                                    ctx->stream));
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (t) *t = ds->t;
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_ds_import_state(ising_ds* ds, const float* theta, const float* m,
                                     const float* v, int64_t t, int mem) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (!theta || !m || !v) return fail(ctx, ISING_EINVAL, "theta, m and v are required");
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  if (t < 0 || t > ds->T) return fail(ctx, ISING_EINVAL, "t must lie in [0, T]");
  if (ds->finished) return fail(ctx, ISING_EINVAL, "session already finished");
  const int64_t n = ds->n, B = ds->B;
  cudaMemcpyKind kind = mem == ISING_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const float* ins[3] = {theta, m, v};
  DevMem* dsts[3] = {&ds->theta, &ds->m, &ds->v};
  DevMem tmp;
  for (int a = 0; a < 3; ++a) {
    if (ds->path == ISING_PATH_SPARSE) {
      if (!tmp.p) ISING_TRY(dev_alloc(ctx, tmp, (size_t)B * n * 4));
      ISING_CUDA(ctx, cudaMemcpyAsync(tmp.p, ins[a], (size_t)B * n * 4, kind, ctx->stream));
      restart_major_to_spin_major<<<grid1d(ctx, B * n), 256, 0, ctx->stream>>>(
          n, B, ds->Bp, tmp.as<float>(), dsts[a]->as<float>(), a == 0);
      ISING_CUDA(ctx, cudaGetLastError());
      ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    } else {
      ISING_CUDA(ctx, cudaMemcpy2DAsync(dsts[a]->p, ds->ld * 4, ins[a], n * 4, n * 4, B, kind,
                                        ctx->stream));
      if (a == 0) {
        wrap_rows_kernel<<<grid1d(ctx, B * n), 256, 0, ctx->stream>>>(n, B, ds->ld,
                                                                      ds->theta.as<float>());
        ISING_CUDA(ctx, cudaGetLastError());
      }
    }
  }
  ds->t = t;
  // (step t has no energies in this session: it counts as tracked)
  long long cnt[4] = {(long long)t, 0, (long long)t, 0};
  ISING_CUDA(ctx, cudaMemcpyAsync(ds->counters.p, cnt, 32, cudaMemcpyHostToDevice, ctx->stream));
  const int slot = (int)((t + 1) % 3);
  if (ds->path == ISING_PATH_SPARSE) {
    spins_from_theta_bits<<<grid1d(ctx, n * ds->Bp / 32), 256, 0, ctx->stream>>>(
        n, ds->Bp, ds->theta.as<float>(), ds->spins[slot].as<uint32_t>());
  } else {
    int g = grid1d(ctx, ds->Bp * ds->ld);
    switch (ds->spin_kind) {
      case kSpinF32: spins_from_theta_dense<kSpinF32><<<g, 256, 0, ctx->stream>>>(n, ds->Bp, ds->ld, ds->theta.as<float>(), ds->spins[slot].p); break;
      case kSpinBF16: spins_from_theta_dense<kSpinBF16><<<g, 256, 0, ctx->stream>>>(n, ds->Bp, ds->ld, ds->theta.as<float>(), ds->spins[slot].p); break;
      case kSpinF16: spins_from_theta_dense<kSpinF16><<<g, 256, 0, ctx->stream>>>(n, ds->Bp, ds->ld, ds->theta.as<float>(), ds->spins[slot].p); break;
      default: spins_from_theta_dense<kSpinE4M3><<<g, 256, 0, ctx->stream>>>(n, ds->Bp, ds->ld, ds->theta.as<float>(), ds->spins[slot].p); break;
    }
  }
  ISING_CUDA(ctx, cudaGetLastError());
  if (ds->relaxed()) ISING_TRY(derive_x(ds, (int)((t + 1) % 2)));
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_ds_coupling(ising_ds* ds, float* G_out, int mem) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (!G_out) return fail(ctx, ISING_EINVAL, "G_out is NULL");
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  if (ds->finished) return fail(ctx, ISING_EINVAL, "session already finished");
  const int64_t n = ds->n, B = ds->B;
  cudaMemcpyKind kind = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  DevMem G;
  if (ds->path == ISING_PATH_SPARSE) {
    DevMem Gt;
    ISING_TRY(dev_alloc(ctx, Gt, (size_t)n * ds->Bp * 4));
    ISING_TRY(dev_alloc(ctx, G, (size_t)B * n * 4));
    ISING_TRY(sparse_step(ds, kModeCoupling, Gt.as<float>()));
    spin_major_to_restart_major<<<grid1d(ctx, B * n), 256, 0, ctx->stream>>>(
        n, B, ds->Bp, Gt.as<float>(), G.as<float>());
    ISING_CUDA(ctx, cudaGetLastError());
    ISING_CUDA(ctx, cudaMemcpyAsync(G_out, G.p, (size_t)B * n * 4, kind, ctx->stream));
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    ISING_TRY(dev_alloc(ctx, G, (size_t)ds->Bp * ds->ld * 4));
    if (ds->path == ISING_PATH_PLAIN) ISING_TRY(plain_step(ds, kModeCoupling, G.as<float>()));
    else ISING_TRY(tc_step(ds, kModeCoupling, G.as<float>()));
    ISING_CUDA(ctx, cudaMemcpy2DAsync(G_out, n * 4, G.p, ds->ld * 4, n * 4, B, kind, ctx->stream));
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ds->path == ISING_PATH_TC) ISING_TRY(tc_error(ds));
  }
  return ISING_OK;
}

extern "C" int ising_ds_trace(ising_ds* ds, uint64_t* out, int64_t cap, int64_t* count) {
  if (!ds || !count) return ISING_EINVAL;
  if (cap > 0 && !out) return fail(ds->ctx, ISING_EINVAL, "out is NULL");
  *count = 0;
  if (ds->path != ISING_PATH_TC) return ISING_OK;
  return tc_trace(ds, out, cap, count);
}

extern "C" int ising_ds_last_energies(ising_ds* ds, double* E, int mem) {
  if (!ds) return ISING_EINVAL;
  if (!E) return fail(ds->ctx, ISING_EINVAL, "E is NULL");
  ISING_TRY(copy_out(ds->ctx, E, ds->last_E.p, ds->B * 8, mem));
  ISING_CUDA(ds->ctx, cudaStreamSynchronize(ds->ctx->stream));
  return ISING_OK;
}

extern "C" int ising_ds_set_tiles(ising_ds* ds, int32_t restarts_per_tile, int32_t pair) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (ds->path != ISING_PATH_TC || tc_is_resident(ds))
    return fail(ctx, ISING_ENOTSUP, "tile shapes apply to the tensor-core streaming form");
  if (pair < 0 || pair > 2) return fail(ctx, ISING_EINVAL, "pair must be 0, 1 or 2");
  const int code = restarts_per_tile | (pair ? kTcPair : 0) | (pair == 2 ? kTcSplit : 0);
  int cand[8];
  const int nc = tc_bn_candidates(ds, cand);
  bool ok = restarts_per_tile == 64 || restarts_per_tile == 128 || restarts_per_tile == 224 ||
            restarts_per_tile == 256;
  if (pair) ok = ok && std::find(cand, cand + nc, code) != cand + nc;
  if (!ok) return fail(ctx, ISING_EINVAL, "tile shape %d%s is not available for this session",
                       restarts_per_tile, pair ? " in pairs" : "");
  ISING_TRY(tc_set_bn(ds, code));
  ds->tuned = true;
  return ISING_OK;
}

extern "C" int ising_ds_work(ising_ds* ds, int64_t* restart_steps) {
  if (!ds) return ISING_EINVAL;
  if (!restart_steps) return fail(ds->ctx, ISING_EINVAL, "restart_steps is NULL");
  unsigned long long w = 0;
  ISING_CUDA(ds->ctx, cudaMemcpyAsync(&w, ds->work.p, 8, cudaMemcpyDeviceToHost, ds->ctx->stream));
  ISING_CUDA(ds->ctx, cudaStreamSynchronize(ds->ctx->stream));
  *restart_steps = (int64_t)w + ds->work_host;
  return ISING_OK;
}

extern "C" int ising_ds_convergence(ising_ds* ds, int64_t* step, int mem) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  if (!step) return fail(ctx, ISING_EINVAL, "step is NULL");
  const cudaMemcpyKind kind = mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (ds->conv.p) {
    ISING_CUDA(ctx, cudaMemcpyAsync(step, ds->conv_step(), ds->B * 8, kind, ctx->stream));
  } else if (mem == ISING_MEM_HOST) {
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memset(step, 0, ds->B * 8);
  } else {
    ISING_CUDA(ctx, cudaMemsetAsync(step, 0, ds->B * 8, ctx->stream));
  }
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_ds_restart_best(ising_ds* ds, double* E, int64_t* step, int8_t* spins,
                                     int mem) {
  if (!ds) return ISING_EINVAL;
  if (E) ISING_TRY(copy_out(ds->ctx, E, ds->best_E.p, ds->B * 8, mem));
  if (step) ISING_TRY(copy_out(ds->ctx, step, ds->best_t.p, ds->B * 8, mem));
  if (spins)
    ISING_CUDA(ds->ctx, cudaMemcpy2DAsync(spins, ds->n, ds->best_s.p, ds->bs_ld, ds->n, ds->B,
                                          mem == ISING_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                : cudaMemcpyDeviceToDevice,
                                          ds->ctx->stream));
  ISING_CUDA(ds->ctx, cudaStreamSynchronize(ds->ctx->stream));
  return ISING_OK;
}

extern "C" int ising_ds_result(ising_ds* ds, int8_t* best_spins, double* best_energy,
                               ising_ds_stats* stats, int mem) {
  if (!ds) return ISING_EINVAL;
  ising_ctx* ctx = ds->ctx;
  if (!ds->finished) ISING_TRY(select_best(ds));
  const int64_t b = ds->best_restart;
  if (best_spins)
    ISING_TRY(copy_out(ctx, best_spins, ds->best_s.as<int8_t>() + b * ds->bs_ld, ds->n, mem));
  if (best_energy) {
    if (mem == ISING_MEM_HOST) *best_energy = ds->best_energy;
    else ISING_CUDA(ctx, cudaMemcpyAsync(best_energy, &ds->best_energy, 8, cudaMemcpyHostToDevice, ctx->stream));
  }
  if (stats) {
    long long st = 0;
    ISING_CUDA(ctx, cudaMemcpyAsync(&st, ds->best_t.as<long long>() + b, 8, cudaMemcpyDeviceToHost, ctx->stream));
    ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    stats->best_restart = b;
    stats->best_step = st;
    stats->last_best_energy = ds->last_best_energy;
    stats->last_best_restart = ds->last_best_restart;
    stats->steps_done = ds->t;
    stats->path = ds->path;
    stats->precision = ds->prec;
    stats->device_ms = ds->device_ms;
    stats->kernel_ms = ds->kernel_ms;
    stats->kernel_launches = ds->kernel_launches;
    stats->resident = ds->path == ISING_PATH_TC ? tc_resident_form(ds) : 0;
    stats->operand_planes = ds->path == ISING_PATH_TC ? ds->planes : 1;
    const bool streaming = ds->path == ISING_PATH_TC && tc_resident_form(ds) == 0;
    stats->tile_restarts = streaming ? tc_bn(ds) : 0;
    stats->tile_pair = streaming ? tc_tile_pair(ds) : 0;
  }
  ISING_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ISING_OK;
}

extern "C" int ising_ds_destroy(ising_ds* ds) {
  if (!ds) return ISING_OK;
  if (ds->ctx) cudaStreamSynchronize(ds->ctx->stream);
  for (auto& e : ds->kev)
    if (e) cudaEventDestroy(e);
  if (ds->graph) cudaGraphExecDestroy(ds->graph);
  if (ds->gstream) {
    cudaStreamSynchronize(ds->gstream);
    cudaStreamDestroy(ds->gstream);
  }
  for (auto& e : ds->gev)
    if (e) cudaEventDestroy(e);
  tc_release(ds);
  delete ds;
  return ISING_OK;
}

extern "C" int ising_select_domain(ising_ctx* ctx, const ising_instance* inst,
                                   const ising_ds_params* p, int8_t* best_spins,
                                   double* best_energy, ising_ds_stats* stats, int mem) {
  if (!ctx) return ISING_EINVAL;
  if (mem != ISING_MEM_HOST && mem != ISING_MEM_DEVICE) return fail(ctx, ISING_EINVAL, "bad mem");
  ising_ds* ds = nullptr;
  ISING_TRY(ising_ds_create(ctx, inst, p, &ds));
  int rc = ising_ds_finish(ds);
  if (rc == ISING_OK) rc = ising_ds_result(ds, best_spins, best_energy, stats, mem);
  ising_ds_destroy(ds);
  return rc;
}
