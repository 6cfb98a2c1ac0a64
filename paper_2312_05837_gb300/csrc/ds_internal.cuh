// Domain-selection session (Sec. III-B) shared by the step kernels.
#pragma once

#include "common.cuh"

namespace ising {

// Per-step constants of the update. Adam bias corrections come from a device
// table indexed by the step counter, so launches stay identical across steps
// and can be replayed from a CUDA graph.
struct StepConsts {
  float cq, ch, mu, lr, b1, b2, eps;
  float omb1, omb2;  // 1 - b1 and 1 - b2 formed in FP64, then rounded
};

// theta - 2 pi rint(theta / 2 pi) with 2 pi split in two floats, so that the
// result lies in [-pi, pi] up to one rounding (projection of Sec. III-B
// reading: sin and cos are unchanged).
__device__ __forceinline__ float wrap_angle(float th) {
  const float kInv2Pi = 0.15915494309189535f;
  const float k2PiHi = __int_as_float(0x40C90FDB);  // 2 pi rounded up to float
  const float k2PiLo = -1.7484555314695172e-07f;    // 2 pi - k2PiHi
  float k = rintf(th * kInv2Pi);
  th = fmaf(-k, k2PiHi, th);
  th = fmaf(-k, k2PiLo, th);
  return th;
}

// sgn+(sin theta) for float theta with |theta| < 2 pi, by comparisons: sin is
// >= 0 exactly on [0, pi] and (-2 pi, -pi], i.e. when (theta >= 0) differs
// from (|theta| > pi); pi is not a float, and |theta| > pi holds exactly when
// |theta| exceeds the largest float below pi.
__device__ __forceinline__ bool sin_nonneg(float th) {
  const float kPiDn = __int_as_float(0x40490FDA);  // largest float < pi
  return (th >= 0.0f) != (fabsf(th) > kPiDn);
}

// Adam on one coordinate; returns the projected new angle. The square root and
// the division use the hardware approximations (a few ulp), far inside the
// 1e-5 step tolerance.
__device__ __forceinline__ float adam_update(const StepConsts& k, float c1, float c2, float g,
                                             float th, float& m, float& v) {
  m = fmaf(k.b1, m, k.omb1 * g);
  v = fmaf(k.b2, v, k.omb2 * (g * g));
  const float mhat = m * c1;
  const float vhat = v * c2;
  float rt;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rt) : "f"(vhat));  // relative error ~2^-23
  th = th - __fdividef(k.lr * mhat, rt + k.eps);
  return wrap_angle(th);
}

// sin(theta) on [-pi, pi]: the hardware approximation (absolute error at most
// 2^-21.41 there), for the relaxed spins x = sin(theta) of ISING_DS_RELAXED.
__device__ __forceinline__ float sin_proj(float th) { return __sinf(th); }

// cos(theta) for theta in [-pi, pi] (the projection keeps it there): the
// hardware approximation, absolute error at most 2^-21.41 on that range, so
// the gradient cos(theta) F is within 4e-7 |F| of the exact one.
__device__ __forceinline__ float cos_proj(float th) { return __cosf(th); }

// Convergence rule of Sec. IV-B on the energies of restart b (window 5,
// tolerance 0.005; see ISING_DS_CONVERGE): records E_t, and at t >= 5
// stops the restart when the window's spread is within the tolerance.
// Returns true when the restart stops at this step.
constexpr double kConvTol = 0.005;
__device__ __forceinline__ bool conv_update(double* ring, double* init, long long* step,
                                            unsigned long long* count, int64_t B, int64_t b,
                                            long long t, double E) {
  ring[((t - 1) % 5) * B + b] = E;
  if (t == 1) init[b] = E;
  if (t < 5) return false;
  double mx = ring[b], mn = ring[b];
#pragma unroll
  for (int k = 1; k < 5; ++k) {
    const double x = ring[k * B + b];
    mx = fmax(mx, x);
    mn = fmin(mn, x);
  }
  if (mx - mn <= kConvTol * fabs(E - init[b])) {
    step[b] = t;
    atomicAdd(count, 1ull);
    return true;
  }
  return false;
}

// Early retirement under the convergence rule: live32[k] counts the restarts
// of block [32 k, 32 k + 32) that have not stopped (null when the rule is
// off). A step kernel skips a tile or slice whose restarts [b0, b1) have all
// stopped: their results are final and their state is left as it is.
__device__ __forceinline__ bool restarts_retired(const int* live32, int64_t b0, int64_t b1) {
  if (!live32) return false;
  for (int64_t k = b0 >> 5; k < ((b1 + 31) >> 5); ++k)
    if (live32[k] > 0) return false;
  return true;
}

enum SpinKind { kSpinF32 = 0, kSpinBF16 = 1, kSpinBits = 2, kSpinE4M3 = 3, kSpinF16 = 4 };

// Sign bit of each byte of four E4M3 spins -> four int8 +1 / -1.
__device__ __forceinline__ uint32_t e4m3x4_to_pm1(uint32_t w) {
  const uint32_t m = (w >> 7) & 0x01010101u;
  return 0x01010101u + m * 0xFEu;
}

// Two 16-bit (BF16 or FP16) spins -> two int8 +1 / -1 in the low 16 bits
// (only the sign bits are read).
__device__ __forceinline__ uint32_t bf16x2_to_pm1(uint32_t w) {
  return (((w >> 15) & 1u) ? 0xFFu : 0x01u) | ((((w >> 31) & 1u) ? 0xFFu : 0x01u) << 8);
}

// Copies the spins of restart b from a dense spin slot ([B][ld]) into an int8
// row (16-byte aligned, at least ceil(n / 16) * 16 bytes long); the lanes of a
// warp move 16 source bytes each per iteration.
template <int KIND>
__device__ __forceinline__ void copy_spin_row_dense(int8_t* dst, const void* spins, int64_t n,
                                                    int64_t ld, int64_t b, int lane) {
  if (KIND == kSpinE4M3) {
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(spins) + b * ld);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int64_t v = lane; v < (n + 15) / 16; v += 32) {
      uint4 x = src[v];
      x.x = e4m3x4_to_pm1(x.x);
      x.y = e4m3x4_to_pm1(x.y);
      x.z = e4m3x4_to_pm1(x.z);
      x.w = e4m3x4_to_pm1(x.w);
      d[v] = x;
    }
  } else if (KIND == kSpinBF16 || KIND == kSpinF16) {
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(spins) + b * ld);
    uint2* d = reinterpret_cast<uint2*>(dst);
    for (int64_t v = lane; v < (n + 7) / 8; v += 32) {
      const uint4 x = src[v];
      uint2 y;
      y.x = bf16x2_to_pm1(x.x) | (bf16x2_to_pm1(x.y) << 16);
      y.y = bf16x2_to_pm1(x.z) | (bf16x2_to_pm1(x.w) << 16);
      d[v] = y;
    }
  } else {
    const float* src = static_cast<const float*>(spins) + b * ld;
    for (int64_t i = lane; i < n; i += 32) dst[i] = src[i] > 0.f ? 1 : -1;
  }
}

// What best tracking of one session reads and writes; the partial and spin
// slots of step t are qpart / hpart / epart[t % 2] and spins[t % 3].
struct TrackArgs {
  int64_t n, B, Bp, ld;
  int mtiles;
  bool int_mode;
  double cq, chs;
  const long long* qpart[2];
  const long long* hpart[2];
  const float* epart[2];
  const void* spins[3];
  double* best_E;
  long long* best_t;
  int8_t* best_s;
  double* last_E;
  long long* counters;
  int64_t bs_ld;
  uint8_t* improved;
  int64_t T;
  double* conv_ring;
  double* conv_init;
  long long* conv_step;
  unsigned long long* conv_count;
  int* live32;  // live restarts per block of 32 (convergence rule), or null
  // bit-packed spins: copy an improved restart's spins here (small n)
  // instead of flagging it for track_bits_copy_kernel
  bool inline_bits;
  // track the step counters[0] names, without advancing the counter (the
  // last step of a run whose step launches tracked their predecessors)
  bool flush;
};

// Best tracking of restart b at step t, by one warp: E_t(b) from the
// partials of slot t % 2 (lane l adds rows l, l+32, ... in order, then a
// fixed xor tree across lanes, so the sum is deterministic), strict <
// against the best so far, copy of S_t for an improved restart (for
// bit-packed spins a per-restart flag instead, which track_bits_copy_kernel
// reads). With the convergence rule (conv_step non-null) a stopped restart
// is left alone, and steps t <= T feed the rule.
template <int KIND>
__device__ __forceinline__ void track_restart(const TrackArgs& A, long long t, int64_t b, int lane) {
  const int ps = (int)(t % 2);
  double E;
  if (A.int_mode) {
    const long long* qpart = A.qpart[ps];
    const long long* hpart = A.hpart[ps];
    long long q = 0, hs = 0;
#pragma unroll 4
    for (int r = lane; r < A.mtiles; r += 32) {
      q += qpart[(int64_t)r * A.Bp + b];
      hs += hpart[(int64_t)r * A.Bp + b];
    }
    for (int o = 16; o; o >>= 1) {
      q += __shfl_xor_sync(0xffffffffu, q, o);
      hs += __shfl_xor_sync(0xffffffffu, hs, o);
    }
    E = A.cq * (double)q + A.chs * (double)hs;
  } else {
    const float* epart = A.epart[ps];
    double e = 0.0;
#pragma unroll 4
    for (int r = lane; r < A.mtiles; r += 32) e += (double)epart[(int64_t)r * A.Bp + b];
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    E = e;
  }
  // every lane holds the same E (the xor tree is symmetric)
  const bool active = A.conv_step == nullptr || A.conv_step[b] == 0;
  const bool improved = active && E < A.best_E[b];
  __syncwarp();
  if (lane == 0 && active) {
    A.last_E[b] = E;
    if (improved) {
      A.best_E[b] = E;
      A.best_t[b] = t;
    }
    if (A.conv_step && t <= A.T &&
        conv_update(A.conv_ring, A.conv_init, A.conv_step, A.conv_count, A.B, b, t, E) && A.live32)
      atomicSub(&A.live32[b >> 5], 1);
  }
  if (KIND == kSpinBits) {
    if (A.inline_bits) {
      // bit b of each spin's word column, one spin per lane and pass
      if (improved) {
        const uint32_t* bits = static_cast<const uint32_t*>(A.spins[t % 3]);
        const int64_t words = A.Bp / 32;
        int8_t* dst = A.best_s + b * A.bs_ld;
        for (int64_t i = lane; i < A.n; i += 32)
          dst[i] = ((bits[i * words + (b >> 5)] >> (b & 31)) & 1u) ? 1 : -1;
      }
    } else if (lane == 0) {
      // bit-packed spins are copied by track_bits_copy_kernel
      A.improved[b] = improved ? 1 : 0;
    }
  } else if (improved) {
    copy_spin_row_dense<KIND>(A.best_s + b * A.bs_ld, A.spins[t % 3], A.n, A.ld, b, lane);
  }
}

// What a step launch does: the full update, only the energies of the input
// spins (the final evaluation), or only the coupling product G = J s.
// kModeRelaxed: the update with the coupling product taken on the relaxed
// spins x = sin(theta) (ISING_DS_RELAXED); energies then come from a
// kModeEnergy pass on the rounded spins (dense paths) or from the rounded
// spins gathered alongside (sparse path).
enum StepMode { kModeUpdate = 0, kModeEnergy = 1, kModeCoupling = 2, kModeRelaxed = 3 };

}  // namespace ising

struct ising_ds {
  ising_ctx* ctx = nullptr;
  ising::DevInstance inst;
  ising_ds_params p{};
  int64_t n = 0, B = 0, T = 0;
  int64_t t = 0;          // steps done (host mirror of the device counter)
  int path = ISING_PATH_PLAIN;
  int prec = ISING_PREC_FP32_PLAIN;
  bool int_energy = false; // energies accumulate exactly in integers
  int h_shift = 0;         // integer field = h * 2^h_shift
  ising::StepConsts k{};
  // state layout: dense paths [Bp][ld] restart-major; sparse path [n][Bp]
  int64_t ld = 0;          // leading dimension of restart-major arrays
  int64_t Bp = 0;          // padded restart count (sparse: multiple of 128)
  int spin_kind = ising::kSpinF32;
  ising::DevMem theta, m, v;
  ising::DevMem spins[3];  // S_t lives in spins[t % 3]
  int mtiles = 0;          // number of energy partial rows
  ising::DevMem qpart[2], hpart[2], epart[2];  // [mtiles][Bp], slot t % 2
  ising::DevMem hf;        // float32 field (n)
  ising::DevMem hint;      // int32 field * 2^h_shift (n)
  ising::DevMem best_E, best_t, best_s, last_E;
  ising::DevMem improved;  // per restart: improved at the last tracked step (bit-packed path)
  // convergence rule (ISING_DS_CONVERGE): [5][B] ring of energies, [B] E_1,
  // [B] stopping step, and the count of stopped restarts
  ising::DevMem conv;
  ising::DevMem live;      // convergence rule: int32 live restarts per block of 32
  bool conv_all = false;   // every restart has stopped
  // restart-steps the update kernels computed: a device counter (tiles and
  // slices add their restarts once per step) plus the resident forms' steps
  // x B counted on the host
  ising::DevMem work;
  int64_t work_host = 0;
  // relaxed product (ISING_DS_RELAXED): x_t = sin(theta) in slot t % 2, laid
  // out like the state (FP32; the 16-bit operand type on the tensor-core path)
  ising::DevMem xbuf[2];
  bool relaxed() const { return (p.flags & ISING_DS_RELAXED) != 0; }
  // the update launches being queued also track the step before theirs and
  // advance the step counter (streaming tensor-core form; see ds_advance)
  bool fold_track = false;
  double* conv_ring() const { return conv.as<double>(); }
  double* conv_init() const { return conv.as<double>() + 5 * B; }
  long long* conv_step() const { return reinterpret_cast<long long*>(conv.as<double>() + 6 * B); }
  unsigned long long* conv_count() const { return reinterpret_cast<unsigned long long*>(conv.as<double>() + 7 * B); }
  int64_t bs_ld = 0;       // row pitch of best_s (n rounded up to 16)
  // int64 [0] = steps done, [1] = done-block counter, [2] = the latest step
  // whose energies have been tracked (0: none), [3] unused
  ising::DevMem counters;
  ising::DevMem bias;      // float2 [T + 2]: 1/(1-b1^t), 1/(1-b2^t)
  // dense operands
  ising::DevMem Jf;        // plain path: float n x n
  ising::DevMem Jop[3];    // tensor path: planes (bf16, fp16 or e4m3), [n][ld]
  int planes = 1;
  ising::DevMem rowscale;  // fp8 / fp16-plane paths: float scale per row (null: 1)
  void* tc = nullptr;      // tensor-core path state (tensor maps etc.)
  // sparse operands
  ising::DevMem sp_val;    // int8 or float values
  bool sp_int8 = false;
  int sp_q = 1;            // sparse slice width (x 128 restarts), chosen by the autotuner
  bool tuned = false;
  // results
  bool finished = false;
  int64_t best_restart = -1;
  double best_energy = 0.0;
  double device_ms = 0.0;
  double kernel_ms = 0.0;
  int64_t kernel_launches = 0;
  cudaEvent_t kev[2] = {nullptr, nullptr};
  double last_best_energy = 0.0;
  int64_t last_best_restart = -1;
  ising::DevMem scratch;   // small per-session scratch (argmin etc.)
  // CUDA graph of kGraphSteps consecutive steps starting at t % 6 == 0 (the
  // launches repeat with period 6: spins rotate over 3 slots, partials over 2)
  cudaGraphExec_t graph = nullptr;
  cudaStream_t gstream = nullptr;  // private stream for capture and replay
  cudaEvent_t gev[2] = {nullptr, nullptr};
};

namespace ising {

// Path-specific hooks, implemented in ds_plain.cu, ds_sparse.cu, ds_tc.cu.
// A step launch reads S_t from spins[(t) % 3] with t = ds->t + 1; in coupling
// mode it writes G to Gout (dense: [B][ld], sparse: [n][Bp]) and nothing else.
int plain_setup(ising_ds* ds);
int plain_step(ising_ds* ds, int mode, float* Gout);
int sparse_setup(ising_ds* ds);
int sparse_step(ising_ds* ds, int mode, float* Gout);
int tc_setup(ising_ds* ds);
int tc_step(ising_ds* ds, int mode, float* Gout);
int tc_error(ising_ds* ds);  // ISING_ETIMEOUT if a bounded wait gave up
bool tc_is_resident(ising_ds* ds);            // tensor memory keeps the state between steps
int tc_resident_form(ising_ds* ds);           // 0 streaming, 1 grid-wide resident, 2 small (n <= 128)
int tc_run_resident(ising_ds* ds, int64_t steps);  // `steps` steps in one cooperative launch
int tc_trace(ising_ds* ds, uint64_t* out, int64_t cap, int64_t* count);
void tc_release(ising_ds* ds);

// Shared session services (ds.cu).
int ds_conv_check(ising_ds* ds);
int ds_advance(ising_ds* ds, int64_t todo);  // queue steps without waiting
int ds_create_impl(ising_ctx* ctx, const ising_instance* inst, const ising_ds_params* p,
                   ising_ds** out, bool validate);
int track_step(ising_ds* ds);  // reduce partials of step t+1, best tracking, t += 1
int track_flush(ising_ds* ds);  // best tracking of step t (counter already advanced)
TrackArgs track_args(const ising_ds* ds);
// Best tracking of every member of a pack (device arrays: members[count],
// rstart[count + 1] restart offsets, `done` a zeroed block counter).
// Best tracking of every pack member at counters[0] + 1, advancing the
// counters; with `flush`, at counters[0] (already advanced by packed update
// launches that tracked their predecessors), counters left alone.
int track_pack(ising_ctx* ctx, int spin_kind, const TrackArgs* members, const int64_t* rstart,
               int count, int64_t total_restarts, unsigned long long* done, bool flush = false);
// Pack hooks of the tensor-core path (ds_tc.cu): whether the session can be
// a pack member (streaming form, update-only), its pack key (members of one
// launch share it), the bytes and contents of its device entry, and one
// packed step launch.
bool tc_packable(const ising_ds* ds);
uint64_t tc_pack_key(const ising_ds* ds);
int tc_bn(const ising_ds* ds);                        // restart-tile width
int tc_tile_pair(const ising_ds* ds);                 // 0 single CTAs, 1 multicast pairs, 2 pair MMA
constexpr int kTcPair = 1 << 16;   // flag on a width: clusters of two CTAs share spin tiles
constexpr int kTcSplit = 1 << 17;  // ... and issue their MMAs as one (with kTcPair)
int tc_bn_candidates(const ising_ds* ds, int* out);   // widths the autotuner may try (<= 8)
int tc_set_bn(ising_ds* ds, int code);                // a width, with kTcPair or not
size_t tc_pack_entry_bytes();
int tc_pack_entry(ising_ds* ds, void* host_entry);
// What a packed update launch needs to track every member's previous step
// itself (trk null: a tracking launch follows each step instead).
struct PackFold {
  const TrackArgs* trk = nullptr;  // the members' tracking arguments (device)
  const int64_t* rstart = nullptr;  // their restart offsets (device)
  unsigned long long* done = nullptr;  // the pack's CTA counter
};
int tc_pack_launch(ising_ctx* ctx, uint64_t key, int bn, const void* entries, const int* start,
                   int count, int tiles, int* err, const PackFold& f);
int export_spins_int8(ising_ds* ds, int slot, int8_t* out);  // spins[slot] -> int8 [B][n]

}  // namespace ising
